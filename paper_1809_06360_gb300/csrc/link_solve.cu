// Step A3: the boundary-coupling solve of Section II-A (Eq. 10-11 and the
// J-segment generalisation after it). With the segment summaries
// J_j(z_j, z_{j+1}) of Eq. 9, stationarity of sum_j J_j in the link states
// z_1..z_{K-1} (the condition mu = -lambda of Eq. 10, through the envelope
// identity) is a block-tridiagonal SPD system. It is solved in FP64 by block
// elimination from the end, whose Schur complements are the global value
// function at the boundaries:
//     Pi_{K-1} = P of the last segment,
//     D_j  = V_zz^j + Pi_{j+1} = L_j L_j',   G_j = L_j^{-1} V_zx^j,  g_j = L_j^{-1}(v_z^j + pi_{j+1})
//     Pi_j = V_xx^j - G_j'G_j,               pi_j = v_x^j - G_j'g_j
// followed by the forward substitution z_0 = x0,
//     z_{j+1} = -D_j^{-1}(V_zx^j z_j + v_z^j + pi_{j+1}) = Gam_j z_j + gam_j.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <type_traits>
#include <stdio.h>
#include <stdlib.h>

#include "lqr_internal.cuh"

namespace cg = cooperative_groups;

namespace lqr {

__global__ void __launch_bounds__(kBlock) link_solve_kernel(ProbTable tab, int x0_is_float) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_flag;
  __shared__ double s_rd[256];
  const ProbDesc& pd = prob_at(tab, blockIdx.x);
  if (cta_should_exit(pd, &s_flag)) return;
  const int n = pd.n, K = pd.nseg;
  const long long nn = (long long)n * n;
  const WsLayout wl = ws_layout(n, K);
  double* ws = pd.ws;
  double* z = ws + wl.z;
  // z_0 = x0
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    z[i] = x0_is_float ? (double)static_cast<const float*>(pd.x0)[i] : static_cast<const double*>(pd.x0)[i];
  if (K == 1) return;
  double* L = reinterpret_cast<double*>(smem);  // n x n
  const long long sstride = 3 * nn + 2 * n;
  {
    const double* S = ws + wl.summ + (long long)(K - 1) * sstride;
    double* Pi = ws + wl.Pi + (long long)(K - 1) * nn;
    double* pi = ws + wl.pi + (long long)(K - 1) * n;
    for (int e = threadIdx.x; e < nn; e += blockDim.x) Pi[e] = S[e];
    for (int i = threadIdx.x; i < n; i += blockDim.x) pi[i] = S[3 * nn + i];
  }
  __syncthreads();
  for (int j = K - 2; j >= 0; --j) {
    const double* S = ws + wl.summ + (long long)j * sstride;
    const double* Vxx = S;
    const double* Vzx = S + nn;
    const double* Vzz = S + 2 * nn;
    const double* vx = S + 3 * nn;
    const double* vz = S + 3 * nn + n;
    const double* Pn = ws + wl.Pi + (long long)(j + 1) * nn;
    const double* pn = ws + wl.pi + (long long)(j + 1) * n;
    double* Pj = ws + wl.Pi + (long long)j * nn;
    double* pj = ws + wl.pi + (long long)j * n;
    double* G = ws + wl.Gam + (long long)j * nn;
    double* g = ws + wl.gam + (long long)j * n;
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      const int i = e / n, k = e % n;
      L[e] = 0.5 * (Vzz[(size_t)i * n + k] + Vzz[(size_t)k * n + i]) + Pn[e];
      G[e] = Vzx[e];
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) g[i] = vz[i] + pn[i];
    if (threadIdx.x == 0) s_flag = 0;
    __syncthreads();
    cta_chol(n, L, n, &s_flag, s_rd);
    if (s_flag) {
      if (threadIdx.x == 0) raise_status(pd.status, LQR_ERR_NOT_PD, -1 - j);
      return;
    }
    cta_trsm_lower<double>(n, L, n, s_rd, n, G, n);
    if (threadIdx.x == blockDim.x - 1) {
      // g <- L^{-1} g by one thread (a single right-hand side)
      for (int i = 0; i < n; ++i) {
        double t = g[i];
        for (int k = 0; k < i; ++k) t -= L[(size_t)i * n + k] * g[k];
        g[i] = t * s_rd[i];
      }
    }
    __syncthreads();
    cta_mm<4, 4, true, false, double>(n, n, n, G, n, G, n, EpiAdd<double, double>{Pj, n, -1.0, Vxx, n});
    cta_mv<true, double>(n, n, G, n, g, 1, EpiAdd<double, double>{pj, 1, -1.0, vx, 1});
    __syncthreads();
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      const int i = e / n, k = e % n;
      if (k <= i) continue;
      const double a = 0.5 * (Pj[(size_t)i * n + k] + Pj[(size_t)k * n + i]);
      Pj[(size_t)i * n + k] = a;
      Pj[(size_t)k * n + i] = a;
    }
    // Gam_j = -L'^{-1} G_j, gam_j = -L'^{-1} g_j (in place)
    cta_trsm_lower_t<double>(n, L, n, s_rd, n, G, n);
    if (threadIdx.x == blockDim.x - 1) {
      for (int i = n - 1; i >= 0; --i) {
        double t = g[i];
        for (int k = i + 1; k < n; ++k) t -= L[(size_t)k * n + i] * g[k];
        g[i] = t * s_rd[i];
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nn; e += blockDim.x) G[e] = -G[e];
    for (int i = threadIdx.x; i < n; i += blockDim.x) g[i] = -g[i];
    __syncthreads();
  }
  // forward substitution over the links
  for (int j = 0; j + 1 < K; ++j) {
    const double* G = ws + wl.Gam + (long long)j * nn;
    const double* g = ws + wl.gam + (long long)j * n;
    cta_mv<false, double>(n, n, G, n, z + (long long)j * n, 1,
                          EpiAdd<double, double>{z + (long long)(j + 1) * n, 1, 1.0, g, 1});
    __syncthreads();
  }
}

cudaError_t launch_link_solve(const ProbTable& tab, int nprob, int x0_is_float, cudaStream_t st) {
  // the largest n in the launch decides the shared-memory size
  int nmax = tab.probs ? 0 : tab.single.n;
  if (tab.probs) return cudaErrorInvalidValue;  // batched launches pass nmax through launch_link_solve_n
  const size_t bytes = sizeof(double) * (size_t)nmax * nmax;
  {
    cudaError_t e = raise_dyn_smem((const void*)link_solve_kernel, bytes);
    if (e != cudaSuccess) return e;
  }
  link_solve_kernel<<<nprob, kBlock, bytes, st>>>(tab, x0_is_float);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Link solve on the dual segment summaries (LQR_FORM_MULTIPLIER). Segment j
// carries G_j(s, mu) = 1/2 s'P_j s + mu'Z_j s - 1/2 mu'W_j mu + p_j's + w_j'mu,
// the minimum of its cost plus mu'x_end over its controls, so that
// J_j(s, z) = max_mu G_j(s, mu) - mu'z. Stationarity in the link states
// (Eq. 10-11 with mu the end multiplier) gives, with mu_j = Pi_{j+1} z_{j+1} + pi_{j+1},
//     z_{j+1} = (I + W_j Pi_{j+1})^{-1} (Z_j z_j + w_j - W_j pi_{j+1})
//     Pi_j = P_j + Z_j' Pi_{j+1} (I + W_j Pi_{j+1})^{-1} Z_j
//     pi_j = p_j + Z_j' pi_{j+1} + Z_j' Pi_{j+1} (I + W_j Pi_{j+1})^{-1} (w_j - W_j pi_{j+1}).
// With Pi_{j+1} = C C' and M = I + C'W_j C = Ld Ld' (SPD, eigenvalues >= 1):
//     E = C'Z_j, F = Ld^-1 E, v = w_j - W_j pi_{j+1}, t = Ld^-1 C'v
//     Pi_j = P_j + F'F,  pi_j = p_j + Z_j'pi_{j+1} + F't
//     Gam_j = Z_j - (W_j C) Ld^-T F,  gam_j = v - (W_j C) Ld^-T t      (Woodbury)
// so no inverse of the (possibly huge) Gramian W_j is ever formed.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) link_solve_dual_kernel(ProbTable tab, int x0_is_float, long long smem_bytes) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_flag;
  __shared__ double s_rdc[256];
  __shared__ double s_rdl[256];
  const ProbDesc& pd = prob_at(tab, blockIdx.x);
  if (cta_should_exit(pd, &s_flag)) return;
  const int n = pd.n, K = pd.nseg;
  const long long nn = (long long)n * n;
  const WsLayout wl = ws_layout(n, K);
  double* ws = pd.ws;
  double* z = ws + wl.z;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    z[i] = x0_is_float ? (double)static_cast<const float*>(pd.x0)[i] : static_cast<const double*>(pd.x0)[i];
  if (K == 1) return;
  double* work = (smem_bytes >= (long long)sizeof(double) * (4 * nn + 2 * n)) ? reinterpret_cast<double*>(smem)
                                                                              : ws + wl.lwork;
  double* C = work;            // Cholesky factor of Pi_{j+1}
  double* Tm = work + nn;      // W_j C
  double* Ld = work + 2 * nn;  // Cholesky factor of I + C'W_j C
  double* E = work + 3 * nn;   // C'Z_j -> F -> Ld^-T F
  double* pv = work + 4 * nn;  // pi_j under construction
  double* t2 = pv + n;         // Ld^-T t
  const long long sstride = 3 * nn + 2 * n;
  {
    const double* S = ws + wl.summ + (long long)(K - 1) * sstride;
    double* Pi = ws + wl.Pi + (long long)(K - 1) * nn;
    double* pi = ws + wl.pi + (long long)(K - 1) * n;
    for (int e = threadIdx.x; e < nn; e += blockDim.x) Pi[e] = S[e];
    for (int i = threadIdx.x; i < n; i += blockDim.x) pi[i] = S[3 * nn + i];
  }
  __syncthreads();
  for (int j = K - 2; j >= 0; --j) {
    const double* S = ws + wl.summ + (long long)j * sstride;
    const double* Pj_seg = S;
    const double* Z = S + nn;
    const double* Wneg = S + 2 * nn;  // -W_j
    const double* ps = S + 3 * nn;
    const double* w = S + 3 * nn + n;
    const double* Pn = ws + wl.Pi + (long long)(j + 1) * nn;
    const double* pn = ws + wl.pi + (long long)(j + 1) * n;
    double* Pj = ws + wl.Pi + (long long)j * nn;
    double* pj = ws + wl.pi + (long long)j * n;
    double* Gam = ws + wl.Gam + (long long)j * nn;
    double* gam = ws + wl.gam + (long long)j * n;  // holds v, then gam_j
    double* tv = pj;                               // scratch for t / t2 until pi_j is written
    for (int e = threadIdx.x; e < nn; e += blockDim.x) C[e] = Pn[e];
    // v = w_j - W_j pi_{j+1} = w_j + (-W_j) pi_{j+1}
    cta_mv<false, double>(n, n, Wneg, n, pn, 1, EpiAdd<double, double>{gam, 1, 1.0, w, 1});
    if (threadIdx.x == 0) s_flag = 0;
    __syncthreads();
    cta_chol(n, C, n, &s_flag, s_rdc);
    if (s_flag) {
      if (threadIdx.x == 0) raise_status(pd.status, LQR_ERR_NOT_PD, -1 - j);
      return;
    }
    for (int e = threadIdx.x; e < nn; e += blockDim.x)
      if (e % n > e / n) C[e] = 0.0;  // clear the upper triangle left by the factorisation
    __syncthreads();
    // Tm = W C = -(-W) C
    cta_mm<4, 4, false, false, double>(n, n, n, Wneg, n, C, n, EpiStore<double>{Tm, n, -1.0});
    // E = C'Z ; t (in tv) = C'v
    cta_mm<4, 4, true, false, double>(n, n, n, C, n, Z, n, EpiStore<double>{E, n, 1.0});
    cta_mv<true, double>(n, n, C, n, gam, 1, EpiStore<double>{tv, 1, 1.0});
    __syncthreads();
    // Ld = chol(I + C'Tm)
    cta_mm<4, 4, true, false, double>(n, n, n, C, n, Tm, n, EpiStore<double>{Ld, n, 1.0});
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) Ld[(long long)i * n + i] += 1.0;
    if (threadIdx.x == 0) s_flag = 0;
    __syncthreads();
    cta_chol(n, Ld, n, &s_flag, s_rdl);
    if (s_flag) {
      if (threadIdx.x == 0) raise_status(pd.status, LQR_ERR_NOT_PD, -1 - j);
      return;
    }
    // F = Ld^-1 E ; t = Ld^-1 (C'v)
    cta_trsm_lower<double>(n, Ld, n, s_rdl, n, E, n);
    if (threadIdx.x == blockDim.x - 1) {
      for (int i = 0; i < n; ++i) {
        double a = tv[i];
        for (int k = 0; k < i; ++k) a -= Ld[(long long)i * n + k] * tv[k];
        tv[i] = a * s_rdl[i];
      }
    }
    __syncthreads();
    // Pi_j = P_j + F'F ; pi_j = p_j + Z'pi_{j+1} + F't is assembled in pv while t
    // still occupies the pi_j slot
    cta_mm<4, 4, true, false, double>(n, n, n, E, n, E, n, EpiAdd<double, double>{Pj, n, 1.0, Pj_seg, n});
    cta_mv<true, double>(n, n, Z, n, pn, 1, EpiAdd<double, double>{pv, 1, 1.0, ps, 1});
    __syncthreads();
    cta_mv<true, double>(n, n, E, n, tv, 1, EpiAccum<double>{pv, 1, 1.0});
    __syncthreads();
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      const int i = e / n, k = e % n;
      if (k <= i) continue;
      const double a = 0.5 * (Pj[(size_t)i * n + k] + Pj[(size_t)k * n + i]);
      Pj[(size_t)i * n + k] = a;
      Pj[(size_t)k * n + i] = a;
    }
    // F <- Ld^-T F ; t2 = Ld^-T t
    cta_trsm_lower_t<double>(n, Ld, n, s_rdl, n, E, n);
    if (threadIdx.x == blockDim.x - 1) {
      for (int i = n - 1; i >= 0; --i) {
        double a = tv[i];
        for (int k = i + 1; k < n; ++k) a -= Ld[(long long)k * n + i] * t2[k];
        t2[i] = a * s_rdl[i];
      }
    }
    __syncthreads();
    // pi_j from its temporary; Gam_j = Z - Tm (Ld^-T F); gam_j = v - Tm t2
    for (int i = threadIdx.x; i < n; i += blockDim.x) pj[i] = pv[i];
    cta_mm<4, 4, false, false, double>(n, n, n, Tm, n, E, n, EpiAdd<double, double>{Gam, n, -1.0, Z, n});
    cta_mv<false, double>(n, n, Tm, n, t2, 1, EpiAccum<double>{gam, 1, -1.0});
    __syncthreads();
  }
  // forward substitution over the links
  for (int j = 0; j + 1 < K; ++j) {
    const double* G = ws + wl.Gam + (long long)j * nn;
    const double* g = ws + wl.gam + (long long)j * n;
    cta_mv<false, double>(n, n, G, n, z + (long long)j * n, 1,
                          EpiAdd<double, double>{z + (long long)(j + 1) * n, 1, 1.0, g, 1});
    __syncthreads();
  }
}

// Single right-hand-side triangular solves by one warp (column-oriented: after
// y_i is known every lane updates its later entries). y is in shared memory.
__device__ inline void warp_trsv_lower(int n, const double* L, int ld, const double* rd, double* y) {
  const int lane = threadIdx.x & 31;
  for (int i = 0; i < n; ++i) {
    const double yi = y[i] * rd[i];
    __syncwarp();
    if (lane == 0) y[i] = yi;
    for (int k = i + 1 + lane; k < n; k += 32) y[k] -= L[(size_t)k * ld + i] * yi;
    __syncwarp();
  }
}
__device__ inline void warp_trsv_lower_t(int n, const double* L, int ld, const double* rd, double* y) {
  const int lane = threadIdx.x & 31;
  for (int i = n - 1; i >= 0; --i) {
    const double yi = y[i] * rd[i];
    __syncwarp();
    if (lane == 0) y[i] = yi;
    for (int k = lane; k < i; k += 32) y[k] -= L[(size_t)i * ld + k] * yi;
    __syncwarp();
  }
}

// Copy the column slabs owned by the other CTAs of the cluster into the local
// copy of the n x ld matrix M (distributed shared memory reads; 16-byte loads
// when every slab boundary is 16-byte aligned).
template <int CL, typename T>
__device__ inline void cluster_gather_cols(cg::cluster_group& cluster, T* M, int n, int ncols, int ld, int rank) {
  using T2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
  const bool vec = ((ld & 1) == 0) && (ncols % (2 * CL) == 0);
  for (int r2 = 0; r2 < CL; ++r2) {
    if (r2 == rank) continue;
    const T* rem = cluster.map_shared_rank(M, r2);
    const int d0 = r2 * ncols / CL, d1 = (r2 + 1) * ncols / CL, w = d1 - d0;
    if (w <= 0) continue;
    if (vec) {
      const int w2 = w >> 1;
      for (int e = threadIdx.x; e < n * w2; e += blockDim.x) {
        const int i = e / w2, jj = d0 + 2 * (e % w2);
        *reinterpret_cast<T2*>(M + (size_t)i * ld + jj) = *reinterpret_cast<const T2*>(rem + (size_t)i * ld + jj);
      }
    } else {
      for (int e = threadIdx.x; e < n * w; e += blockDim.x) {
        const int i = e / w, jj = d0 + e % w;
        M[(size_t)i * ld + jj] = rem[(size_t)i * ld + jj];
      }
    }
  }
}

// The serial part of the dual link recursion, each link step spread over a
// cluster of CL CTAs (column slabs exchanged through distributed shared
// memory; the two n x n factorisations are computed redundantly in every CTA,
// deterministic, so all CTAs hold identical factors). The vector recursion
// rides along as column n of [Z_j | v_j]:
//     C = chol(Pi_{j+1}),  v = w_j - W_j pi_{j+1},  Tm = W_j C,
//     E = C'[Z_j | v],  Ld = chol(I + C'Tm),  F = Ld^-1 E,
//     [Pi_j | pi_j] = [P_j | p_j + Z_j'pi_{j+1}] + F'F      (columns 0..n-1 | n)
// Tm, Ld, 1/diag(Ld), F and v are stored per link for the parallel post-pass
// that forms Gam_j and gam_j off the serial chain.
template <int CL, typename T>
__global__ void __launch_bounds__(kBlock) link_solve_dual_cluster_kernel(ProbTable tab, int x0_is_float, int stage_inputs) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_flag;
  __shared__ T s_rdc[256];
  __shared__ T s_rdl[256];
  __shared__ float s_pivf[sizeof(T) == 4 ? 512 : 1];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const ProbDesc& pd = prob_at(tab, blockIdx.x / CL);
  // the exit decision reads state written by earlier kernels only: cluster-uniform
  if (cta_should_exit(pd, &s_flag)) return;
  const int n = pd.n, K = pd.nseg;
  const int n1 = n + 1;
  const long long nn = (long long)n * n;
  const WsLayout wl = ws_layout(n, K);
  double* ws = pd.ws;
  if (K == 1) return;
  T* C = reinterpret_cast<T*>(smem);  // n x n
  T* Tm = C + nn;                      // n x n
  T* Ld = Tm + nn;                     // n x n
  T* E = Ld + nn;                      // n x (n+1): C'[Z | v], then F
  T* v = E + (long long)n * n1;        // n
  T* Wn_s = v + n;                     // staged -W_j (n x n)
  T* Z_s = Wn_s + nn;                  // staged [Z_j | v] (n x (n+1)), column n = v
  T* vec_s = Z_s + (long long)n * n1;  // staged w_j, p_j, pi_{j+1}
  const bool staged = stage_inputs != 0;
  const int c0 = rank * n / CL, c1 = (rank + 1) * n / CL, ns = c1 - c0;         // slab of n columns
  const int e0 = rank * n1 / CL, e1 = (rank + 1) * n1 / CL, ens = e1 - e0;      // slab of n+1 columns
  const long long sstride = 3 * nn + 2 * n;
  if (rank == 0) {
    const double* S = ws + wl.summ + (long long)(K - 1) * sstride;
    double* Pi = ws + wl.Pi + (long long)(K - 1) * nn;
    double* pi = ws + wl.pi + (long long)(K - 1) * n;
    for (int e = threadIdx.x; e < nn; e += blockDim.x) Pi[e] = S[e];
    for (int i = threadIdx.x; i < n; i += blockDim.x) pi[i] = S[3 * nn + i];
  }
  cluster.sync();
  for (int j = K - 2; j >= 0; --j) {
    const double* S = ws + wl.summ + (long long)j * sstride;
    const double* Pseg = S;
    const double* Zg = S + nn;
    const double* Wneg = S + 2 * nn;
    const double* ps = S + 3 * nn;
    const double* w = S + 3 * nn + n;
    const double* Pn = ws + wl.Pi + (long long)(j + 1) * nn;
    const double* pn = ws + wl.pi + (long long)(j + 1) * n;
    double* Pj = ws + wl.Pi + (long long)j * nn;
    double* pj = ws + wl.pi + (long long)j * n;
    // (A) redundant: C = chol(Pi_{j+1}); inputs staged
    for (int e = threadIdx.x; e < nn; e += blockDim.x) C[e] = static_cast<T>(Pn[e]);
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      Wn_s[e] = static_cast<T>(Wneg[e]);
      Z_s[(size_t)(e / n) * n1 + (e % n)] = static_cast<T>(Zg[e]);
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      vec_s[i] = static_cast<T>(w[i]);
      vec_s[n + i] = static_cast<T>(ps[i]);
      vec_s[2 * n + i] = static_cast<T>(pn[i]);
    }
    (void)staged;
    if (threadIdx.x == 0) s_flag = 0;
    __syncthreads();
    // v = w - W pi_{j+1} into column n of Z_s (and v)
    cta_mv<false, T>(n, n, Wn_s, n, vec_s + 2 * n, 1, EpiAdd<T, T>{v, 1, 1.0, vec_s, 1});
    if constexpr (sizeof(T) == 8)
      cta_chol(n, reinterpret_cast<double*>(C), n, &s_flag, reinterpret_cast<double*>(s_rdc));
    else
      cta_chol_f32(n, reinterpret_cast<float*>(C), n, &s_flag, s_pivf, reinterpret_cast<float*>(s_rdc));
    if (s_flag) {  // identical in every CTA of the cluster
      if (rank == 0 && threadIdx.x == 0) raise_status(pd.status, LQR_ERR_NOT_PD, -1 - j);
      return;
    }
    for (int e = threadIdx.x; e < nn; e += blockDim.x)
      if (e % n > e / n) C[e] = T(0);
    for (int i = threadIdx.x; i < n; i += blockDim.x) Z_s[(size_t)i * n1 + n] = v[i];
    __syncthreads();
    // (B) slabs of Tm = W C and E = C'[Z | v]
    cta_mm_auto<false, false, T>(n, ns, n, Wn_s, n, C + c0, n, EpiStore<T>{Tm + c0, n, -1.0});
    cta_mm_auto<true, false, T>(n, ens, n, C, n, Z_s + e0, n1, EpiStore<T>{E + e0, n1, 1.0});
    cluster.sync();
    cluster_gather_cols<CL, T>(cluster, Tm, n, n, n, rank);
    cluster.sync();
    // (C) slab of Ld = I + C'Tm
    cta_mm_auto<true, false, T>(n, ns, n, C, n, Tm + c0, n, EpiStore<T>{Ld + c0, n, 1.0});
    __syncthreads();
    for (int i = c0 + threadIdx.x; i < c1; i += blockDim.x) Ld[(size_t)i * n + i] += T(1);
    cluster.sync();
    cluster_gather_cols<CL, T>(cluster, Ld, n, n, n, rank);
    cluster.sync();
    // (D) redundant: Ld = chol(I + C'W C)
    if (threadIdx.x == 0) s_flag = 0;
    __syncthreads();
    if constexpr (sizeof(T) == 8)
      cta_chol(n, reinterpret_cast<double*>(Ld), n, &s_flag, reinterpret_cast<double*>(s_rdl));
    else
      cta_chol_f32(n, reinterpret_cast<float*>(Ld), n, &s_flag, s_pivf, reinterpret_cast<float*>(s_rdl));
    if (s_flag) {
      if (rank == 0 && threadIdx.x == 0) raise_status(pd.status, LQR_ERR_NOT_PD, -1 - j);
      return;
    }
    // (E) slab of F = Ld^-1 E (in place), then the full F
    cta_trsm_lower_warp<T>(n, Ld, n, ens, E + e0, n1, s_rdl);
    cluster.sync();
    cluster_gather_cols<CL, T>(cluster, E, n, n1, n1, rank);
    cluster.sync();
    // (F) slab of [Pi_j | pi_j] = [P_j | p_j + Z'pi_{j+1}] + F'F; stores for the post-pass
    cta_mm_auto<true, false, T>(n, ns, n, E, n1, E + c0, n1, EpiAdd<double, double>{Pj + c0, n, 1.0, Pseg + c0, n});
    if (rank == CL - 1) {
      // column n: pi_j = p_j + Z'pi_{j+1} + F't  (t = column n of F)
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        T a = vec_s[n + i];
        for (int k = 0; k < n; ++k)
          a = fma(Z_s[(size_t)k * n1 + i], vec_s[2 * n + k], fma(E[(size_t)k * n1 + i], E[(size_t)k * n1 + n], a));
        pj[i] = static_cast<double>(a);
      }
    }
    {
      double* gTm = ws + wl.lkTm + (long long)j * nn;
      double* gLd = ws + wl.lkLd + (long long)j * nn;
      double* gRd = ws + wl.lkRd + (long long)j * n;
      double* gF = ws + wl.lkF + (long long)j * n * n1;
      double* gV = ws + wl.lkV + (long long)j * n;
      for (int e = threadIdx.x; e < n * ns; e += blockDim.x) {
        const int i = e / ns, jj = c0 + e % ns;
        gTm[(size_t)i * n + jj] = static_cast<double>(Tm[(size_t)i * n + jj]);
        gLd[(size_t)i * n + jj] = static_cast<double>(Ld[(size_t)i * n + jj]);
      }
      for (int e = threadIdx.x; e < n * ens; e += blockDim.x) {
        const int i = e / ens, jj = e0 + e % ens;
        gF[(size_t)i * n1 + jj] = static_cast<double>(E[(size_t)i * n1 + jj]);
      }
      if (rank == 0)
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
          gRd[i] = static_cast<double>(s_rdl[i]);
          gV[i] = static_cast<double>(v[i]);
        }
    }
    cluster.sync();  // Pi_j, pi_j visible to the cluster; slabs free for reuse
  }
}

// Off the serial chain, one CTA per link: G2 = Ld^-T F (columns 0..n), then
//     Gam_j = Z_j - Tm G2[:, 0:n],   gam_j = v_j - Tm G2[:, n]      (Woodbury)
// so that z_{j+1} = Gam_j z_j + gam_j.
template <typename T>
__global__ void __launch_bounds__(kBlock) link_post_kernel(ProbTable tab) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_flag;
  const ProbDesc& pd = tab.single;
  if (cta_should_exit(pd, &s_flag)) return;
  const int n = pd.n, K = pd.nseg, n1 = n + 1;
  const int j = blockIdx.x;
  if (j >= K - 1) return;
  const long long nn = (long long)n * n;
  const WsLayout wl = ws_layout(n, K);
  double* ws = pd.ws;
  T* G2 = reinterpret_cast<T*>(smem);    // n x (n+1)
  T* Ld = G2 + (long long)n * n1;        // n x n
  T* Tm = Ld + nn;                       // n x n
  T* rd = Tm + nn;                       // n
  for (int e = threadIdx.x; e < n * n1; e += blockDim.x) G2[e] = static_cast<T>(ws[wl.lkF + (long long)j * n * n1 + e]);
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    Ld[e] = static_cast<T>(ws[wl.lkLd + (long long)j * nn + e]);
    Tm[e] = static_cast<T>(ws[wl.lkTm + (long long)j * nn + e]);
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) rd[i] = static_cast<T>(ws[wl.lkRd + (long long)j * n + i]);
  __syncthreads();
  cta_trsm_lower_t_warp<T>(n, Ld, n, n1, G2, n1, rd);
  __syncthreads();
  const double* Z = ws + wl.summ + (long long)j * (3 * nn + 2 * n) + nn;
  cta_mm_auto<false, false, T>(n, n, n, Tm, n, G2, n1,
                               EpiAdd<double, double>{ws + wl.Gam + (long long)j * nn, n, -1.0, Z, n});
  cta_mv<false, T>(n, n, Tm, n, G2 + n, n1,
                   EpiAdd<double, double>{ws + wl.gam + (long long)j * n, 1, -1.0, ws + wl.lkV + (long long)j * n, 1});
}

// ---------------------------------------------------------------------------
// FP32 link chain in one CTA for the sizes the cluster chain cannot hold
// (n > 67, n a multiple of 8): the serial part of the dual block elimination,
//     C = chol(Pi_{j+1}),  Tm = W_j C,  [E | e] = C'[Z_j | v_j],  v_j = w_j - W_j pi_{j+1},
//     Ld = chol(I + C'Tm),  [F | t] = Ld^-1 [E | e],
//     Pi_j = P_j + F'F,  pi_j = p_j + Z_j'pi_{j+1} + F't,
// with Tm, Ld, 1/diag(Ld), [F | t] and v_j stored per link for the parallel
// post-pass (link_post_kernel<float>) that forms Gam_j, gam_j off the chain.
// Three n x (n + 4) FP32 work matrices in shared memory; products on 4 x 4
// register tiles, in place where the output overwrites an operand (every tile
// computed into registers before any is stored).
// ---------------------------------------------------------------------------
constexpr int kChainF32Block = 512;
constexpr int kChainMaxTiles = 3;  // ceil(32 * 33 / 512) tiles per thread at n = 128

__host__ __device__ inline long long chain_f32_smem_floats(int n) {
  const long long ld = n + 4;
  return 3 * (long long)n * ld + p4_scratch_floats(n) + 4LL * n + 8;
}

// One 4 x 4 tile of op(A) B at (i0, j0) into acc (op(A) = A or A').
template <bool TA>
__device__ __forceinline__ void mm4f_acc(int i0, int j0, int K, const float* A, int lda, const float* B, int ldb,
                                         float (&acc)[4][4]) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
  for (int k = 0; k < K; ++k) {
    float4 av;
    if (TA) {
      av = *reinterpret_cast<const float4*>(A + (size_t)k * lda + i0);
    } else {
      av.x = A[(size_t)i0 * lda + k];
      av.y = A[(size_t)(i0 + 1) * lda + k];
      av.z = A[(size_t)(i0 + 2) * lda + k];
      av.w = A[(size_t)(i0 + 3) * lda + k];
    }
    const float4 bv = *reinterpret_cast<const float4*>(B + (size_t)k * ldb + j0);
    const float ak[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      acc[a][0] = fmaf(ak[a], bv.x, acc[a][0]);
      acc[a][1] = fmaf(ak[a], bv.y, acc[a][1]);
      acc[a][2] = fmaf(ak[a], bv.z, acc[a][2]);
      acc[a][3] = fmaf(ak[a], bv.w, acc[a][3]);
    }
  }
}

// C = epi(op(A) B) over M x N (multiples of 4) where C may alias A or B:
// every tile a thread owns is computed into registers before any is stored.
template <bool TA, typename Epi>
__device__ __forceinline__ void mm4f_inplace(int M, int N, int K, const float* A, int lda, const float* B, int ldb,
                                             Epi epi) {
  const int tn = N >> 2, nt = (M >> 2) * tn;
  float acc[kChainMaxTiles][4][4];
#pragma unroll
  for (int s = 0; s < kChainMaxTiles; ++s) {
    const int tile = (int)threadIdx.x + s * (int)blockDim.x;
    if (tile < nt) mm4f_acc<TA>((tile / tn) << 2, (tile % tn) << 2, K, A, lda, B, ldb, acc[s]);
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < kChainMaxTiles; ++s) {
    const int tile = (int)threadIdx.x + s * (int)blockDim.x;
    if (tile < nt) {
      const int i0 = (tile / tn) << 2, j0 = (tile % tn) << 2;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) epi(i0 + a, j0 + b, acc[s][a][b]);
    }
  }
  __syncthreads();
}

// Y <- L^-1 Y in place (L lower n x n, n a multiple of 4, rd[i] = 1 / L[i][i];
// Y n x nc), by 4-row blocks: the diagonal block solved per column, then a
// rank-4 downdate of the rows below. Ends with a barrier.
__device__ inline void trsm_lower_blk4(int n, const float* L, int ldl, const float* rd, int nc, float* Y, int ldy) {
  const int t = threadIdx.x, nthr = blockDim.x;
  for (int b = 0; b < n; b += 4) {
    const float* Lb = L + (size_t)b * ldl + b;
    for (int c = t; c < nc; c += nthr) {
      float* y = Y + (size_t)b * ldy + c;
      const float y0 = y[0] * rd[b];
      const float y1 = (y[ldy] - Lb[ldl] * y0) * rd[b + 1];
      const float y2 = (y[2 * ldy] - Lb[2 * ldl] * y0 - Lb[2 * ldl + 1] * y1) * rd[b + 2];
      const float y3 = (y[3 * ldy] - Lb[3 * ldl] * y0 - Lb[3 * ldl + 1] * y1 - Lb[3 * ldl + 2] * y2) * rd[b + 3];
      y[0] = y0;
      y[ldy] = y1;
      y[2 * ldy] = y2;
      y[3 * ldy] = y3;
    }
    __syncthreads();
    const int rows = n - b - 4;
    for (int e = t; e < rows * nc; e += nthr) {
      const int i = b + 4 + e / nc, c = e % nc;
      const float4 l = *reinterpret_cast<const float4*>(L + (size_t)i * ldl + b);
      float v = Y[(size_t)i * ldy + c];
      v -= l.x * Y[(size_t)b * ldy + c];
      v -= l.y * Y[(size_t)(b + 1) * ldy + c];
      v -= l.z * Y[(size_t)(b + 2) * ldy + c];
      v -= l.w * Y[(size_t)(b + 3) * ldy + c];
      Y[(size_t)i * ldy + c] = v;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kChainF32Block, 1) link_chain_f32_kernel(ProbTable tab) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_flag;
  const ProbDesc& pd = tab.single;
  if (cta_should_exit(pd, &s_flag)) return;
  const int n = pd.n, K = pd.nseg, ld = n + 4, n1 = n + 1;
  const long long nn = (long long)n * n;
  const WsLayout wl = ws_layout(n, K);
  double* ws = pd.ws;
  const long long sstride = 3 * nn + 2 * n;
  float* X = reinterpret_cast<float*>(smem);  // Pi_{j+1} -> C -> I + C'Tm -> Ld -> Pi_j
  float* Y = X + (size_t)n * ld;              // [Z | v] -> [E | e] -> [F | t]
  float* Wb = Y + (size_t)n * ld;             // -W -> Tm
  float* scr = Wb + (size_t)n * ld;           // Cholesky scratch
  float* rdv = scr + p4_scratch_floats(n);    // 1 / diag of the current factor
  float* pin = rdv + n;                       // pi_{j+1}
  float* pnew = pin + n;                      // pi_j under construction
  float* vv = pnew + n;                       // v_j
  const int t = threadIdx.x, nthr = blockDim.x;
  {  // the last segment carries the global value function at its start
    const double* S = ws + wl.summ + (long long)(K - 1) * sstride;
    double* Pi = ws + wl.Pi + (long long)(K - 1) * nn;
    double* pi = ws + wl.pi + (long long)(K - 1) * n;
    for (int e = t; e < nn; e += nthr) {
      Pi[e] = S[e];
      X[(size_t)(e / n) * ld + e % n] = static_cast<float>(S[e]);
    }
    for (int i = t; i < n; i += nthr) {
      pi[i] = S[3 * nn + i];
      pin[i] = static_cast<float>(S[3 * nn + i]);
    }
  }
  __syncthreads();
  for (int j = K - 2; j >= 0; --j) {
    const double* S = ws + wl.summ + (long long)j * sstride;
    const double* Pseg = S;
    const double* Z = S + nn;
    const double* Wneg = S + 2 * nn;  // -W_j
    const double* ps = S + 3 * nn;
    const double* w = S + 3 * nn + n;
    // v_j = w_j + (-W_j) pi_{j+1}; stage [Z_j | v_j | 0] and -W_j
    for (int i = t; i < n; i += nthr) {
      float a = static_cast<float>(w[i]);
      for (int k = 0; k < n; ++k) a = fmaf(static_cast<float>(Wneg[(size_t)i * n + k]), pin[k], a);
      vv[i] = a;
    }
    for (int e = t; e < nn; e += nthr) {
      const int i = e / n, k = e - i * n;
      Y[(size_t)i * ld + k] = static_cast<float>(Z[e]);
      Wb[(size_t)i * ld + k] = static_cast<float>(Wneg[e]);
    }
    if (t == 0) s_flag = 0;
    __syncthreads();
    for (int i = t; i < n; i += nthr) {
      Y[(size_t)i * ld + n] = vv[i];
      Y[(size_t)i * ld + n + 1] = 0.0f;
      Y[(size_t)i * ld + n + 2] = 0.0f;
      Y[(size_t)i * ld + n + 3] = 0.0f;
      float a = static_cast<float>(ps[i]);  // pi_j = p_j + Z_j'pi_{j+1} + F't, first two terms
      for (int k = 0; k < n; ++k) a = fmaf(Y[(size_t)k * ld + i], pin[k], a);
      pnew[i] = a;
    }
    cta_chol_p4<4, 8>(n, X, ld, &s_flag, scr, rdv);  // C
    if (s_flag) {
      if (t == 0) raise_status(pd.status, LQR_ERR_NOT_PD, -1 - j);
      return;
    }
    // Tm = W C = -(-W) C ;  [E | e] = C'[Z | v]
    mm4f_inplace<false>(n, n, n, Wb, ld, X, ld, [&](int i, int k, float v) { Wb[(size_t)i * ld + k] = -v; });
    mm4f_inplace<true>(n, n + 4, n, X, ld, Y, ld, [&](int i, int k, float v) { Y[(size_t)i * ld + k] = v; });
    {
      double* gT = ws + wl.lkTm + (long long)j * nn;
      for (int e = t; e < nn; e += nthr) gT[e] = static_cast<double>(Wb[(size_t)(e / n) * ld + e % n]);
      double* gV = ws + wl.lkV + (long long)j * n;
      for (int i = t; i < n; i += nthr) gV[i] = static_cast<double>(vv[i]);
    }
    // X = I + C'Tm, then Ld = chol(X)
    mm4f_inplace<true>(n, n, n, X, ld, Wb, ld,
                       [&](int i, int k, float v) { X[(size_t)i * ld + k] = v + (i == k ? 1.0f : 0.0f); });
    cta_chol_p4<4, 8>(n, X, ld, &s_flag, scr, rdv);
    if (s_flag) {
      if (t == 0) raise_status(pd.status, LQR_ERR_NOT_PD, -1 - j);
      return;
    }
    {
      double* gL = ws + wl.lkLd + (long long)j * nn;
      for (int e = t; e < nn; e += nthr) gL[e] = static_cast<double>(X[(size_t)(e / n) * ld + e % n]);
      double* gR = ws + wl.lkRd + (long long)j * n;
      for (int i = t; i < n; i += nthr) gR[i] = static_cast<double>(rdv[i]);
    }
    // [F | t] = Ld^-1 [E | e]
    trsm_lower_blk4(n, X, ld, rdv, n1, Y, ld);
    {
      double* gF = ws + wl.lkF + (long long)j * n * n1;
      for (int e = t; e < n * n1; e += nthr) gF[e] = static_cast<double>(Y[(size_t)(e / n1) * ld + e % n1]);
    }
    // Pi_j = P_j + F'F (into X: Ld is stored), pi_j += F't
    cta_mm4f<true>(n, n, n, Y, ld, Y, ld, [&](int i, int k, float v) {
      X[(size_t)i * ld + k] = v + static_cast<float>(Pseg[(size_t)i * n + k]);
    });
    for (int i = t; i < n; i += nthr) {
      float a = pnew[i];
      for (int k = 0; k < n; ++k) a = fmaf(Y[(size_t)k * ld + i], Y[(size_t)k * ld + n], a);
      pnew[i] = a;
    }
    __syncthreads();
    {
      double* Pj = ws + wl.Pi + (long long)j * nn;
      double* pj = ws + wl.pi + (long long)j * n;
      for (int e = t; e < nn; e += nthr) {
        const int i = e / n, k = e - i * n;
        if (k < i) continue;
        const float a = 0.5f * (X[(size_t)i * ld + k] + X[(size_t)k * ld + i]);
        X[(size_t)i * ld + k] = a;
        X[(size_t)k * ld + i] = a;
        Pj[(size_t)i * n + k] = a;
        Pj[(size_t)k * n + i] = a;
      }
      for (int i = t; i < n; i += nthr) {
        pj[i] = static_cast<double>(pnew[i]);
        pin[i] = pnew[i];
      }
    }
    __syncthreads();
  }
}

// The link states: z_0 = x0, z_{j+1} = Gam_j z_j + gam_j (one CTA, serial, O(K n^2)).
__global__ void __launch_bounds__(kBlock) link_forward_kernel(ProbTable tab, int x0_is_float) {
  __shared__ int s_flag;
  const ProbDesc& pd = tab.single;
  if (cta_should_exit(pd, &s_flag)) return;
  const int n = pd.n, K = pd.nseg;
  const long long nn = (long long)n * n;
  const WsLayout wl = ws_layout(n, K);
  double* z = pd.ws + wl.z;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    z[i] = x0_is_float ? (double)static_cast<const float*>(pd.x0)[i] : static_cast<const double*>(pd.x0)[i];
  __syncthreads();
  for (int j = 0; j + 1 < K; ++j) {
    cta_mv<false, double>(n, n, pd.ws + wl.Gam + (long long)j * nn, n, z + (long long)j * n, 1,
                          EpiAdd<double, double>{z + (long long)(j + 1) * n, 1, 1.0, pd.ws + wl.gam + (long long)j * n, 1});
    __syncthreads();
  }
}

template <int CL, typename T>
static cudaError_t launch_dual_cluster(const ProbTable& tab, int nprob, int x0_is_float, size_t bytes,
                                       cudaStream_t st) {
  {
    cudaError_t e = raise_dyn_smem((const void*)link_solve_dual_cluster_kernel<CL, T>, bytes);
    if (e != cudaSuccess) return e;
    if (CL > 8) {
      e = cudaFuncSetAttribute(link_solve_dual_cluster_kernel<CL, T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL * nprob, 1, 1);
  cfg.blockDim = dim3(kBlock, 1, 1);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, link_solve_dual_cluster_kernel<CL, T>, tab, x0_is_float, 1);
}

// link method of the last single-problem solve: -1 none yet, 0 single CTA,
// 2 single-CTA FP32 chain, 8/16 cluster chain width, 1000 + levels for the FP32 scan
static int g_link_cluster = -1;
cudaError_t launch_link_solve_dual_impl(const ProbTable& tab, int nprob, int x0_is_float, cudaStream_t st,
                                        int* nlaunch);
// set per call by launch_link_solve_dual: 0 FP64, 1 FP32, 2 FP64 where the cluster
// chain holds the problem and the single-CTA FP32 chain beyond it
static int g_link_fp32 = 0;

int link_cluster_width() { return g_link_cluster; }

cudaError_t launch_link_solve_dual(const ProbTable& tab, int nprob, int x0_is_float, cudaStream_t st, int link_fp32,
                                   int method, int* nlaunch) {
  if (tab.probs) return cudaErrorInvalidValue;
  g_link_fp32 = link_fp32;
  cudaError_t r = cudaErrorNotSupported;
  int nl = 0;
  if (link_fp32 == 1 && method != LQR_LINK_CHAIN) {
    r = launch_link_scan(tab, x0_is_float, st, &nl);
    if (r == cudaSuccess) g_link_cluster = 1000 + nl - 3;
    if (r == cudaErrorNotSupported && method == LQR_LINK_SCAN) return r;
  }
  if (r == cudaErrorNotSupported) r = launch_link_solve_dual_impl(tab, nprob, x0_is_float, st, &nl);
  if (nlaunch) *nlaunch = nl;
  static int reported = -2;
  if (getenv("LQR_DEBUG") && reported != g_link_cluster) {
    fprintf(stderr, "liblqr: link solve method %d (0 single CTA, 8/16 cluster chain, 1000+levels scan), n=%d K=%d\n",
            g_link_cluster, tab.single.n, tab.single.nseg);
    reported = g_link_cluster;
  }
  return r;
}

cudaError_t launch_link_solve_dual_batched(const ProbTable& tab, int nprob, int nmax, int x0_is_float,
                                          cudaStream_t st) {
  size_t bytes = sizeof(double) * (4 * (size_t)nmax * nmax + 2 * (size_t)nmax);
  int optin = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (bytes > (size_t)optin - kStaticSmemReserve) bytes = 0;
  {
    cudaError_t e = raise_dyn_smem((const void*)link_solve_dual_kernel, bytes);
    if (e != cudaSuccess) return e;
  }
  link_solve_dual_kernel<<<nprob, kBlock, bytes, st>>>(tab, x0_is_float, (long long)bytes);
  return cudaGetLastError();
}

cudaError_t launch_link_solve_dual_impl(const ProbTable& tab, int nprob, int x0_is_float, cudaStream_t st,
                                        int* nlaunch) {
  *nlaunch = 1;
  {
    const int n = tab.single.n;
    const size_t nn = (size_t)n * n, n1 = (size_t)n + 1;
    const size_t es = g_link_fp32 == 1 ? sizeof(float) : sizeof(double);
    // C, Tm, Ld, E (n x (n+1)), v | staged -W, [Z | v], w, p, pi
    const size_t cbytes = es * (3 * nn + n * n1 + n + nn + n * n1 + 3 * (size_t)n);
    int optin = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (n >= 16 && tab.single.nseg > 1 && cbytes <= (size_t)optin - kStaticSmemReserve) {
      int width = 16;
      cudaError_t e = g_link_fp32 == 1 ? launch_dual_cluster<16, float>(tab, nprob, x0_is_float, cbytes, st)
                                  : launch_dual_cluster<16, double>(tab, nprob, x0_is_float, cbytes, st);
      if (e != cudaSuccess) {
        cudaGetLastError();  // 16-CTA clusters not available: portable width
        width = 8;
        e = g_link_fp32 == 1 ? launch_dual_cluster<8, float>(tab, nprob, x0_is_float, cbytes, st)
                        : launch_dual_cluster<8, double>(tab, nprob, x0_is_float, cbytes, st);
      }
      if (e == cudaSuccess) {
        g_link_cluster = width;
        const size_t pbytes = es * (n * n1 + 2 * nn + n);
        const void* post = g_link_fp32 == 1 ? (const void*)link_post_kernel<float> : (const void*)link_post_kernel<double>;
        e = raise_dyn_smem(post, pbytes);
        if (e != cudaSuccess) return e;
        if (g_link_fp32 == 1)
          link_post_kernel<float><<<tab.single.nseg - 1, kBlock, pbytes, st>>>(tab);
        else
          link_post_kernel<double><<<tab.single.nseg - 1, kBlock, pbytes, st>>>(tab);
        link_forward_kernel<<<1, kBlock, 0, st>>>(tab, x0_is_float);
        *nlaunch = 3;
        return cudaGetLastError();
      }
      cudaGetLastError();
    }
  }
  {  // FP32: the single-CTA FP32 chain with its work matrices in shared memory
    const int n = tab.single.n, K = tab.single.nseg;
    const size_t fbytes = sizeof(float) * (size_t)chain_f32_smem_floats(n);
    int optin = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (g_link_fp32 && n >= 8 && n % 8 == 0 && n <= 128 && K > 1 && fbytes <= (size_t)optin - kStaticSmemReserve) {
      const int n1 = n + 1;
      const size_t pbytes = sizeof(float) * ((size_t)n * n1 + 2 * (size_t)n * n + n);
      cudaError_t e = raise_dyn_smem((const void*)link_chain_f32_kernel, fbytes);
      if (e == cudaSuccess) e = raise_dyn_smem((const void*)link_post_kernel<float>, pbytes);
      if (e != cudaSuccess) return e;
      link_chain_f32_kernel<<<1, kChainF32Block, fbytes, st>>>(tab);
      link_post_kernel<float><<<K - 1, kBlock, pbytes, st>>>(tab);
      link_forward_kernel<<<1, kBlock, 0, st>>>(tab, x0_is_float);
      *nlaunch = 3;
      g_link_cluster = 2;
      return cudaGetLastError();
    }
  }
  g_link_cluster = 0;
  const int n = tab.single.n;
  size_t bytes = sizeof(double) * (4 * (size_t)n * n + 2 * (size_t)n);
  int optin = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (bytes > (size_t)optin - kStaticSmemReserve) bytes = 0;  // work matrices go to the global workspace
  {
    cudaError_t e = raise_dyn_smem((const void*)link_solve_dual_kernel, bytes);
    if (e != cudaSuccess) return e;
  }
  link_solve_dual_kernel<<<nprob, kBlock, bytes, st>>>(tab, x0_is_float, (long long)bytes);
  return cudaGetLastError();
}

}  // namespace lqr
