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
#include <cuda_runtime.h>

#include "lqr_internal.cuh"

namespace lqr {

__global__ void __launch_bounds__(kBlock) link_solve_kernel(ProbTable tab, int x0_is_float) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_flag;
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
    cta_chol(n, L, n, &s_flag);
    if (s_flag) {
      if (threadIdx.x == 0) raise_status(pd.status, LQR_ERR_NOT_PD, -1 - j);
      return;
    }
    cta_trsm_lower<double>(n, L, n, n, G, n);
    if (threadIdx.x == blockDim.x - 1) {
      // g <- L^{-1} g by one thread (a single right-hand side)
      for (int i = 0; i < n; ++i) {
        double t = g[i];
        for (int k = 0; k < i; ++k) t -= L[(size_t)i * n + k] * g[k];
        g[i] = t / L[(size_t)i * n + i];
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
    cta_trsm_lower_t<double>(n, L, n, n, G, n);
    if (threadIdx.x == blockDim.x - 1) {
      for (int i = n - 1; i >= 0; --i) {
        double t = g[i];
        for (int k = i + 1; k < n; ++k) t -= L[(size_t)k * n + i] * g[k];
        g[i] = t / L[(size_t)i * n + i];
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
  static size_t configured = 0;
  if (bytes > 48 * 1024 && bytes > configured) {
    cudaError_t e = cudaFuncSetAttribute(link_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    configured = bytes;
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
    cta_chol(n, C, n, &s_flag);
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
    cta_chol(n, Ld, n, &s_flag);
    if (s_flag) {
      if (threadIdx.x == 0) raise_status(pd.status, LQR_ERR_NOT_PD, -1 - j);
      return;
    }
    // F = Ld^-1 E ; t = Ld^-1 (C'v)
    cta_trsm_lower<double>(n, Ld, n, n, E, n);
    if (threadIdx.x == blockDim.x - 1) {
      for (int i = 0; i < n; ++i) {
        double a = tv[i];
        for (int k = 0; k < i; ++k) a -= Ld[(long long)i * n + k] * tv[k];
        tv[i] = a / Ld[(long long)i * n + i];
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
    cta_trsm_lower_t<double>(n, Ld, n, n, E, n);
    if (threadIdx.x == blockDim.x - 1) {
      for (int i = n - 1; i >= 0; --i) {
        double a = tv[i];
        for (int k = i + 1; k < n; ++k) a -= Ld[(long long)k * n + i] * t2[k];
        t2[i] = a / Ld[(long long)i * n + i];
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

cudaError_t launch_link_solve_dual(const ProbTable& tab, int nprob, int x0_is_float, cudaStream_t st) {
  if (tab.probs) return cudaErrorInvalidValue;
  const int n = tab.single.n;
  size_t bytes = sizeof(double) * (4 * (size_t)n * n + 2 * (size_t)n);
  int optin = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (bytes > (size_t)optin - kStaticSmemReserve) bytes = 0;  // work matrices go to the global workspace
  static size_t configured = 0;
  if (bytes > 48 * 1024 && bytes > configured) {
    cudaError_t e = cudaFuncSetAttribute(link_solve_dual_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    configured = bytes;
  }
  link_solve_dual_kernel<<<nprob, kBlock, bytes, st>>>(tab, x0_is_float, (long long)bytes);
  return cudaGetLastError();
}

}  // namespace lqr
