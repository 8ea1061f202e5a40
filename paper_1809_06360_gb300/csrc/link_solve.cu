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
  if (threadIdx.x == 0) s_flag = *(volatile int*)pd.status;
  __syncthreads();
  if (s_flag != 0) return;
  __syncthreads();
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

}  // namespace lqr
