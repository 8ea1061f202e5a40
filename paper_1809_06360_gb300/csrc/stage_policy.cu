// Per-stage reconstruction of the global policy, all stages at once.
//
// The constraint-explicit sweep of Section II-B leaves, at every stage t of a
// segment j < K-1, the cost to go of the rest of the segment as a function of
// the stage's state and the segment's end state (Eq. 9 at stage t),
//   J_t(x, z) = 1/2 x'Vxx x + z'Vzx x + 1/2 z'Vzz z + vx'x + vz'z,
// and the stage's own policy u_t = Kx x + Kz z + k1. Once the link solve has
// given the global value 1/2 z'P_e z + p_e'z at the segment's end point
// (Section III-A), every stage whose constraint_to_go has no rows left (any end
// state is reachable from it) gets its global cost to go and policy from the
// minimising end state z* = -(Vzz + P_e)^-1 (Vzx x + vz + p_e):
//   P_t = Vxx - Vzx'(Vzz + P_e)^-1 Vzx,   p_t = vx - Vzx'(Vzz + P_e)^-1 (vz + p_e),
//   K_t = Kx - Kz (Vzz + P_e)^-1 Vzx,      k_t = k1 - Kz (Vzz + P_e)^-1 (vz + p_e),
// independently of the other stages: one CTA per stage, in place of the
// sequential policy sweep of step A4. P_t comes out as a difference of two
// terms that both grow near the segment end, so the cancellation there costs
// digits that the sequential sweep keeps.
// FP64: one Cholesky factor of Vzz + P_e = L L', then X = L^-1 [Vzx | vz + p_e],
// P_t = Vxx - X_x'X_x, p_t = vx - X_x'x_v, Y = L^-T X, K_t = Kx - Kz Y_x,
// k_t = k1 - Kz y_v.
#include <cuda_runtime.h>

#include "cta_linalg.cuh"
#include "lqr_internal.cuh"

namespace lqr {

namespace {
constexpr int kSpBlock = 256;
}

size_t stage_policy_smem_bytes(int n, int on_chip) {
  return sizeof(double) * ((on_chip ? (size_t)n * n + (size_t)n * (n + 1) : 0) + (size_t)n);
}

__global__ void __launch_bounds__(kSpBlock) stage_policy_kernel(ProbDesc pd, int on_chip, double* scratch) {
  extern __shared__ __align__(16) double ssm[];
  __shared__ int s_flag;
  if (cta_should_exit(pd, &s_flag)) return;
  const int n = pd.n, m = pd.m, T = pd.T, K = pd.nseg;
  const int t = blockIdx.x;
  if (pd.stage_rank[t] != 0) return;  // the policy sweep covers this stage
  // segment of stage t: seg_begin(j) <= t < seg_begin(j + 1)
  int j = (int)(((long long)t * K) / T);
  while (j > 0 && seg_begin(T, K, j) > t) --j;
  while (j + 1 < K && seg_begin(T, K, j + 1) <= t) ++j;
  const size_t nn = (size_t)n * n;
  const int ld = n + 1;
  const WsLayout wl = ws_layout(n, K);
  const double* Pe = pd.ws + wl.Pi + (long long)(j + 1) * nn;
  const double* pe = pd.ws + wl.pi + (long long)(j + 1) * n;
  const double* sv = pd.stageV + (size_t)t * (3 * nn + 2 * n);
  const double* Vxx = sv;
  const double* Vzx = sv + nn;
  const double* Vzz = sv + 2 * nn;
  const double* vx = sv + 3 * nn;
  const double* vz = vx + n;
  double* Sm = on_chip ? ssm : scratch + (size_t)t * (nn + (size_t)n * ld);
  double* X = Sm + nn;  // n x (n + 1): [Vzx | vz + p_e]
  double* rd = ssm + (on_chip ? nn + (size_t)n * ld : 0);
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    Sm[e] = Vzz[e] + 0.5 * (Pe[e] + Pe[(size_t)(e % n) * n + e / n]);
    X[(size_t)(e / n) * ld + e % n] = Vzx[e];
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) X[(size_t)i * ld + n] = vz[i] + pe[i];
  if (threadIdx.x == 0) s_flag = 0;
  __syncthreads();
  cta_chol(n, Sm, n, &s_flag, rd);
  if (s_flag) {
    if (threadIdx.x == 0) raise_status(pd.status, LQR_ERR_NOT_PD, t);
    return;
  }
  cta_trsm_lower_warp(n, (const double*)Sm, n, ld, X, ld, (const double*)rd);
  __syncthreads();
  // P_t = Vxx - X_x'X_x, p_t = vx - X_x'x_v
  double* gP = static_cast<double*>(pd.P);
  double* gp = static_cast<double*>(pd.p);
  if (gP)
    cta_mm<4, 4, true, false, double>(n, n, n, X, ld, X, ld, EpiAdd<double, double>{gP + nn * t, n, -1.0, Vxx, n});
  if (gp) cta_mv<true, double>(n, n, X, ld, X + n, ld, EpiAdd<double, double>{gp + (size_t)n * t, 1, -1.0, vx, 1});
  __syncthreads();
  // Y = L^-T X, K_t = Kx - Kz Y_x, k_t = k1 - Kz y_v  ([Kx | Kz | k1] rows of the segment policy)
  cta_trsm_lower_t_warp(n, (const double*)Sm, n, ld, X, ld, (const double*)rd);
  __syncthreads();
  const int ldp = 2 * n + 1;
  const double* G = pd.segpol + (size_t)m * ldp * t;
  double* gK = static_cast<double*>(pd.K);
  double* gk = static_cast<double*>(pd.k);
  if (gK) cta_mm<4, 4, false, false, double>(m, n, n, G + n, ldp, X, ld, EpiAdd<double, double>{gK + (size_t)m * n * t, n, -1.0, G, ldp});
  if (gk) cta_mv<false, double>(m, n, G + n, ldp, X + n, ld, EpiAdd<double, double>{gk + (size_t)m * t, 1, -1.0, G + 2 * n, ldp});
  if (gP) {  // symmetric part of P_t
    __syncthreads();
    double* Pt = gP + nn * t;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e / n, c = e % n;
      if (c <= i) continue;
      const double a = 0.5 * (Pt[(size_t)i * n + c] + Pt[(size_t)c * n + i]);
      Pt[(size_t)i * n + c] = a;
      Pt[(size_t)c * n + i] = a;
    }
  }
}

cudaError_t launch_stage_policy(const ProbDesc& pd, int nstages, int on_chip, double* scratch, cudaStream_t st) {
  if (nstages <= 0) return cudaSuccess;
  const size_t bytes = stage_policy_smem_bytes(pd.n, on_chip);
  cudaError_t e = raise_dyn_smem((const void*)stage_policy_kernel, bytes);
  if (e != cudaSuccess) return e;
  stage_policy_kernel<<<nstages, kSpBlock, bytes, st>>>(pd, on_chip, scratch);
  return cudaGetLastError();
}

}  // namespace lqr
