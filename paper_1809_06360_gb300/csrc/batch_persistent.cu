// Step A10: a batch of independent problems of uneven n, m, T in one
// persistent launch. When every problem runs as one segment (the batch has at
// least one problem per SM, or the autotuner found this schedule faster), a
// grid of resident 512-thread CTAs takes problems from a queue ordered by
// decreasing work (longest processing time first, so the long problems do not
// end up in the tail) through an atomic ticket, and solves each one whole:
// the FP32 Riccati sweep from the terminal cost (the serial recursion of
// Section III-A; the body of the FP32 segment sweep), then the rollout with
// the multipliers of Eq. 3 and the objective (the body of the FP32 rollout),
// then the objective into the problem's report. No CTA waits for another.
#include <cuda_runtime.h>

#include "lqr_internal.cuh"
#include "rollout_f32_body.cuh"
#include "sweep_f32_body.cuh"

namespace lqr {

template <int SHAPE>  // p4_shape of the largest m of the batch
__global__ void __launch_bounds__(kSweepBlock, 1) batch_persistent_kernel(ProbTable tab, const int* order, int* ticket,
                                                                          int want_lam, int nmax, int mmax,
                                                                          int store_P) {
  __shared__ int s_p;
  for (;;) {
    if (threadIdx.x == 0) {
      const int i = atomicAdd(ticket, 1);
      s_p = i < tab.nprob ? order[i] : -1;
    }
    __syncthreads();
    const int p = s_p;
    __syncthreads();  // every thread has read the ticket before it is reused
    if (p < 0) return;
    const ProbDesc& pd = tab.probs[p];
    const int unit = pd.unit0;  // one segment per problem
    {
      const WsLayout wl = ws_layout(pd.n, 1);
      double* z = pd.ws + wl.z;  // the start state of the one segment
      const float* x0 = static_cast<const float*>(pd.x0);
      for (int i = threadIdx.x; i < pd.n; i += blockDim.x) z[i] = static_cast<double>(x0[i]);
    }
    seg_sweep_f32_unit<SHAPE>(tab, unit, 0, store_P);  // K_t, k_t from the terminal cost
    __threadfence();
    __syncthreads();
    rollout_f32_unit(tab, unit, want_lam, nmax, mmax);  // x_t, u_t, lambda_t, objective partial
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      if (*(volatile int*)pd.status != 0) {
        pd.report[0] = 0.0;
      } else {
        const WsLayout wl = ws_layout(pd.n, 1);
        const double s = pd.ws[wl.costp];
        if (!isfinite(s)) raise_status(pd.status, LQR_ERR_NONFINITE, -1);
        pd.report[0] = s;
      }
    }
  }
}

bool batch_persistent_supported(int nmax, int mmax, long long smem_budget) {
  return p4_shape(mmax) >= 0 && fast_sweep_smem_bytes(nmax, mmax) <= smem_budget &&
         rollout_f32_smem_bytes(nmax, mmax) <= smem_budget && ((nmax + 3) & ~3) <= kRollBlock;
}

cudaError_t launch_batch_persistent(const ProbTable& tab, const int* order, int* ticket, int want_lam, int nmax,
                                    int mmax, int store_P, int num_sms, cudaStream_t st) {
  const long long a = fast_sweep_smem_bytes(nmax, mmax), b = rollout_f32_smem_bytes(nmax, mmax);
  const size_t bytes = (size_t)(a > b ? a : b);
  const int shape = p4_shape(mmax);
  const void* fn = shape == 0 ? (const void*)batch_persistent_kernel<0>
                 : shape == 1 ? (const void*)batch_persistent_kernel<1>
                 : shape == 2 ? (const void*)batch_persistent_kernel<2>
                              : (const void*)batch_persistent_kernel<3>;
  cudaError_t e = raise_dyn_smem(fn, bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kSweepBlock, bytes);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int grid = per_sm * num_sms;  // every CTA resident: the queue needs no more
  if (grid > tab.nprob) grid = tab.nprob;
  switch (shape) {
    case 0: batch_persistent_kernel<0><<<grid, kSweepBlock, bytes, st>>>(tab, order, ticket, want_lam, nmax, mmax, store_P); break;
    case 1: batch_persistent_kernel<1><<<grid, kSweepBlock, bytes, st>>>(tab, order, ticket, want_lam, nmax, mmax, store_P); break;
    case 2: batch_persistent_kernel<2><<<grid, kSweepBlock, bytes, st>>>(tab, order, ticket, want_lam, nmax, mmax, store_P); break;
    default: batch_persistent_kernel<3><<<grid, kSweepBlock, bytes, st>>>(tab, order, ticket, want_lam, nmax, mmax, store_P); break;
  }
  return cudaGetLastError();
}

}  // namespace lqr
