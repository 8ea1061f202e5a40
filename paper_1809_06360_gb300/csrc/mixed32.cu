// LQR_MIXED_FP32 support: element-type conversions between the caller's FP64
// arrays and the FP32 working copies, and the refinement update from FP32
// corrections (w <- w - delta in FP64; Section II-C's KKT system, Eq. 3).
#include <cuda_runtime.h>

#include "lqr_internal.cuh"

namespace lqr {

// Up to kMaxConv arrays converted in one launch; grid-stride over each.
template <typename S, typename D>
__global__ void convert_kernel(ConvTable<S, D> tab, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int a = 0; a < tab.count; ++a) {
    const S* src = tab.src[a];
    D* dst = tab.dst[a];
    const size_t n = tab.n[a];
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += stride)
      dst[e] = static_cast<D>(src[e]);
  }
}

template <typename S, typename D>
cudaError_t launch_convert(const ConvTable<S, D>& tab, const int* skip, cudaStream_t st) {
  if (tab.count == 0) return cudaSuccess;
  convert_kernel<S, D><<<4 * device_sm_count(), 256, 0, st>>>(tab, skip);
  return cudaGetLastError();
}

// w <- w - delta with FP64 w (the caller's solution) and FP32 delta.
__global__ void refine_update_f32_kernel(ProbDesc pd, const float* dk, const float* dx, const float* du,
                                         const float* dl, const float* dp, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  if (*(volatile int*)pd.status != 0) return;
  const int n = pd.n, m = pd.m, T = pd.T;
  const size_t nx = (size_t)(T + 1) * n, nu = (size_t)T * m;
  double* k = static_cast<double*>(pd.k);
  double* x = static_cast<double*>(pd.x);
  double* u = static_cast<double*>(pd.u);
  double* l = static_cast<double*>(pd.lam);
  double* p = static_cast<double*>(pd.p);
  // x, lambda, p have (T+1) n entries and u, k have T m: either may be the longer
  const size_t ne = nx > nu ? nx : nu;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < ne; e += (size_t)gridDim.x * blockDim.x) {
    if (e < nx) {
      if (x) x[e] -= (double)dx[e];
      if (l) l[e] -= (double)dl[e];
      if (p && dp) p[e] -= (double)dp[e];
    }
    if (e < nu) {
      if (u) u[e] -= (double)du[e];
      if (k) k[e] -= (double)dk[e];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) pd.report[3] += 1.0;
}

cudaError_t launch_refine_update_f32(const ProbDesc& pd, const float* dk, const float* dx, const float* du,
                                     const float* dl, const float* dp, const int* skip, cudaStream_t st) {
  refine_update_f32_kernel<<<2 * device_sm_count(), 256, 0, st>>>(pd, dk, dx, du, dl, dp, skip);
  return cudaGetLastError();
}

template cudaError_t launch_convert<double, float>(const ConvTable<double, float>&, const int*, cudaStream_t);
template cudaError_t launch_convert<float, double>(const ConvTable<float, double>&, const int*, cudaStream_t);

}  // namespace lqr
