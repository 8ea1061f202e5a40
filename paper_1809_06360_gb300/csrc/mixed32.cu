// LQR_MIXED_FP32 support: element-type conversions between the caller's FP64
// arrays and the FP32 working copies, and the refinement update from FP32
// corrections (w <- w - delta in FP64; Section II-C's KKT system, Eq. 3).
#include <cuda_runtime.h>

#include "lqr_internal.cuh"

namespace lqr {

// FP64 -> FP32 with rounding to nearest, ties to even (IEEE), by integer
// operations on the bit pattern: the conversion instruction would hold the
// sub-partition's FP64 pipe for 64 cycles per warp. Normal results round the
// 52-bit significand at bit 29; results below the normal range are formed as
// multiples of 2^-149 the same way; beyond the range infinity; NaN stays NaN.
__device__ __forceinline__ float f64_to_f32_rn(double v) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  const unsigned int sign = static_cast<unsigned int>(b >> 32) & 0x80000000u;
  const int e = static_cast<int>((b >> 52) & 0x7FF);
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  unsigned int r;
  if (e >= 897 && e <= 1150) {
    const unsigned int m24 = static_cast<unsigned int>(mant >> 29);
    const unsigned int rem = static_cast<unsigned int>(mant & 0x1FFFFFFFull);
    const unsigned int up = (rem > 0x10000000u) | ((rem == 0x10000000u) & (m24 & 1u));
    r = ((static_cast<unsigned int>(e - 896) << 23) | m24) + up;
  } else if (e > 1150) {
    r = 0x7F800000u | ((e == 0x7FF && mant) ? 0x400000u : 0u);
  } else {
    const int shift = 926 - e;  // >= 30
    if (shift >= 54) {
      r = 0u;
    } else {
      const unsigned long long F = mant | (1ull << 52);
      const unsigned int q = static_cast<unsigned int>(F >> shift);
      const unsigned long long rem = F & ((1ull << shift) - 1), half = 1ull << (shift - 1);
      r = q + static_cast<unsigned int>((rem > half) | ((rem == half) & (q & 1u)));
    }
  }
  return __uint_as_float(sign | r);
}

template <typename S, typename D>
__device__ __forceinline__ D convert_one(S v) {
  return static_cast<D>(v);
}
template <>
__device__ __forceinline__ float convert_one<double, float>(double v) {
  return f64_to_f32_rn(v);
}

// Up to kMaxConv arrays converted in one launch; grid-stride over each, four
// independent loads per thread in flight (coalesced across the warp). A source
// may be host memory mapped into the device's address space, read once over the
// host link, with `raw` taking the unconverted copy into device memory.
constexpr int kConvUnroll = 4;
template <typename S, typename D>
__global__ void __launch_bounds__(256) convert_kernel(ConvTable<S, D> tab, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int a = 0; a < tab.count; ++a) {
    const S* __restrict__ src = tab.src[a];
    D* __restrict__ dst = tab.dst[a];
    S* __restrict__ raw = tab.raw[a];
    const size_t n = tab.n[a];
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += kConvUnroll * stride) {
      S v[kConvUnroll];
#pragma unroll
      for (int u = 0; u < kConvUnroll; ++u) {
        const size_t i = e + u * stride;
        v[u] = i < n ? src[i] : S(0);
      }
#pragma unroll
      for (int u = 0; u < kConvUnroll; ++u) {
        const size_t i = e + u * stride;
        if (i < n) {
          dst[i] = convert_one<S, D>(v[u]);
          if (raw) raw[i] = v[u];
        }
      }
    }
  }
}

template <typename S, typename D>
cudaError_t launch_convert(const ConvTable<S, D>& tab, const int* skip, cudaStream_t st) {
  if (tab.count == 0) return cudaSuccess;
  // one wave: as many CTAs as the multiprocessors hold at once
  static int per_sm = 0;
  if (per_sm == 0 &&
      (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, convert_kernel<S, D>, 256, 0) != cudaSuccess ||
       per_sm < 1))
    per_sm = 4;
  convert_kernel<S, D><<<per_sm * device_sm_count(), 256, 0, st>>>(tab, skip);
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

}  // namespace lqr

extern "C" lqr_status lqr_convert_f64_to_f32(const double* src, float* dst, long long count, void* stream) {
  if (count < 0 || (count > 0 && (!src || !dst))) return LQR_ERR_INVALID_ARG;
  if (count == 0) return LQR_OK;
  lqr::ConvTable<double, float> ct;
  ct.count = 0;
  ct.add(src, dst, static_cast<size_t>(count));
  return lqr::launch_convert(ct, nullptr, static_cast<cudaStream_t>(stream)) == cudaSuccess ? LQR_OK : LQR_ERR_CUDA;
}

namespace lqr {
template cudaError_t launch_convert<float, double>(const ConvTable<float, double>&, const int*, cudaStream_t);

}  // namespace lqr
