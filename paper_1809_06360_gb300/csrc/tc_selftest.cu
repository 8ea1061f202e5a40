// Self-test of the tensor-core product unit of the segment sweep on the
// current GPU: the tcgen05 TF32 products in the forms the sweep issues them
// (A from shared memory and from TMEM, 128-row tiles at row offsets 0 and 64,
// N = 64, 128 and 192, accumulation with a negated A) against CUDA-core FP32
// products of the same operands. Deterministic operands from a hash of the
// indices; one CTA.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lqr_internal.cuh"
#include "tc_sm100.cuh"

namespace lqr {
namespace {

constexpr int kTB = 512;
constexpr int kRab = 192, kRv = 128, kK = 128;
constexpr long long kSpin = 1LL << 24;

__device__ __forceinline__ float hval(int r, int k, int salt) {
  uint32_t x = (uint32_t)r * 0x9E3779B1u ^ (uint32_t)k * 0x85EBCA77u ^ (uint32_t)salt * 0xC2B2AE3Du;
  x ^= x >> 15;
  x *= 0x2C1B3C6Du;
  x ^= x >> 12;
  x *= 0x297A2D39u;
  x ^= x >> 15;
  return (float)(x & 0xFFFF) / 32768.0f - 1.0f;
}

// out: [0] |D1 - ref|/|ref| (SS, N=128), [1] TS N=192, [2] TS N=64 at row
// offset 64, [3] |D5| / |ref5| after D5 = X - X with X = SS at row offset 64,
// [4] 1 if a wait ran out.
__global__ void __launch_bounds__(kTB, 1) tc_selftest_kernel(double* out, float* ref1) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t s_bar;
  __shared__ uint32_t s_tmem;
  __shared__ float s_red[4][kTB / 32];
  __shared__ float s_mag[4][kTB / 32];
  // swizzle atoms need a 1024-byte-aligned base (1024 bytes of slack are allocated)
  unsigned char* smem = smem_raw + ((1024u - (tc::smem_addr(smem_raw) & 1023u)) & 1023u);
  float* sAB = reinterpret_cast<float*>(smem);  // 192 rows x 128 K, swizzled
  float* sV = sAB + kRab * kK;                  // 128 rows x 128 K, swizzled
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  for (int e = t; e < kRab * kK; e += kTB) tc::sw_at(sAB, kRab, e / kK, e % kK) = hval(e / kK, e % kK, 1);
  for (int e = t; e < kRv * kK; e += kTB) tc::sw_at(sV, kRv, e / kK, e % kK) = hval(e / kK, e % kK, 2);
  if (warp == 0) tc::tmem_alloc(&s_tmem, 512);
  if (t == 0) {
    tc::mbar_init(&s_bar, 1);
    tc::mbar_fence_init();
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = s_tmem;
  const uint32_t aAB = tc::smem_addr(sAB), aV = tc::smem_addr(sV);
  int timed_out = 0;
  if (t == 0) {
    // D1 (cols 0..127) = AB[0:128] V'
    for (int s = 0; s < kK / 8; ++s)
      tc::mma_ss(tm + 0, tc::sdesc_k(aAB, kRab, s), tc::sdesc_k(aV, kRv, s), tc::idesc_tf32(128, 128, false), s > 0);
    // D5 (cols 384..511) = AB[64:192] V' - AB[64:192] V'
    for (int s = 0; s < kK / 8; ++s)
      tc::mma_ss(tm + 384, tc::sdesc_k(aAB + 64 * 128, kRab, s), tc::sdesc_k(aV, kRv, s),
                 tc::idesc_tf32(128, 128, false), s > 0);
    for (int s = 0; s < kK / 8; ++s)
      tc::mma_ss(tm + 384, tc::sdesc_k(aAB + 64 * 128, kRab, s), tc::sdesc_k(aV, kRv, s),
                 tc::idesc_tf32(128, 128, true), 1);
    tc::commit(&s_bar);
  }
  if (!tc::mbar_wait(&s_bar, 0, kSpin)) timed_out = 1;
  tc::fence_after_sync();
  if (t == 0 && !timed_out) {
    // D2 (cols 128..319) = D1 AB', A from TMEM; D3 (cols 320..383) = D1 AB[128:192]'
    for (int s = 0; s < kK / 8; ++s)
      tc::mma_ts(tm + 128, tm + 8 * s, tc::sdesc_k(aAB, kRab, s), tc::idesc_tf32(128, 192, false), s > 0);
    for (int s = 0; s < kK / 8; ++s)
      tc::mma_ts(tm + 320, tm + 8 * s, tc::sdesc_k(aAB + 128 * 128, kRab, s), tc::idesc_tf32(128, 64, false), s > 0);
    tc::commit(&s_bar);
  }
  if (!timed_out && !tc::mbar_wait(&s_bar, 1, kSpin)) timed_out = 1;
  tc::fence_after_sync();
  // references on the CUDA cores from the same shared-memory operands (ref1: 128 x 128 in global memory)
  for (int e = t; e < 128 * 128; e += kTB) {
    const int j = e / 128, i = e % 128;
    float a = 0.0f;
    for (int k = 0; k < kK; ++k) a = fmaf(tc::sw_get(sAB, kRab, j, k), tc::sw_get(sV, kRv, i, k), a);
    ref1[e] = a;
  }
  __syncthreads();
  // each thread: its TMEM lane row, 16-column groups dealt over the 4 warps of its quadrant
  const int row = 32 * (warp & 3) + lane, grp = warp >> 2;
  const uint32_t lane_base = tm + ((uint32_t)(32 * (warp & 3)) << 16);
  float err[4] = {0, 0, 0, 0}, mag[4] = {0, 0, 0, 0};
  for (int c0 = 16 * grp; c0 < 512; c0 += 64) {
    float v[16];
    tc::tmem_ld16(lane_base + c0, v);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int c = c0 + q;
      float ref;
      int slot;
      if (c < 128) {
        ref = ref1[row * 128 + c];
        slot = 0;
      } else if (c < 320) {
        const int l = c - 128;
        float a = 0.0f;
        for (int i = 0; i < 128; ++i) a = fmaf(ref1[row * 128 + i], tc::sw_get(sAB, kRab, l, i), a);
        ref = a;
        slot = 1;
      } else if (c < 384) {
        const int l = 128 + (c - 320);
        float a = 0.0f;
        for (int i = 0; i < 128; ++i) a = fmaf(ref1[row * 128 + i], tc::sw_get(sAB, kRab, l, i), a);
        ref = a;
        slot = 2;
      } else {  // X - X: compared with the magnitude of X
        float a = 0.0f;
        for (int k = 0; k < kK; ++k) a = fmaf(tc::sw_get(sAB, kRab, row + 64, k), tc::sw_get(sV, kRv, c - 384, k), a);
        ref = a;
        slot = 3;
      }
      const float d = (slot == 3) ? v[q] : v[q] - ref;
      err[slot] = fmaxf(err[slot], fabsf(d));
      mag[slot] = fmaxf(mag[slot], fabsf(ref));
    }
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    float e = err[s], m = mag[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e = fmaxf(e, __shfl_xor_sync(0xffffffffu, e, o));
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if (lane == 0) {
      s_red[s][warp] = e;
      s_mag[s][warp] = m;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (t == 0) {
    for (int s = 0; s < 4; ++s) {
      float e = 0.0f, m = 0.0f;
      for (int w = 0; w < kTB / 32; ++w) {
        e = fmaxf(e, s_red[s][w]);
        m = fmaxf(m, s_mag[s][w]);
      }
      out[s] = m > 0.0f ? (double)e / (double)m : (double)e;
    }
  }
  if (t == 0) out[4] = 0.0;
  __syncthreads();
  if (timed_out && lane == 0) out[4] = 1.0;
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tm, 512);
}

}  // namespace
}  // namespace lqr

using namespace lqr;

extern "C" lqr_status lqr_tc_selftest(int device, double* errs) {
  if (!errs) return LQR_ERR_INVALID_ARG;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return LQR_ERR_CUDA;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  double* d = nullptr;
  lqr_status st = LQR_OK;
  const size_t bytes = sizeof(float) * ((size_t)kRab * kK + (size_t)kRv * kK) + 1024;
  if (cudaMalloc(&d, 5 * sizeof(double) + sizeof(float) * 128 * 128) != cudaSuccess) {
    cudaGetLastError();
    st = LQR_ERR_OOM;
  } else if (cudaFuncSetAttribute(tc_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
             cudaSuccess) {
    cudaGetLastError();
    st = LQR_ERR_CUDA;
  } else {
    tc_selftest_kernel<<<1, kTB, bytes>>>(d, reinterpret_cast<float*>(d + 5));
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(errs, d, 5 * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = LQR_ERR_CUDA;
    else if (errs[4] != 0.0)
      st = LQR_ERR_TIMEOUT;
  }
  if (d) cudaFree(d);
  if (prev >= 0) cudaSetDevice(prev);
  return st;
}

namespace lqr {
namespace {
__global__ void rcp_newton_kernel(const double* d, double* y, int count) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) y[i] = rcp_newton(d[i]);
}
}  // namespace
}  // namespace lqr

extern "C" lqr_status lqr_rcp_newton_check(const double* d, double* y, int count, void* stream) {
  if (!d || !y || count < 0) return LQR_ERR_INVALID_ARG;
  if (count == 0) return LQR_OK;
  const int grid = (count + 255) / 256 < 1024 ? (count + 255) / 256 : 1024;
  rcp_newton_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(d, y, count);
  return cudaGetLastError() == cudaSuccess ? LQR_OK : LQR_ERR_CUDA;
}
