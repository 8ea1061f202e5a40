// Steps A1 and A4 for FP32 data in the multiplier form: the same stage
// recursion as seg_sweep.cu (Eq. 13 terms, the Riccati update of Section II-B
// with the end-point multiplier as parameter, and the policy of Section III-A),
// laid out for throughput:
//  - the stage data [A_t | B_t | c_t] of the next stage is copied into the
//    other half of a two-slot shared-memory ring with cp.async while the
//    current stage computes, and Q_t, R_t, S_t, q_t, r_t of the current stage
//    arrive while T1 = V [A|B|c] is formed;
//  - every product runs on 4 x 4 register tiles with 128-bit shared loads over
//    n and m rounded up to multiples of 4 (zero padding);
//  - M_uu is inverted in place by the register-blocked Gauss-Jordan sweep (one
//    barrier per pivot) and the value update uses H = M_uu^-1 [M_ux | M_zu' | m_u]:
//        V_xx = M_xx - M_ux'H_x   v_x = m_x - M_ux'h
//        Z    = M_zx - M_zu H_x    -W  = -W - M_zu H_z    w = m_z - M_zu h
//    (K_t = -H_x, k_t = -h), algebraically the Cholesky form W'W of the
//    generic kernel.
// One CTA per segment; used when the padded plan fits in shared memory.
#include "sweep_f32_body.cuh"

namespace lqr {

long long fast_sweep_smem_bytes(int n, int m) { return fast_sweep_smem_bytes_inl(n, m); }

template <int SHAPE>
__global__ void __launch_bounds__(kSweepBlock, 1) seg_sweep_f32_kernel(ProbTable tab, int phase, int store_P) {
  seg_sweep_f32_unit<SHAPE>(tab, (int)blockIdx.x, phase, store_P);
}

bool fast_sweep_supported(int n, int m, long long smem_budget) {
  return fast_sweep_smem_bytes(n, m) <= smem_budget && p4_shape(m) >= 0;
}

// cudaErrorNotSupported (nothing launched) when the plan does not fit.
cudaError_t launch_seg_sweep_f32(const ProbTable& tab, int nunits, int phase, int nmax, int mmax,
                                 long long smem_budget, int store_P, cudaStream_t st) {
  const long long bytes = fast_sweep_smem_bytes(nmax, mmax);
  if (bytes > smem_budget || p4_shape(mmax) < 0) return cudaErrorNotSupported;
  const int shape = p4_shape(mmax);
  const void* fn = shape == 0 ? (const void*)seg_sweep_f32_kernel<0>
                 : shape == 1 ? (const void*)seg_sweep_f32_kernel<1>
                 : shape == 2 ? (const void*)seg_sweep_f32_kernel<2>
                              : (const void*)seg_sweep_f32_kernel<3>;
  cudaError_t e = raise_dyn_smem(fn, (size_t)bytes);
  if (e != cudaSuccess) return e;
  switch (shape) {
    case 0: seg_sweep_f32_kernel<0><<<nunits, kSweepBlock, (size_t)bytes, st>>>(tab, phase, store_P); break;
    case 1: seg_sweep_f32_kernel<1><<<nunits, kSweepBlock, (size_t)bytes, st>>>(tab, phase, store_P); break;
    case 2: seg_sweep_f32_kernel<2><<<nunits, kSweepBlock, (size_t)bytes, st>>>(tab, phase, store_P); break;
    default: seg_sweep_f32_kernel<3><<<nunits, kSweepBlock, (size_t)bytes, st>>>(tab, phase, store_P); break;
  }
  return cudaGetLastError();
}

}  // namespace lqr
