// The FP32 multiplier-form segment sweep (steps A1/A4) as a device function of
// one CTA, shared by seg_sweep_f32_kernel and the persistent batched kernel.
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
#pragma once
#include <cuda_runtime.h>

#include "cta_linalg.cuh"
#include "lqr_internal.cuh"

namespace lqr {

struct FastPlan {
  int N, M, ldAB, ldF, ldV, ldM;  // ldV, ldM: padded row strides of the n x n and m x m buffers
  long long V, Z, Wn, vx, vz, ab, Q, R, S, q, r, T1, F, Muu, Mzx, mz, colbuf, total;  // float offsets
};

__host__ __device__ inline FastPlan fast_plan(int n, int m) {
  FastPlan P;
  P.N = (n + 3) & ~3;
  P.M = (m + 3) & ~3;
  P.ldAB = P.N + P.M + 4;
  P.ldF = 2 * P.N + 4;
  P.ldV = P.N + 4;  // rows four apart in different banks
  P.ldM = P.M + 4;
  const long long N = P.N, M = P.M, LV = P.ldV, LM = P.ldM;
  long long o = 0;
  P.V = o;   o += N * LV;
  P.Z = o;   o += N * LV;
  P.Wn = o;  o += N * LV;
  P.vx = o;  o += N;
  P.vz = o;  o += N;
  P.ab = o;  o += 2 * N * P.ldAB;
  P.Q = o;   o += N * LV;
  P.R = o;   o += M * M;
  P.S = o;   o += M * N;
  P.q = o;   o += N;
  P.r = o;   o += M;
  P.T1 = o;  o += (N * P.ldAB > M * P.ldF) ? N * P.ldAB : M * P.ldF;  // T1, then H
  P.F = o;   o += M * P.ldF;
  P.Muu = o; o += M * LM;
  P.Mzx = o; o += N * LV;
  P.mz = o;  o += N;
  P.colbuf = o; o += p4_scratch_floats(m);  // scratch of the block elimination
  P.total = (o + 3) & ~3LL;
  return P;
}

inline long long fast_sweep_smem_bytes_inl(int n, int m) { return 4 * fast_plan(n, m).total; }

namespace {

// rows x cols floats from global (row stride lds) into shared (row stride ldd);
// 16-byte copies when v16 (rows and pointers 16-byte aligned), else 4-byte.
__device__ __forceinline__ void copy_rows(float* dst, int ldd, const float* src, int lds, int rows, int cols,
                                          bool v16) {
  if (v16) {
    const int per = cols >> 2;
    for (int e = threadIdx.x; e < rows * per; e += blockDim.x) {
      const int i = e / per, c = e - i * per;
      cp_async16(dst + (long long)i * ldd + 4 * c, src + (long long)i * lds + 4 * c);
    }
  } else {
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
      const int i = e / cols, c = e - i * cols;
      cp_async4(dst + (long long)i * ldd + c, src + (long long)i * lds + c);
    }
  }
}

__device__ __forceinline__ bool al16(const void* p) { return (reinterpret_cast<unsigned long long>(p) & 15) == 0; }

// M_uu^-1 in place, 4 x 4 pivot blocks, one register block per thread (512 threads)
template <int SHAPE>
__device__ __forceinline__ void invert_muu(int m, float* Muu, int M, int* flag, float* scr) {
  if (SHAPE == 0) cta_spd_inverse_p4<1, 4>(m, Muu, M, flag, scr, true);
  else if (SHAPE == 1) cta_spd_inverse_p4<2, 4>(m, Muu, M, flag, scr, true);
  else if (SHAPE == 2) cta_spd_inverse_p4<4, 4>(m, Muu, M, flag, scr, true);
  else cta_spd_inverse_p4<4, 8>(m, Muu, M, flag, scr, true);
}

}  // namespace

constexpr int kSweepBlock = 512;  // 16 warps: latency hiding for the small products

// The sweep of one unit (segment) by the calling 512-thread CTA: the body of
// seg_sweep_f32_kernel, also called per problem by the persistent batched kernel.
template <int SHAPE>  // p4_shape(m) of the largest m in the launch
__device__ __forceinline__ void seg_sweep_f32_unit(const ProbTable& tab, int unit, int phase, int store_P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_flag;
  const ProbDesc& pd = prob_of_unit(tab, unit);
  const int seg = unit - pd.unit0;
  const int n = pd.n, m = pd.m, T = pd.T, K = pd.nseg;
  if (cta_should_exit(pd, &s_flag)) return;
  const bool last = (seg == K - 1);
  int mode;
  if (phase == 0) {
    mode = last ? MODE_TERMINAL : MODE_PARAM;
  } else {
    if (last) return;
    mode = MODE_POLICY;
  }
  const bool param = (mode == MODE_PARAM);
  const int t0 = seg_begin(T, K, seg), t1 = seg_begin(T, K, seg + 1);
  const FastPlan P = fast_plan(n, m);
  const int N = P.N, M = P.M, ldAB = P.ldAB, ldF = P.ldF, LV = P.ldV, LM = P.ldM;
  float* sm = reinterpret_cast<float*>(smem);
  float* V = sm + P.V;
  float* Z = sm + P.Z;
  float* Wn = sm + P.Wn;
  float* vx = sm + P.vx;
  float* vz = sm + P.vz;
  float* Qs = sm + P.Q;
  float* Rs = sm + P.R;
  float* Ss = sm + P.S;
  float* qs = sm + P.q;
  float* rs = sm + P.r;
  float* T1 = sm + P.T1;
  float* H = T1;  // after the M terms
  float* F = sm + P.F;
  float* Muu = sm + P.Muu;
  float* Mzx = sm + P.Mzx;
  float* mz = sm + P.mz;
  float* colbuf = sm + P.colbuf;
  const int cN = N + M;  // column of c in [A | B | c]

  const WsLayout wl = ws_layout(n, K);
  double* summ = pd.ws + wl.summ + (long long)seg * (3LL * n * n + 2 * n);
  const float* gA = static_cast<const float*>(pd.A);
  const float* gB = static_cast<const float*>(pd.B);
  const float* gc = static_cast<const float*>(pd.c);
  const float* gQ = static_cast<const float*>(pd.Q);
  const float* gR = static_cast<const float*>(pd.R);
  const float* gS = static_cast<const float*>(pd.S);
  const float* gq = static_cast<const float*>(pd.q);
  const float* gr = static_cast<const float*>(pd.r);
  float* gK = static_cast<float*>(pd.K);
  float* gk = static_cast<float*>(pd.k);
  float* gP = static_cast<float*>(pd.P);
  float* gp = static_cast<float*>(pd.p);
  const long long nn = (long long)n * n, nm = (long long)n * m, mm = (long long)m * m;
  const bool v16 = (n % 4 == 0) && (m % 4 == 0) && al16(gA) && al16(gB) && al16(gQ) && al16(gR) &&
                   (gS == nullptr || al16(gS));

  // ---- zero everything (padding stays zero), initial value function -----------
  {
    float4* z4 = reinterpret_cast<float4*>(smem);
    for (long long i = threadIdx.x; i < P.total / 4; i += blockDim.x) z4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (threadIdx.x == 0) s_flag = 0;
  }
  __syncthreads();
  auto issue_ab = [&](int t) {  // [A_t | B_t | c_t] into ring slot (t1 - 1 - t) & 1
    if (t >= t0) {
      float* ab = sm + P.ab + (long long)((t1 - 1 - t) & 1) * N * ldAB;
      copy_rows(ab, ldAB, gA + nn * t, n, n, n, v16);
      copy_rows(ab + N, ldAB, gB + nm * t, m, n, m, v16);
      for (int i = threadIdx.x; i < n; i += blockDim.x) cp_async4(ab + (long long)i * ldAB + cN, gc + (long long)n * t + i);
    }
    cp_async_commit();
  };
  issue_ab(t1 - 1);
  if (mode == MODE_PARAM) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) Z[i * LV + i] = 1.0f;
  } else if (mode == MODE_TERMINAL) {
    const float* QT = gQ + nn * T;
    for (long long e = threadIdx.x; e < nn; e += blockDim.x) {
      const int i = (int)(e / n), j = (int)(e - (long long)i * n);
      V[i * LV + j] = 0.5f * (QT[(long long)i * n + j] + QT[(long long)j * n + i]);
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) vx[i] = gq[(long long)n * T + i];
  } else {
    const double* Pi = pd.ws + wl.Pi + (long long)(seg + 1) * nn;
    const double* pi = pd.ws + wl.pi + (long long)(seg + 1) * n;
    for (long long e = threadIdx.x; e < nn; e += blockDim.x) {
      const int i = (int)(e / n), j = (int)(e - (long long)i * n);
      V[i * LV + j] = static_cast<float>(Pi[e]);
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) vx[i] = static_cast<float>(pi[i]);
  }
  __syncthreads();
  if (store_P && gP && mode != MODE_PARAM && last) {  // P_T, p_T
    for (long long e = threadIdx.x; e < nn; e += blockDim.x) gP[nn * T + e] = V[(e / n) * LV + (e % n)];
    for (int i = threadIdx.x; i < n; i += blockDim.x) gp[(long long)n * T + i] = vx[i];
  }

  for (int t = t1 - 1; t >= t0; --t) {
    cp_async_wait<0>();
    __syncthreads();  // [A|B|c]_t in its slot; the previous stage is finished
    const float* ab = sm + P.ab + (long long)((t1 - 1 - t) & 1) * N * ldAB;
    // Q, R, S, q, r of this stage; the next stage's [A|B|c] is issued once they are
    // in, so that they do not queue behind it
    copy_rows(Qs, LV, gQ + nn * t, n, n, n, v16);
    copy_rows(Rs, M, gR + mm * t, m, m, m, v16);
    if (gS) copy_rows(Ss, N, gS + nm * t, n, m, n, v16);
    for (int i = threadIdx.x; i < n; i += blockDim.x) cp_async4(qs + i, gq + (long long)n * t + i);
    for (int a = threadIdx.x; a < m; a += blockDim.x) cp_async4(rs + a, gr + (long long)m * t + a);
    cp_async_commit();
    // ---- T1 = V [A|B|c] + [0|0|v_x] ----------------------------------------------
    if (SHAPE == 0) {
      // m <= 32: only T1_B = V B and T1_c = V c + v_x here, the inputs of M_uu and
      // m_u; T1_A = V A is formed beside the inverse below
      cta_mm4f<false>(N, M, N, V, LV, ab + N, ldAB, [&](int i, int j, float v) { T1[i * ldAB + N + j] = v; });
      cta_mm4f<false>(N, 4, N, V, LV, ab + cN, ldAB, [&](int i, int j, float v) {
        if (j == 0) T1[i * ldAB + cN] = v + vx[i];
      }, (N / 4) * (M / 4));
    } else {
      cta_mm4f<false>(N, ldAB, N, V, LV, ab, ldAB,
                      [&](int i, int j, float v) { T1[i * ldAB + j] = (j == cN) ? v + vx[i] : v; });
    }
    cp_async_wait<0>();  // this stage's Q, R, S, q, r
    __syncthreads();
    issue_ab(t - 1);  // in flight during the rest of this stage
    // ---- the M terms ---------------------------------------------------------------
    if (SHAPE == 0) {
      // M_uu = R + B'T1_B and m_u = r + B'T1_c first; then warp 0 inverts M_uu
      // (pivot columns by shuffles, no barrier) while the other 15 warps form
      // T1_A = V A, then M_xx, m_x, M_ux and (parametric) M_zu, m_z, M_zx, which
      // do not depend on the inverse.
      cta_mm4f<true>(M, M, N, ab + N, ldAB, T1 + N, ldAB,
                     [&](int a, int b, float v) { Muu[a * LM + b] = v + Rs[a * M + b]; });
      cta_mm4f<true>(M, 4, N, ab + N, ldAB, T1 + cN, ldAB, [&](int a, int j, float v) {
        if (j == 0) F[a * ldF + 2 * N] = v + rs[a];
      }, (M / 4) * (M / 4));
      __syncthreads();
      const int warp = (int)threadIdx.x >> 5;
      if (warp == 0) {
        warp_spd_inverse32(m, Muu, LM, &s_flag);
      } else {
        constexpr int kWorkers = kSweepBlock - 32;
        const int gtid = (int)threadIdx.x - 32;
        grp_mm4f<false>(gtid, kWorkers, N, N, N, V, LV, ab, ldAB, [&](int i, int j, float v) { T1[i * ldAB + j] = v; });
        NamedBar{2, kWorkers}();  // T1_A complete before M_xx overwrites V
        int rot = 0;
        grp_mm4f<true>(gtid, kWorkers, N, N, N, ab, ldAB, T1, ldAB,
                       [&](int i, int j, float v) { V[i * LV + j] = v + Qs[i * LV + j]; }, rot);
        rot += (N / 4) * (N / 4);
        grp_mm4f<true>(gtid, kWorkers, N, 4, N, ab, ldAB, T1 + cN, ldAB, [&](int i, int j, float v) {
          if (j == 0) vx[i] = v + qs[i];
        }, rot);
        rot += N / 4;
        grp_mm4f<true>(gtid, kWorkers, M, N, N, ab + N, ldAB, T1, ldAB,
                       [&](int a, int j, float v) { F[a * ldF + j] = v + Ss[a * N + j]; }, rot);
        rot += (M / 4) * (N / 4);
        if (param) {
          grp_mm4f<false>(gtid, kWorkers, N, M, N, Z, LV, ab + N, ldAB,
                          [&](int i, int a, float v) { F[a * ldF + N + i] = v; }, rot);
          rot += (N / 4) * (M / 4);
          grp_mm4f<false>(gtid, kWorkers, N, 4, N, Z, LV, ab + cN, ldAB, [&](int i, int j, float v) {
            if (j == 0) mz[i] = v + vz[i];
          }, rot);
          rot += N / 4;
          grp_mm4f<false>(gtid, kWorkers, N, N, N, Z, LV, ab, ldAB,
                          [&](int i, int j, float v) { Mzx[i * LV + j] = v; }, rot);
        }
      }
      __syncthreads();
    } else if (param && SHAPE == 1) {
      // Parametric sweep, m <= 64: B'T1 = [M_ux - S | M_uu - R | m_u - r] first;
      // then the first 256 threads invert M_uu (named barrier 1) while the others
      // form M_xx, m_x, M_zu, m_z, M_zx, which do not depend on it.
      cta_mm4f<true>(M, ldAB, N, ab + N, ldAB, T1, ldAB, [&](int a, int j, float v) {
        if (j < N) F[a * ldF + j] = v + Ss[a * N + j];
        else if (j < cN) Muu[a * LM + (j - N)] = v + Rs[a * M + (j - N)];
        else if (j == cN) F[a * ldF + 2 * N] = v + rs[a];
      });
      __syncthreads();
      constexpr int GT = 256;
      if ((int)threadIdx.x < GT) {
        grp_spd_inverse<4, 4>(m, Muu, LM, &s_flag, colbuf, colbuf + 2 * M, true, (int)threadIdx.x, GT, NamedBar{1, GT});
      } else {
        // M_xx = Q + A'T1_A (into V; the end-of-stage symmetrisation of V_xx takes
        // care of Q's antisymmetric part), m_x = q + A'T1_c, M_zu' = (Z B)' into
        // F[:, N:2N], m_z = w + Z c, M_zx = Z A, dealt round the group (rot)
        const int gtid = (int)threadIdx.x - GT, gthr = kSweepBlock - GT;
        int rot = 0;
        grp_mm4f<true>(gtid, gthr, N, N, N, ab, ldAB, T1, ldAB,
                       [&](int i, int j, float v) { V[i * LV + j] = v + Qs[i * LV + j]; }, rot);
        rot += (N / 4) * (N / 4);
        grp_mm4f<true>(gtid, gthr, N, 4, N, ab, ldAB, T1 + cN, ldAB, [&](int i, int j, float v) {
          if (j == 0) vx[i] = v + qs[i];
        }, rot);
        rot += N / 4;
        if (param) {
          grp_mm4f<false>(gtid, gthr, N, M, N, Z, LV, ab + N, ldAB,
                          [&](int i, int a, float v) { F[a * ldF + N + i] = v; }, rot);
          rot += (N / 4) * (M / 4);
          grp_mm4f<false>(gtid, gthr, N, 4, N, Z, LV, ab + cN, ldAB, [&](int i, int j, float v) {
            if (j == 0) mz[i] = v + vz[i];
          }, rot);
          rot += N / 4;
          grp_mm4f<false>(gtid, gthr, N, N, N, Z, LV, ab, ldAB, [&](int i, int j, float v) { Mzx[i * LV + j] = v; }, rot);
        }
      }
      __syncthreads();
    } else {
      // [A|B]'T1 in one product over the block: rows of A' give M_xx - Q (into V)
      // and m_x - q (columns [0, N) and cN), rows of B' give [M_ux - S | M_uu - R |
      // m_u - r]; the tiles of A'T1_B (= M_ux', not needed) are not formed. With the
      // parametric terms (m > 64) Z B, Z c, Z A join the same phase; then the whole
      // block inverts M_uu.
      const int tA = (N / 4) * (N / 4 + 1), tB = (M / 4) * (ldAB / 4);
      for (int tile = threadIdx.x; tile < tA + tB; tile += kSweepBlock) {
        int i0, j0;
        if (tile < tA) {
          i0 = (tile / (N / 4 + 1)) * 4;
          const int c = tile % (N / 4 + 1);
          j0 = (c < N / 4) ? 4 * c : cN;
        } else {
          i0 = N + ((tile - tA) / (ldAB / 4)) * 4;
          j0 = ((tile - tA) % (ldAB / 4)) * 4;
        }
        mm4f_tile<true>(i0, j0, N, ab, ldAB, T1, ldAB, [&](int i, int j, float v) {
          if (i < N) {
            if (j < N) V[i * LV + j] = v + Qs[i * LV + j];
            else if (j == cN) vx[i] = v + qs[i];
          } else {
            const int a = i - N;
            if (j < N) F[a * ldF + j] = v + Ss[a * N + j];
            else if (j < cN) Muu[a * LM + (j - N)] = v + Rs[a * M + (j - N)];
            else if (j == cN) F[a * ldF + 2 * N] = v + rs[a];
          }
        });
      }
      if (param) {
        int rot = (tA + tB) % kSweepBlock;
        cta_mm4f<false>(N, M, N, Z, LV, ab + N, ldAB, [&](int i, int a, float v) { F[a * ldF + N + i] = v; }, rot);
        rot += (N / 4) * (M / 4);
        cta_mm4f<false>(N, 4, N, Z, LV, ab + cN, ldAB, [&](int i, int j, float v) {
          if (j == 0) mz[i] = v + vz[i];
        }, rot);
        rot += N / 4;
        cta_mm4f<false>(N, N, N, Z, LV, ab, ldAB, [&](int i, int j, float v) { Mzx[i * LV + j] = v; }, rot);
      }
      __syncthreads();
      if (SHAPE == 1)
        grp_spd_inverse<2, 4>(m, Muu, LM, &s_flag, colbuf, colbuf + 2 * M, true, (int)threadIdx.x, kSweepBlock,
                              NamedBar{1, kSweepBlock});
      __syncthreads();
    }
    if (SHAPE >= 2) invert_muu<SHAPE>(m, Muu, LM, &s_flag, colbuf);
    if (s_flag) {
      if (threadIdx.x == 0) raise_status(pd.status, LQR_ERR_NOT_PD, t);
      cp_async_wait<0>();
      return;
    }
    // ---- H = M_uu^-1 [M_ux | M_zu' | m_u] ---------------------------------------------
    const int hcols = param ? ldF : ldF;  // [x | z | h] columns (the z block is zero outside the param mode)
    cta_mm4f<false>(M, hcols, M, Muu, LM, F, ldF, [&](int a, int j, float v) { H[a * ldF + j] = v; });
    __syncthreads();
    // ---- value update ---------------------------------------------------------------------
    int rot = 0;
    cta_mm4f<true>(N, N, M, F, ldF, H, ldF, [&](int i, int j, float v) { V[i * LV + j] -= v; }, rot);
    rot += (N / 4) * (N / 4);
    cta_mm4f<true>(N, 4, M, F, ldF, H + 2 * N, ldF, [&](int i, int j, float v) {
      if (j == 0) vx[i] -= v;
    }, rot);
    rot += N / 4;
    if (param) {
      cta_mm4f<true>(N, N, M, F + N, ldF, H, ldF, [&](int i, int j, float v) { Z[i * LV + j] = Mzx[i * LV + j] - v; },
                     rot);
      rot += (N / 4) * (N / 4);
      cta_mm4f<true>(N, N, M, F + N, ldF, H + N, ldF, [&](int i, int j, float v) { Wn[i * LV + j] -= v; }, rot);
      rot += (N / 4) * (N / 4);
      cta_mm4f<true>(N, 4, M, F + N, ldF, H + 2 * N, ldF, [&](int i, int j, float v) {
        if (j == 0) vz[i] = mz[i] - v;
      }, rot);
    } else {
      // policy K_t = -H_x, k_t = -h
      if (gK)
        for (int e = threadIdx.x; e < (int)nm; e += blockDim.x) {
          const int a = e / n, j = e - a * n;
          gK[nm * t + e] = -H[a * ldF + j];
        }
      if (gk)
        for (int a = threadIdx.x; a < m; a += blockDim.x) gk[(long long)m * t + a] = -H[a * ldF + 2 * N];
      if (pd.Minv) {  // M_uu^-1, kept for refinement corrections that reuse the factorisation
        float* gM = static_cast<float*>(pd.Minv) + mm * t;
        for (int e = threadIdx.x; e < (int)mm; e += blockDim.x) {
          const int a = e / m, b = e - a * m;
          gM[e] = Muu[a * LM + b];
        }
      }
    }
    __syncthreads();
    // symmetrise V_xx
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
      const int i = e / N, j = e - i * N;
      if (j > i) {
        const float s = 0.5f * (V[i * LV + j] + V[j * LV + i]);
        V[i * LV + j] = s;
        V[j * LV + i] = s;
      }
    }
    if (store_P && gP && !param) {
      __syncthreads();
      for (int e = threadIdx.x; e < (int)nn; e += blockDim.x) {
        const int i = e / n;
        gP[nn * t + e] = V[i * LV + (e - i * n)];
      }
      for (int i = threadIdx.x; i < n; i += blockDim.x) gp[(long long)n * t + i] = vx[i];
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  // ---- the summary at the segment start ----------------------------------------------
  if (mode == MODE_POLICY) return;
  for (long long e = threadIdx.x; e < nn; e += blockDim.x) {
    const int i = (int)(e / n), j = (int)(e - (long long)i * n);
    summ[e] = static_cast<double>(V[i * LV + j]);
    if (param) {
      summ[nn + e] = static_cast<double>(Z[i * LV + j]);
      summ[2 * nn + e] = 0.5 * (static_cast<double>(Wn[i * LV + j]) + static_cast<double>(Wn[j * LV + i]));
    } else {
      summ[nn + e] = 0.0;
      summ[2 * nn + e] = 0.0;
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    summ[3 * nn + i] = static_cast<double>(vx[i]);
    summ[3 * nn + n + i] = param ? static_cast<double>(vz[i]) : 0.0;
  }
}


}  // namespace lqr
