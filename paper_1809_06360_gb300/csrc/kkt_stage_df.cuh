// The per-stage block of the KKT residual of Eq. 3 for FP64 data in
// double-FP32 arithmetic, for the refinement passes.
//
// On this GPU every FP64 warp instruction holds its sub-partition's FP64 pipe
// for 64 cycles, so the FP64 residual pass (two FP64 multiply-adds per matrix
// element) runs at a fraction of the rate HBM delivers the elements at. Here
// every FP64 element v is split into an FP32 pair v = h + l (h: v with its
// significand cut to 24 bits, by integer operations on the bit pattern; l: the
// exact rest rounded to FP32), every FP64 vector entry likewise, and each
// product is accumulated as an unevaluated FP32 pair:
//   p = fl(a_h b_h), e = a_h b_h - p            (exact, one FMA)
//   (s_h, t) = TwoSum(s_h, p)                   (exact, Knuth's six additions)
//   s_l += t + e + a_h b_l + a_l b_h            (the small terms in FP32)
// i.e. the compensated dot product of Ogita, Rump and Oishi (Dot2) applied to
// the pair representations. The split errs by at most 2^-47 |v|, the
// accumulation by a few units of 2^-48 of the sum of |terms|: about 47 bits
// where FP64 keeps 53. The mixed-precision refinement uses it for its first
// pass only, whose residual (of the FP32 solve, some 2^-24 of the same scale)
// it resolves to ~1e-7, far finer than the FP32 correction it drives; every
// operation runs on the FP32 and integer pipes. All additions and products use
// the _rn intrinsics so that no contraction into an FMA changes the error-free
// steps.
//
// The layout of the work is that of kkt_stage (kkt_stage.cuh): rows of a
// matrix to warps, columns to lanes, each element used for its row and its
// column product; the |KKT| row sums are not formed here (the mixed-precision
// refinement takes |KKT|_inf from the FP32 copy of the data once per solve).
#pragma once

#include <cuda_runtime.h>

#include "kkt_stage.cuh"

namespace lqr {

struct DF {
  float h, l;
};

// v = h + l (+ at most 2^-47 |v|) for 2^-74 <= |v| < 2^127; smaller magnitudes
// give 0 (an absolute error below 2^-74), larger ones a signed infinity (the
// pass then reports a non-finite residual). Integer and FP32 operations only: a
// conversion instruction would occupy the FP64 pipe for every element.
__device__ __forceinline__ DF df_split(double v) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  const int e = static_cast<int>((b >> 52) & 0x7FF);  // biased FP64 exponent
  const unsigned int sign = static_cast<unsigned int>(b >> 32) & 0x80000000u;
  const unsigned int hm = static_cast<unsigned int>((b >> 29) & 0x7FFFFFull);  // top 23 stored bits
  const unsigned int lm = static_cast<unsigned int>(b & 0x1FFFFFFFull);       // the other 29 bits
  const bool in = (e >= 949) & (e <= 1149);
  const int ec = in ? e : 949;  // keeps the exponent fields below in range
  const float hi = __uint_as_float(sign | (static_cast<unsigned int>(ec - 1023 + 127) << 23) | hm);
  const float scale = __uint_as_float(static_cast<unsigned int>(ec - 1075 + 127) << 23);  // 2^(e - 1075)
  const float lf = __fmul_rn(__uint2float_rn(lm), scale);
  const float big = __uint_as_float(sign | 0x7F800000u);
  DF r;
  r.h = in ? hi : (e > 1149 ? big : 0.0f);
  r.l = in ? (sign ? -lf : lf) : 0.0f;
  return r;
}

__device__ __forceinline__ DF df_zero() { return DF{0.0f, 0.0f}; }

// acc += a b
__device__ __forceinline__ void df_mac(DF& acc, const DF& a, const DF& b) {
  const float p = __fmul_rn(a.h, b.h);
  const float e = __fmaf_rn(a.h, b.h, -p);
  const float s = __fadd_rn(acc.h, p);
  const float z = __fsub_rn(s, acc.h);
  const float t = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, z)), __fsub_rn(p, z));
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(t, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e))));
}

// a += b
__device__ __forceinline__ void df_add(DF& a, const DF& b) {
  const float s = __fadd_rn(a.h, b.h);
  const float z = __fsub_rn(s, a.h);
  const float t = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, z)), __fsub_rn(b.h, z));
  a.h = s;
  a.l = __fadd_rn(a.l, __fadd_rn(b.l, t));
}

__device__ __forceinline__ DF df_scale(const DF& a, float s) {  // s a power of two
  return DF{__fmul_rn(a.h, s), __fmul_rn(a.l, s)};
}

__device__ __forceinline__ double df_value(const DF& a) {
  return static_cast<double>(a.h) + static_cast<double>(a.l);
}

__device__ __forceinline__ DF df_shfl_xor(const DF& a, int o) {
  return DF{__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o)};
}

// kkt_rows_reduce for pairs: RB rows summed over the 32 lanes at once
template <int RB>
__device__ __forceinline__ DF df_rows_reduce(DF (&d)[RB], int lane) {
  int o = 16;
#pragma unroll
  for (int cnt = RB; cnt > 1; cnt >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < cnt / 2; ++j) {
      const DF send = upper ? d[j] : d[j + cnt / 2];
      DF keep = upper ? d[j + cnt / 2] : d[j];
      df_add(keep, df_shfl_xor(send, o));
      d[j] = keep;
    }
    o >>= 1;
  }
  DF v = d[0];
#pragma unroll
  for (; o > 0; o >>= 1) df_add(v, df_shfl_xor(v, o));
  return v;
}

template <int NC>
struct DfCols {
  DF v[NC];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int c = 0; c < NC; ++c) v[c] = df_zero();
  }
};

// One pass over the row-major R x C FP64 matrix M (kkt_mat_pass in pairs):
//   rowout[i] (+)= rscale sum_k M[i,k] vc[k]     (first: assign, else add)
//   col.v[c]  +=  sum_i M[i,k] wr[i]
template <int NCP, int NC>
__device__ __forceinline__ void df_mat_pass(const double* __restrict__ M, int R, int C, const DF* vc, const DF* wr,
                                            float rscale, DF* rowout, bool first, DfCols<NC>& col, int warp,
                                            int lane) {
  static_assert(NCP <= NC, "pass columns beyond the register plan");
  constexpr int RB = NCP >= 4 ? 2 : kKktRB;  // rows per batch: the pairs double the registers
  constexpr int kShift = 5 - KktLog2<RB>::value;
  DF vcl[NCP];
#pragma unroll
  for (int c = 0; c < NCP; ++c) {
    const int k = lane + 32 * c;
    vcl[c] = k < C ? vc[k] : df_zero();
  }
  for (int i0 = warp; i0 < R; i0 += kKktWarps * RB) {
    double v[RB][NCP];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int i = i0 + r * kKktWarps;
#pragma unroll
      for (int c = 0; c < NCP; ++c) {
        const int k = lane + 32 * c;
        v[r][c] = (i < R && k < C) ? __ldg(M + (size_t)i * C + k) : 0.0;
      }
    }
    DF d[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int i = i0 + r * kKktWarps;
      const DF w = i < R ? wr[i] : df_zero();
      d[r] = df_zero();
#pragma unroll
      for (int c = 0; c < NCP; ++c) {
        const DF a = df_split(v[r][c]);
        df_mac(d[r], a, vcl[c]);
        df_mac(col.v[c], a, w);
      }
    }
    const DF dr = df_scale(df_rows_reduce<RB>(d, lane), rscale);
    const int i = i0 + (lane >> kShift) * kKktWarps;
    if ((lane & ((1 << kShift) - 1)) == 0 && i < R) {
      if (first) {
        rowout[i] = dr;
      } else {
        DF acc = rowout[i];
        df_add(acc, dr);
        rowout[i] = acc;
      }
    }
  }
}

template <int NC>
__device__ __forceinline__ void df_pass(const double* __restrict__ M, int R, int C, const DF* vc, const DF* wr,
                                        float rscale, DF* rowout, bool first, DfCols<NC>& col, int warp, int lane) {
  if (NC >= 4 && C > 64)
    df_mat_pass<(NC >= 4 ? 4 : 1), NC>(M, R, C, vc, wr, rscale, rowout, first, col, warp, lane);
  else if (NC >= 2 && C > 32)
    df_mat_pass<(NC >= 2 ? 2 : 1), NC>(M, R, C, vc, wr, rscale, rowout, first, col, warp, lane);
  else
    df_mat_pass<1, NC>(M, R, C, vc, wr, rscale, rowout, first, col, warp, lane);
}

// dynamic shared memory of kkt_stage_df, in doubles (a pair takes one double's room)
__host__ __device__ inline size_t kkt_stage_df_smem_doubles(int n, int m) {
  return (size_t)(7 + kKktWarps) * n + (size_t)(4 + kKktWarps) * m;
}

// Stage t < T of the residual (kkt_stage without the |KKT| row sums), FP64 data,
// products in pairs, the assembly of rx, ru, rd in FP64. Called by all kKktBlock
// threads of a CTA (it synchronises the CTA). Returns this thread's share of
// the stage objective.
template <int NC>
__device__ double kkt_stage_df(const KktData<double>& g, int t, double* sm, KktMax& mx, const KktOut& out) {
  const int n = g.n, m = g.m;
  const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm = (size_t)m * m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* xt = sm;                          // x_t (FP64)
  double* lt = xt + n;                      // lambda_t
  double* ut = lt + n;                      // u_t (m)
  DF* xd = reinterpret_cast<DF*>(ut + m);   // x_t
  DF* xhd = xd + n;                         // x_t / 2
  DF* lnd = xhd + n;                        // -lambda_{t+1}
  DF* ud = lnd + n;                         // u_t (m)
  DF* uhd = ud + m;                         // u_t / 2 (m)
  DF* rowx = uhd + m;                       // (Q x)_i / 2
  DF* rowd = rowx + n;                      // (A x + B u)_i
  DF* rowu = rowd + n;                      // (S x + R u / 2)_a (m)
  DF* px = rowu + m;                        // [nw][n] column partials of rx
  DF* pu = px + kKktWarps * n;              // [nw][m] column partials of ru
  for (int i = threadIdx.x; i < n; i += kKktBlock) {
    const double x = g.x[(size_t)n * t + i];
    xt[i] = x;
    lt[i] = g.lam[(size_t)n * t + i];
    xd[i] = df_split(x);
    xhd[i] = df_scale(xd[i], 0.5f);
    lnd[i] = df_split(-g.lam[(size_t)n * (t + 1) + i]);
  }
  for (int a = threadIdx.x; a < m; a += kKktBlock) {
    const double u = g.u[(size_t)m * t + a];
    ut[a] = u;
    ud[a] = df_split(u);
    uhd[a] = df_scale(ud[a], 0.5f);
  }
  __syncthreads();
  DfCols<NC> cxs, cus;
  cxs.zero();
  cus.zero();
  // A_t: rows A x, columns -A'lambda_{t+1}
  df_pass<NC>(g.A + nn * t, n, n, xd, lnd, 1.0f, rowd, true, cxs, warp, lane);
  // B_t: rows B u, columns -B'lambda_{t+1}
  df_pass<NC>(g.B + nm * t, n, m, ud, lnd, 1.0f, rowd, false, cus, warp, lane);
  // Q_t: rows Q x / 2, columns Q'x / 2
  df_pass<NC>(g.Q + nn * t, n, n, xd, xhd, 0.5f, rowx, true, cxs, warp, lane);
  if (g.S) {  // S_t: rows S x, columns S'u
    df_pass<NC>(g.S + nm * t, m, n, xd, ud, 1.0f, rowu, true, cxs, warp, lane);
  } else {
    if (lane == 0)  // row a belongs to warp a % nw in the R pass below too
      for (int a = warp; a < m; a += kKktWarps) rowu[a] = df_zero();
    __syncwarp();
  }
  // R_t: rows R u / 2, columns R'u / 2
  df_pass<NC>(g.R + mm * t, m, m, ud, uhd, 0.5f, rowu, false, cus, warp, lane);
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int k = lane + 32 * c;
    if (k < n) px[warp * n + k] = cxs.v[c];
    if (k < m) pu[warp * m + k] = cus.v[c];
  }
  __syncthreads();
  double cost = 0.0;
  for (int i = threadIdx.x; i < n; i += kKktBlock) {
    DF sxd = px[i];
#pragma unroll
    for (int w = 1; w < kKktWarps; ++w) df_add(sxd, px[w * n + i]);
    const double sx = df_value(sxd);
    const double qx = df_value(rowx[i]);
    const double x = xt[i];
    const double q = g.q[(size_t)n * t + i];
    const double l = lt[i];
    const double c = g.c[(size_t)n * t + i];
    const double rx = sx + qx + q + l;
    const double rd = g.x[(size_t)n * (t + 1) + i] - df_value(rowd[i]) - c;
    cost += x * (qx + q);
    mx.r = fmax(mx.r, fmax(fabs(rx), fabs(rd)));
    mx.w = fmax(mx.w, fmax(fabs(x), fabs(l)));
    mx.b = fmax(mx.b, fmax(fabs(q), fabs(c)));
    if (out.q) {
      out.put(out.q, (size_t)n * t + i, -rx);
      out.put(out.c, (size_t)n * t + i, rd);
    }
  }
  for (int a = threadIdx.x; a < m; a += kKktBlock) {
    DF sud = pu[a];
#pragma unroll
    for (int w = 1; w < kKktWarps; ++w) df_add(sud, pu[w * m + a]);
    const double ru_row = df_value(rowu[a]);
    const double r = g.r[(size_t)m * t + a];
    const double ru = df_value(sud) + ru_row + r;
    cost += ut[a] * (ru_row + r);
    mx.r = fmax(mx.r, fabs(ru));
    mx.w = fmax(mx.w, fabs(ut[a]));
    mx.b = fmax(mx.b, fabs(r));
    if (out.q) out.put(out.r, (size_t)m * t + a, -ru);
  }
  __syncthreads();
  return cost;
}

}  // namespace lqr
