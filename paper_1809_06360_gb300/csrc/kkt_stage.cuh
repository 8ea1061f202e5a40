// The per-stage block of the FP64 residual of the KKT system of Eq. 3, shared
// by the refinement residual pass and the no-allocation residual entry point
// so that both produce the same numbers for the same solution.
//
// For stage t < T (blocks of Q and R read symmetrised):
//   rx_t = Q x_t + S'u_t + q_t + lambda_t - A_t'lambda_{t+1}
//   ru_t = S x_t + R u_t + r_t - B_t'lambda_{t+1}
//   rd_t = x_{t+1} - A_t x_t - B_t u_t - c_t
// and the stage's share of the objective of Eq. 1.
//
// The FP64 products dominate (about 2(2n^2 + 2nm + m^2) multiply-adds per
// stage, on the FP64 pipe), so every matrix element is read once and used
// twice: for its row product and for its column product. Rows go to warps
// (row i to warp i % nw in every pass, so each row accumulator in shared
// memory has one writer), columns to lanes (k = lane + 32 c, c < NCP, the
// narrowest plan that covers the matrix's columns), and a batch of kKktRB rows
// is loaded before it is used; the row products of a batch are reduced over the
// lanes together (kkt_rows_reduce). Column products stay in registers until the
// end of the stage and are then summed over the warps through shared memory.
#pragma once

#include <cuda_runtime.h>

#include "lqr_internal.cuh"

namespace lqr {

constexpr int kKktBlock = 256;  // threads per CTA of every kernel calling kkt_stage
constexpr int kKktWarps = kKktBlock / 32;
constexpr int kKktMaxDim = 128;  // n, m <= 32 * 4

__device__ __forceinline__ double kkt_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// register columns per lane for max(n, m); 0 = beyond kKktMaxDim
__host__ __device__ inline int kkt_stage_cols(int n, int m) {
  const int d = n > m ? n : m;
  return d <= 32 ? 1 : (d <= 64 ? 2 : (d <= kKktMaxDim ? 4 : 0));
}

// dynamic shared memory of kkt_stage, in doubles (without the stash)
__host__ __device__ inline size_t kkt_stage_smem_doubles(int n, int m) {
  return (size_t)(7 + 2 * kKktWarps) * n + (size_t)(5 + 2 * kKktWarps) * m;
}

// the optional stash of the |KKT| pass: one padded copy of Q_t, then of R_t
__host__ __device__ inline size_t kkt_stash_doubles(int n, int m) {
  const size_t d = (size_t)(n > m ? n : m);
  return d * (d + 1);
}

template <typename TS>
struct KktData {
  const TS *x, *u, *lam, *A, *B, *c, *Q, *R, *S, *q, *r;
  int n, m;
};

// running maxima of |r|, |KKT| row sums, |w| and |b| (per thread)
struct KktMax {
  double r = 0.0, k = 0.0, w = 0.0, b = 0.0;
};

template <int NC>
struct KktCols {
  double v[NC];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int c = 0; c < NC; ++c) v[c] = 0.0;
  }
};

// Sums d[r] over the 32 lanes for RB rows at once (RB a power of two <= 32):
// log2(RB) exchange steps in which each lane keeps half of the remaining rows
// and adds its partner's half, then a plain butterfly over the low lane bits.
// Every lane returns the full sum of row lane >> (5 - log2 RB), about one add
// per row and lane instead of five.
template <int RB>
__device__ __forceinline__ double kkt_rows_reduce(double (&d)[RB], int lane) {
  int o = 16;
#pragma unroll
  for (int cnt = RB; cnt > 1; cnt >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < cnt / 2; ++j) {
      const double send = upper ? d[j] : d[j + cnt / 2];
      const double keep = upper ? d[j + cnt / 2] : d[j];
      d[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
    o >>= 1;
  }
  double v = d[0];
#pragma unroll
  for (; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int RB>
struct KktLog2 {
  static constexpr int value = RB <= 1 ? 0 : 1 + KktLog2<RB / 2>::value;
};
template <>
struct KktLog2<1> {
  static constexpr int value = 0;
};

// One pass over the row-major R x C matrix M (NCP = ceil(C / 32) register
// columns per lane, NCP <= NC, so that no lane of a narrow matrix works on
// padding):
//   rowout[i] (+)= rscale sum_k M[i,k] vc[k]     (first: assign, else add)
//   col.v[c]  +=  sum_i M[i,k] wr[i]             (wr pre-scaled by the caller)
//   rowabs[i] (+)= sum_k |M[i,k]|,  colabs.v[c] += sum_i |M[i,k]|   (KN only)
//   stash[i (C + 1) + k] = M[i,k]                                   (stash given)
// Batches of kKktRB rows (row i0 + r nw, r < kKktRB) are loaded, then reduced
// together.
constexpr int kKktRB = 4;

template <int NCP, int NC, bool KN, typename TS>
__device__ __forceinline__ void kkt_mat_pass(const TS* __restrict__ M, int R, int C, const double* vc,
                                             const double* wr, double rscale, double* rowout, bool first,
                                             KktCols<NC>& col, double* rowabs, KktCols<NC>& colabs, int warp,
                                             int lane, double* stash) {
  static_assert(NCP <= NC, "pass columns beyond the register plan");
  constexpr int RB = kKktRB;
  constexpr int kShift = 5 - KktLog2<RB>::value;  // lanes per row after the reduction: 1 << kShift
  double vcl[NCP];
#pragma unroll
  for (int c = 0; c < NCP; ++c) {
    const int k = lane + 32 * c;
    vcl[c] = k < C ? vc[k] : 0.0;
  }
  for (int i0 = warp; i0 < R; i0 += kKktWarps * RB) {
    double v[RB][NCP];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int i = i0 + r * kKktWarps;
#pragma unroll
      for (int c = 0; c < NCP; ++c) {
        const int k = lane + 32 * c;
        v[r][c] = (i < R && k < C) ? (double)__ldg(M + (size_t)i * C + k) : 0.0;
      }
    }
    double d[RB], a[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int i = i0 + r * kKktWarps;
      const double w = i < R ? wr[i] : 0.0;
      d[r] = 0.0;
      a[r] = 0.0;
#pragma unroll
      for (int c = 0; c < NCP; ++c) {
        if (stash && i < R && lane + 32 * c < C) stash[(size_t)i * (C + 1) + lane + 32 * c] = v[r][c];
        d[r] = fma(v[r][c], vcl[c], d[r]);
        col.v[c] = fma(v[r][c], w, col.v[c]);
        if (KN) {
          a[r] += fabs(v[r][c]);
          colabs.v[c] += fabs(v[r][c]);
        }
      }
    }
    const double dr = rscale * kkt_rows_reduce<RB>(d, lane);
    double ar = 0.0;
    if (KN) ar = kkt_rows_reduce<RB>(a, lane);
    const int i = i0 + (lane >> kShift) * kKktWarps;
    if ((lane & ((1 << kShift) - 1)) == 0 && i < R) {
      rowout[i] = first ? dr : rowout[i] + dr;
      if (KN) rowabs[i] = first ? ar : rowabs[i] + ar;
    }
  }
}

// kkt_mat_pass with the narrowest column plan that covers C
template <int NC, bool KN, typename TS>
__device__ __forceinline__ void kkt_pass(const TS* __restrict__ M, int R, int C, const double* vc, const double* wr,
                                         double rscale, double* rowout, bool first, KktCols<NC>& col,
                                         double* rowabs, KktCols<NC>& colabs, int warp, int lane,
                                         double* stash = nullptr) {
  if (NC >= 4 && C > 64)
    kkt_mat_pass<(NC >= 4 ? 4 : 1), NC, KN>(M, R, C, vc, wr, rscale, rowout, first, col, rowabs, colabs, warp, lane,
                                            stash);
  else if (NC >= 2 && C > 32)
    kkt_mat_pass<(NC >= 2 ? 2 : 1), NC, KN>(M, R, C, vc, wr, rscale, rowout, first, col, rowabs, colabs, warp, lane,
                                            stash);
  else
    kkt_mat_pass<1, NC, KN>(M, R, C, vc, wr, rscale, rowout, first, col, rowabs, colabs, warp, lane, stash);
}

// Row sums of |(M + M')/2| for a square d x d matrix with leading dimension
// ld (KN only): from the matrix itself (ld = d) or from its stash in shared
// memory (ld = d + 1, the padding keeps the column reads conflict-free); the
// same values in the same order either way.
template <typename TM>
__device__ __forceinline__ void kkt_sym_abs_rows(const TM* M, int d, int ld, double* out, int warp, int lane) {
  for (int i = warp; i < d; i += kKktWarps) {
    double a = 0.0;
    for (int k = lane; k < d; k += 32)
      a += fabs(0.5 * ((double)M[(size_t)i * ld + k] + (double)M[(size_t)k * ld + i]));
    a = kkt_warp_sum(a);
    if (lane == 0) out[i] = a;
  }
}

// Stage t < T, called by all kKktBlock threads of a CTA (it synchronises the
// CTA). Folds |rx|, |ru|, |rd|, the |KKT| row sums (KN), |w| and |b| into mx;
// writes -rx, -ru, rd to out when out.q is given; returns this thread's
// share of the stage objective x'(Qx/2 + q) + u'(Sx + Ru/2 + r). stash (KN,
// optional, kkt_stash_doubles): shared memory for the symmetric row sums.
template <int NC, bool KN, typename TS>
__device__ double kkt_stage(const KktData<TS>& g, int t, double* sm, KktMax& mx, const KktOut& out,
                            double* stash = nullptr) {
  const int n = g.n, m = g.m;
  const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm = (size_t)m * m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* xt = sm;                  // x_t
  double* ln = xt + n;              // -lambda_{t+1}
  double* ut = ln + n;              // u_t
  double* rowx = ut + m;            // (Q x)_i / 2
  double* rowd = rowx + n;          // (A x + B u)_i
  double* rowu = rowd + n;          // (S x + R u / 2)_a
  double* kx = rowu + m;            // KN: |Q_sym| row sums
  double* kd = kx + n;              // KN: |A| + |B| row sums
  double* ku = kd + n;              // KN: |S| row sums
  double* kr = ku + m;              // KN: |R_sym| row sums
  double* px = kr + m;              // [nw][n] column partials of rx
  double* pu = px + kKktWarps * n;  // [nw][m] column partials of ru
  double* pxa = pu + kKktWarps * m; // KN: [nw][n] column |.| partials of rx rows
  double* pua = pxa + kKktWarps * n;// KN: [nw][m] column |.| partials of ru rows
  double* xh = pua + kKktWarps * m; // x_t / 2
  double* uh = xh + n;              // u_t / 2
  for (int i = threadIdx.x; i < n; i += kKktBlock) {
    xt[i] = (double)g.x[(size_t)n * t + i];
    xh[i] = 0.5 * xt[i];
    ln[i] = -(double)g.lam[(size_t)n * (t + 1) + i];
  }
  for (int a = threadIdx.x; a < m; a += kKktBlock) {
    ut[a] = (double)g.u[(size_t)m * t + a];
    uh[a] = 0.5 * ut[a];
  }
  __syncthreads();
  KktCols<NC> cxs, cus, cxa, cua;
  cxs.zero(); cus.zero(); cxa.zero(); cua.zero();
  // A_t: rows A x, columns -A'lambda_{t+1}
  kkt_pass<NC, KN>(g.A + nn * t, n, n, xt, ln, 1.0, rowd, true, cxs, kd, cxa, warp, lane);
  // B_t: rows B u, columns -B'lambda_{t+1}
  kkt_pass<NC, KN>(g.B + nm * t, n, m, ut, ln, 1.0, rowd, false, cus, kd, cua, warp, lane);
  // Q_t: rows Q x / 2, columns Q'x / 2
  kkt_pass<NC, false>(g.Q + nn * t, n, n, xt, xh, 0.5, rowx, true, cxs, nullptr, cxa, warp, lane,
                          KN ? stash : nullptr);
  if (KN) {
    if (stash) {
      __syncthreads();
      kkt_sym_abs_rows(stash, n, n + 1, kx, warp, lane);
      __syncthreads();  // the R pass below reuses the stash
    } else {
      kkt_sym_abs_rows(g.Q + nn * t, n, n, kx, warp, lane);
    }
  }
  if (g.S) {  // S_t: rows S x, columns S'u
    kkt_pass<NC, KN>(g.S + nm * t, m, n, xt, ut, 1.0, rowu, true, cxs, ku, cxa, warp, lane);
  } else if (lane == 0) {  // the same writer as the R pass below
    for (int a = warp; a < m; a += kKktWarps) {
      rowu[a] = 0.0;
      if (KN) ku[a] = 0.0;
    }
  }
  // R_t: rows R u / 2, columns R'u / 2
  kkt_pass<NC, false>(g.R + mm * t, m, m, ut, uh, 0.5, rowu, false, cus, nullptr, cua, warp, lane,
                          KN ? stash : nullptr);
  if (KN) {
    if (stash) {
      __syncthreads();
      kkt_sym_abs_rows(stash, m, m + 1, kr, warp, lane);
    } else {
      kkt_sym_abs_rows(g.R + mm * t, m, m, kr, warp, lane);
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int k = lane + 32 * c;
    if (k < n) {
      px[warp * n + k] = cxs.v[c];
      if (KN) pxa[warp * n + k] = cxa.v[c];
    }
    if (k < m) {
      pu[warp * m + k] = cus.v[c];
      if (KN) pua[warp * m + k] = cua.v[c];
    }
  }
  __syncthreads();
  double cost = 0.0;
  for (int i = threadIdx.x; i < n; i += kKktBlock) {
    double sx = 0.0, sxa = 0.0;
#pragma unroll
    for (int w = 0; w < kKktWarps; ++w) {
      sx += px[w * n + i];
      if (KN) sxa += pxa[w * n + i];
    }
    const double qx = rowx[i];
    const double x = xt[i];
    const double q = (double)g.q[(size_t)n * t + i];
    const double lt = (double)g.lam[(size_t)n * t + i];
    const double c = (double)g.c[(size_t)n * t + i];
    const double rx = sx + qx + q + lt;
    const double rd = (double)g.x[(size_t)n * (t + 1) + i] - rowd[i] - c;
    cost += x * (qx + q);
    mx.r = fmax(mx.r, fmax(fabs(rx), fabs(rd)));
    mx.w = fmax(mx.w, fmax(fabs(x), fabs(lt)));
    mx.b = fmax(mx.b, fmax(fabs(q), fabs(c)));
    if (KN) mx.k = fmax(mx.k, fmax(kx[i] + sxa + 1.0, 1.0 + kd[i]));
    if (out.q) {
      out.put(out.q, (size_t)n * t + i, -rx);
      out.put(out.c, (size_t)n * t + i, rd);
    }
  }
  for (int a = threadIdx.x; a < m; a += kKktBlock) {
    double su = 0.0, sua = 0.0;
#pragma unroll
    for (int w = 0; w < kKktWarps; ++w) {
      su += pu[w * m + a];
      if (KN) sua += pua[w * m + a];
    }
    const double r = (double)g.r[(size_t)m * t + a];
    const double ru = su + rowu[a] + r;
    cost += ut[a] * (rowu[a] + r);
    mx.r = fmax(mx.r, fabs(ru));
    mx.w = fmax(mx.w, fabs(ut[a]));
    mx.b = fmax(mx.b, fabs(r));
    if (KN) mx.k = fmax(mx.k, ku[a] + kr[a] + sua);
    if (out.q) out.put(out.r, (size_t)m * t + a, -ru);
  }
  __syncthreads();
  return cost;
}

}  // namespace lqr
