// The FP32 rollout (steps A5/A6) as a device function of one CTA, shared by
// rollout_f32_kernel and the persistent batched kernel.
#pragma once
#include <cuda_runtime.h>

#include "cta_linalg.cuh"
#include "lqr_internal.cuh"
#include "tc_sm100.cuh"

namespace lqr {

// block-wide sum of one value per thread (red: one slot per warp, shared)
template <typename T>
__device__ __forceinline__ T roll_block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T s = T(0);
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) s += red[w];
  return s;  // valid in thread 0
}

// ---------------------------------------------------------------------------
// FP32 variant (x and u outputs present), 512 threads. The forward walk
// streams [K | A | B | Q | R | S | c | k | q | r]_t through a two-slot
// shared-memory ring and forms, besides x_{t+1} and u_t, the objective terms
// and the part of the multiplier recursion that does not involve lambda,
//     g_t = (Q_t + Q_t')/2 x_t + S_t'u_t + q_t      (stored in lambda_t),
// so that the backward walk lambda_t = A_t'lambda_{t+1} - g_t streams A_t only.
// Row products: four threads per row, 128-bit loads; transposed products:
// column partials over 512 / n4 row groups. With n and m multiples of 4 (and
// 16-byte aligned arrays) every region of a slot has its array's global
// layout, and one thread moves a stage with one bulk asynchronous copy per
// array (completion counted in bytes on the slot's mbarrier); otherwise every
// thread issues 16- or 4-byte cp.async copies.
// ---------------------------------------------------------------------------
constexpr int kRollBlock = 512;
constexpr long long kRollSpin = 1LL << 25;  // polls of a stage-data wait (32 ns apart) before LQR_ERR_TIMEOUT

struct FastRollSlot {
  int n4, m4;
  long long K, A, B, Q, R, S, c, k, q, r, elems;
};
__host__ __device__ inline FastRollSlot fast_roll_slot(int n, int m) {
  FastRollSlot L;
  L.n4 = (n + 3) & ~3;
  L.m4 = (m + 3) & ~3;
  const long long n4 = L.n4, m4 = L.m4;
  long long o = 0;
  L.K = o; o += m4 * n4;
  L.A = o; o += n4 * n4;
  L.B = o; o += n4 * m4;
  L.Q = o; o += n4 * n4;
  L.R = o; o += m4 * m4;
  L.S = o; o += m4 * n4;
  L.c = o; o += n4;
  L.k = o; o += m4;
  L.q = o; o += n4;
  L.r = o; o += m4;
  L.elems = o;
  return L;
}
// vectors: x[2] n4, u m4, qx n4, sx m4, ru m4, lam[2] n4, partQ and partS
// (kRollBlock each: (kRollBlock / n4) row groups x n4 for any n4 of the launch)
__host__ __device__ inline long long fast_roll_vec(int nmax, int mmax) {
  const long long n4 = (nmax + 3) & ~3, m4 = (mmax + 3) & ~3;
  return 2 * n4 + m4 + n4 + 2 * m4 + 2 * n4 + 2 * kRollBlock;
}

namespace {
__device__ __forceinline__ void roll_copy_rows(float* dst, int ldd, const float* src, int lds, int rows, int cols,
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
__device__ __forceinline__ bool ral16(const void* p) { return (reinterpret_cast<unsigned long long>(p) & 15) == 0; }
}  // namespace

// The rollout of one unit (segment) by the calling 512-thread CTA: the body of
// rollout_f32_kernel, also called per problem by the persistent batched kernel.
__device__ __forceinline__ void rollout_f32_unit(const ProbTable& tab, int unit, int want_lam, int nmax, int mmax) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_flag;
  __shared__ double s_red[kRollBlock / 32];
  __shared__ __align__(8) uint64_t s_rbar[2];
  const ProbDesc& pd = prob_of_unit(tab, unit);
  if (cta_should_exit(pd, &s_flag)) return;
  const int seg = unit - pd.unit0;
  const int n = pd.n, m = pd.m, T = pd.T, K = pd.nseg;
  const bool last = (seg == K - 1);
  const int t0 = seg_begin(T, K, seg), t1 = seg_begin(T, K, seg + 1);
  const long long nn = (long long)n * n, nm = (long long)n * m, mm = (long long)m * m;
  const WsLayout wl = ws_layout(n, K);
  const int tid = threadIdx.x;
  const FastRollSlot L = fast_roll_slot(n, m);
  const FastRollSlot Lx = fast_roll_slot(nmax, mmax);
  const long long stride = Lx.elems;
  const int n4 = L.n4, m4 = L.m4, n4x = Lx.n4, m4x = Lx.m4;
  const int G = kRollBlock / n4 > 0 ? kRollBlock / n4 : 1;  // row groups of the column partials
  float* ring = reinterpret_cast<float*>(smem);
  float* xb = ring + 2 * stride;  // 2 x n4x
  float* ub = xb + 2 * n4x;       // m4x
  float* qx = ub + m4x;           // n4x
  float* sx = qx + n4x;           // m4x
  float* ru = sx + m4x;           // m4x
  float* lb = ru + m4x;           // 2 x n4x
  float* pQ = lb + 2 * n4x;       // G x n4 (<= kRollBlock)
  float* pS = pQ + kRollBlock;     // G x n4

  const float* gA = static_cast<const float*>(pd.A);
  const float* gB = static_cast<const float*>(pd.B);
  const float* gc = static_cast<const float*>(pd.c);
  const float* gQ = static_cast<const float*>(pd.Q);
  const float* gR = static_cast<const float*>(pd.R);
  const float* gS = static_cast<const float*>(pd.S);
  const float* gq = static_cast<const float*>(pd.q);
  const float* gr = static_cast<const float*>(pd.r);
  const float* gK = static_cast<const float*>(pd.K);
  const float* gk = static_cast<const float*>(pd.k);
  float* ox = static_cast<float*>(pd.x);
  float* ou = static_cast<float*>(pd.u);
  float* olam = (want_lam && pd.lam) ? static_cast<float*>(pd.lam) : nullptr;
  const bool v16 = (n % 4 == 0) && (m % 4 == 0) && ral16(gA) && ral16(gB) && ral16(gQ) && ral16(gR) && ral16(gK) &&
                   (gS == nullptr || ral16(gS));

  // bulk copies: slot regions laid out like the arrays (n4 = n, m4 = m)
  const bool bulk = v16 && ral16(gc) && ral16(gq) && ral16(gk) && ral16(gr);
  // zero the ring and vectors once (padding stays zero)
  {
    const long long tot = 2 * stride + fast_roll_vec(nmax, mmax);
    float4* z4 = reinterpret_cast<float4*>(smem);
    for (long long i = tid; i < tot / 4; i += blockDim.x) z4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (bulk && tid == 0) {
      tc::mbar_init(&s_rbar[0], 1);
      tc::mbar_init(&s_rbar[1], 1);
      tc::mbar_fence_init();
    }
  }
  __syncthreads();
  uint32_t rph = 0u;  // bit s: the parity of slot s's next completion
  // waits for slot s (bulk) or for this thread's copies, then a barrier; false on
  // a timeout (the same answer in every thread)
  auto slot_ready = [&](int s) -> bool {
    bool ok = true;
    if (bulk) {
      ok = tc::mbar_wait(&s_rbar[s], (rph >> s) & 1u, kRollSpin);
      rph ^= 1u << s;
    } else {
      cp_async_wait<0>();
    }
    return __syncthreads_or(!ok) == 0;
  };
  auto fwd_issue = [&](int t) {
    if (bulk) {
      if (t < t1 && tid == 0) {
        const int s = (t - t0) & 1;
        float* d = ring + (long long)s * stride;
        uint64_t* bar = &s_rbar[s];
        const uint32_t bytes = (uint32_t)(4 * (2 * nm + 2 * nn + mm + (gS ? nm : 0) + 2 * n + 2 * m));
        tc::mbar_expect_tx(bar, bytes);
        tc::bulk_g2s(d + L.K, gK + nm * t, (uint32_t)(4 * nm), bar);
        tc::bulk_g2s(d + L.A, gA + nn * t, (uint32_t)(4 * nn), bar);
        tc::bulk_g2s(d + L.B, gB + nm * t, (uint32_t)(4 * nm), bar);
        tc::bulk_g2s(d + L.Q, gQ + nn * t, (uint32_t)(4 * nn), bar);
        tc::bulk_g2s(d + L.R, gR + mm * t, (uint32_t)(4 * mm), bar);
        if (gS) tc::bulk_g2s(d + L.S, gS + nm * t, (uint32_t)(4 * nm), bar);
        tc::bulk_g2s(d + L.c, gc + (long long)n * t, (uint32_t)(4 * n), bar);
        tc::bulk_g2s(d + L.k, gk + (long long)m * t, (uint32_t)(4 * m), bar);
        tc::bulk_g2s(d + L.q, gq + (long long)n * t, (uint32_t)(4 * n), bar);
        tc::bulk_g2s(d + L.r, gr + (long long)m * t, (uint32_t)(4 * m), bar);
      }
      return;
    }
    if (t < t1) {
      float* d = ring + (long long)((t - t0) & 1) * stride;
      roll_copy_rows(d + L.K, n4, gK + nm * t, n, m, n, v16);
      roll_copy_rows(d + L.A, n4, gA + nn * t, n, n, n, v16);
      roll_copy_rows(d + L.B, m4, gB + nm * t, m, n, m, v16);
      roll_copy_rows(d + L.Q, n4, gQ + nn * t, n, n, n, v16);
      roll_copy_rows(d + L.R, m4, gR + mm * t, m, m, m, v16);
      if (gS) roll_copy_rows(d + L.S, n4, gS + nm * t, n, m, n, v16);
      for (int i = tid; i < n; i += blockDim.x) {
        cp_async4(d + L.c + i, gc + (long long)n * t + i);
        cp_async4(d + L.q + i, gq + (long long)n * t + i);
      }
      for (int a = tid; a < m; a += blockDim.x) {
        cp_async4(d + L.k + a, gk + (long long)m * t + a);
        cp_async4(d + L.r + a, gr + (long long)m * t + a);
      }
    }
    cp_async_commit();
  };
  // four threads per row: rows [0, nrows) of a virtual row set, 128 rows per pass
  const int q4 = tid & 3;
  auto rows4 = [&](int nrows, auto rowinfo, auto epi) {
    for (int base = 0; base < nrows; base += kRollBlock / 4) {
      const int r = base + (tid >> 2);
      float acc = 0.0f;
      if (r < nrows) {
        const float* row;
        const float* vec;
        int len4;
        rowinfo(r, row, vec, len4);
        for (int c = q4; c < len4; c += 4) {
          const float4 a = *reinterpret_cast<const float4*>(row + 4 * c);
          const float4 b = *reinterpret_cast<const float4*>(vec + 4 * c);
          acc = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, acc))));
        }
      }
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if (q4 == 0 && r < nrows) epi(r, acc);
    }
  };
  // column partials part[g][j] = sum over rows i of group g of M[i][j] v[i] (M rows x n, ld n4)
  const int cg = tid / n4, cj = tid - (tid / n4) * n4;
  auto colpart = [&](const float* M, int rows, const float* v, float* part) {
    if (cg < G) {
      const int per = (rows + G - 1) / G, i0 = cg * per, i1 = min(rows, i0 + per);
      float acc = 0.0f;
      for (int i = i0; i < i1; ++i) acc = fmaf(M[(long long)i * n4 + cj], v[i], acc);
      part[cg * n4 + cj] = acc;
    }
  };

  fwd_issue(t0);
  {
    const double* zj = pd.ws + wl.z + (long long)seg * n;
    for (int i = tid; i < n; i += blockDim.x) xb[i] = static_cast<float>(zj[i]);
  }
  double cost = 0.0;
  bool timed_out = false;
  for (int t = t0; t < t1; ++t) {
    // slot t and x_t ready; the previous stage is finished
    if (!slot_ready((t - t0) & 1)) {
      timed_out = true;
      break;
    }
    fwd_issue(t + 1);
    const float* d = ring + (long long)((t - t0) & 1) * stride;
    const float* xc = xb + ((t - t0) & 1) * n4x;
    float* xn = xb + (((t - t0) + 1) & 1) * n4x;
    // (1) u = K x + k, A x, Q x, S x
    const int nr1 = m + n + n + (gS ? m : 0);
    rows4(nr1,
          [&](int r, const float*& row, const float*& vec, int& len4) {
            vec = xc;
            len4 = n4 / 4;
            if (r < m) row = d + L.K + (long long)r * n4;
            else if (r < m + n) row = d + L.A + (long long)(r - m) * n4;
            else if (r < m + 2 * n) row = d + L.Q + (long long)(r - m - n) * n4;
            else row = d + L.S + (long long)(r - m - 2 * n) * n4;
          },
          [&](int r, float v) {
            if (r < m) ub[r] = v + d[L.k + r];
            else if (r < m + n) xn[r - m] = v;
            else if (r < m + 2 * n) qx[r - m - n] = v;
            else sx[r - m - 2 * n] = v;
          });
    if (olam) colpart(d + L.Q, n, xc, pQ);
    __syncthreads();
    // (2) x_{t+1} += B u + c, R u, S'u partials, outputs
    rows4(n + m,
          [&](int r, const float*& row, const float*& vec, int& len4) {
            vec = ub;
            len4 = m4 / 4;
            row = (r < n) ? d + L.B + (long long)r * m4 : d + L.R + (long long)(r - n) * m4;
          },
          [&](int r, float v) {
            if (r < n) xn[r] += v + d[L.c + r];
            else ru[r - n] = v;
          });
    if (olam && gS) colpart(d + L.S, m, ub, pS);
    for (int i = tid; i < n; i += blockDim.x) ox[(long long)n * t + i] = xc[i];
    for (int a = tid; a < m; a += blockDim.x) ou[(long long)m * t + a] = ub[a];
    __syncthreads();
    // (3) objective terms and g_t
    for (int j = tid; j < n; j += blockDim.x) {
      cost += static_cast<double>(xc[j]) * (0.5 * static_cast<double>(qx[j]) + static_cast<double>(d[L.q + j]));
      if (olam) {
        float tq = 0.0f, ts = 0.0f;
        for (int g = 0; g < G; ++g) tq += pQ[g * n4 + j];
        if (gS)
          for (int g = 0; g < G; ++g) ts += pS[g * n4 + j];
        olam[(long long)n * t + j] = 0.5f * (qx[j] + tq) + ts + d[L.q + j];
      }
    }
    for (int a = tid; a < m; a += blockDim.x)
      cost += static_cast<double>(ub[a]) *
              (0.5 * static_cast<double>(ru[a]) + (gS ? static_cast<double>(sx[a]) : 0.0) + static_cast<double>(d[L.r + a]));
  }
  if (timed_out) {
    // a stage's copy did not arrive: report it, give the copy issued after it one
    // more bounded wait, stop
    if (tid == 0) {
      raise_status(pd.status, LQR_ERR_TIMEOUT, -1);
      for (int s = 0; s < 2; ++s) tc::mbar_wait(&s_rbar[s], (rph >> s) & 1u, kRollSpin);
    }
    return;
  }
  cp_async_wait<0>();
  __syncthreads();
  const float* xe = xb + ((t1 - t0) & 1) * n4x;  // x_{t1}
  float* lcur = lb;
  if (last) {
    // x_T, its objective term and lambda_T = -((Q_T + Q_T')/2 x_T + q_T)
    const float* QT = gQ + nn * T;
    const float* qT = gq + (long long)n * T;
    for (int i = tid; i < n; i += blockDim.x) ox[(long long)n * T + i] = xe[i];
    for (int base = 0; base < n; base += kRollBlock / 4) {  // Q_T x_T rows (global, four threads per row)
      const int i = base + (tid >> 2);
      float acc = 0.0f;
      if (i < n)
        for (int k = q4; k < n; k += 4) acc = fmaf(QT[(long long)i * n + k], xe[k], acc);
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if (q4 == 0 && i < n) qx[i] = acc;
    }
    if (cg < G) {  // Q_T' x_T partials
      const int per = (n + G - 1) / G, i0 = cg * per, i1 = min(n, i0 + per);
      float acc = 0.0f;
      if (cj < n)
        for (int i = i0; i < i1; ++i) acc = fmaf(QT[(long long)i * n + cj], xe[i], acc);
      pQ[cg * n4 + cj] = acc;
    }
    __syncthreads();
    for (int j = tid; j < n; j += blockDim.x) {
      float tq = 0.0f;
      for (int g = 0; g < G; ++g) tq += pQ[g * n4 + j];
      const float l = -(0.5f * (qx[j] + tq) + qT[j]);
      lcur[j] = l;
      if (olam) olam[(long long)n * T + j] = l;
      cost += static_cast<double>(xe[j]) * (0.5 * static_cast<double>(qx[j]) + static_cast<double>(qT[j]));
    }
  } else if (olam) {
    const double* Pn = pd.ws + wl.Pi + (long long)(seg + 1) * nn;
    const double* pn = pd.ws + wl.pi + (long long)(seg + 1) * n;
    const double* zn = pd.ws + wl.z + (long long)(seg + 1) * n;
    for (int base = 0; base < n; base += kRollBlock / 4) {
      const int i = base + (tid >> 2);
      double acc = 0.0;
      if (i < n)
        for (int k = q4; k < n; k += 4) acc = fma(Pn[(long long)i * n + k], zn[k], acc);
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if (q4 == 0 && i < n) lcur[i] = static_cast<float>(-(acc + pn[i]));
    }
  }
  {
    const double tot = roll_block_sum(cost, s_red);
    if (tid == 0) pd.ws[wl.costp + seg] = tot;
  }
  if (!olam) {
    if (bulk) {
      __syncthreads();
      if (tid == 0) {
        tc::mbar_inval(&s_rbar[0]);
        tc::mbar_inval(&s_rbar[1]);
      }
    }
    return;
  }
  __syncthreads();
  // ---- backward: lambda_t = A_t'lambda_{t+1} - g_t, A_t streamed ----------------
  auto bwd_issue = [&](int t) {
    const int s = (t1 - 1 - t) & 1;
    if (bulk) {
      if (t >= t0 && tid == 0) {
        tc::mbar_expect_tx(&s_rbar[s], (uint32_t)(4 * nn));
        tc::bulk_g2s(ring + (long long)s * stride + L.A, gA + nn * t, (uint32_t)(4 * nn), &s_rbar[s]);
      }
      return;
    }
    if (t >= t0) roll_copy_rows(ring + (long long)s * stride + L.A, n4, gA + nn * t, n, n, n, v16);
    cp_async_commit();
  };
  bwd_issue(t1 - 1);
  for (int t = t1 - 1; t >= t0; --t) {
    if (!slot_ready((t1 - 1 - t) & 1)) {
      if (tid == 0) {
        raise_status(pd.status, LQR_ERR_TIMEOUT, -1);
        for (int s = 0; s < 2; ++s) tc::mbar_wait(&s_rbar[s], (rph >> s) & 1u, kRollSpin);
      }
      return;
    }
    bwd_issue(t - 1);
    const float* Ad = ring + (long long)((t1 - 1 - t) & 1) * stride + L.A;
    float* lnext = lb + (((t1 - 1 - t) + 1) & 1) * n4x;
    colpart(Ad, n, lcur, pQ);
    __syncthreads();
    for (int j = tid; j < n; j += blockDim.x) {
      float s2 = 0.0f;
      for (int g = 0; g < G; ++g) s2 += pQ[g * n4 + j];
      const float l = s2 - olam[(long long)n * t + j];
      lnext[j] = l;
      olam[(long long)n * t + j] = l;
    }
    lcur = lnext;
  }
  cp_async_wait<0>();
  if (bulk) {
    __syncthreads();
    if (tid == 0) {
      tc::mbar_inval(&s_rbar[0]);
      tc::mbar_inval(&s_rbar[1]);
    }
  }
}

}  // namespace lqr
