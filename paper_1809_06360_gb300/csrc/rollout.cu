// Steps A5/A6: per-segment forward reconstruction from the link state
// (Section II-A: with x_link known the sub-problem solutions are evaluated),
//     x_{b_j} = z_j,  u_t = K_t x_t + k_t,  x_{t+1} = A_t x_t + B_t u_t + c_t,
// the objective of Eq. 1 along the trajectory, and the multipliers of Eq. 3
// by the backward adjoint recursion inside the segment,
//     lambda_{b_{j+1}} = -(Pi_{j+1} z_{j+1} + pi_{j+1})   (lambda_T = -(Q_T x_T + q_T)),
//     lambda_t = A_t'lambda_{t+1} - Q_t x_t - S_t'u_t - q_t.
// One CTA per segment; matrix-vector products read the stage data straight
// from global memory (warp per row, or thread per column for transposes, so
// every global read is coalesced).
#include <cuda_runtime.h>

#include "cta_linalg.cuh"
#include "lqr_internal.cuh"

namespace lqr {

namespace {

// y_i = sum_k M[i][k] v[k] for i < rows: one warp per row, lanes stride k.
template <typename TS, typename Tacc, typename Out>
__device__ __forceinline__ void warp_rows(int rows, int cols, const TS* M, const Tacc* v, Out out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < rows; i += nw) {
    Tacc s = Tacc(0);
    for (int k = lane; k < cols; k += 32) s = fma(static_cast<Tacc>(M[(size_t)i * cols + k]), v[k], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out(i, s);
  }
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
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

}  // namespace

template <typename TS>
__global__ void __launch_bounds__(kBlock) rollout_kernel(ProbTable tab, int want_lam) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_flag;
  __shared__ double s_red[kBlock / 32];
  const int unit = blockIdx.x;
  const ProbDesc& pd = prob_of_unit(tab, unit);
  if (cta_should_exit(pd, &s_flag)) return;
  const int seg = unit - pd.unit0;
  const int n = pd.n, m = pd.m, T = pd.T, K = pd.nseg;
  const bool last = (seg == K - 1);
  const int t0 = seg_begin(T, K, seg), t1 = seg_begin(T, K, seg + 1);
  const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm = (size_t)m * m;
  const WsLayout wl = ws_layout(n, K);

  double* x = reinterpret_cast<double*>(smem);  // n
  double* xn = x + n;                           // n
  double* u = xn + n;                           // m
  double* w1 = u + m;                           // n   (stage-cost partials)
  double* w2 = w1 + n;                          // m

  const TS* gA = static_cast<const TS*>(pd.A);
  const TS* gB = static_cast<const TS*>(pd.B);
  const TS* gc = static_cast<const TS*>(pd.c);
  const TS* gQ = static_cast<const TS*>(pd.Q);
  const TS* gR = static_cast<const TS*>(pd.R);
  const TS* gS = static_cast<const TS*>(pd.S);
  const TS* gq = static_cast<const TS*>(pd.q);
  const TS* gr = static_cast<const TS*>(pd.r);
  const TS* gK = static_cast<const TS*>(pd.K);
  const TS* gk = static_cast<const TS*>(pd.k);
  TS* ox = static_cast<TS*>(pd.x);
  TS* ou = static_cast<TS*>(pd.u);
  TS* olam = static_cast<TS*>(pd.lam);

  const double* zj = pd.ws + wl.z + (long long)seg * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = zj[i];
  __syncthreads();

  double cost = 0.0;  // per-thread partial
  for (int t = t0; t < t1; ++t) {
    const TS* Kt = gK + nm * t;
    const TS* kt = gk + (size_t)m * t;
    // u = K x + k
    warp_rows<TS, double>(m, n, Kt, x, [&](int a, double s) { u[a] = s + static_cast<double>(kt[a]); });
    __syncthreads();
    if (ox)
      for (int i = threadIdx.x; i < n; i += blockDim.x) ox[(size_t)n * t + i] = static_cast<TS>(x[i]);
    if (ou)
      for (int a = threadIdx.x; a < m; a += blockDim.x) ou[(size_t)m * t + a] = static_cast<TS>(u[a]);
    const TS* At = gA + nn * t;
    const TS* Bt = gB + nm * t;
    const TS* ct = gc + (size_t)n * t;
    const TS* Qt = gQ + nn * t;
    const TS* Rt = gR + mm * t;
    const TS* qt = gq + (size_t)n * t;
    const TS* rt = gr + (size_t)m * t;
    // x_{t+1} = A x + B u + c   (two passes: A x into xn, then += B u + c)
    warp_rows<TS, double>(n, n, At, x, [&](int i, double s) { xn[i] = s; });
    // stage cost terms: w1 = Q x, w2 = R u
    warp_rows<TS, double>(n, n, Qt, x, [&](int i, double s) { w1[i] = s; });
    warp_rows<TS, double>(m, m, Rt, u, [&](int a, double s) { w2[a] = s; });
    __syncthreads();
    warp_rows<TS, double>(n, m, Bt, u, [&](int i, double s) { xn[i] += s + static_cast<double>(ct[i]); });
    if (gS) {
      // u'S x: w2 += 2 * S x  (so that 1/2 u'w2 = 1/2 u'R u + u'S x)
      warp_rows<TS, double>(m, n, gS + nm * t, x, [&](int a, double s) { w2[a] += 2.0 * s; });
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      cost += x[i] * (0.5 * w1[i] + static_cast<double>(qt[i]));
    for (int a = threadIdx.x; a < m; a += blockDim.x)
      cost += u[a] * (0.5 * w2[a] + static_cast<double>(rt[a]));
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = xn[i];
    __syncthreads();
  }
  if (last) {
    const TS* QT = gQ + nn * T;
    const TS* qT = gq + (size_t)n * T;
    if (ox)
      for (int i = threadIdx.x; i < n; i += blockDim.x) ox[(size_t)n * T + i] = static_cast<TS>(x[i]);
    warp_rows<TS, double>(n, n, QT, x, [&](int i, double s) { w1[i] = s; });
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      cost += x[i] * (0.5 * w1[i] + static_cast<double>(qT[i]));
  }
  {
    const double tot = block_sum(cost, s_red);
    if (threadIdx.x == 0) pd.ws[wl.costp + seg] = tot;
  }
  if (!want_lam || !olam) return;
  __syncthreads();
  // ---- multipliers: lambda at the segment end, then backwards -------------------
  double* lam = w1;  // n : lambda_{t+1}
  double* ln = xn;   // n : lambda_t under construction
  if (last) {
    // lambda_T = -(sym(Q_T) x_T + q_T), x still holds x_T
    const TS* QT = gQ + nn * T;
    const TS* qT = gq + (size_t)n * T;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double s = 0.0;
      for (int i = 0; i < n; ++i) s += 0.5 * (static_cast<double>(QT[(size_t)i * n + j]) + static_cast<double>(QT[(size_t)j * n + i])) * x[i];
      lam[j] = -(s + static_cast<double>(qT[j]));
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) olam[(size_t)n * T + j] = static_cast<TS>(lam[j]);
  } else {
    const double* Pn = pd.ws + wl.Pi + (long long)(seg + 1) * nn;
    const double* pn = pd.ws + wl.pi + (long long)(seg + 1) * n;
    const double* zn = pd.ws + wl.z + (long long)(seg + 1) * n;
    warp_rows<double, double>(n, n, Pn, zn, [&](int i, double s) { lam[i] = -(s + pn[i]); });
  }
  __syncthreads();
  for (int t = t1 - 1; t >= t0; --t) {
    const TS* At = gA + nn * t;
    const TS* Qt = gQ + nn * t;
    const TS* qt = gq + (size_t)n * t;
    // x_t and u_t back from the outputs written above (same block: visible after the barriers)
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = static_cast<double>(ox[(size_t)n * t + i]);
    for (int a = threadIdx.x; a < m; a += blockDim.x) u[a] = static_cast<double>(ou[(size_t)m * t + a]);
    __syncthreads();
    // lambda_t[j] = sum_i A[i][j] lam[i] - sum_i Qs[j][i] x[i] - sum_a S[a][j] u[a] - q[j]
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double s = 0.0;
      for (int i = 0; i < n; ++i) {
        s = fma(static_cast<double>(At[(size_t)i * n + j]), lam[i], s);
        s -= 0.5 * (static_cast<double>(Qt[(size_t)i * n + j]) + static_cast<double>(Qt[(size_t)j * n + i])) * x[i];
      }
      if (gS)
        for (int a = 0; a < m; ++a) s -= static_cast<double>(gS[nm * t + (size_t)a * n + j]) * u[a];
      ln[j] = s - static_cast<double>(qt[j]);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      lam[j] = ln[j];
      olam[(size_t)n * t + j] = static_cast<TS>(ln[j]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Streaming variant (x and u outputs present): the stage data of the next
// stages is copied into a ring of shared-memory slots with cp.async while the
// current stage is evaluated, so the segment's walk is bound by the copy
// stream rather than by one global-load latency per product. Products are in
// the data type (FP32 data: FP32 products; the objective is summed in FP64).
// Forward slot: K_t, A_t, B_t, k_t, c_t. Backward slot (the objective and the
// multipliers, t from the segment end down): A_t, Q_t, S_t, R_t, q_t, r_t;
// x_t and u_t are re-read from the outputs one stage ahead.
// ---------------------------------------------------------------------------
struct RollSlot {
  long long K, A, B, k, c;        // forward
  long long Ab, Q, S, R, q, r;    // backward
  long long elems;
};

__host__ __device__ inline long long al16(long long cnt, int es) {
  const int per = 16 / es;
  return (cnt + per - 1) / per * per;
}

__host__ __device__ inline RollSlot roll_slot(int n, int m, int es) {
  RollSlot L;
  const long long nn = (long long)n * n, nm = (long long)n * m, mm = (long long)m * m;
  long long o = 0;
  L.K = o; o += al16(nm, es);
  L.A = o; o += al16(nn, es);
  L.B = o; o += al16(nm, es);
  L.k = o; o += al16(m, es);
  L.c = o; o += al16(n, es);
  const long long f = o;
  o = 0;
  L.Ab = o; o += al16(nn, es);
  L.Q = o;  o += al16(nn, es);
  L.S = o;  o += al16(nm, es);
  L.R = o;  o += al16(mm, es);
  L.q = o;  o += al16(n, es);
  L.r = o;  o += al16(m, es);
  L.elems = f > o ? f : o;
  return L;
}

__host__ __device__ inline long long roll_vec_elems(int nmax, int mmax, int nwarps) {
  const long long n4 = (nmax + 3) & ~3, m4 = (mmax + 3) & ~3;
  return 2 * n4 + 2 * m4 + 2 * n4 + n4 + 2 * m4 + (long long)nwarps * n4;
}

template <typename TS>
__global__ void __launch_bounds__(kBlock) rollout_stream_kernel(ProbTable tab, int want_lam, int depth, int nmax,
                                                                int mmax) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_flag;
  __shared__ double s_red[kBlock / 32];
  const int unit = blockIdx.x;
  const ProbDesc& pd = prob_of_unit(tab, unit);
  if (cta_should_exit(pd, &s_flag)) return;
  const int seg = unit - pd.unit0;
  const int n = pd.n, m = pd.m, T = pd.T, K = pd.nseg;
  const bool last = (seg == K - 1);
  const int t0 = seg_begin(T, K, seg), t1 = seg_begin(T, K, seg + 1);
  const long long nn = (long long)n * n, nm = (long long)n * m, mm = (long long)m * m;
  const WsLayout wl = ws_layout(n, K);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const RollSlot L = roll_slot(n, m, sizeof(TS));
  const long long stride = roll_slot(nmax, mmax, sizeof(TS)).elems;
  const int n4 = (nmax + 3) & ~3, m4 = (mmax + 3) & ~3;
  TS* ring = reinterpret_cast<TS*>(smem);
  TS* xb = ring + depth * stride;  // 2 x n4
  TS* ub = xb + 2 * n4;            // 2 x m4
  TS* lb = ub + 2 * m4;            // 2 x n4
  TS* w1 = lb + 2 * n4;            // n4   Q x
  TS* w2 = w1 + n4;                // m4   R u
  TS* w3 = w2 + m4;                // m4   S x
  TS* part = w3 + m4;              // nw x n4

  const TS* gA = static_cast<const TS*>(pd.A);
  const TS* gB = static_cast<const TS*>(pd.B);
  const TS* gc = static_cast<const TS*>(pd.c);
  const TS* gQ = static_cast<const TS*>(pd.Q);
  const TS* gR = static_cast<const TS*>(pd.R);
  const TS* gS = static_cast<const TS*>(pd.S);
  const TS* gq = static_cast<const TS*>(pd.q);
  const TS* gr = static_cast<const TS*>(pd.r);
  const TS* gK = static_cast<const TS*>(pd.K);
  const TS* gk = static_cast<const TS*>(pd.k);
  TS* ox = static_cast<TS*>(pd.x);
  TS* ou = static_cast<TS*>(pd.u);
  TS* olam = static_cast<TS*>(pd.lam);

  auto wait_ring = [&]() {
    if (depth >= 3) cp_async_wait<1>();
    else cp_async_wait<0>();
  };
  auto warp_sum = [&](TS v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  };
  // ---- forward: x_{t+1} = A x + B (K x + k) + c ----------------------------
  auto fwd_issue = [&](int t) {
    if (t < t1) {
      TS* d = ring + (long long)((t - t0) % depth) * stride;
      cta_copy_async(d + L.K, gK + nm * t, nm);
      cta_copy_async(d + L.A, gA + nn * t, nn);
      cta_copy_async(d + L.B, gB + nm * t, nm);
      cta_copy_async(d + L.k, gk + (long long)m * t, (long long)m);
      cta_copy_async(d + L.c, gc + (long long)n * t, (long long)n);
    }
    cp_async_commit();
  };
  for (int q = 0; q < depth - 1; ++q) fwd_issue(t0 + q);
  {
    const double* zj = pd.ws + wl.z + (long long)seg * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) xb[i] = static_cast<TS>(zj[i]);
  }
  for (int t = t0; t < t1; ++t) {
    wait_ring();
    __syncthreads();
    fwd_issue(t + depth - 1);
    const TS* d = ring + (long long)((t - t0) % depth) * stride;
    const TS* xc = xb + ((t - t0) & 1) * n4;
    TS* xn = xb + (((t - t0) + 1) & 1) * n4;
    TS* uc = ub + ((t - t0) & 1) * m4;
    for (int rr = warp; rr < m + n; rr += nw) {
      const TS* row = (rr < m) ? d + L.K + (long long)rr * n : d + L.A + (long long)(rr - m) * n;
      TS acc = TS(0);
      for (int k = lane; k < n; k += 32) acc = fma(row[k], xc[k], acc);
      acc = warp_sum(acc);
      if (lane == 0) {
        if (rr < m) uc[rr] = acc + d[L.k + rr];
        else xn[rr - m] = acc;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) ox[(long long)n * t + i] = xc[i];
    for (int a = threadIdx.x; a < m; a += blockDim.x) ou[(long long)m * t + a] = uc[a];
    for (int i = warp; i < n; i += nw) {
      const TS* row = d + L.B + (long long)i * m;
      TS acc = TS(0);
      for (int a = lane; a < m; a += 32) acc = fma(row[a], uc[a], acc);
      acc = warp_sum(acc);
      if (lane == 0) xn[i] += acc + d[L.c + i];
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  // ---- the segment end: x_T, or lambda at b_{j+1} from the link ------------
  const int Ls = t1 - t0;
  const TS* xe = xb + (Ls & 1) * n4;  // x_{t1}
  double cost = 0.0;
  TS* lcur = lb;
  const int rows_per = (n + nw - 1) / nw;
  // part[w][j] = sum over this warp's rows i of (M1[i][j] v1[i] + M2[i][j] v2[i]) (+ -S[a][j] u[a] for its S rows)
  auto col_partials = [&](const TS* M1, const TS* v1, const TS* M2, const TS* v2, const TS* Sm, const TS* us) {
    TS acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = TS(0);
    const int i0 = warp * rows_per, i1 = min(n, i0 + rows_per);
    for (int i = i0; i < i1; ++i) {
      const TS a1 = M1 ? v1[i] : TS(0), a2 = v2[i];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int j = lane + 32 * c;
        if (j < n) {
          TS v = M2[(long long)i * n + j] * a2;
          if (M1) v = fma(M1[(long long)i * n + j], a1, v);
          acc[c] += v;
        }
      }
    }
    if (Sm) {
      const int sper = (m + nw - 1) / nw, a0 = warp * sper, a1e = min(m, a0 + sper);
      for (int a = a0; a < a1e; ++a) {
        const TS ua = us[a];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int j = lane + 32 * c;
          if (j < n) acc[c] = fma(-Sm[(long long)a * n + j], ua, acc[c]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int j = lane + 32 * c;
      if (j < n) part[warp * n4 + j] = acc[c];
    }
  };
  if (last) {
    const TS* QT = gQ + nn * T;
    const TS* qT = gq + (long long)n * T;
    for (int i = threadIdx.x; i < n; i += blockDim.x) ox[(long long)n * T + i] = xe[i];
    for (int i = warp; i < n; i += nw) {
      TS acc = TS(0);
      for (int k = lane; k < n; k += 32) acc = fma(QT[(long long)i * n + k], xe[k], acc);
      acc = warp_sum(acc);
      if (lane == 0) w1[i] = acc;
    }
    col_partials(nullptr, nullptr, QT, xe, nullptr, nullptr);  // Q_T' x_T
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      TS tq = TS(0);
      for (int w = 0; w < nw; ++w) tq += part[w * n4 + j];
      const TS l = -(TS(0.5) * (w1[j] + tq) + qT[j]);
      lcur[j] = l;
      if (want_lam && olam) olam[(long long)n * T + j] = l;
      cost += static_cast<double>(xe[j]) * (0.5 * static_cast<double>(w1[j]) + static_cast<double>(qT[j]));
    }
  } else {
    const double* Pn = pd.ws + wl.Pi + (long long)(seg + 1) * nn;
    const double* pn = pd.ws + wl.pi + (long long)(seg + 1) * n;
    const double* zn = pd.ws + wl.z + (long long)(seg + 1) * n;
    for (int i = warp; i < n; i += nw) {
      double acc = 0.0;
      for (int k = lane; k < n; k += 32) acc = fma(Pn[(long long)i * n + k], zn[k], acc);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) lcur[i] = static_cast<TS>(-(acc + pn[i]));
    }
  }
  __syncthreads();
  // ---- backward: objective and lambda_t = A'lambda_{t+1} - Qs x - S'u - q ---
  auto bwd_issue = [&](int t) {
    if (t >= t0) {
      TS* d = ring + (long long)((t1 - 1 - t) % depth) * stride;
      cta_copy_async(d + L.Ab, gA + nn * t, nn);
      cta_copy_async(d + L.Q, gQ + nn * t, nn);
      if (gS) cta_copy_async(d + L.S, gS + nm * t, nm);
      cta_copy_async(d + L.R, gR + mm * t, mm);
      cta_copy_async(d + L.q, gq + (long long)n * t, (long long)n);
      cta_copy_async(d + L.r, gr + (long long)m * t, (long long)m);
    }
    cp_async_commit();
  };
  for (int q = 0; q < depth - 1; ++q) bwd_issue(t1 - 1 - q);
  // x_t, u_t of the next stage down, one element pair per thread (n, m <= 256 = blockDim)
  TS px = TS(0), pu = TS(0);
  const int tid = threadIdx.x;
  if (t1 - 1 >= t0) {
    if (tid < n) px = ox[(long long)n * (t1 - 1) + tid];
    if (tid < m) pu = ou[(long long)m * (t1 - 1) + tid];
  }
  for (int t = t1 - 1; t >= t0; --t) {
    const int bsel = (t1 - 1 - t) & 1;
    TS* xv = xb + bsel * n4;
    TS* uv = ub + bsel * m4;
    if (tid < n) xv[tid] = px;
    if (tid < m) uv[tid] = pu;
    wait_ring();
    __syncthreads();
    bwd_issue(t - depth + 1);
    if (t - 1 >= t0) {
      if (tid < n) px = ox[(long long)n * (t - 1) + tid];
      if (tid < m) pu = ou[(long long)m * (t - 1) + tid];
    }
    const TS* d = ring + (long long)((t1 - 1 - t) % depth) * stride;
    const TS* Ad = d + L.Ab;
    const TS* Qd = d + L.Q;
    const TS* Sd = gS ? d + L.S : nullptr;
    const TS* Rd = d + L.R;
    // rows: Q x (n), R u (m), S x (m)
    const int nrows = n + m + (gS ? m : 0);
    for (int rr = warp; rr < nrows; rr += nw) {
      const TS* row;
      const TS* v;
      int len;
      if (rr < n) { row = Qd + (long long)rr * n; v = xv; len = n; }
      else if (rr < n + m) { row = Rd + (long long)(rr - n) * m; v = uv; len = m; }
      else { row = Sd + (long long)(rr - n - m) * n; v = xv; len = n; }
      TS acc = TS(0);
      for (int k = lane; k < len; k += 32) acc = fma(row[k], v[k], acc);
      acc = warp_sum(acc);
      if (lane == 0) {
        if (rr < n) w1[rr] = acc;
        else if (rr < n + m) w2[rr - n] = acc;
        else w3[rr - n - m] = acc;
      }
    }
    // columns: A'lambda - (1/2) Q'x - S'u, the -(1/2) folded into a scaled copy of x
    TS* xh = lb + (1 - (lcur == lb ? 0 : 1)) * n4;  // the free lambda buffer holds -x/2 for this pass
    if (tid < n) xh[tid] = TS(-0.5) * xv[tid];
    __syncthreads();
    col_partials(Ad, lcur, Qd, xh, Sd, uv);
    __syncthreads();
    TS* lnext = xh;  // overwritten with lambda_t below (x/2 no longer read after the barrier)
    for (int j = tid; j < n; j += blockDim.x) {
      TS tq = TS(0);
      for (int w = 0; w < nw; ++w) tq += part[w * n4 + j];
      const TS l = tq - TS(0.5) * w1[j] - d[L.q + j];
      lnext[j] = l;
      if (want_lam && olam) olam[(long long)n * t + j] = l;
      cost += static_cast<double>(xv[j]) * (0.5 * static_cast<double>(w1[j]) + static_cast<double>(d[L.q + j]));
    }
    for (int a = tid; a < m; a += blockDim.x)
      cost += static_cast<double>(uv[a]) *
              (0.5 * static_cast<double>(w2[a]) + (gS ? static_cast<double>(w3[a]) : 0.0) + static_cast<double>(d[L.r + a]));
    lcur = lnext;
  }
  cp_async_wait<0>();
  const double tot = block_sum(cost, s_red);
  if (threadIdx.x == 0) pd.ws[wl.costp + seg] = tot;
}

}  // namespace lqr

#include "rollout_f32_body.cuh"

namespace lqr {

__global__ void __launch_bounds__(kRollBlock, 1) rollout_f32_kernel(ProbTable tab, int want_lam, int nmax, int mmax) {
  rollout_f32_unit(tab, (int)blockIdx.x, want_lam, nmax, mmax);
}

long long rollout_f32_smem_bytes(int nmax, int mmax) {
  return 4 * (2 * fast_roll_slot(nmax, mmax).elems + fast_roll_vec(nmax, mmax));
}

__global__ void finalize_kernel(ProbTable tab) {
  const ProbDesc& pd = prob_at(tab, blockIdx.x);
  if (threadIdx.x != 0) return;
  if (pd.skip && *(volatile const int*)pd.skip) return;
  if (*(volatile int*)pd.status != 0) {
    pd.report[0] = 0.0;
    return;
  }
  const WsLayout wl = ws_layout(pd.n, pd.nseg);
  double s = 0.0;
  for (int j = 0; j < pd.nseg; ++j) s += pd.ws[wl.costp + j];
  if (!isfinite(s)) raise_status(pd.status, LQR_ERR_NONFINITE, -1);
  pd.report[0] = s;
}

template <typename TS, typename TC>
cudaError_t launch_rollout(const ProbTable& tab, int nunits, int want_lam, cudaStream_t st, int nmax_, int mmax_,
                           int has_xu) {
  const int nmax = nmax_ > 0 ? nmax_ : tab.single.n, mmax = mmax_ > 0 ? mmax_ : tab.single.m;
  if (has_xu) {
    int optin = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const long long budget = (long long)optin - kStaticSmemReserve;
    if (sizeof(TS) == 4 && ((nmax + 3) & ~3) <= kRollBlock) {
      const long long fb = rollout_f32_smem_bytes(nmax, mmax);
      if (fb <= budget) {
        cudaError_t e = raise_dyn_smem((const void*)rollout_f32_kernel, (size_t)fb);
        if (e != cudaSuccess) return e;
        rollout_f32_kernel<<<nunits, kRollBlock, (size_t)fb, st>>>(tab, want_lam, nmax, mmax);
        return cudaGetLastError();
      }
    }
    const long long slot = roll_slot(nmax, mmax, sizeof(TS)).elems * (long long)sizeof(TS);
    const long long vec = roll_vec_elems(nmax, mmax, kBlock / 32) * (long long)sizeof(TS);
    long long depth = (budget - vec) / slot;
    if (depth > 3) depth = 3;
    if (depth >= 2) {
      const size_t bytes = (size_t)(depth * slot + vec);
      cudaError_t e = raise_dyn_smem((const void*)rollout_stream_kernel<TS>, bytes);
      if (e != cudaSuccess) return e;
      rollout_stream_kernel<TS><<<nunits, kBlock, bytes, st>>>(tab, want_lam, (int)depth, nmax, mmax);
      return cudaGetLastError();
    }
  }
  const size_t bytes = sizeof(double) * (size_t)(3 * nmax + 2 * mmax);
  rollout_kernel<TS><<<nunits, kBlock, bytes, st>>>(tab, want_lam);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const ProbTable& tab, int nprob, cudaStream_t st) {
  finalize_kernel<<<nprob, 32, 0, st>>>(tab);
  return cudaGetLastError();
}

template cudaError_t launch_rollout<double, double>(const ProbTable&, int, int, cudaStream_t, int, int, int);
template cudaError_t launch_rollout<float, float>(const ProbTable&, int, int, cudaStream_t, int, int, int);
template cudaError_t launch_rollout<double, float>(const ProbTable&, int, int, cudaStream_t, int, int, int);

}  // namespace lqr
