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
cudaError_t launch_rollout(const ProbTable& tab, int nunits, int want_lam, cudaStream_t st, int nmax_, int mmax_) {
  const int nmax = nmax_ > 0 ? nmax_ : tab.single.n, mmax = mmax_ > 0 ? mmax_ : tab.single.m;
  const size_t bytes = sizeof(double) * (size_t)(3 * nmax + 2 * mmax);
  rollout_kernel<TS><<<nunits, kBlock, bytes, st>>>(tab, want_lam);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const ProbTable& tab, int nprob, cudaStream_t st) {
  finalize_kernel<<<nprob, 32, 0, st>>>(tab);
  return cudaGetLastError();
}

template cudaError_t launch_rollout<double, double>(const ProbTable&, int, int, cudaStream_t, int, int);
template cudaError_t launch_rollout<float, float>(const ProbTable&, int, int, cudaStream_t, int, int);
template cudaError_t launch_rollout<double, float>(const ProbTable&, int, int, cudaStream_t, int, int);

}  // namespace lqr
