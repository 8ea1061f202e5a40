// Steps A7/A8: the FP64 residual of the global KKT system of Eq. 3 at a
// computed (x, u, lambda), its normwise backward error, the objective of
// Eq. 1 along (x, u), and the update of iterative refinement.
//
// With r = KKT w - b (blocks, Q and R read symmetrised):
//   rx_t = Q x_t + S'u_t + q_t + lambda_t - A_t'lambda_{t+1}     (t < T)
//   ru_t = S x_t + R u_t + r_t - B_t'lambda_{t+1}
//   rxT  = Q_T x_T + q_T + lambda_T
//   r0   = x_0 - x0
//   rd_t = x_{t+1} - A_t x_t - B_t u_t - c_t
// the correction delta solves KKT delta = r, which is the LQR problem with the
// same matrices and the vector data q~ = -rx (q~_T = -rxT), r~ = -ru,
// c~ = rd, x0~ = r0; then w <- w - delta. The backward error is
//   eta = |r|_inf / (|KKT|_inf |w|_inf + |b|_inf),  rel = |r|_inf / |b|_inf,
// with |KKT|_inf the largest absolute row sum.
#include <cuda_runtime.h>

#include "kkt_stage.cuh"
#include "kkt_stage_df.cuh"
#include "lqr_internal.cuh"

namespace lqr {

namespace {

// max of non-negative doubles through their bit patterns (monotone for x >= 0)
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  if (!(v >= 0.0)) v = __longlong_as_double(0x7ff0000000000000LL);  // NaN -> +inf
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace

// Residual-pass accumulators (FP64, in the refinement workspace).
enum ResidSlot { RS_RNORM = 0, RS_KNORM, RS_WNORM, RS_BNORM, RS_COST, RS_COUNT };

// One CTA per stage (grid-stride). Stage t < T, plus the terminal / initial
// rows handled by the CTA that owns t = T-1 / t = 0.
// want_knorm: also the |KKT| row sums of the backward error (the final pass and
// the first refinement pass); the other refinement passes only need |r| and |b|.
template <typename TS>
__global__ void __launch_bounds__(kBlock) kkt_residual_kernel(ProbDesc pd, double* acc, KktOut out, const int* skip,
                                                              int want_knorm) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (skip && *(volatile const int*)skip) return;
  if (*(volatile int*)pd.status != 0) return;
  const int n = pd.n, m = pd.m, T = pd.T;
  const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm = (size_t)m * m;
  double* xt = reinterpret_cast<double*>(smem);
  double* xn = xt + n;
  double* lt = xn + n;
  double* ln = lt + n;
  double* ut = ln + n;
  double* rxv = ut + m;   // n: accumulates rx_t
  double* ruv = rxv + n;  // m: accumulates ru_t
  double* rdv = ruv + m;  // n: accumulates rd_t
  const TS* gx = static_cast<const TS*>(pd.x);
  const TS* gu = static_cast<const TS*>(pd.u);
  const TS* gl = static_cast<const TS*>(pd.lam);
  const TS* gA = static_cast<const TS*>(pd.A);
  const TS* gB = static_cast<const TS*>(pd.B);
  const TS* gc = static_cast<const TS*>(pd.c);
  const TS* gQ = static_cast<const TS*>(pd.Q);
  const TS* gR = static_cast<const TS*>(pd.R);
  const TS* gS = static_cast<const TS*>(pd.S);
  const TS* gq = static_cast<const TS*>(pd.q);
  const TS* gr = static_cast<const TS*>(pd.r);
  const TS* gx0 = static_cast<const TS*>(pd.x0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double rmax = 0.0, kmax = 0.0, wmax = 0.0, bmax = 0.0, cost = 0.0;  // per-thread partials

  for (int t = blockIdx.x; t < T; t += gridDim.x) {
    const TS* At = gA + nn * t;
    const TS* Bt = gB + nm * t;
    const TS* Qt = gQ + nn * t;
    const TS* Rt = gR + mm * t;
    const TS* St = gS ? gS + nm * t : nullptr;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      xt[i] = (double)gx[(size_t)n * t + i];
      xn[i] = (double)gx[(size_t)n * (t + 1) + i];
      lt[i] = (double)gl[(size_t)n * t + i];
      ln[i] = (double)gl[(size_t)n * (t + 1) + i];
      rxv[i] = (double)gq[(size_t)n * t + i] + lt[i];
      rdv[i] = xn[i] - (double)gc[(size_t)n * t + i];
    }
    for (int a = threadIdx.x; a < m; a += blockDim.x) {
      ut[a] = (double)gu[(size_t)m * t + a];
      ruv[a] = (double)gr[(size_t)m * t + a];
    }
    __syncthreads();
    // columns j < n: -A'lambda_{t+1}, Q'x/2 (half of the symmetrised product), S'u; row-sum pieces
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double s = 0.0, absA = 0.0, absS = 0.0;
#pragma unroll 8
      for (int i = 0; i < n; ++i) {
        const double a = (double)At[(size_t)i * n + j];
        s = fma(-a, ln[i], s);
        s = fma(0.5 * (double)Qt[(size_t)i * n + j], xt[i], s);
        if (want_knorm) absA += fabs(a);
      }
      if (St)
        for (int a = 0; a < m; ++a) {
          const double v = (double)St[(size_t)a * n + j];
          s = fma(v, ut[a], s);
          if (want_knorm) absS += fabs(v);
        }
      rxv[j] += s;
      if (want_knorm) {  // |Q_sym| row sum of row j
        double absQ = 0.0;
        for (int k = 0; k < n; ++k)
          absQ += fabs(0.5 * ((double)Qt[(size_t)j * n + k] + (double)Qt[(size_t)k * n + j]));
        kmax = fmax(kmax, absQ + absS + 1.0 + absA);
      }
    }
    // columns a < m: -B'lambda_{t+1}, R'u/2
    for (int a = threadIdx.x; a < m; a += blockDim.x) {
      double s = 0.0, absB = 0.0, absR = 0.0, absSr = 0.0;
#pragma unroll 8
      for (int i = 0; i < n; ++i) {
        const double b = (double)Bt[(size_t)i * m + a];
        s = fma(-b, ln[i], s);
        if (want_knorm) absB += fabs(b);
      }
      for (int b = 0; b < m; ++b) {
        s = fma(0.5 * (double)Rt[(size_t)b * m + a], ut[b], s);
        if (want_knorm) absR += fabs(0.5 * ((double)Rt[(size_t)a * m + b] + (double)Rt[(size_t)b * m + a]));
      }
      if (St && want_knorm)
        for (int k = 0; k < n; ++k) absSr += fabs((double)St[(size_t)a * n + k]);
      ruv[a] += s;
      if (want_knorm) kmax = fmax(kmax, absSr + absR + absB);
    }
    __syncthreads();
    // rows i < n (warp per row): Q x/2, -A x - B u ; dynamics-row sums ; stage cost 1/2 x'Qx + q'x
    for (int i = warp; i < n; i += nw) {
      double qx = 0.0, ax = 0.0, absr = 0.0;
      for (int k = lane; k < n; k += 32) {
        const double a = (double)At[(size_t)i * n + k];
        ax = fma(a, xt[k], ax);
        qx = fma((double)Qt[(size_t)i * n + k], xt[k], qx);
        if (want_knorm) absr += fabs(a);
      }
      for (int b = lane; b < m; b += 32) {
        const double v = (double)Bt[(size_t)i * m + b];
        ax = fma(v, ut[b], ax);
        if (want_knorm) absr += fabs(v);
      }
      qx = warp_sum(qx);
      ax = warp_sum(ax);
      absr = warp_sum(absr);
      if (lane == 0) {
        rxv[i] += 0.5 * qx;
        rdv[i] -= ax;
        kmax = fmax(kmax, 1.0 + absr);
        cost += xt[i] * (0.5 * qx + (double)gq[(size_t)n * t + i]);
      }
    }
    // rows a < m: S x, R u/2 ; stage cost u'S x + 1/2 u'R u + r'u
    for (int a = warp; a < m; a += nw) {
      double sx = 0.0, ru = 0.0;
      if (St)
        for (int k = lane; k < n; k += 32) sx = fma((double)St[(size_t)a * n + k], xt[k], sx);
      for (int b = lane; b < m; b += 32) ru = fma((double)Rt[(size_t)a * m + b], ut[b], ru);
      sx = warp_sum(sx);
      ru = warp_sum(ru);
      if (lane == 0) {
        ruv[a] += sx + 0.5 * ru;
        cost += ut[a] * (sx + 0.5 * ru + (double)gr[(size_t)m * t + a]);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      rmax = fmax(rmax, fmax(fabs(rxv[i]), fabs(rdv[i])));
      wmax = fmax(wmax, fmax(fabs(xt[i]), fabs(lt[i])));
      bmax = fmax(bmax, fmax(fabs((double)gq[(size_t)n * t + i]), fabs((double)gc[(size_t)n * t + i])));
      if (out.q) {
        out.put(out.q, (size_t)n * t + i, -rxv[i]);
        out.put(out.c, (size_t)n * t + i, rdv[i]);
      }
    }
    for (int a = threadIdx.x; a < m; a += blockDim.x) {
      rmax = fmax(rmax, fabs(ruv[a]));
      wmax = fmax(wmax, fabs(ut[a]));
      bmax = fmax(bmax, fabs((double)gr[(size_t)m * t + a]));
      if (out.q) out.put(out.r, (size_t)m * t + a, -ruv[a]);
    }
    __syncthreads();
  }
  // terminal row (Q_T x_T + q_T + lambda_T) and the initial row (x_0 - x0)
  if (blockIdx.x == 0) {
    const TS* QT = gQ + nn * T;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double s = (double)gq[(size_t)n * T + i] + (double)gl[(size_t)n * T + i];
      double absQ = 0.0, qx = 0.0;
      for (int k = 0; k < n; ++k) {
        const double qs = 0.5 * ((double)QT[(size_t)i * n + k] + (double)QT[(size_t)k * n + i]);
        s = fma(qs, (double)gx[(size_t)n * T + k], s);
        qx = fma((double)QT[(size_t)i * n + k], (double)gx[(size_t)n * T + k], qx);
        absQ += fabs(qs);
      }
      const double xT = (double)gx[(size_t)n * T + i];
      cost += xT * (0.5 * qx + (double)gq[(size_t)n * T + i]);
      const double r0 = (double)gx[i] - (double)gx0[i];
      rmax = fmax(rmax, fmax(fabs(s), fabs(r0)));
      kmax = fmax(kmax, absQ + 1.0);
      wmax = fmax(wmax, fmax(fabs(xT), fabs((double)gl[(size_t)n * T + i])));
      bmax = fmax(bmax, fmax(fabs((double)gq[(size_t)n * T + i]), fabs((double)gx0[i])));
      if (out.q) {
        out.put(out.q, (size_t)n * T + i, -s);
        out.put(out.x0, i, r0);
      }
    }
  }
  // block reduction then one atomic per block
  __shared__ double red[5][kBlock / 32];
  rmax = warp_max(rmax);
  kmax = warp_max(kmax);
  wmax = warp_max(wmax);
  bmax = warp_max(bmax);
  cost = warp_sum(cost);
  if (lane == 0) {
    red[0][warp] = rmax; red[1][warp] = kmax; red[2][warp] = wmax; red[3][warp] = bmax; red[4][warp] = cost;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a[5] = {0, 0, 0, 0, 0};
    for (int w = 0; w < nw; ++w) {
      for (int k = 0; k < 4; ++k) a[k] = fmax(a[k], red[k][w]);
      a[4] += red[4][w];
    }
    atomic_max_nonneg(acc + RS_RNORM, a[0]);
    atomic_max_nonneg(acc + RS_KNORM, a[1]);
    atomic_max_nonneg(acc + RS_WNORM, a[2]);
    atomic_max_nonneg(acc + RS_BNORM, a[3]);
    // per-block cost partials, summed in a fixed order by the finalize kernel
    acc[RS_COUNT + blockIdx.x] = a[4];
  }
}

// Streaming form of the same residual (the stage block of kkt_stage.cuh);
// grid-stride over the stages like kkt_residual_kernel.
template <int NC, bool KN, typename TS>
__global__ void __launch_bounds__(kKktBlock, 2)
    kkt_residual_stream_kernel(ProbDesc pd, double* acc, KktOut out, const int* skip, int use_stash, int gate) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (skip && *(volatile const int*)skip) return;
  if (gate && (((volatile const int*)skip)[2] == 0) != (gate == 1)) return;  // not this iteration's form
  if (*(volatile int*)pd.status != 0) return;
  const int n = pd.n, T = pd.T;
  KktData<TS> g;
  g.x = static_cast<const TS*>(pd.x);
  g.u = static_cast<const TS*>(pd.u);
  g.lam = static_cast<const TS*>(pd.lam);
  g.A = static_cast<const TS*>(pd.A);
  g.B = static_cast<const TS*>(pd.B);
  g.c = static_cast<const TS*>(pd.c);
  g.Q = static_cast<const TS*>(pd.Q);
  g.R = static_cast<const TS*>(pd.R);
  g.S = static_cast<const TS*>(pd.S);
  g.q = static_cast<const TS*>(pd.q);
  g.r = static_cast<const TS*>(pd.r);
  g.n = pd.n;
  g.m = pd.m;
  const TS* gx0 = static_cast<const TS*>(pd.x0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* sm = reinterpret_cast<double*>(smem);
  double* stash = use_stash ? sm + kkt_stage_smem_doubles(pd.n, pd.m) : nullptr;
  KktMax mx;
  double cost = 0.0;
  for (int t = blockIdx.x; t < T; t += gridDim.x) cost += kkt_stage<NC, KN>(g, t, sm, mx, out, stash);
  // terminal row (Q_T x_T + q_T + lambda_T) and the initial row (x_0 - x0)
  if (blockIdx.x == 0) {
    const TS* QT = g.Q + (size_t)n * n * T;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double s = (double)g.q[(size_t)n * T + i] + (double)g.lam[(size_t)n * T + i];
      double absQ = 0.0, qx = 0.0;
      for (int k = 0; k < n; ++k) {
        const double qs = 0.5 * ((double)QT[(size_t)i * n + k] + (double)QT[(size_t)k * n + i]);
        s = fma(qs, (double)g.x[(size_t)n * T + k], s);
        qx = fma((double)QT[(size_t)i * n + k], (double)g.x[(size_t)n * T + k], qx);
        absQ += fabs(qs);
      }
      const double xT = (double)g.x[(size_t)n * T + i];
      cost += xT * (0.5 * qx + (double)g.q[(size_t)n * T + i]);
      const double r0 = (double)g.x[i] - (double)gx0[i];
      mx.r = fmax(mx.r, fmax(fabs(s), fabs(r0)));
      if (KN) mx.k = fmax(mx.k, absQ + 1.0);
      mx.w = fmax(mx.w, fmax(fabs(xT), fabs((double)g.lam[(size_t)n * T + i])));
      mx.b = fmax(mx.b, fmax(fabs((double)g.q[(size_t)n * T + i]), fabs((double)gx0[i])));
      if (out.q) {
        out.put(out.q, (size_t)n * T + i, -s);
        out.put(out.x0, i, r0);
      }
    }
  }
  __shared__ double red[5][kKktWarps];
  const double rm = warp_max(mx.r), km = warp_max(mx.k), wm = warp_max(mx.w), bm = warp_max(mx.b);
  cost = warp_sum(cost);
  if (lane == 0) {
    red[0][warp] = rm; red[1][warp] = km; red[2][warp] = wm; red[3][warp] = bm; red[4][warp] = cost;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a[5] = {0, 0, 0, 0, 0};
    for (int w = 0; w < kKktWarps; ++w) {
      for (int k = 0; k < 4; ++k) a[k] = fmax(a[k], red[k][w]);
      a[4] += red[4][w];
    }
    atomic_max_nonneg(acc + RS_RNORM, a[0]);
    atomic_max_nonneg(acc + RS_KNORM, a[1]);
    atomic_max_nonneg(acc + RS_WNORM, a[2]);
    atomic_max_nonneg(acc + RS_BNORM, a[3]);
    acc[RS_COUNT + blockIdx.x] = a[4];
  }
}

// The refinement pass for FP64 data in double-FP32 arithmetic (kkt_stage_df):
// the stages as in kkt_residual_stream_kernel, without the |KKT| row sums; the
// terminal and initial rows (O(n^2) once) in FP64.
template <int NC>
__global__ void __launch_bounds__(kKktBlock, NC >= 4 ? 3 : 4)  // 80 / 64 registers, no spills
    kkt_residual_df_kernel(ProbDesc pd, double* acc, KktOut out, const int* skip, int gate) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (skip && *(volatile const int*)skip) return;
  if (gate && (((volatile const int*)skip)[2] == 0) != (gate == 1)) return;  // not this iteration's form
  if (*(volatile int*)pd.status != 0) return;
  const int n = pd.n, T = pd.T;
  KktData<double> g;
  g.x = static_cast<const double*>(pd.x);
  g.u = static_cast<const double*>(pd.u);
  g.lam = static_cast<const double*>(pd.lam);
  g.A = static_cast<const double*>(pd.A);
  g.B = static_cast<const double*>(pd.B);
  g.c = static_cast<const double*>(pd.c);
  g.Q = static_cast<const double*>(pd.Q);
  g.R = static_cast<const double*>(pd.R);
  g.S = static_cast<const double*>(pd.S);
  g.q = static_cast<const double*>(pd.q);
  g.r = static_cast<const double*>(pd.r);
  g.n = pd.n;
  g.m = pd.m;
  const double* gx0 = static_cast<const double*>(pd.x0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* sm = reinterpret_cast<double*>(smem);
  KktMax mx;
  double cost = 0.0;
  for (int t = blockIdx.x; t < T; t += gridDim.x) cost += kkt_stage_df<NC>(g, t, sm, mx, out);
  if (blockIdx.x == 0) {
    const double* QT = g.Q + (size_t)n * n * T;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double s = g.q[(size_t)n * T + i] + g.lam[(size_t)n * T + i];
      double qx = 0.0;
      for (int k = 0; k < n; ++k) {
        s = fma(0.5 * (QT[(size_t)i * n + k] + QT[(size_t)k * n + i]), g.x[(size_t)n * T + k], s);
        qx = fma(QT[(size_t)i * n + k], g.x[(size_t)n * T + k], qx);
      }
      const double xT = g.x[(size_t)n * T + i];
      cost += xT * (0.5 * qx + g.q[(size_t)n * T + i]);
      const double r0 = g.x[i] - gx0[i];
      mx.r = fmax(mx.r, fmax(fabs(s), fabs(r0)));
      mx.w = fmax(mx.w, fmax(fabs(xT), fabs(g.lam[(size_t)n * T + i])));
      mx.b = fmax(mx.b, fmax(fabs(g.q[(size_t)n * T + i]), fabs(gx0[i])));
      if (out.q) {
        out.put(out.q, (size_t)n * T + i, -s);
        out.put(out.x0, i, r0);
      }
    }
  }
  __shared__ double red[4][kKktWarps];
  const double rm = warp_max(mx.r), wm = warp_max(mx.w), bm = warp_max(mx.b);
  cost = warp_sum(cost);
  if (lane == 0) {
    red[0][warp] = rm; red[1][warp] = wm; red[2][warp] = bm; red[3][warp] = cost;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a[4] = {0, 0, 0, 0};
    for (int w = 0; w < kKktWarps; ++w) {
      for (int k = 0; k < 3; ++k) a[k] = fmax(a[k], red[k][w]);
      a[3] += red[3][w];
    }
    atomic_max_nonneg(acc + RS_RNORM, a[0]);
    atomic_max_nonneg(acc + RS_WNORM, a[1]);
    atomic_max_nonneg(acc + RS_BNORM, a[2]);
    acc[RS_COUNT + blockIdx.x] = a[3];
  }
}

// Turns the accumulators into eta, rel and the cost; decides convergence.
// report: [0] cost, [1] eta, [2] rel, [3] refinement iterations applied.
// cost: the sum of the per-block objective partial sums of the pass.
__device__ void finalize_body(ProbDesc pd, double* acc, double cost, double tol, int* skip, int is_final,
                              int check_convergence) {
  if (*(volatile int*)pd.status != 0) return;
  // already converged: the solution has not changed since the pass that found
  // it converged, whose numbers stand (the final pass was skipped as well)
  if (skip && *skip) return;
  const double r = acc[RS_RNORM], k = acc[RS_KNORM], w = acc[RS_WNORM], bn = acc[RS_BNORM];
  const double eta = r / (k * w + bn);
  const double rel = bn > 0.0 ? r / bn : r;
  pd.report[0] = cost;
  pd.report[1] = eta;
  pd.report[2] = rel;
  if (!isfinite(eta) || !isfinite(cost)) raise_status(pd.status, LQR_ERR_NONFINITE, -1);
  if (skip && !is_final && rel <= tol) *skip = 1;
  if (is_final && check_convergence && !(rel <= tol)) raise_status(pd.status, LQR_ERR_NO_CONVERGENCE, -1);
  // ready for the next pass; |KKT|_inf, a function of the data, stays until the final pass
  for (int i = 0; i < RS_COUNT; ++i)
    if (i != RS_KNORM || is_final) acc[i] = 0.0;
}

// In the refinement loop of a graph (loop: max iterations > 0): skip[2] counts
// the iterations and the loop's condition is set to continue while the
// solution has not converged, no error was raised and the count is below the
// maximum.
__global__ void residual_finalize_kernel(ProbDesc pd, double* acc, int nblocks, double tol, int* skip,
                                         int is_final, int check_convergence, int loop,
                                         cudaGraphConditionalHandle cond) {
  // the objective's block partial sums over the warp's lanes (one dependent
  // FP64 add per 32 blocks instead of one per block)
  double cost = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += 32) cost += acc[RS_COUNT + b];
  cost = kkt_warp_sum(cost);
  if (threadIdx.x != 0) return;
  finalize_body(pd, acc, cost, tol, skip, is_final, check_convergence);
  if (loop > 0) {
    const int it = skip[2] + 1;
    skip[2] = it;
    const bool go = skip[0] == 0 && *(volatile int*)pd.status == 0 && it < loop;
    cudaGraphSetConditional(cond, go ? 1u : 0u);
  }
}

// w <- w - delta for the outputs the correction solve refreshed.
template <typename TS>
__global__ void refine_update_kernel(ProbDesc pd, const double* dk, const double* dx, const double* du,
                                     const double* dl, const double* dp, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  if (*(volatile int*)pd.status != 0) return;
  const int n = pd.n, m = pd.m, T = pd.T;
  const size_t nx = (size_t)(T + 1) * n, nu = (size_t)T * m;
  TS* k = static_cast<TS*>(pd.k);
  TS* x = static_cast<TS*>(pd.x);
  TS* u = static_cast<TS*>(pd.u);
  TS* l = static_cast<TS*>(pd.lam);
  TS* p = static_cast<TS*>(pd.p);
  // x, lambda, p have (T+1) n entries and u, k have T m: either may be the longer
  const size_t ne = nx > nu ? nx : nu;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < ne; e += (size_t)gridDim.x * blockDim.x) {
    if (e < nx) {
      if (x) x[e] = static_cast<TS>((double)x[e] - dx[e]);
      if (l) l[e] = static_cast<TS>((double)l[e] - dl[e]);
      if (p) p[e] = static_cast<TS>((double)p[e] - dp[e]);
    }
    if (e < nu) {
      if (u) u[e] = static_cast<TS>((double)u[e] - du[e]);
      if (k) k[e] = static_cast<TS>((double)k[e] - dk[e]);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) pd.report[3] += 1.0;
}

int residual_grid(int T) {
  int g = 4 * device_sm_count();
  if (g > kMaxResidBlocks) g = kMaxResidBlocks;
  return T < g ? T : g;
}

template <typename TS>
cudaError_t launch_kkt_residual(const ProbDesc& pd, double* acc, const KktOut& out, const int* skip, cudaStream_t st,
                                int knorm, int df) {
  // by default the refinement passes (correction vectors requested) skip the |KKT| row sums
  const int want_knorm = knorm >= 0 ? knorm : (out.q == nullptr) ? 1 : 0;
  const int nc = kkt_stage_cols(pd.n, pd.m);
  const bool df_ok = nc > 0 && sizeof(TS) == 8 && !want_knorm && out.q;
  // df = 3 (a graph's loop body): both forms, gated on the iteration count skip[2]
  const int gate_df = (df == 3 && df_ok && skip) ? 1 : 0, gate_fp64 = gate_df ? 2 : 0;
  if (df && df_ok) {
    const size_t bytes = sizeof(double) * kkt_stage_df_smem_doubles(pd.n, pd.m);
    const int g = residual_grid(pd.T);
    if (nc == 1)
      kkt_residual_df_kernel<1><<<g, kKktBlock, bytes, st>>>(pd, acc, out, skip, gate_df);
    else if (nc == 2)
      kkt_residual_df_kernel<2><<<g, kKktBlock, bytes, st>>>(pd, acc, out, skip, gate_df);
    else
      kkt_residual_df_kernel<4><<<g, kKktBlock, bytes, st>>>(pd, acc, out, skip, gate_df);
    if (!gate_df) return cudaGetLastError();
  }
  if (nc > 0) {
    const size_t base = sizeof(double) * kkt_stage_smem_doubles(pd.n, pd.m);  // <= 45056 B at n = m = 128
    // the |KKT| pass stages Q_t and R_t in shared memory for their symmetric row sums
    const size_t bytes = want_knorm ? base + sizeof(double) * kkt_stash_doubles(pd.n, pd.m) : base;
    const int g = residual_grid(pd.T);
#define LQR_RES_LAUNCH(NC, KN)                                                                               \
  do {                                                                                                       \
    if (bytes > 48 * 1024 && cudaFuncSetAttribute(kkt_residual_stream_kernel<NC, KN, TS>,                     \
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize,              \
                                                  (int)bytes) != cudaSuccess)                                \
      return cudaGetLastError();                                                                             \
    kkt_residual_stream_kernel<NC, KN, TS><<<g, kKktBlock, bytes, st>>>(pd, acc, out, skip, KN, gate_fp64); \
  } while (0)
    if (nc == 1) {
      if (want_knorm) LQR_RES_LAUNCH(1, true); else LQR_RES_LAUNCH(1, false);
    } else if (nc == 2) {
      if (want_knorm) LQR_RES_LAUNCH(2, true); else LQR_RES_LAUNCH(2, false);
    } else {
      if (want_knorm) LQR_RES_LAUNCH(4, true); else LQR_RES_LAUNCH(4, false);
    }
#undef LQR_RES_LAUNCH
    return cudaGetLastError();
  }
  const size_t bytes = sizeof(double) * (6 * (size_t)pd.n + 3 * (size_t)pd.m);
  kkt_residual_kernel<TS><<<residual_grid(pd.T), kBlock, bytes, st>>>(pd, acc, out, skip, want_knorm);
  return cudaGetLastError();
}

// |KKT|_inf of Eq. 3's matrix (the largest absolute row sum, Q and R read
// symmetrised) from the FP32 copy of the data, into the accumulators of the
// residual passes: per stage the x rows (|Q_sym| row + |S| column + 1 + |A|
// column), the u rows (|S| row + |R_sym| row + |B| column) and the dynamics
// rows (1 + |A| row + |B| row); the terminal rows (|Q_T,sym| row + 1) and the
// initial-condition rows (1). It depends on the data alone, so the mixed-
// precision refinement takes it once per solve, in FP32 (it only scales the
// reported backward error), instead of in an FP64 residual pass.
//
// A CTA takes stages blockIdx.x, blockIdx.x + gridDim.x, ...; each stage is a
// sequence of items (Q_t, A_t, B_t, S_t, R_t; Q_T alone for t = T), one matrix
// each, copied whole into a ring of S shared-memory slots (16-byte cp.async
// where aligned) S - 1 items ahead of the one being summed. Each row or column
// sum is one thread's loop: columns read down (consecutive threads, distinct
// banks), rows read from the thread's own diagonal on (thread i starts at
// column i mod C), and a symmetrised row i of Q pairs row i with column i.
template <int S>
__global__ void __launch_bounds__(256) kkt_norm_f32_kernel(ProbDesc pd, double* acc) {
  extern __shared__ __align__(16) float nsm[];
  if (*(volatile int*)pd.status != 0) return;
  const int n = pd.n, m = pd.m, T = pd.T, tid = threadIdx.x, nthr = blockDim.x;
  const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm = (size_t)m * m;
  const int slot = (int)((((nn > nm ? nn : nm) > mm ? (nn > nm ? nn : nm) : mm) + 3) & ~(size_t)3);
  const float* gA = static_cast<const float*>(pd.A);
  const float* gB = static_cast<const float*>(pd.B);
  const float* gQ = static_cast<const float*>(pd.Q);
  const float* gR = static_cast<const float*>(pd.R);
  const float* gS = static_cast<const float*>(pd.S);
  float* xr = nsm + S * slot;  // x rows
  float* dr = xr + n;          // dynamics rows
  float* ur = dr + n;          // u rows
  const int ipt = gS ? 5 : 4;  // items of a stage t < T
  const int nst = (T + 1 - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int last_t = (int)blockIdx.x + (nst - 1) * (int)gridDim.x;
  const int nitems = nst <= 0 ? 0 : (nst - 1) * ipt + (last_t == T ? 1 : ipt);
  // item k: stage t = blockIdx.x + (k / ipt) gridDim.x, matrix k % ipt (0 Q, 1 A, 2 B, 3 R, 4 S)
  auto item_src = [&](int k, int* rows, int* cols) -> const float* {
    const int t = (int)blockIdx.x + (k / ipt) * (int)gridDim.x, w = k % ipt;
    switch (w) {
      case 0: *rows = n; *cols = n; return gQ + nn * t;
      case 1: *rows = n; *cols = n; return gA + nn * t;
      case 2: *rows = n; *cols = m; return gB + nm * t;
      case 3: *rows = m; *cols = m; return gR + mm * t;
      default: *rows = m; *cols = n; return gS + nm * t;
    }
  };
  auto issue = [&](int k) {
    if (k < nitems) {
      int r, c;
      const float* src = item_src(k, &r, &c);
      cta_copy_async(nsm + (k % S) * slot, src, (long long)r * c);
    }
    cp_async_commit();
  };
  // |M| row sums (rotated start) into rows[], column sums into cols[] (either may be null)
  auto abs_sums = [&](const float* M, int R, int C, float* rows, float* cols) {
    const int nr = rows ? R : 0, tasks = nr + (cols ? C : 0);
    for (int x = tid; x < tasks; x += nthr) {
      float s = 0.0f;
      if (x < nr) {
        const float* row = M + x * C;
        int c = x % C;
        for (int l = 0; l < C; ++l) {
          s += fabsf(row[c]);
          c = c + 1 == C ? 0 : c + 1;
        }
        rows[x] += s;
      } else {
        const int j = x - nr;
        for (int i = 0; i < R; ++i) s += fabsf(M[i * C + j]);
        cols[j] += s;
      }
    }
  };
  // |(M + M')/2| row sums of a d x d block into rows[]
  auto sym_sums = [&](const float* M, int d, float* rows) {
    for (int i = tid; i < d; i += nthr) {
      float s = 0.0f;
      int c = i;
      for (int l = 0; l < d; ++l) {
        s += fabsf(0.5f * (M[i * d + c] + M[c * d + i]));
        c = c + 1 == d ? 0 : c + 1;
      }
      rows[i] += s;
    }
  };
  float kmax = 1.0f;  // the initial-condition rows
  for (int i = tid; i < n; i += nthr) xr[i] = dr[i] = 1.0f;
  for (int a = tid; a < m; a += nthr) ur[a] = 0.0f;
  for (int k = 0; k < S - 1; ++k) issue(k);
  for (int k = 0; k < nitems; ++k) {
    cp_async_wait<(S >= 2 ? S - 2 : 0)>();
    __syncthreads();  // item k in its slot; item k - 1 (and its slot) finished
    issue(k + S - 1);
    if (S == 1) {
      cp_async_wait<0>();
      __syncthreads();
    }
    const float* M = nsm + (k % S) * slot;
    const int w = k % ipt;
    if (w == 0) sym_sums(M, n, xr);
    else if (w == 1) abs_sums(M, n, n, dr, xr);
    else if (w == 2) abs_sums(M, n, m, dr, ur);
    else if (w == 3) sym_sums(M, m, ur);
    else abs_sums(M, m, n, ur, xr);
    const int t = (int)blockIdx.x + (k / ipt) * (int)gridDim.x;
    if (w == ipt - 1 || t == T) {  // the stage's last item
      __syncthreads();
      for (int i = tid; i < n; i += nthr) {
        kmax = fmaxf(kmax, t == T ? xr[i] : fmaxf(xr[i], dr[i]));
        xr[i] = dr[i] = 1.0f;
      }
      for (int a = tid; a < m; a += nthr) {
        if (t != T) kmax = fmaxf(kmax, ur[a]);
        ur[a] = 0.0f;
      }
    }
    if (S == 1) __syncthreads();  // the single slot is refilled at the next item
  }
  cp_async_wait<0>();
  __shared__ double red[32];
  const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
  const double v = warp_max((double)kmax);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (tid == 0) {
    double b = red[0];
    for (int w = 1; w < nw; ++w) b = fmax(b, red[w]);
    atomic_max_nonneg(acc + RS_KNORM, b);
  }
}

static size_t kkt_norm_slot_floats(int n, int m) {
  size_t s = (size_t)n * n;
  if ((size_t)n * m > s) s = (size_t)n * m;
  if ((size_t)m * m > s) s = (size_t)m * m;
  return (s + 3) & ~(size_t)3;
}

cudaError_t launch_kkt_norm_f32(const ProbDesc& pd, double* acc, cudaStream_t st) {
  const size_t slot = kkt_norm_slot_floats(pd.n, pd.m), vec = 2 * (size_t)pd.n + pd.m;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return cudaGetLastError();
  const size_t budget = (size_t)optin - 1024;
  const int g = residual_grid(pd.T + 1);
  for (int S = 3; S >= 1; --S) {
    const size_t bytes = sizeof(float) * (S * slot + vec);
    if (bytes > budget) continue;
    const void* f = S == 3 ? (const void*)kkt_norm_f32_kernel<3>
                           : S == 2 ? (const void*)kkt_norm_f32_kernel<2> : (const void*)kkt_norm_f32_kernel<1>;
    cudaError_t e = raise_dyn_smem(f, bytes);
    if (e != cudaSuccess) return e;
    if (S == 3) kkt_norm_f32_kernel<3><<<g, 256, bytes, st>>>(pd, acc);
    else if (S == 2) kkt_norm_f32_kernel<2><<<g, 256, bytes, st>>>(pd, acc);
    else kkt_norm_f32_kernel<1><<<g, 256, bytes, st>>>(pd, acc);
    return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_residual_finalize_loop(const ProbDesc& pd, double* acc, double tol, int* skip, int loop,
                                          cudaGraphConditionalHandle cond, cudaStream_t st) {
  residual_finalize_kernel<<<1, 32, 0, st>>>(pd, acc, residual_grid(pd.T), tol, skip, 0, 0, loop, cond);
  return cudaGetLastError();
}

cudaError_t launch_residual_finalize(const ProbDesc& pd, double* acc, double tol, int* skip, int is_final,
                                     int check, cudaStream_t st) {
  residual_finalize_kernel<<<1, 32, 0, st>>>(pd, acc, residual_grid(pd.T), tol, skip, is_final, check, 0,
                                             cudaGraphConditionalHandle{});
  return cudaGetLastError();
}

template <typename TS>
cudaError_t launch_refine_update(const ProbDesc& pd, const double* dk, const double* dx, const double* du,
                                 const double* dl, const double* dp, const int* skip, cudaStream_t st) {
  refine_update_kernel<TS><<<2 * device_sm_count(), 256, 0, st>>>(pd, dk, dx, du, dl, dp, skip);
  return cudaGetLastError();
}

template cudaError_t launch_kkt_residual<double>(const ProbDesc&, double*, const KktOut&, const int*, cudaStream_t,
                                                 int, int);
template cudaError_t launch_kkt_residual<float>(const ProbDesc&, double*, const KktOut&, const int*, cudaStream_t,
                                                int, int);
template cudaError_t launch_refine_update<double>(const ProbDesc&, const double*, const double*, const double*,
                                                  const double*, const double*, const int*, cudaStream_t);
template cudaError_t launch_refine_update<float>(const ProbDesc&, const double*, const double*, const double*,
                                                 const double*, const double*, const int*, cudaStream_t);

}  // namespace lqr
