// The trajectory-optimisation outer loop of Section I, whose subproblems are
// LQR problems: Gauss-Newton multiple-shooting SQP on the nonlinear tracking
// model
//   x_{t+1} = f(x_t, u_t) = A x_t + B u_t + beta tanh(C x_t),  x_0 = x_init,
//   J = sum_t 1/2 (x_t - xref_t)'Q (x_t - xref_t) + 1/2 u_t'R u_t
//       + 1/2 (x_T - xref_T)'Q_T (x_T - xref_T).
// Per iteration, at the iterate (x, u): the linearisation kernel writes the LQR
// subproblem in the step (dx, du) (A_t = A + beta diag(1 - tanh^2(C x_t)) C,
// c_t = f(x_t, u_t) - x_{t+1}, q_t = Q (x_t - xref_t), r_t = R u_t,
// dx_0 = x_init - x_0; B_t, Q_t, R_t are the model's, written once per
// call); the segment-parallel solver solves it; the merit kernel evaluates,
// for every candidate step length alpha at once, the objective and the l1 norm
// of the defects at (x + alpha dx, u + alpha du); the update kernel takes the
// step the host picked. All in FP64.
//
// The merit kernel uses that both are cheap in alpha once a stage's products
// are formed: with e = x_t - xref_t, J_t(alpha) = 1/2 (e'Qe + 2 alpha dx'Qe +
// alpha^2 dx'Q dx) + the same in u, and
//   f(x + alpha dx, u + alpha du) = (A x + B u) + alpha (A dx + B du) + beta tanh(C x + alpha C dx),
// so each stage forms six matrix-vector products once and every candidate
// costs O(n).
#include <cuda_runtime.h>

#include "lqr_internal.cuh"

namespace lqr {

namespace {

constexpr int kSqpBlock = 256;
constexpr int kSqpWarps = kSqpBlock / 32;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum (op 0) or max (op 1) of one value per thread; every thread gets it.
__device__ double block_reduce(double v, int op, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = op ? warp_max_d(v) : warp_sum_d(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = threadIdx.x < kSqpWarps ? red[threadIdx.x] : 0.0;
    r = op ? warp_max_d(r) : warp_sum_d(r);
    if (threadIdx.x == 0) red[kSqpWarps] = r;
  }
  __syncthreads();
  return red[kSqpWarps];
}

// y = M v for an r x c row-major matrix, one thread per row
__device__ __forceinline__ double row_dot(const double* M, int c, int i, const double* v) {
  double s = 0.0;
  for (int k = 0; k < c; ++k) s = fma(M[(size_t)i * c + k], v[k], s);
  return s;
}

}  // namespace

__global__ void sqp_fill_kernel(NlModelDev md, double* Bt, double* Qt, double* Rt) {
  const int n = md.n, m = md.m, T = md.T;
  const size_t nb = (size_t)T * n * m, nq = (size_t)(T + 1) * n * n, nr = (size_t)T * m * m;
  const size_t tot = nb + nq + nr;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    if (e < nb) {
      Bt[e] = md.B[e % ((size_t)n * m)];
    } else if (e < nb + nq) {
      const size_t f = e - nb, t = f / ((size_t)n * n);
      Qt[f] = (t < (size_t)T ? md.Q : md.QT)[f % ((size_t)n * n)];
    } else {
      const size_t f = e - nb - nq;
      Rt[f] = md.R[f % ((size_t)m * m)];
    }
  }
}

// One CTA per stage t = 0..T: the subproblem's stage data at the iterate.
__global__ void __launch_bounds__(kSqpBlock) sqp_linearize_kernel(NlModelDev md, const double* x, const double* u,
                                                                   double* At, double* c, double* q, double* r,
                                                                   double* dx0) {
  extern __shared__ __align__(16) double lsm[];
  const int n = md.n, m = md.m, T = md.T, t = blockIdx.x;
  double* xs = lsm;       // x_t
  double* us = xs + n;    // u_t
  double* sc = us + m;    // 1 - tanh^2(C x_t), then x_t - xref_t
  double* es = sc + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    xs[i] = x[(size_t)n * t + i];
    es[i] = xs[i] - md.xref[(size_t)n * t + i];
  }
  if (t < T)
    for (int k = threadIdx.x; k < m; k += blockDim.x) us[k] = u[(size_t)m * t + k];
  __syncthreads();
  if (t == T) {  // the terminal gradient
    for (int i = threadIdx.x; i < n; i += blockDim.x) q[(size_t)n * T + i] = row_dot(md.QT, n, i, es);
    return;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double th = tanh(row_dot(md.C, n, i, xs));
    const double f = row_dot(md.A, n, i, xs) + row_dot(md.B, m, i, us) + md.beta * th;
    c[(size_t)n * t + i] = f - x[(size_t)n * (t + 1) + i];
    q[(size_t)n * t + i] = row_dot(md.Q, n, i, es);
    sc[i] = md.beta * (1.0 - th * th);
    if (t == 0) dx0[i] = md.x0[i] - xs[i];
  }
  for (int k = threadIdx.x; k < m; k += blockDim.x) r[(size_t)m * t + k] = row_dot(md.R, m, k, us);
  __syncthreads();
  double* Ad = At + (size_t)n * n * t;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) Ad[e] = md.A[e] + sc[e / n] * md.C[e];
}

// One CTA per stage t = 0..T; writes part[t][0..kSqpOut): the objective and
// defect l1 norm of each candidate alpha, then g'd, max|lambda|, max|dx|,
// max|du|, max|x|, max|u| of the stage.
__global__ void __launch_bounds__(kSqpBlock) sqp_merit_kernel(NlModelDev md, const double* x, const double* u,
                                                               const double* dx, const double* du, const double* q,
                                                               const double* r, const double* lam, double* part) {
  extern __shared__ __align__(16) double msm[];
  __shared__ double red[kSqpWarps + 1];
  const int n = md.n, m = md.m, T = md.T, t = blockIdx.x;
  double* xs = msm;        // x_t
  double* dxs = xs + n;    // dx_t
  double* es = dxs + n;    // x_t - xref_t
  double* us = es + n;     // u_t
  double* dus = us + m;    // du_t
  double* base = dus + m;  // A x_t + B u_t - x_{t+1}
  double* lin = base + n;  // A dx_t + B du_t - dx_{t+1}
  double* cx = lin + n;    // C x_t
  double* cdx = cx + n;    // C dx_t
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    xs[i] = x[(size_t)n * t + i];
    dxs[i] = dx[(size_t)n * t + i];
    es[i] = xs[i] - md.xref[(size_t)n * t + i];
  }
  if (t < T)
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
      us[k] = u[(size_t)m * t + k];
      dus[k] = du[(size_t)m * t + k];
    }
  __syncthreads();
  const bool term = (t == T);
  const double* Qm = term ? md.QT : md.Q;
  // quadratic-form pieces and the stage's alpha-independent reductions
  double qee = 0.0, qde = 0.0, qdd = 0.0, gd = 0.0, lmax = 0.0, dmax = 0.0, xmax = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double qe = row_dot(Qm, n, i, es), qd = row_dot(Qm, n, i, dxs);
    qee = fma(es[i], qe, qee);
    qde = fma(dxs[i], qe, qde);
    qdd = fma(dxs[i], qd, qdd);
    gd = fma(q[(size_t)n * t + i], dxs[i], gd);
    lmax = fmax(lmax, fabs(lam[(size_t)n * t + i]));
    dmax = fmax(dmax, fabs(dxs[i]));
    xmax = fmax(xmax, fabs(xs[i]));
  }
  double ree = 0.0, rde = 0.0, rdd = 0.0, umax = 0.0, dumax = 0.0;
  if (!term)
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
      const double re = row_dot(md.R, m, k, us), rd = row_dot(md.R, m, k, dus);
      ree = fma(us[k], re, ree);
      rde = fma(dus[k], re, rde);
      rdd = fma(dus[k], rd, rdd);
      gd = fma(r[(size_t)m * t + k], dus[k], gd);
      umax = fmax(umax, fabs(us[k]));
      dumax = fmax(dumax, fabs(dus[k]));
    }
  const double Se = block_reduce(qee + ree, 0, red), Sd = block_reduce(qde + rde, 0, red),
               Sdd = block_reduce(qdd + rdd, 0, red);
  double* out = part + (size_t)t * kSqpOut;
  const double g_all = block_reduce(gd, 0, red);
  const double l_all = block_reduce(lmax, 1, red), dx_all = block_reduce(dmax, 1, red),
               du_all = block_reduce(dumax, 1, red), x_all = block_reduce(xmax, 1, red),
               u_all = block_reduce(umax, 1, red);
  // the defects of each candidate: the dynamics into stage t + 1 (t < T) and,
  // at t = 0, the initial condition; the stage's products formed once
  if (!term)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      base[i] = row_dot(md.A, n, i, xs) + row_dot(md.B, m, i, us) - x[(size_t)n * (t + 1) + i];
      lin[i] = row_dot(md.A, n, i, dxs) + row_dot(md.B, m, i, dus) - dx[(size_t)n * (t + 1) + i];
      cx[i] = row_dot(md.C, n, i, xs);
      cdx[i] = row_dot(md.C, n, i, dxs);
    }
  __syncthreads();
  for (int a = 0; a < kSqpCand; ++a) {
    const double al = sqp_alpha(a);
    double d = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if (!term) d += fabs(base[i] + al * lin[i] + md.beta * tanh(cx[i] + al * cdx[i]));
      if (t == 0) d += fabs(xs[i] + al * dxs[i] - md.x0[i]);
    }
    const double D = block_reduce(d, 0, red);
    if (threadIdx.x == 0) {
      out[a] = 0.5 * (Se + 2.0 * al * Sd + al * al * Sdd);
      out[kSqpCand + a] = D;
    }
  }
  if (threadIdx.x == 0) {
    out[2 * kSqpCand + 0] = g_all;
    out[2 * kSqpCand + 1] = l_all;
    out[2 * kSqpCand + 2] = dx_all;
    out[2 * kSqpCand + 3] = du_all;
    out[2 * kSqpCand + 4] = x_all;
    out[2 * kSqpCand + 5] = u_all;
  }
}

// res[j] = sum over stages (j < 2 kSqpCand + 1) or max over stages (the rest)
// of part[.][j], one warp per output, each lane a fixed stride of stages.
__global__ void sqp_merit_final_kernel(const double* part, int nst, double* res) {
  const int lane = threadIdx.x & 31, j = threadIdx.x >> 5;
  if (j >= kSqpOut) return;
  const bool is_max = j > 2 * kSqpCand;
  double v = 0.0;
  for (int s = lane; s < nst; s += 32) {
    const double p = part[(size_t)s * kSqpOut + j];
    v = is_max ? fmax(v, p) : v + p;
  }
  v = is_max ? warp_max_d(v) : warp_sum_d(v);
  if (lane == 0) res[j] = v;
}

__global__ void sqp_update_kernel(double* x, double* u, const double* dx, const double* du, double alpha,
                                  long long nx, long long nu) {
  const long long ne = nx > nu ? nx : nu;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
    if (e < nx) x[e] += alpha * dx[e];
    if (e < nu) u[e] += alpha * du[e];
  }
}

cudaError_t launch_sqp_fill(const NlModelDev& md, double* Bt, double* Qt, double* Rt, cudaStream_t st) {
  sqp_fill_kernel<<<2 * device_sm_count(), 256, 0, st>>>(md, Bt, Qt, Rt);
  return cudaGetLastError();
}

cudaError_t launch_sqp_linearize(const NlModelDev& md, const double* x, const double* u, double* At, double* c,
                                 double* q, double* r, double* dx0, cudaStream_t st) {
  const size_t bytes = sizeof(double) * (3 * (size_t)md.n + md.m);
  sqp_linearize_kernel<<<md.T + 1, kSqpBlock, bytes, st>>>(md, x, u, At, c, q, r, dx0);
  return cudaGetLastError();
}

cudaError_t launch_sqp_merit(const NlModelDev& md, const double* x, const double* u, const double* dx,
                             const double* du, const double* q, const double* r, const double* lam, double* part,
                             double* res, cudaStream_t st) {
  const size_t bytes = sizeof(double) * (7 * (size_t)md.n + 2 * (size_t)md.m);
  sqp_merit_kernel<<<md.T + 1, kSqpBlock, bytes, st>>>(md, x, u, dx, du, q, r, lam, part);
  sqp_merit_final_kernel<<<1, 32 * kSqpOut, 0, st>>>(part, md.T + 1, res);
  return cudaGetLastError();
}

cudaError_t launch_sqp_update(double* x, double* u, const double* dx, const double* du, double alpha, long long nx,
                              long long nu, cudaStream_t st) {
  sqp_update_kernel<<<2 * device_sm_count(), 256, 0, st>>>(x, u, dx, du, alpha, nx, nu);
  return cudaGetLastError();
}

}  // namespace lqr
