// The multipliers of every segment problem from the least-squares system of
// Section II-B ("Lagrange Multipliers"), at a given trajectory (x, u).
//
// Segment j (stages b .. e-1, L = e - b) is the problem of the
// constraint-explicit section: its first state fixed (multiplier lambda_0),
// the dynamics (lambda_1 .. lambda_L) and, for every segment but the last,
// its end state fixed (multiplier mu) with no terminal cost; the last segment
// carries the terminal cost and no end constraint. The stationarity rows
//   x rows:  lambda_i - A_t'lambda_{i+1} = g_i = -(Q_t x_t + S_t'u_t + q_t)
//   u rows:           -B_t'lambda_{i+1} = h_i = -(S_t x_t + R_t u_t + r_t)
//   end row: lambda_L (+ mu)             = g_L  (-(Q_T x_T + q_T), or 0)
// (t = b + i) form the paper's over-determined system A'lambda = b; its
// normal equations A A' lambda = A b are block tridiagonal in the unknown
// blocks lambda_0 .. lambda_L (, mu):
//   diagonal   D_0 = I,  D_i = I + A_t A_t' + B_t B_t' (t = b + i - 1, 1 <= i <= L),  D_mu = I
//   coupling   block (i, i-1) = -A_t (1 <= i <= L),  block (mu, L) = I
//   right side f_0 = g_0,  f_i = g_i - A_t g_{i-1} - B_t h_{i-1},  f_mu = g_L.
// One CTA per segment solves them by block Cholesky, D~_i = L_i L_i' with
// D~_i = D_i - C_i C_i', C_i = E_i L_{i-1}^-T (E_i the coupling block), the
// forward substitution y_i = L_i^-1 (f_i - C_i y_{i-1}) along the way, then the
// backward substitution lambda_i = L_i^-T (y_i - C_{i+1}' lambda_{i+1}).
// Arithmetic in FP64: the normal equations square the condition number of
// the stationarity system.
#include <cuda_runtime.h>

#include "cta_linalg.cuh"
#include "lqr_internal.cuh"

namespace lqr {

namespace {

constexpr int kLsBlock = 256;

// per block of the workspace: L_i, C_i' (n x n each), y_i, 1 / diag(L_i)
__host__ __device__ inline long long ls_block_doubles(int n) { return 2LL * n * n + 2LL * n; }

// g = -(Q_sym x + S'u + q), h = -(S x + R_sym u + r) at stage t (h only when m > 0)
__device__ void ls_stage_rhs(const LsArgs& a, int t, double* g, double* h) {
  const int n = a.n, m = a.m;
  const double* Q = a.Q + (size_t)n * n * t;
  const double* R = a.R + (size_t)m * m * t;
  const double* S = a.S ? a.S + (size_t)m * n * t : nullptr;
  const double* x = a.x + (size_t)n * t;
  const double* u = a.u + (size_t)m * t;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = a.q[(size_t)n * t + i];
    for (int k = 0; k < n; ++k) s = fma(0.5 * (Q[(size_t)i * n + k] + Q[(size_t)k * n + i]), x[k], s);
    if (S)
      for (int k = 0; k < m; ++k) s = fma(S[(size_t)k * n + i], u[k], s);
    g[i] = -s;
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double s = a.r[(size_t)m * t + i];
    for (int k = 0; k < m; ++k) s = fma(0.5 * (R[(size_t)i * m + k] + R[(size_t)k * m + i]), u[k], s);
    if (S)
      for (int k = 0; k < n; ++k) s = fma(S[(size_t)i * n + k], x[k], s);
    h[i] = -s;
  }
}

}  // namespace

size_t ls_mult_smem_bytes(int n, int m, int on_chip) {
  return sizeof(double) * ((on_chip ? 3 * (size_t)n * n : 0) + 6 * (size_t)n + 2 * (size_t)m);
}

long long ls_mult_scratch_doubles(int n, int T, int K) {
  int lmax = 0;
  for (int j = 0; j < K; ++j) {
    const int L = seg_begin(T, K, j + 1) - seg_begin(T, K, j);
    if (L > lmax) lmax = L;
  }
  return (long long)(lmax + 2) * ls_block_doubles(n);
}

__global__ void __launch_bounds__(kLsBlock) ls_mult_kernel(LsArgs a) {
  extern __shared__ __align__(16) double lsm[];
  __shared__ int s_flag;
  const int n = a.n, m = a.m, T = a.T, K = a.K, j = blockIdx.x;
  if (threadIdx.x == 0) s_flag = *(volatile int*)a.status;
  __syncthreads();
  if (s_flag) return;
  const int b = seg_begin(T, K, j), e = seg_begin(T, K, j + 1), L = e - b;
  const bool last = (j == K - 1);
  const int N = L + 1 + (last ? 0 : 1);
  const size_t nn = (size_t)n * n, nm = (size_t)n * m;
  const long long bd = ls_block_doubles(n);
  double* blk = a.scratch + (long long)j * a.scratch_per_seg;  // block i at blk + i * bd
  double* bufs = lsm;                                           // [Lprev | Dcur | Wt] when on chip
  double* vec = lsm + (a.on_chip ? 3 * nn : 0);
  double* gp = vec;          // g_{i-1}
  double* gc = gp + n;       // g_i
  double* f = gc + n;        // f_i, then y_i
  double* yp = f + n;        // y_{i-1}
  double* rdp = yp + n;      // 1 / diag(L_{i-1})
  double* rdc = rdp + n;     // 1 / diag(L_i)
  double* hp = rdc + n;      // h_{i-1}
  double* hc = hp + m;       // h_i

  const double* Lprev = nullptr;
  for (int i = 0; i < N; ++i) {
    double* Lg = blk + (long long)i * bd;  // this block's slots in the workspace
    double* Wg = Lg + nn;
    double* yg = Wg + nn;
    double* rg = yg + n;
    double* D = a.on_chip ? bufs + (size_t)((i & 1) ? nn : 0) : Lg;
    double* Wt = a.on_chip ? bufs + 2 * nn : Wg;
    const bool stage = (i >= 1 && i <= L);  // a dynamics block
    const int t = b + i - 1;
    // (1) g_i, h_i and the diagonal block D_i
    if (i < L) {
      ls_stage_rhs(a, b + i, gc, hc);
    } else if (i == L) {
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double s = 0.0;
        if (last) {
          const double* QT = a.Q + nn * T;
          s = a.q[(size_t)n * T + k];
          for (int c = 0; c < n; ++c) s = fma(0.5 * (QT[(size_t)k * n + c] + QT[(size_t)c * n + k]), a.x[(size_t)n * T + c], s);
        }
        gc[k] = -s;
      }
    }
    if (stage) {
      const double* At = a.A + nn * t;
      const double* Bt = a.B + nm * t;
      cta_mm<4, 4, false, true, double>(n, n, n, At, n, At, n, EpiStore<double>{D, n, 1.0});
      __syncthreads();
      if (m > 0) cta_mm<4, 4, false, true, double>(n, n, m, Bt, m, Bt, m, EpiAccum<double>{D, n, 1.0});
      // E' = -A_t' into Wt (the coupling block of lambda_i with lambda_{i-1})
      for (int x = threadIdx.x; x < n * n; x += blockDim.x) Wt[x] = -At[(size_t)(x % n) * n + x / n];
    } else {
      for (int x = threadIdx.x; x < n * n; x += blockDim.x) D[x] = 0.0;
      if (i > 0)  // the mu block: coupling I
        for (int x = threadIdx.x; x < n * n; x += blockDim.x) Wt[x] = (x / n == x % n) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) D[(size_t)k * n + k] += 1.0;
    // (2) the right side f_i
    if (i == 0) {
      for (int k = threadIdx.x; k < n; k += blockDim.x) f[k] = gc[k];
    } else if (stage) {
      const double* At = a.A + nn * t;
      const double* Bt = a.B + nm * t;
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double s = gc[k];
        for (int c = 0; c < n; ++c) s = fma(-At[(size_t)k * n + c], gp[c], s);
        for (int c = 0; c < m; ++c) s = fma(-Bt[(size_t)k * m + c], hp[c], s);
        f[k] = s;
      }
    } else {
      for (int k = threadIdx.x; k < n; k += blockDim.x) f[k] = gc[k];  // f_mu = g_L
    }
    __syncthreads();
    // (3) elimination of the coupling: Wt = L_{i-1}^-1 E' (= C_i'), D -= C_i C_i', f -= C_i y_{i-1}
    if (i > 0) {
      cta_trsm_lower_warp(n, Lprev, n, n, Wt, n, (const double*)rdp);
      __syncthreads();
      cta_mm<4, 4, true, false, double>(n, n, n, Wt, n, Wt, n, EpiAccum<double>{D, n, -1.0});
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < n; ++c) s = fma(Wt[(size_t)c * n + k], yp[c], s);
        f[k] -= s;
      }
      __syncthreads();
    }
    // (4) D~_i = L_i L_i', y_i = L_i^-1 f_i
    if (threadIdx.x == 0) s_flag = 0;
    __syncthreads();
    cta_chol(n, D, n, &s_flag, rdc);
    if (s_flag) {
      if (threadIdx.x == 0) raise_status(a.status, LQR_ERR_NOT_PD, b + i);
      return;
    }
    cta_trsm_lower_warp(n, (const double*)D, n, 1, f, 1, (const double*)rdc);
    __syncthreads();
    // keep the block for the backward substitution; roll the vectors
    if (a.on_chip) {
      for (int x = threadIdx.x; x < n * n; x += blockDim.x) Lg[x] = D[x];
      if (i > 0)
        for (int x = threadIdx.x; x < n * n; x += blockDim.x) Wg[x] = Wt[x];
    }
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      yg[k] = f[k];
      rg[k] = rdc[k];
      yp[k] = f[k];
      rdp[k] = rdc[k];
      gp[k] = gc[k];
    }
    for (int k = threadIdx.x; k < m; k += blockDim.x) hp[k] = hc[k];
    Lprev = D;
    __syncthreads();
  }
  // backward substitution: lambda_i = L_i^-T (y_i - C_{i+1}' lambda_{i+1})
  double* lam = f;   // lambda_{i+1}, then lambda_i
  double* tmp = gc;
  for (int i = N - 1; i >= 0; --i) {
    const double* Lg = blk + (long long)i * bd;
    const double* yg = Lg + 2 * nn;
    const double* rg = yg + n;
    if (i == N - 1) {
      for (int k = threadIdx.x; k < n; k += blockDim.x) tmp[k] = yg[k];
    } else {
      const double* Wn = blk + (long long)(i + 1) * bd + nn;  // C_{i+1}'
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double s = yg[k];
        for (int c = 0; c < n; ++c) s = fma(-Wn[(size_t)k * n + c], lam[c], s);
        tmp[k] = s;
      }
    }
    __syncthreads();
    cta_trsm_lower_t_warp(n, Lg, n, 1, tmp, 1, rg);
    __syncthreads();
    double* out = (i < L) ? a.lam + (size_t)n * (b + i)
                : (i == L) ? (last ? a.lam + (size_t)n * T : (a.lam_end ? a.lam_end + (size_t)n * j : nullptr))
                           : (a.mu ? a.mu + (size_t)n * j : nullptr);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      lam[k] = tmp[k];
      if (out) out[k] = tmp[k];
    }
    __syncthreads();
  }
}

cudaError_t launch_ls_mult(const LsArgs& a, cudaStream_t st) {
  const size_t bytes = ls_mult_smem_bytes(a.n, a.m, a.on_chip);
  cudaError_t e = raise_dyn_smem((const void*)ls_mult_kernel, bytes);
  if (e != cudaSuccess) return e;
  ls_mult_kernel<<<a.K, kLsBlock, bytes, st>>>(a);
  return cudaGetLastError();
}

}  // namespace lqr
