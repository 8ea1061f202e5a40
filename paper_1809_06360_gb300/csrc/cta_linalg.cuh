// CTA-cooperative dense linear algebra on small row-major matrices held in
// shared or global memory (generic addressing). Every routine is executed by
// all threads of the block; routines do NOT end with a barrier unless stated,
// so independent routines can run back to back and the caller places the
// __syncthreads() that orders dependent phases.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace lqr {

// ---------------------------------------------------------------------------
// Matrix product with a per-element epilogue.
//   acc(i,j) = sum_k opA(i,k) * opB(k,j),  0 <= i < M, 0 <= j < N
//   opA(i,k) = TA ? A[k*lda + i] : A[i*lda + k]
//   opB(k,j) = TB ? B[j*ldb + k] : B[k*ldb + j]
// Each thread owns RM x RN output tiles; tiles are dealt round-robin over the
// block, consecutive threads take consecutive column tiles of one row tile.
// ---------------------------------------------------------------------------
template <int RM, int RN, bool TA, bool TB, typename Tacc, typename XA, typename XB, typename Epi>
__device__ __forceinline__ void cta_mm(int M, int N, int K, const XA* A, int lda,
                                       const XB* B, int ldb, Epi epi) {
  const int tm = (M + RM - 1) / RM, tn = (N + RN - 1) / RN;
  const int ntiles = tm * tn;
  for (int tile = threadIdx.x; tile < ntiles; tile += blockDim.x) {
    const int i0 = (tile / tn) * RM, j0 = (tile % tn) * RN;
    Tacc acc[RM][RN];
#pragma unroll
    for (int a = 0; a < RM; ++a)
#pragma unroll
      for (int b = 0; b < RN; ++b) acc[a][b] = Tacc(0);
    int ia[RM], jb[RN];
#pragma unroll
    for (int a = 0; a < RM; ++a) ia[a] = min(i0 + a, M - 1);  // clamp: rows past M are discarded
#pragma unroll
    for (int b = 0; b < RN; ++b) jb[b] = min(j0 + b, N - 1);
    for (int k = 0; k < K; ++k) {
      Tacc av[RM], bv[RN];
#pragma unroll
      for (int a = 0; a < RM; ++a)
        av[a] = static_cast<Tacc>(TA ? A[(size_t)k * lda + ia[a]] : A[(size_t)ia[a] * lda + k]);
#pragma unroll
      for (int b = 0; b < RN; ++b)
        bv[b] = static_cast<Tacc>(TB ? B[(size_t)jb[b] * ldb + k] : B[(size_t)k * ldb + jb[b]]);
#pragma unroll
      for (int a = 0; a < RM; ++a)
#pragma unroll
        for (int b = 0; b < RN; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < RM; ++a)
#pragma unroll
      for (int b = 0; b < RN; ++b)
        if (i0 + a < M && j0 + b < N) epi(i0 + a, j0 + b, acc[a][b]);
  }
}

// Picks the register tile from the output shape so that thin products still
// occupy the block: 4x4 when there are enough tiles, else 2x2, else 1x1.
template <bool TA, bool TB, typename Tacc, typename XA, typename XB, typename Epi>
__device__ __forceinline__ void cta_mm_auto(int M, int N, int K, const XA* A, int lda, const XB* B, int ldb, Epi epi) {
  const int nthr = blockDim.x;
  if (((M + 3) / 4) * ((N + 3) / 4) >= nthr / 2)
    cta_mm<4, 4, TA, TB, Tacc>(M, N, K, A, lda, B, ldb, epi);
  else if (((M + 1) / 2) * ((N + 1) / 2) >= nthr / 2)
    cta_mm<2, 2, TA, TB, Tacc>(M, N, K, A, lda, B, ldb, epi);
  else
    cta_mm<1, 1, TA, TB, Tacc>(M, N, K, A, lda, B, ldb, epi);
}

// --- epilogues --------------------------------------------------------------
template <typename XC>
struct EpiStore {  // C = alpha * acc
  XC* C; int ldc; double alpha;
  template <typename T>
  __device__ __forceinline__ void operator()(int i, int j, T v) const {
    C[(size_t)i * ldc + j] = static_cast<XC>(static_cast<T>(alpha) * v);
  }
};
template <typename XC>
struct EpiStoreT {  // C' = alpha * acc  (writes C[j][i])
  XC* C; int ldc; double alpha;
  template <typename T>
  __device__ __forceinline__ void operator()(int i, int j, T v) const {
    C[(size_t)j * ldc + i] = static_cast<XC>(static_cast<T>(alpha) * v);
  }
};
template <typename XC>
struct EpiAccum {  // C += alpha * acc
  XC* C; int ldc; double alpha;
  template <typename T>
  __device__ __forceinline__ void operator()(int i, int j, T v) const {
    XC* p = C + (size_t)i * ldc + j;
    *p = static_cast<XC>(static_cast<T>(*p) + static_cast<T>(alpha) * v);
  }
};
template <typename XC, typename XD>
struct EpiAdd {  // C = alpha * acc + D (D == nullptr means 0)
  XC* C; int ldc; double alpha; const XD* D; int ldd;
  template <typename T>
  __device__ __forceinline__ void operator()(int i, int j, T v) const {
    T d = D ? static_cast<T>(D[(size_t)i * ldd + j]) : T(0);
    C[(size_t)i * ldc + j] = static_cast<XC>(static_cast<T>(alpha) * v + d);
  }
};
template <typename XC, typename XD>
struct EpiAddSym {  // C = alpha * acc + (D + D')/2, D square with leading dimension ldd
  XC* C; int ldc; double alpha; const XD* D; int ldd;
  template <typename T>
  __device__ __forceinline__ void operator()(int i, int j, T v) const {
    T d = T(0.5) * (static_cast<T>(D[(size_t)i * ldd + j]) + static_cast<T>(D[(size_t)j * ldd + i]));
    C[(size_t)i * ldc + j] = static_cast<XC>(static_cast<T>(alpha) * v + d);
  }
};

// y[i] (op)= alpha * sum_k opA(i,k) x[k] ; one thread per output row.
template <bool TA, typename Tacc, typename XA, typename XX, typename Epi>
__device__ __forceinline__ void cta_mv(int M, int K, const XA* A, int lda,
                                       const XX* x, int incx, Epi epi) {
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    Tacc acc = Tacc(0);
    for (int k = 0; k < K; ++k)
      acc = fma(static_cast<Tacc>(TA ? A[(size_t)k * lda + i] : A[(size_t)i * lda + k]),
                static_cast<Tacc>(x[(size_t)k * incx]), acc);
    epi(i, 0, acc);
  }
}

// FP64 reciprocal for the serial pivot chain. On GB300 every FP64 warp
// instruction holds the sub-partition's FP64 pipe for 64 cycles and a library
// FP64 division costs ~430 cycles, so the pivot reciprocal is taken from the
// FP32 hardware reciprocal and refined by two Newton-Raphson steps
// y <- y + y (1 - d y), each of which doubles the number of correct bits
// (24 -> 48 -> full FP64). Outside the FP32 exponent range the division is used.
__device__ __forceinline__ double rcp_newton(double d) {
  const double ad = fabs(d);
  if (!(ad > 1e-30 && ad < 1e30)) return 1.0 / d;
  double y = (double)__frcp_rn((float)d);
  double e = fma(-d, y, 1.0);
  y = fma(y, e, y);
  e = fma(-d, y, 1.0);
  return fma(y, e, y);
}

// ---------------------------------------------------------------------------
// In-place lower Cholesky (FP64) of the d x d SPD matrix G (leading dim ld),
// computed as LDL' so that the serial pivot chain needs one reciprocal per
// column and no square root; the square roots that turn L D L' into the
// Cholesky factor are taken afterwards for all columns at once.
// One barrier per column: in step j every thread applies the rank-1 update of
// column j (still unscaled: A[i][k] -= A[i][j] A[k][j] / D_j) to the trailing
// elements it owns, and scales column j-1 by 1/D_{j-1} (unit lower L), which
// nobody reads in step j. Thread t owns row (t >> 2) + j + 1 + 64 r and the
// columns k = t (mod 4) of that row. The thread that writes the final value of
// the next pivot D_{j+1} also computes its reciprocal.
// On exit rdiag[j] = 1 / L[j][j] (if rdiag is non-null). `flag` (shared) is
// set to 1 when a pivot is not positive. `piv` (shared) holds d doubles of
// scratch. Ends with a barrier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ldl_pivot_prep(double v, int j, double* inv, int* flag) {
  const bool ok = (v > 0.0) && isfinite(v);
  if (!ok) *flag = 1;
  inv[j] = ok ? rcp_newton(v) : 0.0;
}

__device__ inline void cta_chol_piv(int d, double* G, int ld, int* flag, double* piv, double* rdiag) {
  const int t = threadIdx.x;
  const int nthr = blockDim.x;
  double* inv = piv;           // 1 / D_j                     (d)
  double* lc0 = piv + d;       // L[:, j] for even j          (d)
  double* lc1 = piv + 2 * d;   // L[:, j] for odd j           (d)
  double* gc = piv + 3 * d;    // unscaled column j, contiguous (bank-conflict-free reads)
  if (t == 0) ldl_pivot_prep(G[0], 0, inv, flag);
  __syncthreads();
  for (int j = 0; j < d; ++j) {
    double* lc = (j & 1) ? lc1 : lc0;
    const double* lp = (j & 1) ? lc0 : lc1;
    // (a) column j copied to contiguous scratch, its scaled form l_ij = a_ij / D_j,
    // and column j-1 written back as unit L
    const double invj = inv[j];
    for (int i = j + 1 + t; i < d; i += nthr) {
      const double g = G[(size_t)i * ld + j];
      gc[i] = g;
      lc[i] = g * invj;
    }
    if (j > 0)
      for (int i = j + t; i < d; i += nthr) G[(size_t)i * ld + (j - 1)] = lp[i];
    __syncthreads();
    // (b) trailing update of the lower triangle, elements dealt flat over the
    // block so that every FP64 warp instruction carries full lanes; element 0
    // is the next pivot, whose owner (thread 0) prepares its reciprocal first
    const int w = d - j - 1;
    const int ne = w * (w + 1) / 2;
    for (int e = t; e < ne; e += nthr) {
      int ii = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
      while ((ii + 1) * (ii + 2) / 2 <= e) ++ii;
      while (ii * (ii + 1) / 2 > e) --ii;
      const int kk = e - ii * (ii + 1) / 2;
      const int i = j + 1 + ii, k = j + 1 + kk;
      const double v = G[(size_t)i * ld + k] - lc[i] * gc[k];
      G[(size_t)i * ld + k] = v;
      if (e == 0) ldl_pivot_prep(v, j + 1, inv, flag);
    }
    __syncthreads();
  }
  // L D L' -> Cholesky: column j times sqrt(D_j); one square root per column,
  // all columns at once (off the pivot chain)
  double* sq = lc0;  // the scaled-column scratch is free now
  double* isq = lc1;
  for (int j = t; j < d; j += nthr) {
    const double Dj = G[(size_t)j * ld + j];
    const double r = (Dj > 0.0) ? rsqrt(Dj) : 1.0;
    isq[j] = r;
    sq[j] = (Dj > 0.0) ? Dj * r : 1.0;
  }
  __syncthreads();
  for (int e = t; e < d * d; e += nthr) {
    const int i = e / d, j = e % d;
    if (j > i) continue;
    G[(size_t)i * ld + j] = (i == j) ? sq[j] : G[(size_t)i * ld + j] * sq[j];
  }
  if (rdiag)
    for (int j = t; j < d; j += nthr) rdiag[j] = isq[j];
  __syncthreads();
}

// Convenience wrapper with static scratch (d <= 256); rdiag may be null.
__device__ inline void cta_chol(int d, double* G, int ld, int* flag, double* rdiag = nullptr) {
  __shared__ double s_piv[4 * 256];
  cta_chol_piv(d, G, ld, flag, s_piv, rdiag);
}

// ---------------------------------------------------------------------------
// FP32 Cholesky of the d x d SPD matrix G in place (lower), same column
// scheme as the FP64 one but with the FP32 hardware reciprocal square root on
// the pivot chain: one pivot per barrier, full-lane trailing updates.
// rdiag[j] = 1 / L[j][j]. `piv` (shared) holds d floats. Ends with a barrier.
// ---------------------------------------------------------------------------
__device__ inline void cta_chol_f32(int d, float* G, int ld, int* flag, float* piv, float* rdiag) {
  // piv: 2d floats: [0, d) reciprocal square roots of the pivots, [d, 2d) the
  // current scaled column (contiguous, bank-conflict-free reads)
  const int t = threadIdx.x;
  const int nthr = blockDim.x;
  float* lc = piv + d;
  if (t == 0) {
    const float v = G[0];
    const bool ok = (v > 0.0f) && isfinite(v);
    if (!ok) *flag = 1;
    const float r = ok ? rsqrtf(v) : 1.0f;
    piv[0] = r;
    G[0] = ok ? v * r : 1.0f;
  }
  __syncthreads();
  for (int j = 0; j < d; ++j) {
    const float r = piv[j];
    for (int i = j + 1 + t; i < d; i += nthr) {
      const float l = G[(size_t)i * ld + j] * r;
      G[(size_t)i * ld + j] = l;
      lc[i] = l;
    }
    __syncthreads();
    const int w = d - j - 1;
    const int ne = w * (w + 1) / 2;
    for (int e = t; e < ne; e += nthr) {
      int ii = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
      while ((ii + 1) * (ii + 2) / 2 <= e) ++ii;
      while (ii * (ii + 1) / 2 > e) --ii;
      const int kk = e - ii * (ii + 1) / 2;
      const int i = j + 1 + ii, k = j + 1 + kk;
      const float v = G[(size_t)i * ld + k] - lc[i] * lc[k];
      G[(size_t)i * ld + k] = v;
      if (e == 0) {  // the next pivot, by its only writer
        const bool ok = (v > 0.0f) && isfinite(v);
        if (!ok) *flag = 1;
        const float rr = ok ? rsqrtf(v) : 1.0f;
        piv[j + 1] = rr;
        G[(size_t)(j + 1) * ld + (j + 1)] = ok ? v * rr : 1.0f;
      }
    }
    __syncthreads();
  }
  if (rdiag)
    for (int j = t; j < d; j += nthr) rdiag[j] = piv[j];
  __syncthreads();
}

// Inverse of the lower-triangular d x d factor L (leading dim ldl, with
// rdiag[i] = 1 / L[i][i]) into X (lower, leading dim ldx; the strict upper
// part is set to zero). Column c of L^{-1} is the forward substitution of
// e_c; one thread per column. Ends with a barrier.
template <typename T>
__device__ inline void cta_trinv_lower(int d, const T* L, int ldl, const T* rdiag, T* X, int ldx) {
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) X[(size_t)(e / d) * ldx + (e % d)] = T(0);
  __syncthreads();
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    X[(size_t)c * ldx + c] = rdiag[c];
    for (int i = c + 1; i < d; ++i) {
      T s = T(0);
      for (int k = c; k < i; ++k) s = fma(L[(size_t)i * ldl + k], X[(size_t)k * ldx + c], s);
      X[(size_t)i * ldx + c] = -s * rdiag[i];
    }
  }
  __syncthreads();
}

// Triangular solves with few right-hand sides: one warp per column, the
// column-oriented elimination spread over the lanes.
template <typename XX, typename TL>
__device__ __forceinline__ void cta_trsm_lower_warp(int d, const TL* L, int ldl, int nc, XX* X, int ldx,
                                                    const TL* rdiag) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = warp; c < nc; c += nw) {
    for (int i = 0; i < d; ++i) {
      const TL xi = static_cast<TL>(X[(size_t)i * ldx + c]) * rdiag[i];
      __syncwarp();
      if (lane == 0) X[(size_t)i * ldx + c] = static_cast<XX>(xi);
      for (int k = i + 1 + lane; k < d; k += 32)
        X[(size_t)k * ldx + c] = static_cast<XX>(static_cast<TL>(X[(size_t)k * ldx + c]) - L[(size_t)k * ldl + i] * xi);
      __syncwarp();
    }
  }
}
template <typename XX, typename TL>
__device__ __forceinline__ void cta_trsm_lower_t_warp(int d, const TL* L, int ldl, int nc, XX* X, int ldx,
                                                      const TL* rdiag) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = warp; c < nc; c += nw) {
    for (int i = d - 1; i >= 0; --i) {
      const TL xi = static_cast<TL>(X[(size_t)i * ldx + c]) * rdiag[i];
      __syncwarp();
      if (lane == 0) X[(size_t)i * ldx + c] = static_cast<XX>(xi);
      for (int k = lane; k < i; k += 32)
        X[(size_t)k * ldx + c] = static_cast<XX>(static_cast<TL>(X[(size_t)k * ldx + c]) - L[(size_t)i * ldl + k] * xi);
      __syncwarp();
    }
  }
}

// Solve L Y = X in place (L lower d x d, leading dim ldl; X d x nc, leading dim
// ldx) with rdiag[i] = 1 / L[i][i]; arithmetic in Tacc. One thread per column.
// No barrier at the end.
template <typename Tacc, typename TL, typename XX>
__device__ __forceinline__ void cta_trsm_lower(int d, const TL* L, int ldl, const TL* rdiag, int nc, XX* X, int ldx) {
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    for (int i = 0; i < d; ++i) {
      Tacc t = static_cast<Tacc>(X[(size_t)i * ldx + c]);
      for (int k = 0; k < i; ++k) t -= static_cast<Tacc>(L[(size_t)i * ldl + k]) * static_cast<Tacc>(X[(size_t)k * ldx + c]);
      X[(size_t)i * ldx + c] = static_cast<XX>(t * static_cast<Tacc>(rdiag[i]));
    }
  }
}

// Solve L' Y = X in place (L lower), rdiag[i] = 1 / L[i][i]. No barrier.
template <typename Tacc, typename TL, typename XX>
__device__ __forceinline__ void cta_trsm_lower_t(int d, const TL* L, int ldl, const TL* rdiag, int nc, XX* X, int ldx) {
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    for (int i = d - 1; i >= 0; --i) {
      Tacc t = static_cast<Tacc>(X[(size_t)i * ldx + c]);
      for (int k = i + 1; k < d; ++k) t -= static_cast<Tacc>(L[(size_t)k * ldl + i]) * static_cast<Tacc>(X[(size_t)k * ldx + c]);
      X[(size_t)i * ldx + c] = static_cast<XX>(t * static_cast<Tacc>(rdiag[i]));
    }
  }
}

// Solve U Y = X in place (U upper d x d, row-major, leading dim ldu). No barrier.
__device__ __forceinline__ void cta_trsm_upper(int d, const double* U, int ldu, int nc, double* X, int ldx) {
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    for (int i = d - 1; i >= 0; --i) {
      double t = X[(size_t)i * ldx + c];
      for (int k = i + 1; k < d; ++k) t -= U[(size_t)i * ldu + k] * X[(size_t)k * ldx + c];
      X[(size_t)i * ldx + c] = t / U[(size_t)i * ldu + i];
    }
  }
}

// Solve U' Y = X in place (U upper, so U' is lower). No barrier.
__device__ __forceinline__ void cta_trsm_upper_t(int d, const double* U, int ldu, int nc, double* X, int ldx) {
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    for (int i = 0; i < d; ++i) {
      double t = X[(size_t)i * ldx + c];
      for (int k = 0; k < i; ++k) t -= U[(size_t)k * ldu + i] * X[(size_t)k * ldx + c];
      X[(size_t)i * ldx + c] = t / U[(size_t)i * ldu + i];
    }
  }
}

// ---------------------------------------------------------------------------
// Householder QR, FP64, in place on X (nr x nc, leading dim ld): reflects the
// first p columns (p <= nr, p <= nc) and applies every reflection to all
// columns to their right. On exit X[0:p,0:p] upper holds R, X[i][j] (i > j,
// j < p) holds the reflector tail, vhead[j] its head and beta[j] its scale,
// so that H_j = I - beta_j v_j v_j' and Q' X_in = H_{p-1} ... H_0 X_in.
// scal must point to 4 shared doubles. Ends with a barrier.
// ---------------------------------------------------------------------------
__device__ inline void cta_householder_qr(int nr, int nc, int p, double* X, int ld, double* vhead,
                                          double* beta, double* scal) {
  for (int j = 0; j < p; ++j) {
    if (threadIdx.x < 32) {
      double s = 0.0;
      for (int i = j + threadIdx.x; i < nr; i += 32) {
        const double v = X[(size_t)i * ld + j];
        s = fma(v, v, s);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (threadIdx.x == 0) {
        const double x0 = X[(size_t)j * ld + j];
        const double sigma = sqrt(s);
        if (sigma == 0.0) {
          scal[0] = 0.0;   // alpha
          beta[j] = 0.0;
          vhead[j] = 0.0;
        } else {
          const double alpha = x0 >= 0.0 ? -sigma : sigma;
          vhead[j] = x0 - alpha;
          beta[j] = 1.0 / (sigma * (sigma + fabs(x0)));
          scal[0] = alpha;
        }
      }
    }
    __syncthreads();
    const double bj = beta[j], v0 = vhead[j];
    for (int c = j + 1 + threadIdx.x; c < nc; c += blockDim.x) {
      double s = v0 * X[(size_t)j * ld + c];
      for (int i = j + 1; i < nr; ++i) s = fma(X[(size_t)i * ld + j], X[(size_t)i * ld + c], s);
      s *= bj;
      X[(size_t)j * ld + c] -= s * v0;
      for (int i = j + 1; i < nr; ++i) X[(size_t)i * ld + c] -= s * X[(size_t)i * ld + j];
    }
    __syncthreads();
    if (threadIdx.x == 0) X[(size_t)j * ld + j] = (bj == 0.0) ? X[(size_t)j * ld + j] : scal[0];
    __syncthreads();
  }
}

// Apply H_j (j = 0..p-1 in that order, i.e. Q') or in reverse order (i.e. Q)
// to the columns of Y (nr x nc, leading dim ldy), using reflectors stored by
// cta_householder_qr in V (leading dim ldv). Ends with a barrier.
__device__ inline void cta_householder_apply(int nr, int p, const double* V, int ldv, const double* vhead,
                                             const double* beta, int nc, double* Y, int ldy, bool transpose_q) {
  for (int jj = 0; jj < p; ++jj) {
    const int j = transpose_q ? jj : p - 1 - jj;
    const double bj = beta[j], v0 = vhead[j];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      double s = v0 * Y[(size_t)j * ldy + c];
      for (int i = j + 1; i < nr; ++i) s = fma(V[(size_t)i * ldv + j], Y[(size_t)i * ldy + c], s);
      s *= bj;
      Y[(size_t)j * ldy + c] -= s * v0;
      for (int i = j + 1; i < nr; ++i) Y[(size_t)i * ldy + c] -= s * V[(size_t)i * ldv + j];
    }
    __syncthreads();
  }
}

// Calls f(e, i, j) for e = threadIdx.x, threadIdx.x + blockDim.x, ... < rows *
// cols with (i, j) = (e / cols, e % cols): each thread steps its (i, j) by the
// block's quotient and remainder, one division per call instead of one per
// element (an integer division costs tens of instructions, a 64-bit one about a
// hundred).
template <typename F>
__device__ __forceinline__ void cta_for_rc(int rows, int cols, F f) {
  const int total = rows * cols, step = blockDim.x;
  const int dq = step / cols, dr = step - dq * cols;
  int i = threadIdx.x / cols, j = threadIdx.x - i * cols;
  for (int e = threadIdx.x; e < total; e += step) {
    f(e, i, j);
    i += dq;
    j += dr;
    if (j >= cols) {
      j -= cols;
      ++i;
    }
  }
}

// --- asynchronous global -> shared copies (cp.async, sm_80+) ----------------
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// cnt elements of T from global src to shared dst by all threads of the block
// (not committed): 16-byte copies when both ends are 16-byte aligned and the
// size is a multiple of 16 bytes, else one copy per element.
template <typename T>
__device__ __forceinline__ void cta_copy_async(T* dst, const T* src, long long cnt) {
  const bool v16 = (((reinterpret_cast<unsigned long long>(dst) | reinterpret_cast<unsigned long long>(src)) & 15) == 0) &&
                   ((cnt * (long long)sizeof(T)) % 16 == 0);
  if (v16) {
    constexpr int per = 16 / sizeof(T);
    const long long n16 = cnt / per;
    for (long long e = threadIdx.x; e < n16; e += blockDim.x) cp_async16(dst + e * per, src + e * per);
  } else {
    for (long long e = threadIdx.x; e < cnt; e += blockDim.x) {
      if (sizeof(T) == 8) cp_async8(dst + e, src + e);
      else cp_async4(dst + e, src + e);
    }
  }
}

__device__ __forceinline__ float rsqrt_pos(float v) { return rsqrtf(v); }
__device__ __forceinline__ double rsqrt_pos(double v) { return rsqrt(v); }

// Reciprocal of a pivot on a dependent chain.
__device__ __forceinline__ float recip_fast(float p) {
  // hardware approximation refined by one Newton-Raphson step r += r (1 - p r)
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(p));
  return fmaf(r, fmaf(-p, r, 1.0f), r);
}
__device__ __forceinline__ double recip_fast(double p) { return rcp_newton(p); }

// ---------------------------------------------------------------------------
// 4 x 4 block eliminations: d/4 pivot steps instead of d, each a rank-4
// update. Thread t owns the BR x BC register block (BC a multiple of 4, BR in
// {1, 2, 4}); the block grid must not exceed blockDim.x. Rows and columns
// past d are padding (zero; padded pivots are taken as 1).
// Per step: (a) the threads i < d4 invert the 4 x 4 pivot block in registers
// (redundantly) and form w_i = P^-1 c_i from the published pivot columns;
// (b) every owner applies the update and the owners of the next pivot
// columns publish them. Two barriers per step.
// Shared scratch: p4_scratch_floats(d) floats, 16-byte aligned.
// ---------------------------------------------------------------------------
__host__ __device__ inline int p4_scratch_floats(int d) {
  const int d4 = (d + 3) & ~3;
  return 16 * d4 + 16;
}

// Register-block shape for d on 512 threads: 0 = (1,4), 1 = (2,4), 2 = (4,4),
// 3 = (4,8) (block grid (d4/BR) x (d4/BC) <= 512 and both dividing d4), -1 = none.
__host__ __device__ inline int p4_shape(int d) {
  const int d4 = (d + 3) & ~3;
  if (d4 <= 32) return 0;
  if (d4 <= 64) return 1;
  if (d4 <= 88) return 2;
  if (d4 <= 128 && d4 % 8 == 0) return 3;
  return -1;
}

// In-register lower Cholesky factor L of the 4 x 4 SPD matrix m (row-major,
// lower triangle read) and Li = L^-1 (lower). bad |= a pivot that is not
// positive and finite.
template <typename T>
__device__ __forceinline__ void chol4(const T m[16], T L[16], T Li[16], bool& bad) {
  T rs[4];
#pragma unroll
  for (int e = 0; e < 16; ++e) L[e] = T(0);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    T dj = m[j * 4 + j];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < j) dj = fma(-L[j * 4 + k], L[j * 4 + k], dj);
    bad |= !(dj > T(0) && isfinite(dj));
    rs[j] = dj > T(0) ? rsqrt_pos(dj) : T(1);
    L[j * 4 + j] = dj > T(0) ? dj * rs[j] : T(1);
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (i > j) {
        T a = m[i * 4 + j];
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (k < j) a = fma(-L[i * 4 + k], L[j * 4 + k], a);
        L[i * 4 + j] = a * rs[j];
      }
  }
  // Li by forward substitution, 1/L_ii = rs[i]
#pragma unroll
  for (int e = 0; e < 16; ++e) Li[e] = T(0);
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (i < c) continue;
      T a = (i == c) ? T(1) : T(0);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k >= c && k < i) a = fma(-L[i * 4 + k], Li[k * 4 + c], a);
      Li[i * 4 + c] = a * rs[i];
    }
}

__device__ __forceinline__ float comp4(const float4& v, int r) {
  return r == 0 ? v.x : (r == 1 ? v.y : (r == 2 ? v.z : v.w));
}
__device__ __forceinline__ float dot4(const float4& a, const float4& b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}

// Inverse of the SPD matrix G in place; sym: the input is taken as (G + G')/2.
// Step J with the 4 x 4 pivot block P = L L': w_i = L^-1 c_i, u_i = L^-T w_i
// (= P^-1 c_i); a_ik -= w_i'w_k off the pivot rows and columns (symmetric),
// u_k / u_i on them, -P^-1 on the pivot block. *flag = 1 on a pivot block that
// is not positive definite.
template <int BR, int BC>
__device__ inline void cta_spd_inverse_p4(int d, float* G, int ld, int* flag, float* scr, bool sym) {
  static_assert(BC % 4 == 0 && (BR == 1 || BR == 2 || BR == 4), "block shape");
  const int t = threadIdx.x;
  const int d4 = (d + 3) & ~3;
  const int nbr = d4 / BR, nbc = d4 / BC;
  // row-fast mapping: the lanes of a warp share k0 and take consecutive row blocks
  // (broadcast loads of w_k, conflict-free loads of w_i and of the matrix)
  const bool own = t < nbr * nbc;
  const int i0 = own ? (t % nbr) * BR : 0, k0 = own ? (t / nbr) * BC : 0;
  float4* Cb = reinterpret_cast<float4*>(scr);  // 2 x d4: pivot columns, row i = (a_i,p0 .. a_i,p0+3)
  float4* Wb = Cb + 2 * d4;                     // d4: w_i
  float4* Ub = Wb + d4;                         // d4: u_i
  float4* Pn = reinterpret_cast<float4*>(scr + 16 * d4);  // 4 rows of -P^-1
  float v[BR][BC];
#pragma unroll
  for (int a = 0; a < BR; ++a)
#pragma unroll
    for (int b = 0; b < BC; ++b) {
      const int i = i0 + a, k = k0 + b;
      float g = 0.0f;
      if (own && i < d && k < d) {  // read transposed: symmetric in exact arithmetic
        g = G[(size_t)k * ld + i];
        if (sym) g = 0.5f * (g + G[(size_t)i * ld + k]);
      }
      v[a][b] = g;
    }
  if (own && k0 == 0)
#pragma unroll
    for (int a = 0; a < BR; ++a) Cb[i0 + a] = make_float4(v[a][0], v[a][1], v[a][2], v[a][3]);
  bool bad = false;
  __syncthreads();
  for (int J = 0; J < d4 / 4; ++J) {
    const int p0 = 4 * J;
    const float4* C = Cb + (J & 1) * d4;
    float4* Cn = Cb + ((J + 1) & 1) * d4;
    if (t < d4) {  // (a) the pivot factor (redundantly), w_t and u_t
      float m[16], L[16], Li[16];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float4 c = C[p0 + r];
        m[r * 4 + 0] = c.x; m[r * 4 + 1] = c.y; m[r * 4 + 2] = c.z; m[r * 4 + 3] = c.w;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (p0 + r >= d) {  // padded pivot: identity
#pragma unroll
          for (int q = 0; q < 4; ++q) { m[r * 4 + q] = 0.0f; m[q * 4 + r] = 0.0f; }
          m[r * 4 + r] = 1.0f;
        }
      bool b2 = false;
      chol4(m, L, Li, b2);
      const float4 c = C[t];
      float w[4], u[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k <= r; ++k) s = fmaf(Li[r * 4 + k], comp4(c, k), s);
        w[r] = s;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {  // u = Li' w
        float s = 0.0f;
#pragma unroll
        for (int k = r; k < 4; ++k) s = fmaf(Li[k * 4 + r], w[k], s);
        u[r] = s;
      }
      Wb[t] = make_float4(w[0], w[1], w[2], w[3]);
      Ub[t] = make_float4(u[0], u[1], u[2], u[3]);
      if (t == 0) {
        bad |= b2;
#pragma unroll
        for (int r = 0; r < 4; ++r) {  // rows of -P^-1 = -Li' Li
          float pr[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float s = 0.0f;
#pragma unroll
            for (int k = 0; k < 4; ++k) s = fmaf(Li[k * 4 + r], Li[k * 4 + q], s);
            pr[q] = -s;
          }
          Pn[r] = make_float4(pr[0], pr[1], pr[2], pr[3]);
        }
      }
    }
    __syncthreads();
    if (own) {  // (b) the update of the owned block
      float4 wk[BC];
#pragma unroll
      for (int b = 0; b < BC; ++b) wk[b] = Wb[k0 + b];
#pragma unroll
      for (int a = 0; a < BR; ++a) {
        const float4 wi = Wb[i0 + a];
#pragma unroll
        for (int b = 0; b < BC; ++b) v[a][b] -= dot4(wi, wk[b]);
      }
      // the pivot columns (u_i, or -P^-1 on the pivot rows) and the pivot rows (u_k)
      const int kJ = p0 - k0;
      if (kJ >= 0 && kJ < BC) {
#pragma unroll
        for (int a = 0; a < BR; ++a) {
          const int i = i0 + a;
          const float4 x = (i >= p0 && i < p0 + 4) ? Pn[i - p0] : Ub[i];
#pragma unroll
          for (int bq = 0; bq < BC / 4; ++bq)
            if (4 * bq == kJ) {
              v[a][4 * bq] = x.x; v[a][4 * bq + 1] = x.y; v[a][4 * bq + 2] = x.z; v[a][4 * bq + 3] = x.w;
            }
        }
      }
      if ((i0 <= p0 && p0 < i0 + BR) || (p0 <= i0 && i0 < p0 + 4)) {
#pragma unroll
        for (int a = 0; a < BR; ++a) {
          const int r = i0 + a - p0;
          if (r < 0 || r >= 4) continue;
#pragma unroll
          for (int b = 0; b < BC; ++b)
            if (k0 + b < p0 || k0 + b >= p0 + 4) v[a][b] = comp4(Ub[k0 + b], r);
        }
      }
      const int kN = p0 + 4 - k0;  // publish the next pivot columns
      if (kN >= 0 && kN < BC)
#pragma unroll
        for (int bq = 0; bq < BC / 4; ++bq)
          if (4 * bq == kN)
#pragma unroll
            for (int a = 0; a < BR; ++a)
              Cn[i0 + a] = make_float4(v[a][4 * bq], v[a][4 * bq + 1], v[a][4 * bq + 2], v[a][4 * bq + 3]);
    }
    __syncthreads();
  }
  if (__syncthreads_or(bad ? 1 : 0) && t == 0) *flag = 1;
  if (own)
#pragma unroll
    for (int a = 0; a < BR; ++a)
#pragma unroll
      for (int b = 0; b < BC; ++b) {
        const int i = i0 + a, k = k0 + b;
        if (i < d && k < d) G[(size_t)k * ld + i] = -v[a][b];  // the inverse is symmetric
      }
  __syncthreads();
}

// Lower Cholesky factor of the SPD matrix G in place (strict upper part set to
// zero) by 4 x 4 block elimination: step J factors the pivot block D_J = L_J L_J'
// and writes the final block column, L_J on the diagonal and w_i = L_J^-1 c_i
// below it; the trailing matrix is downdated by w_i'w_k (symmetric).
// rdiag[k] = 1 / L[k][k] if non-null. *flag = 1 on a non-SPD pivot block.
template <int BR, int BC>
__device__ inline void cta_chol_p4(int d, float* G, int ld, int* flag, float* scr, float* rdiag) {
  static_assert(BC % 4 == 0 && (BR == 1 || BR == 2 || BR == 4), "block shape");
  const int t = threadIdx.x;
  const int d4 = (d + 3) & ~3, nJ = d4 / 4;
  const int nbr = d4 / BR, nbc = d4 / BC;
  bool own = t < nbr * nbc;
  const int i0 = own ? (t / nbc) * BR : 0, k0 = own ? (t % nbc) * BC : 0;
  own = own && (i0 + BR - 1 >= k0);
  float4* Cb = reinterpret_cast<float4*>(scr);  // 2 x d4
  float4* Wb = Cb + 2 * d4;                     // d4
  float v[BR][BC];
#pragma unroll
  for (int a = 0; a < BR; ++a)
#pragma unroll
    for (int b = 0; b < BC; ++b) {
      const int i = i0 + a, k = k0 + b;
      float g = 0.0f;
      if (own && i < d && k < d) g = G[(size_t)(i >= k ? i : k) * ld + (i >= k ? k : i)];  // from the lower part
      if (i >= d && i == k) g = 1.0f;  // padded pivots
      v[a][b] = g;
    }
  if (own && k0 == 0)
#pragma unroll
    for (int a = 0; a < BR; ++a) Cb[i0 + a] = make_float4(v[a][0], v[a][1], v[a][2], v[a][3]);
  bool bad = false;
  __syncthreads();
  for (int J = 0; J < nJ; ++J) {
    const int p0 = 4 * J;
    const float4* C = Cb + (J & 1) * d4;
    float4* Cn = Cb + ((J + 1) & 1) * d4;
    if (t >= p0 && t < d4) {  // (a) the pivot factor (redundantly) and the final block column
      float m[16], L[16], Li[16];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float4 c = C[p0 + r];
        m[r * 4 + 0] = c.x; m[r * 4 + 1] = c.y; m[r * 4 + 2] = c.z; m[r * 4 + 3] = c.w;
      }
      bool b2 = false;
      chol4(m, L, Li, b2);
      if (t == p0) bad |= b2;
      float o[4];
      if (t >= p0 + 4) {
        const float4 c = C[t];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          float s = 0.0f;
#pragma unroll
          for (int k = 0; k <= r; ++k) s = fmaf(Li[r * 4 + k], comp4(c, k), s);
          o[r] = s;
        }
        Wb[t] = make_float4(o[0], o[1], o[2], o[3]);
      } else {
        float rd = 1.0f;
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (t - p0 == r) {
#pragma unroll
            for (int q = 0; q < 4; ++q) o[q] = L[r * 4 + q];
            rd = Li[r * 4 + r];
          }
        if (rdiag && t < d) rdiag[t] = rd;
      }
      if (t < d)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (p0 + q < d) G[(size_t)t * ld + p0 + q] = o[q];
    }
    __syncthreads();
    if (own && k0 + BC > p0 + 4) {  // (b) the trailing downdate
#pragma unroll
      for (int bq = 0; bq < BC / 4; ++bq) {
        const int kb = k0 + 4 * bq;
        if (kb < p0 + 4) continue;
        float4 wk[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) wk[q] = Wb[kb + q];
#pragma unroll
        for (int a = 0; a < BR; ++a) {
          if (i0 + a < kb) continue;
          const float4 wi = Wb[i0 + a];
#pragma unroll
          for (int q = 0; q < 4; ++q) v[a][4 * bq + q] -= dot4(wi, wk[q]);
        }
        if (kb == p0 + 4)
#pragma unroll
          for (int a = 0; a < BR; ++a)
            if (i0 + a >= kb) Cn[i0 + a] = make_float4(v[a][4 * bq], v[a][4 * bq + 1], v[a][4 * bq + 2], v[a][4 * bq + 3]);
      }
    }
    __syncthreads();
  }
  if (__syncthreads_or(bad ? 1 : 0) && t == 0) *flag = 1;
  for (int e = t; e < d * d; e += blockDim.x) {  // block columns right of the diagonal block
    const int i = e / d, k = e - i * d;
    if ((k >> 2) > (i >> 2)) G[(size_t)i * ld + k] = 0.0f;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Gauss-Jordan inverse of an SPD matrix by a group of threads (gtid < nthr)
// that synchronise through bar() (a named barrier), so that the rest of the
// block can work on something else meanwhile. Scalar pivots, one BR x BC
// register block per thread (row-fast mapping; (ceil(d/BR)) x (ceil(d/BC))
// blocks <= nthr), the pivot column and its reciprocal published by their
// owners. sym: the input is taken as (G + G')/2. colbuf: 2 dp floats, rpv: 2
// floats (shared), dp = max(BR ceil(d/BR), BC ceil(d/BC)). *flag = 1 on a
// pivot that is not positive and finite. Ends with bar().
// ---------------------------------------------------------------------------
template <int BR, int BC, typename Bar>
__device__ inline void grp_spd_inverse(int d, float* G, int ld, int* flag, float* colbuf, float* rpv, bool sym,
                                       int gtid, int nthr, Bar bar) {
  const int nbr = (d + BR - 1) / BR, nbc = (d + BC - 1) / BC;
  const int dp = (nbr * BR > nbc * BC) ? nbr * BR : nbc * BC;
  const bool own = gtid < nbr * nbc;
  const int i0 = own ? (gtid % nbr) * BR : 0, k0 = own ? (gtid / nbr) * BC : 0;
  float v[BR][BC];
#pragma unroll
  for (int a = 0; a < BR; ++a)
#pragma unroll
    for (int b = 0; b < BC; ++b) {
      const int i = i0 + a, k = k0 + b;
      float g = 0.0f;
      if (own && i < d && k < d) {
        g = G[(size_t)k * ld + i];
        if (sym) g = 0.5f * (g + G[(size_t)i * ld + k]);
      }
      v[a][b] = g;
    }
  for (int i = gtid; i < dp; i += nthr) {
    float g = 0.0f;
    if (i < d) {
      g = G[i];
      if (sym) g = 0.5f * (g + G[(size_t)i * ld]);
    }
    colbuf[i] = g;
    if (i == 0) rpv[0] = recip_fast(g);
  }
  bool bad = false;
  if (gtid == 0) {
    const float g = G[0];
    bad = !(g > 0.0f && isfinite(g));
  }
  bar();
  for (int j = 0; j < d; ++j) {
    const float* col = colbuf + (j & 1) * dp;
    float* nxt = colbuf + ((j + 1) & 1) * dp;
    if (own) {
      const float rp = rpv[j & 1];
      float ci[BR], ckr[BC];
#pragma unroll
      for (int a = 0; a < BR; ++a) ci[a] = col[i0 + a];
#pragma unroll
      for (int b = 0; b < BC; ++b) ckr[b] = col[k0 + b] * rp;
      // rank-1 update; the pivot row becomes a_jk / p, the pivot column a_ij / p
      // and the pivot -1/p (selects, no data-dependent branches)
#pragma unroll
      for (int a = 0; a < BR; ++a)
#pragma unroll
        for (int b = 0; b < BC; ++b) {
          const float upd = fmaf(-ci[a], ckr[b], v[a][b]);
          const bool ri = (i0 + a == j), cj = (k0 + b == j);
          v[a][b] = cj ? (ri ? -rp : ci[a] * rp) : (ri ? ckr[b] : upd);
        }
      const int bn = j + 1 - k0;  // publish the next pivot column
      if (bn >= 0 && bn < BC) {
#pragma unroll
        for (int b = 0; b < BC; ++b)
          if (b == bn)
#pragma unroll
            for (int a = 0; a < BR; ++a) {
              nxt[i0 + a] = v[a][b];
              if (i0 + a == j + 1 && j + 1 < d) {
                const float pn = v[a][b];
                bad |= !(pn > 0.0f && isfinite(pn));
                rpv[(j + 1) & 1] = recip_fast(pn);
              }
            }
      }
    }
    bar();
  }
  if (bad) *flag = 1;
  if (own)
#pragma unroll
    for (int a = 0; a < BR; ++a)
#pragma unroll
      for (int b = 0; b < BC; ++b) {
        const int i = i0 + a, k = k0 + b;
        if (i < d && k < d) G[(size_t)k * ld + i] = -v[a][b];
      }
  bar();
}

// Inverse of the SPD m x m matrix (G + G')/2 (m <= 32, row stride ld) in
// place by one warp: lane j holds column j in registers (rows and columns
// beyond m are the identity), Gauss-Jordan elimination without pivoting, the
// pivot column broadcast by shuffles; no shared-memory round trip or barrier
// on the pivot chain. The pivot loop stays rolled (a fully unrolled 32-pivot
// body is ~50 KB of straight-line code that one warp streams through the
// instruction cache, measured 10x slower): blocks of four pivots, after
// which the register column is rotated by four rows, so that pivot kb + u
// always sits in register u. *flag = 1 on a pivot that is not positive and
// finite. Only the calling warp takes part.
__device__ inline void warp_spd_inverse32(int m, float* G, int ld, int* flag) {
  constexpr int U = 4;
  const int lane = threadIdx.x & 31;
  float b[32];  // b[i] = row (kb + i) mod 32 of this lane's column at the start of block kb
#pragma unroll
  for (int i = 0; i < 32; ++i)
    b[i] = (i < m && lane < m) ? 0.5f * (G[i * ld + lane] + G[lane * ld + i]) : (i == lane ? 1.0f : 0.0f);
  bool bad = false;
#pragma unroll 1
  for (int kb = 0; kb < 32; kb += U) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = kb + u;
      const float d = __shfl_sync(0xffffffffu, b[u], k);
      bad |= !(d > 0.0f && isfinite(d));
      const float r = recip_fast(d);
      const bool piv = (lane == k);
      // column k becomes -a_ik / d (pivot 1/d), row k a_kj / d, the rest a_ij - a_ik a_kj / d
      const float f = piv ? r : b[u] * r;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        if (i == u) continue;
        const float ci = __shfl_sync(0xffffffffu, b[i], k);
        b[i] = fmaf(-ci, f, piv ? 0.0f : b[i]);
      }
      b[u] = f;
    }
    float t[U];
#pragma unroll
    for (int u = 0; u < U; ++u) t[u] = b[u];
#pragma unroll
    for (int i = 0; i < 32 - U; ++i) b[i] = b[i + U];
#pragma unroll
    for (int u = 0; u < U; ++u) b[32 - U + u] = t[u];
  }
  __syncwarp();  // every lane has read G before it is overwritten
  if (lane < m)
#pragma unroll
    for (int i = 0; i < 32; ++i)
      if (i < m) G[i * ld + lane] = b[i];
  if (bad && lane == 0) *flag = 1;
  __syncwarp();
}

// named barrier over the first nthr threads of the block (id > 0)
struct NamedBar {
  int id, nthr;
  __device__ __forceinline__ void operator()() const {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthr) : "memory");
  }
};

// FP32 product on 4-aligned shapes with 128-bit shared/global loads:
//   acc(i,j) = sum_k opA(i,k) B[k][j],  0 <= i < M, 0 <= j < N (M, N multiples of 4)
//   opA(i,k) = TA ? A[k*lda + i] : A[i*lda + k]
// A, B 16-byte aligned, lda and ldb multiples of 4. Padding rows/columns of
// the operands must hold zeros (or finite values whose products the epilogue
// discards). Each thread owns 4 x 4 output tiles; epi(i, j, v) for every
// element of the padded M x N range.
// rot: tile 0 goes to thread rot (mod blockDim.x), so that consecutive
// products of one phase can be dealt where the previous one left off.
// One 4 x 4 output tile at (i0, j0) of the product below (the shared body of
// the CTA and group forms, also usable with a caller's own tile order).
template <bool TA, typename Epi>
__device__ __forceinline__ void mm4f_tile(int i0, int j0, int K, const float* A, int lda, const float* B, int ldb,
                                          Epi epi) {
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
  int k = 0;
  if (!TA) {
    for (; k + 4 <= K; k += 4) {
      float4 av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = *reinterpret_cast<const float4*>(A + (size_t)(i0 + a) * lda + k);
#pragma unroll
      for (int q = 0; q < 4; ++q) bv[q] = *reinterpret_cast<const float4*>(B + (size_t)(k + q) * ldb + j0);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float ak[4] = {av[a].x, av[a].y, av[a].z, av[a].w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[a][0] = fmaf(ak[q], bv[q].x, acc[a][0]);
          acc[a][1] = fmaf(ak[q], bv[q].y, acc[a][1]);
          acc[a][2] = fmaf(ak[q], bv[q].z, acc[a][2]);
          acc[a][3] = fmaf(ak[q], bv[q].w, acc[a][3]);
        }
      }
    }
  }
  for (; k < K; ++k) {
    float ak[4];
    if (TA) {
      const float4 t4 = *reinterpret_cast<const float4*>(A + (size_t)k * lda + i0);
      ak[0] = t4.x; ak[1] = t4.y; ak[2] = t4.z; ak[3] = t4.w;
    } else {
#pragma unroll
      for (int a = 0; a < 4; ++a) ak[a] = A[(size_t)(i0 + a) * lda + k];
    }
    const float4 bv = *reinterpret_cast<const float4*>(B + (size_t)k * ldb + j0);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      acc[a][0] = fmaf(ak[a], bv.x, acc[a][0]);
      acc[a][1] = fmaf(ak[a], bv.y, acc[a][1]);
      acc[a][2] = fmaf(ak[a], bv.z, acc[a][2]);
      acc[a][3] = fmaf(ak[a], bv.w, acc[a][3]);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) epi(i0 + a, j0 + b, acc[a][b]);
}

// grp_mm4f: the same over a group of nthr threads, gtid the index in the group.
template <bool TA, typename Epi>
__device__ __forceinline__ void grp_mm4f(int gtid, int nthr, int M, int N, int K, const float* A, int lda,
                                         const float* B, int ldb, Epi epi, int rot = 0) {
  const int tm = M >> 2, tn = N >> 2;
  const int tid = (gtid + nthr - (rot % nthr)) % nthr;
  for (int tile = tid; tile < tm * tn; tile += nthr)
    mm4f_tile<TA>((tile / tn) << 2, (tile % tn) << 2, K, A, lda, B, ldb, epi);
}

template <bool TA, typename Epi>
__device__ __forceinline__ void cta_mm4f(int M, int N, int K, const float* A, int lda, const float* B, int ldb,
                                         Epi epi, int rot = 0) {
  grp_mm4f<TA>((int)threadIdx.x, (int)blockDim.x, M, N, K, A, lda, B, ldb, epi, rot);
}

// y_i = epi(i, sum_k A[i*lda + k] x[k]) for i < M: one warp per row, lanes
// stride k (conflict-free shared reads), shuffle reduction.
template <typename T, typename Epi>
__device__ __forceinline__ void cta_mv_warp(int M, int K, const T* A, int lda, const T* x, Epi epi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < M; i += nw) {
    T s = T(0);
    for (int k = lane; k < K; k += 32) s = fma(A[(size_t)i * lda + k], x[k], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) epi(i, s);
  }
}

}  // namespace lqr
