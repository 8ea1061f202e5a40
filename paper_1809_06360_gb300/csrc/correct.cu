// Step A8: refinement corrections that reuse the factorisation of the solve.
//
// A correction solves the LQR problem with the solve's matrices and new vector
// data (q~, r~, c~, x0~). With the solve's global policies K_t, value matrices
// P_t and the inverses M_uu,t^-1 = (R_t + B_t'P_{t+1}B_t)^-1 kept, it is an
// affine recursion in the vectors alone (the serial Riccati recursion of
// Section III-A with the matrices fixed):
//   s_t = P_{t+1} c~_t + p_{t+1},  g_u = r~_t + B_t's_t,  g_x = q~_t + A_t's_t
//   k~_t = -M_uu,t^-1 g_u,  p_t = g_x + K_t'g_u,  p_T = q~_T
//   u~_t = K_t x~_t + k~_t,  x~_{t+1} = A_t x~_t + B_t u~_t + c~_t,
//   lambda~_t = -(P_t x~_t + p_t).
// With the closed-loop matrices Phi_t = A_t + B_t K_t (formed once per solve)
// both recursions are one n x n matrix-vector product per stage:
//   p_t = Phi_t'p_{t+1} + e_t,      e_t = Phi_t'(P_{t+1} c~_t) + q~_t + K_t'r~_t
//   x~_{t+1} = Phi_t x~_t + w_t,    w_t = B_t k~_t + c~_t,
// and everything else (e_t; k~_t, w_t once p is known; u~_t, lambda~_t once x~
// is known) is independent across stages. The recursions split over the
// solve's K segments: with the segment map Psi_j = Phi_{e-1} ... Phi_b
// (b = b_j, e = b_{j+1}), p_b = Psi_j'p_e + eps_j and x~_e = Psi_j x~_b +
// delta_j, where eps_j (delta_j) is the segment's own pass started from p_e = 0
// (x~_b = 0). One correction is then:
//   e_t (all stages)  ->  eps_j (segment passes)  ->  backward link chain for p
//   at the boundaries  ->  p_t (segment passes)  ->  k~_t, w_t (all stages)  ->
//   delta_j (segment passes)  ->  forward link chain for x~ at the boundaries
//   ->  x~_t (segment passes)  ->  u~_t, lambda~_t (all stages),
// O(T (n^2 + nm)) work instead of the solve's O(T n^3). A link chain is the
// same kind of recursion over the K segment maps (two levels over groups of
// about sqrt(K) links when K is large). FP32 data and arithmetic (the
// corrections of the mixed FP32 mode, whose FP64 residual decides convergence).
//
// Every recursion runs in one kernel, corr_rec_kernel: one CTA per run of
// consecutive steps. A step's matrix and offset vector are stored as one block
// (n + 1 rows of stride ld, row n the offset vector; the per-stage kernels
// write the offsets into the blocks) and stream into a ring of shared-memory
// slots by one bulk asynchronous copy per step (cp.async.bulk, completion
// counted in bytes on an mbarrier per slot), up to slots - 1 steps ahead. The
// CTA is warp-specialised: one warp issues the copies, one waits for them, and
// eight warps compute, all meeting at one barrier per step. Both directions
// read the stored block by columns (M' y from M, M y from the stored
// transpose); each consumer warp owns corr_opw(n) outputs, and the 32 /
// corr_opw(n) lanes of one output sum interleaved rows (q, q + P, ...) that
// the row stride ld places in distinct banks, combined by shuffles. The
// independent per-stage work runs one warp per stage straight from global
// memory (coalesced rows; a row-wise product reduces across the warp by
// shuffles).
#include <cuda_runtime.h>
#include <stdint.h>

#include "cta_linalg.cuh"
#include "lqr_internal.cuh"
#include "tc_sm100.cuh"

namespace lqr {

namespace {

constexpr int kCorrBlock = 256;         // closed-loop and group maps
constexpr int kRecMaxSlots = 6;         // ring slots of the recursion kernel
constexpr int kRecConsumers = 8;        // computing warps of the recursion kernel
constexpr int kRecBlock = (kRecConsumers + 2) * 32;  // + the issuing and the waiting warp
constexpr int kParWarps = 8;            // per-stage kernels: warps per CTA, one stage per warp
constexpr long long kCorrSpin = 1LL << 25;  // polls of a stage-data wait (32 ns apart) before LQR_ERR_TIMEOUT

__device__ __forceinline__ bool corr_exit(const int* status, const int* skip, int* s_flag) {
  if (threadIdx.x == 0) *s_flag = (*(volatile const int*)status != 0) || (skip && *(volatile const int*)skip);
  __syncthreads();
  const bool ex = *s_flag != 0;
  __syncthreads();
  return ex;
}

// rows x cols floats (source row stride lds) into shared memory with row stride ldd
__device__ __forceinline__ void copy_pad(float* dst, int ldd, const float* src, int lds, int rows, int cols) {
  cta_for_rc(rows, cols, [&](int, int i, int j) { cp_async4(dst + i * ldd + j, src + (long long)i * lds + j); });
}

}  // namespace

size_t corr_rec_smem_bytes(int n, int slots) {
  const size_t ld = (size_t)corr_ld(n);
  return sizeof(float) * ((size_t)slots * (n + 1) * ld + 2 * ld);
}
size_t corr_psi_smem_bytes(int n, int m, int psi_global) {
  const size_t N = (n + 3) & ~3, M = (m + 3) & ~3;
  return sizeof(float) * (3 * N * (N + 4) + (psi_global ? 0 : N * (M + 4) + M * (N + 4)));
}
size_t corr_group_smem_bytes(int n) {
  const size_t N = (n + 3) & ~3;
  return sizeof(float) * 3 * N * (N + 4);
}
static size_t corr_par_smem_bytes(int n, int m) {
  const int v = corr_ld(n > m ? n : m);
  return sizeof(float) * (size_t)kParWarps * 4 * v;
}
void corr_plan(int n, int m, long long smem_budget, int* slots, int* psi_global) {
  *slots = 0;
  *psi_global = 0;
  if ((long long)corr_psi_smem_bytes(n, m, 0) > smem_budget) {
    // B_t, K_t straight from global memory: float4 rows need n, m multiples of 4
    if (n % 4 != 0 || m % 4 != 0 || (long long)corr_psi_smem_bytes(n, m, 1) > smem_budget) return;
    *psi_global = 1;
  }
  if ((long long)corr_par_smem_bytes(n, m) > smem_budget) return;
  for (int s = kRecMaxSlots; s >= 2; --s)
    if ((long long)corr_rec_smem_bytes(n, s) <= smem_budget) {
      *slots = s;
      return;
    }
}

// ---------------------------------------------------------------------------
// Once per solve: Phi_t = A_t + B_t K_t (written for every stage) and
// Psi_j = Phi_{e-1} ... Phi_b. One CTA per segment, the two products of a stage
// on 4 x 4 register tiles (n, m padded to multiples of 4 with zeros; row
// strides N + 4, M + 4), A_t staged in the free Psi buffer. Both are stored,
// with their transposes, as rows 0..n-1 of blocks of stride ld (zero padding).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kCorrBlock) corr_psi_kernel(CorrArgs a) {
  extern __shared__ __align__(16) float csm[];
  __shared__ int s_flag;
  if (corr_exit(a.status, a.skip, &s_flag)) return;
  const int n = a.n, m = a.m, j = blockIdx.x;
  const int b = seg_begin(a.T, a.nseg, j), e = seg_begin(a.T, a.nseg, j + 1);
  const int N = (n + 3) & ~3, M = (m + 3) & ~3, LD = N + 4, LDm = M + 4;
  float* X = csm;            // Psi so far
  float* Y = X + N * LD;     // free: A_t, then Phi_t Psi
  float* Phi = Y + N * LD;
  float* Bs = Phi + N * LD;  // N x LDm (unless read from global memory)
  float* Ks = Bs + N * LDm;  // M x LD
  const int total = 3 * N * LD + (a.psi_global ? 0 : N * LDm + M * LD);
  for (int x = threadIdx.x; x < total; x += blockDim.x) csm[x] = 0.0f;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) X[i * LD + i] = 1.0f;
  const int ld = corr_ld(n);
  const long long nn = (long long)n * n, nm = (long long)n * m, blk = (long long)(n + 1) * ld;
  for (int t = b; t < e; ++t) {
    copy_pad(Y, LD, a.A + nn * t, n, n, n);
    if (!a.psi_global) {
      copy_pad(Bs, LDm, a.B + nm * t, m, n, m);
      copy_pad(Ks, LD, a.K + nm * t, n, m, n);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();  // stage data in; the previous stage's products are finished
    auto phi = [&](int i, int l, float v) { Phi[i * LD + l] = (i < n && l < n) ? v + Y[i * LD + l] : 0.0f; };
    if (a.psi_global)  // n, m multiples of 4: the unpadded rows of B_t and K_t
      cta_mm4f<false>(N, N, M, a.B + nm * t, m, a.K + nm * t, n, phi);
    else
      cta_mm4f<false>(N, N, M, Bs, LDm, Ks, LD, phi);
    __syncthreads();
    float* gPhi = a.Phit + blk * t;
    float* gPhiT = a.PhiTt + blk * t;
    cta_for_rc(n, ld, [&](int x, int i, int l) {
      gPhi[x] = l < n ? Phi[i * LD + l] : 0.0f;
      gPhiT[x] = l < n ? Phi[l * LD + i] : 0.0f;
    });
    cta_mm4f<false>(N, N, N, Phi, LD, X, LD, [&](int i, int l, float v) { Y[i * LD + l] = v; });
    __syncthreads();
    float* tmp = X;
    X = Y;
    Y = tmp;
  }
  float* gPsi = a.Psi + blk * j;
  float* gPsiT = a.PsiT + blk * j;
  cta_for_rc(n, ld, [&](int x, int i, int l) {
    gPsi[x] = l < n ? X[i * LD + l] : 0.0f;
    gPsiT[x] = l < n ? X[l * LD + i] : 0.0f;
  });
}

// Theta_g = Psi_{hi-1} ... Psi_lo per group of links (once per solve): one CTA
// per group, products on 4 x 4 register tiles (row stride N + 4); stored like Psi.
__global__ void __launch_bounds__(kCorrBlock) corr_group_maps_kernel(CorrArgs a) {
  extern __shared__ __align__(16) float csm[];
  __shared__ int s_flag;
  if (corr_exit(a.status, a.skip, &s_flag)) return;
  const int n = a.n, K = a.nseg, G = a.G;
  const int g = blockIdx.x;
  const int lo = g * G, hi = (lo + G < K) ? lo + G : K;
  const int N = (n + 3) & ~3, LD = N + 4;
  float* X = csm;  // product so far
  float* Y = X + N * LD;
  float* M = Y + N * LD;  // Psi_j
  for (int x = threadIdx.x; x < 3 * N * LD; x += blockDim.x) csm[x] = 0.0f;
  __syncthreads();
  const int ld = corr_ld(n);
  const long long blk = (long long)(n + 1) * ld;
  copy_pad(X, LD, a.Psi + blk * lo, ld, n, n);
  cp_async_commit();
  for (int j = lo + 1; j < hi; ++j) {
    copy_pad(M, LD, a.Psi + blk * j, ld, n, n);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    cta_mm4f<false>(N, N, N, M, LD, X, LD, [&](int i, int l, float val) { Y[i * LD + l] = val; });
    __syncthreads();
    float* tmp = X;
    X = Y;
    Y = tmp;
  }
  cp_async_wait<0>();
  __syncthreads();
  float* gT = a.Theta + blk * g;
  float* gTT = a.ThetaT + blk * g;
  cta_for_rc(n, ld, [&](int x, int i, int l) {
    gT[x] = l < n ? X[i * LD + l] : 0.0f;
    gTT[x] = l < n ? X[l * LD + i] : 0.0f;
  });
}

// ---------------------------------------------------------------------------
// The recursion y <- M_k'y + o_k (dir 0, k descending) or y <- M_k y + o_k
// (dir 1, k ascending) over runs of consecutive k, one run per CTA:
// run j = [jG, min(count, jG + G)) when G > 0, else segment j of a nruns-way
// split of count. Block k at C + cstride k holds, read by columns, M_k (dir 0)
// or the transpose of M_k (dir 1) in rows 0..n-1 and o_k in row n (stride ld,
// 16-byte aligned). The start value of run j is y0[y0stride (j + 1)] (dir 0) or
// y0[y0stride j] (dir 1), zero when y0 is null. Outputs: `all` (nullable) gets,
// dir 0, the value after step k at all[k] and, from the last run, its start
// value at all[hi]; dir 1, the value before step k at all[k] and, from the last
// run, its final value at all[hi]. `end` (nullable) gets run j's final value at
// end[estride j].
// ---------------------------------------------------------------------------
struct RecArgs {
  const float* C;
  long long cstride;
  const float* y0;
  long long y0stride;
  float* all;
  long long astride;
  float* end;
  long long estride;
  int n, ld, count, nruns, G, slots;
  long long spin;  // polls of a copy wait (0: kCorrSpin)
  const int* skip;
  int* status;
};

__global__ void __launch_bounds__(kRecBlock) corr_rec_kernel(RecArgs a, int dir) {
  extern __shared__ __align__(16) float csm[];
  __shared__ __align__(8) uint64_t s_bar[kRecMaxSlots];
  __shared__ int s_flag, s_fail;  // s_fail: 1 + the step whose copy did not arrive
  if (corr_exit(a.status, a.skip, &s_flag)) return;
  const int n = a.n, ld = a.ld, j = blockIdx.x, S = a.slots, tid = threadIdx.x, nthr = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31;
  int lo, hi;
  if (a.G > 0) {
    lo = j * a.G;
    hi = lo + a.G < a.count ? lo + a.G : a.count;
  } else {
    lo = seg_begin(a.count, a.nruns, j);
    hi = seg_begin(a.count, a.nruns, j + 1);
  }
  const int cnt = hi > lo ? hi - lo : 0;
  const bool last = j == a.nruns - 1;
  const int slot_f = (n + 1) * ld;
  const uint32_t bytes = (uint32_t)slot_f * 4u;
  float* ybuf = csm + S * slot_f;  // two value buffers: step idx reads ybuf[idx & 1]
  if (tid == 0) {
    for (int s = 0; s < S; ++s) tc::mbar_init(&s_bar[s], 1);
    tc::mbar_fence_init();
    s_fail = 0;
  }
  for (int e = tid; e < n; e += nthr)
    ybuf[e] = a.y0 ? a.y0[a.y0stride * (long long)(dir == 0 ? j + 1 : j) + e] : 0.0f;
  __syncthreads();
  if (dir == 0 && last && a.all)
    for (int e = tid; e < n; e += nthr) a.all[a.astride * hi + e] = ybuf[e];
  auto issue = [&](int idx, int sl) {  // one thread of the issuing warp
    const int k = dir == 0 ? hi - 1 - idx : lo + idx;
    tc::mbar_expect_tx(&s_bar[sl], bytes);
    tc::bulk_g2s(csm + sl * slot_f, a.C + a.cstride * k, bytes, &s_bar[sl]);
  };
  // Each step starts at a barrier of the whole CTA, after which: the consumers
  // have finished step idx - 1 (its slot may be refilled), the waiting warp has
  // seen step idx's copy complete (or set s_fail).
  if (warp == kRecConsumers) {  // issuing warp
    if (lane == 0)
      for (int idx = 0; idx < S - 1 && idx < cnt; ++idx) issue(idx, idx);
    int isl = S - 1;  // the slot of step idx + S - 1: that of step idx - 1
    for (int idx = 0; idx < cnt; ++idx) {
      __syncthreads();
      if (s_fail) break;
      if (lane == 0 && idx + S - 1 < cnt) issue(idx + S - 1, isl);
      if (++isl == S) isl = 0;
    }
  } else if (warp == kRecConsumers + 1) {  // waiting warp
    int s = 0;
    uint32_t par = 0u;
    for (int idx = 0; idx < cnt; ++idx) {
      int ok = 1;
      if (lane == 0) {
        ok = tc::mbar_wait(&s_bar[s], par, a.spin > 0 ? a.spin : kCorrSpin) ? 1 : 0;
        if (!ok) s_fail = idx + 1;
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      __syncthreads();
      if (!ok) break;
      if (++s == S) {
        s = 0;
        par ^= 1u;
      }
    }
  } else {  // consumers: warp w owns outputs w opw .. w opw + opw - 1
    const int opw = corr_opw(n), P = 32 / opw;
    const int q = lane / opw, i = warp * opw + (lane - q * opw);
    const bool act = i < n;
    int s = 0;
    for (int idx = 0; idx < cnt; ++idx) {
      __syncthreads();
      if (s_fail) break;
      const float* Cs = csm + s * slot_f;
      const float* yc = ybuf + (idx & 1) * ld;
      float* yx = ybuf + ((idx + 1) & 1) * ld;
      const int k = dir == 0 ? hi - 1 - idx : lo + idx;
      float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
      if (act) {
        const float* col = Cs + i;
        int l = q;
        for (; l + 3 * P < n; l += 4 * P) {
          s0 = fmaf(col[l * ld], yc[l], s0);
          s1 = fmaf(col[(l + P) * ld], yc[l + P], s1);
          s2 = fmaf(col[(l + 2 * P) * ld], yc[l + 2 * P], s2);
          s3 = fmaf(col[(l + 3 * P) * ld], yc[l + 3 * P], s3);
        }
        for (; l < n; l += P) s0 = fmaf(col[l * ld], yc[l], s0);
      }
      float sum = (s0 + s1) + (s2 + s3);
      for (int o = opw; o < 32; o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (act && q == 0) {
        const float v = sum + Cs[n * ld + i];
        yx[i] = v;
        if (a.all) a.all[a.astride * k + i] = dir == 0 ? v : yc[i];
      }
      if (++s == S) s = 0;
    }
  }
  __syncthreads();  // the last step's values written, or a failure seen by every warp
  if (s_fail) {
    // a copy that did not arrive (step s_fail - 1): report it, give the copies
    // still in flight (that step and up to S - 2 after it) one more bounded wait, stop
    if (tid == 0) {
      raise_status(a.status, LQR_ERR_TIMEOUT, -1);
      const int f = s_fail - 1;
      for (int p = f; p < f + S - 1 && p < cnt; ++p)
        tc::mbar_wait(&s_bar[p % S], (uint32_t)(p / S) & 1u, kCorrSpin);
    }
    return;
  }
  const float* yf = ybuf + (cnt & 1) * ld;
  if (a.end)
    for (int e = tid; e < n; e += nthr) a.end[a.estride * j + e] = yf[e];
  if (dir == 1 && last && a.all)
    for (int e = tid; e < n; e += nthr) a.all[a.astride * hi + e] = yf[e];
}

// ---------------------------------------------------------------------------
// Per-stage products from global memory, one warp each.
// ---------------------------------------------------------------------------
// float4 rows apply when the row length is 4 C4 floats with C4 a power of two
// up to 32 (32 / C4 rows per warp load) and the rows are 16-byte aligned
__device__ __forceinline__ int vec4_lanes(const float* M, int ldm, int len) {
  const int c4 = len >> 2;
  const bool ok = (len & 3) == 0 && c4 >= 1 && c4 <= 32 && (c4 & (c4 - 1)) == 0 && (ldm & 3) == 0 &&
                  (reinterpret_cast<unsigned long long>(M) & 15) == 0;
  return ok ? c4 : 0;
}

// out[i] += sum_{l < rows} M[l ldm + i] v[l] for i < cols: lanes over i
// (coalesced rows of M). With float4 rows, lane (r, c) reads columns 4c..4c+3
// of rows r, r + 32/C4, ..., eight rows in flight, and the row groups are
// summed by shuffles.
__device__ __forceinline__ void warp_colmv(const float* __restrict__ M, int ldm, int rows, int cols,
                                           const float* v, float* out) {
  const int lane = threadIdx.x & 31;
  const int c4 = vec4_lanes(M, ldm, cols);
  if (c4) {
    const int rp = 32 / c4, r = lane / c4, c = lane - r * c4;
    float ax = 0.0f, ay = 0.0f, az = 0.0f, aw = 0.0f;
    const float* p = M + 4 * c;
    int l = r;
    for (; l + 7 * rp < rows; l += 8 * rp) {
      float4 m4[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) m4[u] = __ldg(reinterpret_cast<const float4*>(p + (long long)(l + u * rp) * ldm));
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float vl = v[l + u * rp];
        ax = fmaf(m4[u].x, vl, ax);
        ay = fmaf(m4[u].y, vl, ay);
        az = fmaf(m4[u].z, vl, az);
        aw = fmaf(m4[u].w, vl, aw);
      }
    }
    for (; l < rows; l += rp) {
      const float4 m = __ldg(reinterpret_cast<const float4*>(p + (long long)l * ldm));
      const float vl = v[l];
      ax = fmaf(m.x, vl, ax);
      ay = fmaf(m.y, vl, ay);
      az = fmaf(m.z, vl, az);
      aw = fmaf(m.w, vl, aw);
    }
    for (int o = c4; o < 32; o <<= 1) {
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
      az += __shfl_xor_sync(0xffffffffu, az, o);
      aw += __shfl_xor_sync(0xffffffffu, aw, o);
    }
    if (r == 0) {
      out[4 * c] += ax;
      out[4 * c + 1] += ay;
      out[4 * c + 2] += az;
      out[4 * c + 3] += aw;
    }
    return;
  }
  for (int i = lane; i < cols; i += 32) {
    const float* p = M + i;
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
    int l = 0;
#pragma unroll 2
    for (; l + 4 <= rows; l += 4) {
      const float m0 = __ldg(p + (long long)l * ldm), m1 = __ldg(p + (long long)(l + 1) * ldm);
      const float m2 = __ldg(p + (long long)(l + 2) * ldm), m3 = __ldg(p + (long long)(l + 3) * ldm);
      s0 = fmaf(m0, v[l], s0);
      s1 = fmaf(m1, v[l + 1], s1);
      s2 = fmaf(m2, v[l + 2], s2);
      s3 = fmaf(m3, v[l + 3], s3);
    }
    for (; l < rows; ++l) s0 = fmaf(__ldg(p + (long long)l * ldm), v[l], s0);
    out[i] += (s0 + s1) + (s2 + s3);
  }
}

// out[i] += sum_{l < cols} M[i ldm + l] v[l] for i < rows. With float4 rows,
// lane (r, c) takes columns 4c..4c+3 of rows r, r + 32/C4, ... (four row groups
// in flight), the C4 lanes of a row summed by shuffles; otherwise lanes over l,
// four rows at a time, shuffle reductions.
__device__ __forceinline__ void warp_rowmv(const float* __restrict__ M, int ldm, int rows, int cols,
                                           const float* v, float* out) {
  const int lane = threadIdx.x & 31;
  const int c4 = vec4_lanes(M, ldm, cols);
  if (c4) {
    const int rp = 32 / c4, r = lane / c4, c = lane - r * c4;
    const float4 v4 = *reinterpret_cast<const float4*>(v + 4 * c);
    const float* p = M + 4 * c;
    for (int i0 = 0; i0 < rows; i0 += 4 * rp) {
      float d[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int row = i0 + u * rp + r;
        d[u] = 0.0f;
        if (row < rows) {
          const float4 m = __ldg(reinterpret_cast<const float4*>(p + (long long)row * ldm));
          d[u] = fmaf(m.x, v4.x, fmaf(m.y, v4.y, fmaf(m.z, v4.z, m.w * v4.w)));
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        for (int o = 1; o < c4; o <<= 1) d[u] += __shfl_xor_sync(0xffffffffu, d[u], o);
        const int row = i0 + u * rp + r;
        if (c == 0 && row < rows) out[row] += d[u];
      }
    }
    return;
  }
  for (int i = 0; i < rows; i += 4) {
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
    const float* r0 = M + (long long)i * ldm;
    for (int l = lane; l < cols; l += 32) {
      const float vl = v[l];
      s0 = fmaf(__ldg(r0 + l), vl, s0);
      if (i + 1 < rows) s1 = fmaf(__ldg(r0 + ldm + l), vl, s1);
      if (i + 2 < rows) s2 = fmaf(__ldg(r0 + 2 * (long long)ldm + l), vl, s2);
      if (i + 3 < rows) s3 = fmaf(__ldg(r0 + 3 * (long long)ldm + l), vl, s3);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      s3 += __shfl_xor_sync(0xffffffffu, s3, o);
    }
    if (lane < 4 && i + lane < rows) out[i + lane] += lane == 0 ? s0 : lane == 1 ? s1 : lane == 2 ? s2 : s3;
  }
}

__device__ __forceinline__ void warp_load(float* dst, const float* src, int cnt) {
  for (int i = threadIdx.x & 31; i < cnt; i += 32) dst[i] = src ? src[i] : 0.0f;
}

// e_t = Phi_t'(P_{t+1} c~_t) + q~_t + K_t'r~_t (into row n of Phi_t's block) and
// Pc_t = P_{t+1} c~_t, t < T
__global__ void __launch_bounds__(kParWarps * 32) corr_rhs_kernel(CorrArgs a) {
  extern __shared__ __align__(16) float psm[];
  __shared__ int s_flag;
  if (corr_exit(a.status, a.skip, &s_flag)) return;
  const int n = a.n, m = a.m, ld = corr_ld(n), v = corr_ld(n > m ? n : m), w = threadIdx.x >> 5;
  const int t = blockIdx.x * kParWarps + w;
  if (t >= a.T) return;
  float* c = psm + w * 4 * v;
  float* pc = c + v;
  float* r = pc + v;
  float* e = r + v;
  const long long nn = (long long)n * n, nm = (long long)n * m;
  warp_load(c, a.cc + (long long)n * t, n);
  warp_load(r, a.cr + (long long)m * t, m);
  warp_load(pc, nullptr, n);
  warp_load(e, a.cq + (long long)n * t, n);
  __syncwarp();
  warp_colmv(a.P + nn * (t + 1), n, n, n, c, pc);  // P symmetric: column i is row i
  __syncwarp();
  float* blk = a.Phit + (long long)(n + 1) * ld * t;
  warp_colmv(blk, ld, n, n, pc, e);
  __syncwarp();  // the two products may split e over the lanes differently
  warp_colmv(a.K + nm * t, n, m, n, r, e);
  __syncwarp();
  for (int i = threadIdx.x & 31; i < n; i += 32) {
    blk[n * ld + i] = e[i];
    a.pcv[(long long)ld * t + i] = pc[i];
  }
}

// with p_{t+1} known: k~_t = -M_uu,t^-1 (r~_t + B_t'(Pc_t + p_{t+1})) and
// w_t = B_t k~_t + c~_t (into row n of the block of Phi_t'), t < T
__global__ void __launch_bounds__(kParWarps * 32) corr_ctrl_kernel(CorrArgs a) {
  extern __shared__ __align__(16) float psm[];
  __shared__ int s_flag;
  if (corr_exit(a.status, a.skip, &s_flag)) return;
  const int n = a.n, m = a.m, ld = corr_ld(n), v = corr_ld(n > m ? n : m), w = threadIdx.x >> 5;
  const int t = blockIdx.x * kParWarps + w;
  if (t >= a.T) return;
  float* s = psm + w * 4 * v;
  float* gu = s + v;
  float* k = gu + v;
  float* wv = k + v;
  const long long nm = (long long)n * m, mm = (long long)m * m;
  for (int i = threadIdx.x & 31; i < n; i += 32)
    s[i] = a.pcv[(long long)ld * t + i] + a.dp[(long long)n * (t + 1) + i];
  warp_load(gu, a.cr + (long long)m * t, m);
  warp_load(k, nullptr, m);
  warp_load(wv, a.cc + (long long)n * t, n);
  __syncwarp();
  warp_colmv(a.B + nm * t, m, n, m, s, gu);
  __syncwarp();
  warp_colmv(a.Minv + mm * t, m, m, m, gu, k);  // M_uu^-1 symmetric
  __syncwarp();
  for (int c = threadIdx.x & 31; c < m; c += 32) {
    k[c] = -k[c];
    a.dk[(long long)m * t + c] = k[c];
  }
  __syncwarp();
  warp_rowmv(a.B + nm * t, m, n, m, k, wv);
  __syncwarp();
  float* wrow = a.PhiTt + (long long)(n + 1) * ld * t + (long long)n * ld;
  for (int i = threadIdx.x & 31; i < n; i += 32) wrow[i] = wv[i];
}

// with x~ known: u~_t = K_t x~_t + k~_t (t < T), lambda~_t = -(P_t x~_t + p_t) (t <= T)
__global__ void __launch_bounds__(kParWarps * 32) corr_out_kernel(CorrArgs a) {
  extern __shared__ __align__(16) float psm[];
  __shared__ int s_flag;
  if (corr_exit(a.status, a.skip, &s_flag)) return;
  const int n = a.n, m = a.m, v = corr_ld(n > m ? n : m), w = threadIdx.x >> 5;
  const int t = blockIdx.x * kParWarps + w;
  if (t > a.T) return;
  float* x = psm + w * 4 * v;
  float* l = x + v;
  float* u = l + v;
  const long long nn = (long long)n * n, nm = (long long)n * m;
  warp_load(x, a.dx + (long long)n * t, n);
  warp_load(l, a.dp + (long long)n * t, n);
  if (t < a.T) warp_load(u, a.dk + (long long)m * t, m);
  __syncwarp();
  warp_colmv(a.P + nn * t, n, n, n, x, l);  // P symmetric
  if (t < a.T) warp_rowmv(a.K + nm * t, n, m, n, x, u);  // another output vector
  __syncwarp();
  for (int i = threadIdx.x & 31; i < n; i += 32) a.dl[(long long)n * t + i] = -l[i];
  if (t < a.T)
    for (int c = threadIdx.x & 31; c < m; c += 32) a.du[(long long)m * t + c] = u[c];
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
cudaError_t launch_corr_groups(const CorrArgs& a, cudaStream_t st) {
  if (a.ng <= 0) return cudaSuccess;
  const size_t bytes = corr_group_smem_bytes(a.n);
  cudaError_t e = raise_dyn_smem((const void*)corr_group_maps_kernel, bytes);
  if (e != cudaSuccess) return e;
  corr_group_maps_kernel<<<a.ng, kCorrBlock, bytes, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_corr_psi(const CorrArgs& a, cudaStream_t st) {
  const size_t bytes = corr_psi_smem_bytes(a.n, a.m, a.psi_global);
  cudaError_t e = raise_dyn_smem((const void*)corr_psi_kernel, bytes);
  if (e != cudaSuccess) return e;
  corr_psi_kernel<<<a.nseg, kCorrBlock, bytes, st>>>(a);
  return cudaGetLastError();
}

// one correction: e, eps, backward links, p, k~ and w, delta, forward links, x~, u~ and lambda~
cudaError_t launch_correction(const CorrArgs& a, cudaStream_t st, int* launches) {
  const int n = a.n, ld = corr_ld(n), K = a.nseg, T = a.T;
  const size_t rb = corr_rec_smem_bytes(n, a.slots), pb = corr_par_smem_bytes(n, a.m);
  cudaError_t e = raise_dyn_smem((const void*)corr_rec_kernel, rb);
  if (e == cudaSuccess) e = raise_dyn_smem((const void*)corr_rhs_kernel, pb);
  if (e == cudaSuccess) e = raise_dyn_smem((const void*)corr_ctrl_kernel, pb);
  if (e == cudaSuccess) e = raise_dyn_smem((const void*)corr_out_kernel, pb);
  if (e != cudaSuccess) return e;
  const long long blk = (long long)(n + 1) * ld, orow = (long long)n * ld;
  int cnt = 0;
  auto rec = [&](const float* C, const float* y0, long long y0s, float* all, long long as, float* end, int count,
                 int nruns, int G, int dir) {
    RecArgs r;
    r.C = C; r.cstride = blk;
    r.y0 = y0; r.y0stride = y0s; r.all = all; r.astride = as; r.end = end; r.estride = blk;
    r.n = n; r.ld = ld; r.count = count; r.nruns = nruns; r.G = G; r.slots = a.slots; r.spin = a.spin;
    r.skip = a.skip; r.status = a.status;
    corr_rec_kernel<<<nruns, kRecBlock, rb, st>>>(r, dir);
    ++cnt;
  };
  const int pgrid = (T + kParWarps) / kParWarps;  // T + 1 stages for the outputs
  const float* qT = a.cq + (long long)n * T;
  // the link chain of one direction: one run over all K links, or two levels over groups
  auto chain = [&](int dir) {
    const float* psi = dir == 0 ? a.Psi : a.PsiT;  // offsets eps_j / delta_j in row n
    const float* start = dir == 0 ? qT : a.cx0;
    float* bound = dir == 0 ? a.pb : a.xb;
    if (a.ng > 0) {
      float* th = dir == 0 ? a.Theta : a.ThetaT;
      float* gv = dir == 0 ? a.gY : a.gX;
      rec(psi, nullptr, 0, nullptr, 0, th + orow, K, a.ng, a.G, dir);
      rec(th, start, 0, gv, n, nullptr, a.ng, 1, a.ng, dir);
      rec(psi, gv, n, bound, n, nullptr, K, a.ng, a.G, dir);
    } else {
      rec(psi, start, 0, bound, n, nullptr, K, 1, K, dir);
    }
  };
  corr_rhs_kernel<<<(T + kParWarps - 1) / kParWarps, kParWarps * 32, pb, st>>>(a);
  rec(a.Phit, nullptr, 0, nullptr, 0, a.Psi + orow, T, K, 0, 0);
  chain(0);
  rec(a.Phit, a.pb, n, a.dp, n, nullptr, T, K, 0, 0);
  corr_ctrl_kernel<<<(T + kParWarps - 1) / kParWarps, kParWarps * 32, pb, st>>>(a);
  rec(a.PhiTt, nullptr, 0, nullptr, 0, a.PsiT + orow, T, K, 0, 1);
  chain(1);
  rec(a.PhiTt, a.xb, n, a.dx, n, nullptr, T, K, 0, 1);
  corr_out_kernel<<<pgrid, kParWarps * 32, pb, st>>>(a);
  if (launches) *launches += cnt + 3;
  return cudaGetLastError();
}

}  // namespace lqr
