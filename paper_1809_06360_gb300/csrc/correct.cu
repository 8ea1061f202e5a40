// Step A8: refinement corrections that reuse the factorisation of the solve.
//
// A correction solves the LQR problem with the solve's matrices and new vector
// data (q~, r~, c~, x0~). With the solve's global policies K_t, value matrices
// P_t and the inverses M_uu,t^-1 = (R_t + B_t'P_{t+1}B_t)^-1 kept, it is an
// affine recursion in the vectors alone (the serial Riccati recursion of
// Section III-A with the matrices fixed):
//   s_t = P_{t+1} c~_t + p_{t+1},  g_u = r~_t + B_t's_t,  g_x = q~_t + A_t's_t
//   k~_t = -M_uu,t^-1 g_u,  p_t = g_x + K_t'g_u  (= Phi_t'p_{t+1} + e_t, Phi_t = A_t + B_t K_t)
//   u~_t = K_t x~_t + k~_t,  x~_{t+1} = A_t x~_t + B_t u~_t + c~_t,
//   lambda~_t = -(P_t x~_t + p_t),  p_T = q~_T.
// It splits over the solve's K segments: with the closed-loop segment map
// Psi_j = Phi_{e-1} ... Phi_b (b = b_j, e = b_{j+1}), p_b = Psi_j'p_e + eps_j and
// x~_e = Psi_j x~_b + delta_j, where eps_j (delta_j) is the segment's own pass
// started from p_e = 0 (x~_b = 0). One correction is then: the segment passes
// for eps_j (parallel), the backward link chain for p at the boundaries, the
// segment passes for p_t, k~_t (parallel), the segment passes for delta_j, the
// forward link chain for x~ at the boundaries, and the final segment passes for
// x~_t, u~_t, lambda~_t: O(T (n^2 + nm)) work instead of the solve's O(T n^3).
// Psi_j is formed once per solve. FP32 data and arithmetic (the corrections of
// the mixed FP32 mode, whose FP64 residual decides convergence).
//
// Shared-memory matrices are stored with odd row strides (n + 1, m + 1) so
// that both row-per-thread and column-per-thread reads are conflict-free; the
// stage data of the next stage is copied with cp.async while the current one
// computes.
#include <cuda_runtime.h>

#include "cta_linalg.cuh"
#include "lqr_internal.cuh"

namespace lqr {

namespace {

constexpr int kCorrBlock = 256;
constexpr int kLinkDepth = 3;  // Psi_j ring depth of the link chains
constexpr int kLinkSplit = 4;  // threads per output of a link step (partial sums over l)

__device__ __forceinline__ bool corr_exit(const CorrArgs& a, int* s_flag) {
  if (threadIdx.x == 0) *s_flag = (*(volatile int*)a.status != 0) || (a.skip && *(volatile const int*)a.skip);
  __syncthreads();
  const bool ex = *s_flag != 0;
  __syncthreads();
  return ex;
}

// rows x cols floats (row stride cols) into shared memory with row stride ldd
__device__ __forceinline__ void copy_pad(float* dst, int ldd, const float* src, int rows, int cols) {
  cta_for_rc(rows, cols, [&](int e, int i, int j) { cp_async4(dst + i * ldd + j, src + e); });
}
__device__ __forceinline__ void copy_vec(float* dst, const float* src, int cnt) {
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) cp_async4(dst + e, src + e);
}

// one ring slot of the segment passes: A, B, K, P, M_uu^-1 and the stage vectors
struct CorrSlot {
  int ldn, ldm;  // n + 1, m + 1
  int oA, oB, oK, oP, oM, oc, oq, or_, ok, op, size;
};

__host__ __device__ inline CorrSlot corr_slot(int n, int m) {
  CorrSlot s;
  s.ldn = n + 1;
  s.ldm = m + 1;
  int o = 0;
  s.oA = o; o += n * s.ldn;
  s.oB = o; o += n * s.ldm;
  s.oK = o; o += m * s.ldn;
  s.oP = o; o += n * s.ldn;
  s.oM = o; o += m * s.ldm;
  s.oc = o; o += n;
  s.oq = o; o += n;
  s.or_ = o; o += m;
  s.ok = o; o += m;
  s.op = o; o += n;
  s.size = (o + 3) & ~3;
  return s;
}

}  // namespace

size_t corr_seg_smem_bytes(int n, int m, int slots) {
  return sizeof(float) * ((size_t)slots * corr_slot(n, m).size + 4 * n + 2 * m);
}
size_t corr_psi_smem_bytes(int n, int m, int psi_global) {
  const size_t N = (n + 3) & ~3, M = (m + 3) & ~3;
  return sizeof(float) * (3 * N * (N + 4) + (psi_global ? 0 : N * (M + 4) + M * (N + 4)));
}
void corr_plan(int n, int m, long long smem_budget, int* slots, int* psi_global) {
  *slots = 0;
  *psi_global = 0;
  if ((long long)corr_link_smem_bytes(n) > smem_budget) return;
  if ((long long)corr_psi_smem_bytes(n, m, 0) > smem_budget) {
    // B_t, K_t straight from global memory: float4 rows need n, m multiples of 4
    if (n % 4 != 0 || m % 4 != 0 || (long long)corr_psi_smem_bytes(n, m, 1) > smem_budget) return;
    *psi_global = 1;
  }
  if ((long long)corr_seg_smem_bytes(n, m, 2) <= smem_budget) *slots = 2;
  else if ((long long)corr_seg_smem_bytes(n, m, 1) <= smem_budget) *slots = 1;
}
size_t corr_link_smem_bytes(int n) {
  return sizeof(float) * ((size_t)kLinkDepth * n * (n + 1) + (1 + kLinkSplit) * (size_t)n);
}

// Psi_j = Phi_{e-1} ... Phi_b, Phi_t = A_t + B_t K_t: one CTA per segment, the
// two products of a stage on 4 x 4 register tiles (n, m padded to multiples of
// 4 with zeros; row strides N + 4, M + 4), A_t staged in the free Psi buffer.
__global__ void __launch_bounds__(kCorrBlock) corr_psi_kernel(CorrArgs a) {
  extern __shared__ __align__(16) float csm[];
  __shared__ int s_flag;
  if (corr_exit(a, &s_flag)) return;
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
  const long long nn = (long long)n * n, nm = (long long)n * m;
  for (int t = b; t < e; ++t) {
    copy_pad(Y, LD, a.A + nn * t, n, n);
    if (!a.psi_global) {
      copy_pad(Bs, LDm, a.B + nm * t, n, m);
      copy_pad(Ks, LD, a.K + nm * t, m, n);
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
    cta_mm4f<false>(N, N, N, Phi, LD, X, LD, [&](int i, int l, float v) { Y[i * LD + l] = v; });
    __syncthreads();
    float* tmp = X;
    X = Y;
    Y = tmp;
  }
  for (int x = threadIdx.x; x < n * n; x += blockDim.x) {
    const int i = x / n, l = x - i * n;
    a.Psi[nn * j + x] = X[i * LD + l];
  }
}

// Backward segment pass. mode 0: from p_e = 0, writes eps_j. mode 1: from
// p_e = pb[j + 1], writes p_t (dp) and k~_t (dk) for the segment's stages (and
// the last segment p_T).
__global__ void __launch_bounds__(kCorrBlock) corr_back_kernel(CorrArgs a, int mode) {
  extern __shared__ __align__(16) float csm[];
  __shared__ int s_flag;
  if (corr_exit(a, &s_flag)) return;
  const int n = a.n, m = a.m, T = a.T, j = blockIdx.x;
  const int b = seg_begin(T, a.nseg, j), e = seg_begin(T, a.nseg, j + 1);
  if (e <= b) return;  // an empty segment (uniform over the CTA)
  const CorrSlot L = corr_slot(n, m);
  float* ring = csm;
  float* p = ring + (a.slots > 1 ? 2 : 1) * L.size;
  float* s = p + n;
  float* gx = s + n;
  float* gu = gx + n;
  const long long nn = (long long)n * n, nm = (long long)n * m, mm = (long long)m * m;
  const int two = a.slots > 1;
  auto slot = [&](int t) { return ring + (two ? ((e - 1 - t) & 1) : 0) * L.size; };
  auto issue = [&](int t) {
    float* sl = slot(t);
    copy_pad(sl + L.oA, L.ldn, a.A + nn * t, n, n);
    copy_pad(sl + L.oB, L.ldm, a.B + nm * t, n, m);
    copy_pad(sl + L.oK, L.ldn, a.K + nm * t, m, n);
    copy_pad(sl + L.oP, L.ldn, a.P + nn * (t + 1), n, n);
    if (mode == 1) copy_pad(sl + L.oM, L.ldm, a.Minv + mm * t, m, m);
    copy_vec(sl + L.oc, a.cc + (long long)n * t, n);
    copy_vec(sl + L.oq, a.cq + (long long)n * t, n);
    copy_vec(sl + L.or_, a.cr + (long long)m * t, m);
    cp_async_commit();
  };
  if (two) issue(e - 1);
  for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = (mode == 0) ? 0.0f : a.pb[(long long)n * (j + 1) + i];
  if (mode == 1 && j == a.nseg - 1)
    for (int i = threadIdx.x; i < n; i += blockDim.x) a.dp[(long long)n * T + i] = a.pb[(long long)n * a.nseg + i];
  for (int t = e - 1; t >= b; --t) {
    const float* sl = slot(t);
    if (!two) {  // one slot: the previous stage has finished with it
      __syncthreads();
      issue(t);
    }
    cp_async_wait<0>();
    __syncthreads();  // stage t in its slot; p of stage t + 1 complete
    if (two && t - 1 >= b) issue(t - 1);
    const float* As = sl + L.oA;
    const float* Bs = sl + L.oB;
    const float* Ks = sl + L.oK;
    const float* Ps = sl + L.oP;
    const float* Ms = sl + L.oM;
    // s = P_{t+1} c~_t + p_{t+1} (P symmetric: column reads)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      float v = p[i];
      for (int l = 0; l < n; ++l) v = fmaf(Ps[l * L.ldn + i], sl[L.oc + l], v);
      s[i] = v;
    }
    __syncthreads();
    // g_x = q~ + A's, g_u = r~ + B's
    for (int x = threadIdx.x; x < n + m; x += blockDim.x) {
      if (x < n) {
        float v = sl[L.oq + x];
        for (int i = 0; i < n; ++i) v = fmaf(As[i * L.ldn + x], s[i], v);
        gx[x] = v;
      } else {
        const int c = x - n;
        float v = sl[L.or_ + c];
        for (int i = 0; i < n; ++i) v = fmaf(Bs[i * L.ldm + c], s[i], v);
        gu[c] = v;
      }
    }
    __syncthreads();
    // p_t = g_x + K'g_u ; k~_t = -M_uu^-1 g_u
    for (int x = threadIdx.x; x < n + m; x += blockDim.x) {
      if (x < n) {
        float v = gx[x];
        for (int c = 0; c < m; ++c) v = fmaf(Ks[c * L.ldn + x], gu[c], v);
        p[x] = v;
        if (mode == 1) a.dp[(long long)n * t + x] = v;
      } else if (mode == 1) {
        const int c = x - n;
        float v = 0.0f;
        for (int d = 0; d < m; ++d) v = fmaf(Ms[c * L.ldm + d], gu[d], v);
        a.dk[(long long)m * t + c] = -v;
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  if (mode == 0)
    for (int i = threadIdx.x; i < n; i += blockDim.x) a.eps[(long long)n * j + i] = p[i];
}

// Forward segment pass. mode 0: from x~_b = 0, writes delta_j. mode 1: from
// x~_b = xb[j], writes x~_t, u~_t, lambda~_t (and the last segment x~_T, lambda~_T).
__global__ void __launch_bounds__(kCorrBlock) corr_fwd_kernel(CorrArgs a, int mode) {
  extern __shared__ __align__(16) float csm[];
  __shared__ int s_flag;
  if (corr_exit(a, &s_flag)) return;
  const int n = a.n, m = a.m, T = a.T, j = blockIdx.x;
  const int b = seg_begin(T, a.nseg, j), e = seg_begin(T, a.nseg, j + 1);
  if (e <= b) return;  // an empty segment (uniform over the CTA)
  const CorrSlot L = corr_slot(n, m);
  float* ring = csm;
  float* x0 = ring + (a.slots > 1 ? 2 : 1) * L.size;  // two state buffers
  float* x1 = x0 + n;
  float* u = x1 + n;
  const long long nn = (long long)n * n, nm = (long long)n * m;
  const int two = a.slots > 1;
  auto slot = [&](int t) { return ring + (two ? ((t - b) & 1) : 0) * L.size; };
  auto issue = [&](int t) {
    float* sl = slot(t);
    copy_pad(sl + L.oA, L.ldn, a.A + nn * t, n, n);
    copy_pad(sl + L.oB, L.ldm, a.B + nm * t, n, m);
    copy_pad(sl + L.oK, L.ldn, a.K + nm * t, m, n);
    if (mode == 1) {
      copy_pad(sl + L.oP, L.ldn, a.P + nn * t, n, n);
      copy_vec(sl + L.op, a.dp + (long long)n * t, n);
    }
    copy_vec(sl + L.oc, a.cc + (long long)n * t, n);
    copy_vec(sl + L.ok, a.dk + (long long)m * t, m);
    cp_async_commit();
  };
  if (two) issue(b);
  for (int i = threadIdx.x; i < n; i += blockDim.x) x0[i] = (mode == 0) ? 0.0f : a.xb[(long long)n * j + i];
  float* xc = x0;
  float* xn = x1;
  for (int t = b; t < e; ++t) {
    const float* sl = slot(t);
    if (!two) {  // one slot: the previous stage has finished with it
      __syncthreads();
      issue(t);
    }
    cp_async_wait<0>();
    __syncthreads();  // stage t in its slot; x~_t complete
    if (two && t + 1 < e) issue(t + 1);
    const float* As = sl + L.oA;
    const float* Bs = sl + L.oB;
    const float* Ks = sl + L.oK;
    const float* Ps = sl + L.oP;
    // u~ = K x~ + k~ ; lambda~ = -(P x~ + p) (P symmetric: column reads)
    for (int x = threadIdx.x; x < n + m; x += blockDim.x) {
      if (x < m) {
        float v = sl[L.ok + x];
        for (int l = 0; l < n; ++l) v = fmaf(Ks[x * L.ldn + l], xc[l], v);
        u[x] = v;
        if (mode == 1) a.du[(long long)m * t + x] = v;
      } else if (mode == 1) {
        const int i = x - m;
        float v = sl[L.op + i];
        for (int l = 0; l < n; ++l) v = fmaf(Ps[l * L.ldn + i], xc[l], v);
        a.dl[(long long)n * t + i] = -v;
        a.dx[(long long)n * t + i] = xc[i];
      }
    }
    __syncthreads();
    // x~_{t+1} = A x~ + B u~ + c~
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      float v = sl[L.oc + i];
      for (int l = 0; l < n; ++l) v = fmaf(As[i * L.ldn + l], xc[l], v);
      for (int c = 0; c < m; ++c) v = fmaf(Bs[i * L.ldm + c], u[c], v);
      xn[i] = v;
    }
    float* tmp = xc;
    xc = xn;
    xn = tmp;
  }
  cp_async_wait<0>();
  __syncthreads();
  if (mode == 0) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) a.delta[(long long)n * j + i] = xc[i];
  } else if (j == a.nseg - 1) {
    // x~_T and lambda~_T = -(P_T x~_T + p_T)
    const float* PT = a.P + nn * T;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      float v = a.dp[(long long)n * T + i];
      for (int l = 0; l < n; ++l) v = fmaf(PT[(long long)l * n + i], xc[l], v);
      a.dl[(long long)n * T + i] = -v;
      a.dx[(long long)n * T + i] = xc[i];
    }
  }
}

// A run of dependent link steps by one CTA. dir 0 (backward): links l = hi-1
// down to lo, v <- M_l' v + off_l, out[l] = v. dir 1 (forward): links l = lo ..
// hi-1, v <- M_l v + off_l, out[l + 1] = v. M_l (n x n) arrive through a ring of
// kLinkDepth slots, kLinkDepth - 1 links ahead; each output of a step is summed
// by kLinkSplit threads over a quarter of l each (output index fastest over the
// threads: conflict-free reads of M's rows and columns at the odd row stride),
// the partial sums combined through shared memory. v (shared) holds the start
// value on entry and the end value on exit; out may be null.
__device__ inline void chain_run(const float* mats, const float* offs, int lo, int hi, int dir, int n, float* v,
                                 float* out, float* csm) {
  const long long nn = (long long)n * n;
  const int ldn = n + 1;
  constexpr int kRows = kCorrBlock / kLinkSplit;  // outputs per pass of the thread block
  float* ring = csm;
  float* part = ring + kLinkDepth * n * ldn;  // [kLinkSplit][n]
  const int q = (int)threadIdx.x / kRows, r0 = (int)threadIdx.x % kRows;
  const int chunk = (n + kLinkSplit - 1) / kLinkSplit;
  const int l0 = q * chunk < n ? q * chunk : n, l1 = (q + 1) * chunk < n ? (q + 1) * chunk : n;
  const int cnt = hi - lo;
  auto link_of = [&](int idx) { return dir == 0 ? hi - 1 - idx : lo + idx; };
  auto issue = [&](int idx) {
    if (idx < cnt) copy_pad(ring + (idx % kLinkDepth) * n * ldn, ldn, mats + nn * link_of(idx), n, n);
    cp_async_commit();
  };
  for (int d = 0; d < kLinkDepth - 1; ++d) issue(d);
  for (int idx = 0; idx < cnt; ++idx) {
    issue(idx + kLinkDepth - 1);
    cp_async_wait<kLinkDepth - 1>();
    __syncthreads();  // M of this link in its slot; v complete
    const float* Ms = ring + (idx % kLinkDepth) * n * ldn;
    const int jl = link_of(idx);
    for (int i = r0; i < n; i += kRows) {
      float acc = 0.0f;
      if (dir == 0)
        for (int l = l0; l < l1; ++l) acc = fmaf(Ms[l * ldn + i], v[l], acc);
      else
        for (int l = l0; l < l1; ++l) acc = fmaf(Ms[i * ldn + l], v[l], acc);
      part[q * n + i] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      float acc = offs[(long long)n * jl + i];
#pragma unroll
      for (int g = 0; g < kLinkSplit; ++g) acc += part[g * n + i];
      v[i] = acc;
      if (out) out[(long long)n * (dir == 0 ? jl : jl + 1) + i] = acc;
    }
  }
  cp_async_wait<0>();
  __syncthreads();
}

// The single link chain, one CTA. dir 0: pb[K] = q~_T, pb[j] = Psi_j'pb[j + 1] + eps_j
// (j = K-1 .. 0). dir 1: xb[0] = x0~, xb[j + 1] = Psi_j xb[j] + delta_j.
__global__ void __launch_bounds__(kCorrBlock) corr_link_kernel(CorrArgs a, int dir) {
  extern __shared__ __align__(16) float csm[];
  __shared__ int s_flag;
  if (corr_exit(a, &s_flag)) return;
  const int n = a.n, K = a.nseg;
  float* v = csm + kLinkDepth * n * (n + 1) + kLinkSplit * n;
  float* out = dir == 0 ? a.pb : a.xb;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    v[i] = dir == 0 ? a.cq[(long long)n * a.T + i] : a.cx0[i];
    out[(long long)n * (dir == 0 ? K : 0) + i] = v[i];
  }
  chain_run(a.Psi, dir == 0 ? a.eps : a.delta, 0, K, dir, n, v, out, csm);
}

// The two-level chain over groups of G links (a depth of about 2 G + K / G steps
// instead of K). stage 0, one CTA per group: the group's own steps from zero give
// its offset (e_g backward, d_g forward: pb_lo = Phi_g' pb_hi + e_g,
// x_hi = Phi_g x_lo + d_g). stage 1, one CTA: the chain over the groups with the
// group maps Phi_g = Psi_{hi-1} ... Psi_lo gives the group boundary values.
// stage 2, one CTA per group: the group's steps from its boundary value write
// every link value.
__global__ void __launch_bounds__(kCorrBlock) corr_chain2_kernel(CorrArgs a, int dir, int stage) {
  extern __shared__ __align__(16) float csm[];
  __shared__ int s_flag;
  if (corr_exit(a, &s_flag)) return;
  const int n = a.n, K = a.nseg, G = a.G, ng = a.ng;
  float* v = csm + kLinkDepth * n * (n + 1) + kLinkSplit * n;
  const float* offs = dir == 0 ? a.eps : a.delta;
  if (stage == 1) {
    float* gv = dir == 0 ? a.gY : a.gX;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      v[i] = dir == 0 ? a.cq[(long long)n * a.T + i] : a.cx0[i];
      gv[(long long)n * (dir == 0 ? ng : 0) + i] = v[i];
    }
    chain_run(a.Phi, dir == 0 ? a.ge : a.gd, 0, ng, dir, n, v, gv, csm);
    return;
  }
  const int g = blockIdx.x;
  const int lo = g * G, hi = (lo + G < K) ? lo + G : K;
  float* out = nullptr;
  if (stage == 0) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = 0.0f;
  } else {
    const float* gv = dir == 0 ? a.gY : a.gX;
    out = dir == 0 ? a.pb : a.xb;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      v[i] = gv[(long long)n * (dir == 0 ? g + 1 : g) + i];
      if (dir == 0 && g == ng - 1) out[(long long)n * K + i] = v[i];  // pb[K] = q~_T
      if (dir == 1 && g == 0) out[i] = v[i];                          // xb[0] = x0~
    }
  }
  __syncthreads();
  chain_run(a.Psi, offs, lo, hi, dir, n, v, out, csm);
  if (stage == 0) {
    float* go = dir == 0 ? a.ge : a.gd;
    for (int i = threadIdx.x; i < n; i += blockDim.x) go[(long long)n * g + i] = v[i];
  }
}

// Phi_g = Psi_{hi-1} ... Psi_lo per group (once per solve): one CTA per group,
// products on 4 x 4 register tiles (n padded to a multiple of 4, row stride N + 4).
__global__ void __launch_bounds__(kCorrBlock) corr_group_maps_kernel(CorrArgs a) {
  extern __shared__ __align__(16) float csm[];
  __shared__ int s_flag;
  if (corr_exit(a, &s_flag)) return;
  const int n = a.n, K = a.nseg, G = a.G;
  const int g = blockIdx.x;
  const int lo = g * G, hi = (lo + G < K) ? lo + G : K;
  const int N = (n + 3) & ~3, LD = N + 4;
  float* X = csm;        // product so far
  float* Y = X + N * LD;
  float* M = Y + N * LD;  // Psi_j
  for (int x = threadIdx.x; x < 3 * N * LD; x += blockDim.x) csm[x] = 0.0f;
  __syncthreads();
  const long long nn = (long long)n * n;
  copy_pad(X, LD, a.Psi + nn * lo, n, n);
  cp_async_commit();
  for (int j = lo + 1; j < hi; ++j) {
    copy_pad(M, LD, a.Psi + nn * j, n, n);
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
  for (int x = threadIdx.x; x < n * n; x += blockDim.x) a.Phi[nn * g + x] = X[(x / n) * LD + x % n];
}

size_t corr_group_smem_bytes(int n) {
  const size_t N = (n + 3) & ~3;
  return sizeof(float) * 3 * N * (N + 4);
}

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

// one correction: eps, backward links, p and k~, delta, forward links, x~ u~ lambda~
cudaError_t launch_correction(const CorrArgs& a, cudaStream_t st, int* launches) {
  const size_t sb = corr_seg_smem_bytes(a.n, a.m, a.slots), lb = corr_link_smem_bytes(a.n);
  cudaError_t e = raise_dyn_smem((const void*)corr_back_kernel, sb);
  if (e == cudaSuccess) e = raise_dyn_smem((const void*)corr_fwd_kernel, sb);
  if (e == cudaSuccess) e = raise_dyn_smem((const void*)corr_link_kernel, lb);
  if (e != cudaSuccess) return e;
  if (a.ng > 0) {
    e = raise_dyn_smem((const void*)corr_chain2_kernel, lb);
    if (e != cudaSuccess) return e;
  }
  // a link chain: one CTA over all K links, or the two-level form over groups
  auto chain = [&](int dir) {
    if (a.ng > 0) {
      corr_chain2_kernel<<<a.ng, kCorrBlock, lb, st>>>(a, dir, 0);
      corr_chain2_kernel<<<1, kCorrBlock, lb, st>>>(a, dir, 1);
      corr_chain2_kernel<<<a.ng, kCorrBlock, lb, st>>>(a, dir, 2);
      if (launches) *launches += 3;
    } else {
      corr_link_kernel<<<1, kCorrBlock, lb, st>>>(a, dir);
      if (launches) *launches += 1;
    }
  };
  corr_back_kernel<<<a.nseg, kCorrBlock, sb, st>>>(a, 0);
  chain(0);
  corr_back_kernel<<<a.nseg, kCorrBlock, sb, st>>>(a, 1);
  corr_fwd_kernel<<<a.nseg, kCorrBlock, sb, st>>>(a, 0);
  chain(1);
  corr_fwd_kernel<<<a.nseg, kCorrBlock, sb, st>>>(a, 1);
  if (launches) *launches += 4;
  return cudaGetLastError();
}

}  // namespace lqr
