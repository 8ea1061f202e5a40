// Step A3 as a parallel scan (FP32 mode). The link recursion of Section II-C
// (Eq. 10-11 in the multiplier form) composes segment summaries
//     S_j = (P_j, Z_j, W_j, p_j, w_j):   x_end = Z_j x - W_j mu + w_j,
//                                          lambda_start = P_j x + p_j + Z_j' mu
// (x the segment's start state, mu its end costate). Two adjacent segments a
// (earlier) and b compose into one summary with, for M = I + W_a P_b,
//     P_ab = P_a + Z_a' P_b M^-1 Z_a          p_ab = p_a + Z_a'(p_b + P_b M^-1 v)
//     Z_ab = Z_b M^-1 Z_a                     w_ab = w_b + Z_b M^-1 v
//     W_ab = W_b + Z_b M^-1 W_a Z_b'          v = w_a - W_a p_b
// and this composition is associative, so the global value functions
// Pi_j = P(S_j o S_{j+1} o ... o S_{K-1}) follow from a suffix scan in
// ceil(log2 K) levels of independent compositions instead of K-1 dependent
// link steps. Every M^-1 is evaluated in the symmetric form
//     C = chol(P_b),  Tm = W_a C,  Y = (I + C'Tm)^-1 (SPD, eigenvalues <= 1),
//     E = C'[Z_a | v],  F2 = Y E,
//     P_b M^-1 = C Y C',  M^-1 [Z_a | v] = [Z_a | v] - Tm F2,
//     M^-1 W_a = W_a - Tm Y Tm'.
// A last pass composes each S_j with the final Pi_{j+1} to get the link
// feedback Gam_j, gam_j (z_{j+1} = Gam_j z_j + gam_j; gam_j refined in FP64),
// and one CTA runs the O(K n^2) chain of link states (FP32 products, FP64
// sums) with the Gam_j prefetched into shared memory.
// One CTA per composition; all operands in shared memory in FP32, row-major,
// n rounded up to n4 (multiple of 4) with zero padding so that every product
// runs on 4 x 4 register tiles with 128-bit loads.
#include <cuda_runtime.h>

#include "cta_linalg.cuh"
#include "lqr_internal.cuh"

namespace lqr {

// Summaries (FP64, [P | Z | -W | p | w]) to FP32 scan elements (buffer 0);
// the last segment's summary is already its global value function.
__global__ void link_scan_init_kernel(ProbTable tab) {
  __shared__ int s_flag;
  const ProbDesc& pd = tab.single;
  if (cta_should_exit(pd, &s_flag)) return;
  const int n = pd.n, K = pd.nseg, j = blockIdx.x;
  const long long nn = (long long)n * n, ss = 3 * nn + 2 * n;
  const WsLayout wl = ws_layout(n, K);
  const double* S = pd.ws + wl.summ + (long long)j * ss;
  float* e = reinterpret_cast<float*>(pd.ws + wl.scan) + (long long)j * scan_elem_floats(n);
  for (long long i = threadIdx.x; i < ss; i += blockDim.x) e[i] = static_cast<float>(S[i]);
  if (j == K - 1) {
    for (long long i = threadIdx.x; i < nn; i += blockDim.x) pd.ws[wl.Pi + (long long)j * nn + i] = S[i];
    for (int i = threadIdx.x; i < n; i += blockDim.x) pd.ws[wl.pi + (long long)j * n + i] = S[3 * nn + i];
  }
}

// shared-memory plan of one composition (floats): Cb, Wa, Zb, Tm, Y (n4 x n4),
// Za, E, F2 (n4 x (n4 + 4)), pb, wa (n4), the block-elimination scratch, then
// gd, t1, gbk (n4 doubles each) and 1/diag(C) (n4).
// ldn: leading dimension of the n4 x n4 buffers, n4 + 4 (rows four apart fall
// in different banks) when that fits, else n4.
__host__ __device__ inline long long scan_tail_offset(int n, int ldn) {
  const long long n4 = (n + 3) & ~3, ld1 = n4 + 4;
  return 5 * n4 * ldn + 3 * n4 * ld1 + 2 * n4;
}
__host__ __device__ inline long long scan_smem_floats(int n, int ldn) {
  const long long n4 = (n + 3) & ~3;
  return scan_tail_offset(n, ldn) + p4_scratch_floats(n) + 6 * n4 + n4 + 4;
}

// mode 0: one level of the suffix scan with stride s. CTA j composes element
//         j (buffer src) with element b = j + s; when b + s >= K element b
//         already covers the last segment, its value function is final
//         (Pi_b, pi_b in the workspace) and so is the result (written to
//         Pi_j, pi_j); otherwise the full composite goes to buffer dst.
// mode 1: the feedback pass. CTA j composes the original S_j (buffer 0) with
//         the final Pi_{j+1} and keeps M^-1 [Z_j | v] = [Gam_j | gam_j].
constexpr int kScanBlock = 512;  // 16 warps per composition

template <int SHAPE>  // p4_shape(n): register-block shape of the block eliminations
__global__ void __launch_bounds__(kScanBlock, 1) link_scan_kernel(ProbTable tab, int s, int mode, int src_buf, int dst_buf,
                                                                 int ldn) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_flag;
  const ProbDesc& pd = tab.single;
  if (cta_should_exit(pd, &s_flag)) return;
  const int n = pd.n, K = pd.nseg, j = blockIdx.x;
  const int n4 = (n + 3) & ~3, ld1 = n4 + 4;
  const long long nn = (long long)n * n, es = scan_elem_floats(n);
  const WsLayout wl = ws_layout(n, K);
  double* ws = pd.ws;
  float* sbase = reinterpret_cast<float*>(ws + wl.scan);
  const int b = j + (mode == 0 ? s : 1);
  const bool bfin = (mode == 1) || (b + s >= K);
  const float* ea = sbase + ((long long)(mode == 0 ? src_buf : 0) * K + j) * es;
  const float* eb = sbase + ((long long)src_buf * K + b) * es;  // read only when !bfin
  float* ed = sbase + ((long long)dst_buf * K + j) * es;

  float* Cb = reinterpret_cast<float*>(smem);  // C = chol(P_b), later U = Y Tm'
  float* Wa = Cb + n4 * ldn;                   // -W_a, later -(M^-1 W_a)
  float* Zb = Wa + n4 * ldn;                   // Z_b
  float* Tm = Zb + n4 * ldn;                   // W_a C
  float* Y = Tm + n4 * ldn;                    // (I + C'W_a C)^-1
  float* Za = Y + n4 * ldn;                    // [Z_a | v], later [Gam | gam]     (n4 x ld1)
  float* E = Za + (long long)n4 * ld1;         // C'[Z_a | v], later (Z_b Hn)'
  float* F2 = E + (long long)n4 * ld1;         // Y E
  float* pb = F2 + (long long)n4 * ld1;        // p_b
  float* wa = pb + n4;                         // w_a
  float* colbuf = wa + n4;                     // block-elimination scratch (16-byte aligned)
  double* dtail = reinterpret_cast<double*>(colbuf + p4_scratch_floats(n));  // 3 n4 doubles (mode 1 refinement)
  float* rdc = reinterpret_cast<float*>(dtail + 3 * n4);  // 1 / diag(C)

  {
    float4* z4 = reinterpret_cast<float4*>(smem);
    const long long n4f = scan_smem_floats(n, ldn) / 4;
    for (long long i = threadIdx.x; i < n4f; i += blockDim.x) z4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (threadIdx.x == 0) s_flag = 0;
  }
  __syncthreads();
  const double* Pfin = ws + wl.Pi + (long long)b * nn;
  const double* pfin = ws + wl.pi + (long long)b * n;
  for (int e = threadIdx.x; e < (int)nn; e += blockDim.x) {
    const int i = e / n, k = e - i * n;
    Cb[i * ldn + k] = bfin ? static_cast<float>(Pfin[e]) : eb[e];
    Za[i * ld1 + k] = ea[nn + e];
    Wa[i * ldn + k] = ea[2 * nn + e];
    if (!bfin) Zb[i * ldn + k] = eb[nn + e];
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    pb[i] = bfin ? static_cast<float>(pfin[i]) : eb[3 * nn + i];
    wa[i] = ea[3 * nn + n + i];
  }
  __syncthreads();
  // v = w_a - W_a p_b (column n4 of Za); C = chol(P_b)
  cta_mv_warp<float>(n, n, Wa, ldn, pb, [&](int i, float v) { Za[i * ld1 + n4] = v + wa[i]; });
  if (SHAPE == 0) cta_chol_p4<1, 4>(n, Cb, ldn, &s_flag, colbuf, rdc);
  else if (SHAPE == 1) cta_chol_p4<2, 4>(n, Cb, ldn, &s_flag, colbuf, rdc);
  else cta_chol_p4<4, 4>(n, Cb, ldn, &s_flag, colbuf, rdc);
  if (s_flag) {
    if (threadIdx.x == 0) raise_status(pd.status, LQR_ERR_NOT_PD, -1 - j);
    return;
  }
  // Tm = W_a C;  E = C'[Z_a | v]
  cta_mm4f<false>(n4, n4, n4, Wa, ldn, Cb, ldn, [&](int i, int k, float v) { Tm[i * ldn + k] = -v; });
  cta_mm4f<true>(n4, ld1, n4, Cb, ldn, Za, ld1, [&](int i, int k, float v) { E[i * ld1 + k] = v; },
                 (n4 / 4) * (n4 / 4));
  __syncthreads();
  // Y = (I + C'Tm)^-1
  cta_mm4f<true>(n4, n4, n4, Cb, ldn, Tm, ldn,
                 [&](int i, int k, float v) { Y[i * ldn + k] = (i == k && i < n) ? v + 1.0f : v; });
  __syncthreads();
  if (SHAPE == 0) cta_spd_inverse_p4<1, 4>(n, Y, ldn, &s_flag, colbuf, false);
  else if (SHAPE == 1) cta_spd_inverse_p4<2, 4>(n, Y, ldn, &s_flag, colbuf, false);
  else cta_spd_inverse_p4<4, 4>(n, Y, ldn, &s_flag, colbuf, false);
  if (s_flag) {
    if (threadIdx.x == 0) raise_status(pd.status, LQR_ERR_NOT_PD, -1 - j);
    return;
  }
  // F2 = Y E
  cta_mm4f<false>(n4, ld1, n4, Y, ldn, E, ld1, [&](int i, int k, float v) { F2[i * ld1 + k] = v; });
  __syncthreads();
  if (mode == 1) {  // [Gam_j | gam_j] = [Z_j | v] - Tm F2
    // Gam_j (FP32) replaces Z_j in element j of buffer 0, read only by this CTA
    float* G = sbase + (long long)j * es + nn;
    double* g = ws + wl.gam + (long long)j * n;
    double* gd = dtail;  // gam (FP64)
    double* t1 = gd + n4;
    double* gbk = t1 + n4;
    float* rf = pb;      // residual (p_b, w_a no longer needed)
    float* c1 = wa;
    float* c2 = colbuf;
    cta_mm4f<false>(n4, ld1, n4, Tm, ldn, F2, ld1, [&](int i, int k, float v) {
      if (i < n) {
        if (k < n) G[(long long)i * n + k] = Za[i * ld1 + k] - v;
        else if (k == n4) gd[i] = static_cast<double>(Za[i * ld1 + n4] - v);
      }
    });
    __syncthreads();
    // gam = M^-1 v is small next to v (the affine link terms mostly cancel),
    // so its FP32 value is refined: r = v - M gam in FP64 from the stored
    // summary and Pi_{j+1}, pi_{j+1}; gam += M^-1 r with M^-1 applied as
    // C^-T Y C' (no cancellation). A correction is kept only while the
    // residual decreases; at most two.
    const double* Sj = ws + wl.summ + (long long)j * (3 * nn + 2 * n);
    const double* Wn64 = Sj + 2 * nn;
    const double* w64 = Sj + 3 * nn + n;
    const double* Pi1 = ws + wl.Pi + (long long)(j + 1) * nn;
    const double* pi1 = ws + wl.pi + (long long)(j + 1) * n;
    __shared__ double s_wmax[kScanBlock / 32];
    __shared__ double s_rn;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double rprev = INFINITY;
    for (int it = 0; it < 3; ++it) {
      cta_mv_warp<double>(n, n, Pi1, n, gd, [&](int i, double v) { t1[i] = v + pi1[i]; });
      __syncthreads();
      // r = w - W (pi + Pi gam) - gam
      double wmax = 0.0;
      cta_mv_warp<double>(n, n, Wn64, n, t1, [&](int i, double v) {
        const double r = v + w64[i] - gd[i];
        rf[i] = static_cast<float>(r);
        wmax = fmax(wmax, fabs(r));
      });
      if (lane == 0) s_wmax[warp] = wmax;
      __syncthreads();
      if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, s_wmax[w]);
        s_rn = mx;
      }
      __syncthreads();
      const double rn = s_rn;
      if (!(rn < rprev)) {  // no progress: back to the previous iterate
        if (it > 0)
          for (int i = threadIdx.x; i < n; i += blockDim.x) gd[i] = gbk[i];
        __syncthreads();
        break;
      }
      if (it == 2) break;
      rprev = rn;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        gbk[i] = gd[i];
        float a = 0.0f;
        for (int k = 0; k < n; ++k) a = fmaf(Cb[k * ldn + i], rf[k], a);
        c1[i] = a;
      }
      __syncthreads();
      cta_mv_warp<float>(n, n, Y, ldn, c1, [&](int i, float v) { c2[i] = v; });
      __syncthreads();
      cta_trsm_lower_t_warp<float, float>(n, Cb, ldn, 1, c2, 1, rdc);
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) gd[i] += static_cast<double>(c2[i]);
      __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) g[i] = gd[i];
    return;
  }
  // P_ab = P_a + E_Z' F2_Z;  p_ab = p_a + Z_a'p_b + E_Z' F2_v
  double* Pj = ws + wl.Pi + (long long)j * nn;
  double* pj = ws + wl.pi + (long long)j * n;
  cta_mm4f<true>(n4, n4, n4, E, ld1, F2, ld1, [&](int i, int k, float v) {
    if (i < n && k < n) {
      const float r = ea[(long long)i * n + k] + v;
      if (bfin) Pj[(long long)i * n + k] = static_cast<double>(r);
      else ed[(long long)i * n + k] = r;
    }
  });
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float acc = ea[3 * nn + i];
    for (int k = 0; k < n; ++k) acc = fmaf(Za[k * ld1 + i], pb[k], fmaf(E[k * ld1 + i], F2[k * ld1 + n4], acc));
    if (bfin) pj[i] = static_cast<double>(acc);
    else ed[3 * nn + i] = acc;
  }
  if (bfin) return;
  __syncthreads();
  // [Gam | gam] = [Z_a | v] - Tm F2 (in place);  U = Y Tm' (as (Tm Y)', Y symmetric)
  cta_mm4f<false>(n4, ld1, n4, Tm, ldn, F2, ld1, [&](int i, int k, float v) { Za[i * ld1 + k] -= v; });
  cta_mm4f<false>(n4, n4, n4, Tm, ldn, Y, ldn, [&](int i, int k, float v) { Cb[k * ldn + i] = v; },
                  (n4 / 4) * (ld1 / 4));
  __syncthreads();
  // Z_ab = Z_b Gam, w_ab = w_b + Z_b gam;  -(M^-1 W_a) = -W_a + Tm U
  cta_mm4f<false>(n4, ld1, n4, Zb, ldn, Za, ld1, [&](int i, int k, float v) {
    if (i < n) {
      if (k < n) ed[nn + (long long)i * n + k] = v;
      else if (k == n4) ed[3 * nn + n + i] = eb[3 * nn + n + i] + v;
    }
  });
  cta_mm4f<false>(n4, n4, n4, Tm, ldn, Cb, ldn, [&](int i, int k, float v) { Wa[i * ldn + k] += v; },
                  (n4 / 4) * (ld1 / 4));
  __syncthreads();
  // -W_ab = -W_b + Z_b (-(M^-1 W_a)) Z_b': V = Z_b Hn stored transposed, then Z_b V'
  cta_mm4f<false>(n4, n4, n4, Zb, ldn, Wa, ldn, [&](int i, int k, float v) { E[k * ldn + i] = v; });
  __syncthreads();
  cta_mm4f<false>(n4, n4, n4, Zb, ldn, E, ldn, [&](int i, int k, float v) {
    if (i < n && k < n) ed[2 * nn + (long long)i * n + k] = eb[2 * nn + (long long)i * n + k] + v;
  });
}

constexpr int kFwdDepth = 4;  // link feedback matrices in flight

__host__ __device__ inline long long scan_forward_smem_bytes(int n) {
  const long long n4 = (n + 3) & ~3, ldg = n4 + 4;
  return 8 * (2 * n4 + kFwdDepth * n4) + 4 * (2 * n4 + kFwdDepth * n4 * ldg);
}

// The link states: z_0 = x0, z_{j+1} = Gam_j z_j + gam_j. One CTA; the FP32
// Gam_j stream through a ring of kFwdDepth shared-memory slots (cp.async
// issued kFwdDepth-1 links ahead; rows padded to n4 + 4 floats), four threads
// per row form the FP32 product and the refined FP64 gam_j is added in FP64.
__global__ void __launch_bounds__(kBlock) link_scan_forward_kernel(ProbTable tab, int x0_is_float) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_flag;
  const ProbDesc& pd = tab.single;
  if (cta_should_exit(pd, &s_flag)) return;
  const int n = pd.n, K = pd.nseg;
  const int n4 = (n + 3) & ~3, ldg = n4 + 4;
  const long long nn = (long long)n * n, es = scan_elem_floats(n);
  const WsLayout wl = ws_layout(n, K);
  const float* sbase = reinterpret_cast<const float*>(pd.ws + wl.scan);
  double* zd = reinterpret_cast<double*>(smem);  // 2 x n4: z_j (FP64), ping-pong
  double* gr = zd + 2 * n4;                      // kFwdDepth x n4: gam ring
  float* zf = reinterpret_cast<float*>(gr + kFwdDepth * n4);  // 2 x n4: z_j (FP32), zero padded
  float* Gr = zf + 2 * n4;                                     // kFwdDepth x n4 x ldg: Gam ring
  double* z = pd.ws + wl.z;
  const bool rows16 = (n % 4) == 0;  // rows start on 16-byte boundaries in global memory
  auto issue = [&](int j) {
    if (j < K - 1) {
      const float* src = sbase + (long long)j * es + nn;
      float* dst = Gr + (long long)(j % kFwdDepth) * n4 * ldg;
      if (rows16)
        cta_for_rc(n, n / 4, [&](int, int i, int c) {
          cp_async16(dst + (long long)i * ldg + 4 * c, src + (long long)i * n + 4 * c);
        });
      else
        cta_for_rc(n, n, [&](int e, int i, int k) { cp_async4(dst + (long long)i * ldg + k, src + e); });
      const double* gs = pd.ws + wl.gam + (long long)j * n;
      double* gdst = gr + (j % kFwdDepth) * n4;
      for (int i = threadIdx.x; i < n; i += blockDim.x) cp_async8(gdst + i, gs + i);
    }
    cp_async_commit();
  };
  // padding columns of every slot (never copied) and of z stay zero
  for (long long e = threadIdx.x; e < (long long)kFwdDepth * n4 * ldg; e += blockDim.x) Gr[e] = 0.0f;
  for (int i = threadIdx.x; i < 2 * n4; i += blockDim.x) zf[i] = 0.0f;
  __syncthreads();
  for (int j = 0; j < kFwdDepth - 1; ++j) issue(j);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = x0_is_float ? (double)static_cast<const float*>(pd.x0)[i] : static_cast<const double*>(pd.x0)[i];
    zd[i] = v;
    zf[i] = static_cast<float>(v);
    z[i] = v;
  }
  const int q = threadIdx.x & 3;  // quarter of the row
  const int nq = n4 / 4;          // float4 chunks per row, dealt over the 4 threads
  for (int j = 0; j + 1 < K; ++j) {
    cp_async_wait<kFwdDepth - 2>();
    __syncthreads();  // Gam_j, gam_j and z_j visible; slot (j-1) % depth free
    issue(j + kFwdDepth - 1);
    const float* G = Gr + (long long)(j % kFwdDepth) * n4 * ldg;
    const double* g = gr + (j % kFwdDepth) * n4;
    const float* zc = zf + (j & 1) * n4;
    float* zfn = zf + ((j + 1) & 1) * n4;
    double* zdn = zd + ((j + 1) & 1) * n4;
    double* zg = z + (long long)(j + 1) * n;
    for (int base = 0; base < n4; base += (int)(blockDim.x >> 2)) {  // uniform trip count: full-warp shuffles
      const int i = base + (int)(threadIdx.x >> 2);
      float acc = 0.0f;
      if (i < n4)
        for (int c = q; c < nq; c += 4) {
          const float4 gv = *reinterpret_cast<const float4*>(G + (long long)i * ldg + 4 * c);
          const float4 zv = *reinterpret_cast<const float4*>(zc + 4 * c);
          acc = fmaf(gv.x, zv.x, fmaf(gv.y, zv.y, fmaf(gv.z, zv.z, fmaf(gv.w, zv.w, acc))));
        }
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if (q == 0 && i < n) {
        const double v = static_cast<double>(acc) + g[i];
        zdn[i] = v;
        zfn[i] = static_cast<float>(v);
        zg[i] = v;
      }
    }
  }
  cp_async_wait<0>();
}

size_t link_scan_smem_bytes(int n) { return sizeof(float) * (size_t)scan_smem_floats(n, (n + 3) & ~3); }

// levels: the scan levels (true) or the feedback pass (false)
template <int SHAPE>
static cudaError_t launch_scan_levels(const ProbTable& tab, size_t bytes, int ldn, cudaStream_t st, bool levels) {
  const int K = tab.single.nseg;
  cudaError_t e = raise_dyn_smem((const void*)link_scan_kernel<SHAPE>, bytes);
  if (e != cudaSuccess) return e;
  if (levels) {
    int src = 0, dst = 1;
    for (int s = 1; s < K; s *= 2) {
      link_scan_kernel<SHAPE><<<K - s, kScanBlock, bytes, st>>>(tab, s, 0, src, dst, ldn);
      src = dst;
      dst = (dst == 1) ? 2 : 1;
    }
  } else {
    link_scan_kernel<SHAPE><<<K - 1, kScanBlock, bytes, st>>>(tab, 1, 1, 0, 0, ldn);
  }
  return cudaGetLastError();
}

// Returns cudaErrorNotSupported (nothing launched) when the shape does not fit.
// part: 0 = the whole solve; 1 = the summaries' conversion and the levels (Pi_j,
// pi_j final afterwards); 2 = the feedback pass and the link states.
cudaError_t launch_link_scan(const ProbTable& tab, int x0_is_float, cudaStream_t st, int* launches, int part) {
  const int n = tab.single.n, K = tab.single.nseg;
  if (K < 2 || tab.probs) return cudaErrorNotSupported;
  int optin = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int n4 = (n + 3) & ~3;
  int ldn = n4 + 4;
  if (sizeof(float) * (size_t)scan_smem_floats(n, ldn) > (size_t)optin - kStaticSmemReserve) ldn = n4;
  const size_t bytes = sizeof(float) * (size_t)scan_smem_floats(n, ldn);
  const int shape = p4_shape(n);
  if (bytes > (size_t)optin - kStaticSmemReserve || shape < 0 || shape > 2 ||
      (size_t)scan_forward_smem_bytes(n) > (size_t)optin - kStaticSmemReserve)
    return cudaErrorNotSupported;
  int lv = 0;
  for (int s = 1; s < K; s *= 2) ++lv;
  int nl = 0;
  cudaError_t e = cudaSuccess;
  if (part != 2) {
    link_scan_init_kernel<<<K, kBlock, 0, st>>>(tab);
    e = shape == 0 ? launch_scan_levels<0>(tab, bytes, ldn, st, true)
        : shape == 1 ? launch_scan_levels<1>(tab, bytes, ldn, st, true)
                     : launch_scan_levels<2>(tab, bytes, ldn, st, true);
    if (e != cudaSuccess) return e;
    nl += 1 + lv;
  }
  if (part != 1) {
    e = shape == 0 ? launch_scan_levels<0>(tab, bytes, ldn, st, false)
        : shape == 1 ? launch_scan_levels<1>(tab, bytes, ldn, st, false)
                     : launch_scan_levels<2>(tab, bytes, ldn, st, false);
    if (e != cudaSuccess) return e;
    const size_t fbytes = (size_t)scan_forward_smem_bytes(n);
    e = raise_dyn_smem((const void*)link_scan_forward_kernel, fbytes);
    if (e != cudaSuccess) return e;
    link_scan_forward_kernel<<<1, kBlock, fbytes, st>>>(tab, x0_is_float);
    nl += 2;
  }
  if (launches) *launches = nl;
  return cudaGetLastError();
}

}  // namespace lqr
