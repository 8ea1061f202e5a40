// Step A4 (the policy sweep of Section III-A, started from the global value
// function at each segment end) with the stage products on the fifth-
// generation tensor cores: tcgen05.mma of kind::tf32 with FP32 accumulators
// in tensor memory, for 64 < n <= 128 and m <= 64 (padded to 128 and 64 with
// zeros). Per stage t, with V = V_{t+1}:
//   alpha  T1' = [A|B]' V                     two 128-row tiles (rows 0..127 and
//                                             64..191 of [A|B]') into TMEM
//   beta   [A'VA | A'VB] = (A'V) [A|B]        A operand from TMEM; B'VB from the
//          B'VB = (B'V) B                     second tile's rows 64..127
//   factor M_uu = R + B'VB: FP64 Cholesky L, FP32 L^-1, M_uu^-1 = L^-T L^-1
//   P4     H_x' = M_ux' M_uu^-1               (M_ux' = S' + A'VB)
//   P5     A'VA <- A'VA - M_ux' H_x           in place, negated A
//   V_t = Q + A'VA - M_ux' H_x (symmetrised), v_t = m_x - M_ux' h,
//   h = M_uu^-1 m_u, K_t = -H_x, k_t = -h, with the vectors (V c + v, m_x, m_u)
//   on the CUDA cores beside the tensor-core work.
// The next stage's [A|B] is copied, transposed element by element (4-byte
// cp.async), into the K-major operand tile while the factor runs.
// One 512-thread CTA per segment, all of tensor memory (512 columns).
#include <cuda_runtime.h>
#include <stdint.h>

#include "cta_linalg.cuh"
#include "lqr_internal.cuh"
#include "tc_sm100.cuh"

namespace lqr {

namespace {

constexpr int kTcBlock = 512;
constexpr int NP = 128, MP = 64, NMP = NP + MP;  // padded n, m
constexpr long long kTcSpin = 1LL << 26;         // polls of a completion wait (32 ns apart) before LQR_ERR_TIMEOUT

// Shared-memory plan (bytes from a 1024-byte-aligned base).
constexpr uint32_t kOffAB = 0;                       // [A|B]': 192 rows x 128 K, swizzled
constexpr uint32_t kOffV = kOffAB + NMP * NP * 4;    // V: 128 x 128 K, swizzled
constexpr uint32_t kOffMux = kOffV;                  // M_ux': 128 x 64 K (after alpha)
constexpr uint32_t kOffHx = kOffV + NP * MP * 4;     // H_x': 128 x 64 K (after P4)
constexpr uint32_t kOffL64 = kOffHx;                 // FP64 M_uu / L, 64 x 64 (before P4)
constexpr uint32_t kOffMinv = kOffV + NP * NP * 4;   // M_uu^-1: 64 x 64 K, swizzled
constexpr uint32_t kOffX = kOffMinv + MP * MP * 4;   // L^-1 FP32, 64 x 64 plain
constexpr uint32_t kOffVec = kOffX + MP * MP * 4;    // vectors
constexpr int kVecFloats = 8 * NP;
constexpr uint32_t kSmemBytes = kOffVec + kVecFloats * 4 + 1024;  // + alignment slack

// TMEM columns
constexpr uint32_t kTRa = 0, kTRb = 128, kTAA = 256, kTBB = 448, kTH = 0;

// Waits for the next completion of the mbarrier; the phase advances only when
// it arrived, so that after a timeout `phase` still names the pending one.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t& phase, long long limit) {
  const bool ok = tc::mbar_wait(bar, phase & 1u, limit);
  if (ok) ++phase;
  tc::fence_after_sync();
  return ok;
}

// X = L^-1 (lower, FP32, leading dimension ldx) of the FP64 Cholesky factor L
// (leading dimension ldl, rd[i] = 1 / L[i][i]): the factor is converted to
// FP32 once into Lf (every conversion from FP64 takes the FP64 pipe), then
// L X = I is solved row by row with all threads, each step scaling row k and
// downdating the rows below it. Ends with a barrier.
__device__ inline void trinv_f64_to_f32(int d, const double* L, int ldl, const double* rd, float* Lf, float* rdf,
                                        float* X, int ldx) {
  const int t = threadIdx.x, nthr = blockDim.x;
  for (int e = t; e < d * d; e += nthr) {
    const int i = e / d, k = e - i * d;
    Lf[i * ldx + k] = k < i ? (float)L[i * ldl + k] : 0.0f;
    X[i * ldx + k] = (i == k) ? 1.0f : 0.0f;
  }
  for (int i = t; i < d; i += nthr) rdf[i] = (float)rd[i];
  __syncthreads();
  // thread -> (row offset t / 64, column t % 64): 8 rows of 64 columns per pass
  const int c = t & 63, r0 = t >> 6, rstep = nthr >> 6;
  for (int k = 0; k < d; ++k) {
    if (r0 == 0 && c <= k) X[k * ldx + c] *= rdf[k];
    __syncthreads();
    if (c <= k) {
      const float xk = X[k * ldx + c];
      for (int i = k + 1 + r0; i < d; i += rstep) X[i * ldx + c] = fmaf(-Lf[i * ldx + k], xk, X[i * ldx + c]);
    }
    __syncthreads();
  }
}

}  // namespace

bool tc_sweep_supported(int n, int m) { return n > 64 && n <= NP && m >= 1 && m <= MP; }

__global__ void __launch_bounds__(kTcBlock, 1) seg_sweep_tc_kernel(ProbTable tab, int store_P, long long spin) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t s_bar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_flag;
  __shared__ double s_rd[MP];
  const int unit = blockIdx.x;
  const ProbDesc& pd = prob_of_unit(tab, unit);
  const int seg = unit - pd.unit0;
  const int n = pd.n, m = pd.m, T = pd.T, K = pd.nseg;
  if (seg >= K - 1) return;  // the policy sweep covers segments 0 .. K-2
  if (cta_should_exit(pd, &s_flag)) return;
  const int t0 = seg_begin(T, K, seg), t1 = seg_begin(T, K, seg + 1);
  unsigned char* smem = smem_raw + ((1024u - (tc::smem_addr(smem_raw) & 1023u)) & 1023u);
  float* sAB = reinterpret_cast<float*>(smem + kOffAB);
  float* sV = reinterpret_cast<float*>(smem + kOffV);
  float* sMux = reinterpret_cast<float*>(smem + kOffMux);
  float* sHx = reinterpret_cast<float*>(smem + kOffHx);
  double* L64 = reinterpret_cast<double*>(smem + kOffL64);
  float* sMinv = reinterpret_cast<float*>(smem + kOffMinv);
  float* X = reinterpret_cast<float*>(smem + kOffX);
  float* vec = reinterpret_cast<float*>(smem + kOffVec);
  float* vx = vec;            // v_{t+1} -> v_t
  float* T1c = vec + NP;      // V c + v
  float* mx = vec + 2 * NP;   // m_x
  float* mu = vec + 3 * NP;   // m_u (64)
  float* hv = mu + MP;        // h (64)
  float* cs = vec + 4 * NP;   // c_t
  float* qs = vec + 5 * NP;   // q_t
  float* rs = vec + 6 * NP;   // r_t (64)
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int quad = warp & 3, grp = warp >> 2;  // TMEM lane quadrant, column group
  const float* gA = static_cast<const float*>(pd.A);
  const float* gB = static_cast<const float*>(pd.B);
  const float* gc = static_cast<const float*>(pd.c);
  const float* gQ = static_cast<const float*>(pd.Q);
  const float* gR = static_cast<const float*>(pd.R);
  const float* gS = static_cast<const float*>(pd.S);
  const float* gq = static_cast<const float*>(pd.q);
  const float* gr = static_cast<const float*>(pd.r);
  float* gK = static_cast<float*>(pd.K);
  float* gk = static_cast<float*>(pd.k);
  float* gP = static_cast<float*>(pd.P);
  float* gp = static_cast<float*>(pd.p);
  const long long nn = (long long)n * n, nm = (long long)n * m, mm = (long long)m * m;
  const WsLayout wl = ws_layout(n, K);

  // ---- set-up: zero the operand tiles (padding stays zero), TMEM, mbarrier ----
  for (uint32_t e = t; e < (kOffVec + kVecFloats * 4) / 16; e += kTcBlock)
    reinterpret_cast<float4*>(smem)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (warp == 0) tc::tmem_alloc(&s_tmem, 512);
  if (t == 0) {
    tc::mbar_init(&s_bar, 1);
    tc::mbar_fence_init();
    s_flag = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = s_tmem;
  const uint32_t lane_base = tm + ((uint32_t)(32 * quad) << 16);
  const uint32_t aAB = tc::smem_addr(sAB), aV = tc::smem_addr(sV), aMux = tc::smem_addr(sMux),
                 aHx = tc::smem_addr(sHx), aMinv = tc::smem_addr(sMinv);
  uint32_t phase = 0;
  int fail = 0;     // 0, LQR_ERR_TIMEOUT or LQR_ERR_NOT_PD (CTA-uniform once decided)
  int my_wait = 0;  // this thread's own wait ran out

  // stage data of stage s: [A|B]' element by element into the K-major tile
  // (lane -> 8 rows x 4 K positions of one 32-wide K block: conflict-free
  // shared stores, 32-byte global segments), c, q, r into their vectors
  auto issue_stage = [&](int s) {
    const float* A = gA + nn * s;
    const float* B = gB + nm * s;
    // work items: (row group of 8 rows of [A|B]', K group of 4): rows 0..n-1 of A', 128..128+m-1 of B'
    const int kgroups = (n + 3) >> 2;
    const int rgA = (n + 7) >> 3, rgB = (m + 7) >> 3;
    const int items = (rgA + rgB) * kgroups;
    for (int it = warp; it < items; it += kTcBlock / 32) {
      const int rg = it / kgroups, kg = it - rg * kgroups;
      const bool isA = rg < rgA;
      const int r = (isA ? rg * 8 : NP + (rg - rgA) * 8) + (lane & 7);
      const int col = isA ? r : r - NP;  // column of A or B
      const int k = kg * 4 + (lane >> 3);
      const bool ok = isA ? (col < n && k < n) : (col < m && k < n);
      if (ok) {
        float* dst = &tc::sw_at(sAB, NMP, r, k);
        const float* src = isA ? (A + (long long)k * n + col) : (B + (long long)k * m + col);
        cp_async4(dst, src);
      }
    }
    for (int i = t; i < n; i += kTcBlock) {
      cp_async4(cs + i, gc + (long long)n * s + i);
      cp_async4(qs + i, gq + (long long)n * s + i);
    }
    for (int a = t; a < m; a += kTcBlock) cp_async4(rs + a, gr + (long long)m * s + a);
    cp_async_commit();
  };

  // ---- initial value function: the global one at the segment end ----------------
  {
    const double* Pi = pd.ws + wl.Pi + (long long)(seg + 1) * nn;
    const double* pi = pd.ws + wl.pi + (long long)(seg + 1) * n;
    for (long long e = t; e < nn; e += kTcBlock) {
      const int i = (int)(e / n), j = (int)(e - (long long)i * n);
      tc::sw_at(sV, NP, i, j) = static_cast<float>(Pi[e]);
    }
    for (int i = t; i < n; i += kTcBlock) vx[i] = static_cast<float>(pi[i]);
  }
  __syncthreads();
  issue_stage(t1 - 1);

  for (int st = t1 - 1; st >= t0; --st) {
    cp_async_wait<0>();
    tc::fence_proxy_async();
    __syncthreads();  // [A|B]'_t, c, q, r and V in place
    // ---- alpha: T1' = [A|B]' V (two 128-row tiles) ---------------------------------
    if (t == 0) {
      tc::fence_after_sync();
      for (int s = 0; s < NP / 8; ++s) {
        const uint64_t bV = tc::sdesc_k(aV, NP, s);
        tc::mma_ss(tm + kTRa, tc::sdesc_k(aAB, NMP, s), bV, tc::idesc_tf32(128, 128, false), s > 0);
        tc::mma_ss(tm + kTRb, tc::sdesc_k(aAB + 64 * 128, NMP, s), bV, tc::idesc_tf32(128, 128, false), s > 0);
      }
      tc::commit(&s_bar);
    }
    // T1c = V c + v (warp per row, lanes over K: 4 consecutive K positions each)
    for (int i = warp; i < n; i += kTcBlock / 32) {
      const float4 v4 = *reinterpret_cast<const float4*>(
          reinterpret_cast<const unsigned char*>(sV) + tc::sw_off(NP, i, 4 * lane));
      const int k = 4 * lane;
      float a = v4.x * cs[k] + v4.y * cs[k + 1] + v4.z * cs[k + 2] + v4.w * cs[k + 3];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) T1c[i] = a + vx[i];
    }
    __syncthreads();
    // m_x = q + A'T1c, m_u = r + B'T1c (rows of [A|B]')
    for (int r = warp; r < NP + m; r += kTcBlock / 32) {
      if (r >= n && r < NP) continue;
      const float4 a4 = *reinterpret_cast<const float4*>(
          reinterpret_cast<const unsigned char*>(sAB) + tc::sw_off(NMP, r, 4 * lane));
      const int k = 4 * lane;
      float a = a4.x * T1c[k] + a4.y * T1c[k + 1] + a4.z * T1c[k + 2] + a4.w * T1c[k + 3];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) {
        if (r < NP) mx[r] = a + qs[r];
        else mu[r - NP] = a + rs[r - NP];
      }
    }
    if (!wait_phase(&s_bar, phase, spin)) my_wait = 1;
    if (__syncthreads_or(my_wait)) {
      fail = LQR_ERR_TIMEOUT;
      break;
    }
    // ---- beta: [A'VA | A'VB] = (A'V)[A|B],  B'VB = (B'V) B ------------------------------
    if (t == 0) {
      for (int s = 0; s < NP / 8; ++s) {
        tc::mma_ts(tm + kTAA, tm + kTRa + 8 * s, tc::sdesc_k(aAB, NMP, s), tc::idesc_tf32(128, NMP, false), s > 0);
        tc::mma_ts(tm + kTBB, tm + kTRb + 8 * s, tc::sdesc_k(aAB + NP * 128, NMP, s), tc::idesc_tf32(128, MP, false),
                   s > 0);
      }
      tc::commit(&s_bar);
    }
    if (!wait_phase(&s_bar, phase, spin)) my_wait = 1;
    if (__syncthreads_or(my_wait)) {
      fail = LQR_ERR_TIMEOUT;
      break;
    }
    // M_uu = R + B'VB (rows of TMEM lanes 64..127) into FP64; M_ux' = S' + A'VB
    if (quad >= 2) {
      float v[16];
      tc::tmem_ld16(lane_base + kTBB + 16 * grp, v);
      const int a = 32 * (quad - 2) + lane;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int b = 16 * grp + q;
        // R read transposed (coalesced over the lanes): M_uu is symmetrised below
        double val = (a < m && b < m) ? (double)(v[q] + gR[mm * st + (long long)b * m + a]) : 0.0;
        L64[a * MP + b] = val;
      }
    }
    {
      float v[16];
      tc::tmem_ld16(lane_base + kTAA + NP + 16 * grp, v);
      const int j = 32 * quad + lane;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int a = 16 * grp + q;
        float val = v[q];
        if (gS && j < n && a < m) val += gS[nm * st + (long long)a * n + j];
        tc::sw_at(sMux, NP, j, a) = (j < n && a < m) ? val : 0.0f;
      }
    }
    tc::fence_before_sync();
    tc::fence_proxy_async();
    __syncthreads();
    // the next stage's data into the free operand tile while the factor runs
    if (st - 1 >= t0) issue_stage(st - 1);
    // M_uu symmetrised, factored in FP64
    for (int e = t; e < m * m; e += kTcBlock) {
      const int a = e / m, b = e - a * m;
      if (b < a) {
        const double s = 0.5 * (L64[a * MP + b] + L64[b * MP + a]);
        L64[a * MP + b] = s;
        L64[b * MP + a] = s;
      }
    }
    if (t == 0) s_flag = 0;
    __syncthreads();
    cta_chol(m, L64, MP, &s_flag, s_rd);
    if (s_flag) {
      if (t == 0) raise_status(pd.status, LQR_ERR_NOT_PD, st);
      fail = LQR_ERR_NOT_PD;
      break;
    }
    // M_uu^-1 = L^-T L^-1 (FP32), into the swizzled operand tile and, when kept, to global
    // (the M_uu^-1 tile holds the FP32 copy of the factor until it is overwritten below)
    trinv_f64_to_f32(m, L64, MP, s_rd, sMinv, vec + 7 * NP, X, MP);
    {
      float* gM = pd.Minv ? static_cast<float*>(pd.Minv) + mm * st : nullptr;
      // over the padded 64 x 64 tile: rows and columns of X beyond m are zero
      cta_mm<4, 4, true, false, float>(MP, MP, m, X, MP, X, MP, [&](int i, int j, float v) {
        tc::sw_at(sMinv, MP, i, j) = v;
        if (gM && i < m && j < m) gM[(long long)i * m + j] = v;
      });
    }
    tc::fence_proxy_async();
    __syncthreads();
    // ---- P4: H_x' = M_ux' M_uu^-1 ----------------------------------------------------------
    if (t == 0) {
      tc::fence_after_sync();
      for (int s = 0; s < MP / 8; ++s)
        tc::mma_ss(tm + kTH, tc::sdesc_k(aMux, NP, s), tc::sdesc_k(aMinv, MP, s), tc::idesc_tf32(128, MP, false),
                   s > 0);
      tc::commit(&s_bar);
    }
    // h = M_uu^-1 m_u, k_t = -h
    for (int a = warp; a < m; a += kTcBlock / 32) {
      float s = 0.0f;
      for (int b = lane; b < m; b += 32) s = fmaf(tc::sw_get(sMinv, MP, a, b), mu[b], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        hv[a] = s;
        if (gk) gk[(long long)m * st + a] = -s;
      }
    }
    __syncthreads();
    // v_t = m_x - M_ux' h
    for (int i = warp; i < n; i += kTcBlock / 32) {
      float s = 0.0f;
      for (int a = lane; a < m; a += 32) s = fmaf(tc::sw_get(sMux, NP, i, a), hv[a], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) vx[i] = mx[i] - s;
    }
    if (!wait_phase(&s_bar, phase, spin)) my_wait = 1;
    if (__syncthreads_or(my_wait)) {
      fail = LQR_ERR_TIMEOUT;
      break;
    }
    // H_x' into its operand tile (the FP64 factor is done), K_t = -H_x
    {
      float v[16];
      tc::tmem_ld16(lane_base + kTH + 16 * grp, v);
      const int j = 32 * quad + lane;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int a = 16 * grp + q;
        tc::sw_at(sHx, NP, j, a) = v[q];
        if (gK && j < n && a < m) gK[nm * st + (long long)a * n + j] = -v[q];
      }
    }
    tc::fence_before_sync();
    tc::fence_proxy_async();
    __syncthreads();
    // ---- P5: A'VA - M_ux' H_x (in place, negated A) ------------------------------------------
    if (t == 0) {
      tc::fence_after_sync();
      for (int s = 0; s < MP / 8; ++s)
        tc::mma_ss(tm + kTAA, tc::sdesc_k(aMux, NP, s), tc::sdesc_k(aHx, NP, s), tc::idesc_tf32(128, NP, true), 1);
      tc::commit(&s_bar);
    }
    if (!wait_phase(&s_bar, phase, spin)) my_wait = 1;
    if (__syncthreads_or(my_wait)) {
      fail = LQR_ERR_TIMEOUT;
      break;
    }
    // V_t = Q + (A'VA - M_ux' H_x), then symmetrised
    {
      const int i = 32 * quad + lane;
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        float v[16];
        const int j0 = 32 * grp + 16 * h2;
        tc::tmem_ld16(lane_base + kTAA + j0, v);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int j = j0 + q;
          // Q read transposed (coalesced over the lanes): V_t is symmetrised below
          const float qv = (i < n && j < n) ? gQ[nn * st + (long long)j * n + i] : 0.0f;
          tc::sw_at(sV, NP, i, j) = (i < n && j < n) ? v[q] + qv : 0.0f;
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    for (int e = t; e < n * n; e += kTcBlock) {
      const int i = e / n, j = e - i * n;
      if (j > i) {
        float& a = tc::sw_at(sV, NP, i, j);
        float& b = tc::sw_at(sV, NP, j, i);
        const float s = 0.5f * (a + b);
        a = s;
        b = s;
      }
    }
    if (store_P && gP) {
      __syncthreads();
      for (long long e = t; e < nn; e += kTcBlock) {
        const int i = (int)(e / n), j = (int)(e - (long long)i * n);
        gP[nn * st + e] = tc::sw_get(sV, NP, i, j);
      }
      for (int i = t; i < n; i += kTcBlock) gp[(long long)n * st + i] = vx[i];
    }
  }
  // ---- clean-up: a failed wait gets one more bounded wait for the tensor core -------
  if (fail == LQR_ERR_TIMEOUT) {
    if (t == 0) raise_status(pd.status, LQR_ERR_TIMEOUT, -1);
    // the threads whose wait ran out wait once more, with the default limit, for
    // the pending products (a thread that saw them complete has nothing pending)
    if (my_wait) tc::mbar_wait(&s_bar, phase & 1u, kTcSpin);
  }
  cp_async_wait<0>();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tm, 512);
}

cudaError_t launch_seg_sweep_tc(const ProbTable& tab, int nunits, int store_P, long long spin_limit, cudaStream_t st) {
  cudaError_t e = raise_dyn_smem((const void*)seg_sweep_tc_kernel, kSmemBytes);
  if (e != cudaSuccess) return e;
  seg_sweep_tc_kernel<<<nunits, kTcBlock, kSmemBytes, st>>>(tab, store_P, spin_limit > 0 ? spin_limit : kTcSpin);
  return cudaGetLastError();
}

}  // namespace lqr
