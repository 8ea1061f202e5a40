// Segment sweeps: step A1 (the constraint-explicit backward sweep of Section
// II-B with the segment end state x_term as a parameter, Eq. 9-16) and step A4
// (the exact smoothing sweep of Section III-A started from the global value
// function at the segment end). One CTA per segment; the segment's value
// function stays on chip across its stages while the stage data streams
// through shared memory.
#include <cuda_runtime.h>

#include "lqr_internal.cuh"

namespace lqr {

namespace {

// Stage term T1 = Vxx [A|B|c] with v_x added to the last column (-> V_xx c + v_x).
template <typename TC>
struct EpiT1 {
  TC* T1; int ld; const TC* vx; int lastcol;
  template <typename T>
  __device__ __forceinline__ void operator()(int i, int j, T v) const {
    if (j == lastcol) v += static_cast<T>(vx[i]);
    T1[(size_t)i * ld + j] = static_cast<TC>(v);
  }
};

// Scatter of N = H_x [A|B|c] (r x (n+m+1)) into [N_u | N_x | N_z | n_1] with n_1 += h.
struct EpiAug {
  double* aug; int ldaug; int n, m; const double* H; int ldH;
  __device__ __forceinline__ void operator()(int i, int j, double v) const {
    if (j < n) {
      aug[(size_t)i * ldaug + m + j] = v;
    } else if (j < n + m) {
      aug[(size_t)i * ldaug + (j - n)] = v;
    } else {
      aug[(size_t)i * ldaug + m + 2 * n] = v + H[(size_t)i * ldH + 2 * n];
    }
  }
};

template <typename TC>
__device__ __forceinline__ void cta_copy(int rows, int cols, const TC* src, int lds, TC* dst, int ldd) {
  for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
    const int i = e / cols, j = e % cols;
    dst[(size_t)i * ldd + j] = src[(size_t)i * lds + j];
  }
}

template <typename TC>
__device__ __forceinline__ void cta_symmetrize(int n, TC* V, int ld) {
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    if (j <= i) continue;
    const TC a = TC(0.5) * (V[(size_t)i * ld + j] + V[(size_t)j * ld + i]);
    V[(size_t)i * ld + j] = a;
    V[(size_t)j * ld + i] = a;
  }
}

constexpr int RMg = 4, RNg = 4;  // register tile of the stage products

}  // namespace

// grid: one CTA per (problem, segment) unit; block: kBlock threads.
// phase 0 = A1: segments j < K-1 run the parametric sweep (MODE_PARAM) and
//               segment K-1 the terminal Riccati sweep (MODE_TERMINAL);
// phase 1 = A4: segments j < K-1 run MODE_POLICY from (Pi_{j+1}, pi_{j+1});
//               segment K-1 has nothing to do.
template <typename TS, typename TC>
__global__ void __launch_bounds__(kBlock) seg_sweep_kernel(ProbTable tab, int phase, long long smem_budget,
                                                           int store_P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_flag;
  __shared__ double s_scal[4];
  __shared__ double s_rd[256];   // 1 / L[i][i] of the current FP64 factor
  __shared__ TC s_rdc[256];      // the same in the compute type
  __shared__ float s_pivf[512];  // pivot scratch of the FP32 factorisation

  const int unit = blockIdx.x;
  const ProbDesc& pd = prob_of_unit(tab, unit);
  const int seg = unit - pd.unit0;
  const int n = pd.n, m = pd.m, T = pd.T, K = pd.nseg;
  if (cta_should_exit(pd, &s_flag)) return;  // an earlier step failed or the correction is not needed
  const bool last = (seg == K - 1);
  int mode;
  if (phase == 0) {
    mode = last ? MODE_TERMINAL : MODE_PARAM;
  } else {
    if (last) return;
    mode = MODE_POLICY;
  }
  const bool param = (mode == MODE_PARAM);
  const bool cons = param && (pd.form == LQR_FORM_CONSTRAINED);
  const int t0 = seg_begin(T, K, seg), t1 = seg_begin(T, K, seg + 1);

  SweepPlan P;
  make_plan(P, n, m, mode, (int)sizeof(TC), smem_budget, pd.form == LQR_FORM_CONSTRAINED);
  unsigned char* scratch = reinterpret_cast<unsigned char*>(pd.scratch + (long long)seg * pd.scratch_per_unit);
  TC* Vxx = plan_ptr<TC>(P, SB_VXX, smem, scratch);
  TC* AB = plan_ptr<TC>(P, SB_AB, smem, scratch);
  TC* T1 = plan_ptr<TC>(P, SB_T1, smem, scratch);
  TC* F = plan_ptr<TC>(P, SB_F, smem, scratch);
  TC* Muu = plan_ptr<TC>(P, SB_MUU, smem, scratch);
  double* L64 = (sizeof(TC) == 8) ? reinterpret_cast<double*>(Muu) : plan_ptr<double>(P, SB_L64, smem, scratch);
  TC* vec = plan_ptr<TC>(P, SB_VEC, smem, scratch);
  TC* Wbuf = (sizeof(TC) == 8) ? F : plan_ptr<TC>(P, SB_W, smem, scratch);
  TC* vx = vec;
  TC* vz = vec + n;
  TC* mz = vec + 2 * n;
  TC* Vzx = param ? plan_ptr<TC>(P, SB_VZX, smem, scratch) : nullptr;
  TC* Vzz = param ? plan_ptr<TC>(P, SB_VZZ, smem, scratch) : nullptr;
  double* HH = cons ? plan_ptr<double>(P, SB_HH, smem, scratch) : nullptr;
  double* Gc = cons ? plan_ptr<double>(P, SB_G, smem, scratch) : nullptr;
  double* Ec = cons ? plan_ptr<double>(P, SB_E, smem, scratch) : nullptr;
  double* H = cons ? plan_ptr<double>(P, SB_H, smem, scratch) : nullptr;
  double* AUG = cons ? plan_ptr<double>(P, SB_AUG, smem, scratch) : nullptr;
  const int ldAB = P.ldAB, ldF = P.ldF, ldG = P.ldG, ldH = P.ldH;
  const int cmu = ldF - 1;  // column of m_u in F

  const WsLayout wl = ws_layout(n, K);
  double* summ = pd.ws + wl.summ + (long long)seg * (3LL * n * n + 2 * n);
  double* Vzz_g = summ + 2LL * n * n;  // the summary slot of V_zz (written at the end)

  const TS* gA = static_cast<const TS*>(pd.A);
  const TS* gB = static_cast<const TS*>(pd.B);
  const TS* gc = static_cast<const TS*>(pd.c);
  const TS* gQ = static_cast<const TS*>(pd.Q);
  const TS* gR = static_cast<const TS*>(pd.R);
  const TS* gS = static_cast<const TS*>(pd.S);
  const TS* gq = static_cast<const TS*>(pd.q);
  const TS* gr = static_cast<const TS*>(pd.r);
  TS* gK = static_cast<TS*>(pd.K);
  TS* gk = static_cast<TS*>(pd.k);
  TS* gP = static_cast<TS*>(pd.P);
  TS* gp = static_cast<TS*>(pd.p);
  const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm = (size_t)m * m;

  // ---- initial value function at the segment end --------------------------
  int rr = 0;  // rows of constraint_to_go still to absorb (uniform)
  if (mode == MODE_PARAM && cons) {
    // Eq. 11 without the terminal cost: V = 0, v = 0, H_x = I, H_z = -I, h = 0
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      Vxx[e] = TC(0);
      Vzx[e] = TC(0);
      Vzz[e] = TC(0);
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) { vx[i] = TC(0); vz[i] = TC(0); }
    for (int e = threadIdx.x; e < n * ldH; e += blockDim.x) {
      const int i = e / ldH, j = e % ldH;
      H[e] = (j == i) ? 1.0 : ((j == n + i) ? -1.0 : 0.0);
    }
    rr = n;
  } else if (mode == MODE_PARAM) {
    // dual form: value of (segment cost + mu'x_end) at the segment end is mu'x:
    // P = 0, Z (the V_zx slot) = I, -W (the V_zz slot) = 0, p = 0, w (the v_z slot) = 0.
    // Every stage is then a plain stage of the same recursion (Z <-> V_zx, -W <-> V_zz).
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      Vxx[e] = TC(0);
      Vzx[e] = (e / n == e % n) ? TC(1) : TC(0);
      Vzz[e] = TC(0);
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) { vx[i] = TC(0); vz[i] = TC(0); }
    rr = 0;
  } else if (mode == MODE_TERMINAL) {
    const TS* QT = gQ + nn * T;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e / n, j = e % n;
      Vxx[e] = static_cast<TC>(0.5 * (static_cast<double>(QT[(size_t)i * n + j]) +
                                      static_cast<double>(QT[(size_t)j * n + i])));
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) vx[i] = static_cast<TC>(gq[(size_t)n * T + i]);
  } else if (pd.smooth) {
    // the smoothing pass of Section III-A: the next segment's cost to go at its
    // start with its own end pinned at its link point, J_{j+1}(x, z_{j+2}):
    // V = Vxx^{j+1}, v = vx^{j+1} + Vzx^{j+1}' z_{j+2} (the last segment: its value)
    const double* S1 = pd.ws + wl.summ + (long long)(seg + 1) * (3LL * n * n + 2 * n);
    const double* z2 = pd.ws + wl.z + (long long)(seg + 2) * n;
    const bool pinned = seg + 1 < K - 1;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) Vxx[e] = static_cast<TC>(S1[e]);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double a = S1[3 * nn + i];
      if (pinned)
        for (int k = 0; k < n; ++k) a += S1[nn + (size_t)k * n + i] * z2[k];
      vx[i] = static_cast<TC>(a);
    }
  } else {
    const double* Pi = pd.ws + wl.Pi + (long long)(seg + 1) * nn;
    const double* pi = pd.ws + wl.pi + (long long)(seg + 1) * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) Vxx[e] = static_cast<TC>(Pi[e]);
    for (int i = threadIdx.x; i < n; i += blockDim.x) vx[i] = static_cast<TC>(pi[i]);
  }
  __syncthreads();
  if (store_P && gP && mode != MODE_PARAM && last) {  // P_T, p_T
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) gP[nn * T + e] = static_cast<TS>(Vxx[e]);
    for (int i = threadIdx.x; i < n; i += blockDim.x) gp[(size_t)n * T + i] = static_cast<TS>(vx[i]);
  }

  bool failed = false;
  for (int t = t1 - 1; t >= t0; --t) {
    // with the per-stage reconstruction, the policy sweep only covers the stages
    // whose constraint_to_go still has rows (the end of the segment)
    if (mode == MODE_POLICY && pd.stage_rank && pd.stage_rank[t] == 0) break;
    // ---- (1) stage the dynamics [A_t | B_t | c_t] ---------------------------
    {
      const TS* At = gA + nn * t;
      const TS* Bt = gB + nm * t;
      const TS* ct = gc + (size_t)n * t;
      for (int e = threadIdx.x; e < n * n; e += blockDim.x) AB[(size_t)(e / n) * ldAB + (e % n)] = static_cast<TC>(At[e]);
      for (int e = threadIdx.x; e < n * m; e += blockDim.x) AB[(size_t)(e / m) * ldAB + n + (e % m)] = static_cast<TC>(Bt[e]);
      for (int i = threadIdx.x; i < n; i += blockDim.x) AB[(size_t)i * ldAB + n + m] = static_cast<TC>(ct[i]);
    }
    __syncthreads();
    // ---- (2) T1 = V_xx [A|B|c] + [0|0|v_x] -----------------------------------
    cta_mm<RMg, RNg, false, false, TC>(n, ldAB, n, Vxx, n, AB, ldAB, EpiT1<TC>{T1, ldAB, vx, n + m});
    __syncthreads();
    // ---- (3) the M terms of Eq. 13 (with the affine and parameter terms) ------
    {
      const TS* St = gS ? gS + nm * t : nullptr;
      const TS* Rt = gR + mm * t;
      const TS* Qt = gQ + nn * t;
      // M_ux = S + B'V A
      cta_mm<RMg, RNg, true, false, TC>(m, n, n, AB + n, ldAB, T1, ldAB, EpiAdd<TC, TS>{F, ldF, 1.0, St, n});
      // m_u = r + B'(V c + v)
      cta_mm<RMg, 1, true, false, TC>(m, 1, n, AB + n, ldAB, T1 + n + m, ldAB,
                                      EpiAdd<TC, TS>{F + cmu, ldF, 1.0, gr + (size_t)m * t, 1});
      // M_uu = R + B'V B
      cta_mm<RMg, RNg, true, false, TC>(m, m, n, AB + n, ldAB, T1 + n, ldAB, EpiAddSym<TC, TS>{Muu, m, 1.0, Rt, m});
      if (param) {
        // M_zu' = (V_zx B)'  and  m_z = v_z + V_zx c
        cta_mm<RMg, RNg, false, false, TC>(n, m, n, Vzx, n, AB + n, ldAB, EpiStoreT<TC>{F + n, ldF, 1.0});
        cta_mv<false, TC>(n, n, Vzx, n, AB + n + m, ldAB, EpiAdd<TC, TC>{mz, 1, 1.0, vz, 1});
      }
      // M_xx = Q + A'V A  (into the V_xx buffer), m_x = q + A'(V c + v)  (into v_x)
      cta_mm<RMg, RNg, true, false, TC>(n, n, n, AB, ldAB, T1, ldAB, EpiAddSym<TC, TS>{Vxx, n, 1.0, Qt, n});
      cta_mm<RMg, 1, true, false, TC>(n, 1, n, AB, ldAB, T1 + n + m, ldAB,
                                      EpiAdd<TC, TS>{vx, 1, 1.0, gq + (size_t)n * t, 1});
    }
    __syncthreads();
    if (param) {  // M_zx = V_zx A, kept in T1[:, 0:n]
      cta_mm<RMg, RNg, false, false, TC>(n, n, n, Vzx, n, AB, ldAB, EpiStore<TC>{T1, ldAB, 1.0});
      __syncthreads();
    }

    if (rr == 0) {
      // ---- (4a) unconstrained stage: factor M_uu = L L' ------------------------
      // FP64 path: FP64 factor, in-place triangular solve. Mixed path: FP64
      // factor of the FP32-formed M_uu, applied in FP32 through L^{-1}. FP32
      // path: FP32 factor (hardware rsqrt pivots), applied through L^{-1}.
      TC* Wp = F;              // W = L^{-1} [M_ux | M_zu' | m_u]
      const TC* Linv = nullptr;
      if (threadIdx.x == 0) s_flag = 0;
      if (sizeof(TC) == 8) {
        __syncthreads();
        cta_chol(m, L64, m, &s_flag, s_rd);
        if (s_flag) {
          if (threadIdx.x == 0) raise_status(pd.status, LQR_ERR_NOT_PD, t);
          failed = true;
          break;
        }
        for (int i = threadIdx.x; i < m; i += blockDim.x) s_rdc[i] = static_cast<TC>(s_rd[i]);
        __syncthreads();
        cta_trsm_lower<TC>(m, reinterpret_cast<const TC*>(L64), m, s_rdc, ldF, F, ldF);
        __syncthreads();
      } else {
        if (sizeof(TS) == 8) {
          for (int e = threadIdx.x; e < m * m; e += blockDim.x) L64[e] = static_cast<double>(Muu[e]);
          __syncthreads();
          cta_chol(m, L64, m, &s_flag, s_rd);
          if (s_flag) {
            if (threadIdx.x == 0) raise_status(pd.status, LQR_ERR_NOT_PD, t);
            failed = true;
            break;
          }
          for (int e = threadIdx.x; e < m * m; e += blockDim.x) Muu[e] = static_cast<TC>(L64[e]);
          for (int i = threadIdx.x; i < m; i += blockDim.x) s_rdc[i] = static_cast<TC>(s_rd[i]);
          __syncthreads();
        } else {
          __syncthreads();
          cta_chol_f32(m, reinterpret_cast<float*>(Muu), m, &s_flag, s_pivf, reinterpret_cast<float*>(s_rdc));
          if (s_flag) {
            if (threadIdx.x == 0) raise_status(pd.status, LQR_ERR_NOT_PD, t);
            failed = true;
            break;
          }
        }
        TC* Li = reinterpret_cast<TC*>(L64);  // the FP64 factor buffer is free now
        cta_trinv_lower<TC>(m, Muu, m, s_rdc, Li, m);
        Wp = Wbuf;
        cta_mm_auto<false, false, TC>(m, ldF, m, Li, m, F, ldF, EpiStore<TC>{Wp, ldF, 1.0});
        __syncthreads();
        Linv = Li;
      }
      // V_xx = M_xx - W_x'W_x ;  v_x = m_x - W_x'w
      cta_mm<RMg, RNg, true, false, TC>(n, n, m, Wp, ldF, Wp, ldF, EpiAccum<TC>{Vxx, n, -1.0});
      cta_mm<RMg, 1, true, false, TC>(n, 1, m, Wp, ldF, Wp + cmu, ldF, EpiAccum<TC>{vx, 1, -1.0});
      if (param) {
        // V_zx = M_zx - W_z'W_x ; V_zz -= W_z'W_z ; v_z = m_z - W_z'w
        cta_mm<RMg, RNg, true, false, TC>(n, n, m, Wp + n, ldF, Wp, ldF, EpiAccum<TC>{T1, ldAB, -1.0});
        cta_mm<RMg, RNg, true, false, TC>(n, n, m, Wp + n, ldF, Wp + n, ldF, EpiAccum<TC>{Vzz, n, -1.0});
        cta_mm<RMg, 1, true, false, TC>(n, 1, m, Wp + n, ldF, Wp + cmu, ldF, EpiAdd<TC, TC>{vz, 1, -1.0, mz, 1});
      }
      __syncthreads();
      if (!param) {
        // policy [K_t | k_t] = -L'^{-1} W
        if (Linv) {
          cta_mm_auto<true, false, TC>(m, ldF, m, Linv, m, Wp, ldF, EpiStore<TC>{F, ldF, 1.0});
        } else {
          cta_trsm_lower_t<TC>(m, reinterpret_cast<const TC*>(L64), m, s_rdc, ldF, F, ldF);
        }
        __syncthreads();
        if (gK)
          for (int e = threadIdx.x; e < m * n; e += blockDim.x)
            gK[nm * t + e] = static_cast<TS>(-F[(size_t)(e / n) * ldF + (e % n)]);
        if (gk)
          for (int a = threadIdx.x; a < m; a += blockDim.x) gk[(size_t)m * t + a] = static_cast<TS>(-F[(size_t)a * ldF + cmu]);
        if (pd.segpol && mode == MODE_TERMINAL) {  // the last segment's policy [K_t | 0 | k_t]
          const int ld = 2 * n + 1;
          double* sp = pd.segpol + (size_t)m * ld * t;
          for (int e = threadIdx.x; e < m * ld; e += blockDim.x) {
            const int a = e / ld, j = e % ld;
            sp[e] = j < n ? -static_cast<double>(F[(size_t)a * ldF + j])
                          : (j < 2 * n ? 0.0 : -static_cast<double>(F[(size_t)a * ldF + cmu]));
          }
        }
        if (pd.Minv && Linv && sizeof(TS) == 4) {
          // M_uu^-1 = L^-T L^-1, kept for refinement corrections that reuse the factorisation
          cta_mm_auto<true, false, TC>(m, m, m, Linv, m, Linv, m,
                                       EpiStore<TS>{static_cast<TS*>(pd.Minv) + (size_t)m * m * t, m, 1.0});
        }
      } else {
        cta_copy<TC>(n, n, T1, ldAB, Vzx, n);
        if (pd.segpol && sizeof(TC) == 8) {
          // the paper's segment policy [K_x | K_z | k_1] = -L^-T W (W = L^-1 [M_ux | M_zu' | m_u])
          __syncthreads();
          cta_trsm_lower_t<TC>(m, reinterpret_cast<const TC*>(L64), m, s_rdc, ldF, F, ldF);
          __syncthreads();
          double* sp = pd.segpol + (size_t)m * ldF * t;
          for (int e = threadIdx.x; e < m * ldF; e += blockDim.x) sp[e] = -static_cast<double>(F[e]);
        }
      }
      cta_symmetrize<TC>(n, Vxx, n);
      __syncthreads();
    } else {
      // ---- (4b) constrained stage (Eq. 13-16, Section II-B) -------------------
      // Requires param. The constraint_to_go has rr > 0 rows [H_x | H_z | h].
      double* vhead = HH;
      double* beta = HH + m;
      const int ldAug1 = m + 2 * n + 1;
      if (rr >= m) {
        // N = H_x [A|B|c] scattered into [N_u | N_x | N_z | n_1] (r x (m+2n+1))
        cta_mm<RMg, RNg, false, false, double>(rr, n + m + 1, n, H, ldH, AB, ldAB,
                                               EpiAug{AUG, ldAug1, n, m, H, ldH});
        for (int e = threadIdx.x; e < rr * n; e += blockDim.x) {
          const int i = e / n, j = e % n;
          AUG[(size_t)i * ldAug1 + m + n + j] = H[(size_t)i * ldH + n + j];
        }
        __syncthreads();
        // N_u has full column rank m: P_y = I, Z_w empty; Q'[N_u | N] by Householder
        cta_householder_qr(rr, ldAug1, m, AUG, ldAug1, vhead, beta, s_scal);
        if (threadIdx.x == 0) {
          double dmax = 0.0, dmin = 1e300;
          for (int j = 0; j < m; ++j) {
            const double d = fabs(AUG[(size_t)j * ldAug1 + j]);
            dmax = fmax(dmax, d);
            dmin = fmin(dmin, d);
          }
          s_flag = !(dmin > 1e-12 * (double)(rr > m ? rr : m) * dmax) ? 1 : 0;
        }
        __syncthreads();
        if (s_flag) {
          if (threadIdx.x == 0) raise_status(pd.status, LQR_ERR_SEGMENT_INFEASIBLE, t);
          failed = true;
          break;
        }
        // policy G = -R_1^{-1} (Q_1'[N_x | N_z | n_1]); new constraint rows Q_2'[N_x | N_z | n_1]
        for (int e = threadIdx.x; e < m * ldG; e += blockDim.x) {
          const int a = e / ldG, j = e % ldG;
          Gc[e] = -AUG[(size_t)a * ldAug1 + m + j];
        }
        for (int e = threadIdx.x; e < (rr - m) * ldH; e += blockDim.x) {
          const int i = e / ldH, j = e % ldH;
          H[e] = AUG[(size_t)(m + i) * ldAug1 + m + j];
        }
        __syncthreads();
        cta_trsm_upper(m, AUG, ldAug1, ldG, Gc, ldG);
        __syncthreads();
        rr -= m;
      } else {
        // 0 < rr < m: N_u has full row rank rr. QR of N_u' gives P_y (first rr
        // columns of Q_f) and Z_w (the rest); y solves the constraint exactly
        // and w minimises the cost with u = P_y y + Z_w w substituted.
        const int ld2 = rr + ldF + m;
        // AUG[:, 0:rr] = N_u' = (H_x B)'
        cta_mm<RMg, RNg, true, true, double>(m, rr, n, AB + n, ldAB, H, ldH, EpiStore<double>{AUG, ld2, 1.0});
        // Gc rows 0..rr-1 = [N_x | N_z | n_1]
        cta_mm<RMg, RNg, false, false, double>(rr, n, n, H, ldH, AB, ldAB, EpiStore<double>{Gc, ldG, 1.0});
        cta_mv<false, double>(rr, n, H, ldH, AB + n + m, ldAB, EpiAdd<double, double>{Gc + 2 * n, ldG, 1.0, H + 2 * n, ldH});
        for (int e = threadIdx.x; e < rr * n; e += blockDim.x) {
          const int i = e / n, j = e % n;
          Gc[(size_t)i * ldG + n + j] = H[(size_t)i * ldH + n + j];
        }
        // AUG[:, rr:rr+ldF] = F, AUG[:, rr+ldF:] = M_uu
        for (int e = threadIdx.x; e < m * ldF; e += blockDim.x) {
          const int a = e / ldF, j = e % ldF;
          AUG[(size_t)a * ld2 + rr + j] = static_cast<double>(F[e]);
        }
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
          const int a = e / m, b = e % m;
          AUG[(size_t)a * ld2 + rr + ldF + b] = static_cast<double>(Muu[e]);
        }
        __syncthreads();
        cta_householder_qr(m, ld2, rr, AUG, ld2, vhead, beta, s_scal);
        if (threadIdx.x == 0) {
          double dmax = 0.0, dmin = 1e300;
          for (int j = 0; j < rr; ++j) {
            const double d = fabs(AUG[(size_t)j * ld2 + j]);
            dmax = fmax(dmax, d);
            dmin = fmin(dmin, d);
          }
          s_flag = !(dmin > 1e-12 * (double)m * dmax) ? 1 : 0;
        }
        __syncthreads();
        if (s_flag) {
          if (threadIdx.x == 0) raise_status(pd.status, LQR_ERR_SEGMENT_INFEASIBLE, t);
          failed = true;
          break;
        }
        // M~ = Q_f' M_uu Q_f: Ec (ld m) = (Q_f'M_uu)' = M_uu Q_f, then Q_f' from the left
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
          const int a = e / m, b = e % m;
          Ec[e] = AUG[(size_t)b * ld2 + rr + ldF + a];
        }
        // Y = -T'^{-1} [N_x | N_z | n_1]   (T = R factor of N_u', so N_u P_y = T')
        for (int e = threadIdx.x; e < rr * ldG; e += blockDim.x) Gc[e] = -Gc[e];
        __syncthreads();
        cta_householder_apply(m, rr, AUG, ld2, vhead, beta, m, Ec, m, true);
        cta_trsm_upper_t(rr, AUG, ld2, ldG, Gc, ldG);
        __syncthreads();
        // rhs_w = F~_w + M~_wy Y   (in place in AUG rows rr..m-1, columns rr..rr+ldF-1)
        cta_mm<RMg, RNg, false, false, double>(m - rr, ldG, rr, Ec + (size_t)rr * m, m, Gc, ldG,
                                               EpiAccum<double>{AUG + (size_t)rr * ld2 + rr, ld2, 1.0});
        if (threadIdx.x == 0) s_flag = 0;
        __syncthreads();
        cta_chol(m - rr, Ec + (size_t)rr * m + rr, m, &s_flag, s_rd);
        if (s_flag) {
          if (threadIdx.x == 0) raise_status(pd.status, LQR_ERR_NOT_PD, t);
          failed = true;
          break;
        }
        // W = -M~_ww^{-1} rhs_w  (Gc rows rr..m-1)
        for (int e = threadIdx.x; e < (m - rr) * ldG; e += blockDim.x) {
          const int a = e / ldG, j = e % ldG;
          Gc[(size_t)(rr + a) * ldG + j] = -AUG[(size_t)(rr + a) * ld2 + rr + j];
        }
        __syncthreads();
        cta_trsm_lower<double>(m - rr, Ec + (size_t)rr * m + rr, m, s_rd, ldG, Gc + (size_t)rr * ldG, ldG);
        __syncthreads();
        cta_trsm_lower_t<double>(m - rr, Ec + (size_t)rr * m + rr, m, s_rd, ldG, Gc + (size_t)rr * ldG, ldG);
        __syncthreads();
        // G = Q_f [Y; W]
        cta_householder_apply(m, rr, AUG, ld2, vhead, beta, ldG, Gc, ldG, false);
        rr = 0;
      }
      __syncthreads();
      if (pd.segpol) {  // the paper's segment policy of this constrained stage, u = G [x; z; 1]
        double* sp = pd.segpol + (size_t)m * ldG * t;
        for (int e = threadIdx.x; e < m * ldG; e += blockDim.x) sp[e] = Gc[e];
      }
      // ---- value update by substitution of u = G [x; z; 1] (Eq. 16, symmetric form)
      // E = F + M_uu G
      cta_mm<RMg, RNg, false, false, double>(m, ldG, m, Muu, m, Gc, ldG, EpiAdd<double, TC>{Ec, ldG, 1.0, F, ldF});
      __syncthreads();
      // V_xx = M_xx + F_x'G_x + G_x'E_x ; v_x = m_x + F_x'g + G_x'e
      cta_mm<RMg, RNg, true, false, double>(n, n, m, F, ldF, Gc, ldG, EpiAccum<TC>{Vxx, n, 1.0});
      cta_mm<RMg, 1, true, false, double>(n, 1, m, F, ldF, Gc + 2 * n, ldG, EpiAccum<TC>{vx, 1, 1.0});
      // V_zx = M_zx + F_z'G_x + G_z'E_x (T1 holds M_zx) ; V_zz += F_z'G_z + G_z'E_z ; v_z = m_z + F_z'g + G_z'e
      cta_mm<RMg, RNg, true, false, double>(n, n, m, F + n, ldF, Gc, ldG, EpiAccum<TC>{T1, ldAB, 1.0});
      cta_mm<RMg, RNg, true, false, double>(n, n, m, F + n, ldF, Gc + n, ldG, EpiAccum<TC>{Vzz, n, 1.0});
      cta_mm<RMg, 1, true, false, double>(n, 1, m, F + n, ldF, Gc + 2 * n, ldG, EpiAdd<TC, TC>{vz, 1, 1.0, mz, 1});
      __syncthreads();
      cta_mm<RMg, RNg, true, false, double>(n, n, m, Gc, ldG, Ec, ldG, EpiAccum<TC>{Vxx, n, 1.0});
      cta_mm<RMg, 1, true, false, double>(n, 1, m, Gc, ldG, Ec + 2 * n, ldG, EpiAccum<TC>{vx, 1, 1.0});
      cta_mm<RMg, RNg, true, false, double>(n, n, m, Gc + n, ldG, Ec, ldG, EpiAccum<TC>{T1, ldAB, 1.0});
      cta_mm<RMg, RNg, true, false, double>(n, n, m, Gc + n, ldG, Ec + n, ldG, EpiAccum<TC>{Vzz, n, 1.0});
      cta_mm<RMg, 1, true, false, double>(n, 1, m, Gc + n, ldG, Ec + 2 * n, ldG, EpiAccum<TC>{vz, 1, 1.0});
      __syncthreads();
      cta_copy<TC>(n, n, T1, ldAB, Vzx, n);
      cta_symmetrize<TC>(n, Vxx, n);
      __syncthreads();
    }
    if (pd.stageV && param) {
      // the cost to go at stage t as a function of (x_t, x_term) (Eq. 9 at stage
      // t) and the rows of its constraint_to_go, for the per-stage reconstruction
      // of the global policy
      double* sv = pd.stageV + (size_t)t * (3 * nn + 2 * n);
      for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        sv[e] = static_cast<double>(Vxx[e]);
        sv[nn + e] = static_cast<double>(Vzx[e]);
        sv[2 * nn + e] = 0.5 * (static_cast<double>(Vzz[(size_t)i * n + j]) + static_cast<double>(Vzz[(size_t)j * n + i]));
      }
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        sv[3 * nn + i] = static_cast<double>(vx[i]);
        sv[3 * nn + n + i] = static_cast<double>(vz[i]);
      }
      if (threadIdx.x == 0) pd.stage_rank[t] = rr;
    }
    if (store_P && gP && !param) {
      for (int e = threadIdx.x; e < n * n; e += blockDim.x) gP[nn * t + e] = static_cast<TS>(Vxx[e]);
      for (int i = threadIdx.x; i < n; i += blockDim.x) gp[(size_t)n * t + i] = static_cast<TS>(vx[i]);
    }
  }
  if (failed) return;
  if (param && rr != 0) {  // the segment is too short to reach an arbitrary end state
    if (threadIdx.x == 0) raise_status(pd.status, LQR_ERR_SEGMENT_INFEASIBLE, t0);
    return;
  }
  // ---- write the summary (Eq. 9 at the segment start) --------------------------
  if (mode == MODE_POLICY) return;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) summ[e] = static_cast<double>(Vxx[e]);
  for (int i = threadIdx.x; i < n; i += blockDim.x) summ[3 * nn + i] = static_cast<double>(vx[i]);
  if (param) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) summ[nn + e] = static_cast<double>(Vzx[e]);
    for (int i = threadIdx.x; i < n; i += blockDim.x) summ[3 * nn + n + i] = static_cast<double>(vz[i]);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e / n, j = e % n;
      Vzz_g[e] = 0.5 * (static_cast<double>(Vzz[(size_t)i * n + j]) + static_cast<double>(Vzz[(size_t)j * n + i]));
    }
  } else {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) { summ[nn + e] = 0.0; summ[2 * nn + e] = 0.0; }
    for (int i = threadIdx.x; i < n; i += blockDim.x) summ[3 * nn + n + i] = 0.0;
  }
}

template <typename TS, typename TC>
long long sweep_smem_needed(int n, int m, long long smem_budget, bool constrained, long long* scratch_doubles) {
  SweepPlan a, b, c;
  make_plan(a, n, m, MODE_PARAM, (int)sizeof(TC), smem_budget, constrained);
  make_plan(b, n, m, MODE_TERMINAL, (int)sizeof(TC), smem_budget, constrained);
  make_plan(c, n, m, MODE_POLICY, (int)sizeof(TC), smem_budget, constrained);
  long long s = a.smem_bytes;
  if (b.smem_bytes > s) s = b.smem_bytes;
  if (c.smem_bytes > s) s = c.smem_bytes;
  long long g = a.scratch_bytes;
  if (b.scratch_bytes > g) g = b.scratch_bytes;
  if (c.scratch_bytes > g) g = c.scratch_bytes;
  if (scratch_doubles) *scratch_doubles = (g + 7) / 8;
  return s;
}

template <typename TS, typename TC>
cudaError_t launch_seg_sweep(const ProbTable& tab, int nunits, int phase, long long smem_bytes,
                             long long smem_budget, int store_P, cudaStream_t st) {
  cudaError_t e = raise_dyn_smem((const void*)seg_sweep_kernel<TS, TC>, (size_t)smem_bytes);
  if (e != cudaSuccess) return e;
  seg_sweep_kernel<TS, TC><<<nunits, kBlock, (size_t)smem_bytes, st>>>(tab, phase, smem_budget, store_P);
  return cudaGetLastError();
}

template cudaError_t launch_seg_sweep<double, double>(const ProbTable&, int, int, long long, long long, int,
                                                      cudaStream_t);
template cudaError_t launch_seg_sweep<float, float>(const ProbTable&, int, int, long long, long long, int,
                                                    cudaStream_t);
template cudaError_t launch_seg_sweep<double, float>(const ProbTable&, int, int, long long, long long, int,
                                                     cudaStream_t);
template long long sweep_smem_needed<double, double>(int, int, long long, bool, long long*);
template long long sweep_smem_needed<double, float>(int, int, long long, bool, long long*);
template long long sweep_smem_needed<float, float>(int, int, long long, bool, long long*);

}  // namespace lqr
