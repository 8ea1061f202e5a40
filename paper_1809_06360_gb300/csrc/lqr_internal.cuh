// Internal types shared by the liblqr kernels and the host orchestration.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cta_linalg.cuh"
#include "lqr.h"

namespace lqr {

constexpr int kBlock = 256;           // threads per CTA of the sweep / rollout kernels
constexpr int kStaticSmemReserve = 12 * 1024;  // static shared memory of the kernels (pivot scratch, flags)

// Segment j of a K-way split of T stages covers [seg_begin(j), seg_begin(j+1)).
__host__ __device__ inline int seg_begin(int T, int K, int j) {
  return (int)(((long long)j * (long long)T) / (long long)K);
}

// Per-problem FP64 workspace, offsets in doubles from ProbDesc::ws.
struct WsLayout {
  long long summ;   // K * (3n^2 + 2n)   segment summaries (Eq. 9 at each segment start)
  long long Pi;     // (K+1) * n^2       global value Hessian at b_j (j = 0..K-1 used)
  long long pi;     // (K+1) * n         global value gradient at b_j
  long long Gam;    // K * n^2           link feedback z_{j+1} = Gam_j z_j + gam_j
  long long gam;    // K * n
  long long z;      // (K+1) * n         link states z_j = x_{b_j}
  long long costp;  // K                 partial objective per segment
  long long lwork;  // 4 n^2 + 2n        link-solve work matrices when they do not fit in shared memory
  // per-link factors stored by the cluster link chain for the parallel post-pass
  long long lkTm;   // K * n^2           W_j C_{j+1}
  long long lkLd;   // K * n^2           Cholesky factor of I + C'W_j C
  long long lkRd;   // K * n             1 / diag(Ld)
  long long lkF;    // K * n (n+1)       Ld^-1 C'[Z_j | v_j]
  long long lkV;    // K * n             v_j = w_j - W_j pi_{j+1}
  long long scan;   // 3 K scan_elem_floats(n) / 2   FP32 link-scan elements (base, ping, pong)
  long long total;
};

__host__ __device__ inline WsLayout ws_layout(int n, int K) {
  WsLayout w;
  const long long nn = (long long)n * n;
  long long o = 0;
  w.summ = o;  o += (long long)K * (3 * nn + 2 * n);
  w.Pi = o;    o += (long long)(K + 1) * nn;
  w.pi = o;    o += (long long)(K + 1) * n;
  w.Gam = o;   o += (long long)K * nn;
  w.gam = o;   o += (long long)K * n;
  w.z = o;     o += (long long)(K + 1) * n;
  w.costp = o; o += K;
  o = (o + 31) & ~31LL;
  w.lwork = o; o += 4 * nn + 2 * n;
  o = (o + 31) & ~31LL;
  w.lkTm = o;  o += (long long)K * nn;
  w.lkLd = o;  o += (long long)K * nn;
  w.lkRd = o;  o += (long long)K * n;
  w.lkF = o;   o += (long long)K * n * (n + 1);
  w.lkV = o;   o += (long long)K * n;
  o = (o + 31) & ~31LL;
  w.scan = o;
  if (K > 1) o += (3LL * K * (((3 * nn + 2 * n) + 3) & ~3LL) + 1) / 2;
  w.total = (o + 31) & ~31LL;
  return w;
}

// Floats per element of the FP32 link scan: P | Z | -W (n x n each) | p | w,
// rounded up to a multiple of 4 (16-byte aligned elements).
__host__ __device__ inline long long scan_elem_floats(int n) {
  return ((3LL * n * n + 2LL * n) + 3) & ~3LL;
}

// One problem as the kernels see it.
struct ProbDesc {
  const void *A, *B, *c, *Q, *R, *S, *q, *r, *x0;   // element type TS
  void *K, *k, *x, *u, *P, *p, *lam;                 // element type TS, may be null
  double* ws;                 // WsLayout base
  double* scratch;            // nseg * scratch_per_unit doubles (spilled sweep buffers)
  long long scratch_per_unit; // doubles
  int* status;                // [0] = lqr_status, [1] = first flagged stage
  const int* skip;            // when non-null and set, every kernel of this solve returns at once
  double* report;             // [0] cost, [1] eta, [2] rel, [3] refinement corrections applied
  int n, m, T, nseg;
  int unit0;                  // first unit (segment) index of this problem in a launch
  int form;                   // lqr_form of the parametric sweeps
  void* Minv;                 // FP32 fast path: T x m x m M_uu^-1 of the policy stages, may be null
  double* segpol;             // FP64 constrained sweep: T x m x (2n+1) segment policies [K_x | K_z | k_1], may be null
  int smooth;                 // policy sweep started from the next segment's cost with its end pinned (Section III-A)
  double* stageV;             // FP64 constrained sweep: T x (3n^2 + 2n) per-stage [Vxx | Vzx | Vzz | vx | vz], may be null
  int* stage_rank;            // T: rows of the constraint_to_go at each stage (with stageV); the policy
                              // sweep stops at the first stage of rank 0 when set
};

// Kernel-argument view of the problems of one launch: a single problem is
// passed by value, a batch through a device array plus a unit -> problem map.
struct ProbTable {
  ProbDesc single;
  const ProbDesc* probs;      // device array (batched) or nullptr
  const int* unit_prob;       // device array: unit -> problem index (batched)
  int nprob;
};

__device__ __forceinline__ const ProbDesc& prob_of_unit(const ProbTable& tab, int unit) {
  return tab.probs ? tab.probs[tab.unit_prob[unit]] : tab.single;
}
__device__ __forceinline__ const ProbDesc& prob_at(const ProbTable& tab, int i) {
  return tab.probs ? tab.probs[i] : tab.single;
}

// Uniform early exit of a CTA: an earlier step failed, or this is a
// refinement correction that is no longer needed. Ends with a barrier.
__device__ __forceinline__ bool cta_should_exit(const ProbDesc& pd, int* s_flag) {
  if (threadIdx.x == 0) *s_flag = (*(volatile int*)pd.status != 0) || (pd.skip && *(volatile const int*)pd.skip);
  __syncthreads();
  const bool ex = *s_flag != 0;
  __syncthreads();
  return ex;
}

// First error wins; records the stage that raised it.
__device__ __forceinline__ void raise_status(int* st, int code, int stage) {
  if (atomicCAS(st, 0, code) == 0) atomicExch(st + 1, stage);
}

// ---------------------------------------------------------------------------
// Placement plan of the segment-sweep buffers: each buffer lives in dynamic
// shared memory while the budget lasts (in priority order), otherwise in the
// unit's slice of global scratch. Identical on host and device.
// ---------------------------------------------------------------------------
enum SweepBuf {
  SB_VXX = 0,  // TC  n x n        V_xx (then M_xx)
  SB_AB,       // TC  n x ldAB     [A_t | B_t | c_t]
  SB_T1,       // TC  n x ldAB     V_xx [A|B|c] (+v_x), later V_zx A
  SB_F,        // TC  m x ldF      [M_ux | M_zu' | m_u]  (then W = L^-1 F, then policy)
  SB_MUU,      // TC  m x m        M_uu
  SB_L64,      // f64 m x m        Cholesky factor of M_uu (aliases SB_MUU when TC = double)
  SB_VEC,      // TC  4n           v_x, v_z, m_z, spare
  SB_W,        // TC  m x ldF      W = L^-1 F when TC is float (TC = double solves in place)
  SB_VZX,      // TC  n x n        V_zx          (parametric sweep only)
  SB_VZZ,      // TC  n x n        V_zz          (parametric sweep only)
  SB_HH,       // f64 2m           Householder heads and scales
  SB_G,        // f64 m x (2n+1)   constrained-stage policy [K_x | K_z | k_1]
  SB_E,        // f64 m x (2n+1)   F + M_uu G, also M~ (m x m)
  SB_H,        // f64 n x (2n+1)   constraint_to_go [H_x | H_z | h_1] (Eq. 9b), r rows used
  SB_AUG,      // f64 workspace of the range/null-space split
  SB_COUNT
};

enum SweepMode { MODE_PARAM = 0, MODE_TERMINAL = 1, MODE_POLICY = 2 };

struct SweepPlan {
  int ldAB, ldF, ldG, ldH, ldAug;
  long long off[SB_COUNT];    // byte offset (smem or scratch)
  unsigned smem_mask;         // bit b set = buffer b in shared memory
  long long smem_bytes;       // dynamic shared memory used
  long long scratch_bytes;    // global scratch per unit
};

__host__ __device__ inline long long align16(long long b) { return (b + 15) & ~15LL; }

__host__ __device__ inline void make_plan(SweepPlan& P, int n, int m, int mode, int tc_size,
                                          long long smem_budget, bool constrained) {
  const bool param = (mode == MODE_PARAM);
  const bool cons = param && constrained;  // range/null-space workspace
  P.ldAB = n + m + 1;
  P.ldF = param ? 2 * n + 1 : n + 1;
  P.ldG = 2 * n + 1;
  P.ldH = 2 * n + 1;
  // [N_u | N_x | N_z | n_1] (n rows) or [N_u' | F | M_uu] (m rows, at most n + ldF + m columns)
  const long long aug1 = (long long)n * (m + 2 * n + 1);
  const long long aug2 = (long long)m * (n + (2 * n + 1) + m);
  P.ldAug = 0;  // chosen per stage
  long long bytes[SB_COUNT];
  const long long tc = tc_size;
  bytes[SB_VXX] = tc * n * n;
  bytes[SB_AB] = tc * n * P.ldAB;
  bytes[SB_T1] = tc * n * P.ldAB;
  bytes[SB_F] = tc * m * P.ldF;
  bytes[SB_MUU] = tc * m * m;
  bytes[SB_L64] = (tc_size == 8) ? 0 : 8LL * m * m;
  bytes[SB_VEC] = tc * 4 * n;
  bytes[SB_W] = (tc_size == 8) ? 0 : tc * m * P.ldF;
  bytes[SB_VZX] = param ? tc * n * n : 0;
  bytes[SB_VZZ] = param ? tc * n * n : 0;
  bytes[SB_HH] = cons ? 8LL * 2 * m : 0;
  bytes[SB_G] = cons ? 8LL * m * P.ldG : 0;
  bytes[SB_E] = cons ? 8LL * m * (P.ldG > m ? P.ldG : m) : 0;
  bytes[SB_H] = cons ? 8LL * n * P.ldH : 0;
  bytes[SB_AUG] = cons ? 8LL * (aug1 > aug2 ? aug1 : aug2) : 0;
  long long s = 0, g = 0;
  P.smem_mask = 0;
  for (int b = 0; b < SB_COUNT; ++b) {
    const long long sz = align16(bytes[b]);
    if (sz == 0) { P.off[b] = 0; continue; }
    if (s + sz <= smem_budget) {
      P.off[b] = s; s += sz; P.smem_mask |= (1u << b);
    } else {
      P.off[b] = g; g += sz;
    }
  }
  P.smem_bytes = s;
  P.scratch_bytes = g;
}

template <typename T>
__device__ __forceinline__ T* plan_ptr(const SweepPlan& P, int b, unsigned char* smem, unsigned char* scratch) {
  return reinterpret_cast<T*>(((P.smem_mask >> b) & 1u) ? smem + P.off[b] : scratch + P.off[b]);
}

// Multiprocessor count of the current device (looked up once per device).
int device_sm_count();

// Raises (never lowers) a kernel's dynamic shared-memory limit; one registry
// for all launchers of the same kernel (lqr_api.cu).
cudaError_t raise_dyn_smem(const void* func, size_t bytes);

// Refinement corrections that reuse the factorisation (correct.cu): FP32
// arrays of one problem, K = the solve's segment count. The step matrices of
// the correction recursions are stored as blocks of n + 1 rows of stride ld
// (corr_ld): rows 0..n-1 the matrix, row n the step's offset vector.
struct CorrArgs {
  const float *A, *B, *K, *P, *Minv;   // the solve's data, policies, value matrices, M_uu^-1
  const float *cq, *cr, *cc, *cx0;     // correction data q~ ((T+1) n), r~ (T m), c~ (T n), x0~ (n)
  float *Phit, *PhiTt;                 // T blocks: Phi_t with e_t, Phi_t' with w_t
  float *Psi, *PsiT;                   // K blocks: Psi_j with eps_j, Psi_j' with delta_j
  float* pcv;                          // P_{t+1} c~_t (T ld)
  float *pb, *xb;                      // (K+1) n each: p and x~ at the segment boundaries
  float *dk, *dp, *dx, *du, *dl;       // the correction: k~, p, x~, u~, lambda~
  const int* skip;                     // set: converged, every kernel returns at once
  int* status;
  int n, m, T, nseg;
  long long spin;  // polls of a copy wait before LQR_ERR_TIMEOUT (0: the default)
  int slots;       // ring slots of the recursion kernel (2..6)
  int psi_global;  // 1: the closed-loop maps read B_t, K_t from global memory
  // two-level link chains (ng > 0): groups of G consecutive links, blocks of
  // their maps Theta_g with e_g and Theta_g' with d_g (ng each), group boundary
  // values Y, X ((ng+1) n)
  float *Theta, *ThetaT, *gY, *gX;
  int G, ng;
};

// ---------------------------------------------------------------------------
// Host-side launchers (defined in the .cu files, called by lqr_api.cu).
// ---------------------------------------------------------------------------
// phase 0: A1 (parametric sweeps + terminal sweep); phase 1: A4 (policy sweeps)
template <typename TS, typename TC>
cudaError_t launch_seg_sweep(const ProbTable& tab, int nunits, int phase, long long smem_bytes,
                             long long smem_budget, int store_P, cudaStream_t st);
template <typename TS, typename TC>
long long sweep_smem_needed(int n, int m, long long smem_budget, bool constrained, long long* scratch_doubles);

cudaError_t launch_link_solve(const ProbTable& tab, int nprob, int x0_is_float, cudaStream_t st);
// The FP32 multiplier-form segment sweep (steps A1/A4) on padded 4 x 4 tiles;
// cudaErrorNotSupported (nothing launched) when its plan does not fit.
cudaError_t launch_seg_sweep_f32(const ProbTable& tab, int nunits, int phase, int nmax, int mmax,
                                 long long smem_budget, int store_P, cudaStream_t st);
long long fast_sweep_smem_bytes(int n, int m);
long long rollout_f32_smem_bytes(int nmax, int mmax);
// Step A10 in one persistent launch for batches of one-segment problems
// (batch_persistent.cu): CTAs take problems from the LPT-ordered queue `order`
// through the zeroed int `ticket`.
bool batch_persistent_supported(int nmax, int mmax, long long smem_budget);
cudaError_t launch_batch_persistent(const ProbTable& tab, const int* order, int* ticket, int want_lam, int nmax,
                                    int mmax, int store_P, int num_sms, cudaStream_t st);
// The policy sweep (step A4) with TF32 tensor-core stage products and the FP64
// Cholesky factor of M_uu (seg_sweep_tc.cu), FP32 data, 64 < n <= 128, m <= 64.
bool tc_sweep_supported(int n, int m);
cudaError_t launch_seg_sweep_tc(const ProbTable& tab, int nunits, int store_P, long long spin_limit, cudaStream_t st);
// the FP32 fast sweeps (and with them the kept M_uu^-1) apply to (n, m)
bool fast_sweep_supported(int n, int m, long long smem_budget);
// refinement corrections that reuse the factorisation (correct.cu)
// Outputs per consumer warp of a correction recursion step (a power of two,
// 4..32): eight warps cover n, and 32 / corr_opw(n) lanes share each output.
__host__ __device__ inline int corr_opw(int n) {
  const int need = (n + 7) / 8;
  int o = 4;
  while (o < need) o <<= 1;
  return o > 32 ? 32 : o;
}
// The row stride of the stored correction blocks: a multiple of 4 floats (16-byte
// rows) at least n, and congruent to corr_opw(n) mod 32 when lanes share an
// output, so that the lanes summing rows q, q + P, ... of one column block read
// distinct shared-memory banks.
__host__ __device__ inline int corr_ld(int n) {
  const int opw = corr_opw(n);
  int ld = (n + 3) & ~3;
  if (opw < 32)
    while ((ld & 31) != opw) ld += 4;
  return ld;
}
size_t corr_rec_smem_bytes(int n, int slots);
size_t corr_psi_smem_bytes(int n, int m, int psi_global);
// the plan of the correction kernels for (n, m) within the shared-memory
// budget (slots 0: they do not apply)
void corr_plan(int n, int m, long long smem_budget, int* slots, int* psi_global);
cudaError_t launch_corr_psi(const CorrArgs& a, cudaStream_t st);
cudaError_t launch_correction(const CorrArgs& a, cudaStream_t st, int* launches);
// the group maps of the two-level link chains (once per solve, after launch_corr_psi)
cudaError_t launch_corr_groups(const CorrArgs& a, cudaStream_t st);
size_t corr_group_smem_bytes(int n);

// Element-type conversion of up to kMaxConv arrays in one launch (skip: when
// non-null and set, nothing is done).
constexpr int kMaxConv = 16;
template <typename S, typename D>
struct ConvTable {
  const S* src[kMaxConv];
  D* dst[kMaxConv];
  S* raw[kMaxConv];  // when non-null: also an unconverted copy of the source
  size_t n[kMaxConv];
  int count;
  void add(const void* s, void* d, size_t cnt, void* raw_copy = nullptr) {
    if (!s || !d || cnt == 0) return;
    src[count] = static_cast<const S*>(s);
    dst[count] = static_cast<D*>(d);
    raw[count] = static_cast<S*>(raw_copy);
    n[count] = cnt;
    ++count;
  }
};
template <typename S, typename D>
cudaError_t launch_convert(const ConvTable<S, D>& tab, const int* skip, cudaStream_t st);
cudaError_t launch_refine_update_f32(const ProbDesc& pd, const float* dk, const float* dx, const float* du,
                                     const float* dl, const float* dp, const int* skip, cudaStream_t st);

// Dual link solve of one problem. link_fp32 selects FP32 arithmetic; method
// is an lqr_link value (the scan needs link_fp32). *nlaunch = kernels launched.
cudaError_t launch_link_solve_dual(const ProbTable& tab, int nprob, int x0_is_float, cudaStream_t st,
                                   int link_fp32, int method, int* nlaunch);
// The FP32 suffix-scan link solve; cudaErrorNotSupported (nothing launched)
// when the problem shape does not fit. part 0: all; 1: up to the final Pi_j, pi_j;
// 2: the link feedback and the link states.
cudaError_t launch_link_scan(const ProbTable& tab, int x0_is_float, cudaStream_t st, int* launches, int part = 0);
size_t link_scan_smem_bytes(int n);

template <typename TS, typename TC>
// has_xu: every problem of the launch has x and u outputs (the streaming
// kernel re-reads them for the multiplier pass).
cudaError_t launch_rollout(const ProbTable& tab, int nunits, int want_lam, cudaStream_t st, int nmax = 0, int mmax = 0,
                           int has_xu = 0);
cudaError_t launch_link_solve_dual_batched(const ProbTable& tab, int nprob, int nmax, int x0_is_float, cudaStream_t st);

cudaError_t launch_finalize(const ProbTable& tab, int nprob, cudaStream_t st);

// adjoint (adjoint.cu)
template <typename TS>
cudaError_t launch_adjoint_rhs(int n, int m, int T, const void* gx, const void* gu, void* q, void* r, void* c,
                               void* x0, cudaStream_t st);
template <typename TS>
cudaError_t launch_adjoint_grad(int n, int m, int T, const void* x, const void* u, const void* lam, const void* xix,
                                const void* xiu, const void* xil, const lqr_problem* g, cudaStream_t st);

// the batched adjoint's per-problem jobs (adjoint.cu): adjoint_job_bytes() per
// job, filled on the host, one launch each over a device table
size_t adjoint_job_bytes();
void adjoint_job_fill(void* dst, int n, int m, int T, const void* gx, const void* gu, void* q, void* r, void* c,
                      void* x0, const void* x, const void* u, const void* lam, const void* xix, const void* xiu,
                      const void* xil, const lqr_problem* g);
template <typename TS>
cudaError_t launch_adjoint_rhs_batched(const void* jobs, int njobs, cudaStream_t st);
template <typename TS>
cudaError_t launch_adjoint_grad_batched(const void* jobs, int njobs, int Tmax, cudaStream_t st);

// per-stage reconstruction of the global policy (stage_policy.cu)
size_t stage_policy_smem_bytes(int n, int on_chip);
cudaError_t launch_stage_policy(const ProbDesc& pd, int nstages, int on_chip, double* scratch, cudaStream_t st);

// the trajectory-optimisation outer loop (sqp.cu): model data on the device
struct NlModelDev {
  const double *A, *B, *C, *Q, *R, *QT, *xref, *x0;
  double beta;
  int n, m, T;
};
constexpr int kSqpCand = 9;                 // candidate step lengths: 0, 1, 1/2, ..., 1/128
constexpr int kSqpOut = 2 * kSqpCand + 6;   // per stage: J(alpha), D(alpha), g'd, max|lam|, |dx|, |du|, |x|, |u|
__host__ __device__ inline double sqp_alpha(int a) { return a == 0 ? 0.0 : ldexp(1.0, -(a - 1)); }
cudaError_t launch_sqp_fill(const NlModelDev& md, double* Bt, double* Qt, double* Rt, cudaStream_t st);
cudaError_t launch_sqp_linearize(const NlModelDev& md, const double* x, const double* u, double* At, double* c,
                                 double* q, double* r, double* dx0, cudaStream_t st);
cudaError_t launch_sqp_merit(const NlModelDev& md, const double* x, const double* u, const double* dx,
                             const double* du, const double* q, const double* r, const double* lam, double* part,
                             double* res, cudaStream_t st);
cudaError_t launch_sqp_update(double* x, double* u, const double* dx, const double* du, double alpha, long long nx,
                              long long nu, cudaStream_t st);

// least-squares multipliers of the segment problems (ls_mult.cu)
struct LsArgs {
  const double *A, *B, *Q, *R, *S, *q, *r, *x, *u;
  double *lam, *lam_end, *mu;
  double* scratch;             // per segment: (longest segment + 2) factor blocks
  long long scratch_per_seg;   // doubles
  int* status;
  int n, m, T, K;
  int on_chip;                 // 1: the working blocks in shared memory
};
size_t ls_mult_smem_bytes(int n, int m, int on_chip);
long long ls_mult_scratch_doubles(int n, int T, int K);
cudaError_t launch_ls_mult(const LsArgs& a, cudaStream_t st);

// Destinations of the correction problem's vectors that a residual pass
// writes (-rx, -ru, rd and x_0 - x0): FP64, or FP32 for the FP32 correction
// solves of the mixed-precision refinement; q == nullptr: none.
struct KktOut {
  void *q, *r, *c, *x0;
  int f32;
  __device__ __forceinline__ void put(void* p, size_t i, double v) const {
    if (f32)
      static_cast<float*>(p)[i] = static_cast<float>(v);
    else
      static_cast<double*>(p)[i] = v;
  }
};

// refinement (refine.cu)
// per-CTA objective partials of the residual pass: at most kMaxResidBlocks CTAs
constexpr int kMaxResidBlocks = 1024;
constexpr int kResidAccDoubles = 8 + kMaxResidBlocks;
// knorm: also accumulate |KKT|_inf (1), not (0), or only when no correction
// vectors are requested (-1). |KKT|_inf depends on the data alone: a pass that
// computes it once keeps it in the accumulators until the solve's final pass.
// df: 1 the double-FP32 kernel where it applies (FP64 data, correction vectors
// requested, no |KKT| row sums, n, m <= 128), else the FP64 one; 3 (the loop
// body of a refinement graph) both, the double-FP32 one running in the first
// iteration (skip[2] == 0) and the FP64 one in the later ones.
template <typename TS>
cudaError_t launch_kkt_residual(const ProbDesc& pd, double* acc, const KktOut& out, const int* skip, cudaStream_t st,
                                int knorm = -1, int df = 0);
// |KKT|_inf from the FP32 copy of the data (pd: the FP32 problem), once per mixed-precision solve
cudaError_t launch_kkt_norm_f32(const ProbDesc& pd, double* acc, cudaStream_t st);
// The finalize of a refinement graph's loop body: also counts the iterations
// in skip[2] and sets the loop condition `cond` (continue while not converged,
// no error and fewer than `loop` iterations).
cudaError_t launch_residual_finalize_loop(const ProbDesc& pd, double* acc, double tol, int* skip, int loop,
                                          cudaGraphConditionalHandle cond, cudaStream_t st);
cudaError_t launch_residual_finalize(const ProbDesc& pd, double* acc, double tol, int* skip, int is_final,
                                     int check, cudaStream_t st);
template <typename TS>
cudaError_t launch_refine_update(const ProbDesc& pd, const double* dk, const double* dx, const double* du,
                                 const double* dl, const double* dp, const int* skip, cudaStream_t st);

}  // namespace lqr
