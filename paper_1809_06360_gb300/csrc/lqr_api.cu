// C-ABI of liblqr: argument validation, workspace management and the launch
// sequence of one solve (Section II-C: split -> parametric segment sweeps ->
// link solve -> redistribution to the segments).
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>

#include "kkt_stage.cuh"
#include "lqr_internal.cuh"

using namespace lqr;

namespace lqr {
int device_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 1;
  }
  int v = cache[dev].load(std::memory_order_acquire);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
    cudaGetLastError();
    return 1;
  }
  cache[dev].store(v, std::memory_order_release);
  return v;
}

cudaError_t raise_dyn_smem(const void* func, size_t bytes) {
  struct Entry { const void* f; int dev; size_t bytes; };
  static Entry table[64];
  static int count = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  for (int i = 0; i < count; ++i)
    if (table[i].f == func && table[i].dev == dev) {
      if (bytes <= table[i].bytes) return cudaSuccess;
      cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e == cudaSuccess) table[i].bytes = bytes;
      return e;
    }
  cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && count < 64) table[count++] = Entry{func, dev, bytes};
  return e;
}
}  // namespace lqr

struct lqr_handle {
  int device = 0;
  int num_sms = 0;
  long long smem_optin = 0;
  unsigned char* ws = nullptr;  // device workspace
  size_t ws_bytes = 0;
  unsigned char* stage = nullptr;  // device staging for lqr_solve_host
  size_t stage_bytes = 0;
  int* d_status = nullptr;     // [2]
  double* d_report = nullptr;  // [4]
  int last_K = 0;
  int last_launches = 0;
  int last_resid = 0;
  // batched solves: device descriptor table, per-problem status/report, pinned staging
  unsigned char* bdev = nullptr;
  size_t bdev_bytes = 0;
  unsigned char* bhost = nullptr;  // pinned
  size_t bhost_bytes = 0;
  cudaEvent_t bhost_ev = nullptr;  // last copy out of bhost
  unsigned char* adj = nullptr;    // adjoint problems' vectors and solutions
  size_t adj_bytes = 0;
  int last_batch = 0;
  size_t bstatus_off = 0, breport_off = 0;
  // phase profiling: one event pair per phase per solve, summed on read
  static constexpr int kPhases = LQR_NUM_PHASES;
  static constexpr int kMaxProfiled = 256;
  int prof_on = 0;
  int prof_count = 0;                       // solves recorded since enable
  cudaEvent_t ev[kMaxProfiled][kPhases + 1];
  int ev_created = 0;
  int prof_launches[kPhases] = {0};
  // side stream: the A4 sweep runs on it next to the link tail (fork/join by events)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // lqr_solve_host: the policies' copy back to the host beside the refinement
  cudaStream_t copy = nullptr;
  cudaEvent_t ev_kready = nullptr, ev_kdone = nullptr;
  // LQR_MIXED_FP32: FP32 copy of the data, FP32 solution and correction buffers
  unsigned char* f32 = nullptr;
  size_t f32_bytes = 0;
  unsigned char* nl = nullptr;  // the outer loop's subproblem data and merit partials
  size_t nl_bytes = 0;
  // the refinement loop of the mixed modes as a CUDA graph: a WHILE node around
  // one iteration, the condition set by the iteration's finalize kernel, so
  // that the iterations after convergence are not launched at all. Rebuilt when
  // the arguments of its kernels change (key); plain launches if a graph call fails.
  static constexpr int kRKeyBytes = 1024;
  cudaStream_t cap = nullptr;
  cudaGraph_t rgraph = nullptr;
  cudaGraphExec_t rexec = nullptr;
  unsigned char rkey[kRKeyBytes];
  int rkey_valid = 0;
  int rbody = 0;                  // kernels of the loop body
  int rgraph_broken = 0;
  // launches of the last solve that ran the graph: last_launches + rbody * *last_iters
  const int* last_iters = nullptr;
  cudaStream_t last_stream = nullptr;
  // batch-schedule autotuner: per batch-shape bucket, 1 = the persistent
  // one-segment schedule was measured faster than the per-step launches
  struct TuneEntry { int key[4]; int persistent; float ms[2]; };
  TuneEntry tune[64];
  int ntune = 0;
  int last_schedule = 0;  // schedule of the last batched solve: 0 per-step launches, 1 persistent
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

lqr_status grow(unsigned char** buf, size_t* cap, size_t need) {
  if (need <= *cap) return LQR_OK;
  if (*buf) {
    cudaDeviceSynchronize();
    cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
  }
  size_t sz = need + need / 8 + (1 << 20);
  if (cudaMalloc(buf, sz) != cudaSuccess) {
    cudaGetLastError();
    *buf = nullptr;
    return LQR_ERR_OOM;
  }
  *cap = sz;
  return LQR_OK;
}

int ceil_div(int a, int b) { return (a + b - 1) / b; }

// The least stages a parametric segment needs to reach an arbitrary end state
// in the generic case: the constraint rank drops by m per stage (Section II-B).
int min_segment_len(int n, int m) { return ceil_div(n, m); }

int auto_segments(const lqr_handle* h, int n, int m, int T) {
  const int lmin = min_segment_len(n, m);
  int kmax = T / (lmin > 1 ? lmin : 1);
  // one segment per SM keeps every SM busy while the link chain stays short
  int K = h->num_sms > 0 ? h->num_sms : 128;
  if (K > T / 16) K = T / 16;
  if (K > kmax) K = kmax;
  if (K < 1) K = 1;
  return K;
}

bool elem_size(lqr_precision p, size_t* es) {
  switch (p) {
    case LQR_FP64: *es = 8; return true;
    case LQR_MIXED_TF32: *es = 8; return true;
    case LQR_FP32: *es = 4; return true;
    case LQR_MIXED_FP32: *es = 8; return true;
    default: return false;
  }
}

lqr_status validate(const lqr_problem* p, const lqr_opts* o, const lqr_solution* s) {
  if (!p || !o || !s) return LQR_ERR_INVALID_ARG;
  if (p->n < 1 || p->m < 1 || p->T < 1) return LQR_ERR_INVALID_ARG;
  if (p->n > 256 || p->m > 256) return LQR_ERR_INVALID_ARG;
  if (!p->A || !p->B || !p->c || !p->Q || !p->R || !p->q || !p->r || !p->x0) return LQR_ERR_INVALID_ARG;
  if ((s->P == nullptr) != (s->p == nullptr)) return LQR_ERR_INVALID_ARG;
  if (s->lam && (!s->x || !s->u)) return LQR_ERR_INVALID_ARG;
  if ((s->x || s->u) && (!s->K || !s->k)) return LQR_ERR_INVALID_ARG;  // the rollout reads K_t, k_t
  if (o->num_segments < 0 || o->num_segments > p->T) return LQR_ERR_INVALID_ARG;
  if (o->prec != LQR_FP64 && o->prec != LQR_FP32 && o->prec != LQR_MIXED_TF32 && o->prec != LQR_MIXED_FP32)
    return LQR_ERR_UNSUPPORTED;
  if (o->prec == LQR_MIXED_FP32 && o->form != LQR_FORM_MULTIPLIER) return LQR_ERR_UNSUPPORTED;
  if (o->form != LQR_FORM_MULTIPLIER && o->form != LQR_FORM_CONSTRAINED) return LQR_ERR_INVALID_ARG;
  if (o->max_refine < 0 || o->max_refine > 64) return LQR_ERR_INVALID_ARG;
  if ((o->max_refine > 0 || o->residual) && (!s->x || !s->u || !s->lam || !s->K || !s->k))
    return LQR_ERR_INVALID_ARG;
  if (o->max_refine > 0 && o->prec == LQR_FP32) return LQR_ERR_UNSUPPORTED;  // refinement needs FP64 data
  if (o->link != LQR_LINK_AUTO && o->link != LQR_LINK_CHAIN && o->link != LQR_LINK_SCAN) return LQR_ERR_INVALID_ARG;
  if (o->spin_limit < 0) return LQR_ERR_INVALID_ARG;
  if (o->link == LQR_LINK_SCAN && ((o->prec != LQR_FP32 && o->prec != LQR_MIXED_FP32) || o->form != LQR_FORM_MULTIPLIER))
    return LQR_ERR_UNSUPPORTED;
  return LQR_OK;
}

struct SolvePlan {
  int K;
  long long smem;
  long long scratch_doubles;  // per unit
  WsLayout wl;
  long long rbase;            // refinement buffers (doubles from the workspace base), or -1
  size_t ws_need;             // bytes
};

// Refinement buffers: correction data q~ r~ c~ x0~, corrections dk dx du dl dp,
// residual accumulators, skip flag.
struct RefineLayout {
  long long cq, cr, cc, cx0, dk, dx, du, dl, dp, acc, skip, total;
};
RefineLayout refine_layout(long long base, int n, int m, int T) {
  RefineLayout r;
  long long o = base;
  auto take = [&](long long cnt) { long long a = o; o += (cnt + 31) & ~31LL; return a; };
  r.cq = take((long long)(T + 1) * n);
  r.cr = take((long long)T * m);
  r.cc = take((long long)T * n);
  r.cx0 = take(n);
  r.dk = take((long long)T * m);
  r.dx = take((long long)(T + 1) * n);
  r.du = take((long long)T * m);
  r.dl = take((long long)(T + 1) * n);
  r.dp = take((long long)(T + 1) * n);
  r.acc = take(kResidAccDoubles);
  r.skip = take(4);
  r.total = o - base;
  return r;
}

lqr_status plan_solve(lqr_handle* h, const lqr_problem* p, const lqr_opts* o, SolvePlan* sp) {
  int K = o->num_segments > 0 ? o->num_segments : auto_segments(h, p->n, p->m, p->T);
  if (K > 1 && p->T / K < min_segment_len(p->n, p->m)) return LQR_ERR_SEGMENT_INFEASIBLE;
  sp->K = K;
  const long long budget = h->smem_optin - kStaticSmemReserve;
  const bool cons = (o->form == LQR_FORM_CONSTRAINED);
  if (o->prec == LQR_FP64)
    sp->smem = sweep_smem_needed<double, double>(p->n, p->m, budget, cons, &sp->scratch_doubles);
  else if (o->prec == LQR_MIXED_TF32)
    sp->smem = sweep_smem_needed<double, float>(p->n, p->m, budget, cons, &sp->scratch_doubles);
  else
    sp->smem = sweep_smem_needed<float, float>(p->n, p->m, budget, cons, &sp->scratch_doubles);
  sp->wl = ws_layout(p->n, K);
  long long total = sp->wl.total + (long long)K * sp->scratch_doubles;
  sp->rbase = -1;
  if (o->max_refine > 0 || o->residual) {
    sp->rbase = (total + 31) & ~31LL;
    total = sp->rbase + refine_layout(0, p->n, p->m, p->T).total;
  }
  sp->ws_need = sizeof(double) * (size_t)total + 256;
  return LQR_OK;
}

ProbDesc make_desc(lqr_handle* h, const lqr_problem* p, const lqr_solution* s, const SolvePlan& sp, int form) {
  ProbDesc d;
  memset(&d, 0, sizeof(d));
  d.A = p->A; d.B = p->B; d.c = p->c; d.Q = p->Q; d.R = p->R; d.S = p->S; d.q = p->q; d.r = p->r; d.x0 = p->x0;
  d.K = s->K; d.k = s->k; d.x = s->x; d.u = s->u; d.P = s->P; d.p = s->p; d.lam = s->lam;
  d.ws = reinterpret_cast<double*>(h->ws);
  d.scratch = d.ws + sp.wl.total;
  d.scratch_per_unit = sp.scratch_doubles;
  d.status = h->d_status;
  d.skip = nullptr;
  d.report = h->d_report;
  d.n = p->n; d.m = p->m; d.T = p->T; d.nseg = sp.K;
  d.unit0 = 0;
  d.form = form;
  return d;
}

// Records the boundary event `k` (0..kPhases) of the current profiled solve.
void prof_mark(lqr_handle* h, int k, cudaStream_t st) {
  if (!h->prof_on || h->prof_count >= lqr_handle::kMaxProfiled) return;
  cudaEventRecord(h->ev[h->prof_count][k], st);
}

// The arguments of the kernels of one refinement iteration (the key of the
// cached graph: compared byte by byte, so built from a zeroed struct).
struct RefineGraphArgs {
  ProbDesc main;
  CorrArgs ca;
  KktOut cvec;
  double* acc;
  int* skip;
  float* dp;
  double tol;
  int max_refine;
};
static_assert(sizeof(RefineGraphArgs) <= lqr_handle::kRKeyBytes, "graph key too large");

// One refinement iteration of the mixed modes (reuse path) on stream s: the
// residual pass (both forms, gated on the iteration count), the finalize that
// counts the iteration and sets the loop condition, the correction and the
// update. *cnt += kernels launched.
static bool refine_iteration(const RefineGraphArgs& a, cudaGraphConditionalHandle cond, cudaStream_t s, int* cnt) {
  const int n = a.main.n, m = a.main.m;
  if (launch_kkt_residual<double>(a.main, a.acc, a.cvec, a.skip, s, 0, 3) != cudaSuccess) return false;
  if (launch_residual_finalize_loop(a.main, a.acc, a.tol, a.skip, a.max_refine, cond, s) != cudaSuccess) return false;
  *cnt += (kkt_stage_cols(n, m) > 0 ? 2 : 1) + 1;
  if (launch_correction(a.ca, s, cnt) != cudaSuccess) return false;
  if (launch_refine_update_f32(a.main, a.ca.dk, a.ca.dx, a.ca.du, a.ca.dl, a.dp, a.skip, s) != cudaSuccess) return false;
  *cnt += 1;
  return true;
}

static void refine_graph_drop(lqr_handle* h) {
  if (h->rexec) cudaGraphExecDestroy(h->rexec);
  if (h->rgraph) cudaGraphDestroy(h->rgraph);
  h->rexec = nullptr;
  h->rgraph = nullptr;
  h->rkey_valid = 0;
}

// Launches the refinement loop as a graph on st (building it when the
// arguments differ from the cached graph's). false: no graph (a graph call
// failed; the caller launches the iterations itself from then on).
static bool refine_graph_launch(lqr_handle* h, const RefineGraphArgs& a, cudaStream_t st) {
  if (!h->rkey_valid || memcmp(h->rkey, &a, sizeof(a)) != 0) {
    refine_graph_drop(h);
    bool ok = (h->cap || cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) == cudaSuccess);
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle cond;
    alignas(cudaGraphNodeParams) unsigned char npbuf[sizeof(cudaGraphNodeParams)];
    memset(npbuf, 0, sizeof(npbuf));
    cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(npbuf);
    cudaGraphNode_t node;
    ok = ok && cudaGraphCreate(&g, 0) == cudaSuccess;
    ok = ok && cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = cond;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) == cudaSuccess;
    }
    int body = 0;
    if (ok) {
      cudaGraph_t bg = np.conditional.phGraph_out[0];
      ok = cudaStreamBeginCaptureToGraph(h->cap, bg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) == cudaSuccess;
      if (ok) {
        const bool launched = refine_iteration(a, cond, h->cap, &body);
        cudaGraph_t out = nullptr;
        ok = cudaStreamEndCapture(h->cap, &out) == cudaSuccess && launched;
      }
    }
    ok = ok && cudaGraphInstantiate(&h->rexec, g, 0) == cudaSuccess;
    h->rgraph = g;
    if (!ok) {
      cudaGetLastError();  // clear a sticky launch error of the capture, if any
      refine_graph_drop(h);
      h->rgraph_broken = 1;
      return false;
    }
    memcpy(h->rkey, &a, sizeof(a));
    h->rkey_valid = 1;
    h->rbody = body;
  }
  if (cudaGraphLaunch(h->rexec, st) != cudaSuccess) {
    refine_graph_drop(h);
    h->rgraph_broken = 1;
    return false;
  }
  return true;
}

// Steps A1 (and, unless summary_only, A3, A4, A5/A6) for the problem in tab.
// `profile` marks the phase boundaries of this pipeline.
lqr_status enqueue_pipeline(lqr_handle* h, const ProbTable& tab, const SolvePlan& sp, const lqr_opts* o,
                            bool want_traj, bool want_lam, int store_P, bool summary_only, bool profile,
                            cudaStream_t st, int* launches, bool tensor_cores = false) {
  const long long budget = h->smem_optin - kStaticSmemReserve;
  const int prec = o->prec;
  const bool dual = (o->form != LQR_FORM_CONSTRAINED);
  cudaError_t e;
  auto sweep = [&](int phase, cudaStream_t sst) {
    if (tensor_cores && phase == 1 && prec == LQR_FP32 && dual && tc_sweep_supported(tab.single.n, tab.single.m))
      return launch_seg_sweep_tc(tab, sp.K, store_P, o->spin_limit, sst);
    if (prec == LQR_FP64) return launch_seg_sweep<double, double>(tab, sp.K, phase, sp.smem, budget, store_P, sst);
    if (prec == LQR_MIXED_TF32) return launch_seg_sweep<double, float>(tab, sp.K, phase, sp.smem, budget, store_P, sst);
    if (dual) {
      const cudaError_t r = launch_seg_sweep_f32(tab, sp.K, phase, tab.single.n, tab.single.m, budget, store_P, sst);
      if (r != cudaErrorNotSupported) return r;
    }
    return launch_seg_sweep<float, float>(tab, sp.K, phase, sp.smem, budget, store_P, sst);
  };
  if (profile) prof_mark(h, LQR_PHASE_SWEEP, st);
  e = sweep(0, st);
  ++*launches;
  if (e != cudaSuccess) return LQR_ERR_CUDA;
  if (profile) prof_mark(h, LQR_PHASE_LINK, st);
  if (summary_only) {
    if (profile) {
      prof_mark(h, LQR_PHASE_POLICY, st);
      prof_mark(h, LQR_PHASE_ROLLOUT, st);
    }
    return LQR_OK;
  }
  const int x0f = (prec == LQR_FP32) ? 1 : 0;
  // FP32 multiplier form: the scan up to the final Pi_j, then the A4 sweep on the
  // side stream while the link feedback and link states run here
  bool scan_split = false;
  if (dual && prec == LQR_FP32 && o->link != LQR_LINK_CHAIN && sp.K > 1) {
    if (!h->side) {
      if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return LQR_ERR_CUDA;
    }
    int nl = 0;
    e = launch_link_scan(tab, x0f, st, &nl, 1);
    if (e == cudaSuccess) {
      scan_split = true;
      *launches += nl;
    } else if (e != cudaErrorNotSupported) {
      return LQR_ERR_CUDA;
    }
  }
  if (!scan_split) {
    // the boundary-coupling solve runs in FP64 except in the all-FP32 mode
    if (dual) {
      int nl = 0;
      // FP32 in the all-FP32 path; FP64 in the mixed modes where the cluster
      // chain holds the problem (n <= 67), beyond it the FP32 chain (an FP64
      // link step at n = 128 takes 4.4 ms on one SM)
      e = launch_link_solve_dual(tab, 1, x0f, st, prec == LQR_FP32 ? 1 : (prec == LQR_MIXED_TF32 ? 2 : 0), o->link,
                                 &nl);
      *launches += nl;
      if (e == cudaErrorNotSupported) return LQR_ERR_UNSUPPORTED;
    } else {
      e = launch_link_solve(tab, 1, x0f, st);
      ++*launches;
    }
    if (e != cudaSuccess) return LQR_ERR_CUDA;
  }
  if (profile) prof_mark(h, LQR_PHASE_POLICY, st);
  if (scan_split) {
    if (cudaEventRecord(h->ev_fork, st) != cudaSuccess || cudaStreamWaitEvent(h->side, h->ev_fork, 0) != cudaSuccess)
      return LQR_ERR_CUDA;
    e = sweep(1, h->side);
    ++*launches;
    if (e != cudaSuccess) return LQR_ERR_CUDA;
    if (cudaEventRecord(h->ev_join, h->side) != cudaSuccess) return LQR_ERR_CUDA;
    int nl = 0;
    e = launch_link_scan(tab, x0f, st, &nl, 2);
    *launches += nl;
    if (e != cudaSuccess) return LQR_ERR_CUDA;
    if (cudaStreamWaitEvent(st, h->ev_join, 0) != cudaSuccess) return LQR_ERR_CUDA;
  } else if (sp.K > 1) {
    e = sweep(1, st);
    ++*launches;
    if (e != cudaSuccess) return LQR_ERR_CUDA;
  }
  if (profile) prof_mark(h, LQR_PHASE_ROLLOUT, st);
  if (want_traj) {
    const int xu = (tab.single.x && tab.single.u) ? 1 : 0;
    if (prec == LQR_FP32)
      e = launch_rollout<float, float>(tab, sp.K, want_lam ? 1 : 0, st, 0, 0, xu);
    else
      e = launch_rollout<double, double>(tab, sp.K, want_lam ? 1 : 0, st, 0, 0, xu);
    ++*launches;
    if (e != cudaSuccess) return LQR_ERR_CUDA;
    e = launch_finalize(tab, 1, st);
    ++*launches;
    if (e != cudaSuccess) return LQR_ERR_CUDA;
  }
  return LQR_OK;
}

// LQR_MIXED_FP32: the FP32 path on an FP32 copy of the data, solution kept in
// FP64, FP64 residual and refinement corrections by the FP32 path.
// src (may be null): the inputs as device-visible pointers to host memory; the
// conversion then reads them once and also writes the FP64 copies into p's
// arrays. k_ready (may be null) is recorded once s->K holds its final values.
lqr_status run_solve_mixed32(lqr_handle* h, const lqr_problem* p, const lqr_opts* o, const lqr_solution* s,
                             cudaStream_t st, bool summary_only, SolvePlan* sp_out, bool tensor_cores = false,
                             const lqr_problem* src = nullptr, cudaEvent_t k_ready = nullptr) {
  SolvePlan sp;
  lqr_status rs = plan_solve(h, p, o, &sp);
  if (rs != LQR_OK) return rs;
  rs = grow(&h->ws, &h->ws_bytes, sp.ws_need);
  if (rs != LQR_OK) return rs;
  const int n = p->n, m = p->m, T = p->T, K = sp.K;
  const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm = (size_t)m * m;
  const bool want_P = (s->P != nullptr);
  // Corrections reuse the factorisation (K_t, P_t, M_uu^-1 of the solve; correct.cu)
  // when the FP32 fast sweeps run and the correction kernels' plans fit; otherwise
  // every correction is a whole FP32 solve.
  const long long budget = h->smem_optin - kStaticSmemReserve;
  int cslots = 0, cpsi_global = 0;
  corr_plan(n, m, budget, &cslots, &cpsi_global);
  const bool reuse = !summary_only && sp.rbase >= 0 && o->max_refine > 0 && cslots > 0;
  const bool keep_P = want_P || reuse;
  // FP32 working arrays (each 256-byte aligned)
  size_t off = 0;
  auto take = [&](size_t cnt) { const size_t a = off; off += (cnt + 63) & ~(size_t)63; return a; };
  const size_t oA = take((size_t)T * nn), oB = take((size_t)T * nm), oc = take((size_t)T * n),
               oQ = take((size_t)(T + 1) * nn), oR = take((size_t)T * mm), oS = p->S ? take((size_t)T * nm) : 0,
               oq = take((size_t)(T + 1) * n), orr = take((size_t)T * m), ox0 = take(n);
  const size_t oK = take((size_t)T * nm), ok = take((size_t)T * m), ox = take((size_t)(T + 1) * n),
               ou = take((size_t)T * m), ol = take((size_t)(T + 1) * n), oP = keep_P ? take((size_t)(T + 1) * nn) : 0,
               op = keep_P ? take((size_t)(T + 1) * n) : 0;
  const size_t ocq = take((size_t)(T + 1) * n), ocr = take((size_t)T * m), occ = take((size_t)T * n),
               ocx0 = take(n), odk = take((size_t)T * m), odx = take((size_t)(T + 1) * n), odu = take((size_t)T * m),
               odl = take((size_t)(T + 1) * n), odp = keep_P ? take((size_t)(T + 1) * n) : 0;
  const size_t cld = (size_t)corr_ld(n), blk = (size_t)(n + 1) * cld;
  const size_t oMi = reuse ? take((size_t)T * mm) : 0, oPhit = reuse ? take((size_t)T * blk) : 0,
               oPhiTt = reuse ? take((size_t)T * blk) : 0, oPsi = reuse ? take((size_t)K * blk) : 0,
               oPsiT = reuse ? take((size_t)K * blk) : 0, opcv = reuse ? take((size_t)T * cld) : 0,
               opb = reuse ? take((size_t)(K + 1) * n) : 0, oxb = reuse ? take((size_t)(K + 1) * n) : 0;
  // two-level correction link chains for long chains: groups of about sqrt(K) links
  int cG = 0, cng = 0;
  if (reuse && K >= 32 && (long long)corr_group_smem_bytes(n) <= budget) {
    cG = 1;
    while (cG * cG < K) ++cG;
    cng = (K + cG - 1) / cG;
  }
  const size_t oTh = cng ? take((size_t)cng * blk) : 0, oThT = cng ? take((size_t)cng * blk) : 0,
               ogY = cng ? take((size_t)(cng + 1) * n) : 0, ogX = cng ? take((size_t)(cng + 1) * n) : 0;
  rs = grow(&h->f32, &h->f32_bytes, sizeof(float) * off);
  if (rs != LQR_OK) return rs;
  float* f = reinterpret_cast<float*>(h->f32);
  lqr_problem p32 = *p;
  p32.A = f + oA; p32.B = f + oB; p32.c = f + oc; p32.Q = f + oQ; p32.R = f + oR; p32.S = p->S ? f + oS : nullptr;
  p32.q = f + oq; p32.r = f + orr; p32.x0 = f + ox0;
  lqr_solution s32;
  memset(&s32, 0, sizeof(s32));
  if (!summary_only) {
    s32.K = f + oK; s32.k = f + ok; s32.x = f + ox; s32.u = f + ou; s32.lam = f + ol;
    if (keep_P) { s32.P = f + oP; s32.p = f + op; }
  }
  {
    ConvTable<double, float> ct;
    ct.count = 0;
    const lqr_problem* cs = src ? src : p;  // where the conversion reads
    auto raw = [&](const void* d) { return src ? const_cast<void*>(d) : nullptr; };
    ct.add(cs->A, (void*)p32.A, (size_t)T * nn, raw(p->A));
    ct.add(cs->B, (void*)p32.B, (size_t)T * nm, raw(p->B));
    ct.add(cs->c, (void*)p32.c, (size_t)T * n, raw(p->c));
    ct.add(cs->Q, (void*)p32.Q, (size_t)(T + 1) * nn, raw(p->Q));
    ct.add(cs->R, (void*)p32.R, (size_t)T * mm, raw(p->R));
    ct.add(cs->S, (void*)p32.S, (size_t)T * nm, raw(p->S));
    ct.add(cs->q, (void*)p32.q, (size_t)(T + 1) * n, raw(p->q));
    ct.add(cs->r, (void*)p32.r, (size_t)T * m, raw(p->r));
    ct.add(cs->x0, (void*)p32.x0, (size_t)n, raw(p->x0));
    if (launch_convert(ct, nullptr, st) != cudaSuccess) return LQR_ERR_CUDA;
  }
  lqr_opts o32 = *o;
  o32.prec = LQR_FP32;
  ProbTable tab;
  memset(&tab, 0, sizeof(tab));
  tab.single = make_desc(h, &p32, &s32, sp, (int)o->form);
  if (reuse) tab.single.Minv = f + oMi;
  tab.nprob = 1;
  int launches = 1;
  if (cudaMemsetAsync(h->d_status, 0, 2 * sizeof(int), st) != cudaSuccess) return LQR_ERR_CUDA;
  if (cudaMemsetAsync(h->d_report, 0, 4 * sizeof(double), st) != cudaSuccess) return LQR_ERR_CUDA;
  rs = enqueue_pipeline(h, tab, sp, &o32, !summary_only, !summary_only, keep_P ? 1 : 0, summary_only, true, st,
                        &launches, tensor_cores);
  if (rs != LQR_OK) return rs;
  if (!summary_only) {
    ConvTable<float, double> ct;
    ct.count = 0;
    ct.add(s32.K, s->K, (size_t)T * nm);
    ct.add(s32.k, s->k, (size_t)T * m);
    ct.add(s32.x, s->x, (size_t)(T + 1) * n);
    ct.add(s32.u, s->u, (size_t)T * m);
    ct.add(s32.lam, s->lam, (size_t)(T + 1) * n);
    if (want_P) {
      ct.add(s32.P, s->P, (size_t)(T + 1) * nn);
      ct.add(s32.p, s->p, (size_t)(T + 1) * n);
    }
    if (launch_convert(ct, nullptr, st) != cudaSuccess) return LQR_ERR_CUDA;
    ++launches;
    // K_t is final here (the refinement corrects k, x, u, lambda and p only)
    if (k_ready && cudaEventRecord(k_ready, st) != cudaSuccess) return LQR_ERR_CUDA;
  }
  prof_mark(h, LQR_PHASE_REFINE, st);
  if (!summary_only && sp.rbase >= 0) {
    double* base = reinterpret_cast<double*>(h->ws);
    const RefineLayout rl = refine_layout(sp.rbase, n, m, T);
    double* acc = base + rl.acc;
    int* skip = reinterpret_cast<int*>(base + rl.skip);
    if (cudaMemsetAsync(acc, 0, sizeof(double) * kResidAccDoubles, st) != cudaSuccess) return LQR_ERR_CUDA;
    if (cudaMemsetAsync(skip, 0, 4 * sizeof(int), st) != cudaSuccess) return LQR_ERR_CUDA;
    const ProbDesc main = make_desc(h, p, s, sp, (int)o->form);
    // the correction problem: the FP32 matrices, FP32 copies of the residual vectors
    lqr_problem cp = p32;
    cp.q = f + ocq; cp.r = f + ocr; cp.c = f + occ; cp.x0 = f + ocx0;
    lqr_solution cs;
    cs.K = s32.K; cs.k = f + odk; cs.x = f + odx; cs.u = f + odu; cs.lam = f + odl;
    cs.P = want_P ? s32.P : nullptr;
    cs.p = want_P ? (void*)(f + odp) : nullptr;
    ProbTable ctab;
    memset(&ctab, 0, sizeof(ctab));
    ctab.single = make_desc(h, &cp, &cs, sp, (int)o->form);
    ctab.single.skip = skip;
    ctab.nprob = 1;
    CorrArgs ca;
    memset(&ca, 0, sizeof(ca));
    if (reuse) {
      ca.A = f + oA; ca.B = f + oB; ca.K = f + oK; ca.P = f + oP; ca.Minv = f + oMi;
      ca.cq = f + ocq; ca.cr = f + ocr; ca.cc = f + occ; ca.cx0 = f + ocx0;
      ca.Phit = f + oPhit; ca.PhiTt = f + oPhiTt; ca.Psi = f + oPsi; ca.PsiT = f + oPsiT; ca.pcv = f + opcv;
      ca.pb = f + opb; ca.xb = f + oxb;
      ca.dk = f + odk; ca.dp = f + odp; ca.dx = f + odx; ca.du = f + odu; ca.dl = f + odl;
      ca.skip = skip; ca.status = h->d_status;
      ca.n = n; ca.m = m; ca.T = T; ca.nseg = K;
      ca.slots = cslots; ca.psi_global = cpsi_global; ca.spin = o->spin_limit;
      ca.G = cG; ca.ng = cng;
      if (cng) { ca.Theta = f + oTh; ca.ThetaT = f + oThT; ca.gY = f + ogY; ca.gX = f + ogX; }
      if (launch_corr_psi(ca, st) != cudaSuccess) return LQR_ERR_CUDA;
      ++launches;
      if (cng) {
        if (launch_corr_groups(ca, st) != cudaSuccess) return LQR_ERR_CUDA;
        ++launches;
      }
    }
    // |KKT|_inf (data only) once, from the FP32 copy, so that whichever pass finds
    // the solution converged has the whole backward error
    if (o->max_refine > 0) {
      if (launch_kkt_norm_f32(tab.single, acc, st) != cudaSuccess) return LQR_ERR_CUDA;
      ++launches;
    }
    // the residual passes write the correction problem's vectors in FP32 directly
    KktOut cvec;
    memset(&cvec, 0, sizeof(cvec));
    cvec.q = (void*)cp.q; cvec.r = (void*)cp.r; cvec.c = (void*)cp.c; cvec.x0 = (void*)cp.x0; cvec.f32 = 1;
    h->last_iters = nullptr;
    bool looped = false;
    if (reuse && o->max_refine > 0 && !h->rgraph_broken && !o->refine_plain) {
      // the loop as a graph: one iteration's kernels under a WHILE node
      RefineGraphArgs ga;
      memset(&ga, 0, sizeof(ga));
      ga.main = main; ga.ca = ca; ga.cvec = cvec; ga.acc = acc; ga.skip = skip; ga.tol = o->tol;
      ga.max_refine = o->max_refine; ga.dp = want_P ? f + odp : nullptr;
      if (refine_graph_launch(h, ga, st)) {
        looped = true;
        h->last_iters = skip + 2;
        h->last_stream = st;
      }
    }
    for (int it = 0; it < o->max_refine && !looped; ++it) {
      // the first pass (the residual of the FP32 solve, some 2^-24 of |KKT| |w|)
      // in double-FP32 arithmetic (~2^-47 of it), the later ones in FP64
      if (launch_kkt_residual<double>(main, acc, cvec, skip, st, 0, it == 0 ? 1 : 0) != cudaSuccess)
        return LQR_ERR_CUDA;
      if (launch_residual_finalize(main, acc, o->tol, skip, 0, 0, st) != cudaSuccess) return LQR_ERR_CUDA;
      launches += 2;
      if (reuse) {
        if (launch_correction(ca, st, &launches) != cudaSuccess) return LQR_ERR_CUDA;
      } else {
        rs = enqueue_pipeline(h, ctab, sp, &o32, true, true, want_P ? 1 : 0, false, false, st, &launches,
                              tensor_cores);
        if (rs != LQR_OK) return rs;
      }
      if (launch_refine_update_f32(main, f + odk, f + odx, f + odu, f + odl, want_P ? f + odp : nullptr, skip, st) !=
          cudaSuccess)
        return LQR_ERR_CUDA;
      ++launches;
    }
    // final residual and objective, skipped on the device once refinement has converged
    if (launch_kkt_residual<double>(main, acc, KktOut{}, skip, st) != cudaSuccess) return LQR_ERR_CUDA;
    if (launch_residual_finalize(main, acc, o->tol, skip, 1, (o->max_refine > 0 && o->tol > 0) ? 1 : 0, st) !=
        cudaSuccess)
      return LQR_ERR_CUDA;
    launches += 2;
    h->last_resid = 1;
  } else {
    h->last_resid = 0;
  }
  prof_mark(h, LQR_NUM_PHASES, st);
  if (h->prof_on && h->prof_count < lqr_handle::kMaxProfiled) ++h->prof_count;
  h->last_K = sp.K;
  h->last_launches = launches;
  if (sp_out) *sp_out = sp;
  return LQR_OK;
}


// The launch sequence of one solve. `summary_only` stops after step A1.
lqr_status run_solve(lqr_handle* h, const lqr_problem* p, const lqr_opts* o, const lqr_solution* s,
                     cudaStream_t st, bool summary_only, SolvePlan* sp_out) {
  if (o->prec == LQR_MIXED_FP32) return run_solve_mixed32(h, p, o, s, st, summary_only, sp_out);
  // the mixed TF32 mode on the tensor-core plan: an FP32 copy of the data, the
  // policy sweeps on the tensor cores (FP64 factor of M_uu), FP64 refinement
  if (o->prec == LQR_MIXED_TF32 && o->form == LQR_FORM_MULTIPLIER && tc_sweep_supported(p->n, p->m))
    return run_solve_mixed32(h, p, o, s, st, summary_only, sp_out, true);
  SolvePlan sp;
  lqr_status rs = plan_solve(h, p, o, &sp);
  if (rs != LQR_OK) return rs;
  rs = grow(&h->ws, &h->ws_bytes, sp.ws_need);
  if (rs != LQR_OK) return rs;
  ProbTable tab;
  memset(&tab, 0, sizeof(tab));
  tab.single = make_desc(h, p, s, sp, (int)o->form);
  tab.nprob = 1;
  const int store_P = (s->P != nullptr) ? 1 : 0;
  int launches = 0;
  if (cudaMemsetAsync(h->d_status, 0, 2 * sizeof(int), st) != cudaSuccess) return LQR_ERR_CUDA;
  if (cudaMemsetAsync(h->d_report, 0, 4 * sizeof(double), st) != cudaSuccess) return LQR_ERR_CUDA;
  const bool want_traj = (s->x || s->u);
  rs = enqueue_pipeline(h, tab, sp, o, want_traj, s->lam != nullptr, store_P, summary_only, true, st, &launches);
  if (rs != LQR_OK) return rs;
  prof_mark(h, LQR_PHASE_REFINE, st);
  if (!summary_only && sp.rbase >= 0) {
    // ---- A7/A8: FP64 KKT residual and iterative refinement ---------------------
    double* base = reinterpret_cast<double*>(h->ws);
    const RefineLayout rl = refine_layout(sp.rbase, p->n, p->m, p->T);
    double* acc = base + rl.acc;
    int* skip = reinterpret_cast<int*>(base + rl.skip);
    if (cudaMemsetAsync(acc, 0, sizeof(double) * kResidAccDoubles, st) != cudaSuccess) return LQR_ERR_CUDA;
    if (cudaMemsetAsync(skip, 0, 4 * sizeof(int), st) != cudaSuccess) return LQR_ERR_CUDA;
    const ProbDesc& main = tab.single;
    // the correction problem: same matrices, residual vectors, corrections into the workspace
    lqr_problem cp = *p;
    cp.c = base + rl.cc; cp.q = base + rl.cq; cp.r = base + rl.cr; cp.x0 = base + rl.cx0;
    lqr_solution cs;
    cs.K = s->K; cs.k = base + rl.dk; cs.x = base + rl.dx; cs.u = base + rl.du; cs.lam = base + rl.dl;
    cs.P = s->P; cs.p = s->P ? (void*)(base + rl.dp) : nullptr;
    ProbTable ctab;
    memset(&ctab, 0, sizeof(ctab));
    ctab.single = make_desc(h, &cp, &cs, sp, (int)o->form);
    ctab.single.skip = skip;
    ctab.nprob = 1;
    for (int it = 0; it < o->max_refine; ++it) {
      // the first pass also takes |KKT|_inf, so that the pass that finds the
      // solution converged has the whole backward error
      const KktOut out{base + rl.cq, base + rl.cr, base + rl.cc, base + rl.cx0, 0};
      if (launch_kkt_residual<double>(main, acc, out, skip, st, it == 0 ? 1 : 0) != cudaSuccess) return LQR_ERR_CUDA;
      if (launch_residual_finalize(main, acc, o->tol, skip, 0, 0, st) != cudaSuccess) return LQR_ERR_CUDA;
      launches += 2;
      rs = enqueue_pipeline(h, ctab, sp, o, true, true, store_P, false, false, st, &launches);
      if (rs != LQR_OK) return rs;
      if (launch_refine_update<double>(main, base + rl.dk, base + rl.dx, base + rl.du, base + rl.dl,
                                       s->p ? base + rl.dp : nullptr, skip, st) != cudaSuccess)
        return LQR_ERR_CUDA;
      ++launches;
    }
    // final residual and objective of the returned solution (in the data's element
    // type), skipped on the device once refinement has converged
    const cudaError_t er = (o->prec == LQR_FP32)
        ? launch_kkt_residual<float>(main, acc, KktOut{}, skip, st)
        : launch_kkt_residual<double>(main, acc, KktOut{}, skip, st);
    if (er != cudaSuccess) return LQR_ERR_CUDA;
    if (launch_residual_finalize(main, acc, o->tol, skip, 1, (o->max_refine > 0 && o->tol > 0) ? 1 : 0, st) !=
        cudaSuccess)
      return LQR_ERR_CUDA;
    launches += 2;
    h->last_resid = 1;
  } else {
    h->last_resid = 0;
  }
  prof_mark(h, LQR_NUM_PHASES, st);
  if (h->prof_on && h->prof_count < lqr_handle::kMaxProfiled) ++h->prof_count;
  h->last_K = sp.K;
  h->last_launches = launches;
  if (sp_out) *sp_out = sp;
  return LQR_OK;
}

// Segment count per problem of a batch. With at least one problem per SM the
// batch alone fills the GPU and every problem runs as one plain Riccati sweep
// (K = 1: no parametric sweep, no link solve). Otherwise the stages are spread
// so that the batch forms about two units per SM, with segments of at least
// max(16, ceil(n/m)) stages.
int batch_segments(const lqr_handle* h, int nprob, const lqr_problem* probs, int i, long long total_T, int fixedK) {
  const lqr_problem& p = probs[i];
  const int lmin = min_segment_len(p.n, p.m);
  const int kmax = (lmin > 0) ? p.T / lmin : p.T;
  int K;
  if (fixedK > 0) {
    K = fixedK;
  } else if (nprob >= h->num_sms) {
    K = 1;
  } else {
    const double share = (double)p.T / (double)total_T;
    K = (int)(2.0 * h->num_sms * share + 0.5);
    const int by_len = p.T / (lmin > 16 ? lmin : 16);
    if (K > by_len) K = by_len;
  }
  if (K > kmax) K = kmax;
  if (K < 1) K = 1;
  return K;
}

lqr_status run_batched_impl(lqr_handle* h, int nprob, const lqr_problem* probs, const lqr_opts* o,
                            const lqr_solution* sols, int* segments_out, cudaStream_t st, bool persistent) {
  long long total_T = 0;
  int nmax = 0, mmax = 0;
  for (int i = 0; i < nprob; ++i) {
    total_T += probs[i].T;
    if (probs[i].n > nmax) nmax = probs[i].n;
    if (probs[i].m > mmax) mmax = probs[i].m;
  }
  const long long budget = h->smem_optin - kStaticSmemReserve;
  const bool cons = (o->form == LQR_FORM_CONSTRAINED);
  // pass 1: sizes
  long long ws_total = 0, smem_max = 0;
  int nunits = 0;
  bool any_split = false;
  struct Item { int K; long long off; long long scratch; };
  Item* items = (Item*)malloc(sizeof(Item) * (size_t)nprob);
  if (!items) return LQR_ERR_OOM;
  for (int i = 0; i < nprob; ++i) {
    const lqr_problem& p = probs[i];
    const int K = persistent ? 1 : batch_segments(h, nprob, probs, i, total_T, o->num_segments);
    if (K > 1 && p.T / K < min_segment_len(p.n, p.m)) { free(items); return LQR_ERR_SEGMENT_INFEASIBLE; }
    long long scratch = 0, smem = 0;
    if (o->prec == LQR_FP64) smem = sweep_smem_needed<double, double>(p.n, p.m, budget, cons, &scratch);
    else if (o->prec == LQR_MIXED_TF32) smem = sweep_smem_needed<double, float>(p.n, p.m, budget, cons, &scratch);
    else smem = sweep_smem_needed<float, float>(p.n, p.m, budget, cons, &scratch);
    if (smem > smem_max) smem_max = smem;
    const WsLayout wl = ws_layout(p.n, K);
    items[i].K = K;
    items[i].off = ws_total;
    items[i].scratch = scratch;
    ws_total += ((wl.total + (long long)K * scratch) + 31) & ~31LL;
    nunits += K;
    if (K > 1) any_split = true;
    if (segments_out) segments_out[i] = K;
  }
  lqr_status rs = grow(&h->ws, &h->ws_bytes, sizeof(double) * (size_t)ws_total + 256);
  if (rs != LQR_OK) { free(items); return rs; }
  // device table: descriptors | unit map | status (2 ints each) | report (4 doubles each)
  // device table: descriptors | unit map | LPT order | status (2 ints each) |
  // report (4 doubles each) | ticket of the persistent schedule
  const size_t desc_bytes = sizeof(ProbDesc) * (size_t)nprob;
  const size_t unit_bytes = sizeof(int) * (size_t)nunits + sizeof(int) * (size_t)nprob;
  const size_t stat_off = (desc_bytes + unit_bytes + 255) & ~(size_t)255;
  const size_t rep_off = (stat_off + sizeof(int) * 2 * (size_t)nprob + 255) & ~(size_t)255;
  const size_t tick_off = (rep_off + sizeof(double) * 4 * (size_t)nprob + 255) & ~(size_t)255;
  const size_t table_bytes = tick_off + 256;
  rs = grow(&h->bdev, &h->bdev_bytes, table_bytes);
  if (rs != LQR_OK) { free(items); return rs; }
  if (h->bhost_bytes < desc_bytes + unit_bytes) {
    if (h->bhost) { if (h->bhost_ev) cudaEventSynchronize(h->bhost_ev); cudaFreeHost(h->bhost); h->bhost = nullptr; }
    const size_t sz = desc_bytes + unit_bytes + (1 << 16);
    if (cudaMallocHost(&h->bhost, sz) != cudaSuccess) { cudaGetLastError(); h->bhost_bytes = 0; free(items); return LQR_ERR_OOM; }
    h->bhost_bytes = sz;
  }
  if (!h->bhost_ev && cudaEventCreateWithFlags(&h->bhost_ev, cudaEventDisableTiming) != cudaSuccess) {
    free(items);
    return LQR_ERR_CUDA;
  }
  cudaEventSynchronize(h->bhost_ev);  // the previous batch's table has left the staging buffer
  ProbDesc* hd = reinterpret_cast<ProbDesc*>(h->bhost);
  int* hu = reinterpret_cast<int*>(h->bhost + desc_bytes);
  double* wsb = reinterpret_cast<double*>(h->ws);
  int* dstat = reinterpret_cast<int*>(h->bdev + stat_off);
  double* drep = reinterpret_cast<double*>(h->bdev + rep_off);
  int u = 0;
  for (int i = 0; i < nprob; ++i) {
    const lqr_problem& p = probs[i];
    const lqr_solution& so = sols[i];
    ProbDesc d;
    memset(&d, 0, sizeof(d));
    d.A = p.A; d.B = p.B; d.c = p.c; d.Q = p.Q; d.R = p.R; d.S = p.S; d.q = p.q; d.r = p.r; d.x0 = p.x0;
    d.K = so.K; d.k = so.k; d.x = so.x; d.u = so.u; d.P = so.P; d.p = so.p; d.lam = so.lam;
    const WsLayout wl = ws_layout(p.n, items[i].K);
    d.ws = wsb + items[i].off;
    d.scratch = d.ws + wl.total;
    d.scratch_per_unit = items[i].scratch;
    d.status = dstat + 2 * i;
    d.skip = nullptr;
    d.report = drep + 4 * i;
    d.n = p.n; d.m = p.m; d.T = p.T; d.nseg = items[i].K;
    d.unit0 = u;
    d.form = (int)o->form;
    hd[i] = d;
    for (int j = 0; j < items[i].K; ++j) hu[u++] = i;
  }
  // longest processing time first: the queue order of the persistent schedule
  int* horder = hu + u;
  {
    for (int i = 0; i < nprob; ++i) horder[i] = i;
    double* work = (double*)malloc(sizeof(double) * (size_t)nprob);
    if (!work) { free(items); return LQR_ERR_OOM; }
    for (int i = 0; i < nprob; ++i) {
      const double n = probs[i].n, m = probs[i].m;
      work[i] = (double)probs[i].T * (4 * n * n * n + 6 * n * n * m + 4 * n * m * m + 2 * m * m * m);
    }
    std::sort(horder, horder + nprob, [&](int a, int b) { return work[a] > work[b] || (work[a] == work[b] && a < b); });
    free(work);
  }
  free(items);
  if (cudaMemcpyAsync(h->bdev, h->bhost, desc_bytes + unit_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return LQR_ERR_CUDA;
  cudaEventRecord(h->bhost_ev, st);
  if (cudaMemsetAsync(h->bdev + stat_off, 0, table_bytes - stat_off, st) != cudaSuccess) return LQR_ERR_CUDA;
  ProbTable tab;
  memset(&tab, 0, sizeof(tab));
  tab.probs = reinterpret_cast<const ProbDesc*>(h->bdev);
  tab.unit_prob = reinterpret_cast<const int*>(h->bdev + desc_bytes);
  tab.nprob = nprob;
  int launches = 0;
  int store_P = 0;
  bool want_traj = false, want_lam = false;
  int all_xu = 1;
  for (int i = 0; i < nprob; ++i) {
    if (sols[i].P) store_P = 1;
    if (sols[i].x || sols[i].u) want_traj = true;
    if (sols[i].lam) want_lam = true;
    if (!sols[i].x || !sols[i].u) all_xu = 0;
  }
  cudaError_t e;
  h->last_schedule = persistent ? 1 : 0;
  if (persistent) {
    prof_mark(h, LQR_PHASE_SWEEP, st);
    e = launch_batch_persistent(tab, reinterpret_cast<const int*>(h->bdev + desc_bytes) + nunits,
                                reinterpret_cast<int*>(h->bdev + tick_off), want_lam ? 1 : 0, nmax, mmax, store_P,
                                h->num_sms, st);
    if (e != cudaSuccess) return LQR_ERR_CUDA;
    for (int k = LQR_PHASE_LINK; k <= LQR_NUM_PHASES; ++k) prof_mark(h, k, st);
    if (h->prof_on && h->prof_count < lqr_handle::kMaxProfiled) ++h->prof_count;
    h->last_batch = nprob;
    h->bstatus_off = stat_off;
    h->breport_off = rep_off;
    h->last_launches = 1;
    h->last_K = nunits;
    return LQR_OK;
  }
  auto sweep = [&](int phase) {
    if (o->prec == LQR_FP64) return launch_seg_sweep<double, double>(tab, nunits, phase, smem_max, budget, store_P, st);
    if (o->prec == LQR_MIXED_TF32)
      return launch_seg_sweep<double, float>(tab, nunits, phase, smem_max, budget, store_P, st);
    if (!cons) {
      const cudaError_t r = launch_seg_sweep_f32(tab, nunits, phase, nmax, mmax, budget, store_P, st);
      if (r != cudaErrorNotSupported) return r;
    }
    return launch_seg_sweep<float, float>(tab, nunits, phase, smem_max, budget, store_P, st);
  };
  prof_mark(h, LQR_PHASE_SWEEP, st);
  e = sweep(0);
  ++launches;
  if (e != cudaSuccess) return LQR_ERR_CUDA;
  prof_mark(h, LQR_PHASE_LINK, st);
  const int x0f = (o->prec == LQR_FP32) ? 1 : 0;
  e = cons ? cudaErrorNotSupported : launch_link_solve_dual_batched(tab, nprob, nmax, x0f, st);
  if (cons) return LQR_ERR_UNSUPPORTED;
  ++launches;
  if (e != cudaSuccess) return LQR_ERR_CUDA;
  prof_mark(h, LQR_PHASE_POLICY, st);
  if (any_split) {
    e = sweep(1);
    ++launches;
    if (e != cudaSuccess) return LQR_ERR_CUDA;
  }
  prof_mark(h, LQR_PHASE_ROLLOUT, st);
  if (want_traj) {
    e = (o->prec == LQR_FP32) ? launch_rollout<float, float>(tab, nunits, want_lam ? 1 : 0, st, nmax, mmax, all_xu)
                              : launch_rollout<double, double>(tab, nunits, want_lam ? 1 : 0, st, nmax, mmax, all_xu);
    ++launches;
    if (e != cudaSuccess) return LQR_ERR_CUDA;
    e = launch_finalize(tab, nprob, st);
    ++launches;
    if (e != cudaSuccess) return LQR_ERR_CUDA;
  }
  prof_mark(h, LQR_PHASE_REFINE, st);
  prof_mark(h, LQR_NUM_PHASES, st);
  if (h->prof_on && h->prof_count < lqr_handle::kMaxProfiled) ++h->prof_count;
  h->last_batch = nprob;
  h->bstatus_off = stat_off;
  h->breport_off = rep_off;
  h->last_launches = launches;
  h->last_K = nunits;
  return LQR_OK;
}

int log2_bucket(long long v) {
  int b = 0;
  while (v > 1) { v >>= 1; ++b; }
  return b;
}

// The batch schedule (step A10). Batches of FP32 multiplier-form problems that
// want trajectories and fit the FP32 sweep and rollout plans can run as one
// persistent launch of one-segment problems; otherwise, or when the per-step
// launches (with the segment split of batch_segments) were measured faster for
// this batch shape, one launch per step. The autotuner times both schedules on
// the first batch of a shape bucket (problem count, largest n, m, horizon: the
// call synchronises the stream then) and keeps the faster in the handle.
lqr_status run_batched(lqr_handle* h, int nprob, const lqr_problem* probs, const lqr_opts* o,
                       const lqr_solution* sols, int* segments_out, cudaStream_t st) {
  int nmax = 0, mmax = 0, Tmax = 0;
  bool all_xu = true;
  for (int i = 0; i < nprob; ++i) {
    if (probs[i].n > nmax) nmax = probs[i].n;
    if (probs[i].m > mmax) mmax = probs[i].m;
    if (probs[i].T > Tmax) Tmax = probs[i].T;
    if (!sols[i].x || !sols[i].u) all_xu = false;
  }
  const long long budget = h->smem_optin - kStaticSmemReserve;
  const bool eligible = o->prec == LQR_FP32 && o->form == LQR_FORM_MULTIPLIER && o->num_segments <= 1 && all_xu &&
                        batch_persistent_supported(nmax, mmax, budget);
  if (!eligible) return run_batched_impl(h, nprob, probs, o, sols, segments_out, st, false);
  if (o->num_segments == 1) return run_batched_impl(h, nprob, probs, o, sols, segments_out, st, true);
  const int key[4] = {log2_bucket(nprob), nmax, mmax, log2_bucket(Tmax)};
  for (int i = 0; i < h->ntune; ++i)
    if (memcmp(h->tune[i].key, key, sizeof(key)) == 0)
      return run_batched_impl(h, nprob, probs, o, sols, segments_out, st, h->tune[i].persistent != 0);
  // measure both schedules on this batch (each once to warm up, once timed)
  cudaEvent_t ev[2];
  if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) return LQR_ERR_CUDA;
  float ms[2] = {0.f, 0.f};
  lqr_status rs = LQR_OK;
  for (int cand = 0; cand < 2 && rs == LQR_OK; ++cand) {
    for (int rep = 0; rep < 2 && rs == LQR_OK; ++rep) {
      if (rep == 1) cudaEventRecord(ev[0], st);
      rs = run_batched_impl(h, nprob, probs, o, sols, segments_out, st, cand == 1);
      if (rep == 1) cudaEventRecord(ev[1], st);
    }
    if (rs == LQR_OK && (cudaEventSynchronize(ev[1]) != cudaSuccess ||
                         cudaEventElapsedTime(&ms[cand], ev[0], ev[1]) != cudaSuccess))
      rs = LQR_ERR_CUDA;
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (rs != LQR_OK) return rs;
  const int pick = ms[1] <= ms[0] ? 1 : 0;
  if (h->ntune < 64) {
    lqr_handle::TuneEntry& te = h->tune[h->ntune++];
    memcpy(te.key, key, sizeof(key));
    te.persistent = pick;
    te.ms[0] = ms[0];
    te.ms[1] = ms[1];
  }
  // the outputs of the last (persistent) run stand; rerun only if the other schedule won
  if (pick == 0) return run_batched_impl(h, nprob, probs, o, sols, segments_out, st, false);
  return LQR_OK;
}

// Per-problem adjoint buffers (element size es): q~ r~ c~ x0~ | K~ k~ xi_x xi_u xi_l.
struct AdjLayout { size_t q, r, c, x0, K, k, x, u, l, total; };
AdjLayout adj_layout(size_t base, int n, int m, int T, size_t es) {
  AdjLayout a;
  size_t o = base;
  auto take = [&](size_t elems) { size_t r = o; o += (elems * es + 255) & ~(size_t)255; return r; };
  a.q = take((size_t)(T + 1) * n); a.r = take((size_t)T * m); a.c = take((size_t)T * n); a.x0 = take(n);
  a.K = take((size_t)T * m * n); a.k = take((size_t)T * m); a.x = take((size_t)(T + 1) * n);
  a.u = take((size_t)T * m); a.l = take((size_t)(T + 1) * n);
  a.total = o - base;
  return a;
}

lqr_status validate_backward(const lqr_problem* p, const lqr_opts* o, const lqr_solution* s, const lqr_problem* g) {
  if (!g) return LQR_ERR_INVALID_ARG;
  if (o && o->prec == LQR_MIXED_FP32) return LQR_ERR_UNSUPPORTED;
  if (!s || !s->x || !s->u || !s->lam) return LQR_ERR_INVALID_ARG;
  lqr_solution none;
  memset(&none, 0, sizeof(none));
  lqr_status v = validate(p, o, &none);
  if (v != LQR_OK) return v;
  if (g->n != p->n || g->m != p->m || g->T != p->T) return LQR_ERR_INVALID_ARG;
  return LQR_OK;
}

}  // namespace

extern "C" {

lqr_status lqr_backward(lqr_handle* h, const lqr_problem* prob, const lqr_opts* opts, const lqr_solution* sol,
                        const void* grad_x, const void* grad_u, const lqr_problem* grads, void* stream) {
  if (!h) return LQR_ERR_INVALID_ARG;
  lqr_status v = validate_backward(prob, opts, sol, grads);
  if (v != LQR_OK) return v;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  size_t es = 0;
  elem_size(opts->prec, &es);
  const int n = prob->n, m = prob->m, T = prob->T;
  const AdjLayout al = adj_layout(0, n, m, T, es);
  lqr_status r = grow(&h->adj, &h->adj_bytes, al.total);
  if (r != LQR_OK) return r;
  unsigned char* b = h->adj;
  cudaError_t e = (es == 8) ? launch_adjoint_rhs<double>(n, m, T, grad_x, grad_u, b + al.q, b + al.r, b + al.c, b + al.x0, st)
                            : launch_adjoint_rhs<float>(n, m, T, grad_x, grad_u, b + al.q, b + al.r, b + al.c, b + al.x0, st);
  if (e != cudaSuccess) return LQR_ERR_CUDA;
  lqr_problem ap = *prob;
  ap.q = b + al.q; ap.r = b + al.r; ap.c = b + al.c; ap.x0 = b + al.x0;
  lqr_solution as;
  memset(&as, 0, sizeof(as));
  as.K = b + al.K; as.k = b + al.k; as.x = b + al.x; as.u = b + al.u; as.lam = b + al.l;
  r = run_solve(h, &ap, opts, &as, st, false, nullptr);
  if (r != LQR_OK) return r;
  e = (es == 8) ? launch_adjoint_grad<double>(n, m, T, sol->x, sol->u, sol->lam, b + al.x, b + al.u, b + al.l, grads, st)
                : launch_adjoint_grad<float>(n, m, T, sol->x, sol->u, sol->lam, b + al.x, b + al.u, b + al.l, grads, st);
  if (e != cudaSuccess) return LQR_ERR_CUDA;
  h->last_launches += 2;
  return LQR_OK;
}

lqr_status lqr_backward_batched(lqr_handle* h, int nprob, const lqr_problem* probs, const lqr_opts* opts,
                                const lqr_solution* sols, const void* const* grad_x, const void* const* grad_u,
                                const lqr_problem* grads, void* stream) {
  if (!h || nprob < 1 || !probs || !opts || !sols || !grads) return LQR_ERR_INVALID_ARG;
  if (opts->max_refine > 0 || opts->residual || opts->form == LQR_FORM_CONSTRAINED) return LQR_ERR_UNSUPPORTED;
  for (int i = 0; i < nprob; ++i) {
    lqr_status v = validate_backward(&probs[i], opts, &sols[i], &grads[i]);
    if (v != LQR_OK) return v;
  }
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  size_t es = 0;
  elem_size(opts->prec, &es);
  size_t total = 0;
  int Tmax = 0;
  for (int i = 0; i < nprob; ++i) {
    total += adj_layout(0, probs[i].n, probs[i].m, probs[i].T, es).total;
    if (probs[i].T > Tmax) Tmax = probs[i].T;
  }
  // the job table of the adjoint's right-hand-side and gradient kernels follows the vectors
  const size_t job_off = (total + 255) & ~(size_t)255;
  const size_t jb = adjoint_job_bytes();
  lqr_status r = grow(&h->adj, &h->adj_bytes, job_off + jb * (size_t)nprob);
  if (r != LQR_OK) return r;
  lqr_problem* ap = (lqr_problem*)malloc(sizeof(lqr_problem) * (size_t)nprob);
  lqr_solution* as = (lqr_solution*)malloc(sizeof(lqr_solution) * (size_t)nprob);
  unsigned char* jobs = (unsigned char*)malloc(jb * (size_t)nprob);
  if (!ap || !as || !jobs) { free(ap); free(as); free(jobs); return LQR_ERR_OOM; }
  size_t off = 0;
  unsigned char* b = h->adj;
  for (int i = 0; i < nprob; ++i) {
    const lqr_problem& p = probs[i];
    const AdjLayout al = adj_layout(off, p.n, p.m, p.T, es);
    off += al.total;
    ap[i] = p;
    ap[i].q = b + al.q; ap[i].r = b + al.r; ap[i].c = b + al.c; ap[i].x0 = b + al.x0;
    memset(&as[i], 0, sizeof(lqr_solution));
    as[i].K = b + al.K; as[i].k = b + al.k; as[i].x = b + al.x; as[i].u = b + al.u; as[i].lam = b + al.l;
    adjoint_job_fill(jobs + jb * i, p.n, p.m, p.T, grad_x ? grad_x[i] : nullptr, grad_u ? grad_u[i] : nullptr,
                     b + al.q, b + al.r, b + al.c, b + al.x0, sols[i].x, sols[i].u, sols[i].lam, as[i].x, as[i].u,
                     as[i].lam, &grads[i]);
  }
  // pageable source: the copy is staged before the call returns, so `jobs` may be freed
  cudaError_t e = cudaMemcpyAsync(b + job_off, jobs, jb * (size_t)nprob, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = (es == 8) ? launch_adjoint_rhs_batched<double>(b + job_off, nprob, st)
                  : launch_adjoint_rhs_batched<float>(b + job_off, nprob, st);
  r = (e == cudaSuccess) ? run_batched(h, nprob, ap, opts, as, nullptr, st) : LQR_ERR_CUDA;
  if (r == LQR_OK) {
    e = (es == 8) ? launch_adjoint_grad_batched<double>(b + job_off, nprob, Tmax, st)
                  : launch_adjoint_grad_batched<float>(b + job_off, nprob, Tmax, st);
    if (e != cudaSuccess) r = LQR_ERR_CUDA;
    h->last_launches += 2;
  }
  free(jobs);
  free(ap);
  free(as);
  return r;
}


lqr_status lqr_solve_batched(lqr_handle* h, int nprob, const lqr_problem* probs, const lqr_opts* o,
                             const lqr_solution* sols, int* segments, void* stream) {
  if (!h || nprob < 1 || !probs || !o || !sols) return LQR_ERR_INVALID_ARG;
  for (int i = 0; i < nprob; ++i) {
    if (o->prec == LQR_MIXED_FP32) return LQR_ERR_UNSUPPORTED;
    lqr_status v = validate(&probs[i], o, &sols[i]);
    if (v != LQR_OK) return v;
  }
  if (o->max_refine > 0 || o->residual) return LQR_ERR_UNSUPPORTED;
  if (o->form == LQR_FORM_CONSTRAINED) return LQR_ERR_UNSUPPORTED;
  DeviceGuard g(h->device);
  return run_batched(h, nprob, probs, o, sols, segments, static_cast<cudaStream_t>(stream));
}

lqr_status lqr_report_batched(lqr_handle* h, void* stream, int nprob, int* status, double* cost) {
  if (!h || nprob < 1 || nprob > h->last_batch || !status) return LQR_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return LQR_ERR_CUDA;
  int* tmp = (int*)malloc(sizeof(int) * 2 * (size_t)nprob);
  double* rep = (double*)malloc(sizeof(double) * 4 * (size_t)nprob);
  if (!tmp || !rep) { free(tmp); free(rep); return LQR_ERR_OOM; }
  lqr_status r = LQR_OK;
  if (cudaMemcpy(tmp, h->bdev + h->bstatus_off, sizeof(int) * 2 * (size_t)nprob, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(rep, h->bdev + h->breport_off, sizeof(double) * 4 * (size_t)nprob, cudaMemcpyDeviceToHost) != cudaSuccess)
    r = LQR_ERR_CUDA;
  else
    for (int i = 0; i < nprob; ++i) {
      status[i] = tmp[2 * i];
      if (cost) cost[i] = rep[4 * i];
    }
  free(tmp);
  free(rep);
  return r;
}

lqr_status lqr_create(lqr_handle** out, int device, size_t workspace_hint) {
  if (!out) return LQR_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return LQR_ERR_CUDA;
  }
  DeviceGuard g(device);
  lqr_handle* h = new lqr_handle();
  h->device = device;
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
  h->num_sms = v;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  h->smem_optin = v;
  if (cudaMalloc(&h->d_status, 4 * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&h->d_report, 4 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    lqr_destroy(h);
    return LQR_ERR_OOM;
  }
  cudaMemset(h->d_status, 0, 4 * sizeof(int));
  cudaMemset(h->d_report, 0, 4 * sizeof(double));
  if (workspace_hint > 0 && grow(&h->ws, &h->ws_bytes, workspace_hint) != LQR_OK) {
    lqr_destroy(h);
    return LQR_ERR_OOM;
  }
  *out = h;
  return LQR_OK;
}

lqr_status lqr_destroy(lqr_handle* h) {
  if (!h) return LQR_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  cudaDeviceSynchronize();
  if (h->ws) cudaFree(h->ws);
  if (h->stage) cudaFree(h->stage);
  if (h->d_status) cudaFree(h->d_status);
  if (h->d_report) cudaFree(h->d_report);
  if (h->bdev) cudaFree(h->bdev);
  if (h->adj) cudaFree(h->adj);
  if (h->bhost) cudaFreeHost(h->bhost);
  if (h->bhost_ev) cudaEventDestroy(h->bhost_ev);
  if (h->ev_created)
    for (int i = 0; i < lqr_handle::kMaxProfiled; ++i)
      for (int k = 0; k <= lqr_handle::kPhases; ++k) cudaEventDestroy(h->ev[i][k]);
  if (h->f32) cudaFree(h->f32);
  if (h->nl) cudaFree(h->nl);
  if (h->rexec) cudaGraphExecDestroy(h->rexec);
  if (h->rgraph) cudaGraphDestroy(h->rgraph);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_kready) cudaEventDestroy(h->ev_kready);
  if (h->ev_kdone) cudaEventDestroy(h->ev_kdone);
  if (h->copy) cudaStreamDestroy(h->copy);
  if (h->side) cudaStreamDestroy(h->side);
  delete h;
  return LQR_OK;
}

lqr_status lqr_partition(int n, int m, int T, int K, int* bounds) {
  if (n < 1 || m < 1 || T < 1 || K < 1 || K > T || !bounds) return LQR_ERR_INVALID_ARG;
  if (K > 1 && T / K < min_segment_len(n, m)) return LQR_ERR_SEGMENT_INFEASIBLE;
  for (int j = 0; j <= K; ++j) bounds[j] = seg_begin(T, K, j);
  return LQR_OK;
}

lqr_status lqr_solve(lqr_handle* h, const lqr_problem* p, const lqr_opts* o, const lqr_solution* s, void* stream) {
  if (!h) return LQR_ERR_INVALID_ARG;
  lqr_status v = validate(p, o, s);
  if (v != LQR_OK) return v;
  DeviceGuard g(h->device);
  return run_solve(h, p, o, s, static_cast<cudaStream_t>(stream), false, nullptr);
}

lqr_status lqr_segment_policies(lqr_handle* h, const lqr_problem* p, const lqr_opts* o, int smooth, void* Kx,
                                void* Kz, void* k1, void* z, void* stream) {
  if (!h || !Kx || !k1) return LQR_ERR_INVALID_ARG;
  lqr_solution none;
  memset(&none, 0, sizeof(none));
  lqr_status v = validate(p, o, &none);
  if (v != LQR_OK) return v;
  if (o->prec != LQR_FP64 || o->form != LQR_FORM_CONSTRAINED || o->max_refine > 0) return LQR_ERR_UNSUPPORTED;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  lqr_opts o2 = *o;
  o2.residual = 0;
  SolvePlan sp;
  lqr_status rs = plan_solve(h, p, &o2, &sp);
  if (rs != LQR_OK) return rs;
  const int n = p->n, m = p->m, T = p->T, K = sp.K;
  const size_t ldp = 2 * (size_t)n + 1;
  const long long pol_off = ((sp.wl.total + (long long)K * sp.scratch_doubles) + 31) & ~31LL;
  const size_t need = sizeof(double) * ((size_t)pol_off + (size_t)T * m * ldp) + 256;
  rs = grow(&h->ws, &h->ws_bytes, need > sp.ws_need ? need : sp.ws_need);
  if (rs != LQR_OK) return rs;
  lqr_solution sol;
  memset(&sol, 0, sizeof(sol));
  if (smooth) { sol.K = Kx; sol.k = k1; }  // the policy sweeps write the smoothed gains
  ProbTable tab;
  memset(&tab, 0, sizeof(tab));
  tab.single = make_desc(h, p, &sol, sp, (int)LQR_FORM_CONSTRAINED);
  tab.nprob = 1;
  double* segpol = reinterpret_cast<double*>(h->ws) + pol_off;
  if (!smooth) tab.single.segpol = segpol;
  const long long budget = h->smem_optin - kStaticSmemReserve;
  int launches = 0;
  if (cudaMemsetAsync(h->d_status, 0, 2 * sizeof(int), st) != cudaSuccess) return LQR_ERR_CUDA;
  if (cudaMemsetAsync(h->d_report, 0, 4 * sizeof(double), st) != cudaSuccess) return LQR_ERR_CUDA;
  // A1: the constraint-explicit segment sweeps (and the last segment's Riccati sweep)
  if (launch_seg_sweep<double, double>(tab, K, 0, sp.smem, budget, 0, st) != cudaSuccess) return LQR_ERR_CUDA;
  ++launches;
  // A3: the link points (block elimination of the primal link system)
  if (launch_link_solve(tab, 1, 0, st) != cudaSuccess) return LQR_ERR_CUDA;
  ++launches;
  if (smooth) {
    tab.single.smooth = 1;
    if (K > 1) {
      if (launch_seg_sweep<double, double>(tab, K, 1, sp.smem, budget, 0, st) != cudaSuccess) return LQR_ERR_CUDA;
      ++launches;
    }
    if (Kz && cudaMemsetAsync(Kz, 0, sizeof(double) * (size_t)T * m * n, st) != cudaSuccess) return LQR_ERR_CUDA;
  } else {
    // [K_x | K_z | k_1] rows into the three outputs
    const size_t pitch = sizeof(double) * ldp;
    if (cudaMemcpy2DAsync(Kx, sizeof(double) * n, segpol, pitch, sizeof(double) * n, (size_t)T * m,
                          cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return LQR_ERR_CUDA;
    if (Kz && cudaMemcpy2DAsync(Kz, sizeof(double) * n, segpol + n, pitch, sizeof(double) * n, (size_t)T * m,
                                cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return LQR_ERR_CUDA;
    if (cudaMemcpy2DAsync(k1, sizeof(double), segpol + 2 * n, pitch, sizeof(double), (size_t)T * m,
                          cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return LQR_ERR_CUDA;
  }
  if (z && cudaMemcpyAsync(z, h->ws + sizeof(double) * sp.wl.z, sizeof(double) * (size_t)(K + 1) * n,
                           cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return LQR_ERR_CUDA;
  h->last_K = K;
  h->last_launches = launches;
  h->last_resid = 0;
  return LQR_OK;
}

lqr_status lqr_sqp_solve(lqr_handle* h, const lqr_nl_model* md, const lqr_sqp_opts* so, double* x, double* u,
                         double* lam, double* Kout, double* kout, lqr_sqp_report* rep, double* hist, void* stream) {
  if (!h || !md || !so || !x || !u || !rep) return LQR_ERR_INVALID_ARG;
  memset(rep, 0, sizeof(*rep));
  const int n = md->n, m = md->m, T = md->T;
  if (n < 1 || m < 1 || T < 1 || n > 256 || m > 256) return LQR_ERR_INVALID_ARG;
  if (!md->A || !md->B || !md->C || !md->Q || !md->R || !md->QT || !md->xref || !md->x0) return LQR_ERR_INVALID_ARG;
  if (so->max_iters < 1 || !(so->tol >= 0.0) || !(so->nu_min >= 0.0)) return LQR_ERR_INVALID_ARG;
  if (so->sub.prec != LQR_FP64 && so->sub.prec != LQR_MIXED_FP32) return LQR_ERR_UNSUPPORTED;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm = (size_t)m * m;
  // workspace: the subproblem's data, its solution where the caller gave none,
  // the merit partials
  size_t off = 0;
  auto take = [&](size_t cnt) { const size_t a = off; off += (cnt + 31) & ~(size_t)31; return a; };
  const size_t oA = take((size_t)T * nn), oB = take((size_t)T * nm), oc = take((size_t)T * n),
               oQ = take((size_t)(T + 1) * nn), oR = take((size_t)T * mm), oq = take((size_t)(T + 1) * n),
               or_ = take((size_t)T * m), ox0 = take(n), odx = take((size_t)(T + 1) * n), odu = take((size_t)T * m),
               olam = lam ? 0 : take((size_t)(T + 1) * n), oK = Kout ? 0 : take((size_t)T * nm),
               ok = kout ? 0 : take((size_t)T * m), opart = take((size_t)(T + 1) * kSqpOut), ores = take(kSqpOut);
  lqr_status rs = grow(&h->nl, &h->nl_bytes, sizeof(double) * off);
  if (rs != LQR_OK) return rs;
  double* b = reinterpret_cast<double*>(h->nl);
  NlModelDev dm;
  dm.A = md->A; dm.B = md->B; dm.C = md->C; dm.Q = md->Q; dm.R = md->R; dm.QT = md->QT;
  dm.xref = md->xref; dm.x0 = md->x0; dm.beta = md->beta; dm.n = n; dm.m = m; dm.T = T;
  lqr_problem sp;
  memset(&sp, 0, sizeof(sp));
  sp.n = n; sp.m = m; sp.T = T;
  sp.A = b + oA; sp.B = b + oB; sp.c = b + oc; sp.Q = b + oQ; sp.R = b + oR; sp.S = nullptr;
  sp.q = b + oq; sp.r = b + or_; sp.x0 = b + ox0;
  lqr_solution sol;
  memset(&sol, 0, sizeof(sol));
  double* dx = b + odx;
  double* du = b + odu;
  double* lm = lam ? lam : b + olam;
  sol.K = Kout ? Kout : b + oK; sol.k = kout ? kout : b + ok;
  sol.x = dx; sol.u = du; sol.lam = lm;
  lqr_opts o = so->sub;
  o.residual = 0;
  rs = validate(&sp, &o, &sol);
  if (rs != LQR_OK) return rs;
  int launches = 0;
  if (launch_sqp_fill(dm, b + oB, b + oQ, b + oR, st) != cudaSuccess) return LQR_ERR_CUDA;
  ++launches;
  double res[kSqpOut];
  int status[2];
  for (int it = 0; it < so->max_iters; ++it) {
    // the LQR subproblem at the iterate, its solution, the merit of every candidate step
    if (launch_sqp_linearize(dm, x, u, b + oA, b + oc, b + oq, b + or_, b + ox0, st) != cudaSuccess)
      return LQR_ERR_CUDA;
    rs = run_solve(h, &sp, &o, &sol, st, false, nullptr);
    if (rs != LQR_OK) return rs;
    launches += 1 + h->last_launches;
    if (launch_sqp_merit(dm, x, u, dx, du, b + oq, b + or_, lm, b + opart, b + ores, st) != cudaSuccess)
      return LQR_ERR_CUDA;
    launches += 2;
    if (cudaMemcpyAsync(res, b + ores, sizeof(res), cudaMemcpyDeviceToHost, st) != cudaSuccess) return LQR_ERR_CUDA;
    if (cudaMemcpyAsync(status, h->d_status, sizeof(status), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return LQR_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return LQR_ERR_CUDA;
    if (status[0] != 0) return static_cast<lqr_status>(status[0]);
    const double* J = res;
    const double* D = res + kSqpCand;
    const double gd = res[2 * kSqpCand], lmax = res[2 * kSqpCand + 1], dxm = res[2 * kSqpCand + 2],
                 dum = res[2 * kSqpCand + 3], xm = res[2 * kSqpCand + 4], um = res[2 * kSqpCand + 5];
    // step length: the first of 1, 1/2, ..., 1/128 with sufficient decrease of
    // the l1 merit J + nu D (Armijo), else the last; the full step once the
    // predicted decrease is at rounding level
    const double nu = fmax(so->nu_min, 2.0 * lmax);
    const double phi0 = J[0] + nu * D[0], slope = gd - nu * D[0];
    int a = 1;
    for (; a < kSqpCand; ++a) {
      const double al = sqp_alpha(a);
      if (fabs(slope) <= 1e-12 * fmax(1.0, fabs(phi0)) || J[a] + nu * D[a] <= phi0 + 1e-4 * al * slope) break;
    }
    if (a == kSqpCand) a = kSqpCand - 1;
    const double al = sqp_alpha(a);
    const double scale = fmax(1.0, fmax(xm, um));
    if (launch_sqp_update(x, u, dx, du, al, (long long)(T + 1) * n, (long long)T * m, st) != cudaSuccess)
      return LQR_ERR_CUDA;
    ++launches;
    const double step = al * fmax(dxm, dum);
    if (hist) {
      double* hr = hist + (size_t)LQR_SQP_HIST * it;
      hr[0] = al; hr[1] = J[a]; hr[2] = D[a]; hr[3] = J[a] + nu * D[a]; hr[4] = step; hr[5] = nu;
    }
    rep->iters = it + 1;
    rep->cost = J[a];
    rep->defect = D[a];
    rep->alpha = al;
    rep->step = step;
    if (step <= so->tol * scale && D[a] <= so->tol) {
      rep->converged = 1;
      break;
    }
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return LQR_ERR_CUDA;
  h->last_launches = launches;
  return LQR_OK;
}

lqr_status lqr_global_policy_parallel(lqr_handle* h, const lqr_problem* p, const lqr_opts* o, void* Kout,
                                      void* kout, void* Pout, void* pout, void* stream) {
  if (!h || !Kout || !kout || (Pout != nullptr) != (pout != nullptr)) return LQR_ERR_INVALID_ARG;
  lqr_solution none;
  memset(&none, 0, sizeof(none));
  lqr_status v = validate(p, o, &none);
  if (v != LQR_OK) return v;
  if (o->prec != LQR_FP64 || o->form != LQR_FORM_CONSTRAINED || o->max_refine > 0) return LQR_ERR_UNSUPPORTED;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  lqr_opts o2 = *o;
  o2.residual = 0;
  SolvePlan sp;
  lqr_status rs = plan_solve(h, p, &o2, &sp);
  if (rs != LQR_OK) return rs;
  const int n = p->n, m = p->m, T = p->T, K = sp.K;
  const long long nn = (long long)n * n;
  const long long budget = h->smem_optin - kStaticSmemReserve;
  const int on_chip = (long long)stage_policy_smem_bytes(n, 1) <= budget ? 1 : 0;
  // workspace: the solve's, then the segment policies, the per-stage values and
  // ranks, and (off chip) the per-stage factor buffers
  const long long pol_off = ((sp.wl.total + (long long)K * sp.scratch_doubles) + 31) & ~31LL;
  const long long sv_off = (pol_off + (long long)T * m * (2 * n + 1) + 31) & ~31LL;
  const long long rk_off = (sv_off + (long long)T * (3 * nn + 2 * n) + 31) & ~31LL;
  const long long sc_off = (rk_off + (T + 1) / 2 + 31) & ~31LL;
  const long long end = sc_off + (on_chip ? 0 : (long long)T * (nn + (long long)n * (n + 1)));
  const size_t need = sizeof(double) * (size_t)end + 256;
  rs = grow(&h->ws, &h->ws_bytes, need > sp.ws_need ? need : sp.ws_need);
  if (rs != LQR_OK) return rs;
  double* base = reinterpret_cast<double*>(h->ws);
  lqr_solution sol;
  memset(&sol, 0, sizeof(sol));
  sol.K = Kout; sol.k = kout; sol.P = Pout; sol.p = pout;
  ProbTable tab;
  memset(&tab, 0, sizeof(tab));
  tab.single = make_desc(h, p, &sol, sp, (int)LQR_FORM_CONSTRAINED);
  tab.single.segpol = base + pol_off;
  tab.single.stageV = base + sv_off;
  tab.single.stage_rank = reinterpret_cast<int*>(base + rk_off);
  tab.nprob = 1;
  const int store_P = (Pout && pout) ? 1 : 0;
  int launches = 0;
  if (cudaMemsetAsync(h->d_status, 0, 2 * sizeof(int), st) != cudaSuccess) return LQR_ERR_CUDA;
  if (cudaMemsetAsync(h->d_report, 0, 4 * sizeof(double), st) != cudaSuccess) return LQR_ERR_CUDA;
  // A1: the constraint-explicit segment sweeps, keeping every stage's cost to go,
  // rank and policy (the last segment: its Riccati sweep, global already)
  prof_mark(h, LQR_PHASE_SWEEP, st);
  if (launch_seg_sweep<double, double>(tab, K, 0, sp.smem, budget, store_P, st) != cudaSuccess) return LQR_ERR_CUDA;
  ++launches;
  prof_mark(h, LQR_PHASE_LINK, st);
  if (K > 1) {
    // A3: the link points and the global value at each of them
    if (launch_link_solve(tab, 1, 0, st) != cudaSuccess) return LQR_ERR_CUDA;
    ++launches;
  }
  prof_mark(h, LQR_PHASE_POLICY, st);
  if (K > 1) {
    // the stages whose constraint_to_go still has rows: the policy sweep from the
    // segment end, stopping at the first stage of rank 0
    if (launch_seg_sweep<double, double>(tab, K, 1, sp.smem, budget, store_P, st) != cudaSuccess)
      return LQR_ERR_CUDA;
    ++launches;
  }
  prof_mark(h, LQR_PHASE_ROLLOUT, st);
  if (K > 1) {
    // every other stage of segments 0 .. K-2 at once
    if (launch_stage_policy(tab.single, seg_begin(T, K, K - 1), on_chip, base + sc_off, st) != cudaSuccess)
      return LQR_ERR_CUDA;
    ++launches;
  }
  prof_mark(h, LQR_PHASE_REFINE, st);
  prof_mark(h, LQR_NUM_PHASES, st);
  if (h->prof_on && h->prof_count < lqr_handle::kMaxProfiled) ++h->prof_count;
  h->last_K = K;
  h->last_launches = launches;
  h->last_resid = 0;
  return LQR_OK;
}

lqr_status lqr_kkt_residual_vectors(lqr_handle* h, const lqr_problem* p, const lqr_solution* s, double* qt,
                                    double* rt, double* ct, double* x0t, void* stream) {
  if (!h || !p || !s || !qt || !rt || !ct || !x0t) return LQR_ERR_INVALID_ARG;
  if (!s->x || !s->u || !s->lam) return LQR_ERR_INVALID_ARG;
  lqr_opts o;
  memset(&o, 0, sizeof(o));
  o.prec = LQR_FP64;
  lqr_solution none;
  memset(&none, 0, sizeof(none));
  lqr_status v = validate(p, &o, &none);
  if (v != LQR_OK) return v;
  if (kkt_stage_cols(p->n, p->m) == 0) return LQR_ERR_UNSUPPORTED;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  lqr_status rs = grow(&h->ws, &h->ws_bytes, sizeof(double) * kResidAccDoubles);
  if (rs != LQR_OK) return rs;
  double* acc = reinterpret_cast<double*>(h->ws);
  SolvePlan sp;
  memset(&sp, 0, sizeof(sp));
  sp.K = 1;
  ProbDesc d = make_desc(h, p, s, sp, (int)LQR_FORM_MULTIPLIER);
  if (cudaMemsetAsync(h->d_status, 0, 2 * sizeof(int), st) != cudaSuccess) return LQR_ERR_CUDA;
  if (cudaMemsetAsync(acc, 0, sizeof(double) * kResidAccDoubles, st) != cudaSuccess) return LQR_ERR_CUDA;
  const KktOut out{qt, rt, ct, x0t, 0};
  if (launch_kkt_residual<double>(d, acc, out, nullptr, st, 0, 1) != cudaSuccess) return LQR_ERR_CUDA;
  h->last_launches = 1;
  h->last_resid = 0;
  return LQR_OK;
}

lqr_status lqr_ls_multipliers(lqr_handle* h, const lqr_problem* p, const lqr_opts* o, const double* x,
                              const double* u, double* lam, double* lam_end, double* mu, void* stream) {
  if (!h || !x || !u || !lam) return LQR_ERR_INVALID_ARG;
  lqr_solution none;
  memset(&none, 0, sizeof(none));
  lqr_status v = validate(p, o, &none);
  if (v != LQR_OK) return v;
  if (o->prec != LQR_FP64 || o->max_refine > 0) return LQR_ERR_UNSUPPORTED;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  lqr_opts o2 = *o;
  o2.residual = 0;
  SolvePlan sp;
  lqr_status rs = plan_solve(h, p, &o2, &sp);
  if (rs != LQR_OK) return rs;
  const int n = p->n, m = p->m, T = p->T, K = sp.K;
  if (K > 1 && (!lam_end || !mu)) return LQR_ERR_INVALID_ARG;
  LsArgs a;
  memset(&a, 0, sizeof(a));
  a.A = static_cast<const double*>(p->A); a.B = static_cast<const double*>(p->B);
  a.Q = static_cast<const double*>(p->Q); a.R = static_cast<const double*>(p->R);
  a.S = static_cast<const double*>(p->S); a.q = static_cast<const double*>(p->q);
  a.r = static_cast<const double*>(p->r);
  a.x = x; a.u = u; a.lam = lam; a.lam_end = lam_end; a.mu = mu;
  a.n = n; a.m = m; a.T = T; a.K = K;
  a.status = h->d_status;
  const long long budget = h->smem_optin - kStaticSmemReserve;
  a.on_chip = (long long)ls_mult_smem_bytes(n, m, 1) <= budget ? 1 : 0;
  if ((long long)ls_mult_smem_bytes(n, m, 0) > budget) return LQR_ERR_UNSUPPORTED;
  a.scratch_per_seg = (ls_mult_scratch_doubles(n, T, K) + 31) & ~31LL;
  rs = grow(&h->ws, &h->ws_bytes, sizeof(double) * (size_t)a.scratch_per_seg * K + 256);
  if (rs != LQR_OK) return rs;
  a.scratch = reinterpret_cast<double*>(h->ws);
  if (cudaMemsetAsync(h->d_status, 0, 2 * sizeof(int), st) != cudaSuccess) return LQR_ERR_CUDA;
  if (cudaMemsetAsync(h->d_report, 0, 4 * sizeof(double), st) != cudaSuccess) return LQR_ERR_CUDA;
  if (launch_ls_mult(a, st) != cudaSuccess) return LQR_ERR_CUDA;
  h->last_K = K;
  h->last_launches = 1;
  h->last_resid = 0;
  return LQR_OK;
}

lqr_status lqr_segment_summaries(lqr_handle* h, const lqr_problem* p, const lqr_opts* o, double* summaries,
                                 void* stream) {
  if (!h || !summaries) return LQR_ERR_INVALID_ARG;
  lqr_solution none;
  memset(&none, 0, sizeof(none));
  lqr_status v = validate(p, o, &none);
  if (v != LQR_OK) return v;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SolvePlan sp;
  lqr_status r = run_solve(h, p, o, &none, st, true, &sp);
  if (r != LQR_OK) return r;
  const size_t bytes = sizeof(double) * (size_t)sp.K * LQR_SUMMARY_DOUBLES(p->n);
  if (cudaMemcpyAsync(summaries, h->ws + sizeof(double) * sp.wl.summ, bytes, cudaMemcpyDeviceToDevice, st) !=
      cudaSuccess)
    return LQR_ERR_CUDA;
  return LQR_OK;
}

lqr_status lqr_solve_host(lqr_handle* h, const lqr_problem* ph, const lqr_opts* o, const lqr_solution* sh,
                          void* stream) {
  if (!h) return LQR_ERR_INVALID_ARG;
  lqr_status v = validate(ph, o, sh);
  if (v != LQR_OK) return v;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  size_t es = 0;
  elem_size(o->prec, &es);
  const size_t n = ph->n, m = ph->m, T = ph->T;
  struct Arr { const void* src; void* dst_host; size_t elems; bool in; };
  Arr arrs[16] = {
      {ph->A, nullptr, T * n * n, true},        {ph->B, nullptr, T * n * m, true},
      {ph->c, nullptr, T * n, true},            {ph->Q, nullptr, (T + 1) * n * n, true},
      {ph->R, nullptr, T * m * m, true},        {ph->S, nullptr, T * m * n, true},
      {ph->q, nullptr, (T + 1) * n, true},      {ph->r, nullptr, T * m, true},
      {ph->x0, nullptr, n, true},               {nullptr, sh->K, T * m * n, false},
      {nullptr, sh->k, T * m, false},           {nullptr, sh->x, (T + 1) * n, false},
      {nullptr, sh->u, T * m, false},           {nullptr, sh->P, (T + 1) * n * n, false},
      {nullptr, sh->p, (T + 1) * n, false},     {nullptr, sh->lam, (T + 1) * n, false}};
  size_t off[16], total = 0;
  for (int i = 0; i < 16; ++i) {
    off[i] = total;
    const bool used = arrs[i].in ? (arrs[i].src != nullptr) : (arrs[i].dst_host != nullptr);
    // K and k are needed on the device whenever x or u are requested
    const bool needed = used || (i == 9 || i == 10);
    if (needed) total += (arrs[i].elems * es + 255) & ~(size_t)255;
  }
  lqr_status r = grow(&h->stage, &h->stage_bytes, total);
  if (r != LQR_OK) return r;
  void* dptr[16];
  for (int i = 0; i < 16; ++i) dptr[i] = h->stage + off[i];
  // LQR_MIXED_FP32 with every input in page-locked host memory mapped into the
  // device's address space: the FP64 -> FP32 conversion reads the inputs over
  // the host link once and writes both the FP32 working copy and the FP64 copy
  // (the copy engines move the same bytes no faster; this saves the separate
  // pass over the FP64 copy). Anything else: copies by the copy engines.
  const void* mapped[9] = {nullptr};
  bool zero_copy = (o->prec == LQR_MIXED_FP32);
  for (int i = 0; i < 9 && zero_copy; ++i) {
    if (!arrs[i].src) continue;
    // both ends of the array mapped, at the same offset apart on the device side
    const size_t bytes = arrs[i].elems * es;
    const unsigned char* last = static_cast<const unsigned char*>(arrs[i].src) + bytes - 1;
    cudaPointerAttributes at, at_end;
    if (cudaPointerGetAttributes(&at, arrs[i].src) != cudaSuccess || at.type != cudaMemoryTypeHost ||
        at.devicePointer == nullptr || cudaPointerGetAttributes(&at_end, last) != cudaSuccess ||
        at_end.type != cudaMemoryTypeHost ||
        static_cast<const unsigned char*>(at_end.devicePointer) !=
            static_cast<const unsigned char*>(at.devicePointer) + (bytes - 1)) {
      cudaGetLastError();  // clear a lookup error of unregistered memory
      zero_copy = false;
    } else {
      mapped[i] = at.devicePointer;
    }
  }
  for (int i = 0; i < 9; ++i) {
    if (!arrs[i].src) { dptr[i] = nullptr; continue; }
    if (zero_copy) continue;
    if (cudaMemcpyAsync(dptr[i], arrs[i].src, arrs[i].elems * es, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return LQR_ERR_CUDA;
  }
  lqr_problem pd = *ph;
  pd.A = dptr[0]; pd.B = dptr[1]; pd.c = dptr[2]; pd.Q = dptr[3]; pd.R = dptr[4]; pd.S = dptr[5];
  pd.q = dptr[6]; pd.r = dptr[7]; pd.x0 = dptr[8];
  lqr_solution sd;
  sd.K = dptr[9]; sd.k = dptr[10];
  sd.x = sh->x ? dptr[11] : nullptr;
  sd.u = sh->u ? dptr[12] : nullptr;
  sd.P = sh->P ? dptr[13] : nullptr;
  sd.p = sh->p ? dptr[14] : nullptr;
  sd.lam = sh->lam ? dptr[15] : nullptr;
  if (o->prec == LQR_MIXED_FP32) {
    // the policies K_t go back on the copy stream while the refinement runs
    const bool k_early = arrs[9].dst_host != nullptr && o->max_refine > 0;
    if (k_early && !h->copy) {
      if (cudaStreamCreateWithFlags(&h->copy, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->ev_kready, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->ev_kdone, cudaEventDisableTiming) != cudaSuccess)
        return LQR_ERR_CUDA;
    }
    lqr_problem src = *ph;
    if (zero_copy) {
      src.A = mapped[0]; src.B = mapped[1]; src.c = mapped[2]; src.Q = mapped[3]; src.R = mapped[4];
      src.S = mapped[5]; src.q = mapped[6]; src.r = mapped[7]; src.x0 = mapped[8];
    }
    r = run_solve_mixed32(h, &pd, o, &sd, st, false, nullptr, false, zero_copy ? &src : nullptr,
                          k_early ? h->ev_kready : nullptr);
    if (r != LQR_OK) return r;
    if (k_early) {
      if (cudaStreamWaitEvent(h->copy, h->ev_kready, 0) != cudaSuccess ||
          cudaMemcpyAsync(arrs[9].dst_host, dptr[9], arrs[9].elems * es, cudaMemcpyDeviceToHost, h->copy) !=
              cudaSuccess ||
          cudaEventRecord(h->ev_kdone, h->copy) != cudaSuccess || cudaStreamWaitEvent(st, h->ev_kdone, 0) != cudaSuccess)
        return LQR_ERR_CUDA;
      arrs[9].dst_host = nullptr;  // copied
    }
  } else {
    r = run_solve(h, &pd, o, &sd, st, false, nullptr);
    if (r != LQR_OK) return r;
  }
  for (int i = 9; i < 16; ++i) {
    if (!arrs[i].dst_host) continue;
    if (cudaMemcpyAsync(arrs[i].dst_host, dptr[i], arrs[i].elems * es, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return LQR_ERR_CUDA;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return LQR_ERR_CUDA;
  return LQR_OK;
}

lqr_status lqr_report(lqr_handle* h, void* stream, lqr_report_t* out) {
  if (!h || !out) return LQR_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return LQR_ERR_CUDA;
  int stt[2] = {0, -1};
  double rep[4] = {0, 0, 0, 0};
  if (cudaMemcpy(stt, h->d_status, sizeof(stt), cudaMemcpyDeviceToHost) != cudaSuccess) return LQR_ERR_CUDA;
  if (cudaMemcpy(rep, h->d_report, sizeof(rep), cudaMemcpyDeviceToHost) != cudaSuccess) return LQR_ERR_CUDA;
  out->status = stt[0];
  out->bad_stage = stt[0] ? stt[1] : -1;
  out->num_segments = h->last_K;
  out->refine_iters = (int)rep[3];
  out->cost = rep[0];
  out->kkt_residual = h->last_resid ? rep[1] : -1.0;
  out->kkt_rel = h->last_resid ? rep[2] : -1.0;
  return LQR_OK;
}

const char* lqr_status_string(lqr_status s) {
  switch (s) {
    case LQR_OK: return "ok";
    case LQR_ERR_INVALID_ARG: return "invalid argument";
    case LQR_ERR_NOT_PD: return "not positive definite (R + B'PB or a link block)";
    case LQR_ERR_SEGMENT_INFEASIBLE: return "segment cannot absorb its end-point constraint";
    case LQR_ERR_NONFINITE: return "non-finite value";
    case LQR_ERR_NO_CONVERGENCE: return "iterative refinement did not converge";
    case LQR_ERR_TIMEOUT: return "bounded device wait expired";
    case LQR_ERR_CUDA: return "CUDA runtime error";
    case LQR_ERR_OOM: return "out of device memory";
    case LQR_ERR_UNSUPPORTED: return "unsupported request";
    case LQR_ERR_CAPACITY: return "problem exceeds the fixed capacity of this entry point";
  }
  return "unknown status";
}

int lqr_last_launch_count(const lqr_handle* h) {
  if (!h) return 0;
  if (!h->last_iters) return h->last_launches;
  // a refinement graph ran: its loop body ran as many times as the device counted
  DeviceGuard g(h->device);
  int iters = 0;
  if (cudaStreamSynchronize(h->last_stream) != cudaSuccess ||
      cudaMemcpy(&iters, h->last_iters, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return -1;
  return h->last_launches + h->rbody * iters;
}

lqr_status lqr_profile_enable(lqr_handle* h, int enable) {
  if (!h) return LQR_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  if (enable && !h->ev_created) {
    for (int i = 0; i < lqr_handle::kMaxProfiled; ++i)
      for (int k = 0; k <= lqr_handle::kPhases; ++k)
        if (cudaEventCreate(&h->ev[i][k]) != cudaSuccess) return LQR_ERR_CUDA;
    h->ev_created = 1;
  }
  h->prof_on = enable ? 1 : 0;
  h->prof_count = 0;
  return LQR_OK;
}

lqr_status lqr_profile_read(lqr_handle* h, double* phase_ms, int* solves) {
  if (!h || !phase_ms || !solves) return LQR_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  for (int k = 0; k < lqr_handle::kPhases; ++k) phase_ms[k] = 0.0;
  *solves = h->prof_count;
  for (int i = 0; i < h->prof_count; ++i) {
    if (cudaEventSynchronize(h->ev[i][lqr_handle::kPhases]) != cudaSuccess) return LQR_ERR_CUDA;
    for (int k = 0; k < lqr_handle::kPhases; ++k) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, h->ev[i][k], h->ev[i][k + 1]) != cudaSuccess) return LQR_ERR_CUDA;
      phase_ms[k] += ms;
    }
  }
  return LQR_OK;
}

}  // extern "C"
