// C-ABI of liblqr: argument validation, workspace management and the launch
// sequence of one solve (Section II-C: split -> parametric segment sweeps ->
// link solve -> redistribution to the segments).
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "lqr_internal.cuh"

using namespace lqr;

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
  // phase profiling: one event pair per phase per solve, summed on read
  static constexpr int kPhases = LQR_NUM_PHASES;
  static constexpr int kMaxProfiled = 256;
  int prof_on = 0;
  int prof_count = 0;                       // solves recorded since enable
  cudaEvent_t ev[kMaxProfiled][kPhases + 1];
  int ev_created = 0;
  int prof_launches[kPhases] = {0};
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
  if (o->prec != LQR_FP64 && o->prec != LQR_FP32 && o->prec != LQR_MIXED_TF32) return LQR_ERR_UNSUPPORTED;
  if (o->form != LQR_FORM_MULTIPLIER && o->form != LQR_FORM_CONSTRAINED) return LQR_ERR_INVALID_ARG;
  if (o->max_refine < 0 || o->max_refine > 64) return LQR_ERR_INVALID_ARG;
  if ((o->max_refine > 0 || o->residual) && (!s->x || !s->u || !s->lam || !s->K || !s->k))
    return LQR_ERR_INVALID_ARG;
  if (o->max_refine > 0 && o->prec == LQR_FP32) return LQR_ERR_UNSUPPORTED;  // refinement needs FP64 data
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

// Steps A1 (and, unless summary_only, A3, A4, A5/A6) for the problem in tab.
// `profile` marks the phase boundaries of this pipeline.
lqr_status enqueue_pipeline(lqr_handle* h, const ProbTable& tab, const SolvePlan& sp, const lqr_opts* o,
                            bool want_traj, bool want_lam, int store_P, bool summary_only, bool profile,
                            cudaStream_t st, int* launches) {
  const long long budget = h->smem_optin - kStaticSmemReserve;
  const int prec = o->prec;
  const bool dual = (o->form != LQR_FORM_CONSTRAINED);
  cudaError_t e;
  auto sweep = [&](int phase) {
    if (prec == LQR_FP64) return launch_seg_sweep<double, double>(tab, sp.K, phase, sp.smem, budget, store_P, st);
    if (prec == LQR_MIXED_TF32) return launch_seg_sweep<double, float>(tab, sp.K, phase, sp.smem, budget, store_P, st);
    return launch_seg_sweep<float, float>(tab, sp.K, phase, sp.smem, budget, store_P, st);
  };
  if (profile) prof_mark(h, LQR_PHASE_SWEEP, st);
  e = sweep(0);
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
  e = dual ? launch_link_solve_dual(tab, 1, x0f, st) : launch_link_solve(tab, 1, x0f, st);
  ++*launches;
  if (e != cudaSuccess) return LQR_ERR_CUDA;
  if (profile) prof_mark(h, LQR_PHASE_POLICY, st);
  if (sp.K > 1) {
    e = sweep(1);
    ++*launches;
    if (e != cudaSuccess) return LQR_ERR_CUDA;
  }
  if (profile) prof_mark(h, LQR_PHASE_ROLLOUT, st);
  if (want_traj) {
    if (prec == LQR_FP32)
      e = launch_rollout<float, float>(tab, sp.K, want_lam ? 1 : 0, st);
    else
      e = launch_rollout<double, double>(tab, sp.K, want_lam ? 1 : 0, st);
    ++*launches;
    if (e != cudaSuccess) return LQR_ERR_CUDA;
    e = launch_finalize(tab, 1, st);
    ++*launches;
    if (e != cudaSuccess) return LQR_ERR_CUDA;
  }
  return LQR_OK;
}

// The launch sequence of one solve. `summary_only` stops after step A1.
lqr_status run_solve(lqr_handle* h, const lqr_problem* p, const lqr_opts* o, const lqr_solution* s,
                     cudaStream_t st, bool summary_only, SolvePlan* sp_out) {
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
      if (launch_kkt_residual<double>(main, acc, base + rl.cq, base + rl.cr, base + rl.cc, base + rl.cx0, skip, st) !=
          cudaSuccess)
        return LQR_ERR_CUDA;
      if (launch_residual_finalize(main, acc, o->tol, skip, 0, 0, st) != cudaSuccess) return LQR_ERR_CUDA;
      launches += 2;
      rs = enqueue_pipeline(h, ctab, sp, o, true, true, store_P, false, false, st, &launches);
      if (rs != LQR_OK) return rs;
      if (launch_refine_update<double>(main, base + rl.dk, base + rl.dx, base + rl.du, base + rl.dl,
                                       s->p ? base + rl.dp : nullptr, skip, st) != cudaSuccess)
        return LQR_ERR_CUDA;
      ++launches;
    }
    // final residual and objective of the returned solution
    if (launch_kkt_residual<double>(main, acc, nullptr, nullptr, nullptr, nullptr, nullptr, st) != cudaSuccess)
      return LQR_ERR_CUDA;
    if (launch_residual_finalize(main, acc, o->tol, nullptr, 1, (o->max_refine > 0 && o->tol > 0) ? 1 : 0, st) !=
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

}  // namespace

extern "C" {

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
  if (h->ev_created)
    for (int i = 0; i < lqr_handle::kMaxProfiled; ++i)
      for (int k = 0; k <= lqr_handle::kPhases; ++k) cudaEventDestroy(h->ev[i][k]);
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
  for (int i = 0; i < 9; ++i) {
    if (!arrs[i].src) { dptr[i] = nullptr; continue; }
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
  r = run_solve(h, &pd, o, &sd, st, false, nullptr);
  if (r != LQR_OK) return r;
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
  }
  return "unknown status";
}

int lqr_last_launch_count(const lqr_handle* h) { return h ? h->last_launches : 0; }

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
