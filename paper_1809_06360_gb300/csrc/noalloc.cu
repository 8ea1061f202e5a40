// KKT residual of a given solution without any device allocation.
//
// Callers such as hard real-time control loops (an MPC step that must finish
// inside a fixed cycle, with every allocation done at start-up) and code that
// runs inside another framework's stream capture cannot call cudaMalloc on
// their hot path, and cannot own an liblqr handle with its growable
// workspace. This file gives them one entry point whose scratch memory is a
// fixed, file-scope __device__ array instead: they pass the problem, the
// solution and a 3-double output buffer they allocated themselves.
//
// The kernel is a variant of the residual pass of the refinement step: the
// same per-stage residual blocks and row sums, with the objective summed
// from per-stage partials in stage order, and the final reduction done by the
// last CTA to finish (completion counter in the scratch array) so that one
// launch produces eta, rel and the objective.
#include <cuda_runtime.h>

#include <atomic>

#include "kkt_stage.cuh"
#include "lqr_internal.cuh"

namespace lqr {

namespace {

constexpr int kNoallocSlots = 8;  // [0] |r| [1] |KKT| [2] |w| [3] |b| [4] completion counter
constexpr size_t kNoallocDoubles = (size_t)LQR_NOALLOC_MAX_STAGES + 1 + kNoallocSlots;

// Shared by every call on a device: per-stage objective partials [0, T]
// followed by the reduction slots. Holds the last call's contents.
static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

struct NoallocArgs {
  const void *A, *B, *c, *Q, *R, *S, *q, *r, *x0, *x, *u, *lam;
  int n, m, T;
};

__device__ __forceinline__ void na_atomic_max(double* addr, double v) {
  if (!(v >= 0.0)) v = __longlong_as_double(0x7ff0000000000000LL);
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ double na_warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

static_assert(kBlock == kKktBlock, "the stage block of kkt_stage.cuh assumes kKktBlock threads");

// NC > 0: the stage block of kkt_stage.cuh (the arithmetic of the refinement
// residual pass, so both report the same numbers); NC = 0: n or m beyond its
// register plan, the per-stage loop below (the same arithmetic as the
// generic residual kernel of the refinement step).
template <int NC, typename TS>
__global__ void __launch_bounds__(kBlock) kkt_residual_noalloc_kernel(NoallocArgs a, double* scratch, double* out) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[5][kBlock / 32];
  __shared__ bool s_last;
  const int n = a.n, m = a.m, T = a.T;
  const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm = (size_t)m * m;
  double* slots = scratch + LQR_NOALLOC_MAX_STAGES + 1;
  double* xt = reinterpret_cast<double*>(smem);
  double* xn = xt + n;
  double* lt = xn + n;
  double* ln = lt + n;
  double* ut = ln + n;
  double* rxv = ut + m;
  double* ruv = rxv + n;
  double* rdv = ruv + m;
  const TS* gx = static_cast<const TS*>(a.x);
  const TS* gu = static_cast<const TS*>(a.u);
  const TS* gl = static_cast<const TS*>(a.lam);
  const TS* gA = static_cast<const TS*>(a.A);
  const TS* gB = static_cast<const TS*>(a.B);
  const TS* gc = static_cast<const TS*>(a.c);
  const TS* gQ = static_cast<const TS*>(a.Q);
  const TS* gR = static_cast<const TS*>(a.R);
  const TS* gS = static_cast<const TS*>(a.S);
  const TS* gq = static_cast<const TS*>(a.q);
  const TS* gr = static_cast<const TS*>(a.r);
  const TS* gx0 = static_cast<const TS*>(a.x0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double rmax = 0.0, kmax = 0.0, wmax = 0.0, bmax = 0.0;

  KktMax mx;
  KktData<TS> g;
  g.x = gx; g.u = gu; g.lam = gl; g.A = gA; g.B = gB; g.c = gc; g.Q = gQ; g.R = gR; g.S = gS; g.q = gq; g.r = gr;
  g.n = n; g.m = m;

  for (int t = blockIdx.x; t < T; t += gridDim.x) {
    double cost = 0.0;
    if constexpr (NC > 0) {
      cost = kkt_stage<NC, true>(g, t, reinterpret_cast<double*>(smem), mx, KktOut{});
    } else {
      const TS* At = gA + nn * t;
      const TS* Bt = gB + nm * t;
      const TS* Qt = gQ + nn * t;
      const TS* Rt = gR + mm * t;
      const TS* St = gS ? gS + nm * t : nullptr;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        xt[i] = (double)gx[(size_t)n * t + i];
        xn[i] = (double)gx[(size_t)n * (t + 1) + i];
        lt[i] = (double)gl[(size_t)n * t + i];
        ln[i] = (double)gl[(size_t)n * (t + 1) + i];
        rxv[i] = (double)gq[(size_t)n * t + i] + lt[i];
        rdv[i] = xn[i] - (double)gc[(size_t)n * t + i];
      }
      for (int b = threadIdx.x; b < m; b += blockDim.x) {
        ut[b] = (double)gu[(size_t)m * t + b];
        ruv[b] = (double)gr[(size_t)m * t + b];
      }
      __syncthreads();
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double s = 0.0, absA = 0.0, absS = 0.0, absQ = 0.0;
        for (int i = 0; i < n; ++i) {
          const double v = (double)At[(size_t)i * n + j];
          s = fma(-v, ln[i], s);
          s = fma(0.5 * (double)Qt[(size_t)i * n + j], xt[i], s);
          absA += fabs(v);
        }
        if (St)
          for (int b = 0; b < m; ++b) {
            const double v = (double)St[(size_t)b * n + j];
            s = fma(v, ut[b], s);
            absS += fabs(v);
          }
        for (int k = 0; k < n; ++k)
          absQ += fabs(0.5 * ((double)Qt[(size_t)j * n + k] + (double)Qt[(size_t)k * n + j]));
        rxv[j] += s;
        kmax = fmax(kmax, absQ + absS + 1.0 + absA);
      }
      for (int b = threadIdx.x; b < m; b += blockDim.x) {
        double s = 0.0, absB = 0.0, absR = 0.0, absSr = 0.0;
        for (int i = 0; i < n; ++i) {
          const double v = (double)Bt[(size_t)i * m + b];
          s = fma(-v, ln[i], s);
          absB += fabs(v);
        }
        for (int c2 = 0; c2 < m; ++c2) {
          s = fma(0.5 * (double)Rt[(size_t)c2 * m + b], ut[c2], s);
          absR += fabs(0.5 * ((double)Rt[(size_t)b * m + c2] + (double)Rt[(size_t)c2 * m + b]));
        }
        if (St)
          for (int k = 0; k < n; ++k) absSr += fabs((double)St[(size_t)b * n + k]);
        ruv[b] += s;
        kmax = fmax(kmax, absSr + absR + absB);
      }
      __syncthreads();
      for (int i = warp; i < n; i += nw) {
        double qx = 0.0, ax = 0.0, absr = 0.0;
        for (int k = lane; k < n; k += 32) {
          const double v = (double)At[(size_t)i * n + k];
          ax = fma(v, xt[k], ax);
          qx = fma((double)Qt[(size_t)i * n + k], xt[k], qx);
          absr += fabs(v);
        }
        for (int b = lane; b < m; b += 32) {
          const double v = (double)Bt[(size_t)i * m + b];
          ax = fma(v, ut[b], ax);
          absr += fabs(v);
        }
        qx = na_warp_sum(qx);
        ax = na_warp_sum(ax);
        absr = na_warp_sum(absr);
        if (lane == 0) {
          rxv[i] += 0.5 * qx;
          rdv[i] -= ax;
          kmax = fmax(kmax, 1.0 + absr);
          cost += xt[i] * (0.5 * qx + (double)gq[(size_t)n * t + i]);
        }
      }
      for (int b = warp; b < m; b += nw) {
        double sx = 0.0, ru = 0.0;
        if (St)
          for (int k = lane; k < n; k += 32) sx = fma((double)St[(size_t)b * n + k], xt[k], sx);
        for (int c2 = lane; c2 < m; c2 += 32) ru = fma((double)Rt[(size_t)b * m + c2], ut[c2], ru);
        sx = na_warp_sum(sx);
        ru = na_warp_sum(ru);
        if (lane == 0) {
          ruv[b] += sx + 0.5 * ru;
          cost += ut[b] * (sx + 0.5 * ru + (double)gr[(size_t)m * t + b]);
        }
      }
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        rmax = fmax(rmax, fmax(fabs(rxv[i]), fabs(rdv[i])));
        wmax = fmax(wmax, fmax(fabs(xt[i]), fabs(lt[i])));
        bmax = fmax(bmax, fmax(fabs((double)gq[(size_t)n * t + i]), fabs((double)gc[(size_t)n * t + i])));
      }
      for (int b = threadIdx.x; b < m; b += blockDim.x) {
        rmax = fmax(rmax, fabs(ruv[b]));
        wmax = fmax(wmax, fabs(ut[b]));
        bmax = fmax(bmax, fabs((double)gr[(size_t)m * t + b]));
      }
    }
    // this stage's objective partial, summed later in stage order
    cost = na_warp_sum(cost);
    if (lane == 0) red[4][warp] = cost;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += red[4][w];
      scratch[t] = s;
    }
    __syncthreads();
  }
  if (blockIdx.x == 0) {
    const TS* QT = gQ + nn * T;
    double cost = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double s = (double)gq[(size_t)n * T + i] + (double)gl[(size_t)n * T + i];
      double absQ = 0.0, qx = 0.0;
      for (int k = 0; k < n; ++k) {
        const double qs = 0.5 * ((double)QT[(size_t)i * n + k] + (double)QT[(size_t)k * n + i]);
        s = fma(qs, (double)gx[(size_t)n * T + k], s);
        qx = fma((double)QT[(size_t)i * n + k], (double)gx[(size_t)n * T + k], qx);
        absQ += fabs(qs);
      }
      const double xT = (double)gx[(size_t)n * T + i];
      cost += xT * (0.5 * qx + (double)gq[(size_t)n * T + i]);
      const double r0 = (double)gx[i] - (double)gx0[i];
      rmax = fmax(rmax, fmax(fabs(s), fabs(r0)));
      kmax = fmax(kmax, absQ + 1.0);
      wmax = fmax(wmax, fmax(fabs(xT), fabs((double)gl[(size_t)n * T + i])));
      bmax = fmax(bmax, fmax(fabs((double)gq[(size_t)n * T + i]), fabs((double)gx0[i])));
    }
    cost = na_warp_sum(cost);
    if (lane == 0) red[4][warp] = cost;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += red[4][w];
      scratch[T] = s;
    }
  }
  rmax = fmax(rmax, mx.r);
  kmax = fmax(kmax, mx.k);
  wmax = fmax(wmax, mx.w);
  bmax = fmax(bmax, mx.b);
  rmax = na_warp_max(rmax);
  kmax = na_warp_max(kmax);
  wmax = na_warp_max(wmax);
  bmax = na_warp_max(bmax);
  if (lane == 0) {
    red[0][warp] = rmax; red[1][warp] = kmax; red[2][warp] = wmax; red[3][warp] = bmax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double v[4] = {0, 0, 0, 0};
    for (int w = 0; w < nw; ++w)
      for (int k = 0; k < 4; ++k) v[k] = fmax(v[k], red[k][w]);
    for (int k = 0; k < 4; ++k) na_atomic_max(slots + k, v[k]);
    __threadfence();
    const unsigned int ticket = atomicAdd(reinterpret_cast<unsigned int*>(slots + 4), 1u);
    s_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  // the last CTA: the objective from the stage partials in stage order, then eta and rel
  __threadfence();
  const volatile double* vs = scratch;
  const int per = (T + 1 + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per;
  const int b1 = min(T + 1, b0 + per);
  double part = 0.0;
  for (int t = b0; t < b1; ++t) part += vs[t];
  __shared__ double parts[kBlock];
  parts[threadIdx.x] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double cost = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) cost += parts[i];
    const volatile double* vsl = slots;
    const double r = vsl[0], k = vsl[1], w = vsl[2], bn = vsl[3];
    out[0] = r / (k * w + bn);
    out[1] = bn > 0.0 ? r / bn : r;
    out[2] = cost;
  }
}

// Device address of g_noalloc_scratch per device, published with release
// order once looked up (the lookup is idempotent, so two host threads making
// the first call on a device at the same time both store the same address).
static std::atomic<double*> g_dev_scratch[64];

}  // namespace

}  // namespace lqr

using namespace lqr;

extern "C" lqr_status lqr_kkt_residual_noalloc(const lqr_problem* p, const lqr_solution* s, lqr_precision prec,
                                               double* out, void* stream) {
  if (!p || !s || !out) return LQR_ERR_INVALID_ARG;
  if (p->n < 1 || p->m < 1 || p->T < 1 || p->n > 256 || p->m > 256) return LQR_ERR_INVALID_ARG;
  if (!p->A || !p->B || !p->c || !p->Q || !p->R || !p->q || !p->r || !p->x0) return LQR_ERR_INVALID_ARG;
  if (!s->x || !s->u || !s->lam) return LQR_ERR_INVALID_ARG;
  // the mixed modes keep data and solution in FP64
  if (prec != LQR_FP64 && prec != LQR_FP32 && prec != LQR_MIXED_TF32 && prec != LQR_MIXED_FP32)
    return LQR_ERR_UNSUPPORTED;
  if (p->T > LQR_NOALLOC_MAX_STAGES) return LQR_ERR_CAPACITY;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LQR_ERR_CUDA;
  double* scratch = g_dev_scratch[dev].load(std::memory_order_acquire);
  if (!scratch) {
    // once per device, with that device current: the device address of the
    // scratch array (its host-side name is only a stand-in)
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return LQR_ERR_CUDA;
    }
    scratch = static_cast<double*>(ptr);
    g_dev_scratch[dev].store(scratch, std::memory_order_release);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the reduction slots and the completion counter start at zero on every call
  if (cudaMemsetAsync(scratch + LQR_NOALLOC_MAX_STAGES + 1, 0, sizeof(double) * kNoallocSlots, st) != cudaSuccess)
    return LQR_ERR_CUDA;
  NoallocArgs a;
  a.A = p->A; a.B = p->B; a.c = p->c; a.Q = p->Q; a.R = p->R; a.S = p->S; a.q = p->q; a.r = p->r; a.x0 = p->x0;
  a.x = s->x; a.u = s->u; a.lam = s->lam;
  a.n = p->n; a.m = p->m; a.T = p->T;
  const int grid = p->T < 4 * device_sm_count() ? p->T : 4 * device_sm_count();
  const int nc = kkt_stage_cols(p->n, p->m);
  size_t bytes = sizeof(double) * (6 * (size_t)p->n + 3 * (size_t)p->m);
  if (nc > 0) bytes = sizeof(double) * kkt_stage_smem_doubles(p->n, p->m);  // <= 45056 B: no opt-in needed
#define LQR_NA_LAUNCH(NC)                                                  \
  do {                                                                     \
    if (prec == LQR_FP32)                                                  \
      kkt_residual_noalloc_kernel<NC, float><<<grid, kBlock, bytes, st>>>(a, scratch, out);  \
    else                                                                   \
      kkt_residual_noalloc_kernel<NC, double><<<grid, kBlock, bytes, st>>>(a, scratch, out); \
  } while (0)
  switch (nc) {
    case 1: LQR_NA_LAUNCH(1); break;
    case 2: LQR_NA_LAUNCH(2); break;
    case 4: LQR_NA_LAUNCH(4); break;
    default: LQR_NA_LAUNCH(0); break;
  }
#undef LQR_NA_LAUNCH
  return cudaGetLastError() == cudaSuccess ? LQR_OK : LQR_ERR_CUDA;
}
