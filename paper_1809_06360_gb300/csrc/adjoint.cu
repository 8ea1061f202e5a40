// Step A9: gradients of a loss L(x, u) of the optimal trajectory with respect
// to every problem datum, by the implicit function theorem on the KKT system
// of Eq. 3. With F(w, theta) = KKT(theta) w - b(theta) = 0 at the solution
// w = (x, u, lambda) and KKT symmetric,
//     dL/dtheta = -xi' dF/dtheta,   KKT xi = (dL/dx, dL/du, 0).
// KKT xi = g is the LQR problem with the same matrices and the vector data
// q~ = -dL/dx (q~_T = -dL/dx_T), r~ = -dL/du, c~ = 0, x0~ = 0, so xi is one
// more segment-parallel Riccati solve (the adjoint solve). Reading the blocks
// of F (Q and R symmetrised):
//     dL/dq_t = -xi_x,t            dL/dr_t = -xi_u,t          dL/dc_t  = xi_l,t+1
//     dL/dQ_t = -(xi_x x' + x xi_x')/2                        dL/dx0   = xi_l,0
//     dL/dR_t = -(xi_u u' + u xi_u')/2
//     dL/dS_t = -(u xi_x' + xi_u x')
//     dL/dA_t = lambda_{t+1} xi_x,t' + xi_l,t+1 x_t'
//     dL/dB_t = lambda_{t+1} xi_u,t' + xi_l,t+1 u_t'
// (xi_l = the multiplier part of xi, lambda = the forward multipliers).
#include <cuda_runtime.h>
#include <string.h>

#include "lqr_internal.cuh"

namespace lqr {

// One problem's adjoint job: its dimensions, dL/dx and dL/du (null = 0), the
// adjoint problem's vector data, the forward and adjoint solutions, and the
// gradient outputs (null = not wanted).
struct AdjJob {
  int n, m, T;
  const void *gx, *gu;
  void *q, *r, *c, *x0;
  const void *x, *u, *lam, *xix, *xiu, *xil;
  void *dA, *dB, *dc, *dQ, *dR, *dS, *dq, *dr, *dx0;
};

// Loads the adjoint problem's vector data: q~ = -gx, r~ = -gu, c~ = 0, x0~ = 0
// (blocks `blk` of `nblk` of the job).
template <typename TS>
__device__ __forceinline__ void adjoint_rhs_job(const AdjJob& jb, int blk, int nblk) {
  const int n = jb.n, m = jb.m, T = jb.T;
  const TS* gx = static_cast<const TS*>(jb.gx);
  const TS* gu = static_cast<const TS*>(jb.gu);
  TS* q = static_cast<TS*>(jb.q);
  TS* r = static_cast<TS*>(jb.r);
  TS* c = static_cast<TS*>(jb.c);
  TS* x0 = static_cast<TS*>(jb.x0);
  const size_t nx = (size_t)(T + 1) * n, nu = (size_t)T * m, nc = (size_t)T * n;
  const size_t ne = nx > nu ? nx : nu;
  for (size_t e = blk * (size_t)blockDim.x + threadIdx.x; e < ne; e += (size_t)nblk * blockDim.x) {
    if (e < nx) q[e] = gx ? static_cast<TS>(-gx[e]) : TS(0);
    if (e < nu) r[e] = gu ? static_cast<TS>(-gu[e]) : TS(0);
    if (e < nc) c[e] = TS(0);
    if (e < (size_t)n) x0[e] = TS(0);
  }
}
template <typename TS>
__global__ void adjoint_rhs_kernel(AdjJob jb) { adjoint_rhs_job<TS>(jb, blockIdx.x, gridDim.x); }
template <typename TS>
__global__ void adjoint_rhs_batched_kernel(const AdjJob* jobs) { adjoint_rhs_job<TS>(jobs[blockIdx.y], blockIdx.x, gridDim.x); }

// Stages dealt over blocks `blk` of `nblk` of the job; the terminal and initial
// terms by block 0.
template <typename TS>
__device__ __forceinline__ void adjoint_grad_job(const AdjJob& jb, int blk, int nblk) {
  const int n = jb.n, m = jb.m, T = jb.T;
  const TS* x = static_cast<const TS*>(jb.x);
  const TS* u = static_cast<const TS*>(jb.u);
  const TS* lam = static_cast<const TS*>(jb.lam);
  const TS* xix = static_cast<const TS*>(jb.xix);
  const TS* xiu = static_cast<const TS*>(jb.xiu);
  const TS* xil = static_cast<const TS*>(jb.xil);
  TS* dA = static_cast<TS*>(jb.dA);
  TS* dB = static_cast<TS*>(jb.dB);
  TS* dc = static_cast<TS*>(jb.dc);
  TS* dQ = static_cast<TS*>(jb.dQ);
  TS* dR = static_cast<TS*>(jb.dR);
  TS* dS = static_cast<TS*>(jb.dS);
  TS* dq = static_cast<TS*>(jb.dq);
  TS* dr = static_cast<TS*>(jb.dr);
  TS* dx0 = static_cast<TS*>(jb.dx0);
  const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm = (size_t)m * m;
  for (int t = blk; t < T; t += nblk) {
    const TS* xt = x + (size_t)n * t;
    const TS* ut = u + (size_t)m * t;
    const TS* ln = lam + (size_t)n * (t + 1);
    const TS* ax = xix + (size_t)n * t;
    const TS* au = xiu + (size_t)m * t;
    const TS* al = xil + (size_t)n * (t + 1);
    if (dA)
      for (size_t e = threadIdx.x; e < nn; e += blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        dA[nn * t + e] = static_cast<TS>((double)ln[i] * (double)ax[j] + (double)al[i] * (double)xt[j]);
      }
    if (dB)
      for (size_t e = threadIdx.x; e < nm; e += blockDim.x) {
        const int i = (int)(e / m), a = (int)(e % m);
        dB[nm * t + e] = static_cast<TS>((double)ln[i] * (double)au[a] + (double)al[i] * (double)ut[a]);
      }
    if (dQ)
      for (size_t e = threadIdx.x; e < nn; e += blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        dQ[nn * t + e] = static_cast<TS>(-0.5 * ((double)ax[i] * (double)xt[j] + (double)xt[i] * (double)ax[j]));
      }
    if (dR)
      for (size_t e = threadIdx.x; e < mm; e += blockDim.x) {
        const int a = (int)(e / m), b = (int)(e % m);
        dR[mm * t + e] = static_cast<TS>(-0.5 * ((double)au[a] * (double)ut[b] + (double)ut[a] * (double)au[b]));
      }
    if (dS)
      for (size_t e = threadIdx.x; e < nm; e += blockDim.x) {
        const int a = (int)(e / n), j = (int)(e % n);
        dS[nm * t + e] = static_cast<TS>(-((double)ut[a] * (double)ax[j] + (double)au[a] * (double)xt[j]));
      }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if (dc) dc[(size_t)n * t + i] = al[i];
      if (dq) dq[(size_t)n * t + i] = static_cast<TS>(-(double)ax[i]);
    }
    if (dr)
      for (int a = threadIdx.x; a < m; a += blockDim.x) dr[(size_t)m * t + a] = static_cast<TS>(-(double)au[a]);
  }
  if (blk == 0) {
    const TS* xT = x + (size_t)n * T;
    const TS* aT = xix + (size_t)n * T;
    if (dQ)
      for (size_t e = threadIdx.x; e < nn; e += blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        dQ[nn * T + e] = static_cast<TS>(-0.5 * ((double)aT[i] * (double)xT[j] + (double)xT[i] * (double)aT[j]));
      }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if (dq) dq[(size_t)n * T + i] = static_cast<TS>(-(double)aT[i]);
      if (dx0) dx0[i] = xil[i];
    }
  }
}
template <typename TS>
__global__ void __launch_bounds__(kBlock) adjoint_grad_kernel(AdjJob jb) { adjoint_grad_job<TS>(jb, blockIdx.x, gridDim.x); }
template <typename TS>
__global__ void __launch_bounds__(kBlock) adjoint_grad_batched_kernel(const AdjJob* jobs) {
  adjoint_grad_job<TS>(jobs[blockIdx.y], blockIdx.x, gridDim.x);
}

template <typename TS>
cudaError_t launch_adjoint_rhs(int n, int m, int T, const void* gx, const void* gu, void* q, void* r, void* c,
                               void* x0, cudaStream_t st) {
  AdjJob jb;
  memset(&jb, 0, sizeof(jb));
  jb.n = n; jb.m = m; jb.T = T; jb.gx = gx; jb.gu = gu; jb.q = q; jb.r = r; jb.c = c; jb.x0 = x0;
  adjoint_rhs_kernel<TS><<<2 * device_sm_count(), 256, 0, st>>>(jb);
  return cudaGetLastError();
}

template <typename TS>
cudaError_t launch_adjoint_grad(int n, int m, int T, const void* x, const void* u, const void* lam, const void* xix,
                                const void* xiu, const void* xil, const lqr_problem* g, cudaStream_t st) {
  AdjJob jb;
  memset(&jb, 0, sizeof(jb));
  jb.n = n; jb.m = m; jb.T = T; jb.x = x; jb.u = u; jb.lam = lam; jb.xix = xix; jb.xiu = xiu; jb.xil = xil;
  jb.dA = (void*)g->A; jb.dB = (void*)g->B; jb.dc = (void*)g->c; jb.dQ = (void*)g->Q; jb.dR = (void*)g->R;
  jb.dS = (void*)g->S; jb.dq = (void*)g->q; jb.dr = (void*)g->r; jb.dx0 = (void*)g->x0;
  const int grid = T < 4 * device_sm_count() ? T : 4 * device_sm_count();
  adjoint_grad_kernel<TS><<<grid, kBlock, 0, st>>>(jb);
  return cudaGetLastError();
}

// The batched forms: one launch each over a device table of njobs jobs
// (blocks per job on the x dimension, jobs on y).
template <typename TS>
cudaError_t launch_adjoint_rhs_batched(const void* jobs, int njobs, cudaStream_t st) {
  dim3 grid(4, njobs);
  adjoint_rhs_batched_kernel<TS><<<grid, 256, 0, st>>>(static_cast<const AdjJob*>(jobs));
  return cudaGetLastError();
}
template <typename TS>
cudaError_t launch_adjoint_grad_batched(const void* jobs, int njobs, int Tmax, cudaStream_t st) {
  dim3 grid(Tmax < 32 ? Tmax : 32, njobs);
  adjoint_grad_batched_kernel<TS><<<grid, kBlock, 0, st>>>(static_cast<const AdjJob*>(jobs));
  return cudaGetLastError();
}
size_t adjoint_job_bytes() { return sizeof(AdjJob); }
void adjoint_job_fill(void* dst, int n, int m, int T, const void* gx, const void* gu, void* q, void* r, void* c,
                      void* x0, const void* x, const void* u, const void* lam, const void* xix, const void* xiu,
                      const void* xil, const lqr_problem* g) {
  AdjJob jb;
  memset(&jb, 0, sizeof(jb));
  jb.n = n; jb.m = m; jb.T = T; jb.gx = gx; jb.gu = gu; jb.q = q; jb.r = r; jb.c = c; jb.x0 = x0;
  jb.x = x; jb.u = u; jb.lam = lam; jb.xix = xix; jb.xiu = xiu; jb.xil = xil;
  jb.dA = (void*)g->A; jb.dB = (void*)g->B; jb.dc = (void*)g->c; jb.dQ = (void*)g->Q; jb.dR = (void*)g->R;
  jb.dS = (void*)g->S; jb.dq = (void*)g->q; jb.dr = (void*)g->r; jb.dx0 = (void*)g->x0;
  memcpy(dst, &jb, sizeof(jb));
}

template cudaError_t launch_adjoint_rhs<double>(int, int, int, const void*, const void*, void*, void*, void*, void*,
                                                cudaStream_t);
template cudaError_t launch_adjoint_rhs<float>(int, int, int, const void*, const void*, void*, void*, void*, void*,
                                               cudaStream_t);
template cudaError_t launch_adjoint_grad<double>(int, int, int, const void*, const void*, const void*, const void*,
                                                 const void*, const void*, const lqr_problem*, cudaStream_t);
template cudaError_t launch_adjoint_grad<float>(int, int, int, const void*, const void*, const void*, const void*,
                                                const void*, const void*, const lqr_problem*, cudaStream_t);
template cudaError_t launch_adjoint_rhs_batched<double>(const void*, int, cudaStream_t);
template cudaError_t launch_adjoint_rhs_batched<float>(const void*, int, cudaStream_t);
template cudaError_t launch_adjoint_grad_batched<double>(const void*, int, int, cudaStream_t);
template cudaError_t launch_adjoint_grad_batched<float>(const void*, int, int, cudaStream_t);

}  // namespace lqr
