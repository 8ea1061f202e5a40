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

#include "lqr_internal.cuh"

namespace lqr {

// Loads the adjoint problem's vector data: q~ = -gx, r~ = -gu, c~ = 0, x0~ = 0.
template <typename TS>
__global__ void adjoint_rhs_kernel(int n, int m, int T, const TS* gx, const TS* gu, TS* q, TS* r, TS* c, TS* x0) {
  const size_t nx = (size_t)(T + 1) * n, nu = (size_t)T * m, nc = (size_t)T * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nx; e += (size_t)gridDim.x * blockDim.x) {
    q[e] = gx ? static_cast<TS>(-gx[e]) : TS(0);
    if (e < nu) r[e] = gu ? static_cast<TS>(-gu[e]) : TS(0);
    if (e < nc) c[e] = TS(0);
    if (e < (size_t)n) x0[e] = TS(0);
  }
}

// One CTA per stage (grid-stride); writes the gradients of stage t (and the
// terminal / initial terms from the CTA of t = 0). Output pointers may be null.
template <typename TS>
__global__ void __launch_bounds__(kBlock) adjoint_grad_kernel(int n, int m, int T, const TS* x, const TS* u,
                                                              const TS* lam, const TS* xix, const TS* xiu,
                                                              const TS* xil, TS* dA, TS* dB, TS* dc, TS* dQ, TS* dR,
                                                              TS* dS, TS* dq, TS* dr, TS* dx0) {
  const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm = (size_t)m * m;
  for (int t = blockIdx.x; t < T; t += gridDim.x) {
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
  if (blockIdx.x == 0) {
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
cudaError_t launch_adjoint_rhs(int n, int m, int T, const void* gx, const void* gu, void* q, void* r, void* c,
                               void* x0, cudaStream_t st) {
  adjoint_rhs_kernel<TS><<<2 * device_sm_count(), 256, 0, st>>>(n, m, T, static_cast<const TS*>(gx), static_cast<const TS*>(gu),
                                                  static_cast<TS*>(q), static_cast<TS*>(r), static_cast<TS*>(c),
                                                  static_cast<TS*>(x0));
  return cudaGetLastError();
}

template <typename TS>
cudaError_t launch_adjoint_grad(int n, int m, int T, const void* x, const void* u, const void* lam, const void* xix,
                                const void* xiu, const void* xil, const lqr_problem* g, cudaStream_t st) {
  const int grid = T < 4 * device_sm_count() ? T : 4 * device_sm_count();
  adjoint_grad_kernel<TS><<<grid, kBlock, 0, st>>>(
      n, m, T, static_cast<const TS*>(x), static_cast<const TS*>(u), static_cast<const TS*>(lam),
      static_cast<const TS*>(xix), static_cast<const TS*>(xiu), static_cast<const TS*>(xil),
      (TS*)g->A, (TS*)g->B, (TS*)g->c, (TS*)g->Q, (TS*)g->R, (TS*)g->S, (TS*)g->q, (TS*)g->r, (TS*)g->x0);
  return cudaGetLastError();
}

template cudaError_t launch_adjoint_rhs<double>(int, int, int, const void*, const void*, void*, void*, void*, void*,
                                                cudaStream_t);
template cudaError_t launch_adjoint_rhs<float>(int, int, int, const void*, const void*, void*, void*, void*, void*,
                                               cudaStream_t);
template cudaError_t launch_adjoint_grad<double>(int, int, int, const void*, const void*, const void*, const void*,
                                                 const void*, const void*, const lqr_problem*, cudaStream_t);
template cudaError_t launch_adjoint_grad<float>(int, int, int, const void*, const void*, const void*, const void*,
                                                const void*, const void*, const lqr_problem*, cudaStream_t);

}  // namespace lqr
