/*
 * FP64 serial Riccati recursion: the correctness oracle for the LQR solver.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path links, loads or calls
 * this file; the tests, the smoke check and the CPU-baseline leg of the bench
 * are its only users. It shares no code with the CUDA library.
 *
 * What it computes (Section II, Eq. 1-2 and the KKT conditions Eq. 3 of the
 * paper): the unique minimiser of the strictly convex finite-horizon problem
 *     sum_{t<T} 1/2 x'Q_t x + u'S_t x + 1/2 u'R_t u + q_t'x + r_t'u
 *       + 1/2 x_T'Q_T x_T + q_T'x_T
 *     s.t. x_{t+1} = A_t x_t + B_t u_t + c_t,  x_0 = x0,
 * by plain dynamic programming (the serial Riccati recursion that Section III-A
 * compares the parallel method against). With the value function
 * V_t(x) = 1/2 x'P_t x + p_t'x + s_t:
 *     P_T = Q_T, p_T = q_T, s_T = 0
 *     for t = T-1 .. 0:
 *         w   = P_{t+1} c_t + p_{t+1}
 *         Guu = R_t + B'P B,  Gux = S_t + B'P A,  Gxx = Q_t + A'P A
 *         gu  = r_t + B'w,    gx  = q_t + A'w
 *         K_t = -Guu^{-1} Gux,  k_t = -Guu^{-1} gu      (Cholesky of Guu)
 *         P_t = Gxx + Gux'K_t (symmetrised),  p_t = gx + Gux'k_t
 *         s_t = s_{t+1} + p_{t+1}'c_t + 1/2 c_t'P_{t+1}c_t + 1/2 gu'k_t
 *     x_0 = x0, u_t = K_t x_t + k_t, x_{t+1} = A_t x_t + B_t u_t + c_t
 *     lambda_t = -(P_t x_t + p_t)   (sign convention of Eq. 3: Q_T x_T + q_T + lambda_T = 0)
 * Q and R are read symmetrised, 1/2 (M + M').
 *
 * Layout: row-major, stage-major, float64:
 *   A[T][n][n] B[T][n][m] c[T][n] Q[T+1][n][n] R[T][m][m] S[T][m][n] (NULL = 0)
 *   q[T+1][n] r[T][m] x0[n]
 *   outputs (any may be NULL): K[T][m][n] k[T][m] P[T+1][n][n] p[T+1][n]
 *   s[T+1] x[T+1][n] u[T][m] lam[T+1][n] cost[1]
 * Returns 0 on success, 1 if some R_t + B'P B is not positive definite,
 * 2 on bad arguments, 3 on allocation failure.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, ld) ((size_t)(i) * (size_t)(ld) + (size_t)(j))

/* In-place lower Cholesky of the d x d matrix G (row-major); upper part untouched.
 * Returns 0 on success, 1 when a pivot is not positive. */
static int chol_lower(int d, double *G) {
  for (int j = 0; j < d; ++j) {
    double s = G[IDX(j, j, d)];
    for (int k = 0; k < j; ++k) s -= G[IDX(j, k, d)] * G[IDX(j, k, d)];
    if (!(s > 0.0)) return 1;
    double l = sqrt(s);
    G[IDX(j, j, d)] = l;
    for (int i = j + 1; i < d; ++i) {
      double t = G[IDX(i, j, d)];
      for (int k = 0; k < j; ++k) t -= G[IDX(i, k, d)] * G[IDX(j, k, d)];
      G[IDX(i, j, d)] = t / l;
    }
  }
  return 0;
}

/* Solve (L L') X = Y in place for the d x nc right-hand side Y (row-major). */
static void chol_solve(int d, const double *L, int nc, double *Y) {
  for (int col = 0; col < nc; ++col) {
    for (int i = 0; i < d; ++i) { /* L z = y */
      double t = Y[IDX(i, col, nc)];
      for (int k = 0; k < i; ++k) t -= L[IDX(i, k, d)] * Y[IDX(k, col, nc)];
      Y[IDX(i, col, nc)] = t / L[IDX(i, i, d)];
    }
    for (int i = d - 1; i >= 0; --i) { /* L' x = z */
      double t = Y[IDX(i, col, nc)];
      for (int k = i + 1; k < d; ++k) t -= L[IDX(k, i, d)] * Y[IDX(k, col, nc)];
      Y[IDX(i, col, nc)] = t / L[IDX(i, i, d)];
    }
  }
}

int oracle_riccati(int n, int m, int T, const double *A, const double *B, const double *c,
                   const double *Q, const double *R, const double *S, const double *q,
                   const double *r, const double *x0, double *K_out, double *k_out,
                   double *P_out, double *p_out, double *s_out, double *x_out, double *u_out,
                   double *lam_out, double *cost_out) {
  if (n < 1 || m < 1 || T < 1 || !A || !B || !c || !Q || !R || !q || !r || !x0) return 2;
  const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm = (size_t)m * m;
  /* the recursion keeps every P_t, p_t, K_t, k_t (needed for the forward pass) */
  double *P = (double *)malloc(sizeof(double) * nn * (T + 1));
  double *p = (double *)malloc(sizeof(double) * n * (T + 1));
  double *s = (double *)malloc(sizeof(double) * (T + 1));
  double *K = (double *)malloc(sizeof(double) * nm * T);
  double *k = (double *)malloc(sizeof(double) * m * T);
  double *PA = (double *)malloc(sizeof(double) * nn);
  double *PB = (double *)malloc(sizeof(double) * nm);
  double *w = (double *)malloc(sizeof(double) * n);
  double *Guu = (double *)malloc(sizeof(double) * mm);
  double *Gux = (double *)malloc(sizeof(double) * nm);
  double *Gxx = (double *)malloc(sizeof(double) * nn);
  double *gu = (double *)malloc(sizeof(double) * m);
  double *gx = (double *)malloc(sizeof(double) * n);
  double *rhs = (double *)malloc(sizeof(double) * m * (n + 1));
  double *x = (double *)malloc(sizeof(double) * n * (T + 1));
  double *u = (double *)malloc(sizeof(double) * m * T);
  int status = 0;
  if (!P || !p || !s || !K || !k || !PA || !PB || !w || !Guu || !Gux || !Gxx || !gu || !gx ||
      !rhs || !x || !u) {
    status = 3;
    goto done;
  }

  /* terminal value: P_T = sym(Q_T), p_T = q_T, s_T = 0 */
  {
    const double *QT = Q + nn * T;
    double *PT = P + nn * T;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) PT[IDX(i, j, n)] = 0.5 * (QT[IDX(i, j, n)] + QT[IDX(j, i, n)]);
    for (int i = 0; i < n; ++i) p[(size_t)n * T + i] = q[(size_t)n * T + i];
    s[T] = 0.0;
  }

  for (int t = T - 1; t >= 0; --t) {
    const double *At = A + nn * t, *Bt = B + nm * t, *ct = c + (size_t)n * t;
    const double *Qt = Q + nn * t, *Rt = R + mm * t, *St = S ? S + nm * t : NULL;
    const double *qt = q + (size_t)n * t, *rt = r + (size_t)m * t;
    const double *Pn = P + nn * (t + 1), *pn = p + (size_t)n * (t + 1);
    /* w = P_{t+1} c_t + p_{t+1} */
    for (int i = 0; i < n; ++i) {
      double a = pn[i];
      for (int j = 0; j < n; ++j) a += Pn[IDX(i, j, n)] * ct[j];
      w[i] = a;
    }
    /* PA = P A, PB = P B */
    for (int i = 0; i < n; ++i) {
      for (int j = 0; j < n; ++j) {
        double a = 0.0;
        for (int l = 0; l < n; ++l) a += Pn[IDX(i, l, n)] * At[IDX(l, j, n)];
        PA[IDX(i, j, n)] = a;
      }
      for (int j = 0; j < m; ++j) {
        double a = 0.0;
        for (int l = 0; l < n; ++l) a += Pn[IDX(i, l, n)] * Bt[IDX(l, j, m)];
        PB[IDX(i, j, m)] = a;
      }
    }
    /* Guu = sym(R) + B'PB, Gux = S + B'PA, Gxx = sym(Q) + A'PA, gu = r + B'w, gx = q + A'w */
    for (int i = 0; i < m; ++i) {
      for (int j = 0; j < m; ++j) {
        double a = 0.5 * (Rt[IDX(i, j, m)] + Rt[IDX(j, i, m)]);
        for (int l = 0; l < n; ++l) a += Bt[IDX(l, i, m)] * PB[IDX(l, j, m)];
        Guu[IDX(i, j, m)] = a;
      }
      for (int j = 0; j < n; ++j) {
        double a = St ? St[IDX(i, j, n)] : 0.0;
        for (int l = 0; l < n; ++l) a += Bt[IDX(l, i, m)] * PA[IDX(l, j, n)];
        Gux[IDX(i, j, n)] = a;
      }
      double a = rt[i];
      for (int l = 0; l < n; ++l) a += Bt[IDX(l, i, m)] * w[l];
      gu[i] = a;
    }
    for (int i = 0; i < n; ++i) {
      for (int j = 0; j < n; ++j) {
        double a = 0.5 * (Qt[IDX(i, j, n)] + Qt[IDX(j, i, n)]);
        for (int l = 0; l < n; ++l) a += At[IDX(l, i, n)] * PA[IDX(l, j, n)];
        Gxx[IDX(i, j, n)] = a;
      }
      double a = qt[i];
      for (int l = 0; l < n; ++l) a += At[IDX(l, i, n)] * w[l];
      gx[i] = a;
    }
    /* the R + B'PB block must be positive definite (strict convexity, Section II) */
    if (chol_lower(m, Guu)) {
      status = 1;
      goto done;
    }
    /* [K_t | k_t] = -Guu^{-1} [Gux | gu] */
    for (int i = 0; i < m; ++i) {
      for (int j = 0; j < n; ++j) rhs[IDX(i, j, n + 1)] = Gux[IDX(i, j, n)];
      rhs[IDX(i, n, n + 1)] = gu[i];
    }
    chol_solve(m, Guu, n + 1, rhs);
    double *Kt = K + nm * t, *kt = k + (size_t)m * t;
    for (int i = 0; i < m; ++i) {
      for (int j = 0; j < n; ++j) Kt[IDX(i, j, n)] = -rhs[IDX(i, j, n + 1)];
      kt[i] = -rhs[IDX(i, n, n + 1)];
    }
    /* P_t = sym(Gxx + Gux'K_t), p_t = gx + Gux'k_t */
    double *Pt = P + nn * t, *pt = p + (size_t)n * t;
    for (int i = 0; i < n; ++i) {
      for (int j = 0; j < n; ++j) {
        double a = Gxx[IDX(i, j, n)];
        for (int l = 0; l < m; ++l) a += Gux[IDX(l, i, n)] * Kt[IDX(l, j, n)];
        Pt[IDX(i, j, n)] = a;
      }
      double a = gx[i];
      for (int l = 0; l < m; ++l) a += Gux[IDX(l, i, n)] * kt[l];
      pt[i] = a;
    }
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) {
        double a = 0.5 * (Pt[IDX(i, j, n)] + Pt[IDX(j, i, n)]);
        Pt[IDX(i, j, n)] = a;
        Pt[IDX(j, i, n)] = a;
      }
    /* s_t = s_{t+1} + p_{t+1}'c + 1/2 c'P_{t+1}c + 1/2 gu'k */
    {
      double a = s[t + 1];
      for (int i = 0; i < n; ++i) {
        double pc = 0.0;
        for (int j = 0; j < n; ++j) pc += Pn[IDX(i, j, n)] * ct[j];
        a += pn[i] * ct[i] + 0.5 * ct[i] * pc;
      }
      for (int i = 0; i < m; ++i) a += 0.5 * gu[i] * kt[i];
      s[t] = a;
    }
  }

  /* forward pass and the cost along the trajectory */
  {
    double cost = 0.0;
    for (int i = 0; i < n; ++i) x[i] = x0[i];
    for (int t = 0; t < T; ++t) {
      const double *At = A + nn * t, *Bt = B + nm * t, *ct = c + (size_t)n * t;
      const double *Qt = Q + nn * t, *Rt = R + mm * t, *St = S ? S + nm * t : NULL;
      const double *qt = q + (size_t)n * t, *rt = r + (size_t)m * t;
      const double *Kt = K + nm * t, *kt = k + (size_t)m * t;
      const double *xt = x + (size_t)n * t;
      double *ut = u + (size_t)m * t, *xn = x + (size_t)n * (t + 1);
      for (int i = 0; i < m; ++i) {
        double a = kt[i];
        for (int j = 0; j < n; ++j) a += Kt[IDX(i, j, n)] * xt[j];
        ut[i] = a;
      }
      for (int i = 0; i < n; ++i) {
        double a = ct[i];
        for (int j = 0; j < n; ++j) a += At[IDX(i, j, n)] * xt[j];
        for (int j = 0; j < m; ++j) a += Bt[IDX(i, j, m)] * ut[j];
        xn[i] = a;
      }
      /* stage cost 1/2 x'Qx + u'Sx + 1/2 u'Ru + q'x + r'u */
      for (int i = 0; i < n; ++i) {
        double qx = 0.0;
        for (int j = 0; j < n; ++j) qx += Qt[IDX(i, j, n)] * xt[j];
        cost += 0.5 * xt[i] * qx + qt[i] * xt[i];
      }
      for (int i = 0; i < m; ++i) {
        double ru = 0.0, sx = 0.0;
        for (int j = 0; j < m; ++j) ru += Rt[IDX(i, j, m)] * ut[j];
        if (St)
          for (int j = 0; j < n; ++j) sx += St[IDX(i, j, n)] * xt[j];
        cost += 0.5 * ut[i] * ru + ut[i] * sx + rt[i] * ut[i];
      }
    }
    {
      const double *QT = Q + nn * T, *qT = q + (size_t)n * T, *xT = x + (size_t)n * T;
      for (int i = 0; i < n; ++i) {
        double qx = 0.0;
        for (int j = 0; j < n; ++j) qx += QT[IDX(i, j, n)] * xT[j];
        cost += 0.5 * xT[i] * qx + qT[i] * xT[i];
      }
    }
    if (cost_out) *cost_out = cost;
  }

  if (lam_out) {
    for (int t = 0; t <= T; ++t) {
      const double *Pt = P + nn * t, *pt = p + (size_t)n * t, *xt = x + (size_t)n * t;
      for (int i = 0; i < n; ++i) {
        double a = pt[i];
        for (int j = 0; j < n; ++j) a += Pt[IDX(i, j, n)] * xt[j];
        lam_out[(size_t)n * t + i] = -a;
      }
    }
  }
  if (K_out) memcpy(K_out, K, sizeof(double) * nm * T);
  if (k_out) memcpy(k_out, k, sizeof(double) * m * T);
  if (P_out) memcpy(P_out, P, sizeof(double) * nn * (T + 1));
  if (p_out) memcpy(p_out, p, sizeof(double) * n * (T + 1));
  if (s_out) memcpy(s_out, s, sizeof(double) * (T + 1));
  if (x_out) memcpy(x_out, x, sizeof(double) * n * (T + 1));
  if (u_out) memcpy(u_out, u, sizeof(double) * m * T);

done:
  free(P); free(p); free(s); free(K); free(k); free(PA); free(PB); free(w); free(Guu);
  free(Gux); free(Gxx); free(gu); free(gx); free(rhs); free(x); free(u);
  return status;
}
