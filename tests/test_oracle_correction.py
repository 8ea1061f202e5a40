"""The reading behind the refinement corrections of the mixed FP32 mode, checked
on the CPU with the oracle alone.

With the matrices fixed, the serial Riccati recursion (Section III-A) is affine
in the vector data (q, r, c, x0). A correction therefore needs only the solve's
K_t, P_t and M_uu^-1: over a segment [b, e), p_b = Psi'p_e + eps and
x_e = Psi x_b + delta with Psi the product of the closed-loop matrices
A_t + B_t K_t, eps (delta) the segment's own pass from p_e = 0 (x_b = 0). Written
out here step by step in numpy, with the K_t, P_t of the oracle's solve, it must
reproduce the oracle's solution of the problem with new vector data."""
import numpy as np
import pytest

import oracle
import workloads


def _correction(prob, ric, new, K):
    A, B, R = prob["A"], prob["B"], prob["R"]
    T = B.shape[0]
    n = A.shape[1]
    Kt, P = ric["K"], ric["P"]
    Rs = 0.5 * (R + np.swapaxes(R, 1, 2))
    Minv = np.stack([np.linalg.inv(Rs[t] + B[t].T @ P[t + 1] @ B[t]) for t in range(T)])
    q, r, c, x0 = new["q"], new["r"], new["c"], new["x0"]
    b = [(j * T) // K for j in range(K + 1)]
    Psi = []
    for j in range(K):
        M = np.eye(n)
        for t in range(b[j], b[j + 1]):
            M = (A[t] + B[t] @ Kt[t]) @ M
        Psi.append(M)
    k = np.zeros((T, B.shape[2]))
    p = np.zeros((T + 1, n))

    def back(j, pe, store):
        pv = pe.copy()
        for t in range(b[j + 1] - 1, b[j] - 1, -1):
            s = P[t + 1] @ c[t] + pv
            gu = r[t] + B[t].T @ s
            gx = q[t] + A[t].T @ s
            if store:
                k[t] = -Minv[t] @ gu
            pv = gx + Kt[t].T @ gu
            if store:
                p[t] = pv
        return pv

    eps = [back(j, np.zeros(n), False) for j in range(K)]
    pb = [None] * (K + 1)
    pb[K] = q[T].copy()
    for j in range(K - 1, -1, -1):
        pb[j] = Psi[j].T @ pb[j + 1] + eps[j]
    p[T] = q[T]
    for j in range(K):
        back(j, pb[j + 1], True)
    out = {"x": np.zeros((T + 1, n)), "u": np.zeros_like(k), "lam": np.zeros((T + 1, n))}

    def fwd(j, xs, store):
        x = xs.copy()
        for t in range(b[j], b[j + 1]):
            u = Kt[t] @ x + k[t]
            if store:
                out["x"][t], out["u"][t], out["lam"][t] = x, u, -(P[t] @ x + p[t])
            x = A[t] @ x + B[t] @ u + c[t]
        return x

    delta = [fwd(j, np.zeros(n), False) for j in range(K)]
    xb = [x0.copy()]
    for j in range(K):
        xb.append(Psi[j] @ xb[j] + delta[j])
    for j in range(K):
        fwd(j, xb[j], True)
    out["x"][T] = xb[K]
    out["lam"][T] = -(P[T] @ xb[K] + p[T])
    out["k"] = k
    return out


@pytest.mark.parametrize("n,m,T,K,cross", [(8, 3, 40, 5, True), (6, 2, 33, 1, False), (12, 4, 64, 8, True)])
def test_vector_only_correction_matches_new_solve(n, m, T, K, cross):
    prob = workloads.make_problem(n, m, T, seed=60 + n + K, cross=cross)
    ric = oracle.riccati(prob)
    rng = np.random.default_rng(n + T)
    new = dict(prob)
    for key in ("q", "r", "c", "x0"):
        new[key] = rng.standard_normal(prob[key].shape)
    want = oracle.riccati(new)
    got = _correction(prob, ric, new, K)
    for key in ("x", "u", "lam", "k"):
        assert oracle.rel_err(got[key], want[key]) < 1e-12, (key, oracle.rel_err(got[key], want[key]))
