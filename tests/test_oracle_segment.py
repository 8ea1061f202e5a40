"""Pins of the oracle's endpoint-constrained segment summary (Section II-B, Eq. 8-9).

The summary comes from a sparse-KKT solve with parametric right-hand sides. It
is checked against two independent formulations:
  * the serial Riccati recursion: minimising J(x_s, z) + V_{t1}(z) over z must
    give V_{t0} (Bellman's principle on the split of Eq. 5-6);
  * a condensed brute force: states eliminated, the endpoint constraint handled
    by a null-space parametrisation of the controls, J evaluated at random
    (x_s, z) points.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _quad(summ, xs, z):
    return (0.5 * xs @ summ["Vxx"] @ xs + z @ summ["Vzx"] @ xs + 0.5 * z @ summ["Vzz"] @ z
            + summ["vx"] @ xs + summ["vz"] @ z + summ["v0"])


def _condensed_value(prob, t0, t1, xs, z):
    """min over u_{t0..t1-1} of the segment cost with x_{t0}=xs, x_{t1}=z,
    by eliminating the states and parametrising the feasible controls."""
    A, B, c, Q, R, S, q, r = (prob[k] for k in ("A", "B", "c", "Q", "R", "S", "q", "r"))
    T, n, m = B.shape
    L = t1 - t0
    # x_i = Phi_i xs + G_i u + h_i  (u stacked, length L*m)
    Phi = np.eye(n)
    G = np.zeros((n, L * m))
    h = np.zeros(n)
    Hu = np.zeros((L * m, L * m))
    gu = np.zeros(L * m)
    const = 0.0
    for i in range(L):
        t = t0 + i
        x_aff = (Phi @ xs + h, G)  # x_i = x_aff[0] + G u
        E = np.zeros((m, L * m))
        E[:, i * m:(i + 1) * m] = np.eye(m)  # u_i = E u
        xa, Gx = x_aff
        Qs = 0.5 * (Q[t] + Q[t].T)
        Rs = 0.5 * (R[t] + R[t].T)
        # 1/2 x'Qx + u'Sx + 1/2 u'Ru + q'x + r'u with x = xa + Gx u, u_i = E u
        Hu += Gx.T @ Qs @ Gx + E.T @ S[t] @ Gx + Gx.T @ S[t].T @ E + E.T @ Rs @ E
        gu += Gx.T @ (Qs @ xa + q[t]) + E.T @ (S[t] @ xa + r[t])
        const += 0.5 * xa @ Qs @ xa + q[t] @ xa
        Phi = A[t] @ Phi
        G = A[t] @ G + B[t] @ E
        h = A[t] @ h + c[t]
    # endpoint: Phi xs + h + G u = z
    u_p = np.linalg.lstsq(G, z - Phi @ xs - h, rcond=None)[0]
    assert np.abs(G @ u_p - (z - Phi @ xs - h)).max() < 1e-9
    N = scipy.linalg.null_space(G)
    if N.shape[1] == 0:
        u = u_p
    else:
        # min over y of 1/2 (u_p + N y)'Hu(u_p + N y) + gu'(u_p + N y)
        y = np.linalg.solve(N.T @ Hu @ N, -N.T @ (Hu @ u_p + gu))
        u = u_p + N @ y
    return 0.5 * u @ Hu @ u + gu @ u + const


@pytest.mark.parametrize("n,m,L,cross", [(2, 1, 3, False), (3, 1, 5, True), (4, 2, 4, True),
                                         (4, 2, 2, False), (5, 2, 6, True), (3, 3, 1, True),
                                         (5, 3, 4, True)])
def test_summary_vs_condensed_brute_force(n, m, L, cross):
    prob = workloads.make_problem(n, m, L + 3, seed=30 + n + L, cross=cross)
    t0, t1 = 1, 1 + L
    summ = oracle.segment_summary(prob, t0, t1)
    g = np.random.default_rng(0)
    for _ in range(4):
        xs = g.standard_normal(n)
        z = g.standard_normal(n)
        J_ref = _condensed_value(prob, t0, t1, xs, z)
        assert abs(_quad(summ, xs, z) - J_ref) <= 1e-9 * max(1.0, abs(J_ref))
    for k in ("Vxx", "Vzz"):
        assert np.abs(summ[k] - summ[k].T).max() <= 1e-9 * np.abs(summ[k]).max()
    # the two ways of reading the cross block agree (dJ/dx_s vs dJ/dz)
    assert np.abs(summ["Vxz_from_init"] - summ["Vzx"].T).max() <= 1e-9 * np.abs(summ["Vzx"]).max()


@pytest.mark.parametrize("n,m,T,t0,t1", [(4, 2, 12, 3, 8), (6, 2, 20, 0, 9), (5, 5, 8, 2, 3),
                                         (6, 4, 14, 5, 13)])
def test_summary_composes_with_serial_value_function(n, m, T, t0, t1):
    """V_{t0}(x) = min_z J(x, z) + V_{t1}(z):
       P_{t0} = Vxx - Vzx'(Vzz + P_{t1})^{-1} Vzx,
       p_{t0} = vx  - Vzx'(Vzz + P_{t1})^{-1}(vz + p_{t1})."""
    prob = workloads.make_problem(n, m, T, seed=40 + t0, cross=True)
    ric = oracle.riccati(prob)
    summ = oracle.segment_summary(prob, t0, t1)
    D = summ["Vzz"] + ric["P"][t1]
    P0 = summ["Vxx"] - summ["Vzx"].T @ np.linalg.solve(D, summ["Vzx"])
    p0 = summ["vx"] - summ["Vzx"].T @ np.linalg.solve(D, summ["vz"] + ric["p"][t1])
    assert oracle.rel_err(P0, ric["P"][t0]) < 1e-9
    assert oracle.rel_err(p0, ric["p"][t0]) < 1e-9


def test_link_coupling_at_global_optimum():
    """Eq. 10-11: at the optimal link point x_link = x*_tau the multiplier of the
    first sub-problem's end constraint and the second's start multiplier
    cancel, i.e. dJ_1/dz + dJ_2/dx_s = 0 for consecutive segments."""
    n, m, T = 4, 2, 15
    prob = workloads.make_problem(n, m, T, seed=51, cross=True)
    ric = oracle.riccati(prob)
    x = ric["x"]
    b = [0, 5, 10]
    s0 = oracle.segment_summary(prob, b[0], b[1])
    s1 = oracle.segment_summary(prob, b[1], b[2])
    z = x[b[1]]
    g_end = s0["Vzx"] @ x[b[0]] + s0["Vzz"] @ z + s0["vz"]
    g_start = s1["Vxx"] @ z + s1["Vzx"].T @ x[b[2]] + s1["vx"]
    assert np.abs(g_end + g_start).max() <= 1e-9 * np.abs(g_end).max()
    # and -dJ/dx_s at the start of segment 1 is the global multiplier lambda_tau
    assert oracle.rel_err(-g_start, ric["lam"][b[1]]) < 1e-9


def test_double_integrator_split_equals_serial():
    """Section III-A: with J = 3 sub-trajectories the undisturbed optimal
    trajectory of the split method equals the serial Riccati trajectory.
    The split here is carried out with oracle summaries and a dense link solve."""
    with open(os.path.join(GOLDEN, "double_integrator.json")) as f:
        cfg = json.load(f)
    prob = workloads.double_integrator(T=cfg["T_chosen"], dt=cfg["dt_chosen"], alpha=cfg["alpha"],
                                       alpha_T=cfg["alpha_T"], beta=cfg["beta"])
    assert list(prob["x0"]) == cfg["x0"]
    T = prob["B"].shape[0]
    n = 2
    J = cfg["J"]
    bnd = [round(j * T / J) for j in range(J + 1)]
    ric = oracle.riccati(prob)
    summ = [oracle.segment_summary(prob, bnd[j], bnd[j + 1]) for j in range(J - 1)]
    # last segment: serial value function at its start
    P_last, p_last = ric["P"][bnd[J - 1]], ric["p"][bnd[J - 1]]
    # stationarity of sum_j J_j in the link points z_1..z_{J-1}
    N = (J - 1) * n
    M = np.zeros((N, N))
    rhs = np.zeros(N)
    for j in range(1, J):
        sl = slice((j - 1) * n, j * n)
        prev = summ[j - 1]
        M[sl, sl] += prev["Vzz"]
        rhs[sl] -= prev["vz"]
        if j == 1:
            rhs[sl] -= prev["Vzx"] @ prob["x0"]
        else:
            M[sl, slice((j - 2) * n, (j - 1) * n)] += prev["Vzx"]
        if j < J - 1:
            cur = summ[j]
            M[sl, sl] += cur["Vxx"]
            M[sl, slice(j * n, (j + 1) * n)] += cur["Vzx"].T
            rhs[sl] -= cur["vx"]
        else:
            M[sl, sl] += P_last
            rhs[sl] -= p_last
    z = np.linalg.solve(M, rhs).reshape(J - 1, n)
    for j in range(1, J):
        assert np.abs(z[j - 1] - ric["x"][bnd[j]]).max() < 1e-9


# ---------------------------------------------------------------------------
# The dualised segment summary (end cost mu'x_term instead of x_term = z)
# ---------------------------------------------------------------------------

def _condensed_dual_value(prob, t0, t1, xs, mu):
    """min over u_{t0..t1-1} of the segment cost plus mu'x_{t1}, x_{t0} = xs, by
    eliminating the states (no end constraint: one unconstrained solve in u)."""
    A, B, c, Q, R, S, q, r = (prob[k] for k in ("A", "B", "c", "Q", "R", "S", "q", "r"))
    T, n, m = B.shape
    L = t1 - t0
    xa, G = xs.copy(), np.zeros((n, L * m))
    Hu = np.zeros((L * m, L * m))
    gu = np.zeros(L * m)
    const = 0.0
    for i in range(L):
        t = t0 + i
        E = np.zeros((m, L * m))
        E[:, i * m:(i + 1) * m] = np.eye(m)
        Qs = 0.5 * (Q[t] + Q[t].T)
        Rs = 0.5 * (R[t] + R[t].T)
        Hu += G.T @ Qs @ G + E.T @ S[t] @ G + G.T @ S[t].T @ E + E.T @ Rs @ E
        gu += G.T @ (Qs @ xa + q[t]) + E.T @ (S[t] @ xa + r[t])
        const += 0.5 * xa @ Qs @ xa + q[t] @ xa
        xa = A[t] @ xa + c[t]
        G = A[t] @ G + B[t] @ E
    gu = gu + G.T @ mu
    const += mu @ xa
    u = np.linalg.solve(Hu, -gu)
    return 0.5 * u @ Hu @ u + gu @ u + const


def _dual_quad(d, xs, mu):
    return (0.5 * xs @ d["P"] @ xs + mu @ d["Z"] @ xs - 0.5 * mu @ d["W"] @ mu + d["p"] @ xs + d["w"] @ mu)


@pytest.mark.parametrize("n,m,L,cross", [(2, 1, 3, False), (3, 1, 5, True), (4, 2, 4, True),
                                         (4, 2, 1, False), (5, 2, 6, True), (3, 5, 2, True)])
def test_dual_summary_vs_condensed_brute_force(n, m, L, cross):
    """G(x_s, mu) - G(0, 0) from the dense KKT blocks equals the condensed
    minimum at random points (the constant g0 drops out of the difference)."""
    prob = workloads.make_problem(n, m, L + 3, seed=60 + n + L, cross=cross)
    t0, t1 = 1, 1 + L
    d = oracle.segment_dual_summary(prob, t0, t1)
    z0 = np.zeros(n)
    G0 = _condensed_dual_value(prob, t0, t1, z0, z0)
    g = np.random.default_rng(1)
    for _ in range(4):
        xs = g.standard_normal(n)
        mu = g.standard_normal(n)
        ref = _condensed_dual_value(prob, t0, t1, xs, mu) - G0
        assert abs(_dual_quad(d, xs, mu) - ref) <= 1e-9 * max(1.0, abs(ref))
    for k in ("P", "W"):
        assert np.abs(d[k] - d[k].T).max() <= 1e-9 * np.abs(d[k]).max()
    # Z read from dG/dx_s and from dG/dmu agree; W is positive semidefinite
    assert np.abs(d["Zt_from_init"] - d["Z"].T).max() <= 1e-9 * np.abs(d["Z"]).max()
    assert np.linalg.eigvalsh(d["W"]).min() >= -1e-12 * np.abs(d["W"]).max()


@pytest.mark.parametrize("n,m,T,t0,t1", [(4, 2, 12, 3, 8), (5, 2, 30, 0, 6), (6, 3, 24, 4, 8)])
def test_dual_summary_equals_primal_by_legendre(n, m, T, t0, t1):
    """J(x_s, z) = max_mu G(x_s, mu) - mu'z (Eq. 9 from the dual value): with
    W invertible, Vzz = W^-1, Vzx = -W^-1 Z, Vxx = P + Z'W^-1 Z, vz = -W^-1 w,
    vx = p + Z'W^-1 w. The two dense solves share no constraint rows."""
    prob = workloads.make_problem(n, m, T, seed=70 + t0, cross=True)
    d = oracle.segment_dual_summary(prob, t0, t1)
    s = oracle.segment_summary(prob, t0, t1)
    Wi = np.linalg.inv(d["W"])
    assert oracle.rel_err(Wi, s["Vzz"]) < 1e-9
    assert oracle.rel_err(-Wi @ d["Z"], s["Vzx"]) < 1e-9
    assert oracle.rel_err(d["P"] + d["Z"].T @ Wi @ d["Z"], s["Vxx"]) < 1e-9
    assert oracle.rel_err(-Wi @ d["w"], s["vz"]) < 1e-9
    assert oracle.rel_err(d["p"] + d["Z"].T @ Wi @ d["w"], s["vx"]) < 1e-9


@pytest.mark.parametrize("n,m,T,t0,t1", [(4, 2, 12, 3, 8), (6, 2, 20, 0, 9), (5, 5, 8, 2, 3),
                                         (3, 5, 10, 1, 2)])
def test_dual_summary_composes_with_serial_value_function(n, m, T, t0, t1):
    """With the tail's value function V_{t1} = (P1, p1), the end multiplier is
    mu = P1 x_{t1} + p1 and x_{t1} = Z x - W mu + w, so
       P_{t0} = P + Z'P1 (I + W P1)^-1 Z,
       p_{t0} = p + Z'(P1 (I + W P1)^-1 (w - W p1) + p1)
    (the link recursion of the multiplier form), also for one-stage segments
    and m > n, where W is singular or the primal summary does not exist."""
    prob = workloads.make_problem(n, m, T, seed=80 + t0, cross=True)
    ric = oracle.riccati(prob)
    d = oracle.segment_dual_summary(prob, t0, t1)
    P1, p1 = ric["P"][t1], ric["p"][t1]
    M = np.eye(n) + d["W"] @ P1
    P0 = d["P"] + d["Z"].T @ P1 @ np.linalg.solve(M, d["Z"])
    p0 = d["p"] + d["Z"].T @ (P1 @ np.linalg.solve(M, d["w"] - d["W"] @ p1) + p1)
    assert oracle.rel_err(P0, ric["P"][t0]) < 1e-9
    assert oracle.rel_err(p0, ric["p"][t0]) < 1e-9


@pytest.mark.parametrize("n,m,T,t1", [(3, 2, 14, 9), (4, 1, 16, 12), (2, 3, 8, 5), (5, 2, 18, 14)])
def test_global_policy_from_segment_equals_serial(n, m, T, t1):
    """The per-stage reconstruction of the global policy from the end-constrained
    value of the rest of the segment and the global value at its end point
    (the serial recursion's P, p at t1) is Bellman's split: it must return the
    serial recursion's P_t, p_t, K_t, k_t at every stage from which the end
    state is reachable (t1 - t >= ceil(n / m))."""
    prob = workloads.make_problem(n, m, T, seed=40 + n * m + t1, cross=True)
    ref = oracle.riccati(prob)
    reach = -(-n // m)
    scale = {k: np.abs(ref[k][:t1]).max() for k in ("P", "p", "K", "k")}
    for t in range(0, t1 - reach + 1):
        g = oracle.global_policy_from_segment(prob, t, t1, ref["P"][t1], ref["p"][t1])
        for k in ("P", "p", "K", "k"):
            assert np.abs(g[k] - ref[k][t]).max() < 1e-8 * scale[k], (t, k)

