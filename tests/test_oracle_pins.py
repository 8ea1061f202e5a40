"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
brute-force KKT solves, closed forms, a library Riccati solver, invariants.

Each pin targets a class of plausible mistakes:
  * dense KKT (random data, S != 0, c != 0, n != m): dropped c, S transposed,
    wrong sign of k, wrong Q_T handling, lambda sign (Eq. 3);
  * scalar closed form in exact rational arithmetic: every term of the one-step
    problem, including S, r, c and q_T;
  * DARE (scipy): the quadratic recursion with S != 0 over a long horizon;
  * cost identity and P_t symmetric PSD: the constant term s_t and symmetrisation.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

import oracle
import workloads

SHAPES = [(1, 1, 1), (2, 1, 3), (3, 2, 5), (4, 3, 8), (4, 1, 6), (3, 4, 4)]


@pytest.mark.parametrize("n,m,T", SHAPES)
@pytest.mark.parametrize("cross", [False, True])
@pytest.mark.parametrize("seed", [1, 2])
def test_riccati_matches_dense_kkt(n, m, T, cross, seed):
    prob = workloads.make_problem(n, m, T, seed=seed, cross=cross)
    ric = oracle.riccati(prob)
    kkt = oracle.dense_kkt(prob)
    assert oracle.rel_err(ric["x"], kkt["x"]) < 1e-10
    assert oracle.rel_err(ric["u"], kkt["u"]) < 1e-10
    assert oracle.rel_err(ric["lam"], kkt["lam"]) < 1e-10
    assert abs(ric["cost"] - kkt["cost"]) <= 1e-10 * max(1.0, abs(kkt["cost"]))


@pytest.mark.parametrize("n,m,T", [(3, 2, 6), (5, 2, 20), (6, 3, 40)])
def test_cost_identity_and_value_function(n, m, T):
    """J* = 1/2 x0'P_0 x0 + p_0'x0 + s_0 = objective along (x, u)."""
    prob = workloads.make_problem(n, m, T, seed=11, cross=True)
    ric = oracle.riccati(prob)
    x0 = prob["x0"]
    J_value = 0.5 * x0 @ ric["P"][0] @ x0 + ric["p"][0] @ x0 + ric["s"][0]
    J_path = oracle.stage_costs(prob, ric["x"], ric["u"])
    assert abs(J_value - J_path) <= 1e-10 * max(1.0, abs(J_path))
    assert abs(ric["cost"] - J_path) <= 1e-10 * max(1.0, abs(J_path))


@pytest.mark.parametrize("seed", [3, 4])
def test_P_symmetric_psd(seed):
    prob = workloads.make_problem(8, 3, 50, seed=seed)
    P = oracle.riccati(prob)["P"]
    assert np.abs(P - np.swapaxes(P, 1, 2)).max() == 0.0
    for Pt in P:
        ev = np.linalg.eigvalsh(Pt)
        assert ev.min() >= -1e-12 * np.abs(ev).max()


@pytest.mark.parametrize("n,m", [(4, 2), (6, 3), (3, 1)])
def test_dare_limit(n, m):
    """Time-invariant data over a long horizon: P_0 converges to the stabilising
    solution of the discrete algebraic Riccati equation (scipy), with the cross
    weight u'S x entering scipy's convention as s = S'."""
    T = 2000
    prob = workloads.time_invariant(n, m, T, seed=21 + n, cross=True)
    A, B, Q, R, S = prob["A"][0], prob["B"][0], prob["Q"][0], prob["R"][0], prob["S"][0]
    X = scipy.linalg.solve_discrete_are(A, B, Q, R, s=S.T)
    P0 = oracle.riccati(prob)["P"][0]
    assert oracle.rel_err(P0, X) < 1e-9


def _scalar_case():
    # n = m = 1, T = 1, every datum nonzero
    return dict(a=Fraction(2), b=Fraction(1), gam=Fraction(1, 2), Q0=Fraction(3), rho=Fraction(2),
                sig=Fraction(1, 2), q0=Fraction(1), r0=Fraction(-1), QT=Fraction(4), qT=Fraction(2),
                xi=Fraction(1))


def test_scalar_closed_form():
    """One-step scalar problem solved by hand:
       min_u 1/2 Q0 xi^2 + sig u xi + 1/2 rho u^2 + q0 xi + r0 u
             + 1/2 QT x1^2 + qT x1,  x1 = a xi + b u + gam
       => u* = -(sig xi + r0 + b (QT (a xi + gam) + qT)) / (rho + QT b^2),
          lambda_1 = -(QT x1 + qT),
          lambda_0 = a lambda_1 - Q0 xi - sig u* - q0   (Eq. 3)."""
    s = _scalar_case()
    u = -(s["sig"] * s["xi"] + s["r0"] + s["b"] * (s["QT"] * (s["a"] * s["xi"] + s["gam"]) + s["qT"])) / (
        s["rho"] + s["QT"] * s["b"] ** 2)
    x1 = s["a"] * s["xi"] + s["b"] * u + s["gam"]
    lam1 = -(s["QT"] * x1 + s["qT"])
    lam0 = s["a"] * lam1 - s["Q0"] * s["xi"] - s["sig"] * u - s["q0"]
    cost = (s["Q0"] * s["xi"] ** 2 / 2 + s["sig"] * u * s["xi"] + s["rho"] * u ** 2 / 2 + s["q0"] * s["xi"]
            + s["r0"] * u + s["QT"] * x1 ** 2 / 2 + s["qT"] * x1)
    f = lambda v: np.array([[float(v)]])
    prob = dict(A=f(s["a"]).reshape(1, 1, 1), B=f(s["b"]).reshape(1, 1, 1), c=f(s["gam"]).reshape(1, 1),
                Q=np.array([[[float(s["Q0"])]], [[float(s["QT"])]]]), R=f(s["rho"]).reshape(1, 1, 1),
                S=f(s["sig"]).reshape(1, 1, 1), q=np.array([[float(s["q0"])], [float(s["qT"])]]),
                r=f(s["r0"]).reshape(1, 1), x0=np.array([float(s["xi"])]))
    ric = oracle.riccati(prob)
    assert abs(ric["u"][0, 0] - float(u)) < 1e-14
    assert abs(ric["x"][1, 0] - float(x1)) < 1e-14
    assert abs(ric["lam"][1, 0] - float(lam1)) < 1e-13
    assert abs(ric["lam"][0, 0] - float(lam0)) < 1e-13
    assert abs(ric["cost"] - float(cost)) < 1e-13
    # feedback gain of the same problem: K = -(sig + b QT a) / (rho + QT b^2)
    K = -(s["sig"] + s["b"] * s["QT"] * s["a"]) / (s["rho"] + s["QT"] * s["b"] ** 2)
    assert abs(ric["K"][0, 0, 0] - float(K)) < 1e-14


def test_zero_data_gives_zero_solution():
    prob = workloads.make_problem(5, 2, 7, seed=5)
    for k in ("c", "q", "r", "x0"):
        prob[k] = np.zeros_like(prob[k])
    ric = oracle.riccati(prob)
    for k in ("x", "u", "lam", "k", "p"):
        assert np.abs(ric[k]).max() == 0.0
    assert ric["cost"] == 0.0


def test_not_pd_is_reported():
    prob = workloads.make_problem(3, 2, 4, seed=6)
    prob["R"][2] = -np.eye(2) * 100.0
    with pytest.raises(oracle.OracleError):
        oracle.riccati(prob)


def test_kkt_residual_of_exact_solution_is_tiny():
    prob = workloads.make_problem(6, 2, 30, seed=8, cross=True)
    ric = oracle.riccati(prob)
    res = oracle.kkt_residual(prob, ric["x"], ric["u"], ric["lam"])
    assert res["eta"] < 1e-14
    # a perturbed trajectory is visibly not a KKT point
    x = ric["x"].copy()
    x[10, 3] += 1e-6
    res2 = oracle.kkt_residual(prob, x, ric["u"], ric["lam"])
    assert res2["rnorm"] > 1e-7


@pytest.mark.parametrize("cross", [False, True])
def test_kkt_residual_matches_dense_system(cross):
    """The block formulas of the residual, |KKT| row sums and norms against the
    dense KKT matrix of Eq. 3 (assembled entry by entry) at a point that is not
    the solution: r = KKT z - b, eta = |r| / (max_i sum_j |KKT_ij| |z| + |b|)."""
    n, m, T = 5, 2, 7
    prob = workloads.make_problem(n, m, T, seed=31, cross=cross)
    rng = np.random.default_rng(5)
    for k in ("Q", "R"):  # nonsymmetric input: both sides read (M + M')/2
        d = prob[k].shape[-1]
        prob[k] = prob[k] + 0.3 * rng.standard_normal((prob[k].shape[0], d, d))
        prob[k] = 0.5 * (prob[k] + np.swapaxes(prob[k], -1, -2)) + 0.2 * (
            prob[k] - np.swapaxes(prob[k], -1, -2))
    x = rng.standard_normal((T + 1, n))
    u = rng.standard_normal((T, m))
    lam = rng.standard_normal((T + 1, n))
    got = oracle.kkt_residual(prob, x, u, lam)
    dk = oracle.dense_kkt(prob)
    K, b = dk["kkt"], dk["rhs"]
    z = np.concatenate([x.ravel(), u.ravel(), lam.ravel()])
    r = K @ z - b
    rnorm = np.abs(r).max()
    knorm = np.abs(K).sum(axis=1).max()
    eta = rnorm / (knorm * np.abs(z).max() + np.abs(b).max())
    assert got["rnorm"] == pytest.approx(rnorm, rel=1e-13)
    assert got["knorm"] == pytest.approx(knorm, rel=1e-13)
    assert got["eta"] == pytest.approx(eta, rel=1e-13)
    assert got["rel"] == pytest.approx(rnorm / np.abs(b).max(), rel=1e-13)


def test_stage_costs_matches_dense_quadratic():
    """The objective of Eq. 1-2 summed stage by stage against 1/2 w'Hw + g'w with the
    dense Hessian of the KKT system (Q, R read symmetrised, S coupling) at a random w."""
    n, m, T = 4, 3, 6
    prob = workloads.make_problem(n, m, T, seed=41, cross=True)
    rng = np.random.default_rng(9)
    x = rng.standard_normal((T + 1, n))
    u = rng.standard_normal((T, m))
    dk = oracle.dense_kkt(prob)
    nw = (T + 1) * n + T * m
    H = dk["kkt"][:nw, :nw]
    g = -dk["rhs"][:nw]
    w = np.concatenate([x.ravel(), u.ravel()])
    assert oracle.stage_costs(prob, x, u) == pytest.approx(0.5 * w @ H @ w + g @ w, rel=1e-13)
