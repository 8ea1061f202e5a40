"""The paper's own feedback policies (Section III-A, the double-integrator
comparison) through lqr_segment_policies, against the serial Riccati policies
of the oracle.

Unsmoothed: per segment u_t = Kx_t x_t + Kz_t z_{j+1} + k1_t with the segment's
end link point. Smoothed: each segment but the last re-swept from the next
segment's cost to go with its own end pinned at its link point. The paper
states that both reproduce the serial optimal trajectory on the undisturbed
system while their feedback gains differ from the serial ones; that is what
is checked, on the paper's double-integrator problem (its alpha, alpha_T,
beta, x0 and J = 3; T and dt are this test's choice). The disturbed-system
costs (the paper's 2.896e3 / 2.203e3) are printed, parity unpinned: the paper
gives neither dt nor T nor which component x_t(1) is."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06360_gb300 import Solver, build
    build.build()
    s = Solver(0)
    yield s
    s.close()


def rollout(prob, policy, disturb=False):
    """Closed-loop trajectory and its cost under policy(t, x) (host, FP64)."""
    A, B, c = prob["A"], prob["B"], prob["c"]
    T = B.shape[0]
    x = prob["x0"].copy()
    xs, us = [x], []
    for t in range(T):
        u = policy(t, x)
        xn = A[t] @ x + B[t] @ u + c[t]
        if disturb:  # Eq. 18: second component, x(1) read as the velocity (0-based index 1)
            xn = xn + np.array([0.0, x[1] / (x[1] ** 2 + 1e-4)])
        xs.append(xn)
        us.append(u)
        x = xn
    xs, us = np.array(xs), np.array(us)
    return xs, us, oracle.stage_costs(prob, xs, us)


def bounds(T, K):
    return [(j * T) // K for j in range(K + 1)]


@pytest.fixture(scope="module")
def double_integrator():
    with open(os.path.join(GOLDEN, "double_integrator.json")) as f:
        cfg = json.load(f)
    prob = workloads.double_integrator(T=cfg["T_chosen"], dt=cfg["dt_chosen"], alpha=cfg["alpha"],
                                       alpha_T=cfg["alpha_T"], beta=cfg["beta"])
    return cfg, prob


def test_segment_policies_double_integrator(solver, double_integrator):
    cfg, prob = double_integrator
    J, T = cfg["J"], prob["B"].shape[0]
    ser = oracle.riccati(prob)
    dev = {k: torch.from_numpy(v).cuda() for k, v in prob.items()}
    un = {k: v.cpu().numpy() for k, v in solver.segment_policies(dev, J, smooth=False).items()}
    assert solver.report()["status"] == 0
    sm = {k: v.cpu().numpy() for k, v in solver.segment_policies(dev, J, smooth=True).items()}
    assert solver.report()["status"] == 0
    b = bounds(T, J)
    seg_of = np.searchsorted(b, np.arange(T), side="right") - 1
    # the link points are the serial optimal states at the boundaries
    for j in range(J):
        assert np.abs(un["z"][j] - ser["x"][b[j]]).max() < 1e-9
    pol_ser = lambda t, x: ser["K"][t] @ x + ser["k"][t]
    pol_un = lambda t, x: un["Kx"][t] @ x + un["Kz"][t] @ un["z"][seg_of[t] + 1] + un["k1"][t]
    pol_sm = lambda t, x: sm["Kx"][t] @ x + sm["k1"][t]
    xs_s, us_s, J_s = rollout(prob, pol_ser)
    for pol in (pol_un, pol_sm):
        xs, us, _ = rollout(prob, pol)
        assert oracle.rel_err(xs, ser["x"]) < 1e-9 and oracle.rel_err(us, ser["u"]) < 1e-9
    # gains: the last segment is the serial policy in both; the earlier segments
    # of the unsmoothed policy hold their ends at the link points (different
    # gains); smoothing differs from serial where the next segment's end is
    # pinned (segment j < J - 2) and equals it for j = J - 2
    last = slice(b[J - 1], T)
    assert oracle.rel_err(un["Kx"][last], ser["K"][last]) < 1e-9
    assert oracle.rel_err(sm["Kx"][last], ser["K"][last]) < 1e-9
    early = slice(b[0], b[J - 1])
    d_un = np.abs(un["Kx"][early] - ser["K"][early]).max() / np.abs(ser["K"]).max()
    d_sm0 = np.abs(sm["Kx"][b[0]:b[1]] - ser["K"][b[0]:b[1]]).max() / np.abs(ser["K"]).max()
    assert d_un > 1e-3 and d_sm0 > 1e-3, (d_un, d_sm0)
    assert oracle.rel_err(sm["Kx"][b[J - 2]:b[J - 1]], ser["K"][b[J - 2]:b[J - 1]]) < 1e-9
    assert np.abs(sm["Kz"]).max() == 0.0
    # the disturbed system of Eq. 18: the three policies now give different costs
    _, _, c_s = rollout(prob, pol_ser, disturb=True)
    _, _, c_u = rollout(prob, pol_un, disturb=True)
    _, _, c_m = rollout(prob, pol_sm, disturb=True)
    print("disturbed costs: serial %.4e, parallel %.4e, smoothed %.4e (paper, other dt/T: 2.896e3, 2.203e3)"
          % (c_s, c_u, c_m))
    assert np.isfinite([c_s, c_u, c_m]).all()
    assert abs(c_s - c_u) > 1e-6 * abs(c_s)


@pytest.mark.parametrize("n,m,T,K", [(6, 2, 60, 4), (5, 3, 45, 5)])
def test_segment_policies_reproduce_optimum(solver, n, m, T, K):
    """Random problems with a cross term and affine dynamics: both policy
    families reproduce the optimal trajectory; the last segment's gains are the
    serial ones."""
    prob = workloads.make_problem(n, m, T, seed=2300 + n * K, cross=True)
    ser = oracle.riccati(prob)
    dev = {k: torch.from_numpy(v).cuda() for k, v in prob.items()}
    b = bounds(T, K)
    seg_of = np.searchsorted(b, np.arange(T), side="right") - 1
    for smooth in (False, True):
        pol = {k: v.cpu().numpy() for k, v in solver.segment_policies(dev, K, smooth=smooth).items()}
        assert solver.report()["status"] == 0
        f = lambda t, x: pol["Kx"][t] @ x + pol["Kz"][t] @ pol["z"][seg_of[t] + 1] + pol["k1"][t]
        xs, us, _ = rollout(prob, f)
        assert oracle.rel_err(xs, ser["x"]) < 1e-9, smooth
        assert oracle.rel_err(pol["Kx"][b[K - 1]:], ser["K"][b[K - 1]:]) < 1e-9
