"""The multipliers of the segment problems from the least-squares system of
Section II-B ("Lagrange Multipliers") through lqr_ls_multipliers, against the
oracle's dense normal-equation solve (ls_multipliers) on the same trajectory,
and at the optimum against the multipliers of Eq. 3 that the solve returns.

Tolerance 1e-9 (normwise, relative): the block Cholesky of the normal
equations runs in FP64 and its error grows with cond(A A') = cond(A')^2; the
stationarity matrices of these workloads are well conditioned (their blocks
are I, A_t', B_t' with rho(A_t) <= 1.05), so FP64 rounding leaves 1e-12 or
less on these sizes."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06360_gb300 import Solver, build
    build.build()
    s = Solver(0)
    yield s
    s.close()


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", torch.float64)


def _bounds(T, K):
    return [j * T // K for j in range(K + 1)]


def _run(solver, prob, x, u, K):
    dprob = {k: to_dev(v) for k, v in prob.items()}
    out = solver.ls_multipliers(dprob, to_dev(x), to_dev(u), K)
    rep = solver.report()
    assert rep["status"] == 0, rep
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("n,m,T,K,cross", [(3, 2, 12, 3, False), (4, 1, 16, 4, True), (2, 3, 9, 2, True),
                                           (5, 2, 1, 1, False), (7, 3, 61, 7, True), (12, 4, 128, 8, True),
                                           (9, 9, 50, 6, False), (16, 4, 40, 1, True)])
@pytest.mark.parametrize("perturb", [False, True])
def test_ls_multipliers_match_oracle(solver, n, m, T, K, cross, perturb):
    prob = workloads.make_problem(n, m, T, seed=800 + n + T + K, cross=cross, rho_max=1.05)
    ref = oracle.riccati(prob)
    x, u = ref["x"], ref["u"]
    if perturb:  # an inconsistent system: the least-squares multipliers
        rng = np.random.default_rng(n + T)
        x = x + 0.05 * rng.standard_normal(x.shape)
        u = u + 0.05 * rng.standard_normal(u.shape)
    b = _bounds(T, K)
    want = oracle.ls_multipliers(prob, x, u, b)
    got = _run(solver, prob, x, u, K)
    for key in ("lam", "lam_end", "mu"):
        if want[key].size:
            assert oracle.rel_err(got[key], want[key]) < 1e-9, (key, oracle.rel_err(got[key], want[key]))
    if not perturb:
        assert oracle.rel_err(got["lam"], ref["lam"]) < 1e-9
        for j in range(K - 1):
            assert np.abs(got["lam_end"][j] - ref["lam"][b[j + 1]]).max() < 1e-9 * np.abs(ref["lam"]).max()
            assert np.abs(got["mu"][j] + got["lam_end"][j]).max() < 1e-9 * np.abs(ref["lam"]).max()


def test_ls_multipliers_long_horizon(solver):
    """n=64, m=32, T=4096, K=152 (the long-horizon workload): at the solve's own
    optimum, the least-squares multipliers against the multipliers of Eq. 3 the
    solve returns and the serial oracle's; three sampled segments (first, an
    interior one, last) against the oracle's dense normal-equation solve at a
    perturbed trajectory."""
    prob = workloads.config1()
    T, n, m = prob["B"].shape
    K = 152
    dprob = {k: to_dev(v) for k, v in prob.items()}
    sol = solver.solve(dprob, num_segments=K)
    assert solver.report()["status"] == 0
    got = solver.ls_multipliers(dprob, sol["x"], sol["u"], K)
    assert solver.report()["status"] == 0
    lam = got["lam"].cpu().numpy()
    ref = oracle.riccati(prob)
    assert oracle.rel_err(lam, sol["lam"].cpu().numpy()) < 1e-9
    assert oracle.rel_err(lam, ref["lam"]) < 1e-9
    b = _bounds(T, K)
    lam_end = got["lam_end"].cpu().numpy()
    mu = got["mu"].cpu().numpy()
    scale = np.abs(ref["lam"]).max()
    assert np.abs(lam_end - ref["lam"][b[1:K]]).max() < 1e-9 * scale
    assert np.abs(mu + lam_end).max() < 1e-9 * scale
    rng = np.random.default_rng(3)
    x = ref["x"] + 0.01 * rng.standard_normal(ref["x"].shape)
    u = ref["u"] + 0.01 * rng.standard_normal(ref["u"].shape)
    got = _run(solver, prob, x, u, K)
    only = (0, 77, K - 1)
    want = oracle.ls_multipliers(prob, x, u, b, only=only)
    for j in only:
        sl = slice(b[j], b[j + 1] + (1 if j == K - 1 else 0))
        assert oracle.rel_err(got["lam"][sl], want["lam"][sl]) < 1e-9, j
        if j < K - 1:
            assert oracle.rel_err(got["lam_end"][j], want["lam_end"][j]) < 1e-9, j
            assert oracle.rel_err(got["mu"][j], want["mu"][j]) < 1e-9, j
