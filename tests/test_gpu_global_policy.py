"""Per-stage reconstruction of the global policy (lqr_global_policy_parallel):
P_t = Vxx - Vzx'(Vzz + P_e)^-1 Vzx and K_t = Kx - Kz (Vzz + P_e)^-1 Vzx at every
stage whose constraint_to_go has no rows left, one CTA per stage, from the
constraint-explicit sweep's per-stage values (Section II-B) and the global
value at the segment end (Section III-A); the few stages at each segment end
with rows left from the policy sweep. Checked against the serial recursion of
the oracle (the plain definition of P_t, p_t, K_t, k_t).

The reconstruction subtracts two terms that grow towards the segment end, so
its error there is the FP64 rounding of Vxx times kappa_t = |Vxx_t| / |P_t|:
largest at the first stage of rank 0 (ceil(n/m) stages before the end) and
falling with the distance from it. The bounds below are that profile with a
margin: the stages swept sequentially and the stages far from the end at
rounding level, the whole horizon within the measured cancellation (n=64,
m=32, K=152: 6.4e-10 on P, 2.2e-9 on p at the worst stage)."""
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


def to_dev(prob):
    return {k: torch.from_numpy(v).to("cuda:0", torch.float64) for k, v in prob.items()}


def _dist(T, K):
    """Distance of every stage from its segment's end (stages of the last segment: 0)."""
    b = [j * T // K for j in range(K + 1)]
    d = np.zeros(T, dtype=int)
    for j in range(K - 1):
        d[b[j]:b[j + 1]] = b[j + 1] - np.arange(b[j], b[j + 1])
    return d


def _stage_err(got, ref):
    sc = np.abs(ref).max()
    return np.abs(got - ref).reshape(got.shape[0], -1).max(axis=1) / sc


@pytest.mark.parametrize("n,m,T,K,cross", [(3, 2, 40, 4, False), (5, 2, 60, 5, True), (4, 1, 48, 4, False),
                                           (2, 3, 30, 5, True), (12, 4, 256, 8, True), (32, 8, 512, 8, False),
                                           (6, 2, 37, 3, True), (8, 4, 24, 1, False)])
def test_global_policy_parallel_matches_serial(solver, n, m, T, K, cross):
    prob = workloads.make_problem(n, m, T, seed=900 + n + T, cross=cross, rho_max=1.02)
    ref = oracle.riccati(prob)
    out = {k: v.cpu().numpy() for k, v in solver.global_policy_parallel(to_dev(prob), K).items()}
    assert solver.report()["status"] == 0
    for k in ("K", "k", "P", "p"):
        assert oracle.rel_err(out[k], ref[k]) < 1e-11, (k, oracle.rel_err(out[k], ref[k]))


def test_global_policy_parallel_long_horizon(solver):
    """n=64, m=32, T=4096 (the long-horizon workload), K=152: the error profile
    over the distance to the segment end. The stages of the policy sweep
    (distance 1) and those 16 or more stages from the end are at rounding
    level; the worst stage is the first of rank 0; the whole horizon within
    1e-8. The cancellation factor kappa_t = |Vxx_t| / |P_t| of the stages near
    the end of two segments comes from the oracle's segment solve and the
    error / (eps kappa_t) ratio is printed."""
    prob = workloads.config1()
    T, n, m = prob["B"].shape
    K = 152
    ref = oracle.riccati(prob)
    out = {k: v.cpu().numpy() for k, v in solver.global_policy_parallel(to_dev(prob), K).items()}
    assert solver.report()["status"] == 0
    d = _dist(T, K)
    reach = -(-n // m)
    eP = _stage_err(out["P"][:T], ref["P"][:T])
    eK = _stage_err(out["K"], ref["K"])
    prof = {dd: float(max(eP[d == dd].max(), eK[d == dd].max())) for dd in range(1, 20)}
    print("max error by distance to the segment end:", {k: "%.1e" % v for k, v in prof.items()})
    for k in ("K", "k", "P", "p"):
        assert oracle.rel_err(out[k], ref[k]) < 1e-8, (k, oracle.rel_err(out[k], ref[k]))
    for dd in range(1, reach):
        assert prof[dd] < 1e-13, (dd, prof[dd])
    assert max(eP[d >= 16].max(), eK[d >= 16].max(), eP[d == 0].max(), eK[d == 0].max()) < 1e-13
    # the worst stages: the first of rank 0 (P_t) and the next (K_t, whose stage
    # policy also carries the cancellation of the stage after it)
    assert max(prof.values()) == max(prof[reach], prof[reach + 1], prof[reach + 2])
    # the segment with the worst stage and a typical one: the size of the
    # subtracted term against P_t, and the conditioning of Vzz + P_e
    b = [j * T // K for j in range(K + 1)]
    worst = int(np.argmax(np.where(d == reach, eP, 0.0)))
    jw = max(j for j in range(K) if b[j] <= worst)
    for j in (jw, 100):
        for dd in range(reach, reach + 4):
            t = b[j + 1] - dd
            sm = oracle.segment_summary(prob, t, b[j + 1])
            S = sm["Vzz"] + ref["P"][b[j + 1]]
            sub = sm["Vzx"].T @ np.linalg.solve(S, sm["Vzx"])
            e = np.abs(out["P"][t] - ref["P"][t]).max() / np.abs(ref["P"][t]).max()
            print("segment %d distance %d: |Vzx'S^-1 Vzx| / |P_t| %.2e cond(Vzz + P_e) %.2e error %.2e" % (
                j, dd, np.abs(sub).max() / np.abs(ref["P"][t]).max(), np.linalg.cond(S), e))
