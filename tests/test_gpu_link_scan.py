"""The FP32 link solve as an associative suffix scan (lqr_link LQR_LINK_SCAN)
against the block-elimination chain (LQR_LINK_CHAIN) and the FP64 oracle.

The scan composes the segment summaries in a different order than the chain,
so the two FP32 results differ by rounding only: per quantity they agree to
within the FP32 error bound of the chain itself, and both stay within the
FP32 bound against the oracle. Shapes cover K a power of two and not, n a
multiple of 4 and not (zero-padded tiles), K = 2 (one level) and the largest
n the scan's shared-memory plan accepts."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("K", "k", "x", "u", "lam")


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06360_gb300 import Solver, build
    build.build()
    s = Solver(0)
    yield s
    s.close()


def to_dev(prob, dtype=torch.float32):
    return {k: torch.from_numpy(v).to("cuda:0", dtype) for k, v in prob.items()}


def run(solver, prob, K, link):
    out = solver.solve(to_dev(prob), num_segments=K, prec="fp32", link=link, want=KEYS + ("P",))
    rep = solver.report()
    assert rep["status"] == 0, (link, rep)
    return {k: v.double().cpu().numpy() for k, v in out.items()}, rep


def levels(K):
    lv, s = 0, 1
    while s < K:
        lv, s = lv + 1, 2 * s
    return lv


@pytest.mark.parametrize("n,m,T,K", [
    (12, 4, 128, 2),      # one level
    (12, 4, 128, 7),      # K not a power of two
    (12, 4, 128, 32),
    (30, 10, 600, 37),    # n % 4 != 0: padded tiles; ragged segment lengths
    (64, 32, 1024, 16),
    (64, 32, 1024, 64),
    (80, 16, 640, 40),    # the largest n of the shared-memory plan, two register blocks per thread
])
def test_scan_matches_chain_and_oracle(solver, n, m, T, K):
    prob = workloads.make_problem(n, m, T, seed=4242 + n + K, rho_max=1.02)
    ref = oracle.riccati(prob)
    scan, rep_s = run(solver, prob, K, "scan")
    nl_scan = solver.last_launch_count()
    chain, rep_c = run(solver, prob, K, "chain")
    e_scan = {k: oracle.rel_err(scan[k], ref[k]) for k in KEYS + ("P",)}
    e_chain = {k: oracle.rel_err(chain[k], ref[k]) for k in KEYS + ("P",)}
    d = {k: oracle.rel_err(scan[k], chain[k]) for k in KEYS + ("P",)}
    print("n=%d K=%d scan %s chain %s diff %s" % (n, K, e_scan, e_chain, d))
    for k in ("K", "k", "x", "u", "P"):
        assert e_scan[k] < 1e-3, (k, e_scan)
        # same accuracy class as the chain: within 10x of its error, or below 1e-4
        assert e_scan[k] < max(10 * e_chain[k], 1e-4), (k, e_scan, e_chain)
    assert abs(rep_s["cost"] - ref["cost"]) / abs(ref["cost"]) < 1e-4
    # sweep, init, levels, feedback pass, link states, policy sweep, rollout, finalize
    assert nl_scan == 1 + 3 + levels(K) + 1 + 2, nl_scan


def test_scan_auto_is_default_for_fp32(solver):
    prob = workloads.make_problem(64, 32, 512, seed=77, rho_max=1.02)
    a, _ = run(solver, prob, 16, "auto")
    s, _ = run(solver, prob, 16, "scan")
    for k in KEYS:
        np.testing.assert_array_equal(a[k], s[k])


def test_scan_unsupported_requests(solver):
    from paper_1809_06360_gb300 import lqr
    prob = workloads.make_problem(12, 4, 64, seed=5)
    with pytest.raises(lqr.LqrError) as e:  # FP64 has no scan
        solver.solve(to_dev(prob, torch.float64), num_segments=4, prec="fp64", link="scan")
    assert e.value.status == 9
    with pytest.raises(lqr.LqrError) as e:  # nor the constrained form
        solver.solve(to_dev(prob), num_segments=4, prec="fp32", link="scan", form="constrained")
    assert e.value.status == 9
    big = workloads.make_problem(96, 8, 96 * 2, seed=6)
    with pytest.raises(lqr.LqrError) as e:  # beyond the shared-memory plan
        solver.solve(to_dev(big), num_segments=4, prec="fp32", link="scan")
    assert e.value.status == 9
    out = solver.solve(to_dev(big), num_segments=4, prec="fp32")  # auto: the chain
    assert solver.report()["status"] == 0
    ref = oracle.riccati(big)
    assert oracle.rel_err(out["x"].double().cpu().numpy(), ref["x"]) < 1e-3


@pytest.mark.parametrize("n,m,T,K", [(88, 24, 264, 11), (96, 8, 192, 4), (128, 64, 256, 16)])
def test_fp32_chain_beyond_the_scan(solver, n, m, T, K):
    """n beyond the scan's and the cluster chain's shared-memory plans (n a
    multiple of 8, up to 128): the single-CTA FP32 chain (serial link steps
    in shared memory) with the parallel feedback post-pass and the link-state
    chain, 3 launches; the whole solve stays in the FP32 bound against the
    oracle."""
    prob = workloads.make_problem(n, m, T, seed=4343 + n + K, rho_max=1.02)
    ref = oracle.riccati(prob)
    out, rep = run(solver, prob, K, "auto")
    e = {k: oracle.rel_err(out[k], ref[k]) for k in KEYS + ("P",)}
    print("fp32 chain n=%d m=%d K=%d errors %s" % (n, m, K, e))
    for k in ("K", "k", "x", "u", "P"):
        assert e[k] < 1e-3, (k, e)
    # sweep, chain + post-pass + link states, policy sweep, rollout, finalize
    assert solver.last_launch_count() == 1 + 3 + 3, solver.last_launch_count()


@pytest.mark.parametrize("prec", ["mixed", "mixed_fp32"])
def test_fp32_chain_under_refinement(solver, prec):
    """The mixed modes at n = 128 take the FP32 chain for the link solve; FP64
    refinement brings x, u, lambda to the oracle at 1e-9."""
    prob = workloads.make_problem(128, 64, 256, seed=4444, rho_max=1.02)
    ref = oracle.riccati(prob)
    out = solver.solve(to_dev(prob, torch.float64), num_segments=16, prec=prec, max_refine=8, tol=1e-11)
    rep = solver.report()
    assert rep["status"] == 0, rep
    for k in ("x", "u", "lam"):
        err = oracle.rel_err(out[k].cpu().numpy(), ref[k])
        assert err < 1e-9, (prec, k, err, rep)
