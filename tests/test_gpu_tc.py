"""The tensor-core product unit of the segment sweeps (tcgen05, kind::tf32):
its products in every operand form the sweep issues agree with CUDA-core
FP32 products of the same operands to the TF32 rounding of the operands
(10 mantissa bits: unit roundoff 2^-11 ~ 4.9e-4 per operand, normwise
differences of order 1e-3 over K = 128 terms), and X - X with the second
product negated cancels to FP32 accumulation rounding."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06360_gb300 import build, lqr
    build.build()
    return lqr


def test_tensor_core_products_match_cuda_cores(lib):
    errs = lib.lqr_tc_selftest(0)
    print("tc selftest", errs)
    assert errs[4] == 0.0
    for e in errs[:3]:
        assert 1e-6 < e < 1e-2, errs  # TF32 rounding is visible, layout errors are O(1)
    assert errs[3] < 1e-5, errs


@pytest.fixture(scope="module")
def solver(lib):
    from paper_1809_06360_gb300 import Solver
    s = Solver(0)
    yield s
    s.close()


def _dev(prob):
    return {k: torch.from_numpy(v).to("cuda:0", torch.float64) for k, v in prob.items()}


@pytest.mark.parametrize("n,m,T,K", [(128, 64, 256, 16), (96, 24, 192, 8), (72, 8, 144, 6)])
def test_tensor_core_policy_sweep(solver, n, m, T, K):
    """LQR_MIXED_TF32 for 64 < n <= 128, m <= 64: the policy sweeps (step A4)
    run on the tensor cores with TF32 stage products and the FP64 Cholesky
    factor of R + B'PB. Unrefined, the gains carry TF32 rounding (errors of
    order 1e-3 against the FP64 oracle, where FP32 products give ~1e-6: the
    signature of the tensor-core path); FP64 refinement then brings x, u and
    lambda to the oracle at 1e-9."""
    import oracle
    import workloads
    prob = workloads.make_problem(n, m, T, seed=7000 + n + m, rho_max=1.02, cross=(n == 96))
    ref = oracle.riccati(prob)
    dev = _dev(prob)
    raw = solver.solve(dev, num_segments=K, prec="mixed", max_refine=0)
    assert solver.report()["status"] == 0
    e_raw = {k: oracle.rel_err(raw[k].cpu().numpy(), ref[k]) for k in ("K", "k", "x", "u")}
    out = solver.solve(dev, num_segments=K, prec="mixed", max_refine=12, tol=1e-11)
    rep = solver.report()
    assert rep["status"] == 0, rep
    e = {k: oracle.rel_err(out[k].cpu().numpy(), ref[k]) for k in ("K", "k", "x", "u", "lam")}
    print("tc sweep n=%d m=%d K=%d unrefined %s refined %s iters %d rel %.2e" % (n, m, K, e_raw, e,
                                                                                 rep["refine_iters"], rep["kkt_rel"]))
    assert 2e-5 < e_raw["K"] < 3e-2, e_raw
    for k in ("x", "u", "lam"):
        assert e[k] < 1e-9, e
    assert e["K"] < 3e-2
