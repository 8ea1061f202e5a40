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


def test_rcp_newton_against_ieee_division(lib):
    """The FP64 pivot reciprocal (FP32 seed + two Newton-Raphson steps) against
    IEEE 1/d over magnitudes 1e-300 .. 1e300 and both signs: the seed has
    about 23 correct bits, each step doubles them (46, then beyond the 53 of
    FP64), so the result is within 1 ulp of the correctly rounded reciprocal;
    outside the FP32 exponent range the division itself is used."""
    import numpy as np
    g = np.random.default_rng(3)
    mant = g.uniform(1.0, 2.0, size=20000)
    expo = g.integers(-996, 997, size=20000)
    sign = np.where(g.random(20000) < 0.5, -1.0, 1.0)
    d = sign * np.ldexp(mant, expo)
    d = np.concatenate([d, [1.0, -1.0, 3.0, 1e-30 * 1.5, 1e30 / 1.5, 2.0 ** 126, 2.0 ** -125]])
    dd = torch.from_numpy(d).cuda()
    y = torch.empty_like(dd)
    lib.lqr_rcp_newton_check(dd.data_ptr(), y.data_ptr(), dd.numel(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    ref = 1.0 / d
    ulp = np.abs(got - ref) / np.spacing(np.abs(ref))
    print("rcp_newton max ulp", ulp.max())
    assert ulp.max() <= 1.0, ulp.max()


def test_bounded_wait_times_out_and_recovers(solver):
    """A spin limit of one poll makes the tensor-core sweep's completion waits
    run out: the solve reports LQR_ERR_TIMEOUT (the kernel waits once more,
    with the default limit, for its own tensor-core products, frees its tensor
    memory and returns), and the next solve on the same handle succeeds."""
    import workloads
    prob = workloads.make_problem(128, 64, 128, seed=77, rho_max=1.02)
    dev = _dev(prob)
    solver.solve(dev, num_segments=8, prec="mixed", spin_limit=1)
    rep = solver.report()
    assert rep["status_name"] == "LQR_ERR_TIMEOUT", rep
    solver.solve(dev, num_segments=8, prec="mixed", max_refine=10, tol=1e-11)
    assert solver.report()["status"] == 0
