"""The FP64 KKT residual pass against the oracle at points where the residual
is well above rounding level.

At a computed solution the residual is at rounding level, so only its order
of magnitude can be compared with the oracle (summation orders differ). Here
the solution is perturbed first (x, u and lambda each by a seeded random vector
of relative size 1e-3), so that |KKT w - b|, the |KKT| row sums, |w| and |b|
are all O(1) quantities: the normwise backward error eta, the relative
residual rel and the objective of Eq. 1 must then match the oracle to FP64
rounding. The no-allocation entry point is used because it evaluates any given
point; it runs the same per-stage block as the residual pass of the
refinement step. Shapes cover every register column plan (max(n, m) <= 32, <= 64,
<= 128), matrices narrower than the plan, n and m odd, S present and absent,
horizons longer than the grid (several stages per CTA) and the generic loop
beyond 128."""
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


def _perturbed(prob, seed, prec):
    """Solve, then move x, u, lambda off the solution by 1e-3 relative."""
    rng = np.random.default_rng(seed)
    out = {}
    ref = oracle.riccati(prob)
    for k in ("x", "u", "lam"):
        v = ref[k]
        out[k] = v + 1e-3 * np.abs(v).max() * rng.standard_normal(v.shape)
    if prec == "fp32":
        out = {k: v.astype(np.float32).astype(np.float64) for k, v in out.items()}
    return out


@pytest.mark.parametrize("n,m,T,cross,prec", [
    (7, 3, 61, True, "fp64"),       # one register column, odd sizes
    (30, 10, 700, False, "fp64"),   # T > grid: several stages per CTA; S absent
    (64, 32, 1300, True, "fp64"),   # two columns for n, one for m
    (64, 32, 300, True, "fp32"),    # FP32 data, FP64 arithmetic
    (80, 16, 200, True, "fp64"),    # four columns for n, one for m
    (100, 70, 50, True, "fp64"),    # four columns for both
    (130, 5, 20, True, "fp64"),     # beyond the register plan: the generic loop
    (130, 5, 20, False, "fp64"),    # the generic loop without S
    (6, 130, 12, True, "fp64"),     # m > 128: the generic loop over the u rows
])
def test_residual_at_perturbed_point_matches_oracle(solver, n, m, T, cross, prec):
    from paper_1809_06360_gb300 import lqr
    prob = workloads.make_problem(n, m, T, seed=900 + n + m + T, cross=cross)
    if not cross:
        prob["S"] = np.zeros_like(prob["S"])
    dt = torch.float32 if prec == "fp32" else torch.float64
    if prec == "fp32":
        prob = {k: v.astype(np.float32).astype(np.float64) for k, v in prob.items()}
    sol = _perturbed(prob, seed=n * 7 + T, prec=prec)
    dev = {k: torch.from_numpy(v).to("cuda:0", dt) for k, v in prob.items()}
    if not cross:
        dev["S"] = None  # the kernels' S = 0 path
    dsol = {k: torch.from_numpy(v).to("cuda:0", dt) for k, v in sol.items()}
    p = lqr.Solver.make_problem_struct({k: v for k, v in dev.items() if v is not None},
                                       lambda t: t.data_ptr())
    s = lqr.lqr_solution(**{f: (dsol[f].data_ptr() if f in dsol else None) for f in lqr.SOLUTION_FIELDS})
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda:0")
    lqr.lqr_kkt_residual_noalloc(p, s, lqr.PRECISION[prec], out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    eta, rel, cost = out.cpu().numpy()
    ref = oracle.kkt_residual(prob, sol["x"], sol["u"], sol["lam"])
    ref_cost = oracle.stage_costs(prob, sol["x"], sol["u"])
    assert ref["rel"] > 1e-6  # well above rounding level
    assert abs(eta - ref["eta"]) <= 1e-12 * ref["eta"], (eta, ref["eta"])
    assert abs(rel - ref["rel"]) <= 1e-12 * ref["rel"], (rel, ref["rel"])
    assert abs(cost - ref_cost) <= 1e-12 * max(abs(ref_cost), 1.0), (cost, ref_cost)


@pytest.mark.parametrize("n,m,T,cross,perturb", [
    (7, 3, 61, True, True), (30, 10, 700, False, True), (64, 32, 1300, True, True), (128, 64, 300, True, True),
    (5, 9, 40, True, True), (33, 33, 20, False, True), (4, 2, 1, True, True), (64, 32, 512, True, False)])
def test_residual_vectors_double_fp32(solver, n, m, T, cross, perturb):
    """The residual blocks of Eq. 3 from the double-FP32 kernel of the refinement
    (lqr_kkt_residual_vectors) against the oracle's FP64 blocks, element by
    element, at points 1e-3 off the optimum and at the optimum itself: within
    2e-13 of |KKT| |w| + |b| (the scale the backward error divides by; the
    pairs keep about 47 bits, FP64 53)."""
    prob = workloads.make_problem(n, m, T, seed=950 + n + m + T, cross=cross)
    if not cross:
        prob["S"] = np.zeros_like(prob["S"])
    sol = _perturbed(prob, seed=n + 3 * T, prec="fp64") if perturb else {
        k: v for k, v in oracle.riccati(prob).items() if k in ("x", "u", "lam")}
    dev = {k: torch.from_numpy(v).to("cuda:0", torch.float64) for k, v in prob.items()}
    if not cross:
        dev["S"] = None
    dsol = {k: torch.from_numpy(np.ascontiguousarray(v)).to("cuda:0", torch.float64) for k, v in sol.items()}
    got = {k: v.cpu().numpy() for k, v in solver.kkt_residual_vectors(
        {k: v for k, v in dev.items() if v is not None}, dsol).items()}
    ref = oracle.kkt_blocks_residual(prob, sol["x"], sol["u"], sol["lam"])
    nrm = oracle.kkt_residual(prob, sol["x"], sol["u"], sol["lam"])
    scale = nrm["knorm"] * nrm["wnorm"] + nrm["bnorm"]
    err = max(np.abs(got["q"][:T] + ref["rx"]).max(), np.abs(got["q"][T] + ref["rxT"]).max(),
              np.abs(got["r"] + ref["ru"]).max(), np.abs(got["c"] - ref["rd"]).max(),
              np.abs(got["x0"] - ref["r0"]).max())
    print("n=%d m=%d T=%d residual %.2e error %.2e of scale %.2e" % (n, m, T, nrm["rnorm"], err, scale))
    assert err <= 2e-13 * scale, (err, scale)


def test_convert_f64_to_f32_rounds_to_nearest_even(solver):
    """The integer-operation FP64 -> FP32 conversion of the mixed modes'
    working copies (lqr_convert_f64_to_f32) against IEEE rounding (numpy's),
    bit for bit: magnitudes over the whole FP32 range and beyond, halfway
    cases (ties to even), subnormal results, overflow to infinity, signed
    zeros, infinities and NaN."""
    from paper_1809_06360_gb300 import lqr
    import warnings
    g = np.random.default_rng(11)
    v = g.standard_normal(300000) * 10.0 ** g.integers(-50, 50, 300000)
    f = g.standard_normal(5000).astype(np.float32)
    ties = (f.astype(np.float64) + np.nextafter(f, np.float32(np.inf)).astype(np.float64)) / 2
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 3.4028235677973366e38, 3.4028235e38 * 1.0000001,
                        2.0 ** -149, 2.0 ** -150, 2.0 ** -150 * 1.0000001, 1.1754942e-38, 2.0 ** -126 * (1 - 2 ** -25),
                        1e-300, -1e300, 1.0, -1.5])
    d = np.concatenate([v, ties, special])
    dd = torch.from_numpy(d).cuda()
    out = torch.empty(d.shape, dtype=torch.float32, device="cuda")
    lqr.lqr_convert_f64_to_f32(dd.data_ptr(), out.data_ptr(), d.size, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        want = d.astype(np.float32)
    nan = np.isnan(want)
    assert np.isnan(out.cpu().numpy()[nan]).all()
    assert np.array_equal(got[~nan], want.view(np.uint32)[~nan]), np.flatnonzero(got[~nan] != want.view(np.uint32)[~nan])[:5]
