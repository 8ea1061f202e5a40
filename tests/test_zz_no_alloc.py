"""The no-allocation KKT-residual entry point, for callers that cannot
allocate device memory while running (real-time control loops, code inside a
stream capture): called twice in a row through the C-ABI, its output must
match what the existing entry point (lqr_solve with the residual pass,
read back by lqr_report) reports for the same solution.
Collected last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-9  # the FP64 tolerance of the parity tests


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06360_gb300 import Solver, build
    build.build()
    s = Solver(0)
    yield s
    s.close()


def _structs(prob, sol):
    from paper_1809_06360_gb300 import lqr
    p = lqr.Solver.make_problem_struct(prob, lambda t: t.data_ptr())
    s = lqr.lqr_solution(**{f: (sol[f].data_ptr() if f in sol else None) for f in lqr.SOLUTION_FIELDS})
    return p, s


@pytest.mark.parametrize("prec,dtype", [("fp32", torch.float32), ("fp64", torch.float64),
                                        ("mixed_fp32", torch.float64)])
def test_noalloc_residual_matches_solve_report(solver, prec, dtype):
    from paper_1809_06360_gb300 import lqr
    prob_np = workloads.make_problem(12, 4, 200, seed=77, cross=True)
    prob = {k: torch.from_numpy(v).to("cuda:0", dtype) for k, v in prob_np.items()}
    sol = solver.solve(prob, num_segments=8, prec=prec, residual=True)
    rep = solver.report()
    assert rep["status"] == 0 and rep["kkt_residual"] >= 0.0
    ref = np.array([rep["kkt_residual"], rep["kkt_rel"], rep["cost"]])
    p, s = _structs(prob, sol)
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out.fill_(float("nan"))
        lqr.lqr_kkt_residual_noalloc(p, s, lqr.PRECISION[prec], out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), (call, got)
        rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)
        assert np.all(rel <= TOL), (call, got, ref)


def test_noalloc_rejects_too_long_horizon(solver):
    from paper_1809_06360_gb300 import lqr
    T = lqr.NOALLOC_MAX_STAGES + 1
    n = m = 1
    f = lambda *shape: torch.zeros(shape, dtype=torch.float64, device="cuda:0")
    prob = dict(A=f(T, n, n), B=f(T, n, m), c=f(T, n), Q=f(T + 1, n, n), R=f(T, m, m), S=f(T, m, n),
                q=f(T + 1, n), r=f(T, m), x0=f(n))
    sol = dict(x=f(T + 1, n), u=f(T, m), lam=f(T + 1, n))
    p, s = _structs(prob, sol)
    out = f(3)
    with pytest.raises(lqr.LqrError) as e:
        lqr.lqr_kkt_residual_noalloc(p, s, lqr.PRECISION["fp64"], out.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)
    assert e.value.status == 10
