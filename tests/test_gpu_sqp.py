"""The trajectory-optimisation outer loop (lqr_sqp_solve: Gauss-Newton
multiple-shooting SQP whose LQR subproblems the segment-parallel solver
solves; Section I) against the oracle's loop (oracle.sqp: the same steps with
the serial recursion for every subproblem).

Per iteration the step lengths must be the same and the objective and
defects agree to 1e-9 (relative); the returned iterate, multipliers and
feedback gains agree to 1e-8 (the subproblem solutions differ by FP64
rounding, which the iteration carries along; both converge to the same
first-order point); the last feedforward k, the vanishing step's, to 1e-9 of
the controls' size. With linear dynamics one
step lands on the LQR optimum (the dense KKT solve)."""
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


def dev_model(model):
    return {k: (torch.from_numpy(np.ascontiguousarray(v)).to("cuda:0", torch.float64)
                if isinstance(v, np.ndarray) else v) for k, v in model.items()}


def run(solver, model, x, u, **kw):
    xd = torch.from_numpy(x.copy()).to("cuda:0", torch.float64)
    ud = torch.from_numpy(u.copy()).to("cuda:0", torch.float64)
    out = solver.sqp_solve(dev_model(model), xd, ud, **kw)
    return {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in out.items()}


@pytest.mark.parametrize("n,m,T,K,beta", [(6, 3, 50, 5, 0.6), (4, 2, 30, 3, 0.3), (5, 5, 40, 4, 0.4)])
def test_sqp_iterates_match_oracle(solver, n, m, T, K, beta):
    model = workloads.make_nl_model(n, m, T, seed=20 + n, beta=beta)
    x = np.zeros((T + 1, n))
    u = np.zeros((T, m))
    ref = oracle.sqp(model, x, u, iters=30, tol=1e-11)
    got = run(solver, model, x, u, max_iters=30, tol=1e-11, num_segments=K)
    assert got["report"]["converged"] == 1
    assert got["report"]["iters"] == len(ref["hist"])
    for i, (g, r) in enumerate(zip(got["hist"], ref["hist"])):
        assert g["alpha"] == r["alpha"], i
        assert abs(g["cost"] - r["cost"]) <= 1e-9 * abs(r["cost"]), (i, g["cost"], r["cost"])
        assert abs(g["defect"] - r["defect"]) <= 1e-9 * max(1.0, r["defect"]), (i, g["defect"], r["defect"])
    for key in ("x", "u", "lam", "K"):
        assert oracle.rel_err(got[key], ref[key]) < 1e-8, (key, oracle.rel_err(got[key], ref[key]))
    # k is the feedforward of the last (vanishing) step: rounding level against the controls
    assert np.abs(got["k"] - ref["k"]).max() < 1e-9 * max(1.0, np.abs(ref["u"]).max())


def test_sqp_linear_dynamics_one_step(solver):
    model = workloads.make_nl_model(5, 2, 40, seed=11, beta=0.0)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((41, 5))
    u = rng.standard_normal((40, 2))
    got = run(solver, model, x, u, max_iters=1, num_segments=4)
    assert got["hist"][0]["alpha"] == 1.0
    T = 40
    n, m = 5, 2
    Q, R, QT, xr = model["Q"], model["R"], model["QT"], model["xref"]
    lin = dict(A=np.repeat(model["A"][None], T, 0), B=np.repeat(model["B"][None], T, 0), c=np.zeros((T, n)),
               Q=np.concatenate([np.repeat(Q[None], T, 0), QT[None]]), R=np.repeat(R[None], T, 0),
               S=np.zeros((T, m, n)), q=np.concatenate([-xr[:T] @ Q.T, (-xr[T] @ QT.T)[None]]),
               r=np.zeros((T, m)), x0=model["x0"].copy())
    ref = oracle.dense_kkt(lin)
    for key in ("x", "u", "lam"):
        assert oracle.rel_err(got[key], ref[key]) < 1e-10, key


@pytest.mark.parametrize("prec,max_refine", [("fp64", 0), ("mixed_fp32", 6)])
def test_sqp_n64(solver, prec, max_refine):
    """n=64, m=32, T=512, beta=0.05, K=16: the converged iterate against the
    oracle loop's, with FP64 subproblems and with mixed-precision ones refined
    to a relative KKT residual of 1e-12."""
    n, m, T = 64, 32, 512
    model = workloads.make_nl_model(n, m, T, seed=84, beta=0.05)
    x = np.zeros((T + 1, n))
    u = np.zeros((T, m))
    ref = oracle.sqp(model, x, u, iters=30, tol=1e-10)
    got = run(solver, model, x, u, max_iters=30, tol=1e-10, num_segments=16, prec=prec, max_refine=max_refine,
              sub_tol=1e-12)
    assert got["report"]["converged"] == 1
    assert abs(got["report"]["iters"] - len(ref["hist"])) <= 1
    for key in ("x", "u", "lam"):
        assert oracle.rel_err(got[key], ref[key]) < 1e-8, (key, oracle.rel_err(got[key], ref[key]))
    assert np.abs(oracle.nl_dynamics(model, got["x"][:-1], got["u"]) - got["x"][1:]).max() < 1e-9


def test_sqp_rejects_bad_options(solver):
    from paper_1809_06360_gb300.lqr import LqrError
    model = workloads.make_nl_model(3, 2, 10, seed=1, beta=0.1)
    x = np.zeros((11, 3))
    u = np.zeros((10, 2))
    with pytest.raises(LqrError):
        run(solver, model, x, u, max_iters=0)
    with pytest.raises(LqrError):
        run(solver, model, x, u, max_iters=3, prec="fp32")
