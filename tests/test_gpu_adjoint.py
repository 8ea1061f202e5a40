"""Adjoint (gradients of a trajectory loss w.r.t. every datum) on the GPU
against the oracle's dense-KKT implicit gradient and FP64 central finite
differences of the serial oracle (h = 1e-6)."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("A", "B", "c", "Q", "R", "S", "q", "r", "x0")


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06360_gb300 import Solver, build
    build.build()
    s = Solver(0)
    yield s
    s.close()


def to_dev(prob, dtype=torch.float64):
    return {k: torch.from_numpy(v).to("cuda:0", dtype) for k, v in prob.items()}


def sq_loss(out):
    return float((out["x"] ** 2).sum() + (out["u"] ** 2).sum())


@pytest.mark.parametrize("n,m,T,K", [(3, 2, 12, 3), (5, 2, 20, 4), (4, 3, 9, 1)])
def test_backward_vs_dense_kkt_gradient(solver, n, m, T, K):
    prob = workloads.make_problem(n, m, T, seed=80 + n * T, cross=True)
    dev = to_dev(prob)
    sol = solver.solve(dev, num_segments=K)
    gx, gu = 2 * sol["x"], 2 * sol["u"]
    grads = solver.backward(dev, sol, gx, gu, num_segments=K)
    assert solver.report()["status"] == 0
    ref = oracle.kkt_implicit_gradient(prob, gx.cpu().numpy(), gu.cpu().numpy())
    for k in FIELDS:
        err = oracle.rel_err(grads[k].cpu().numpy(), ref[k])
        assert err < 1e-9, (k, err)


def test_backward_differentiable_batch_shape_vs_fd(solver):
    """One problem of the differentiable-batch shape (n=32, m=8, T=256, K=16),
    loss sum |x_t|^2 + |u_t|^2: sampled entries against FP64 central FD."""
    prob = workloads.make_problem(32, 8, 256, seed=5000)
    dev = to_dev(prob)
    sol = solver.solve(dev, num_segments=16)
    grads = solver.backward(dev, sol, 2 * sol["x"], 2 * sol["u"], num_segments=16)
    fd = oracle.fd_gradient(prob, sq_loss, keys=("A", "B", "Q", "R", "q", "r", "x0", "c"), entries=4, h=1e-6)
    for k, v in fd.items():
        g = grads[k].cpu().numpy()
        mask = ~np.isnan(v)
        scale = max(1.0, np.abs(g).max())
        assert np.abs(g[mask] - v[mask]).max() <= 1e-5 * scale, (k, np.abs(g[mask] - v[mask]).max(), scale)


def test_autograd_function_matches_backward(solver):
    from paper_1809_06360_gb300.autograd import lqr
    prob = workloads.make_problem(6, 2, 30, seed=90, cross=True)
    t = {k: torch.from_numpy(v).to("cuda:0").requires_grad_(True) for k, v in prob.items()}
    x, u = lqr(*[t[k] for k in FIELDS], num_segments=3)
    loss = (x ** 2).sum() + (u ** 2).sum()
    loss.backward()
    ref = oracle.kkt_implicit_gradient(prob, 2 * x.detach().cpu().numpy(), 2 * u.detach().cpu().numpy())
    for k in FIELDS:
        assert oracle.rel_err(t[k].grad.cpu().numpy(), ref[k]) < 1e-9, k


def test_autograd_batch_fp32(solver):
    """Stacked equal-shape problems (the differentiable-batch layout) in FP32:
    gradients against the FP64 dense-KKT reference of each problem."""
    from paper_1809_06360_gb300.autograd import lqr_batch
    probs = [workloads.make_problem(4, 2, 16, seed=100 + i) for i in range(6)]
    stacked = {k: torch.from_numpy(np.stack([p[k] for p in probs])).to("cuda:0", torch.float32).requires_grad_(True)
               for k in FIELDS}
    x, u = lqr_batch(*[stacked[k] for k in FIELDS], num_segments=2, prec="fp32")
    ((x ** 2).sum() + (u ** 2).sum()).backward()
    worst = 0.0
    for i, p in enumerate(probs):
        ric = oracle.riccati(p)
        ref = oracle.kkt_implicit_gradient(p, 2 * ric["x"], 2 * ric["u"])
        for k in FIELDS:
            worst = max(worst, oracle.rel_err(stacked[k].grad[i].double().cpu().numpy(), ref[k]))
    print("fp32 batched adjoint worst rel err %.2e" % worst)
    assert worst < 1e-3


@pytest.fixture(scope="module")
def config4():
    return workloads.config4()


def test_config4_differentiable_batch(solver, config4):
    """The differentiable batch at full size: 256 problems n=32, m=8, T=256,
    K=16 in FP32, loss sum |x_t|^2 + |u_t|^2 through torch.autograd
    (lqr_batch: one batched forward solve, one batched adjoint solve). Four
    problems spread over the batch are checked on sampled entries of every
    gradient against FP64 central finite differences of the serial oracle
    (h = 1e-6), at the FP32 bound 1e-3 of each array's largest gradient entry;
    every problem's trajectory is checked against the oracle at the FP32 bound."""
    from paper_1809_06360_gb300.autograd import lqr_batch
    probs = config4
    stacked = {k: torch.from_numpy(np.stack([p[k] for p in probs])).to("cuda:0", torch.float32).requires_grad_(True)
               for k in FIELDS}
    x, u = lqr_batch(*[stacked[k] for k in FIELDS], num_segments=16, prec="fp32")
    ((x ** 2).sum() + (u ** 2).sum()).backward()
    xs = x.detach().double().cpu().numpy()
    us = u.detach().double().cpu().numpy()
    for i, p in enumerate(probs):
        ric = oracle.riccati(p, want_P=False)
        assert oracle.rel_err(xs[i], ric["x"]) < 1e-3 and oracle.rel_err(us[i], ric["u"]) < 1e-3, i
    for i in (0, 63, 128, 255):
        fd = oracle.fd_gradient(probs[i], sq_loss, keys=("A", "B", "Q", "R", "q", "r", "x0", "c"), entries=4,
                                h=1e-6, seed=i)
        for k, v in fd.items():
            g = stacked[k].grad[i].double().cpu().numpy()
            mask = ~np.isnan(v)
            scale = max(1e-12, np.abs(g).max())
            err = np.abs(g[mask] - v[mask]).max() / scale
            assert err < 1e-3, (i, k, err)
