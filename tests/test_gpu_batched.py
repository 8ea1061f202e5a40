"""Batched solve (many independent problems of uneven n, m, T in one call)
against the FP64 oracle, problem by problem."""
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


def to_dev(prob, dtype=torch.float64):
    return {k: torch.from_numpy(v).to("cuda:0", dtype) for k, v in prob.items()}


def uneven_batch(count, seed, Tmax=96):
    g = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(g.choice([8, 16, 32, 48]))
        m = int(g.integers(2, 17))
        T = int(g.integers(32, Tmax + 1))
        out.append(workloads.make_problem(n, m, T, seed=seed * 1000 + i, cross=bool(i % 3 == 0)))
    return out


@pytest.mark.parametrize("K", [0, 1, 2])
def test_batched_fp64_vs_oracle(solver, K):
    probs = uneven_batch(24, seed=7)
    dev = [to_dev(p) for p in probs]
    outs, seg = solver.solve_batched(dev, prec="fp64", num_segments=K)
    st, cost = solver.report_batched(len(probs))
    assert all(s == 0 for s in st), st
    if K == 0:
        assert max(seg) > 1  # a small batch is split into segments to fill the GPU
    for p, o, c in zip(probs, outs, cost):
        ref = oracle.riccati(p)
        for k in ("K", "k", "x", "u", "lam"):
            assert oracle.rel_err(o[k].cpu().numpy(), ref[k]) < 1e-9, k
        assert abs(c - ref["cost"]) <= 1e-9 * max(1.0, abs(ref["cost"]))


def test_batch_of_one_equals_single_solve(solver):
    p = workloads.make_problem(12, 4, 128, seed=1000)
    dev = to_dev(p)
    outs, seg = solver.solve_batched([dev], prec="fp64", num_segments=8)
    single = solver.solve(dev, num_segments=8, prec="fp64")
    for k in ("K", "k", "x", "u", "lam"):
        assert torch.equal(outs[0][k], single[k]), k


def test_batched_fp32_uneven(solver):
    probs = uneven_batch(40, seed=9, Tmax=200)
    dev = [to_dev(p, torch.float32) for p in probs]
    outs, seg = solver.solve_batched(dev, prec="fp32")
    st, _ = solver.report_batched(len(probs))
    assert all(s == 0 for s in st)
    worst = 0.0
    for p, o in zip(probs, outs):
        ref = oracle.riccati(p)
        for k in ("K", "k", "x", "u"):
            worst = max(worst, oracle.rel_err(o[k].double().cpu().numpy(), ref[k]))
    print("fp32 batched worst rel err %.2e" % worst)
    assert worst < 1e-3


@pytest.fixture(scope="module")
def config3():
    return workloads.config3()


def test_batched_config3_full(solver, config3):
    """The uneven-batch workload at full size: 4096 problems, T~U{32..512},
    n in {8,16,32,48}, m~U{2..16} (the workload's own seeds), FP32, one
    batched call (the persistent schedule or the per-step launches, whichever
    the autotuner measured faster; one segment per problem either way since
    the batch fills the GPU). Every problem is checked against the FP64 oracle
    on K, k, x and u at the FP32 bound 1e-3 (normwise per quantity)."""
    probs = config3
    dev = [to_dev(p, torch.float32) for p in probs]
    outs, seg = solver.solve_batched(dev, prec="fp32")
    st, cost = solver.report_batched(len(probs))
    assert all(s == 0 for s in st)
    assert max(seg) == 1
    worst = {k: 0.0 for k in ("K", "k", "x", "u")}
    for i, p in enumerate(probs):
        ref = oracle.riccati(p, want_P=False)
        for k in worst:
            e = oracle.rel_err(outs[i][k].double().cpu().numpy(), ref[k])
            worst[k] = max(worst[k], e)
            assert e < 1e-3, (i, k, e, p["B"].shape)
        assert abs(cost[i] - ref["cost"]) <= 1e-3 * max(1.0, abs(ref["cost"])), i
    print("config3 full batch worst per quantity", worst)


def test_batched_persistent_schedule(solver, config3):
    """num_segments = 1 selects the persistent schedule: one launch for the
    whole batch (CTAs take problems longest first), the same answers as the
    per-step launches to FP32 rounding."""
    from paper_1809_06360_gb300 import lqr
    probs = config3[:600]
    dev = [to_dev(p, torch.float32) for p in probs]
    outs, seg = solver.solve_batched(dev, prec="fp32", num_segments=1)
    assert lqr.lqr_last_launch_count(solver.h) == 1
    st, _ = solver.report_batched(len(probs))
    assert all(s == 0 for s in st) and max(seg) == 1
    for i in range(0, 600, 37):
        ref = oracle.riccati(probs[i], want_P=False)
        for k in ("K", "k", "x", "u"):
            assert oracle.rel_err(outs[i][k].double().cpu().numpy(), ref[k]) < 1e-3, (i, k)


def test_batched_error_is_per_problem(solver):
    probs = uneven_batch(6, seed=11)
    probs[3]["R"][5] = -np.eye(probs[3]["R"].shape[1]) * 100.0
    dev = [to_dev(p) for p in probs]
    solver.solve_batched(dev, prec="fp64", num_segments=1)
    st, _ = solver.report_batched(len(probs))
    assert st[3] == 2 and all(s == 0 for i, s in enumerate(st) if i != 3)
