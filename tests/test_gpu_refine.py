"""Steps A7/A8 on the GPU: the FP64 KKT residual kernel against the oracle's
residual of the same (x, u, lambda), iterative refinement, and the mixed
precision mode (FP64 data, FP32 sweeps, FP64 link solve and residual)."""
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


def host(out):
    return {k: v.double().cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("n,m,T,K,cross", [(12, 4, 128, 8, False), (7, 3, 61, 7, True), (5, 2, 1, 1, True)])
def test_residual_kernel_matches_oracle(solver, n, m, T, K, cross):
    prob = workloads.make_problem(n, m, T, seed=300 + n + T, cross=cross)
    out = host(solver.solve(to_dev(prob), num_segments=K, residual=True))
    rep = solver.report()
    assert rep["status"] == 0
    ref = oracle.kkt_residual(prob, out["x"], out["u"], out["lam"])
    # eta and rel of the same point; the residual itself is at rounding level,
    # so only its order of magnitude is comparable (different summation order)
    assert rep["kkt_residual"] < 1e-14 and ref["eta"] < 1e-14
    assert abs(rep["cost"] - oracle.stage_costs(prob, out["x"], out["u"])) <= 1e-11 * abs(rep["cost"])


def test_refinement_repairs_constrained_form(solver):
    """The constraint-explicit form loses ~1e-8 on the long-horizon workload;
    two FP64 refinement corrections bring x, u, lambda, k to the oracle at 1e-9."""
    prob = workloads.config1()
    ref = oracle.riccati(prob)
    out = host(solver.solve(to_dev(prob), num_segments=64, form="constrained", max_refine=2, tol=1e-13))
    rep = solver.report()
    assert rep["status"] == 0, rep
    for k in ("x", "u", "lam", "k", "K"):
        assert oracle.rel_err(out[k], ref[k]) < 1e-9, (k, oracle.rel_err(out[k], ref[k]))
    assert rep["kkt_rel"] < 1e-13 and rep["refine_iters"] >= 1


@pytest.mark.parametrize("K", [16, 64, 256])
def test_mixed_precision_config1(solver, K):
    """FP64 data, FP32 sweeps (FP64 Cholesky of R+B'PB), FP64 link solve,
    FP64 KKT residual with refinement to |r|/|b| <= 1e-12: x, u and lambda
    reach the oracle at 1e-9. The feedback gains K keep FP32 accuracy, and so
    does k, which refinement keeps consistent with them (u_t = K_t x_t + k_t
    along the refined trajectory to FP64 rounding): both stated, bound 1e-4."""
    prob = workloads.config1()
    ref = oracle.riccati(prob)
    out = host(solver.solve(to_dev(prob), num_segments=K, prec="mixed", max_refine=4, tol=1e-12))
    rep = solver.report()
    assert rep["status"] == 0, rep
    errs = {k: oracle.rel_err(out[k], ref[k]) for k in ("x", "u", "lam", "k", "K")}
    print("mixed K=%d errors %s iters %d rel %.2e eta %.2e" % (K, errs, rep["refine_iters"], rep["kkt_rel"],
                                                              rep["kkt_residual"]))
    for k in ("x", "u", "lam"):
        assert errs[k] < 1e-9, errs
    assert errs["K"] < 1e-4 and errs["k"] < 1e-4
    pol = np.einsum("tij,tj->ti", out["K"], out["x"][:-1]) + out["k"]
    assert oracle.rel_err(pol, out["u"]) < 1e-12
    assert rep["kkt_rel"] <= 1e-12
    assert abs(rep["cost"] - ref["cost"]) <= 1e-10 * abs(ref["cost"])


def test_no_convergence_is_reported(solver):
    prob = workloads.config0()
    solver.solve(to_dev(prob), num_segments=8, prec="mixed", max_refine=1, tol=1e-300)
    rep = solver.report()
    assert rep["status_name"] == "LQR_ERR_NO_CONVERGENCE"
    assert rep["refine_iters"] == 1


def test_refinement_stops_when_converged(solver):
    prob = workloads.config0()
    solver.solve(to_dev(prob), num_segments=8, prec="fp64", max_refine=5, tol=1e-6)
    rep = solver.report()
    assert rep["status"] == 0 and rep["refine_iters"] == 0  # FP64 already meets 1e-6


def test_mixed_host_entry_point(solver):
    prob = workloads.make_problem(16, 4, 96, seed=12)
    ref = oracle.riccati(prob)
    out = solver.solve_host(prob, num_segments=8, prec="mixed", want=("K", "k", "x", "u", "lam"),
                            max_refine=3, tol=1e-12)
    rep = solver.report()
    assert rep["status"] == 0
    assert oracle.rel_err(out["x"], ref["x"]) < 1e-9


def test_correction_copy_wait_timeout_is_reported(solver):
    """The correction recursions wait for their own bulk copies with a bounded
    poll count (opts.spin_limit): with a one-poll limit the first wait runs out
    (an 18 KB block does not land within one poll), the solve reports
    LQR_ERR_TIMEOUT instead of hanging, and the handle's next solve (default
    limit) succeeds and reaches the oracle."""
    prob = workloads.make_problem(64, 32, 512, seed=621, rho_max=1.02)
    dev = to_dev(prob)
    solver.solve(dev, num_segments=32, prec="mixed_fp32", max_refine=4, tol=1e-10, spin_limit=1)
    rep = solver.report()
    assert rep["status_name"] == "LQR_ERR_TIMEOUT", rep
    out = host(solver.solve(dev, num_segments=32, prec="mixed_fp32", max_refine=4, tol=1e-10))
    assert solver.report()["status"] == 0
    assert oracle.rel_err(out["x"], oracle.riccati(prob)["x"]) < 1e-9


def test_mixed_fp32_host_entry_pinned_and_pageable(solver):
    """lqr_solve_host in LQR_MIXED_FP32: with every input in mapped page-locked
    host memory the conversion kernel reads the inputs over the host link and
    writes the FP64 copy itself; with pageable inputs the copy engines stage
    them; K_t goes back on a copy stream beside the refinement. Either way the
    answer is the device entry point's, bit for bit."""
    prob = workloads.make_problem(32, 8, 300, seed=620, rho_max=1.02)
    want = ("K", "k", "x", "u", "lam")
    dev_out = host(solver.solve(to_dev(prob), num_segments=8, prec="mixed_fp32", max_refine=8, tol=1e-10))
    assert solver.report()["status"] == 0
    pinned = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory().numpy() for k, v in prob.items()}
    for inputs in (pinned, prob):
        out = solver.solve_host(inputs, num_segments=8, prec="mixed_fp32", want=want, max_refine=8, tol=1e-10)
        rep = solver.report()
        assert rep["status"] == 0 and rep["refine_iters"] >= 1, rep
        for k in want:
            assert np.array_equal(out[k], dev_out[k]), k


@pytest.mark.parametrize("prec", ["mixed", "mixed_fp32"])
@pytest.mark.parametrize("n,m,T,K", [(3, 5, 20, 4), (8, 16, 96, 8), (2, 9, 40, 5)])
def test_refinement_with_more_controls_than_states(solver, prec, n, m, T, K):
    """m > n: T m entries of u and k exceed the (T + 1) n entries of x and
    lambda, and every one of them must take the refinement update. The FP32
    solve leaves ~1e-6 errors, so a u entry the update skipped stays visibly
    wrong (x, u, lambda at 1e-9 against the oracle). Each correction satisfies
    du_t = K_t dx_t + dk_t, so refinement leaves d_t = u_t - K_t x_t - k_t as the
    unrefined solve had it (FP64 rounding in the mixed mode, FP32 rounding of the
    FP32 rollout in mixed_fp32); a k entry the update skipped would move d_t by
    its correction."""
    prob = workloads.make_problem(n, m, T, seed=500 + n * m, rho_max=1.02, cross=True)
    ref = oracle.riccati(prob)
    dev = to_dev(prob)
    out0 = host(solver.solve(dev, num_segments=K, prec=prec, max_refine=0))
    out = host(solver.solve(dev, num_segments=K, prec=prec, max_refine=6, tol=1e-12))
    rep = solver.report()
    assert rep["status"] == 0, rep
    errs = {k: oracle.rel_err(out[k], ref[k]) for k in ("x", "u", "lam", "k", "K")}
    print("%s m>n (%d,%d,%d,K=%d) errors %s iters %d rel %.2e" % (prec, n, m, T, K, errs, rep["refine_iters"],
                                                                  rep["kkt_rel"]))
    assert rep["refine_iters"] >= 1
    for k in ("x", "u", "lam"):
        assert errs[k] < 1e-9, errs
    assert errs["K"] < 1e-4 and errs["k"] < 1e-3
    assert np.array_equal(out["K"], out0["K"])
    d0 = out0["u"] - np.einsum("tij,tj->ti", out0["K"], out0["x"][:-1]) - out0["k"]
    d = out["u"] - np.einsum("tij,tj->ti", out["K"], out["x"][:-1]) - out["k"]
    assert np.abs(d - d0).max() <= 1e-10 * np.abs(out["u"]).max()
    assert rep["kkt_rel"] <= 1e-12


def _launches_per_correction(solver, prob, K):
    """Kernels one refinement correction enqueues (every correction is enqueued
    up to max_refine; a converged one returns at once on the device)."""
    dev = to_dev(prob)
    counts = []
    for it in (1, 2):
        solver.solve(dev, num_segments=K, prec="mixed_fp32", max_refine=it, tol=0.0)
        counts.append(solver.last_launch_count())
    return counts[1] - counts[0]


def test_mixed_fp32_correction_paths(solver):
    """Which correction path a shape takes. Where the correction kernels' plans
    fit (n=64, m=32: two stage-data slots and the fast sweep; n=72 and n=128:
    the generic FP32 sweep, which also keeps M_uu^-1; n=128 with one slot and
    the closed-loop maps reading B_t, K_t from global memory), corrections
    reuse the solve's K_t, P_t and M_uu^-1 and the refinement loop runs as a
    CUDA graph whose loop body is one iteration: the residual pass writing the
    FP32 correction vectors (two kernels, double-FP32 and FP64, gated on the
    iteration count), finalize, the correction (three per-stage kernels, four
    segment recursions, two link chains), update: 13 kernels per executed
    iteration when a chain is one kernel. With K >= 32 segments each link
    chain runs in two levels over groups of ceil(sqrt(K)) links (group
    offsets, the chain over the groups, the fill: three kernels), 17 kernels
    per iteration; K = 40 leaves a short last group, K = 49 none. n=136: the
    closed-loop maps' plan does not fit the shared memory, so each correction
    is a whole FP32 solve launched from the host (residual, finalize and update
    around the kernels of a plain FP32 solve of that shape). All reach the
    oracle at 1e-9."""
    cases = [(workloads.make_problem(64, 32, 256, seed=611, rho_max=1.02), 16, 13),
             (workloads.make_problem(72, 32, 288, seed=612, rho_max=1.02), 16, 13),
             (workloads.make_problem(128, 64, 256, seed=613, rho_max=1.02), 16, 13),
             (workloads.make_problem(64, 32, 400, seed=615, rho_max=1.02), 40, 17),
             (workloads.make_problem(128, 64, 392, seed=616, rho_max=1.02), 49, 17),
             (workloads.make_problem(136, 8, 160, seed=614, rho_max=1.02), 4, None)]
    for prob, K, expect in cases:
        per = _launches_per_correction(solver, prob, K)
        solver.solve(to_dev(prob, torch.float32), num_segments=K, prec="fp32")
        plain = solver.last_launch_count()
        assert per == (expect if expect is not None else 3 + plain), (prob["B"].shape, per, plain)
        ref = oracle.riccati(prob)
        out = host(solver.solve(to_dev(prob), num_segments=K, prec="mixed_fp32", max_refine=8, tol=1e-11))
        rep = solver.report()
        assert rep["status"] == 0, rep
        for k in ("x", "u", "lam"):
            assert oracle.rel_err(out[k], ref[k]) < 1e-9, (prob["B"].shape, k, oracle.rel_err(out[k], ref[k]))


def test_refinement_graph_stops_at_convergence(solver):
    """The refinement loop of the mixed modes runs as a graph whose WHILE node
    stops once the finalize kernel finds the solution converged: a cap of 8
    iterations launches exactly the kernels a cap of 3 does (two corrections
    and the pass that finds convergence), and the answer is the same bit for
    bit; a third problem in between (other arguments: the graph is rebuilt)
    does not disturb either."""
    prob = workloads.make_problem(64, 32, 512, seed=617, rho_max=1.02)
    other = workloads.make_problem(32, 8, 300, seed=618, rho_max=1.02)
    dev = to_dev(prob)
    res = {}
    for cap in (3, 8, 8, 3):
        out = host(solver.solve(dev, num_segments=32, prec="mixed_fp32", max_refine=cap, tol=1e-10))
        rep = solver.report()
        assert rep["status"] == 0 and rep["refine_iters"] == 2, rep
        res.setdefault(cap, []).append((solver.last_launch_count(), out))
        host(solver.solve(to_dev(other), num_segments=8, prec="mixed_fp32", max_refine=cap, tol=1e-10))
        assert solver.report()["status"] == 0
    counts = {cap: [c for c, _ in v] for cap, v in res.items()}
    assert counts[3][0] == counts[3][1] == counts[8][0] == counts[8][1], counts
    for k in ("x", "u", "lam", "k"):
        assert np.array_equal(res[3][0][1][k], res[8][0][1][k]), k
    ref = oracle.riccati(prob)
    assert oracle.rel_err(res[8][1][1]["x"], ref["x"]) < 1e-9


def test_refinement_plain_launches_match_graph(solver):
    """refine_plain = 1 launches the refinement loop's kernels one by one from
    the host instead of as the graph: the same kernels in the same order, so the
    answer and the report are the same bit for bit; every iteration up to
    max_refine is launched (the converged ones return at once on the device), so
    the plain loop reports more launches."""
    prob = workloads.make_problem(64, 32, 512, seed=619, rho_max=1.02)
    dev = to_dev(prob)
    outs, reps, counts = [], [], []
    for plain in (False, True, False):
        outs.append(host(solver.solve(dev, num_segments=32, prec="mixed_fp32", max_refine=8, tol=1e-10,
                                      refine_plain=plain)))
        reps.append(solver.report())
        counts.append(solver.last_launch_count())
    for rep in reps:
        assert rep["status"] == 0 and rep["refine_iters"] == 2, rep
    for k in ("x", "u", "lam", "k"):
        assert np.array_equal(outs[0][k], outs[1][k]) and np.array_equal(outs[0][k], outs[2][k]), k
    assert reps[0]["kkt_rel"] == reps[1]["kkt_rel"] and reps[0]["cost"] == reps[1]["cost"]
    assert counts[0] == counts[2] < counts[1], counts


@pytest.mark.parametrize("K", [64, 152])
def test_mixed_fp32_config1(solver, K):
    """LQR_MIXED_FP32: FP64 data; the solve runs the FP32 path (FP32 sweeps,
    FP32 M_uu inverse, FP32 link scan) on an FP32 copy of the data, and each
    correction reuses its K_t, P_t and M_uu^-1 (vector-only passes over the
    same segments; test_mixed_fp32_correction_paths pins which path runs); the
    FP64 KKT residual drives refinement to |r|/|b| <= 1e-10. x, u and lambda
    reach the oracle at 1e-9; K keeps FP32 accuracy (1e-4), k stays consistent
    with the refined trajectory."""
    prob = workloads.config1()
    ref = oracle.riccati(prob)
    out = host(solver.solve(to_dev(prob), num_segments=K, prec="mixed_fp32", max_refine=6, tol=1e-10))
    rep = solver.report()
    assert rep["status"] == 0, rep
    errs = {k: oracle.rel_err(out[k], ref[k]) for k in ("x", "u", "lam", "k", "K")}
    print("mixed_fp32 K=%d errors %s iters %d rel %.2e eta %.2e" % (K, errs, rep["refine_iters"], rep["kkt_rel"],
                                                                   rep["kkt_residual"]))
    for k in ("x", "u", "lam"):
        assert errs[k] < 1e-9, errs
    assert errs["K"] < 1e-4 and errs["k"] < 1e-3
    assert rep["kkt_rel"] <= 1e-10
    assert rep["refine_iters"] <= 4
    assert abs(rep["cost"] - ref["cost"]) <= 1e-10 * abs(ref["cost"])


def test_mixed_fp32_small_and_odd_shapes(solver):
    for (n, m, T, K) in ((12, 4, 128, 8), (30, 10, 600, 37), (5, 2, 1, 1)):
        prob = workloads.make_problem(n, m, T, seed=900 + n, rho_max=1.02)
        ref = oracle.riccati(prob)
        out = host(solver.solve(to_dev(prob), num_segments=K, prec="mixed_fp32", max_refine=6, tol=1e-11))
        rep = solver.report()
        assert rep["status"] == 0, (n, rep)
        for k in ("x", "u", "lam"):
            assert oracle.rel_err(out[k], ref[k]) < 1e-9, (n, k, oracle.rel_err(out[k], ref[k]))


def test_mixed_fp32_value_function_outputs(solver):
    """With P and p requested: the trajectory is refined to FP64 accuracy while P
    and p keep FP32 accuracy (they are not unknowns of the KKT system: P comes
    from the FP32 sweeps, and the corrections, which reuse K_t, P_t and M_uu^-1
    of the solve, update p consistently with lambda = -(P x + p) at that P)."""
    prob = workloads.make_problem(12, 4, 256, seed=77, rho_max=1.02, cross=True)
    ref = oracle.riccati(prob)
    out = host(solver.solve(to_dev(prob), num_segments=16, prec="mixed_fp32", max_refine=6, tol=1e-11,
                            want=("K", "k", "x", "u", "lam", "P", "p")))
    rep = solver.report()
    assert rep["status"] == 0, rep
    errs = {k: oracle.rel_err(out[k], ref[k]) for k in ("x", "u", "lam", "p", "P")}
    print("mixed_fp32 with P", errs, rep["refine_iters"])
    for k in ("x", "u", "lam"):
        assert errs[k] < 1e-9, errs
    assert errs["p"] < 1e-4 and errs["P"] < 1e-4, errs


def test_mixed_fp32_unsupported_forms(solver):
    from paper_1809_06360_gb300 import lqr
    prob = workloads.config0()
    with pytest.raises(lqr.LqrError) as e:
        solver.solve(to_dev(prob), num_segments=8, prec="mixed_fp32", form="constrained")
    assert e.value.status == 9


@pytest.fixture(scope="module")
def config2():
    prob = workloads.config2()
    return prob, oracle.riccati(prob)


@pytest.mark.parametrize("prec", ["mixed", "mixed_fp32"])
def test_config2_refined(solver, config2, prec):
    """The mixed-precision workload n=128, m=64, T=1024, K=64: FP64 data, FP32
    segment sweeps (the mixed TF32 mode: policy sweeps on the tensor cores with
    TF32 products and the FP64 Cholesky factor of R + B'PB), FP64 KKT residual
    and refinement to |r|/|b| <= 1e-8. x, u and
    lambda reach the oracle at 1e-9; K_t, k_t, P_t and p_t are not unknowns of
    the KKT system: K, k and P keep the accuracy of the FP32 sweeps (bound
    1e-4), p_t carries that of the FP32 link chain through the boundary values
    pi_j it starts from (bound 1e-3), all stated per quantity."""
    prob, ref = config2
    out = host(solver.solve(to_dev(prob), num_segments=64, prec=prec, max_refine=12, tol=1e-8,
                            want=("K", "k", "x", "u", "lam", "P", "p")))
    rep = solver.report()
    assert rep["status"] == 0, rep
    errs = {k: oracle.rel_err(out[k], ref[k]) for k in ("x", "u", "lam", "K", "k", "P", "p")}
    print("config2 %s errors %s iters %d rel %.2e eta %.2e" % (prec, errs, rep["refine_iters"], rep["kkt_rel"],
                                                             rep["kkt_residual"]))
    assert rep["kkt_rel"] <= 1e-8
    for k in ("x", "u", "lam"):
        assert errs[k] < 1e-9, errs
    # the mixed TF32 mode runs the policy sweeps on the tensor cores: TF32 class
    bound_mat, bound_p = (3e-2, 3e-2) if prec == "mixed" else (1e-4, 1e-3)
    for k in ("K", "k", "P"):
        assert errs[k] < bound_mat, errs
    assert errs["p"] < bound_p, errs
    assert abs(rep["cost"] - ref["cost"]) <= 1e-10 * abs(ref["cost"])
