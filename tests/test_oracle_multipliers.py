"""Pins of the oracle's least-squares multipliers (Section II-B, "Lagrange
Multipliers": the over-determined stationarity system and its normal
equations).

  * At the optimum the system is consistent, so its least-squares solution is
    the exact multiplier vector: it must equal the multipliers of the global
    KKT system of Eq. 3 solved densely, for every partition; each interior
    segment's mu is minus its end multiplier (no terminal cost), and its end
    multiplier is the next segment's first one.
  * Away from the optimum the solution must minimise the sum of squared
    stationarity residuals of the segment, evaluated independently through
    kkt_blocks_residual (the residual of Eq. 3, pinned against the dense KKT
    system): zero gradient and no decrease under random perturbations.
"""
import numpy as np
import pytest

import oracle
import workloads


def _bounds(T, K):
    return [j * T // K for j in range(K + 1)]


@pytest.mark.parametrize("n,m,T,K", [(3, 2, 12, 1), (3, 2, 12, 3), (4, 1, 16, 4), (2, 3, 9, 2), (5, 2, 20, 5)])
def test_ls_multipliers_equal_dense_kkt(n, m, T, K):
    prob = workloads.make_problem(n, m, T, seed=700 + 10 * n + K, rho_max=1.05)
    ref = oracle.dense_kkt(prob)
    out = oracle.ls_multipliers(prob, ref["x"], ref["u"], _bounds(T, K))
    assert oracle.rel_err(out["lam"], ref["lam"]) < 1e-9
    b = _bounds(T, K)
    for j in range(K - 1):
        assert np.abs(out["lam_end"][j] - ref["lam"][b[j + 1]]).max() < 1e-9 * np.abs(ref["lam"]).max()
        assert np.abs(out["mu"][j] + out["lam_end"][j]).max() < 1e-9 * np.abs(ref["lam"]).max()


def _segment_ls_objective(prob, x, u, b, e, lam_seg, last):
    """Sum of squared stationarity residuals of the segment [b, e) with the
    segment's multipliers lam_seg (L + 1 rows), through kkt_blocks_residual on
    the global arrays (the other stages' multipliers do not enter these rows).
    The end row of an interior segment is zeroed by its free mu and drops out."""
    T = prob["B"].shape[0]
    lam = np.zeros((T + 1, prob["B"].shape[1]))
    lam[b:e + 1] = lam_seg
    res = oracle.kkt_blocks_residual(prob, x, u, lam)
    f = np.sum(res["rx"][b:e] ** 2) + np.sum(res["ru"][b:e] ** 2)
    if last:
        f += np.sum(res["rxT"] ** 2)
    return f


@pytest.mark.parametrize("K", [1, 3])
def test_ls_multipliers_minimise_residual_off_optimum(K):
    n, m, T = 4, 2, 15
    prob = workloads.make_problem(n, m, T, seed=731, rho_max=1.05)
    ref = oracle.dense_kkt(prob)
    rng = np.random.default_rng(5)
    x = ref["x"] + 0.1 * rng.standard_normal(ref["x"].shape)
    u = ref["u"] + 0.1 * rng.standard_normal(ref["u"].shape)
    b = _bounds(T, K)
    out = oracle.ls_multipliers(prob, x, u, b)
    for j in range(K):
        last = j == K - 1
        seg = np.vstack([out["lam"][b[j]:b[j + 1]], out["lam"][T][None] if last else out["lam_end"][j][None]])
        f0 = _segment_ls_objective(prob, x, u, b[j], b[j + 1], seg, last)
        assert f0 > 1e-6  # off the optimum the system is inconsistent
        # zero gradient (central differences) and a minimum along random directions
        h = 1e-5
        for _ in range(6):
            d = rng.standard_normal(seg.shape)
            fp = _segment_ls_objective(prob, x, u, b[j], b[j + 1], seg + h * d, last)
            fm = _segment_ls_objective(prob, x, u, b[j], b[j + 1], seg - h * d, last)
            assert abs(fp - fm) / (2 * h) < 1e-6 * max(1.0, f0)
            assert _segment_ls_objective(prob, x, u, b[j], b[j + 1], seg + 0.1 * d, last) >= f0
        if not last:
            assert np.abs(out["mu"][j] + out["lam_end"][j]).max() < 1e-12 * max(1.0, np.abs(seg).max())
