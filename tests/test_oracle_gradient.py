"""Pin of the oracle's dense-KKT implicit gradient against central finite
differences of the serial Riccati oracle (two independent routes to dL/dtheta)."""
import numpy as np
import pytest

import oracle
import workloads


def loss(out):
    return float((out["x"] ** 2).sum() + (out["u"] ** 2).sum())


@pytest.mark.parametrize("n,m,T,cross", [(2, 1, 3, True), (3, 2, 4, True), (3, 1, 5, False)])
def test_implicit_gradient_matches_finite_differences(n, m, T, cross):
    prob = workloads.make_problem(n, m, T, seed=60 + n + T, cross=cross)
    ric = oracle.riccati(prob)
    g = oracle.kkt_implicit_gradient(prob, 2 * ric["x"], 2 * ric["u"])
    fd = oracle.fd_gradient(prob, loss, h=1e-6)
    for k in g:
        scale = max(1.0, np.abs(g[k]).max())
        assert np.abs(g[k] - fd[k]).max() <= 1e-6 * scale, (k, np.abs(g[k] - fd[k]).max())


def test_implicit_gradient_symmetry_of_Q_and_R():
    """Q and R enter symmetrised, so their gradients are symmetric matrices."""
    prob = workloads.make_problem(3, 2, 4, seed=70, cross=True)
    ric = oracle.riccati(prob)
    g = oracle.kkt_implicit_gradient(prob, ric["x"], ric["u"])
    assert np.abs(g["Q"] - np.swapaxes(g["Q"], 1, 2)).max() < 1e-12
    assert np.abs(g["R"] - np.swapaxes(g["R"], 1, 2)).max() < 1e-12
