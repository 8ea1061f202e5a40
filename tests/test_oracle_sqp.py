"""Pins of the oracle's trajectory-optimisation outer loop (Section I: the LQR
problem as the subproblem of trajectory optimisation): the Gauss-Newton
multiple-shooting SQP on the synthetic nonlinear tracking model.

  * The dynamics Jacobian against central finite differences of the dynamics.
  * Linear dynamics (beta = 0): one step from any starting point lands on the
    optimum of the resulting LQR problem, solved independently as the dense
    KKT system of Eq. 3.
  * At convergence: the dynamics hold and the gradient of the Lagrangian
    (Eq. 3's sign convention) vanishes, both evaluated with finite differences
    of the dynamics function alone.
"""
import numpy as np
import pytest

import oracle
import workloads


def test_nl_jacobian_matches_finite_differences():
    model = workloads.make_nl_model(5, 2, 4, seed=3, beta=0.7)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 5))
    J = oracle.nl_jacobian(model, x)
    h = 1e-6
    u = np.zeros((3, 2))
    for j in range(5):
        e = np.zeros(5)
        e[j] = h
        fd = (oracle.nl_dynamics(model, x + e, u) - oracle.nl_dynamics(model, x - e, u)) / (2 * h)
        assert np.abs(fd - J[:, :, j]).max() < 1e-8


def _linear_lqr(model):
    T = model["T"]
    n, m = model["B"].shape
    Q, R, QT, xr = model["Q"], model["R"], model["QT"], model["xref"]
    return dict(A=np.repeat(model["A"][None], T, 0), B=np.repeat(model["B"][None], T, 0), c=np.zeros((T, n)),
                Q=np.concatenate([np.repeat(Q[None], T, 0), QT[None]]), R=np.repeat(R[None], T, 0),
                S=np.zeros((T, m, n)), q=np.concatenate([-xr[:T] @ Q.T, (-xr[T] @ QT.T)[None]]),
                r=np.zeros((T, m)), x0=model["x0"].copy())


def test_sqp_linear_dynamics_one_step():
    model = workloads.make_nl_model(4, 2, 25, seed=11, beta=0.0)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((26, 4))
    u = rng.standard_normal((25, 2))
    out = oracle.sqp(model, x, u, iters=1)
    assert out["hist"][0]["alpha"] == 1.0
    ref = oracle.dense_kkt(_linear_lqr(model))
    assert oracle.rel_err(out["x"], ref["x"]) < 1e-10
    assert oracle.rel_err(out["u"], ref["u"]) < 1e-10
    assert oracle.rel_err(out["lam"], ref["lam"]) < 1e-10


@pytest.mark.parametrize("n,m,T,beta", [(4, 2, 30, 0.3), (6, 3, 50, 0.6)])
def test_sqp_converges_to_first_order_point(n, m, T, beta):
    model = workloads.make_nl_model(n, m, T, seed=20 + n, beta=beta)
    x = np.zeros((T + 1, n))
    u = np.zeros((T, m))
    out = oracle.sqp(model, x, u, iters=40, tol=1e-11)
    assert len(out["hist"]) < 40
    x, u, lam = out["x"], out["u"], out["lam"]
    # the dynamics and the initial condition hold
    assert np.abs(oracle.nl_dynamics(model, x[:-1], u) - x[1:]).max() < 1e-9
    assert np.abs(x[0] - model["x0"]).max() < 1e-9

    # Lagrangian L = J + lam_0'(x_0 - x_init) + sum_t lam_{t+1}'(x_{t+1} - f(x_t, u_t))
    def lagr(xx, uu):
        return (oracle.nl_cost(model, xx, uu) + lam[0] @ (xx[0] - model["x0"])
                + np.sum(lam[1:] * (xx[1:] - oracle.nl_dynamics(model, xx[:-1], uu))))
    rng = np.random.default_rng(7)
    h = 1e-5
    scale = max(1.0, np.abs(lam).max())
    for _ in range(8):
        dx = rng.standard_normal(x.shape)
        du = rng.standard_normal(u.shape)
        g = (lagr(x + h * dx, u + h * du) - lagr(x - h * dx, u - h * du)) / (2 * h)
        assert abs(g) < 1e-6 * scale * np.sqrt(x.size + u.size)
    # the merit decreased along the way and the last steps were full ones
    assert out["hist"][-1]["alpha"] == 1.0
