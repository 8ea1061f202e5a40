"""Seeded synthetic LQR workloads.

This module only draws random problem data. It holds none of the solver's
arithmetic, and it is the one module that both the FP64 oracle tests and the
GPU path (tests, bench) take their inputs from.

Problem statement (Section II, Eq. 1-2 of the paper): minimise
    sum_t  1/2 x'Q_t x + u'S_t x + 1/2 u'R_t u + q_t'x + r_t'u
         + 1/2 x_T'Q_T x_T + q_T'x_T
subject to x_{t+1} = A_t x_t + B_t u_t + c_t and x_0 = x0.
The paper's names are Q_xx=Q, Q_uu=R, Q_ux=S (m x n), q_x1=q, q_u1=r,
F_x=A, F_u=B, f_1=c, x_init=x0.

Array layout (row-major, stage-major, float64 numpy):
    A (T,n,n)  B (T,n,m)  c (T,n)  Q (T+1,n,n) [slot T = Q_T]
    R (T,m,m)  S (T,m,n)  q (T+1,n) [slot T = q_T]  r (T,m)  x0 (n,)

Distributions (the robot-trajectory-shaped synthetic family):
    A_t = I + 0.1*N(0,1)/sqrt(n), optionally rescaled so rho(A_t) <= rho_max
    B_t ~ N(0,1)/sqrt(n)
    Q_t = L L' + 1e-2 I, L ~ N(0,1) n x n (unscaled); Q_T likewise
    R_t = M M' + 1e-1 I, M ~ N(0,1) m x m (unscaled)
    S_t = 0 (or, with cross=True, a jointly PD [[Q,S'],[S,R]])
    q_t, r_t, c_t ~ N(0,1); x0 ~ N(0,I)
Seeds: numpy Generator(PCG64(seed)); config i uses seed 1000+i; problem j of a
batch config i uses 1000*(i+1)+j.
"""
from __future__ import annotations

import numpy as np

FIELDS = ("A", "B", "c", "Q", "R", "S", "q", "r", "x0")


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def make_problem(n: int, m: int, T: int, seed: int, rho_max: float | None = None,
                 cross: bool = False, scale_linear: float = 1.0) -> dict:
    """One seeded LQR problem in float64 (layout in the module docstring)."""
    if n < 1 or m < 1 or T < 1:
        raise ValueError("n, m, T must be >= 1")
    g = _rng(seed)
    eye_n = np.eye(n)
    A = eye_n[None] + 0.1 * g.standard_normal((T, n, n)) / np.sqrt(n)
    if rho_max is not None:
        rho = np.max(np.abs(np.linalg.eigvals(A)), axis=-1)
        A = A * np.minimum(1.0, rho_max / rho)[:, None, None]
    B = g.standard_normal((T, n, m)) / np.sqrt(n)
    c = scale_linear * g.standard_normal((T, n))
    if cross:
        # jointly positive-definite stage Hessian [[Q, S'], [S, R]]
        G = g.standard_normal((T, n + m, n + m)) / np.sqrt(n + m)
        H = G @ np.swapaxes(G, 1, 2) + 1e-1 * np.eye(n + m)[None]
        Q = np.empty((T + 1, n, n))
        Q[:T] = H[:, :n, :n]
        R = np.ascontiguousarray(H[:, n:, n:])
        S = np.ascontiguousarray(H[:, n:, :n])
        LT = g.standard_normal((n, n))
        Q[T] = LT @ LT.T + 1e-2 * eye_n
    else:
        L = g.standard_normal((T + 1, n, n))
        Q = L @ np.swapaxes(L, 1, 2) + 1e-2 * eye_n[None]
        M = g.standard_normal((T, m, m))
        R = M @ np.swapaxes(M, 1, 2) + 1e-1 * np.eye(m)[None]
        S = np.zeros((T, m, n))
    q = scale_linear * g.standard_normal((T + 1, n))
    r = scale_linear * g.standard_normal((T, m))
    x0 = g.standard_normal(n)
    out = dict(A=A, B=B, c=c, Q=Q, R=R, S=S, q=q, r=r, x0=x0)
    return {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in out.items()}


def dims(prob: dict) -> tuple[int, int, int]:
    T, n, m = prob["B"].shape
    return n, m, T


# --- the five workload families -------------------------------------------------

def config0() -> dict:
    """Single LQR, n=12, m=4, T=128 (plain FP64 method, K=8 segments)."""
    return make_problem(12, 4, 128, seed=1000)


def config1(T: int = 4096) -> dict:
    """Long horizon n=64, m=32, T=4096, rho(A_t) <= 1.02 (K swept 16..1024)."""
    return make_problem(64, 32, T, seed=1001, rho_max=1.02)


def config2(T: int = 1024) -> dict:
    """Mixed precision family n=128, m=64, T=1024 (K=64), rho(A_t) <= 1.02."""
    return make_problem(128, 64, T, seed=1002, rho_max=1.02)


def config3_shapes(count: int = 4096, seed: int = 1003) -> list[tuple[int, int, int]]:
    """(n, m, T) per problem of the uneven batch: T~U{32..512}, n in {8,16,32,48},
    m~U{2..16}, drawn problem by problem from the batch seed (so the first k
    shapes of a batch of any size are the same)."""
    g = _rng(seed)
    out = []
    for _ in range(count):
        n = int(g.choice(np.array([8, 16, 32, 48])))
        m = int(g.integers(2, 17))
        T = int(g.integers(32, 513))
        out.append((n, m, T))
    return out


def config3(count: int = 4096) -> list[dict]:
    """Uneven batch: problem i drawn with seed 1000*(3+1)+i."""
    return [make_problem(n, m, T, seed=4000 + i)
            for i, (n, m, T) in enumerate(config3_shapes(count))]


def config4(count: int = 256) -> list[dict]:
    """Differentiable batch: count problems of n=32, m=8, T=256 (K=16)."""
    return [make_problem(32, 8, 256, seed=5000 + i) for i in range(count)]


def double_integrator(T: int, dt: float, alpha: float = 10.0, alpha_T: float = 1e3,
                      beta: float = 1e-2) -> dict:
    """The double-integrator example of Section III-A (Eq. 17): cost
    alpha*|x_t|^2 + beta*|u_t|^2, terminal alpha_T*|x_T|^2, x0 = (1, 0).
    The paper leaves dt and T unstated; callers choose them."""
    n, m = 2, 1
    A = np.tile(np.array([[1.0, dt], [0.0, 1.0]]), (T, 1, 1))
    B = np.tile(np.array([[0.0], [dt]]), (T, 1, 1))
    Q = np.tile(2.0 * alpha * np.eye(n), (T + 1, 1, 1))
    Q[T] = 2.0 * alpha_T * np.eye(n)
    R = np.tile(2.0 * beta * np.eye(m), (T, 1, 1))
    out = dict(A=A, B=B, c=np.zeros((T, n)), Q=Q, R=R, S=np.zeros((T, m, n)),
               q=np.zeros((T + 1, n)), r=np.zeros((T, m)), x0=np.array([1.0, 0.0]))
    return {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in out.items()}


def time_invariant(n: int, m: int, T: int, seed: int, cross: bool = True) -> dict:
    """Stage data repeated over time (for the infinite-horizon limit pin)."""
    one = make_problem(n, m, 1, seed=seed, cross=cross)
    g = _rng(seed + 7)
    out = {}
    for k in ("A", "B", "c", "R", "S", "r"):
        out[k] = np.repeat(one[k], T, axis=0)
    out["Q"] = np.repeat(one["Q"][:1], T + 1, axis=0)
    out["q"] = np.repeat(one["q"][:1], T + 1, axis=0)
    out["x0"] = g.standard_normal(n)
    return {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in out.items()}


def make_nl_model(n: int, m: int, T: int, seed: int, beta: float = 0.2) -> dict:
    """A seeded nonlinear tracking problem for the trajectory-optimisation outer
    loop (the setting of the paper's Section I, whose subproblems are LQR):
        x_{t+1} = A x_t + B u_t + beta tanh(C x_t),  x_0 = x_init,
        cost  sum_t 1/2 (x_t - xref_t)'Q (x_t - xref_t) + 1/2 u_t'R u_t
              + 1/2 (x_T - xref_T)'Q_T (x_T - xref_T).
    Time-invariant A (I + 0.1 N(0,1)/sqrt(n), rescaled to rho(A) <= 1),
    B ~ N(0,1)/sqrt(n), C ~ N(0,1)/sqrt(n); Q = L L'/n + I, Q_T = 10 Q,
    R = M M'/m + 0.1 I; the reference is a sum of three random sinusoids per
    state over the horizon (amplitudes 0.1 N(0,1)); x_init ~ N(0, I)."""
    g = _rng(seed)
    A = np.eye(n) + 0.1 * g.standard_normal((n, n)) / np.sqrt(n)
    A = A / max(1.0, np.max(np.abs(np.linalg.eigvals(A))))
    B = g.standard_normal((n, m)) / np.sqrt(n)
    C = g.standard_normal((n, n)) / np.sqrt(n)
    L = g.standard_normal((n, n))
    Q = L @ L.T / n + np.eye(n)
    M = g.standard_normal((m, m))
    R = M @ M.T / m + 0.1 * np.eye(m)
    t = np.arange(T + 1)[:, None] / max(T, 1)
    xref = np.zeros((T + 1, n))
    for _ in range(3):
        amp = 0.1 * g.standard_normal(n)
        freq = g.uniform(0.5, 4.0, n)
        phase = g.uniform(0.0, 2 * np.pi, n)
        xref += amp * np.sin(2 * np.pi * freq * t + phase)
    x0 = g.standard_normal(n)
    return dict(A=A, B=B, C=C, beta=float(beta), Q=Q, R=R, QT=10.0 * Q, xref=xref, x0=x0, T=T)
