"""FP64 oracle for the segment-parallel Riccati solver.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it. The product path never imports,
links or calls anything here, and nothing here imports the product package.

Contents
--------
riccati(prob)            serial FP64 Riccati recursion in plain C (lqr_oracle.c):
                         the plain definition of the unique optimum (Section II,
                         Eq. 1-3; the serial method of Section III-A).
dense_kkt(prob)          the global KKT system of Eq. 3 assembled densely and solved
                         with numpy.linalg.solve (brute force, tiny sizes only).
segment_summary(...)     the endpoint-constrained segment problem of Section II-B
                         (Eq. 8) solved by a dense KKT solve with the two end states
                         as parameters; returns the quadratic cost_to_go(x, x_term)
                         of Eq. 9 at the segment start: (Vxx, Vzx, Vzz, vx, vz, v0).
segment_dual_summary(...) the same segment problem with its end-point constraint
                         dualised (end cost mu'x_term): the dual value
                         G(x_s, mu) = 1/2 x_s'P x_s + mu'Z x_s - 1/2 mu'W mu + p'x_s + w'mu,
                         by a dense KKT solve with (x_s, mu) as parameters.
kkt_residual(prob, ...)  the residual of Eq. 3 and its normwise backward error.
global_policy_from_segment(...) the global cost to go and policy at one stage
                         from the end-constrained value of the rest of its segment
                         and the global value at the segment end (Section II-B,
                         Section III-A).
nl_dynamics / nl_jacobian / sqp(...)  the nonlinear tracking problem of the
                         trajectory-optimisation outer loop (Section I: its
                         subproblems are LQR problems) and a Gauss-Newton
                         multiple-shooting SQP loop whose subproblems are solved
                         by riccati().
ls_multipliers(...)      the multipliers of every segment problem from the
                         over-determined stationarity system of Section II-B
                         ("Lagrange Multipliers"), solved through its normal
                         equations as the paper states.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lqr_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liblqr_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into oracle/_build (host code, any arch)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        lib.oracle_riccati.restype = ctypes.c_int
        lib.oracle_riccati.argtypes = [ctypes.c_int] * 3 + [d] * 18
        _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dims(prob):
    T, n, m = prob["B"].shape
    return n, m, T


class OracleError(RuntimeError):
    pass


def riccati(prob: dict, want_P: bool = True) -> dict:
    """Serial FP64 Riccati recursion (C). Returns K,k,P,p,s,x,u,lam,cost."""
    lib = _load()
    n, m, T = _dims(prob)
    arr = {k: np.ascontiguousarray(prob[k], dtype=np.float64) for k in
           ("A", "B", "c", "Q", "R", "S", "q", "r", "x0")}
    out = dict(K=np.empty((T, m, n)), k=np.empty((T, m)),
               P=np.empty((T + 1, n, n)) if want_P else None, p=np.empty((T + 1, n)),
               s=np.empty(T + 1), x=np.empty((T + 1, n)), u=np.empty((T, m)),
               lam=np.empty((T + 1, n)) if want_P else None, cost=np.empty(1))
    st = lib.oracle_riccati(n, m, T, _ptr(arr["A"]), _ptr(arr["B"]), _ptr(arr["c"]),
                            _ptr(arr["Q"]), _ptr(arr["R"]), _ptr(arr["S"]), _ptr(arr["q"]),
                            _ptr(arr["r"]), _ptr(arr["x0"]), _ptr(out["K"]), _ptr(out["k"]),
                            _ptr(out["P"]), _ptr(out["p"]), _ptr(out["s"]), _ptr(out["x"]),
                            _ptr(out["u"]), _ptr(out["lam"]), _ptr(out["cost"]))
    if st == 1:
        raise OracleError("R_t + B'P B not positive definite")
    if st != 0:
        raise OracleError("oracle_riccati failed with status %d" % st)
    out["cost"] = float(out["cost"][0])
    return out


# ---------------------------------------------------------------------------
# Dense KKT (brute force) -- Eq. 3 of the paper
# ---------------------------------------------------------------------------

def _sym(M):
    return 0.5 * (M + np.swapaxes(M, -1, -2))


def dense_kkt(prob: dict) -> dict:
    """Assemble the KKT system of Eq. 3 densely and solve it.

    Unknowns w = (x_0..x_T, u_0..u_{T-1}) and multipliers lambda_0..lambda_T,
    with the Lagrangian f(w) + lambda_0'(x_0 - x0)
    + sum_t lambda_{t+1}'(x_{t+1} - A_t x_t - B_t u_t - c_t), so that
    stationarity in x_t reads Q x_t + S'u_t + q_t + lambda_t - A_t'lambda_{t+1} = 0
    exactly as printed in Eq. 3.
    """
    n, m, T = _dims(prob)
    A, B, c, Q, R, S, q, r, x0 = (prob[k] for k in ("A", "B", "c", "Q", "R", "S", "q", "r", "x0"))
    Q = _sym(Q)
    R = _sym(R)
    nx = (T + 1) * n
    nw = nx + T * m
    nc = (T + 1) * n
    H = np.zeros((nw, nw))
    g = np.zeros(nw)
    C = np.zeros((nc, nw))
    d = np.zeros(nc)

    def xs(t):
        return slice(t * n, (t + 1) * n)

    def us(t):
        return slice(nx + t * m, nx + (t + 1) * m)

    for t in range(T):
        H[xs(t), xs(t)] = Q[t]
        H[us(t), us(t)] = R[t]
        H[us(t), xs(t)] = S[t]
        H[xs(t), us(t)] = S[t].T
        g[xs(t)] = q[t]
        g[us(t)] = r[t]
    H[xs(T), xs(T)] = Q[T]
    g[xs(T)] = q[T]
    C[0:n, xs(0)] = np.eye(n)
    d[0:n] = x0
    for t in range(T):
        rows = slice((t + 1) * n, (t + 2) * n)
        C[rows, xs(t + 1)] = np.eye(n)
        C[rows, xs(t)] = -A[t]
        C[rows, us(t)] = -B[t]
        d[rows] = c[t]
    Kmat = np.block([[H, C.T], [C, np.zeros((nc, nc))]])
    rhs = np.concatenate([-g, d])
    sol = np.linalg.solve(Kmat, rhs)
    w = sol[:nw]
    lam = sol[nw:]
    x = w[:nx].reshape(T + 1, n)
    u = w[nx:].reshape(T, m)
    cost = 0.5 * w @ H @ w + g @ w
    return dict(x=x, u=u, lam=lam.reshape(T + 1, n), cost=float(cost), kkt=Kmat, rhs=rhs)


def segment_summary(prob: dict, t0: int, t1: int) -> dict:
    """Endpoint-constrained problem on stages t0..t1-1 (Eq. 8: x_{t0} = x_s,
    x_{t1} = z, no terminal cost), solved by a dense KKT solve with (x_s, z)
    as right-hand-side parameters.

    Its optimal value is the quadratic of Eq. 9,
        J(x_s, z) = 1/2 x_s'Vxx x_s + z'Vzx x_s + 1/2 z'Vzz z + vx'x_s + vz'z + v0,
    read off through the envelope identity dJ/dx_s = -nu_init, dJ/dz = -nu_term
    (nu = the multipliers of the two endpoint constraints, same sign convention
    as Eq. 3 and Eq. 12).
    """
    n, m, T = _dims(prob)
    if not (0 <= t0 < t1 <= T):
        raise ValueError("bad segment")
    L = t1 - t0
    A, B, c, Q, R, S, q, r = (prob[k] for k in ("A", "B", "c", "Q", "R", "S", "q", "r"))
    Q = _sym(Q)
    R = _sym(R)
    nx = (L + 1) * n
    nw = nx + L * m
    nc = (L + 2) * n
    H = np.zeros((nw, nw))
    g = np.zeros(nw)
    C = np.zeros((nc, nw))
    d0 = np.zeros(nc)

    def xs(i):
        return slice(i * n, (i + 1) * n)

    def us(i):
        return slice(nx + i * m, nx + (i + 1) * m)

    for i in range(L):
        t = t0 + i
        H[xs(i), xs(i)] = Q[t]
        H[us(i), us(i)] = R[t]
        H[us(i), xs(i)] = S[t]
        H[xs(i), us(i)] = S[t].T
        g[xs(i)] = q[t]
        g[us(i)] = r[t]
        rows = slice((i + 1) * n, (i + 2) * n)
        C[rows, xs(i + 1)] = np.eye(n)
        C[rows, xs(i)] = -A[t]
        C[rows, us(i)] = -B[t]
        d0[rows] = c[t]
    C[0:n, xs(0)] = np.eye(n)                      # x_{t0} = x_s
    C[(L + 1) * n:(L + 2) * n, xs(L)] = np.eye(n)  # x_{t1} = z
    Kmat = np.block([[H, C.T], [C, np.zeros((nc, nc))]])
    # right-hand sides: [zero parameters | x_s = e_i | z = e_i]
    rhs = np.zeros((nw + nc, 1 + 2 * n))
    rhs[:nw, 0] = -g
    rhs[nw:, 0] = d0
    for i in range(n):
        rhs[nw + i, 1 + i] = 1.0
        rhs[nw + (L + 1) * n + i, 1 + n + i] = 1.0
    sol = np.linalg.solve(Kmat, rhs)
    nu_init = sol[nw:nw + n]                  # (n, 1+2n)
    nu_term = sol[nw + (L + 1) * n:nw + nc]   # (n, 1+2n)
    Vxx = -nu_init[:, 1:1 + n]
    Vzz = -nu_term[:, 1 + n:]
    Vzx = -nu_term[:, 1:1 + n]
    vx = -nu_init[:, 0]
    vz = -nu_term[:, 0]
    w0 = sol[:nw, 0]
    v0 = 0.5 * w0 @ H @ w0 + g @ w0
    u0 = sol[us(0)]  # the first control as an affine function of (x_s, z)
    return dict(Vxx=Vxx, Vzx=Vzx, Vzz=Vzz, vx=vx, vz=vz, v0=float(v0),
                Vxz_from_init=-nu_init[:, 1 + n:], Kx=u0[:, 1:1 + n], Kz=u0[:, 1 + n:], k1=u0[:, 0])


def global_policy_from_segment(prob: dict, t: int, t1: int, P_end, p_end) -> dict:
    """The global cost to go and policy at stage t from the end-constrained
    problem on stages t..t1-1 (Eq. 8-9: its value J(x, z) and its first
    control u_t = Kx x + Kz z + k1, by segment_summary) and the global value
    1/2 z'P_end z + p_end'z at the end link point t1: the minimising end
    state z* = -(Vzz + P_end)^-1 (Vzx x + vz + p_end) gives
        P_t = Vxx - Vzx'(Vzz + P_end)^-1 Vzx,   p_t = vx - Vzx'(Vzz + P_end)^-1 (vz + p_end),
        K_t = Kx - Kz (Vzz + P_end)^-1 Vzx,      k_t = k1 - Kz (Vzz + P_end)^-1 (vz + p_end)
    (the per-stage reconstruction of the global policy from a segment's
    parametric value, Section II-B with Section III-A's global value). Needs
    t1 - t stages enough to reach every end state (a regular J)."""
    sm = segment_summary(prob, t, t1)
    Sm = sm["Vzz"] + np.asarray(P_end)
    X = np.linalg.solve(Sm, np.column_stack([sm["Vzx"], sm["vz"] + np.asarray(p_end)]))
    Xx, xv = X[:, :-1], X[:, -1]
    return dict(P=sm["Vxx"] - sm["Vzx"].T @ Xx, p=sm["vx"] - sm["Vzx"].T @ xv,
                K=sm["Kx"] - sm["Kz"] @ Xx, k=sm["k1"] - sm["Kz"] @ xv)


def segment_dual_summary(prob: dict, t0: int, t1: int) -> dict:
    """The segment problem of Eq. 8 with its end-point constraint dualised:
    stages t0..t1-1, x_{t0} = x_s, no end constraint and, in place of it, the
    linear end cost mu'x_{t1} (mu the end multiplier of Eq. 10). Its optimal
    value is the quadratic
        G(x_s, mu) = 1/2 x_s'P x_s + mu'Z x_s - 1/2 mu'W mu + p'x_s + w'mu + g0,
    and J(x_s, z) of Eq. 9 is max_mu G(x_s, mu) - mu'z. Solved by a dense KKT
    solve with (x_s, mu) as right-hand-side parameters; the blocks are read off
    through dG/dx_s = -nu_init (the multiplier of x_{t0} = x_s, sign of Eq. 3)
    and dG/dmu = x_{t1} at the optimum. Returns P, Z, W, p, w, and Zt_from_init,
    the transpose of Z as it appears in dG/dx_s (equal to Z' in exact
    arithmetic)."""
    n, m, T = _dims(prob)
    if not (0 <= t0 < t1 <= T):
        raise ValueError("bad segment")
    L = t1 - t0
    A, B, c, Q, R, S, q, r = (prob[k] for k in ("A", "B", "c", "Q", "R", "S", "q", "r"))
    Q = _sym(Q)
    R = _sym(R)
    nx = (L + 1) * n
    nw = nx + L * m
    nc = (L + 1) * n
    H = np.zeros((nw, nw))
    g = np.zeros(nw)
    C = np.zeros((nc, nw))
    d0 = np.zeros(nc)

    def xs(i):
        return slice(i * n, (i + 1) * n)

    def us(i):
        return slice(nx + i * m, nx + (i + 1) * m)

    for i in range(L):
        t = t0 + i
        H[xs(i), xs(i)] = Q[t]
        H[us(i), us(i)] = R[t]
        H[us(i), xs(i)] = S[t]
        H[xs(i), us(i)] = S[t].T
        g[xs(i)] = q[t]
        g[us(i)] = r[t]
        rows = slice((i + 1) * n, (i + 2) * n)
        C[rows, xs(i + 1)] = np.eye(n)
        C[rows, xs(i)] = -A[t]
        C[rows, us(i)] = -B[t]
        d0[rows] = c[t]
    C[0:n, xs(0)] = np.eye(n)  # x_{t0} = x_s
    Kmat = np.block([[H, C.T], [C, np.zeros((nc, nc))]])
    # right-hand sides: [zero parameters | x_s = e_i | mu = e_i]; mu enters the
    # gradient of the end state, so its columns sit in the stationarity rows
    rhs = np.zeros((nw + nc, 1 + 2 * n))
    rhs[:nw, 0] = -g
    rhs[nw:, 0] = d0
    for i in range(n):
        rhs[nw + i, 1 + i] = 1.0
        rhs[L * n + i, 1 + n + i] = -1.0
    sol = np.linalg.solve(Kmat, rhs)
    nu_init = sol[nw:nw + n]   # (n, 1+2n): -dG/dx_s
    x_end = sol[L * n:nx]      # (n, 1+2n):  dG/dmu
    P = -nu_init[:, 1:1 + n]
    p = -nu_init[:, 0]
    Z = x_end[:, 1:1 + n]
    W = -x_end[:, 1 + n:]
    w = x_end[:, 0]
    return dict(P=P, Z=Z, W=W, p=p, w=w, Zt_from_init=-nu_init[:, 1 + n:])


def kkt_blocks_residual(prob: dict, x, u, lam):
    """Residual blocks of Eq. 3 at (x, u, lambda), FP64:
      rx_t = Q x_t + S'u_t + q_t + lam_t - A'lam_{t+1}   (t < T)
      ru_t = S x_t + R u_t + r_t - B'lam_{t+1}
      rxT  = Q_T x_T + q_T + lam_T
      r0   = x_0 - x0
      rd_t = x_{t+1} - A x_t - B u_t - c_t
    """
    A, B, c, Q, R, S, q, r, x0 = (prob[k] for k in ("A", "B", "c", "Q", "R", "S", "q", "r", "x0"))
    Q = _sym(Q)
    R = _sym(R)
    T = B.shape[0]
    xt, xn = x[:T], x[1:]
    lt, ln = lam[:T], lam[1:]
    rx = (np.einsum("tij,tj->ti", Q[:T], xt) + np.einsum("tji,tj->ti", S, u) + q[:T] + lt
          - np.einsum("tji,tj->ti", A, ln))
    ru = (np.einsum("tij,tj->ti", S, xt) + np.einsum("tij,tj->ti", R, u) + r
          - np.einsum("tji,tj->ti", B, ln))
    rxT = Q[T] @ x[T] + q[T] + lam[T]
    r0 = x[0] - x0
    rd = xn - np.einsum("tij,tj->ti", A, xt) - np.einsum("tij,tj->ti", B, u) - c
    return dict(rx=rx, ru=ru, rxT=rxT, r0=r0, rd=rd)


def ls_multipliers(prob: dict, x, u, bounds, only=None) -> dict:
    """Multipliers of the segment problems from the paper's least-squares
    system (Section II-B, "Lagrange Multipliers"; Eq. mults, mu, multsglobal,
    pseudoinverse), at the given trajectory (x, u).

    Segment j covers stages bounds[j] .. bounds[j+1]-1 and is the problem of
    the constraint-explicit section: x at its first stage fixed (multiplier
    lambda_0), the dynamics (lambda_1..lambda_L), and for every segment but the
    last its end state fixed (multiplier mu) with no terminal cost; the last
    segment carries the terminal cost Q_T, q_T and no end constraint (the
    splitting of Section II-A). With L stages, the stationarity conditions are
      x rows, i < L:  lambda_i - A_t'lambda_{i+1} = g_i = -(Q_t x_t + S_t'u_t + q_t)
      u rows, i < L:           -B_t'lambda_{i+1} = h_i = -(S_t x_t + R_t u_t + r_t)
      end row:        lambda_L (+ mu)             = g_L
    (t = bounds[j] + i; g_L = -(Q_T x_T + q_T) for the last segment, 0 else).
    The matrix of this system (the paper's A') has full column rank; its
    least-squares solution comes from the normal equations A A' lambda = A b,
    assembled densely here and solved with numpy.linalg.solve.

    Returns lam ((T+1) x n: lambda_t for t in segment j's stages from segment
    j, lambda_T from the last segment), lam_end ((K-1) x n: each interior
    segment's own lambda_L, the multiplier of the dynamics into the next
    segment's first state) and mu ((K-1) x n). With `only` (segment indices),
    just those segments are solved; the other entries stay zero."""
    A, B, Q, R, S, q, r = (prob[k] for k in ("A", "B", "Q", "R", "S", "q", "r"))
    Q = _sym(Q)
    R = _sym(R)
    n, m, T = _dims(prob)
    K = len(bounds) - 1
    lam = np.zeros((T + 1, n))
    lam_end = np.zeros((max(K - 1, 0), n))
    mu = np.zeros((max(K - 1, 0), n))
    for j in (range(K) if only is None else only):
        b, e = bounds[j], bounds[j + 1]
        L = e - b
        last = (j == K - 1)
        nunk = (L + 1) * n + (0 if last else n)
        neq = L * (n + m) + n
        At = np.zeros((neq, nunk))  # the paper's A': equations x unknowns
        rhs = np.zeros(neq)

        def lcol(i):
            return slice(i * n, (i + 1) * n)

        for i in range(L):
            t = b + i
            xr = slice(i * n, (i + 1) * n)
            ur = slice(L * n + i * m, L * n + (i + 1) * m)
            At[xr, lcol(i)] = np.eye(n)
            At[xr, lcol(i + 1)] = -A[t].T
            At[ur, lcol(i + 1)] = -B[t].T
            rhs[xr] = -(Q[t] @ x[t] + S[t].T @ u[t] + q[t])
            rhs[ur] = -(S[t] @ x[t] + R[t] @ u[t] + r[t])
        er = slice(L * (n + m), L * (n + m) + n)
        At[er, lcol(L)] = np.eye(n)
        if last:
            rhs[er] = -(Q[T] @ x[T] + q[T])
        else:
            At[er, (L + 1) * n:] = np.eye(n)
        sol = np.linalg.solve(At.T @ At, At.T @ rhs)
        lam[b:e] = sol[:L * n].reshape(L, n)
        if last:
            lam[T] = sol[L * n:(L + 1) * n]
        else:
            lam_end[j] = sol[L * n:(L + 1) * n]
            mu[j] = sol[(L + 1) * n:]
    return dict(lam=lam, lam_end=lam_end, mu=mu)


def kkt_residual(prob: dict, x, u, lam) -> dict:
    """Normwise backward error of (x, u, lambda) for the KKT system of Eq. 3:
        eta = |KKT w - b|_inf / (|KKT|_inf |w|_inf + |b|_inf),
    with |KKT|_inf the largest absolute row sum, computed block by block, and
    b = (-q, -r, -q_T, x0, c). Also returns rel = |KKT w - b|_inf / |b|_inf."""
    A, B, c, Q, R, S, q, r, x0 = (prob[k] for k in ("A", "B", "c", "Q", "R", "S", "q", "r", "x0"))
    Qs = _sym(Q)
    Rs = _sym(R)
    T = B.shape[0]
    res = kkt_blocks_residual(prob, x, u, lam)
    rnorm = max(np.abs(v).max() for v in res.values())
    # row sums of |KKT|
    row_x = (np.abs(Qs[:T]).sum(-1) + np.abs(S).sum(-2) + 1.0 + np.abs(A).sum(-2))
    row_u = np.abs(S).sum(-1) + np.abs(Rs).sum(-1) + np.abs(B).sum(-2)
    row_xT = np.abs(Qs[T]).sum(-1) + 1.0
    row_d = 1.0 + np.abs(A).sum(-1) + np.abs(B).sum(-1)
    knorm = max(row_x.max(), row_u.max(), row_xT.max(), 1.0, row_d.max())
    wnorm = max(np.abs(x).max(), np.abs(u).max(), np.abs(lam).max())
    bnorm = max(np.abs(q).max(), np.abs(r).max(), np.abs(x0).max(), np.abs(c).max())
    return dict(eta=rnorm / (knorm * wnorm + bnorm), rel=rnorm / bnorm, rnorm=rnorm,
                knorm=knorm, wnorm=wnorm, bnorm=bnorm)


def stage_costs(prob: dict, x, u) -> float:
    """Objective of Eq. 1-2 along a trajectory (x, u)."""
    A, B, c, Q, R, S, q, r = (prob[k] for k in ("A", "B", "c", "Q", "R", "S", "q", "r"))
    T = B.shape[0]
    xt = x[:T]
    J = (0.5 * np.einsum("ti,tij,tj->", xt, Q[:T], xt) + np.einsum("ti,tij,tj->", u, S, xt)
         + 0.5 * np.einsum("ti,tij,tj->", u, R, u) + np.einsum("ti,ti->", q[:T], xt)
         + np.einsum("ti,ti->", r, u))
    J += 0.5 * x[T] @ Q[T] @ x[T] + q[T] @ x[T]
    return float(J)


def rel_err(a, ref) -> float:
    """Normwise relative error max|a - ref| / max|ref| over the stacked tensor."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.abs(ref).max()
    num = np.abs(a - ref).max()
    return float(num / den) if den > 0 else float(num)


# ---------------------------------------------------------------------------
# Gradients of a loss of the optimal trajectory (brute force references)
# ---------------------------------------------------------------------------

def kkt_implicit_gradient(prob: dict, gx, gu) -> dict:
    """dL/dtheta for every datum theta, where L has gradients gx = dL/dx
    ((T+1) x n) and gu = dL/du (T x m) at the optimum, by differentiating the
    KKT system of Eq. 3 entry by entry: the assembly is linear in the data, so
    d(KKT)/dtheta_e and d(rhs)/dtheta_e are the assembly of the unit change of
    theta_e (exactly), and dw/dtheta_e = -KKT^{-1} (dKKT w - drhs).
    Tiny problems only (one assembly per entry)."""
    import scipy.linalg
    base = dense_kkt(prob)
    Kmat, rhs = base["kkt"], base["rhs"]
    lu = scipy.linalg.lu_factor(Kmat)
    w = scipy.linalg.lu_solve(lu, rhs)
    n, m, T = _dims(prob)
    nw = (T + 1) * n + T * m
    g = np.zeros(Kmat.shape[0])
    g[:(T + 1) * n] = np.asarray(gx).ravel()
    g[(T + 1) * n:nw] = np.asarray(gu).ravel()
    out = {}
    for key in ("A", "B", "c", "Q", "R", "S", "q", "r", "x0"):
        arr = prob[key]
        grad = np.zeros_like(arr)
        flat = grad.reshape(-1)
        for e in range(arr.size):
            pert = {k: v.copy() for k, v in prob.items()}
            pert[key].reshape(-1)[e] += 1.0
            pk = dense_kkt(pert)
            dK = pk["kkt"] - Kmat
            db = pk["rhs"] - rhs
            dw = -scipy.linalg.lu_solve(lu, dK @ w - db)
            flat[e] = g @ dw
        out[key] = grad
    return out


def fd_gradient(prob: dict, loss, keys=None, h: float = 1e-6, entries: int | None = None, seed: int = 0) -> dict:
    """Central finite differences (step h) of loss(riccati(prob)) with the
    serial C oracle; loss maps the oracle's output dict to a float. With
    `entries`, only that many randomly chosen entries per array are perturbed
    (the others are NaN)."""
    rng = np.random.default_rng(seed)
    out = {}
    for key in keys or ("A", "B", "c", "Q", "R", "S", "q", "r", "x0"):
        arr = prob[key]
        grad = np.full(arr.shape, np.nan)
        idx = np.arange(arr.size) if entries is None else rng.choice(arr.size, size=min(entries, arr.size),
                                                                       replace=False)
        for e in idx:
            p1 = {k: v.copy() for k, v in prob.items()}
            p2 = {k: v.copy() for k, v in prob.items()}
            p1[key].reshape(-1)[e] += h
            p2[key].reshape(-1)[e] -= h
            grad.reshape(-1)[e] = (loss(riccati(p1)) - loss(riccati(p2))) / (2 * h)
        out[key] = grad
    return out


# ---------------------------------------------------------------------------
# The trajectory-optimisation outer loop (Section I: LQR as the subproblem)
# ---------------------------------------------------------------------------

def nl_dynamics(model: dict, x, u):
    """f(x, u) = A x + B u + beta tanh(C x) (x, u may carry a leading stage axis)."""
    A, B, C, beta = model["A"], model["B"], model["C"], model["beta"]
    return x @ A.T + u @ B.T + beta * np.tanh(x @ C.T)


def nl_jacobian(model: dict, x):
    """df/dx = A + beta diag(1 - tanh(C x)^2) C (df/du = B), for a stack of states."""
    A, C, beta = model["A"], model["C"], model["beta"]
    th = np.tanh(x @ C.T)
    return A[None] + beta * (1.0 - th ** 2)[..., :, None] * C[None]


def nl_cost(model: dict, x, u) -> float:
    """The tracking objective of the model at (x, u)."""
    Q, R, QT, xr = model["Q"], model["R"], model["QT"], model["xref"]
    e = x - xr
    return float(0.5 * np.einsum("ti,ij,tj->", e[:-1], Q, e[:-1]) + 0.5 * np.einsum("ti,ij,tj->", u, R, u)
                 + 0.5 * e[-1] @ QT @ e[-1])


def sqp_subproblem(model: dict, x, u) -> dict:
    """The LQR subproblem in the step (dx, du) at the iterate (x, u): dynamics
    linearised at every stage (A_t = df/dx, B_t = B, c_t = f(x_t, u_t) - x_{t+1}),
    the objective's exact quadratic model (its Hessians Q, R, Q_T and gradients
    q_t = Q (x_t - xref_t), r_t = R u_t), dx_0 = x_init - x_0."""
    T = u.shape[0]
    n, m = model["B"].shape
    Q, R, QT, xr = model["Q"], model["R"], model["QT"], model["xref"]
    prob = dict(A=nl_jacobian(model, x[:T]), B=np.repeat(model["B"][None], T, 0),
                c=nl_dynamics(model, x[:T], u) - x[1:],
                Q=np.concatenate([np.repeat(Q[None], T, 0), QT[None]]), R=np.repeat(R[None], T, 0),
                S=np.zeros((T, m, n)), q=np.concatenate([(x[:T] - xr[:T]) @ Q.T, ((x[T] - xr[T]) @ QT.T)[None]]),
                r=u @ R.T, x0=model["x0"] - x[0])
    return prob


def sqp_merit_terms(model: dict, x, u, dx, du, alpha: float):
    """Objective and l1 norm of the constraint defects (dynamics and initial
    state) at the trial point (x + alpha dx, u + alpha du)."""
    xa, ua = x + alpha * dx, u + alpha * du
    d = np.abs(nl_dynamics(model, xa[:-1], ua) - xa[1:]).sum() + np.abs(xa[0] - model["x0"]).sum()
    return nl_cost(model, xa, ua), float(d)


SQP_ALPHAS = tuple(0.5 ** i for i in range(8))


def sqp(model: dict, x, u, iters: int, tol: float = 1e-10, nu_min: float = 1.0) -> dict:
    """Gauss-Newton multiple-shooting SQP for the nonlinear tracking problem:
    at every iterate the LQR subproblem (sqp_subproblem) is solved by the serial
    recursion (riccati), giving the step (dx, du) and the new multipliers
    lambda; the step length is the first alpha of 1, 1/2, ..., 1/128 whose
    l1 merit phi(alpha) = J + nu D (D the defects' l1 norm,
    nu = max(nu_min, 2 max|lambda|)) satisfies the Armijo condition
    phi(alpha) <= phi(0) + 1e-4 alpha (g'd - nu D(0)) (g'd the objective's
    directional derivative), else the last one; the full step when the
    predicted decrease |g'd - nu D(0)| is below 1e-12 max(1, |phi(0)|) (the
    merit differences are then at rounding level). Stops after `iters`
    iterations or once alpha max|(dx, du)| <= tol max(1, max|(x, u)|) (the
    iterate before the step) and D(alpha) <= tol. Returns the iterate, the last multipliers and policy, and
    per iteration the step length, merit and defects."""
    x = np.array(x, dtype=np.float64)
    u = np.array(u, dtype=np.float64)
    hist = []
    lam = K = k = None
    for it in range(iters):
        prob = sqp_subproblem(model, x, u)
        sol = riccati(prob)
        dx, du, lam, K, k = sol["x"], sol["u"], sol["lam"], sol["K"], sol["k"]
        nu = max(nu_min, 2.0 * np.abs(lam).max())
        gd = float(np.sum(prob["q"] * dx) + np.sum(prob["r"] * du))
        J0, D0 = sqp_merit_terms(model, x, u, dx, du, 0.0)
        phi0 = J0 + nu * D0
        slope = gd - nu * D0
        pick = None
        for a in SQP_ALPHAS:
            Ja, Da = sqp_merit_terms(model, x, u, dx, du, a)
            pick = (a, Ja, Da)
            if abs(slope) <= 1e-12 * max(1.0, abs(phi0)) or Ja + nu * Da <= phi0 + 1e-4 * a * slope:
                break
        a, Ja, Da = pick
        scale = max(1.0, np.abs(x).max(), np.abs(u).max())
        x = x + a * dx
        u = u + a * du
        step = a * max(np.abs(dx).max(), np.abs(du).max())
        hist.append(dict(alpha=a, cost=Ja, defect=Da, merit=Ja + nu * Da, step=step, nu=nu))
        if step <= tol * scale and Da <= tol:
            break
    return dict(x=x, u=u, lam=lam, K=K, k=k, hist=hist)
