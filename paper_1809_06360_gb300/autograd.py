"""torch.autograd.Function over the segment-parallel LQR solve.

Forward: the optimal trajectory (x, u) of the problem given by the data
tensors. Backward: the adjoint segment-parallel Riccati solve of liblqr
(lqr_backward / lqr_backward_batched) returns the gradient with respect to
every datum A, B, c, Q, R, S, q, r, x0. All arithmetic runs in liblqr's CUDA
kernels; this module only marshals tensors.
"""
from __future__ import annotations

import torch

from .lqr import Solver

FIELDS = ("A", "B", "c", "Q", "R", "S", "q", "r", "x0")
_solvers: dict[int, Solver] = {}


def _solver(device: torch.device) -> Solver:
    idx = device.index if device.index is not None else torch.cuda.current_device()
    if idx not in _solvers:
        _solvers[idx] = Solver(idx)
    return _solvers[idx]


class LQRFunction(torch.autograd.Function):
    """x, u = LQRFunction.apply(A, B, c, Q, R, S, q, r, x0, num_segments, prec) for one problem."""

    @staticmethod
    def forward(ctx, A, B, c, Q, R, S, q, r, x0, num_segments=0, prec="fp64"):
        prob = dict(A=A.contiguous(), B=B.contiguous(), c=c.contiguous(), Q=Q.contiguous(), R=R.contiguous(),
                    S=S.contiguous(), q=q.contiguous(), r=r.contiguous(), x0=x0.contiguous())
        s = _solver(A.device)
        out = s.solve(prob, num_segments=num_segments, prec=prec, want=("K", "k", "x", "u", "lam"))
        ctx.save_for_backward(*[prob[k] for k in FIELDS], out["x"], out["u"], out["lam"])
        ctx.num_segments = num_segments
        ctx.prec = prec
        return out["x"], out["u"]

    @staticmethod
    def backward(ctx, gx, gu):
        saved = ctx.saved_tensors
        prob = dict(zip(FIELDS, saved[:9]))
        sol = dict(x=saved[9], u=saved[10], lam=saved[11])
        s = _solver(prob["A"].device)
        g = s.backward(prob, sol, gx.contiguous() if gx is not None else None,
                       gu.contiguous() if gu is not None else None, num_segments=ctx.num_segments, prec=ctx.prec)
        return tuple(g[k] for k in FIELDS) + (None, None)


class LQRBatchFunction(torch.autograd.Function):
    """x, u = LQRBatchFunction.apply(A, B, c, Q, R, S, q, r, x0, num_segments, prec) for a stack of
    equal-shape problems (leading batch dimension), solved as one batched call."""

    @staticmethod
    def forward(ctx, A, B, c, Q, R, S, q, r, x0, num_segments=0, prec="fp32"):
        data = [t.contiguous() for t in (A, B, c, Q, R, S, q, r, x0)]
        nb = A.shape[0]
        probs = [dict(zip(FIELDS, [t[i] for t in data])) for i in range(nb)]
        s = _solver(A.device)
        outs, _ = s.solve_batched(probs, prec=prec, num_segments=num_segments, want=("K", "k", "x", "u", "lam"))
        x = torch.stack([o["x"] for o in outs])
        u = torch.stack([o["u"] for o in outs])
        lam = torch.stack([o["lam"] for o in outs])
        ctx.save_for_backward(*data, x, u, lam)
        ctx.num_segments = num_segments
        ctx.prec = prec
        return x, u

    @staticmethod
    def backward(ctx, gx, gu):
        saved = ctx.saved_tensors
        data = saved[:9]
        x, u, lam = saved[9:12]
        nb = data[0].shape[0]
        probs = [dict(zip(FIELDS, [t[i] for t in data])) for i in range(nb)]
        sols = [dict(x=x[i], u=u[i], lam=lam[i]) for i in range(nb)]
        gx = gx.contiguous() if gx is not None else None
        gu = gu.contiguous() if gu is not None else None
        s = _solver(data[0].device)
        grads = s.backward_batched(probs, sols, [gx[i] if gx is not None else None for i in range(nb)],
                                   [gu[i] if gu is not None else None for i in range(nb)], prec=ctx.prec,
                                   num_segments=ctx.num_segments)
        return tuple(torch.stack([g[k] for g in grads]) for k in FIELDS) + (None, None)


def lqr(A, B, c, Q, R, S, q, r, x0, num_segments=0, prec="fp64"):
    """Differentiable solve of one problem: returns (x, u)."""
    return LQRFunction.apply(A, B, c, Q, R, S, q, r, x0, num_segments, prec)


def lqr_batch(A, B, c, Q, R, S, q, r, x0, num_segments=0, prec="fp32"):
    """Differentiable batched solve of stacked equal-shape problems: returns (x, u)."""
    return LQRBatchFunction.apply(A, B, c, Q, R, S, q, r, x0, num_segments, prec)
