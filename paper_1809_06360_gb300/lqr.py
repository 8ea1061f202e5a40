"""Thin ctypes binding of liblqr (include/lqr.h).

Argument marshalling only: every step of the solve runs in the CUDA kernels of
liblqr.so. The functions carry the C names; `Solver` wraps them for torch
tensors (device memory and the current CUDA stream come from PyTorch).
There is no CPU fallback: without the compiled library every call raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int, c_double, c_void_p, c_size_t = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t

LQR_OK = 0
STATUS_NAMES = {0: "LQR_OK", 1: "LQR_ERR_INVALID_ARG", 2: "LQR_ERR_NOT_PD", 3: "LQR_ERR_SEGMENT_INFEASIBLE",
                4: "LQR_ERR_NONFINITE", 5: "LQR_ERR_NO_CONVERGENCE", 6: "LQR_ERR_TIMEOUT", 7: "LQR_ERR_CUDA",
                8: "LQR_ERR_OOM", 9: "LQR_ERR_UNSUPPORTED", 10: "LQR_ERR_CAPACITY"}
NOALLOC_MAX_STAGES = 65536
PRECISION = {"fp64": 0, "fp32": 1, "mixed": 2, "mixed_tf32": 2, "mixed_bf16": 3, "mixed_fp32": 4}
FORM = {"multiplier": 0, "constrained": 1}
LINK = {"auto": 0, "chain": 1, "scan": 2}

PROBLEM_FIELDS = ("A", "B", "c", "Q", "R", "S", "q", "r", "x0")
SOLUTION_FIELDS = ("K", "k", "x", "u", "P", "p", "lam")

# Exported symbols declared in include/lqr.h
EXPORTS = ("lqr_create", "lqr_destroy", "lqr_partition", "lqr_solve", "lqr_solve_host",
           "lqr_segment_summaries", "lqr_report", "lqr_status_string", "lqr_last_launch_count",
           "lqr_profile_enable", "lqr_profile_read", "lqr_solve_batched", "lqr_report_batched",
           "lqr_backward", "lqr_backward_batched", "lqr_kkt_residual_noalloc", "lqr_tc_selftest",
           "lqr_rcp_newton_check", "lqr_segment_policies", "lqr_ls_multipliers",
           "lqr_global_policy_parallel", "lqr_sqp_solve", "lqr_kkt_residual_vectors",
           "lqr_convert_f64_to_f32")
PHASES = ("sweep", "link", "policy", "rollout", "refine")


class lqr_problem(ctypes.Structure):
    _fields_ = [("n", c_int), ("m", c_int), ("T", c_int)] + [(f, c_void_p) for f in PROBLEM_FIELDS]


class lqr_solution(ctypes.Structure):
    _fields_ = [(f, c_void_p) for f in SOLUTION_FIELDS]


class lqr_opts(ctypes.Structure):
    _fields_ = [("prec", c_int), ("num_segments", c_int), ("tol", c_double), ("max_refine", c_int),
                ("debug_checks", c_int), ("form", c_int), ("residual", c_int), ("link", c_int),
                ("spin_limit", ctypes.c_longlong), ("refine_plain", c_int)]


class lqr_report_t(ctypes.Structure):
    _fields_ = [("status", c_int), ("num_segments", c_int), ("refine_iters", c_int), ("bad_stage", c_int),
                ("cost", c_double), ("kkt_residual", c_double), ("kkt_rel", c_double)]


class lqr_nl_model(ctypes.Structure):
    _fields_ = [("n", c_int), ("m", c_int), ("T", c_int), ("A", c_void_p), ("B", c_void_p), ("C", c_void_p),
                ("beta", c_double), ("Q", c_void_p), ("R", c_void_p), ("QT", c_void_p), ("xref", c_void_p),
                ("x0", c_void_p)]


class lqr_sqp_opts(ctypes.Structure):
    _fields_ = [("max_iters", c_int), ("tol", c_double), ("nu_min", c_double), ("sub", lqr_opts)]


class lqr_sqp_report(ctypes.Structure):
    _fields_ = [("iters", c_int), ("converged", c_int), ("cost", c_double), ("defect", c_double),
                ("alpha", c_double), ("step", c_double)]


SQP_HIST = ("alpha", "cost", "defect", "merit", "step", "nu")


class LqrError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s: %s" % (where, STATUS_NAMES.get(status, str(status))))


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load liblqr.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("liblqr.so not found at %s; run paper_1809_06360_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    lib.lqr_create.argtypes = [P(c_void_p), c_int, c_size_t]
    lib.lqr_destroy.argtypes = [c_void_p]
    lib.lqr_partition.argtypes = [c_int, c_int, c_int, c_int, P(c_int)]
    lib.lqr_solve.argtypes = [c_void_p, P(lqr_problem), P(lqr_opts), P(lqr_solution), c_void_p]
    lib.lqr_solve_host.argtypes = [c_void_p, P(lqr_problem), P(lqr_opts), P(lqr_solution), c_void_p]
    lib.lqr_segment_summaries.argtypes = [c_void_p, P(lqr_problem), P(lqr_opts), c_void_p, c_void_p]
    lib.lqr_report.argtypes = [c_void_p, c_void_p, P(lqr_report_t)]
    lib.lqr_status_string.argtypes = [c_int]
    lib.lqr_status_string.restype = ctypes.c_char_p
    lib.lqr_last_launch_count.argtypes = [c_void_p]
    lib.lqr_profile_enable.argtypes = [c_void_p, c_int]
    lib.lqr_profile_read.argtypes = [c_void_p, P(c_double), P(c_int)]
    lib.lqr_solve_batched.argtypes = [c_void_p, c_int, P(lqr_problem), P(lqr_opts), P(lqr_solution), P(c_int),
                                      c_void_p]
    lib.lqr_report_batched.argtypes = [c_void_p, c_void_p, c_int, P(c_int), P(c_double)]
    lib.lqr_kkt_residual_noalloc.argtypes = [P(lqr_problem), P(lqr_solution), c_int, c_void_p, c_void_p]
    lib.lqr_tc_selftest.argtypes = [c_int, P(c_double)]
    lib.lqr_rcp_newton_check.argtypes = [c_void_p, c_void_p, c_int, c_void_p]
    lib.lqr_segment_policies.argtypes = [c_void_p, P(lqr_problem), P(lqr_opts), c_int, c_void_p, c_void_p, c_void_p,
                                         c_void_p, c_void_p]
    lib.lqr_convert_f64_to_f32.argtypes = [c_void_p, c_void_p, ctypes.c_longlong, c_void_p]
    lib.lqr_kkt_residual_vectors.argtypes = [c_void_p, P(lqr_problem), P(lqr_solution), c_void_p, c_void_p,
                                             c_void_p, c_void_p, c_void_p]
    lib.lqr_sqp_solve.argtypes = [c_void_p, P(lqr_nl_model), P(lqr_sqp_opts), c_void_p, c_void_p, c_void_p,
                                  c_void_p, c_void_p, P(lqr_sqp_report), P(c_double), c_void_p]
    lib.lqr_global_policy_parallel.argtypes = [c_void_p, P(lqr_problem), P(lqr_opts), c_void_p, c_void_p,
                                               c_void_p, c_void_p, c_void_p]
    lib.lqr_ls_multipliers.argtypes = [c_void_p, P(lqr_problem), P(lqr_opts), c_void_p, c_void_p, c_void_p,
                                       c_void_p, c_void_p, c_void_p]
    lib.lqr_backward.argtypes = [c_void_p, P(lqr_problem), P(lqr_opts), P(lqr_solution), c_void_p, c_void_p,
                                 P(lqr_problem), c_void_p]
    lib.lqr_backward_batched.argtypes = [c_void_p, c_int, P(lqr_problem), P(lqr_opts), P(lqr_solution),
                                         P(c_void_p), P(c_void_p), P(lqr_problem), c_void_p]
    for name in ("lqr_create", "lqr_destroy", "lqr_partition", "lqr_solve", "lqr_solve_host",
                 "lqr_segment_summaries", "lqr_report", "lqr_last_launch_count", "lqr_profile_enable",
                 "lqr_profile_read", "lqr_solve_batched", "lqr_report_batched", "lqr_backward",
                 "lqr_backward_batched", "lqr_kkt_residual_noalloc", "lqr_tc_selftest",
                 "lqr_rcp_newton_check", "lqr_segment_policies", "lqr_ls_multipliers",
                 "lqr_global_policy_parallel", "lqr_sqp_solve", "lqr_kkt_residual_vectors",
                 "lqr_convert_f64_to_f32"):
        getattr(lib, name).restype = c_int
    _lib = lib
    return lib


def _check(st: int, where: str):
    if st != LQR_OK:
        raise LqrError(st, where)


# --- C-named wrappers ---------------------------------------------------------

def lqr_create(device: int = 0, workspace_hint: int = 0) -> int:
    h = c_void_p()
    _check(load().lqr_create(ctypes.byref(h), device, workspace_hint), "lqr_create")
    return h.value


def lqr_destroy(h: int) -> None:
    _check(load().lqr_destroy(h), "lqr_destroy")


def lqr_partition(n: int, m: int, T: int, K: int) -> list[int]:
    b = (c_int * (K + 1))()
    _check(load().lqr_partition(n, m, T, K, b), "lqr_partition")
    return list(b)


def lqr_solve(h: int, prob: lqr_problem, opts: lqr_opts, sol: lqr_solution, stream: int | None) -> None:
    _check(load().lqr_solve(h, ctypes.byref(prob), ctypes.byref(opts), ctypes.byref(sol), stream or None),
           "lqr_solve")


def lqr_solve_host(h: int, prob: lqr_problem, opts: lqr_opts, sol: lqr_solution, stream: int | None) -> None:
    _check(load().lqr_solve_host(h, ctypes.byref(prob), ctypes.byref(opts), ctypes.byref(sol), stream or None),
           "lqr_solve_host")


def lqr_segment_summaries(h: int, prob: lqr_problem, opts: lqr_opts, summaries_ptr: int, stream: int | None):
    _check(load().lqr_segment_summaries(h, ctypes.byref(prob), ctypes.byref(opts), summaries_ptr, stream or None),
           "lqr_segment_summaries")


def lqr_report(h: int, stream: int | None) -> dict:
    rep = lqr_report_t()
    _check(load().lqr_report(h, stream or None, ctypes.byref(rep)), "lqr_report")
    return dict(status=rep.status, status_name=STATUS_NAMES.get(rep.status, str(rep.status)),
                num_segments=rep.num_segments, refine_iters=rep.refine_iters, bad_stage=rep.bad_stage,
                cost=rep.cost, kkt_residual=rep.kkt_residual, kkt_rel=rep.kkt_rel)


def lqr_status_string(status: int) -> str:
    return load().lqr_status_string(status).decode()


def lqr_last_launch_count(h: int) -> int:
    return load().lqr_last_launch_count(h)


def lqr_solve_batched(h: int, probs, opts: lqr_opts, sols, stream: int | None) -> list[int]:
    n = len(probs)
    parr = (lqr_problem * n)(*probs)
    sarr = (lqr_solution * n)(*sols)
    seg = (c_int * n)()
    _check(load().lqr_solve_batched(h, n, parr, ctypes.byref(opts), sarr, seg, stream or None),
           "lqr_solve_batched")
    return list(seg)


def lqr_report_batched(h: int, stream: int | None, nprob: int):
    st = (c_int * nprob)()
    cost = (c_double * nprob)()
    _check(load().lqr_report_batched(h, stream or None, nprob, st, cost), "lqr_report_batched")
    return list(st), list(cost)


def lqr_kkt_residual_noalloc(prob: lqr_problem, sol: lqr_solution, prec: int, out_ptr: int,
                             stream: int | None) -> None:
    """KKT residual (eta, rel, objective) into a caller-owned device buffer of 3 doubles; no allocation."""
    _check(load().lqr_kkt_residual_noalloc(ctypes.byref(prob), ctypes.byref(sol), prec, out_ptr, stream or None),
           "lqr_kkt_residual_noalloc")


def lqr_backward(h: int, prob: lqr_problem, opts: lqr_opts, sol: lqr_solution, gx: int | None, gu: int | None,
                 grads: lqr_problem, stream: int | None) -> None:
    _check(load().lqr_backward(h, ctypes.byref(prob), ctypes.byref(opts), ctypes.byref(sol), gx, gu,
                               ctypes.byref(grads), stream or None), "lqr_backward")


def lqr_backward_batched(h: int, probs, opts: lqr_opts, sols, gxs, gus, grads, stream: int | None) -> None:
    n = len(probs)
    parr = (lqr_problem * n)(*probs)
    sarr = (lqr_solution * n)(*sols)
    garr = (lqr_problem * n)(*grads)
    gx = (c_void_p * n)(*gxs)
    gu = (c_void_p * n)(*gus)
    _check(load().lqr_backward_batched(h, n, parr, ctypes.byref(opts), sarr, gx, gu, garr, stream or None),
           "lqr_backward_batched")


def lqr_tc_selftest(device: int = 0) -> list[float]:
    """The tensor-core product unit against CUDA-core products (include/lqr.h)."""
    errs = (c_double * 5)()
    _check(load().lqr_tc_selftest(device, errs), "lqr_tc_selftest")
    return [errs[i] for i in range(5)]


def lqr_rcp_newton_check(d_ptr: int, y_ptr: int, count: int, stream: int | None) -> None:
    _check(load().lqr_rcp_newton_check(d_ptr, y_ptr, count, stream or None), "lqr_rcp_newton_check")


def lqr_convert_f64_to_f32(src: int, dst: int, count: int, stream: int | None = None) -> None:
    _check(load().lqr_convert_f64_to_f32(src, dst, count, stream), "lqr_convert_f64_to_f32")


def lqr_profile_enable(h: int, enable: bool) -> None:
    _check(load().lqr_profile_enable(h, 1 if enable else 0), "lqr_profile_enable")


def lqr_profile_read(h: int) -> tuple[dict, int]:
    ms = (c_double * len(PHASES))()
    n = c_int()
    _check(load().lqr_profile_read(h, ms, ctypes.byref(n)), "lqr_profile_read")
    return {k: ms[i] for i, k in enumerate(PHASES)}, n.value


# --- torch convenience -------------------------------------------------------------

def _torch():
    import torch
    return torch


class Solver:
    """One liblqr handle bound to a CUDA device; problems are dicts of torch tensors."""

    def __init__(self, device: int = 0, workspace_hint: int = 0):
        self.device = device
        self.h = lqr_create(device, workspace_hint)

    def last_launch_count(self) -> int:
        """Kernels launched by the last solve on this handle."""
        return lqr_last_launch_count(self.h)

    def close(self):
        if self.h:
            lqr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _dims(prob):
        T, n, m = prob["B"].shape
        return int(n), int(m), int(T)

    @staticmethod
    def make_problem_struct(prob, ptr) -> lqr_problem:
        n, m, T = Solver._dims(prob)
        p = lqr_problem(n=n, m=m, T=T)
        for f in PROBLEM_FIELDS:
            v = prob.get(f)
            setattr(p, f, ptr(v) if v is not None else None)
        return p

    def _stream(self, stream):
        torch = _torch()
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        return stream.cuda_stream

    def alloc_solution(self, prob, want=("K", "k", "x", "u", "lam")):
        torch = _torch()
        n, m, T = self._dims(prob)
        dt = prob["A"].dtype
        dev = prob["A"].device
        shapes = dict(K=(T, m, n), k=(T, m), x=(T + 1, n), u=(T, m), P=(T + 1, n, n), p=(T + 1, n),
                      lam=(T + 1, n))
        out = {k: torch.empty(shapes[k], dtype=dt, device=dev) for k in want}
        if "P" in out and "p" not in out:
            out["p"] = torch.empty(shapes["p"], dtype=dt, device=dev)
        return out

    def solve(self, prob, num_segments=0, prec="fp64", out=None, want=("K", "k", "x", "u", "lam"),
              stream=None, tol=1e-8, max_refine=0, form="multiplier", residual=False, link="auto", spin_limit=0,
              refine_plain=False):
        """Enqueue a solve on `stream` (torch stream; default current). Returns the output tensors."""
        if out is None:
            out = self.alloc_solution(prob, want)
        ptr = lambda t: t.data_ptr()
        p = self.make_problem_struct(prob, ptr)
        s = lqr_solution(**{f: (out[f].data_ptr() if f in out else None) for f in SOLUTION_FIELDS})
        o = lqr_opts(prec=PRECISION[prec], num_segments=num_segments, tol=tol, max_refine=max_refine,
                     debug_checks=0, form=FORM[form], residual=1 if residual else 0, link=LINK[link],
                     spin_limit=spin_limit, refine_plain=1 if refine_plain else 0)
        lqr_solve(self.h, p, o, s, self._stream(stream))
        return out

    def report(self, stream=None) -> dict:
        return lqr_report(self.h, self._stream(stream))

    def solve_batched(self, probs, prec="fp32", num_segments=0, outs=None, want=("K", "k", "x", "u", "lam"),
                      stream=None):
        """Solve a list of problems (dicts of device tensors, uneven n, m, T) in one batched call.
        Returns (outputs per problem, segment count per problem)."""
        if outs is None:
            outs = [self.alloc_solution(p, want) for p in probs]
        ptr = lambda t: t.data_ptr()
        ps = [self.make_problem_struct(p, ptr) for p in probs]
        ss = [lqr_solution(**{f: (o[f].data_ptr() if f in o else None) for f in SOLUTION_FIELDS}) for o in outs]
        o = lqr_opts(prec=PRECISION[prec], num_segments=num_segments, tol=0.0, max_refine=0, debug_checks=0,
                     form=0, residual=0)
        seg = lqr_solve_batched(self.h, ps, o, ss, self._stream(stream))
        return outs, seg

    def report_batched(self, nprob, stream=None):
        return lqr_report_batched(self.h, self._stream(stream), nprob)

    @staticmethod
    def _alloc_grads(prob):
        torch = _torch()
        return {k: torch.empty_like(prob[k]) if prob.get(k) is not None else
                torch.zeros((prob["B"].shape[0], prob["B"].shape[2], prob["B"].shape[1]), dtype=prob["A"].dtype,
                            device=prob["A"].device) for k in PROBLEM_FIELDS}

    def backward(self, prob, sol, grad_x=None, grad_u=None, num_segments=0, prec="fp64", stream=None,
                 form="multiplier"):
        """dL/d(problem data) for upstream gradients dL/dx, dL/du (device tensors or None)."""
        grads = self._alloc_grads(prob)
        ptr = lambda t: t.data_ptr()
        p = self.make_problem_struct(prob, ptr)
        g = self.make_problem_struct(grads, ptr)
        so = lqr_solution(**{f: (sol[f].data_ptr() if f in sol else None) for f in SOLUTION_FIELDS})
        o = lqr_opts(prec=PRECISION[prec], num_segments=num_segments, tol=0.0, max_refine=0, debug_checks=0,
                     form=FORM[form], residual=0)
        lqr_backward(self.h, p, o, so, grad_x.data_ptr() if grad_x is not None else None,
                     grad_u.data_ptr() if grad_u is not None else None, g, self._stream(stream))
        return grads

    def backward_batched(self, probs, sols, grads_x, grads_u, prec="fp32", num_segments=0, stream=None):
        ptr = lambda t: t.data_ptr()
        grads = [self._alloc_grads(p) for p in probs]
        ps = [self.make_problem_struct(p, ptr) for p in probs]
        gs = [self.make_problem_struct(g, ptr) for g in grads]
        ss = [lqr_solution(**{f: (s[f].data_ptr() if f in s else None) for f in SOLUTION_FIELDS}) for s in sols]
        o = lqr_opts(prec=PRECISION[prec], num_segments=num_segments, tol=0.0, max_refine=0, debug_checks=0,
                     form=0, residual=0)
        gx = [t.data_ptr() if t is not None else None for t in grads_x]
        gu = [t.data_ptr() if t is not None else None for t in grads_u]
        lqr_backward_batched(self.h, ps, o, ss, gx, gu, gs, self._stream(stream))
        return grads

    def segment_policies(self, prob, num_segments, smooth=False, stream=None):
        """The paper's segment policies (lqr_segment_policies): dict Kx, Kz, k1, z (FP64 device tensors)."""
        torch = _torch()
        n, m, T = self._dims(prob)
        dev = prob["A"].device
        out = dict(Kx=torch.empty((T, m, n), dtype=torch.float64, device=dev),
                   Kz=torch.empty((T, m, n), dtype=torch.float64, device=dev),
                   k1=torch.empty((T, m), dtype=torch.float64, device=dev),
                   z=torch.empty((num_segments + 1, n), dtype=torch.float64, device=dev))
        p = self.make_problem_struct(prob, lambda t: t.data_ptr())
        o = lqr_opts(prec=PRECISION["fp64"], num_segments=num_segments, tol=0.0, max_refine=0, debug_checks=0,
                     form=FORM["constrained"], residual=0)
        _check(load().lqr_segment_policies(self.h, ctypes.byref(p), ctypes.byref(o), 1 if smooth else 0,
                                           out["Kx"].data_ptr(), out["Kz"].data_ptr(), out["k1"].data_ptr(),
                                           out["z"].data_ptr(), self._stream(stream) or None),
               "lqr_segment_policies")
        return out

    def kkt_residual_vectors(self, prob, sol, stream=None):
        """The correction solve's right-hand side at sol (lqr_kkt_residual_vectors):
        dict q = -rx ((T+1) x n), r = -ru, c = rd, x0 = r0 (FP64 device tensors)."""
        torch = _torch()
        n, m, T = self._dims(prob)
        dev = prob["A"].device
        out = dict(q=torch.empty((T + 1, n), dtype=torch.float64, device=dev),
                   r=torch.empty((T, m), dtype=torch.float64, device=dev),
                   c=torch.empty((T, n), dtype=torch.float64, device=dev),
                   x0=torch.empty((n,), dtype=torch.float64, device=dev))
        p = self.make_problem_struct(prob, lambda t: t.data_ptr())
        s = lqr_solution(**{f: (sol[f].data_ptr() if f in sol else None) for f in SOLUTION_FIELDS})
        _check(load().lqr_kkt_residual_vectors(self.h, ctypes.byref(p), ctypes.byref(s), out["q"].data_ptr(),
                                               out["r"].data_ptr(), out["c"].data_ptr(), out["x0"].data_ptr(),
                                               self._stream(stream) or None),
               "lqr_kkt_residual_vectors")
        return out

    def sqp_solve(self, model, x, u, max_iters=30, tol=1e-10, nu_min=1.0, num_segments=0, prec="fp64",
                  max_refine=0, sub_tol=1e-10, stream=None):
        """Trajectory-optimisation outer loop (lqr_sqp_solve). model: dict of FP64
        device tensors A, B, C, Q, R, QT, xref, x0 and float beta; x, u: FP64
        device tensors, updated in place. Returns dict x, u, lam, K, k, report
        (dict), hist (list of per-iteration dicts)."""
        torch = _torch()
        n, m = model["B"].shape
        T = u.shape[0]
        dev = x.device
        lam = torch.empty((T + 1, n), dtype=torch.float64, device=dev)
        K = torch.empty((T, m, n), dtype=torch.float64, device=dev)
        k = torch.empty((T, m), dtype=torch.float64, device=dev)
        md = lqr_nl_model(n=n, m=m, T=T, A=model["A"].data_ptr(), B=model["B"].data_ptr(), C=model["C"].data_ptr(),
                          beta=float(model["beta"]), Q=model["Q"].data_ptr(), R=model["R"].data_ptr(),
                          QT=model["QT"].data_ptr(), xref=model["xref"].data_ptr(), x0=model["x0"].data_ptr())
        sub = lqr_opts(prec=PRECISION[prec], num_segments=num_segments, tol=sub_tol, max_refine=max_refine,
                       debug_checks=0, form=FORM["multiplier"], residual=0)
        so = lqr_sqp_opts(max_iters=max_iters, tol=tol, nu_min=nu_min, sub=sub)
        rep = lqr_sqp_report()
        hist = (c_double * (len(SQP_HIST) * max_iters))()
        _check(load().lqr_sqp_solve(self.h, ctypes.byref(md), ctypes.byref(so), x.data_ptr(), u.data_ptr(),
                                    lam.data_ptr(), K.data_ptr(), k.data_ptr(), ctypes.byref(rep), hist,
                                    self._stream(stream) or None),
               "lqr_sqp_solve")
        report = {f: getattr(rep, f) for f, _ in lqr_sqp_report._fields_}
        hl = [dict(zip(SQP_HIST, hist[len(SQP_HIST) * i:len(SQP_HIST) * (i + 1)])) for i in range(rep.iters)]
        return dict(x=x, u=u, lam=lam, K=K, k=k, report=report, hist=hl)

    def global_policy_parallel(self, prob, num_segments, want_P=True, stream=None):
        """Per-stage reconstruction of the global policy (lqr_global_policy_parallel):
        dict K, k (and P, p) as FP64 device tensors."""
        torch = _torch()
        n, m, T = self._dims(prob)
        dev = prob["A"].device
        out = dict(K=torch.empty((T, m, n), dtype=torch.float64, device=dev),
                   k=torch.empty((T, m), dtype=torch.float64, device=dev))
        if want_P:
            out["P"] = torch.empty((T + 1, n, n), dtype=torch.float64, device=dev)
            out["p"] = torch.empty((T + 1, n), dtype=torch.float64, device=dev)
        p = self.make_problem_struct(prob, lambda t: t.data_ptr())
        o = lqr_opts(prec=PRECISION["fp64"], num_segments=num_segments, tol=0.0, max_refine=0, debug_checks=0,
                     form=FORM["constrained"], residual=0)
        _check(load().lqr_global_policy_parallel(self.h, ctypes.byref(p), ctypes.byref(o), out["K"].data_ptr(),
                                                 out["k"].data_ptr(),
                                                 out["P"].data_ptr() if want_P else None,
                                                 out["p"].data_ptr() if want_P else None,
                                                 self._stream(stream) or None),
               "lqr_global_policy_parallel")
        return out

    def ls_multipliers(self, prob, x, u, num_segments, stream=None):
        """Segment multipliers from the least-squares system (lqr_ls_multipliers):
        dict lam, lam_end, mu (FP64 device tensors)."""
        torch = _torch()
        n, m, T = self._dims(prob)
        dev = prob["A"].device
        K = max(num_segments, 1)
        out = dict(lam=torch.empty((T + 1, n), dtype=torch.float64, device=dev),
                   lam_end=torch.empty((max(K - 1, 1), n), dtype=torch.float64, device=dev),
                   mu=torch.empty((max(K - 1, 1), n), dtype=torch.float64, device=dev))
        p = self.make_problem_struct(prob, lambda t: t.data_ptr())
        o = lqr_opts(prec=PRECISION["fp64"], num_segments=num_segments, tol=0.0, max_refine=0, debug_checks=0,
                     form=FORM["multiplier"], residual=0)
        _check(load().lqr_ls_multipliers(self.h, ctypes.byref(p), ctypes.byref(o), x.data_ptr(), u.data_ptr(),
                                         out["lam"].data_ptr(), out["lam_end"].data_ptr(), out["mu"].data_ptr(),
                                         self._stream(stream) or None),
               "lqr_ls_multipliers")
        if K == 1:
            out["lam_end"] = out["lam_end"][:0]
            out["mu"] = out["mu"][:0]
        return out

    def segment_summaries(self, prob, num_segments, prec="fp64", stream=None, form="multiplier"):
        torch = _torch()
        n, m, T = self._dims(prob)
        buf = torch.empty((num_segments, 3 * n * n + 2 * n), dtype=torch.float64, device=prob["A"].device)
        p = self.make_problem_struct(prob, lambda t: t.data_ptr())
        o = lqr_opts(prec=PRECISION[prec], num_segments=num_segments, tol=0.0, max_refine=0, debug_checks=0,
                     form=FORM[form])
        lqr_segment_summaries(self.h, p, o, buf.data_ptr(), self._stream(stream))
        return buf

    def solve_host(self, prob_np, num_segments=0, prec="fp64", out_np=None, want=("K", "k", "x", "u"),
                   stream=None, form="multiplier", tol=1e-8, max_refine=0, residual=False, link="auto"):
        """Host-memory solve (numpy arrays, ideally pinned): copies in, solves, copies out, synchronises."""
        import numpy as np
        n, m, T = self._dims(prob_np)
        if out_np is None:
            dt = prob_np["A"].dtype
            shapes = dict(K=(T, m, n), k=(T, m), x=(T + 1, n), u=(T, m), P=(T + 1, n, n), p=(T + 1, n),
                          lam=(T + 1, n))
            out_np = {k: np.empty(shapes[k], dtype=dt) for k in want}
        p = self.make_problem_struct(prob_np, lambda a: a.ctypes.data)
        s = lqr_solution(**{f: (out_np[f].ctypes.data if f in out_np else None) for f in SOLUTION_FIELDS})
        o = lqr_opts(prec=PRECISION[prec], num_segments=num_segments, tol=tol, max_refine=max_refine,
                     debug_checks=0, form=FORM[form], residual=1 if residual else 0, link=LINK[link])
        lqr_solve_host(self.h, p, o, s, self._stream(stream))
        return out_np
