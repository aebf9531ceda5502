"""Python binding of the matcha C ABI (``include/matcha.h``).

Argument marshalling only: every step of the alignment path runs in the CUDA
kernels of ``_lib/libmatcha.so``.  Device buffers are torch tensors (used for
memory and streams); calls are enqueued on torch's current CUDA stream.
There is no CPU fallback: without the compiled library or a GPU the calls
raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libmatcha.so")

MATCHA_MAX_LEVELS = 16
MATCHA_MAX_L = 64
MATCHA_MAX_P = 32
FP64, FP32, TF32, BF16 = 0, 1, 2, 3

# exported symbols, in include/matcha.h order
SYMBOLS = [
    "matcha_plan_create", "matcha_plan_destroy", "matcha_plan_info", "matcha_plan_table",
    "matcha_workspace_size", "matcha_analyze", "matcha_correlate_coeffs", "matcha_soft_search",
    "matcha_newton_march", "matcha_final_select", "matcha_align", "matcha_host_workspace_size",
    "matcha_align_host", "matcha_status_string", "matcha_last_error",
    "matcha_soft_search_noalloc", "matcha_template_grad_workspace_size", "matcha_template_grad",
    "matcha_plan_device_status", "matcha_plan_autotune", "matcha_plan_set_wait_limit",
    "matcha_transform_volumes", "matcha_shift_search_workspace_size", "matcha_shift_search",
    "matcha_align6d_workspace_size", "matcha_align6d", "matcha_objective",
    "matcha_plan_set_tiles",
]


class MatchaError(RuntimeError):
    pass


class PlanDesc(ctypes.Structure):
    _fields_ = [("box_n", ctypes.c_int), ("n_shells", ctypes.c_int), ("r_max", ctypes.c_double),
                ("L0", ctypes.c_int), ("K_oversample", ctypes.c_int), ("P_max", ctypes.c_int),
                ("M_iter", ctypes.c_int), ("n_levels", ctypes.c_int),
                ("L_sched", ctypes.c_int * MATCHA_MAX_LEVELS), ("precision", ctypes.c_int),
                ("step_tol", ctypes.c_double), ("accept_tol", ctypes.c_double),
                ("refine", ctypes.c_int), ("ball_lambda", ctypes.c_double)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_lm", ctypes.c_int), ("coeff_count", ctypes.c_long),
                ("corr_entries", ctypes.c_long), ("n_pairs", ctypes.c_int),
                ("soft_n", ctypes.c_int), ("real_bytes", ctypes.c_int)]


class TuneReport(ctypes.Structure):
    _fields_ = [("analyze_shells", ctypes.c_int), ("analyze_ms", ctypes.c_float * 4),
                ("tc_ctas_per_sm", ctypes.c_int), ("tc_ms", ctypes.c_float * 2),
                ("soft_kernel", ctypes.c_int), ("soft_ms", ctypes.c_float * 3),
                ("newton_sched", ctypes.c_int), ("newton_ms", ctypes.c_float * 2)]


_lib = None
_vp = ctypes.c_void_p


def lib():
    """Load the compiled library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise MatchaError("libmatcha.so is not built (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        i, l, d, sz = ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_size_t
        sigs = {
            "matcha_plan_create": [ctypes.POINTER(PlanDesc), ctypes.POINTER(_vp)],
            "matcha_plan_destroy": [_vp],
            "matcha_plan_info": [_vp, ctypes.POINTER(PlanInfo)],
            "matcha_plan_table": [_vp, i, _vp, l, ctypes.POINTER(l)],
            "matcha_workspace_size": [_vp, i, ctypes.POINTER(sz)],
            "matcha_analyze": [_vp, _vp, i, _vp, _vp],
            "matcha_correlate_coeffs": [_vp, _vp, _vp, i, i, _vp, _vp],
            "matcha_soft_search": [_vp, _vp, i, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
            "matcha_soft_search_noalloc": [_vp, _vp, i, _vp, _vp, _vp, _vp, _vp, _vp],
            "matcha_newton_march": [_vp, _vp, i, _vp, _vp, _vp, _vp, _vp, _vp],
            "matcha_final_select": [_vp, i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
            "matcha_align": [_vp, _vp, _vp, i, i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, sz, _vp],
            "matcha_host_workspace_size": [_vp, i, i, ctypes.POINTER(sz)],
            "matcha_align_host": [_vp, _vp, _vp, i, i, _vp, _vp, _vp, _vp, _vp, _vp, sz, _vp],
            "matcha_template_grad_workspace_size": [_vp, i, i, ctypes.POINTER(sz)],
            "matcha_plan_device_status": [_vp, ctypes.POINTER(i)],
            "matcha_plan_set_wait_limit": [_vp, l],
            "matcha_plan_autotune": [_vp, _vp, _vp, i, i, _vp, _vp, sz, _vp, ctypes.POINTER(TuneReport)],
            "matcha_template_grad": [_vp, _vp, _vp, i, i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, sz, _vp],
            "matcha_transform_volumes": [i, _vp, i, i, _vp, _vp, i, _vp, _vp],
            "matcha_objective": [_vp, _vp, i, i, i, _vp, _vp, _vp],
            "matcha_plan_set_tiles": [_vp, ctypes.POINTER(TuneReport)],
            "matcha_shift_search_workspace_size": [_vp, i, i, i, ctypes.POINTER(sz)],
            "matcha_shift_search": [_vp, _vp, _vp, i, i, i, _vp, _vp, _vp, _vp, _vp, _vp, sz, _vp],
            "matcha_align6d_workspace_size": [_vp, i, i, i, i, ctypes.POINTER(sz)],
            "matcha_align6d": [_vp, _vp, _vp, i, i, i, i, i, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                               _vp, sz, _vp],
        }
        for name, args in sigs.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.matcha_status_string.argtypes = [ctypes.c_int]
        L.matcha_status_string.restype = ctypes.c_char_p
        L.matcha_last_error.argtypes = []
        L.matcha_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status: int, what: str):
    if status != 0:
        L = lib()
        raise MatchaError("%s: %s (%s)" % (what, L.matcha_status_string(status).decode(),
                                           L.matcha_last_error().decode()))


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise MatchaError("matcha needs a CUDA device; no CPU path exists")
    return torch


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream():
    torch = _torch()
    return torch.cuda.current_stream().cuda_stream


class Plan:
    """A plan: Algorithm 1's parameters plus the device tables (step a0)."""

    def __init__(self, box_n: int, n_shells: int, L0: int, K: int, P: int, M_iter: int,
                 L_sched: Sequence[int], precision: int = FP64, r_max: float = 0.0,
                 step_tol: float = 0.0, accept_tol: float = 0.0, refine: int = 0,
                 ball_lambda: float = 0.0):
        _torch()
        d = PlanDesc()
        d.box_n, d.n_shells, d.r_max = box_n, n_shells, r_max
        d.L0, d.K_oversample, d.P_max, d.M_iter = L0, K, P, M_iter
        d.n_levels = len(L_sched)
        if not 1 <= len(L_sched) <= MATCHA_MAX_LEVELS:
            raise MatchaError("matcha_plan_create: invalid argument (L_sched length)")
        for k, L in enumerate(L_sched):
            d.L_sched[k] = int(L)
        d.precision, d.step_tol, d.accept_tol = precision, step_tol, accept_tol
        d.refine = refine
        d.ball_lambda = ball_lambda
        h = _vp()
        _check(lib().matcha_plan_create(ctypes.byref(d), ctypes.byref(h)), "matcha_plan_create")
        self._h = h
        self.desc = d
        info = PlanInfo()
        _check(lib().matcha_plan_info(h, ctypes.byref(info)), "matcha_plan_info")
        self.info = info
        self.precision = precision
        self.P = P
        self.L_sched = tuple(int(L) for L in L_sched)
        self.L_final = int(L_sched[-1])
        self.box_n = box_n
        self.n_shells = n_shells

    @property
    def handle(self):
        return self._h

    @property
    def real_dtype(self):
        torch = _torch()
        return torch.float64 if self.precision == FP64 else torch.float32

    def close(self):
        if getattr(self, "_h", None):
            lib().matcha_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def table(self, which: int) -> np.ndarray:
        n = ctypes.c_long()
        _check(lib().matcha_plan_table(self._h, which, None, 0, ctypes.byref(n)), "matcha_plan_table")
        out = np.zeros(n.value)
        _check(lib().matcha_plan_table(self._h, which, out.ctypes.data, n.value, ctypes.byref(n)),
               "matcha_plan_table")
        return out

    def autotune(self, particles, templates, ws=None, P_per=None) -> dict:
        """Times the result-invariant tile choices on this batch and keeps the
        fastest in the plan (``matcha_plan_autotune``); returns the report."""
        torch = _torch()
        _need(particles, torch.float32, "particles"); _need(templates, torch.float32, "templates")
        B = particles.shape[0]
        stride = 0 if templates.shape[0] == 1 and B != 1 else 1
        if ws is None:
            ws = alloc_workspace(self, B)
        base = ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        rep = TuneReport()
        if P_per is not None:
            _need(P_per, torch.int32, "P_per")
        _check(lib().matcha_plan_autotune(self.handle, _ptr(particles), _ptr(templates), B, stride,
                                          _ptr(P_per), aligned, ws.numel() - (aligned - base),
                                          _stream(), ctypes.byref(rep)), "matcha_plan_autotune")
        return dict(analyze_shells=rep.analyze_shells, analyze_ms=list(rep.analyze_ms),
                    tc_ctas_per_sm=rep.tc_ctas_per_sm, tc_ms=list(rep.tc_ms),
                    soft_kernel=rep.soft_kernel, soft_ms=list(rep.soft_ms),
                    newton_sched=rep.newton_sched, newton_ms=list(rep.newton_ms))

    def set_tiles(self, analyze_shells: int = 0, tc_ctas_per_sm: int = 0, soft_kernel: int = 0,
                  newton_sched: int = 0):
        """Pins the result-invariant tile choices (0: the built-in rule)."""
        rep = TuneReport()
        rep.analyze_shells, rep.tc_ctas_per_sm, rep.soft_kernel = analyze_shells, tc_ctas_per_sm, soft_kernel
        rep.newton_sched = newton_sched
        _check(lib().matcha_plan_set_tiles(self.handle, ctypes.byref(rep)), "matcha_plan_set_tiles")

    def set_wait_limit(self, polls: int):
        """Polls before a tensor-core wait gives up (-1: built-in; 0: at once, for tests)."""
        _check(lib().matcha_plan_set_wait_limit(self.handle, polls), "matcha_plan_set_wait_limit")

    def device_status(self) -> int:
        """Reads and clears the plan's device status bits (bit 0: a tensor-core
        wait hit its limit)."""
        bits = ctypes.c_int(0)
        lib().matcha_plan_device_status(self.handle, ctypes.byref(bits))
        return bits.value

    def workspace_size(self, B: int) -> int:
        s = ctypes.c_size_t()
        _check(lib().matcha_workspace_size(self._h, B, ctypes.byref(s)), "matcha_workspace_size")
        return s.value

    def host_workspace_size(self, B: int, template_batch_stride: int) -> int:
        s = ctypes.c_size_t()
        _check(lib().matcha_host_workspace_size(self._h, B, template_batch_stride, ctypes.byref(s)),
               "matcha_host_workspace_size")
        return s.value


def _need(t, dtype, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise MatchaError("%s must be a contiguous CUDA tensor of %s" % (name, dtype))


def matcha_analyze(plan: Plan, vols):
    torch = _torch()
    _need(vols, torch.float32, "vols")
    B = vols.shape[0]
    out = torch.empty((B, plan.n_shells, plan.info.n_lm, 2), dtype=plan.real_dtype, device="cuda")
    _check(lib().matcha_analyze(plan.handle, _ptr(vols), B, _ptr(out), _stream()), "matcha_analyze")
    return out


def matcha_correlate_coeffs(plan: Plan, f, h, h_batch_stride: int):
    torch = _torch()
    _need(f, plan.real_dtype, "f"); _need(h, plan.real_dtype, "h")
    B = f.shape[0]
    c = torch.empty((B, plan.info.corr_entries, 2, 2), dtype=plan.real_dtype, device="cuda")
    _check(lib().matcha_correlate_coeffs(plan.handle, _ptr(f), _ptr(h), B, h_batch_stride, _ptr(c),
                                         _stream()), "matcha_correlate_coeffs")
    return c


def matcha_soft_search(plan: Plan, c, P_per=None, grid=None):
    torch = _torch()
    _need(c, plan.real_dtype, "c")
    B = c.shape[0]
    n = plan.info.soft_n
    if grid is None:
        grid = torch.empty((B, n, n, n), dtype=plan.real_dtype, device="cuda")
    P = plan.P
    idx = torch.empty((B, P), dtype=torch.int32, device="cuda")
    euler = torch.empty((B, P, 3), dtype=torch.float64, device="cuda")
    score = torch.empty((B, P), dtype=torch.float64, device="cuda")
    ncand = torch.empty((B,), dtype=torch.int32, device="cuda")
    if P_per is not None:
        _need(P_per, torch.int32, "P_per")
    _check(lib().matcha_soft_search(plan.handle, _ptr(c), B, _ptr(P_per), _ptr(grid), _ptr(idx),
                                    _ptr(euler), _ptr(score), _ptr(ncand), _stream()),
           "matcha_soft_search")
    return dict(grid=grid, idx=idx, euler=euler, score=score, n_cand=ncand)


def matcha_soft_search_noalloc(plan: Plan, c, idx, euler, score, n_cand, P_per=None):
    """matcha_soft_search with the grid in the library's built-in device array.

    For callers that must not allocate device memory: all outputs are passed
    in (preallocated by the caller), and this call allocates nothing.
    """
    torch = _torch()
    _need(c, plan.real_dtype, "c")
    _need(idx, torch.int32, "idx"); _need(euler, torch.float64, "euler")
    _need(score, torch.float64, "score"); _need(n_cand, torch.int32, "n_cand")
    if P_per is not None:
        _need(P_per, torch.int32, "P_per")
    B = c.shape[0]
    _check(lib().matcha_soft_search_noalloc(plan.handle, _ptr(c), B, _ptr(P_per), _ptr(idx),
                                            _ptr(euler), _ptr(score), _ptr(n_cand), _stream()),
           "matcha_soft_search_noalloc")
    return dict(idx=idx, euler=euler, score=score, n_cand=n_cand)


def matcha_newton_march(plan: Plan, c, n_cand, euler, work=None, score=None, flags=None):
    """Refines ``euler`` in place; ``work`` (optional int64 [B][2]) receives
    the recurrence-step counts of derivative and value-only evaluations."""
    torch = _torch()
    _need(c, plan.real_dtype, "c"); _need(n_cand, torch.int32, "n_cand")
    _need(euler, torch.float64, "euler")
    B = c.shape[0]
    if score is None:
        score = torch.full((B, plan.P), float("nan"), dtype=torch.float64, device="cuda")
    if flags is None:
        flags = torch.zeros((B, plan.P), dtype=torch.int32, device="cuda")
    if work is not None:
        _need(work, torch.int64, "work")
    _check(lib().matcha_newton_march(plan.handle, _ptr(c), B, _ptr(n_cand), _ptr(euler), _ptr(score),
                                     _ptr(flags), _ptr(work), _stream()), "matcha_newton_march")
    return dict(euler=euler, score=score, flags=flags, work=work)


def matcha_objective(plan: Plan, c, euler, L=None):
    """C_L, gradient and Hessian at rotations euler [B][Q][3] (float64); returns
    [B][Q][10] (C, C_a, C_b, C_g, C_aa, C_ab, C_ag, C_bb, C_bg, C_gg)."""
    torch = _torch()
    _need(c, plan.real_dtype, "c"); _need(euler, torch.float64, "euler")
    B, Q = euler.shape[0], euler.shape[1]
    out = torch.empty((B, Q, 10), dtype=torch.float64, device="cuda")
    L = plan.L_final if L is None else L
    _check(lib().matcha_objective(plan.handle, _ptr(c), B, L, Q, _ptr(euler), _ptr(out), _stream()),
           "matcha_objective")
    return out


def matcha_final_select(plan: Plan, n_cand, cand_euler, cand_score, cand_flags, P_per=None):
    torch = _torch()
    B = n_cand.shape[0]
    euler = torch.empty((B, 3), dtype=torch.float64, device="cuda")
    R = torch.empty((B, 3, 3), dtype=torch.float64, device="cuda")
    score = torch.empty((B,), dtype=torch.float64, device="cuda")
    best = torch.empty((B,), dtype=torch.int32, device="cuda")
    flags = torch.empty((B,), dtype=torch.int32, device="cuda")
    _check(lib().matcha_final_select(plan.handle, B, _ptr(P_per), _ptr(n_cand), _ptr(cand_euler),
                                     _ptr(cand_score), _ptr(cand_flags), _ptr(euler), _ptr(R),
                                     _ptr(score), _ptr(best), _ptr(flags), _stream()),
           "matcha_final_select")
    return dict(euler=euler, R=R, score=score, best_p=best, flags=flags)


def alloc_workspace(plan: Plan, B: int):
    torch = _torch()
    nbytes = plan.workspace_size(B)
    return torch.empty((nbytes + 256,), dtype=torch.uint8, device="cuda")


def matcha_align(plan: Plan, particles, templates, P_per=None, ws=None, out=None):
    """The whole path on device tensors; ``templates`` holds B volumes or one shared."""
    torch = _torch()
    _need(particles, torch.float32, "particles"); _need(templates, torch.float32, "templates")
    B = particles.shape[0]
    stride = 0 if templates.shape[0] == 1 and B != 1 else 1
    if ws is None:
        ws = alloc_workspace(plan, B)
    if out is None:
        out = dict(euler=torch.empty((B, 3), dtype=torch.float64, device="cuda"),
                   R=torch.empty((B, 3, 3), dtype=torch.float64, device="cuda"),
                   score=torch.empty((B,), dtype=torch.float64, device="cuda"),
                   best_p=torch.empty((B,), dtype=torch.int32, device="cuda"),
                   flags=torch.empty((B,), dtype=torch.int32, device="cuda"))
    base = ws.data_ptr()
    aligned = (base + 255) // 256 * 256
    nbytes = ws.numel() - (aligned - base)
    _check(lib().matcha_align(plan.handle, _ptr(particles), _ptr(templates), B, stride, _ptr(P_per),
                              _ptr(out["euler"]), _ptr(out["R"]), _ptr(out["score"]),
                              _ptr(out["best_p"]), _ptr(out["flags"]), aligned, nbytes, _stream()),
           "matcha_align")
    return out


def _aligned(ws):
    base = ws.data_ptr()
    aligned = (base + 255) // 256 * 256
    return aligned, ws.numel() - (aligned - base)


def matcha_transform_volumes(vols, R=None, shift=None, B=None, precision: int = FP64, out=None):
    """out_b(x) = vol(R_b^T (x - c0) + c0 - shift_b), trilinear (a shared input
    volume when ``vols`` holds one and B > 1)."""
    torch = _torch()
    _need(vols, torch.float32, "vols")
    N = vols.shape[-1]
    B = vols.shape[0] if B is None else B
    stride = 0 if vols.shape[0] == 1 and B != 1 else 1
    if R is not None:
        _need(R, torch.float64, "R")
    if shift is not None:
        _need(shift, torch.float64, "shift")
    if out is None:
        out = torch.empty((B, N, N, N), dtype=torch.float32, device="cuda")
    _check(lib().matcha_transform_volumes(N, _ptr(vols), B, stride, _ptr(R), _ptr(shift), precision,
                                          _ptr(out), _stream()), "matcha_transform_volumes")
    return out


def matcha_shift_search(plan: Plan, particles, rotated, max_shift: int, upsample: int, R=None,
                        ws=None):
    """Translation of each particle against its rotated template (t, tau = R^T t, cc, flags)."""
    torch = _torch()
    _need(particles, torch.float32, "particles"); _need(rotated, torch.float32, "rotated")
    B = particles.shape[0]
    if R is not None:
        _need(R, torch.float64, "R")
    if ws is None:
        n = ctypes.c_size_t()
        _check(lib().matcha_shift_search_workspace_size(plan.handle, B, max_shift, upsample,
                                                        ctypes.byref(n)), "workspace size")
        ws = torch.empty((n.value + 256,), dtype=torch.uint8, device="cuda")
    out = dict(t=torch.empty((B, 3), dtype=torch.float64, device="cuda"),
               tau=torch.empty((B, 3), dtype=torch.float64, device="cuda") if R is not None else None,
               cc=torch.empty((B,), dtype=torch.float64, device="cuda"),
               flags=torch.empty((B,), dtype=torch.int32, device="cuda"))
    a, nb = _aligned(ws)
    _check(lib().matcha_shift_search(plan.handle, _ptr(particles), _ptr(rotated), B, max_shift,
                                     upsample, _ptr(R), _ptr(out["t"]), _ptr(out["tau"]),
                                     _ptr(out["cc"]), _ptr(out["flags"]), a, nb, _stream()),
           "matcha_shift_search")
    return out


def alloc_workspace6d(plan: Plan, B: int, stride: int, max_shift: int, upsample: int):
    torch = _torch()
    n = ctypes.c_size_t()
    _check(lib().matcha_align6d_workspace_size(plan.handle, B, stride, max_shift, upsample,
                                               ctypes.byref(n)), "workspace size")
    return torch.empty((n.value + 256,), dtype=torch.uint8, device="cuda")


def matcha_align6d(plan: Plan, particles, templates, rounds: int, max_shift: int, upsample: int,
                   ws=None, out=None):
    """6-D pose by ``rounds`` rotation-translation alternations (device tensors)."""
    torch = _torch()
    _need(particles, torch.float32, "particles"); _need(templates, torch.float32, "templates")
    B = particles.shape[0]
    stride = 0 if templates.shape[0] == 1 and B != 1 else 1
    if ws is None:
        ws = alloc_workspace6d(plan, B, stride, max_shift, upsample)
    if out is None:
        f64 = dict(dtype=torch.float64, device="cuda")
        out = dict(euler=torch.empty((B, 3), **f64), R=torch.empty((B, 3, 3), **f64),
                   tau=torch.empty((B, 3), **f64), t=torch.empty((B, 3), **f64),
                   score=torch.empty((B,), **f64), cc=torch.empty((B,), **f64),
                   flags=torch.empty((B,), dtype=torch.int32, device="cuda"))
    a, nb = _aligned(ws)
    _check(lib().matcha_align6d(plan.handle, _ptr(particles), _ptr(templates), B, stride, rounds,
                                max_shift, upsample, _ptr(out["euler"]), _ptr(out["R"]),
                                _ptr(out["tau"]), _ptr(out["t"]), _ptr(out["score"]),
                                _ptr(out["cc"]), _ptr(out["flags"]), a, nb, _stream()),
           "matcha_align6d")
    return out


def matcha_align_host(plan: Plan, particles: np.ndarray, templates: np.ndarray, ws=None,
                      out=None):
    """matcha_align on host arrays (float32, [B][N][N][N]); copies are inside the call."""
    torch = _torch()
    B = particles.shape[0]
    stride = 0 if templates.shape[0] == 1 and B != 1 else 1
    if ws is None:
        ws = torch.empty((plan.host_workspace_size(B, stride) + 256,), dtype=torch.uint8,
                         device="cuda")
    base = ws.data_ptr()
    aligned = (base + 255) // 256 * 256
    nbytes = ws.numel() - (aligned - base)
    if out is None:
        out = dict(euler=np.empty((B, 3)), R=np.empty((B, 3, 3)), score=np.empty(B),
                   best_p=np.empty(B, dtype=np.int32), flags=np.empty(B, dtype=np.int32))

    def hp(a):
        if isinstance(a, torch.Tensor):
            return a.data_ptr()
        return a.ctypes.data
    _check(lib().matcha_align_host(plan.handle, hp(particles), hp(templates), B, stride,
                                   hp(out["euler"]), hp(out["R"]), hp(out["score"]),
                                   hp(out["best_p"]), hp(out["flags"]), aligned, nbytes, _stream()),
           "matcha_align_host")
    return out


def align_from_coefs(plan: Plan, f, h, h_batch_stride: int, P_per=None):
    """Steps a3..a7 from SH coefficients (``matcha_analyze`` layout): the
    contraction, the SOFFT search, the Newton march and the final selection.
    Returns the final selection plus ``c`` (the correlation coefficients)."""
    c = matcha_correlate_coeffs(plan, f, h, h_batch_stride)
    soft = matcha_soft_search(plan, c, P_per=P_per)
    nm = matcha_newton_march(plan, c, soft["n_cand"], soft["euler"])
    out = matcha_final_select(plan, soft["n_cand"], nm["euler"], nm["score"], nm["flags"], P_per=P_per)
    out["c"] = c
    return out


def matcha_template_grad(plan: Plan, f, c, euler, weight=None, template_batch_stride: int = 0,
                         voxels: bool = True):
    """Gradient of sum_b weight_b C_{L_J}(theta*_b) with respect to the
    template: ``coef_grad`` [n_t][S][n_lm][2] (plan precision) and
    ``vox_grad`` [n_t][N][N][N] (float64), n_t = 1 for a shared template;
    also ``shift`` [B][4] = (H^{-1} grad C, C) and ``flags`` [B]."""
    torch = _torch()
    _need(f, plan.real_dtype, "f"); _need(c, plan.real_dtype, "c")
    _need(euler, torch.float64, "euler")
    if weight is not None:
        _need(weight, torch.float64, "weight")
    B = f.shape[0]
    nt = B if template_batch_stride else 1
    N = plan.box_n
    coef_grad = torch.empty((nt, plan.n_shells, plan.info.n_lm, 2), dtype=plan.real_dtype, device="cuda")
    vox_grad = torch.empty((nt, N, N, N), dtype=torch.float64, device="cuda") if voxels else None
    shift = torch.empty((B, 4), dtype=torch.float64, device="cuda")
    flags = torch.empty((B,), dtype=torch.int32, device="cuda")
    need = ctypes.c_size_t(0)
    _check(lib().matcha_template_grad_workspace_size(plan.handle, B, template_batch_stride,
                                                     ctypes.byref(need)), "matcha_template_grad")
    ws = torch.empty((need.value + 256,), dtype=torch.uint8, device="cuda")
    base = ws.data_ptr()
    aligned = (base + 255) // 256 * 256
    _check(lib().matcha_template_grad(plan.handle, _ptr(f), _ptr(c), B, template_batch_stride,
                                      _ptr(euler), _ptr(weight), _ptr(coef_grad), _ptr(vox_grad),
                                      _ptr(shift), _ptr(flags), aligned, need.value, _stream()),
           "matcha_template_grad")
    return dict(coef_grad=coef_grad, vox_grad=vox_grad, shift=shift, flags=flags)


def corr_layout(L: int):
    """(m, n, l) of every (pair slot, degree) row of the library's grouped
    correlation layout, in the row order of ``corr_pairs``.

    The pairs (m, n), m >= |n|, of one m are grouped two at a time
    (n = 2j - m and 2j - m + 1, j = 0..m); the second slot of each m's last
    group is empty and is listed with n = m + 1 (its coefficients are zero).
    """
    rows = []
    for m in range(L + 1):
        for j in range(m + 1):
            na = 2 * j - m
            for l in range(m, L + 1):
                rows.append((m, na, l))
                rows.append((m, na + 1, l))
    return np.array(rows, dtype=np.int64)


def corr_pairs(c):
    """Rows (c^l_mn, c^l_nm) of a correlation buffer [..., corr_entries, 2, 2].

    The library interleaves the two partners of a group component by
    component (8 reals per group and degree); this returns the buffer as
    [..., corr_entries, 2, 2] = (row, c_mn | c_nm, re | im) with rows in
    ``corr_layout`` order.  Works on numpy arrays and torch tensors.
    """
    lead, n = tuple(c.shape[:-3]), c.shape[-3]
    g = c.reshape(lead + (n // 2, 4, 2))                 # [group, l][component][slot]
    g = g.transpose(-1, -2) if hasattr(g, "is_cuda") else np.swapaxes(g, -1, -2)
    return g.reshape(lead + (n, 2, 2))


def plan_for_workload(w, precision: int = FP64, **kw) -> Plan:
    """A plan with the parameters of a ``synth.Workload``."""
    return Plan(box_n=w.N, n_shells=w.n_shells, L0=w.L0, K=w.K, P=w.P, M_iter=w.M_iter,
                L_sched=w.L_sched, precision=precision, r_max=w.r_max, **kw)
