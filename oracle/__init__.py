"""FP64 CPU oracle (ctypes binding of ``oracle/*.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg may use this module; the CUDA library never does.
Every function follows the paper's definitions in double precision; see the
C sources for the citation of each step.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)


class OrcParams(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("S", ctypes.c_int), ("L0", ctypes.c_int),
                ("K", ctypes.c_int), ("P", ctypes.c_int), ("M_iter", ctypes.c_int),
                ("n_levels", ctypes.c_int), ("L_sched", ctypes.c_int * 16),
                ("r_max", ctypes.c_double), ("step_tol", ctypes.c_double),
                ("accept_tol", ctypes.c_double), ("refine", ctypes.c_int)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_c_offset.restype = ctypes.c_long
        L.orc_c_size.restype = ctypes.c_long
        L.orc_c_index.restype = ctypes.c_long
        L.orc_plm_bar.restype = ctypes.c_double
        L.orc_plm_bar.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
        L.orc_trilinear.restype = ctypes.c_double
        L.orc_trilinear.argtypes = [_fp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_wigner_d.argtypes = [ctypes.c_int, ctypes.c_double, _dp]
        L.orc_wigner_d_finite_sum.restype = ctypes.c_double
        L.orc_wigner_d_finite_sum.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double]
        L.orc_wigner_d_derivs.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp]
        L.orc_euler_to_matrix.argtypes = [ctypes.c_double] * 3 + [_dp]
        L.orc_rotation_angle.restype = ctypes.c_double
        L.orc_objective.restype = ctypes.c_double
        L.orc_objective.argtypes = [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, _dp, _dp, _dp]
        L.orc_sh_synthesize.argtypes = [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]
        L.orc_soft_angles.argtypes = [ctypes.c_int, ctypes.c_long, _dp]
        L.orc_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _f(a):
    return a.ctypes.data_as(_fp)


def _i(a):
    return a.ctypes.data_as(_ip)


# ---- layouts --------------------------------------------------------------
def c_size(L):
    return (L + 1) * (2 * L + 1) * (2 * L + 3) // 3


def c_index(l, m, n):
    return l * (2 * l - 1) * (2 * l + 1) // 3 + (m + l) * (2 * l + 1) + (n + l)


def lm_size(L):
    return (L + 1) * (L + 2) // 2


def lm_index(l, m):
    return l * (l + 1) // 2 + m


# ---- quadrature -------------------------------------------------------------
def gauss_legendre(n):
    x = np.zeros(n); w = np.zeros(n)
    lib().orc_gauss_legendre(ctypes.c_int(n), _d(x), _d(w))
    return x, w


def radial_nodes(S, R):
    r = np.zeros(S); w = np.zeros(S)
    lib().orc_radial_nodes(ctypes.c_int(S), ctypes.c_double(R), _d(r), _d(w))
    return r, w


def plm_bar(l, m, x):
    return lib().orc_plm_bar(l, m, float(x))


# ---- sampling / analysis ------------------------------------------------------
def trilinear(vol, px, py, pz):
    v = np.ascontiguousarray(vol, dtype=np.float32)
    return lib().orc_trilinear(_f(v), v.shape[-1], float(px), float(py), float(pz))


def sample_shells(vol, S, R, L):
    v = np.ascontiguousarray(vol, dtype=np.float32)
    out = np.zeros((S, L + 1, 2 * L + 2))
    lib().orc_sample_shells(_f(v), ctypes.c_int(v.shape[-1]), ctypes.c_int(S),
                            ctypes.c_double(R), ctypes.c_int(L), _d(out))
    return out


def sh_analyze_shell(samples, L):
    s = np.ascontiguousarray(samples, dtype=np.float64)
    out = np.zeros(2 * lm_size(L))
    lib().orc_sh_analyze_shell(_d(s), ctypes.c_int(L), _d(out))
    return out[0::2] + 1j * out[1::2]


def sh_synthesize(coef, L, theta, phi):
    c = np.zeros(2 * lm_size(L))
    c[0::2] = np.real(coef); c[1::2] = np.imag(coef)
    out = np.zeros(1)
    lib().orc_sh_synthesize(_d(c), L, float(theta), float(phi), _d(out))
    return out[0]


def analyze_volume(vol, S, R, L):
    """Complex SH coefficients [S][lm] of one volume."""
    v = np.ascontiguousarray(vol, dtype=np.float32)
    out = np.zeros(2 * S * lm_size(L))
    lib().orc_analyze_volume(_f(v), ctypes.c_int(v.shape[-1]), ctypes.c_int(S),
                             ctypes.c_double(R), ctypes.c_int(L), _d(out))
    return (out[0::2] + 1j * out[1::2]).reshape(S, lm_size(L))


def _split(z):
    a = np.zeros(2 * z.size)
    a[0::2] = np.real(z).ravel(); a[1::2] = np.imag(z).ravel()
    return a


def correlate(f, h, S, R, L):
    """c^l_mn (complex, full layout, length T(L)) from coefficient arrays [S][lm]."""
    fa, ha = _split(np.asarray(f)), _split(np.asarray(h))
    out = np.zeros(2 * c_size(L))
    lib().orc_correlate(_d(fa), _d(ha), ctypes.c_int(S), ctypes.c_double(R), ctypes.c_int(L), _d(out))
    return out[0::2] + 1j * out[1::2]


# ---- Wigner ---------------------------------------------------------------
def wigner_d(L, beta):
    out = np.zeros(c_size(L))
    lib().orc_wigner_d(L, float(beta), _d(out))
    return out


def wigner_d_matrix(l, beta, full=None):
    d = wigner_d(l, beta) if full is None else full
    o = c_index(l, -l, -l)
    return d[o:o + (2 * l + 1) ** 2].reshape(2 * l + 1, 2 * l + 1)


def wigner_d_finite_sum(l, m, n, beta):
    return lib().orc_wigner_d_finite_sum(l, m, n, float(beta))


def wigner_d_derivs(L, beta):
    d = np.zeros(c_size(L)); d1 = np.zeros_like(d); d2 = np.zeros_like(d)
    lib().orc_wigner_d_derivs(L, float(beta), _d(d), _d(d1), _d(d2))
    return d, d1, d2


def euler_to_matrix(a, b, g):
    R = np.zeros(9)
    lib().orc_euler_to_matrix(float(a), float(b), float(g), _d(R))
    return R.reshape(3, 3)


def matrix_to_euler(R):
    Rm = np.ascontiguousarray(R, dtype=np.float64).reshape(9)
    out = np.zeros(3)
    lib().orc_matrix_to_euler(_d(Rm), _d(out))
    return out


def rotation_angle(R1, R2):
    a = np.ascontiguousarray(R1, dtype=np.float64).reshape(9)
    b = np.ascontiguousarray(R2, dtype=np.float64).reshape(9)
    return lib().orc_rotation_angle(_d(a), _d(b))


def wigner_D(l, a, b, g):
    """Full D^l(a,b,g) matrix, rows m, columns n (both -l..l)."""
    d = wigner_d_matrix(l, b)
    m = np.arange(-l, l + 1)
    return np.exp(-1j * m[:, None] * a) * d * np.exp(-1j * m[None, :] * g)


# ---- objective --------------------------------------------------------------
def objective(c, L, a, b, g, derivs=False):
    ca = _split(np.asarray(c))
    grad = np.zeros(3); hess = np.zeros(9); im = np.zeros(1)
    C = lib().orc_objective(_d(ca), L, float(a), float(b), float(g),
                            _d(grad) if derivs else None, _d(hess) if derivs else None, _d(im))
    if derivs:
        return C, grad, hess.reshape(3, 3), im[0]
    return C, im[0]


# ---- SOFFT ----------------------------------------------------------------
def soft_n(L0, K):
    return 2 * K * (L0 + 1)


def soft_grid(c, L0, K):
    n = soft_n(L0, K)
    ca = _split(np.asarray(c))
    out = np.zeros(n ** 3)
    lib().orc_soft_grid(_d(ca), ctypes.c_int(L0), ctypes.c_int(K), _d(out))
    return out


def soft_angles(n, idx):
    out = np.zeros(3)
    lib().orc_soft_angles(n, idx, _d(out))
    return out


def local_maxima_topk(grid, n, P):
    g = np.ascontiguousarray(grid, dtype=np.float64)
    idx = np.zeros(P, dtype=np.int32); sc = np.zeros(P)
    k = lib().orc_local_maxima_topk(_d(g), ctypes.c_int(n), ctypes.c_int(P), _i(idx), _d(sc))
    return idx[:k], sc[:k]


# ---- Newton ---------------------------------------------------------------
def wrap(abg):
    a = np.array(abg, dtype=np.float64)
    lib().orc_wrap(_d(a))
    return a


def newton_direction(g, H, L):
    ga = np.ascontiguousarray(g, dtype=np.float64); Ha = np.ascontiguousarray(H, dtype=np.float64).reshape(9)
    d = np.zeros(3)
    fl = lib().orc_newton_direction(_d(ga), _d(Ha), ctypes.c_int(L), _d(d))
    return d, fl


def newton_march(c, L_sched, M_iter, abg, step_tol=1e-9, accept_tol=1e-11, method=0):
    """method 0: Newton steps; 1: gradient steps."""
    ca = _split(np.asarray(c))
    Ls = np.ascontiguousarray(L_sched, dtype=np.int32)
    x = np.array(abg, dtype=np.float64)
    sc = np.zeros(1)
    fl = lib().orc_refine_march(_d(ca), _i(Ls), ctypes.c_int(len(Ls)), ctypes.c_int(M_iter),
                                ctypes.c_double(step_tol), ctypes.c_double(accept_tol),
                                ctypes.c_int(method), _d(x), _d(sc))
    return x, sc[0], fl


def gradient_direction(g, H, L):
    ga = np.ascontiguousarray(g, dtype=np.float64); Ha = np.ascontiguousarray(H, dtype=np.float64).reshape(9)
    d = np.zeros(3)
    lib().orc_gradient_direction(_d(ga), _d(Ha), ctypes.c_int(L), _d(d))
    return d


# ---- full path ----------------------------------------------------------------
def max_threads():
    return lib().orc_max_threads()


def make_params(N, S, r_max, L0, K, P, M_iter, L_sched, step_tol=1e-9, accept_tol=1e-11,
                refine=0):
    p = OrcParams()
    p.refine = refine
    p.N, p.S, p.L0, p.K, p.P, p.M_iter = N, S, L0, K, P, M_iter
    p.n_levels = len(L_sched)
    for i, L in enumerate(L_sched):
        p.L_sched[i] = L
    p.r_max = r_max
    p.step_tol = step_tol
    p.accept_tol = accept_tol
    return p


def align_batch(particles, templates, *, S, r_max, L0, K, P, M_iter, L_sched,
                P_per=None, n_threads=0, step_tol=1e-9, accept_tol=1e-11, refine=0):
    """Run Algorithm 1 on each (particle, template) pair; returns a dict of arrays.

    ``templates`` holds one volume per particle, or a single shared volume;
    ``refine`` 1 replaces the Newton steps by gradient steps.
    """
    parts = np.ascontiguousarray(particles, dtype=np.float32)
    temps = np.ascontiguousarray(templates, dtype=np.float32)
    B, N = parts.shape[0], parts.shape[-1]
    tstride = 0 if temps.shape[0] == 1 else N ** 3
    p = make_params(N, S, r_max, L0, K, P, M_iter, L_sched, step_tol, accept_tol, refine)
    out = dict(euler=np.zeros((B, 3)), R=np.zeros((B, 3, 3)), score=np.zeros(B),
               best_p=np.zeros(B, dtype=np.int32), flags=np.zeros(B, dtype=np.int32),
               cand_idx=np.full((B, P), -1, dtype=np.int32), cand_euler0=np.zeros((B, P, 3)),
               cand_euler=np.zeros((B, P, 3)), cand_score=np.full((B, P), np.nan),
               n_cand=np.zeros(B, dtype=np.int32))
    pp = None if P_per is None else np.ascontiguousarray(P_per, dtype=np.int32)
    lib().orc_align_batch(ctypes.byref(p), _f(parts), _f(temps), ctypes.c_int(B), ctypes.c_long(tstride),
                          _i(pp) if pp is not None else None,
                          _d(out["euler"]), _d(out["R"]), _d(out["score"]), _i(out["best_p"]),
                          _i(out["flags"]), _i(out["cand_idx"]), _d(out["cand_euler0"]),
                          _d(out["cand_euler"]), _d(out["cand_score"]), _i(out["n_cand"]),
                          ctypes.c_int(n_threads))
    return out


# ---- align from SH coefficients ---------------------------------------------
def align_coefs_batch(f, h, *, S, r_max, L0, K, P, M_iter, L_sched, N=0, n_threads=0,
                      step_tol=1e-9, accept_tol=1e-11):
    """Algorithm 1 after the analysis: ``f`` complex [B][S][lm], ``h`` complex
    [S][lm] (one shared template) or [B][S][lm]."""
    fa = _split(np.asarray(f))
    hh = np.asarray(h)
    ha = _split(hh)
    B = np.asarray(f).shape[0]
    per = 2 * S * lm_size(L_sched[-1])
    hstride = 0 if hh.ndim == 2 else per
    p = make_params(N, S, r_max, L0, K, P, M_iter, L_sched, step_tol, accept_tol)
    euler = np.zeros((B, 3)); score = np.zeros(B)
    best = np.zeros(B, dtype=np.int32); flags = np.zeros(B, dtype=np.int32)
    lib().orc_align_coefs_batch(ctypes.byref(p), _d(fa), _d(ha), ctypes.c_long(hstride),
                                ctypes.c_int(B), _d(euler), _d(score), _i(best), _i(flags),
                                ctypes.c_int(n_threads))
    return dict(euler=euler, score=score, best_p=best, flags=flags)


# ---- template gradient of the refined score ----------------------------------
def implicit_shift(grad, H):
    g = np.ascontiguousarray(grad, dtype=np.float64)
    Hm = np.ascontiguousarray(H, dtype=np.float64).reshape(9)
    v = np.zeros(3)
    fl = lib().orc_implicit_shift(_d(g), _d(Hm), _d(v))
    return v, fl


def coef_grad(f, S, R, L, abg, v=None, wt=1.0):
    """dLambda/dh_ln(r_s) (complex [S][lm]) of one particle at rotation abg,
    with implicit shift v (None: the partial derivative at fixed abg)."""
    fa = _split(np.asarray(f))
    a = np.ascontiguousarray(abg, dtype=np.float64)
    vv = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
    G = np.zeros(2 * S * lm_size(L))
    lib().orc_coef_grad(_d(fa), ctypes.c_int(S), ctypes.c_double(R), ctypes.c_int(L), _d(a),
                        _d(vv) if vv is not None else None, ctypes.c_double(wt), _d(G))
    return (G[0::2] + 1j * G[1::2]).reshape(S, lm_size(L))


def analysis_adjoint(G, N, S, R, L):
    """Transpose of ``analyze_volume`` applied to G (complex [S][lm]); [N][N][N]."""
    Ga = _split(np.asarray(G))
    vox = np.zeros(N ** 3)
    lib().orc_analysis_adjoint(_d(Ga), ctypes.c_int(N), ctypes.c_int(S), ctypes.c_double(R),
                               ctypes.c_int(L), _d(vox))
    return vox.reshape(N, N, N)


def template_grad_batch(f, h, euler, *, S, r_max, L_sched, wt=None, N=0, n_threads=0):
    """Per-particle dLambda_b/dh (complex [B][S][lm]) at the refined rotations
    ``euler`` [B][3]; also returns (v, C) [B][4] and the singular-Hessian flags."""
    fa = _split(np.asarray(f))
    hh = np.asarray(h)
    ha = _split(hh)
    B = np.asarray(f).shape[0]
    L = L_sched[-1]
    per = 2 * S * lm_size(L)
    hstride = 0 if hh.ndim == 2 else per
    p = make_params(N, S, r_max, 0, 0, 0, 0, L_sched)
    e = np.ascontiguousarray(euler, dtype=np.float64)
    w = None if wt is None else np.ascontiguousarray(wt, dtype=np.float64)
    G = np.zeros(B * per); out4 = np.zeros((B, 4)); flags = np.zeros(B, dtype=np.int32)
    lib().orc_template_grad_batch(ctypes.byref(p), _d(fa), _d(ha), ctypes.c_long(hstride),
                                  ctypes.c_int(B), _d(e), _d(w) if w is not None else None,
                                  _d(G), _d(out4), _i(flags), ctypes.c_int(n_threads))
    return (G[0::2] + 1j * G[1::2]).reshape(B, S, lm_size(L)), out4, flags


def align_from_c(c, *, L0, K, P, M_iter, L_sched, step_tol=1e-9, accept_tol=1e-11, refine=0):
    """Algorithm 1 from one pair's correlation coefficients (oracle layout, up to L_J)."""
    p = make_params(0, 0, 0.0, L0, K, P, M_iter, L_sched, step_tol, accept_tol, refine)
    ca = _split(np.asarray(c))
    out = dict(euler=np.zeros(3), R=np.zeros(9), score=np.zeros(1), best_p=np.zeros(1, dtype=np.int32),
               flags=np.zeros(1, dtype=np.int32), cand_idx=np.full(P, -1, dtype=np.int32),
               cand_euler=np.zeros((P, 3)), cand_score=np.full(P, np.nan),
               n_cand=np.zeros(1, dtype=np.int32))
    lib().orc_align_from_c(ctypes.byref(p), _d(ca), ctypes.c_int(P), _d(out["euler"]), _d(out["R"]),
                           _d(out["score"]), _i(out["best_p"]), _i(out["flags"]), _i(out["cand_idx"]),
                           None, _d(out["cand_euler"]), _d(out["cand_score"]), _i(out["n_cand"]))
    out["R"] = out["R"].reshape(3, 3)
    return out
