"""Oracle: translation search and the 6-D rotation-translation alternation
(the appendix "Alternating search over rotations and translations", and the
T = 3 alternations of Section 5.2).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
bench's CPU legs may use this module; the CUDA library never does.

Readings (the appendix states the scheme, not its discretisation):

* the objective at a fixed rotation g is <f, g o S_tau h> with
  (S_tau h)(x) = h(x - tau); with u = g o h it equals the cross-correlation
  CC(t) = sum_x f(x) u(x - t) at t = g tau, so tau = R^T t;
* CC is the circular correlation a 3-D FFT computes (indices mod N);
* the integer search covers t in [-m, m]^3 (m = max_shift voxels per axis);
* sub-voxel refinement evaluates the trigonometric interpolant of CC,
  CC(t) = N^-3 Re sum_k X(k) exp(2 pi i k.t / N), X = F conj(U), k in
  [-N/2, N/2)^3 (the upsampled DFT of Guizar-Sicairos et al. that the paper
  cites), on a grid of 2 floor(0.75 U) + 1 points per axis at spacing 1/U
  centred on the integer peak (about 1.5 voxels wide);
* maxima on a grid are taken in linear order [z][y][x] with the smaller index
  winning ties;
* the alternation starts from tau = 0 and runs T rounds of (rotation search on
  (f, S_tau h) by Algorithm 1, then the translation search of g o h); the
  result is the last round's (g, tau);
* flag bit 5 (value 32): the integer peak lies on the search window's edge.
"""
from __future__ import annotations

import math

import numpy as np

from . import _d, _f, lib, align_batch


def transform_volume(vol, R=None, s=None):
    """out(x) = vol(R^T (x - c0) + c0 - s), trilinear, zero outside (float32)."""
    v = np.ascontiguousarray(vol, dtype=np.float32)
    N = v.shape[-1]
    Rm = np.eye(3) if R is None else np.ascontiguousarray(R, dtype=np.float64).reshape(3, 3)
    sv = np.zeros(3) if s is None else np.ascontiguousarray(s, dtype=np.float64)
    out = np.empty_like(v)
    Rm = np.ascontiguousarray(Rm)
    lib().orc_transform_volume(_f(v), N, _d(Rm), _d(sv), _f(out))
    return out


def circular_cc(f, u, t):
    """sum_x f(x) u(x - t), indices mod N; t = (x, y, z) integers (the definition)."""
    tx, ty, tz = (int(a) for a in t)
    return float(np.sum(f.astype(np.float64) * np.roll(u.astype(np.float64), (tz, ty, tx), axis=(0, 1, 2))))


def cross_spectrum(f, u):
    """X(k) = F(k) conj(U(k)), [kz][ky][kx], with the library FFT."""
    F = np.fft.fftn(np.asarray(f, dtype=np.float64))
    U = np.fft.fftn(np.asarray(u, dtype=np.float64))
    return F * np.conj(U)


def cc_interp(X, tx, ty, tz):
    """CC(t) = N^-3 Re sum_k X(k) exp(2 pi i k.t / N) on the grid tz x ty x tx;
    returns [len(tz)][len(ty)][len(tx)]."""
    N = X.shape[-1]
    k = np.fft.fftfreq(N) * N          # 0, 1, .., N/2-1, -N/2, .., -1
    E = [np.exp(2j * np.pi * np.outer(k, np.asarray(t, dtype=np.float64)) / N) for t in (tz, ty, tx)]
    v = np.einsum("zyx,za,yb,xc->abc", X, E[0], E[1], E[2], optimize=True)
    return v.real / N ** 3


def grid_argmax(v):
    """Linear index of the maximum of v ([z][y][x] order), smaller index on ties."""
    flat = v.reshape(-1)
    return int(np.flatnonzero(flat == flat.max())[0])


def fine_offsets(U):
    h = int(math.floor(0.75 * U))
    return (np.arange(2 * h + 1) - h) / float(U)


def shift_search(f, u, max_shift, upsample):
    """Best circular shift t = (x, y, z) of u onto f: integer search in the
    window, then the interpolant on the fine grid.  Returns (t, CC(t), flags)."""
    X = cross_spectrum(f, u)
    m = int(max_shift)
    w = np.arange(-m, m + 1, dtype=np.float64)
    v = cc_interp(X, w, w, w)
    i = grid_argmax(v)
    W = 2 * m + 1
    iz, iy, ix = i // (W * W), (i // W) % W, i % W
    t0 = np.array([w[ix], w[iy], w[iz]])
    flags = 32 if m > 0 and (abs(t0) == m).any() else 0
    off = fine_offsets(upsample)
    vf = cc_interp(X, t0[0] + off, t0[1] + off, t0[2] + off)
    j = grid_argmax(vf)
    nf = len(off)
    jz, jy, jx = j // (nf * nf), (j // nf) % nf, j % nf
    t = t0 + np.array([off[jx], off[jy], off[jz]])
    return t, float(vf.reshape(-1)[j]), flags


def align6d_batch(particles, templates, *, S, r_max, L0, K, P, M_iter, L_sched, rounds,
                  max_shift, upsample, n_threads=0, step_tol=1e-9, accept_tol=1e-11):
    """The alternation on every (particle, template) pair; templates: one per
    particle or one shared.  Returns euler, R, tau, t (= R tau), score (C_{L_J} of
    the last rotation step), cc (CC at t) and flags."""
    parts = np.ascontiguousarray(particles, dtype=np.float32)
    temps = np.ascontiguousarray(templates, dtype=np.float32)
    B = parts.shape[0]
    tmpl = [temps[b] if temps.shape[0] == B else temps[0] for b in range(B)]
    tau = np.zeros((B, 3))
    t = np.zeros((B, 3))
    cc = np.zeros(B)
    tflags = np.zeros(B, dtype=np.int32)
    kw = dict(S=S, r_max=r_max, L0=L0, K=K, P=P, M_iter=M_iter, L_sched=L_sched,
              n_threads=n_threads, step_tol=step_tol, accept_tol=accept_tol)
    for r in range(rounds):
        shifted = np.stack([tmpl[b] if r == 0 else transform_volume(tmpl[b], None, tau[b])
                            for b in range(B)])
        rot = align_batch(parts, shifted, **kw)
        for b in range(B):
            u = transform_volume(tmpl[b], rot["R"][b], None)
            t[b], cc[b], tflags[b] = shift_search(parts[b], u, max_shift, upsample)
            tau[b] = rot["R"][b].T @ t[b]
    out = dict(rot)
    out.update(tau=tau, t=t, cc=cc, flags=rot["flags"] | tflags)
    return out
