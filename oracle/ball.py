"""Oracle: ball-harmonic radial basis with the eigenvalue (Bessel-zero)
truncation, and the correlation coefficients it gives (Appendix "Ball
harmonics expansion and eigenvalue-based truncation", Eq. sigmalmm and the
low-rank factorisation of Appendix "Low-rank structure induced by radial
sparsity").

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
bench's CPU legs may use this module; the CUDA library never does.

Reading.  On the ball of radius R the basis is
psi_klm(x) = N_lk j_l(lambda_lk |x| / R) Y_lm(x / |x|), lambda_lk the k-th
positive zero of the spherical Bessel function j_l (Dirichlet condition at
|x| = R), N_lk^2 = 2 / (R^3 j_{l+1}(lambda_lk)^2) (unit norm).  The retained
set is K_l = {k : lambda_lk <= Lambda} for a frequency budget Lambda.  The
coefficient f_klm = <f, psi_klm> = int_0^R f_lm(r) N_lk j_l(lambda_lk r / R) r^2 dr
is evaluated with the same Gauss-Legendre radial shells as the rest of the
path (weights w_s with the r^2 Jacobian), from the shell SH coefficients
f_lm(r_s):  f_klm = sum_s w_s N_lk j_l(lambda_lk r_s / R) f_lm(r_s).
Then sigma_lmn = sum_{k in K_l} f_klm conj(h_kln) (Eq. sigmalmm), so
A_l = sum_k a_lk b_lk^* has rank <= |K_l| (Eq. rank_bound).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq
from scipy.special import spherical_jn

from . import c_index, c_size, lm_index, lm_size, radial_nodes


def bessel_zeros(L, Lam):
    """lambda_lk <= Lam for l = 0..L: list of arrays (the interlacing
    lambda_{l,k} < lambda_{l+1,k} < lambda_{l,k+1} brackets every root)."""
    zs = [np.array([k * math.pi for k in range(1, int(Lam / math.pi) + 2)])]
    for l in range(1, L + 1):
        prev = zs[-1]
        out = []
        for k in range(len(prev) - 1):
            a, b = prev[k], prev[k + 1]
            out.append(brentq(lambda x: spherical_jn(l, x), a, b, xtol=1e-15, rtol=1e-15, maxiter=200))
        # one more root beyond the last bracket, below the next zero of j_{l-1}'s follower
        if len(prev):
            a = prev[-1]
            b = a + math.pi + 1.0
            while spherical_jn(l, a) * spherical_jn(l, b) > 0:
                b += 0.5
            out.append(brentq(lambda x: spherical_jn(l, x), a, b, xtol=1e-15, rtol=1e-15, maxiter=200))
        zs.append(np.array(out))
    return [z[z <= Lam] for z in zs]


def radial_table(S, R, L, Lam):
    """W[l][k][s] = w_s N_lk j_l(lambda_lk r_s / R) for k < |K_l| (zero-padded to
    Kmax = |K_0|), and the counts |K_l|."""
    r, w = radial_nodes(S, R)
    zs = bessel_zeros(L, Lam)
    counts = np.array([len(z) for z in zs], dtype=np.int32)
    Kmax = int(counts.max()) if len(counts) else 0
    W = np.zeros((L + 1, Kmax, S))
    for l in range(L + 1):
        for k, lam in enumerate(zs[l]):
            N = math.sqrt(2.0 / R ** 3) / abs(spherical_jn(l + 1, lam))
            W[l, k] = w * N * spherical_jn(l, lam * r / R)
    return W, counts


def project(coef, W):
    """Shell SH coefficients [S][lm] (complex) -> ball coefficients [Kmax][lm]."""
    L = W.shape[0] - 1
    out = np.zeros((W.shape[1], lm_size(L)), complex)
    for l in range(L + 1):
        for m in range(l + 1):
            out[:, lm_index(l, m)] = W[l] @ coef[:, lm_index(l, m)]
    return out


def correlate_ball(fb, hb, counts, L):
    """sigma^l_mn = sum_{k < |K_l|} f_klm conj(h_kln) in the oracle's c layout."""
    c = np.zeros(c_size(L), complex)
    for l in range(L + 1):
        K = int(counts[l])
        for m in range(-l, l + 1):
            fm = fb[:K, lm_index(l, abs(m))] if m >= 0 else (-1) ** m * np.conj(fb[:K, lm_index(l, -m)])
            for n in range(-l, l + 1):
                hn = hb[:K, lm_index(l, abs(n))] if n >= 0 else (-1) ** n * np.conj(hb[:K, lm_index(l, -n)])
                c[c_index(l, m, n)] = np.sum(fm * np.conj(hn))
    return c


def align_ball(particles, templates, *, S, r_max, Lam, L0, K, P, M_iter, L_sched):
    """Algorithm 1 with the ball-harmonic correlation: shell analysis (the
    oracle's), projection on the retained radial basis, sigma by Eq. sigmalmm,
    then the SOFFT search, the march and the argmax.  Returns per-particle
    euler, R, score and the counts |K_l|."""
    from . import align_from_c, analyze_volume
    L = L_sched[-1]
    W, counts = radial_table(S, r_max, L, Lam)
    B = particles.shape[0]
    out = dict(euler=np.zeros((B, 3)), R=np.zeros((B, 3, 3)), score=np.zeros(B), counts=counts)
    for b in range(B):
        t = templates[b] if templates.shape[0] == B else templates[0]
        fb = project(analyze_volume(particles[b], S, r_max, L), W)
        hb = project(analyze_volume(t, S, r_max, L), W)
        r = align_from_c(correlate_ball(fb, hb, counts, L), L0=L0, K=K, P=P, M_iter=M_iter,
                         L_sched=L_sched)
        out["euler"][b], out["R"][b], out["score"][b] = r["euler"], r["R"], r["score"][0]
    return out
