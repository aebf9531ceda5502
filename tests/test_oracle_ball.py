"""Pins for the oracle's ball-harmonic radial basis (Appendix "Ball harmonics
expansion and eigenvalue-based truncation") and its correlation (Eq. sigmalmm,
the rank bound of Appendix "Low-rank structure induced by radial sparsity")."""
import math

import numpy as np
from scipy.special import spherical_jn

import oracle as O
from oracle import ball

RNG = np.random.default_rng(41)


def test_bessel_zeros_closed_forms_and_interlacing():
    zs = ball.bessel_zeros(6, 40.0)
    assert np.allclose(zs[0], np.pi * np.arange(1, len(zs[0]) + 1), rtol=0, atol=1e-13)
    for x in zs[1]:                 # j_1(x) = 0  <=>  tan x = x
        assert abs(math.tan(x) - x) < 1e-9 * x
    for x in zs[2]:                 # j_2(x) = 0  <=>  tan x = 3x / (3 - x^2)
        assert abs(math.tan(x) - 3 * x / (3 - x * x)) < 1e-9 * (1 + abs(math.tan(x)))
    assert abs(zs[1][0] - 4.493409457909064) < 1e-12
    counts = [len(z) for z in zs]
    assert all(a >= b for a, b in zip(counts, counts[1:]))          # |K_l| decreases with l
    for l in range(1, 7):
        for k in range(len(zs[l])):
            assert zs[l - 1][k] < zs[l][k] < (zs[l - 1][k + 1] if k + 1 < len(zs[l - 1]) else np.inf)


def _synth_shells(a, W_unused, zs, r, R, L):
    """Shell SH coefficients f_lm(r_s) = sum_k a_klm N_lk j_l(lambda_lk r_s / R)."""
    S = len(r)
    f = np.zeros((S, O.lm_size(L)), complex)
    for l in range(L + 1):
        for k, lam in enumerate(zs[l]):
            N = math.sqrt(2.0 / R ** 3) / abs(spherical_jn(l + 1, lam))
            for m in range(l + 1):
                f[:, O.lm_index(l, m)] += a[k, O.lm_index(l, m)] * N * spherical_jn(l, lam * r / R)
    return f


def _rand_ball(counts, L):
    a = np.zeros((int(max(counts)), O.lm_size(L)), complex)
    for l in range(L + 1):
        for k in range(int(counts[l])):
            for m in range(l + 1):
                a[k, O.lm_index(l, m)] = RNG.normal() + (1j * RNG.normal() if m else 0)
    return a


def test_projection_inverts_synthesis_with_a_fine_radial_rule():
    L, R, Lam, S = 6, 10.0, 25.0, 48
    W, counts = ball.radial_table(S, R, L, Lam)
    zs = ball.bessel_zeros(L, Lam)
    r, _ = O.radial_nodes(S, R)
    a = _rand_ball(counts, L)
    got = ball.project(_synth_shells(a, W, zs, r, R, L), W)
    assert np.abs(got - a).max() < 1e-10 * np.abs(a).max()


def test_ball_correlation_equals_shell_correlation_of_ball_limited_functions():
    """For radial profiles inside the retained span, Parseval in the orthonormal
    radial basis makes sum_k f_klm conj(h_kln) the radial inner product that the
    shell contraction computes."""
    L, R, Lam, S = 6, 10.0, 25.0, 48
    W, counts = ball.radial_table(S, R, L, Lam)
    zs = ball.bessel_zeros(L, Lam)
    r, _ = O.radial_nodes(S, R)
    f = _synth_shells(_rand_ball(counts, L), W, zs, r, R, L)
    h = _synth_shells(_rand_ball(counts, L), W, zs, r, R, L)
    cb = ball.correlate_ball(ball.project(f, W), ball.project(h, W), counts, L)
    cs = O.correlate(f, h, S, R, L)
    assert np.abs(cb - cs).max() < 1e-9 * np.abs(cs).max()


def test_rank_bound_and_rotation():
    """rank(A_l) <= |K_l| (Eq. rank_bound), and a template rotated in coefficient
    space leaves the rank alone: A_l(g o h) = A_l D^l(g)^*."""
    L, R, Lam, S = 10, 8.0, 20.0, 24
    W, counts = ball.radial_table(S, R, L, Lam)
    f = np.zeros((S, O.lm_size(L)), complex)
    h = np.zeros_like(f)
    for s in range(S):
        for l in range(L + 1):
            for m in range(l + 1):
                f[s, O.lm_index(l, m)] = RNG.normal() + (1j * RNG.normal() if m else 0)
                h[s, O.lm_index(l, m)] = RNG.normal() + (1j * RNG.normal() if m else 0)
    fb, hb = ball.project(f, W), ball.project(h, W)
    c = ball.correlate_ball(fb, hb, counts, L)
    g = (0.4, 2.1, 5.0)
    hr = np.zeros_like(hb)
    for l in range(L + 1):
        D = O.wigner_D(l, *g)
        for k in range(hb.shape[0]):
            full = np.array([hb[k, O.lm_index(l, n)] if n >= 0 else (-1) ** n * np.conj(hb[k, O.lm_index(l, -n)])
                             for n in range(-l, l + 1)])
            v = D @ full
            for m in range(l + 1):
                hr[k, O.lm_index(l, m)] = v[m + l]
    cr = ball.correlate_ball(fb, hr, counts, L)
    for l in range(L + 1):
        o = O.c_index(l, -l, -l)
        A = c[o:o + (2 * l + 1) ** 2].reshape(2 * l + 1, 2 * l + 1)
        Ar = cr[o:o + (2 * l + 1) ** 2].reshape(2 * l + 1, 2 * l + 1)
        if counts[l] == 0:
            assert np.abs(A).max() == 0
            continue
        sv = np.linalg.svd(A, compute_uv=False)
        assert np.sum(sv > 1e-10 * sv[0]) <= counts[l]
        assert np.abs(Ar - A @ O.wigner_D(l, *g).conj().T).max() < 1e-10 * np.abs(A).max()


def test_alignment_from_correlation_coefficients_is_algorithm_1():
    import synth
    w = synth.WORKLOADS["small32"]
    d = synth.make_batch(w)
    P, H = d["particles"].numpy(), d["templates"].numpy()
    ref = O.align_batch(P, H, S=w.n_shells, r_max=w.r_max, L0=w.L0, K=w.K, P=w.P, M_iter=w.M_iter,
                        L_sched=w.L_sched)
    L = w.L_sched[-1]
    c = O.correlate(O.analyze_volume(P[0], w.n_shells, w.r_max, L),
                    O.analyze_volume(H[0], w.n_shells, w.r_max, L), w.n_shells, w.r_max, L)
    r = O.align_from_c(c, L0=w.L0, K=w.K, P=w.P, M_iter=w.M_iter, L_sched=w.L_sched)
    assert np.array_equal(r["euler"], ref["euler"][0]) and r["score"][0] == ref["score"][0]


def test_planted_rotation_recovered_with_the_ball_basis():
    """Noiseless exact renderings: with the eigenvalue cut Lambda = 20 (six radial
    terms at l = 0, none above l = 17) the planted rotation comes back within
    0.05 deg (0.024 observed; the shell path at L = 16 stays at 0.104)."""
    import synth
    w = synth.WORKLOADS["small32"]
    d = synth.make_batch(w, exact_rotation=True, noise=False)
    out = ball.align_ball(d["particles"].numpy(), d["templates"].numpy(), S=16, r_max=w.r_max,
                          Lam=20.0, L0=w.L0, K=w.K, P=w.P, M_iter=w.M_iter, L_sched=(8, 12, 16, 20))
    assert list(out["counts"][:3]) == [6, 5, 5] and out["counts"][-1] == 0
    assert math.degrees(O.rotation_angle(out["R"][0], d["R_true"][0])) < 0.05
