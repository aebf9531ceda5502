"""Pins for the step control of the oracle's Newton march (Section 2.2's
update with the safeguards read for it, and Section 2.4's stop on the
parameter increment): a trial that lowers C_L is halved, at most twice; when
no trial is accepted theta stays and flag bit 2 is set; a level ends for a
candidate before its step once ||delta|| < step_tol.

Every expected value here comes from outside the march: the step delta is
solved with numpy from the gradient and Hessian (themselves pinned against
central differences), and every value of C that decides acceptance is the
brute-force quadrature correlation <f, g o h> of the synthesised shell
functions, not the oracle's Wigner sum.

Not reached: a step whose full and half trials are both rejected while the
quarter trial is accepted.  The clamp pi / (2 (L+1)) is a quarter period of
the top degree, so within it C_L is close enough to its quadratic model that
no seeded scan (about 10^5 starts, L = 1..10, poles included) produced one;
the "at most twice" count is checked only through the all-rejected case."""
import math

import numpy as np

import oracle as O


def rand_coef(L, S, rng):
    a = np.zeros((S, O.lm_size(L)), complex)
    for s in range(S):
        for l in range(L + 1):
            for m in range(l + 1):
                a[s, O.lm_index(l, m)] = rng.normal() + (1j * rng.normal() if m else 0)
    return a


def brute_C(f, h, S, R, L, abg):
    """sum_s w_s sum_jk w_j (2 pi / n_phi) f_L(r_s w) h_L(r_s g^{-1} w)."""
    r, ws = O.radial_nodes(S, R)
    x, w = O.gauss_legendre(L + 1)
    nphi = 2 * L + 2
    Rg = O.euler_to_matrix(*abg)
    tot = 0.0
    for j in range(L + 1):
        th = math.acos(x[j])
        for k in range(nphi):
            ph = 2 * math.pi * k / nphi
            v = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
            u = Rg.T @ v
            tu, pu = math.acos(max(-1.0, min(1.0, u[2]))), math.atan2(u[1], u[0])
            for s in range(S):
                tot += (ws[s] * w[j] * (2 * math.pi / nphi) * O.sh_synthesize(f[s], L, th, ph)
                        * O.sh_synthesize(h[s], L, tu, pu))
    return tot


def newton_step(c, L, t):
    """delta = -H^{-1} grad C_L, clamped to pi / (2 (L+1)); requires -H positive definite."""
    C, g, H, _ = O.objective(c, L, *t, derivs=True)
    assert np.linalg.eigvalsh(-H).min() > 0
    d = -np.linalg.solve(H, g)
    cap = math.pi / (2 * (L + 1))
    n = np.linalg.norm(d)
    return d * min(1.0, cap / n)


def same_rotation(a, b, tol=1e-12):
    return O.rotation_angle(O.euler_to_matrix(*a), O.euler_to_matrix(*b)) < tol


# A start on the far side of a maximum of C_6 where the full (clamped) Newton
# step overshoots and lowers C while the half step raises it (found by a
# seeded scan; such starts are rare because the clamp is a quarter period of
# the top degree).
L6, S3, R5 = 6, 3, 5.0
_rng = np.random.default_rng(0)
F6, H6 = rand_coef(L6, S3, _rng), rand_coef(L6, S3, _rng)
C6 = O.correlate(F6, H6, S3, R5, L6)
T6 = np.array([0.5553462636654284, 1.0054467546257164, 0.5584720723468534])


def trial_gains():
    d = newton_step(C6, L6, T6)
    c0 = brute_C(F6, H6, S3, R5, L6, T6)
    gains = [(brute_C(F6, H6, S3, R5, L6, O.wrap(T6 + d / 2 ** k)) - c0) / abs(c0) for k in range(3)]
    return d, c0, gains


def test_rejected_full_step_is_halved():
    d, c0, gains = trial_gains()
    assert gains[0] < -1e-3 and gains[1] > 1e-2          # full step lowers C, half step raises it
    x, sc, fl = O.newton_march(C6, [L6], 1, T6.copy())
    assert same_rotation(x, O.wrap(T6 + d / 2))
    assert fl & 4 == 0 and fl & 2 == 0
    assert abs(sc - brute_C(F6, H6, S3, R5, L6, x)) < 1e-10 * abs(sc)


def test_acceptance_threshold_selects_the_trial():
    """The rule accepts theta' when C(theta') >= C(theta) - accept_tol |C(theta)|; a
    negative accept_tol demands a gain of |accept_tol|.  Between the full step's
    and the half step's gain the half step is taken; above every trial's gain
    nothing is, theta stays bit for bit and bit 2 is set."""
    d, c0, gains = trial_gains()
    thr = 0.5 * (max(gains[0], 0.0) + gains[1])
    x, sc, fl = O.newton_march(C6, [L6], 1, T6.copy(), accept_tol=-thr)
    assert same_rotation(x, O.wrap(T6 + d / 2)) and fl & 4 == 0
    thr = max(gains) + 0.02
    x, sc, fl = O.newton_march(C6, [L6], 1, T6.copy(), accept_tol=-thr)
    assert np.array_equal(x, T6)
    assert fl & 4
    assert abs(sc - c0) < 1e-10 * abs(c0)
    # a full step that raises C is taken whole
    x, sc, fl = O.newton_march(C6, [L6], 1, T6.copy(), accept_tol=1.0)
    assert same_rotation(x, O.wrap(T6 + d)) and fl & 4 == 0


def test_rejection_ends_only_that_step():
    """After a step with no accepted trial the march goes on from the same theta
    with the next step (bit 2 stays set): with two steps and a threshold that only
    the second evaluation at theta faces, the result equals one rejected step."""
    d, c0, gains = trial_gains()
    thr = max(gains) + 0.02
    x1, s1, f1 = O.newton_march(C6, [L6], 1, T6.copy(), accept_tol=-thr)
    x2, s2, f2 = O.newton_march(C6, [L6], 2, T6.copy(), accept_tol=-thr)
    assert np.array_equal(x1, T6) and np.array_equal(x2, T6) and f1 & 4 and f2 & 4


def test_step_tol_stops_before_the_step():
    d0 = newton_step(C6, L6, T6)
    n0 = np.linalg.norm(d0)
    # ||delta|| just below step_tol: no step, theta bit for bit, score C(theta)
    x, sc, fl = O.newton_march(C6, [L6], 3, T6.copy(), step_tol=n0 * (1 + 1e-9))
    assert np.array_equal(x, T6) and fl == 0
    assert abs(sc - brute_C(F6, H6, S3, R5, L6, T6)) < 1e-10 * abs(sc)
    # just above it: the step is taken
    x, sc, fl = O.newton_march(C6, [L6], 1, T6.copy(), step_tol=n0 * (1 - 1e-9))
    assert not np.array_equal(x, T6)


def test_step_tol_ends_the_level_after_converging_steps():
    """Near a planted maximum: the first step's increment is above step_tol, the
    second's below; three allowed steps then give exactly the one-step result."""
    L, S, R = 8, 3, 5.0
    rng = np.random.default_rng(3)
    f = rand_coef(L, S, rng)
    g_true = (1.0, 1.2, 2.0)
    h = np.zeros_like(f)
    for s in range(S):
        for l in range(L + 1):
            full = np.array([f[s, O.lm_index(l, n)] if n >= 0 else (-1) ** n * np.conj(f[s, O.lm_index(l, -n)])
                             for n in range(-l, l + 1)])
            hr = O.wigner_D(l, *g_true).conj().T @ full
            for m in range(l + 1):
                h[s, O.lm_index(l, m)] = hr[m + l]
    c = O.correlate(f, h, S, R, L)
    t0 = np.array(g_true) + np.array([0.03, -0.02, 0.025])
    d0 = newton_step(c, L, t0)
    assert brute_C(f, h, S, R, L, O.wrap(t0 + d0)) > brute_C(f, h, S, R, L, t0)
    t1 = O.wrap(t0 + d0)
    n0, n1 = np.linalg.norm(d0), np.linalg.norm(newton_step(c, L, t1))
    assert n1 < 0.1 * n0
    tol = math.sqrt(n0 * n1)
    x1, s1, _ = O.newton_march(c, [L], 1, t0.copy(), step_tol=tol)
    x3, s3, f3 = O.newton_march(c, [L], 3, t0.copy(), step_tol=tol)
    assert same_rotation(x1, t1) and np.array_equal(x1, x3) and s1 == s3 and f3 == 0
    # started exactly at the planted maximum the march takes no step at all
    xs, ss, fs = O.newton_march(c, [L], 3, np.array(g_true))
    assert np.array_equal(xs, np.array(g_true)) and fs == 0
    assert abs(ss - brute_C(f, h, S, R, L, g_true)) < 1e-10 * abs(ss)


def test_gradient_direction_is_the_scaled_gradient():
    g = np.array([0.01, -0.02, 0.005])
    H = -np.array([[4.0, 1.0, 0.5], [1.0, 3.0, 0.2], [0.5, 0.2, 2.0]])
    d = O.gradient_direction(g, H, 32)
    assert np.abs(d - g / np.linalg.norm(H)).max() < 1e-18
    d = O.gradient_direction(np.array([10.0, 0, 0]), H, 8)        # clamped
    assert abs(np.linalg.norm(d) - math.pi / 18) < 1e-15 and d[0] > 0


def test_gradient_steps_converge_linearly_and_newton_faster():
    """Section 5.1's comparison: near a planted maximum the gradient method
    climbs monotonically but needs many more steps than Newton for the same
    accuracy."""
    L, S, R = 8, 3, 5.0
    rng = np.random.default_rng(3)
    f = rand_coef(L, S, rng)
    g_true = (1.0, 1.2, 2.0)
    h = np.zeros_like(f)
    for s in range(S):
        for l in range(L + 1):
            full = np.array([f[s, O.lm_index(l, n)] if n >= 0 else (-1) ** n * np.conj(f[s, O.lm_index(l, -n)])
                             for n in range(-l, l + 1)])
            hr = O.wigner_D(l, *g_true).conj().T @ full
            for m in range(l + 1):
                h[s, O.lm_index(l, m)] = hr[m + l]
    c = O.correlate(f, h, S, R, L)
    Rt = O.euler_to_matrix(*g_true)
    t0 = np.array(g_true) + np.array([0.05, -0.04, 0.03])
    err = lambda x: O.rotation_angle(O.euler_to_matrix(*x), Rt)
    xn, sn, _ = O.newton_march(c, [L], 3, t0.copy(), step_tol=0)
    prev, scores = err(t0), []
    for k in (1, 2, 3, 6, 12):
        xg, sg, fl = O.newton_march(c, [L], k, t0.copy(), step_tol=0, method=1)
        scores.append(sg)
        assert err(xg) < prev and fl & 2 == 0
        prev = err(xg)
    assert all(b >= a for a, b in zip(scores, scores[1:]))
    xg3, _, _ = O.newton_march(c, [L], 3, t0.copy(), step_tol=0, method=1)
    assert err(xn) < 1e-9 and err(xg3) > 100 * err(xn)
    xg, _, _ = O.newton_march(c, [L], 200, t0.copy(), step_tol=1e-12, method=1)
    assert err(xg) < 1e-6
