"""Pins for the oracle's quadrature, spherical harmonics and sampling.

Each check compares the oracle with something other than itself: a library
routine (numpy, scipy), a closed form, or an exactness property.
"""
import math

import numpy as np
import pytest
import scipy.special as sps

import oracle as O


@pytest.mark.parametrize("n", [1, 2, 5, 17, 33, 49])
def test_gauss_legendre_matches_numpy(n):
    x, w = O.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(x, xr, atol=1e-14, rtol=0)
    assert np.allclose(w, wr, atol=1e-14, rtol=0)


def test_radial_rule_integrates_r2_polynomials():
    # integral_0^R r^2 * r^k dr = R^(k+3)/(k+3), exact for 2S-1 >= k+2
    S, R = 12, 15.0
    r, w = O.radial_nodes(S, R)
    for k in range(0, 2 * S - 2):
        exact = R ** (k + 3) / (k + 3)
        assert abs(np.sum(w * r ** k) - exact) <= 1e-12 * exact
    assert np.all((r > 0) & (r < R))


def test_plm_bar_closed_forms():
    for x in [-0.9, -0.1, 0.3, 0.77]:
        assert abs(O.plm_bar(0, 0, x) - 1 / math.sqrt(4 * math.pi)) < 1e-15
        assert abs(O.plm_bar(1, 0, x) - math.sqrt(3 / (4 * math.pi)) * x) < 1e-15
        st = math.sqrt(1 - x * x)
        assert abs(O.plm_bar(1, 1, x) + math.sqrt(3 / (8 * math.pi)) * st) < 1e-15
        assert abs(O.plm_bar(2, 0, x) - 0.25 * math.sqrt(5 / math.pi) * (3 * x * x - 1)) < 1e-15


@pytest.mark.parametrize("l", [0, 1, 2, 5, 16, 32, 48])
def test_plm_bar_matches_scipy(l):
    th = np.array([0.1, 0.7, 1.5, 2.2, 3.0])
    for m in range(0, l + 1):
        ref = sps.sph_harm_y(l, m, th, 0.0).real
        got = np.array([O.plm_bar(l, m, math.cos(t)) for t in th])
        assert np.allclose(got, ref, atol=1e-13, rtol=1e-12), (l, m)


def test_angular_quadrature_orthonormal_and_addition_theorem():
    L = 10
    x, w = O.gauss_legendre(L + 1)
    nphi = 2 * L + 2
    ph = 2 * np.pi * np.arange(nphi) / nphi
    Y = {}
    for l in range(L + 1):
        for m in range(-l, l + 1):
            p = np.array([O.plm_bar(l, abs(m), xx) for xx in x])
            if m < 0:
                p = p * (-1) ** m
            Y[(l, m)] = p[:, None] * np.exp(1j * m * ph)[None, :]
    keys = list(Y)
    Wt = w[:, None] * (2 * np.pi / nphi)
    G = np.array([[np.sum(Wt * Y[a] * np.conj(Y[b])) for b in keys] for a in keys])
    assert np.abs(G - np.eye(len(keys))).max() < 1e-13
    for l in range(L + 1):
        s = sum(abs(Y[(l, m)][3, 1]) ** 2 for m in range(-l, l + 1))
        assert abs(s - (2 * l + 1) / (4 * np.pi)) < 1e-13


def test_trilinear_reproduces_affine_functions_and_zero_outside():
    N = 16
    k, j, i = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    vol = (0.5 * i - 0.25 * j + 0.125 * k + 1.0).astype(np.float32)
    rng = np.random.default_rng(3)
    for _ in range(50):
        p = rng.uniform(0, N - 1, 3)
        assert abs(O.trilinear(vol, *p) - (0.5 * p[0] - 0.25 * p[1] + 0.125 * p[2] + 1.0)) < 1e-12
    assert O.trilinear(vol, 3, 4, 5) == float(vol[5, 4, 3])
    assert O.trilinear(vol, -2.0, 3, 3) == 0.0
    assert O.trilinear(vol, 3, 3, N + 1.5) == 0.0


def test_shell_analysis_of_coordinate_ramps_pins_axes():
    """x, y, z ramps are pure degree-1 functions on every shell.

    On a shell of radius r: z = r cos t has Y_10 coefficient r sqrt(4pi/3);
    x = r sin t cos p has Y_11 coefficient -r sqrt(2pi/3); y = r sin t sin p
    has Y_11 coefficient +i r sqrt(2pi/3).  Trilinear interpolation is exact
    for affine volumes, so these hold to rounding.
    """
    N, S, R, L = 24, 5, 10.0, 6
    c0 = N / 2
    k, j, i = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    r, _ = O.radial_nodes(S, R)
    for name, vol in [("x", i - c0), ("y", j - c0), ("z", k - c0)]:
        f = O.analyze_volume(vol.astype(np.float32), S, R, L)
        for s in range(S):
            expect = np.zeros(O.lm_size(L), complex)
            if name == "z":
                expect[O.lm_index(1, 0)] = r[s] * math.sqrt(4 * math.pi / 3)
            elif name == "x":
                expect[O.lm_index(1, 1)] = -r[s] * math.sqrt(2 * math.pi / 3)
            else:
                expect[O.lm_index(1, 1)] = 1j * r[s] * math.sqrt(2 * math.pi / 3)
            assert np.abs(f[s] - expect).max() < 1e-12 * max(1.0, r[s]), (name, s)


def test_analysis_inverts_synthesis():
    L = 7
    rng = np.random.default_rng(5)
    a = np.zeros(O.lm_size(L), complex)
    for l in range(L + 1):
        for m in range(l + 1):
            a[O.lm_index(l, m)] = rng.normal() + (1j * rng.normal() if m else 0)
    x, _ = O.gauss_legendre(L + 1)
    nphi = 2 * L + 2
    smp = np.array([[O.sh_synthesize(a, L, math.acos(xx), 2 * math.pi * k / nphi)
                     for k in range(nphi)] for xx in x])
    assert np.abs(O.sh_analyze_shell(smp, L) - a).max() < 1e-13


def test_wigner_term_count_closed_form():
    """Appendix A.5: sum_{l<=L} (2l+1)^2 = (L+1)(2L+1)(2L+3)/3."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "wigner_term_counts.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    for L, T in rows:
        L, T = int(L), int(T)
        assert sum((2 * l + 1) ** 2 for l in range(L + 1)) == T
        assert O.lib().orc_c_size(L) == T
