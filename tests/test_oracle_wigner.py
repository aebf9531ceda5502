"""Pins for the oracle's Wigner functions, rotation chart and the rotation rule."""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.special as sps

import oracle as O

RNG = np.random.default_rng(11)


def test_low_degree_closed_forms():
    for b in [0.0, 0.3, 1.2, 2.9, math.pi]:
        d = O.wigner_d(1, b)
        assert d[O.c_index(0, 0, 0)] == 1.0
        assert abs(d[O.c_index(1, 0, 0)] - math.cos(b)) < 1e-15
        assert abs(d[O.c_index(1, 1, 1)] - (1 + math.cos(b)) / 2) < 1e-15
        assert abs(d[O.c_index(1, 1, -1)] - (1 - math.cos(b)) / 2) < 1e-15
        assert abs(d[O.c_index(1, 1, 0)] + math.sin(b) / math.sqrt(2)) < 1e-15
        assert abs(d[O.c_index(1, 0, 1)] - math.sin(b) / math.sqrt(2)) < 1e-15


@pytest.mark.parametrize("b", [0.05, 0.9, 2.0, 3.1])
def test_d_l00_is_legendre_and_dm0_is_spherical_harmonic(b):
    L = 40
    d = O.wigner_d(L, b)
    for l in range(L + 1):
        Pl = np.polynomial.legendre.Legendre.basis(l)(math.cos(b))
        assert abs(d[O.c_index(l, 0, 0)] - Pl) < 1e-13
        # d^l_{m0}(b) = sqrt(4 pi / (2l+1)) Y_lm(b, 0)  (independent library)
        for m in range(0, l + 1):
            y = sps.sph_harm_y(l, m, b, 0.0).real
            assert abs(d[O.c_index(l, m, 0)] - math.sqrt(4 * math.pi / (2 * l + 1)) * y) < 1e-12


def test_recurrence_matches_finite_sum_to_l20():
    for b in [0.2, 1.1, 2.7]:
        d = O.wigner_d(20, b)
        for l in range(21):
            for m in range(-l, l + 1):
                for n in range(-l, l + 1):
                    assert abs(d[O.c_index(l, m, n)] - O.wigner_d_finite_sum(l, m, n, b)) < 1e-12


def _exact_d_half_pi_squared(l, m, n):
    """Exact value of d^l_{mn}(pi/2)^2 and its sign from Wigner's sum with
    cos = sin = 1/sqrt(2): d = 2^{-l} sqrt((l+n)!(l-n)!(l+m)!(l-m)!) * S with
    S = sum_k (-1)^{k-n+m} / ((l+n-k)! k! (l-k-m)! (k-n+m)!) rational."""
    f = math.factorial
    S = Fraction(0)
    for k in range(0, 2 * l + 1):
        a1, a2, a3 = l + n - k, l - k - m, k - n + m
        if min(a1, a2, a3) < 0:
            continue
        S += Fraction((-1) ** (k - n + m), f(a1) * f(k) * f(a2) * f(a3))
    pre = f(l + n) * f(l - n) * f(l + m) * f(l - m)
    return S * S * pre / Fraction(4 ** l), (S > 0) - (S < 0)


def test_finite_sum_exact_at_half_pi():
    for l in range(0, 7):
        for m in range(-l, l + 1):
            for n in range(-l, l + 1):
                sq, sg = _exact_d_half_pi_squared(l, m, n)
                v = O.wigner_d_finite_sum(l, m, n, math.pi / 2)
                assert abs(v - sg * math.sqrt(float(sq))) < 1e-15


@pytest.mark.parametrize("l", [1, 2, 7, 16, 32, 48])
def test_unitary(l):
    for b in [0.01, 0.8, 1.9, 3.13]:
        D = O.wigner_D(l, *RNG.uniform(0, 2 * math.pi, 1), b, *RNG.uniform(0, 2 * math.pi, 1))
        assert np.abs(D @ D.conj().T - np.eye(2 * l + 1)).max() < 1e-12


@pytest.mark.parametrize("l", [1, 3, 10, 24, 32, 48])
def test_homomorphism(l):
    for _ in range(3):
        e1 = (RNG.uniform(0, 2 * math.pi), RNG.uniform(0, math.pi), RNG.uniform(0, 2 * math.pi))
        e2 = (RNG.uniform(0, 2 * math.pi), RNG.uniform(0, math.pi), RNG.uniform(0, 2 * math.pi))
        R12 = O.euler_to_matrix(*e1) @ O.euler_to_matrix(*e2)
        e12 = O.matrix_to_euler(R12)
        assert np.abs(O.euler_to_matrix(*e12) - R12).max() < 1e-13
        lhs = O.wigner_D(l, *e12)
        rhs = O.wigner_D(l, *e1) @ O.wigner_D(l, *e2)
        assert np.abs(lhs - rhs).max() < 1e-12


def test_y_rotations_compose():
    l = 20
    b1, b2 = 0.4, 1.3
    assert np.abs(O.wigner_d_matrix(l, b1 + b2)
                  - O.wigner_d_matrix(l, b1) @ O.wigner_d_matrix(l, b2)).max() < 1e-12


def test_wigner_orthogonality_by_quadrature():
    """Eq. (wigner-orthogonality): int D^l_{mn} conj(D^l'_{m'n'}) dg = delta/(2l+1),
    with dg = da sin(b) db dg / (8 pi^2) discretised exactly by uniform nodes in
    a and g and Gauss-Legendre nodes in cos(b)."""
    L = 4
    na = 2 * L + 2
    x, w = O.gauss_legendre(L + 1)
    A = 2 * math.pi * np.arange(na) / na
    keys = [(l, m, n) for l in range(L + 1) for m in range(-l, l + 1) for n in range(-l, l + 1)]
    vals = np.zeros((len(keys), na, L + 1, na), complex)
    for ib, xb in enumerate(x):
        b = math.acos(xb)
        for l in range(L + 1):
            D = np.array([[[O.wigner_D(l, a, b, g) for g in A] for a in A]])[0]  # [a][g][m][n]
            for m in range(-l, l + 1):
                for n in range(-l, l + 1):
                    vals[keys.index((l, m, n)), :, ib, :] = D[:, :, m + l, n + l]
    wt = (np.ones(na)[:, None, None] * w[None, :, None] * np.ones(na)[None, None, :]) \
        * (2 * math.pi / na) ** 2 / (8 * math.pi ** 2)
    G = np.einsum("pabc,qabc,abc->pq", vals, vals.conj(), wt)
    expect = np.diag([1.0 / (2 * k[0] + 1) for k in keys])
    assert np.abs(G - expect).max() < 1e-13


def test_beta_derivatives_match_central_differences():
    L, h = 24, 1e-5
    for b in [0.3, 1.4, 2.6]:
        d, d1, d2 = O.wigner_d_derivs(L, b)
        dp = O.wigner_d(L, b + h)
        dm = O.wigner_d(L, b - h)
        fd1 = (dp - dm) / (2 * h)
        fd2 = (dp - 2 * d + dm) / (h * h)
        assert np.abs(fd1 - d1).max() < 1e-7 * max(1.0, np.abs(d1).max())
        assert np.abs(fd2 - d2).max() < 1e-4 * max(1.0, np.abs(d2).max())
        # second derivative of d against central differences of d'
        _, d1p, _ = O.wigner_d_derivs(L, b + h)
        _, d1m, _ = O.wigner_d_derivs(L, b - h)
        assert np.abs((d1p - d1m) / (2 * h) - d2).max() < 1e-7 * max(1.0, np.abs(d2).max())


def test_rotation_rule_of_harmonics_pins_convention():
    """Appendix A.4: Y_ln(g^{-1} x) = sum_m D^l_{mn}(g) Y_lm(x).

    A real bandlimited function u is synthesised at g^{-1} w on the analysis
    grid and analysed; its coefficients must equal sum_n D^l_{mn}(g) a_ln."""
    L = 6
    a = np.zeros(O.lm_size(L), complex)
    for l in range(L + 1):
        for m in range(l + 1):
            a[O.lm_index(l, m)] = RNG.normal() + (1j * RNG.normal() if m else 0)
    abg = (0.3, 1.2, 2.5)
    R = O.euler_to_matrix(*abg)
    x, _ = O.gauss_legendre(L + 1)
    nphi = 2 * L + 2
    smp = np.zeros((L + 1, nphi))
    for j in range(L + 1):
        for k in range(nphi):
            th, ph = math.acos(x[j]), 2 * math.pi * k / nphi
            v = R.T @ np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
            smp[j, k] = O.sh_synthesize(a, L, math.acos(max(-1, min(1, v[2]))), math.atan2(v[1], v[0]))
    b = O.sh_analyze_shell(smp, L)
    for l in range(L + 1):
        full = np.array([a[O.lm_index(l, n)] if n >= 0 else (-1) ** n * np.conj(a[O.lm_index(l, -n)])
                         for n in range(-l, l + 1)])
        pred = O.wigner_D(l, *abg) @ full
        for m in range(l + 1):
            assert abs(pred[m + l] - b[O.lm_index(l, m)]) < 1e-12
    # the inverse rotation must NOT match (guards against a transposed convention)
    pred_inv = O.wigner_D(1, *abg).conj().T @ np.array(
        [-np.conj(a[O.lm_index(1, 1)]), a[O.lm_index(1, 0)], a[O.lm_index(1, 1)]])
    assert abs(pred_inv[2] - b[O.lm_index(1, 1)]) > 1e-3


def test_rotation_angle_and_chart():
    R1 = O.euler_to_matrix(0.2, 0.5, 0.9)
    assert abs(np.linalg.det(R1) - 1) < 1e-14 and np.abs(R1 @ R1.T - np.eye(3)).max() < 1e-15
    # r_y(b) alone: angle b
    assert abs(O.rotation_angle(np.eye(3), O.euler_to_matrix(0, 0.37, 0)) - 0.37) < 1e-14
    # r_z(pi) r_y(b) r_z(pi) = r_y(-b)
    assert np.abs(O.euler_to_matrix(math.pi, 0.4, math.pi) - O.euler_to_matrix(0, -0.4, 0)).max() < 1e-15


@pytest.mark.parametrize("b", [0.05, 0.7, 1.9, 3.0])
def test_beta_derivatives_satisfy_the_degree_identity_and_the_differential_equation(b):
    """Exact identities of the Wigner functions (from their Jacobi-polynomial
    form), far tighter than finite differences:
      sin b d'^l_mn = (l cos b - mn/l) d^l_mn - sqrt((l^2-m^2)(l^2-n^2))/l d^{l-1}_mn,
      d''^l_mn = -cot b d'^l_mn + ((m^2 + n^2 - 2mn cos b)/sin^2 b - l(l+1)) d^l_mn."""
    L = 20
    d, d1, d2 = O.wigner_d_derivs(L, b)
    s, c = math.sin(b), math.cos(b)
    worst1 = worst2 = 0.0
    for l in range(1, L + 1):
        D = O.wigner_d_matrix(l, b, d)
        D1 = O.wigner_d_matrix(l, b, d1)
        D2 = O.wigner_d_matrix(l, b, d2)
        Dm = O.wigner_d_matrix(l - 1, b, d)
        for m in range(-l, l + 1):
            for n in range(-l, l + 1):
                prev = Dm[m + l - 1, n + l - 1] if max(abs(m), abs(n)) <= l - 1 else 0.0
                q = math.sqrt((l * l - m * m) * (l * l - n * n))
                rhs1 = (l * c - m * n / l) * D[m + l, n + l] - q / l * prev
                worst1 = max(worst1, abs(s * D1[m + l, n + l] - rhs1))
                Q = (m * m + n * n - 2 * m * n * c) / (s * s)
                rhs2 = -c / s * D1[m + l, n + l] + (Q - l * (l + 1)) * D[m + l, n + l]
                worst2 = max(worst2, abs(D2[m + l, n + l] - rhs2) * s * s)
    assert worst1 < 1e-12
    assert worst2 < 1e-12
