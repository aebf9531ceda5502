"""Pins for the oracle's translation search and 6-D alternation (the appendix
"Alternating search over rotations and translations"): the volume pose
transform against grid-exact rotations and shifts, the interpolated
correlation against the circular correlation's definition, planted integer
and fractional shifts, and a planted 6-D pose on noiseless volumes."""
import math

import numpy as np

import oracle as O
import synth
from oracle import translation as T

RNG = np.random.default_rng(31)


def test_transform_volume_grid_exact_cases():
    N = 16
    v = RNG.standard_normal((N, N, N)).astype(np.float32)
    assert np.array_equal(T.transform_volume(v), v)
    # +90 degrees about z maps voxel centres onto voxel centres (c0 = N/2 is one):
    # out(x, y, z) = v(R^T (x - c0) + c0) = v(c0 + (y - c0), c0 - (x - c0), z)
    Rz = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    out = T.transform_volume(v, Rz)
    c = N // 2
    for k, j, i in [(3, 4, 5), (0, 8, 8), (9, 2, 15), (7, 7, 1)]:
        xs, ys = c + (j - c), c - (i - c)
        want = v[k, ys, xs] if 0 <= xs < N and 0 <= ys < N else 0.0
        assert out[k, j, i] == want
    # an integer shift is a zero-filled translation
    out = T.transform_volume(v, None, np.array([2.0, -1.0, 3.0]))
    ref = np.zeros_like(v)
    ref[3:, :N - 1, 2:] = v[:N - 3, 1:, :N - 2]
    assert np.array_equal(out, ref)
    # a half-voxel shift of an affine ramp is exact away from the border
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    ramp = (0.5 * x - 0.25 * y + 0.125 * z + 1.0).astype(np.float32)
    out = T.transform_volume(ramp, None, np.array([0.5, 0.0, 0.0]))
    want = 0.5 * (x - 0.5) - 0.25 * y + 0.125 * z + 1.0
    assert np.abs(out[:, :, 1:] - want[:, :, 1:]).max() < 1e-6


def test_interpolated_correlation_equals_circular_definition_at_integer_shifts():
    for N in (12, 13):
        f = RNG.standard_normal((N, N, N)).astype(np.float32)
        u = RNG.standard_normal((N, N, N)).astype(np.float32)
        X = T.cross_spectrum(f, u)
        w = np.arange(-3, 4, dtype=np.float64)
        v = T.cc_interp(X, w, w, w)
        scale = np.sqrt(np.sum(f.astype(np.float64) ** 2) * np.sum(u.astype(np.float64) ** 2))
        for tz in range(-3, 4):
            for ty in (-3, 0, 2):
                for tx in (-1, 3):
                    ref = T.circular_cc(f, u, (tx, ty, tz))
                    assert abs(v[tz + 3, ty + 3, tx + 3] - ref) < 1e-12 * scale


def test_planted_integer_circular_shift_found_exactly():
    N = 16
    u = RNG.standard_normal((N, N, N)).astype(np.float32)
    for t in [(2, -3, 1), (0, 0, 0), (-4, 4, -4)]:
        f = np.roll(u, (t[2], t[1], t[0]), axis=(0, 1, 2))      # f(x) = u(x - t)
        for U in (1, 10):
            got, cc, fl = T.shift_search(f, u, 4, U)
            assert np.array_equal(got, np.array(t, dtype=float))
            assert abs(cc - np.sum(u.astype(np.float64) ** 2)) < 1e-9 * cc
            assert fl == (32 if max(abs(a) for a in t) == 4 else 0)


def test_planted_fractional_shift_found_to_the_grid_spacing():
    """f is u translated by a fractional t* through the Fourier shift theorem
    (odd N: no Nyquist term, so f is real and exactly band-limited); the
    correlation's interpolant then peaks at t*, and the fine grid finds it to
    half its spacing."""
    N = 15
    u = RNG.standard_normal((N, N, N))
    k = np.fft.fftfreq(N) * N
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    ts = np.array([0.3, -1.27, 2.61])
    F = np.fft.fftn(u) * np.exp(-2j * np.pi * (kx * ts[0] + ky * ts[1] + kz * ts[2]) / N)
    f = np.fft.ifftn(F).real
    assert np.abs(np.fft.ifftn(F).imag).max() < 1e-12
    for U, tol in ((10, 0.05), (20, 0.025)):
        got, cc, _ = T.shift_search(f, u, 4, U)
        assert np.abs(got - ts).max() <= tol + 1e-12, (U, got)
        assert np.array_equal(got - np.round(got * U) / U, np.zeros(3))


def test_planted_pose_recovered_by_the_alternation():
    """Noiseless exact renderings f = g* o S_tau* h: the alternation, given enough
    rounds, recovers both the rotation and the shift (block coordinate ascent
    converges one round at a time from tau = 0)."""
    w = synth.WORKLOADS["shift32"]
    d = synth.make_batch(w, exact_rotation=True, noise=False)
    out = T.align6d_batch(d["particles"].numpy(), d["templates"].numpy(), S=w.n_shells,
                          r_max=w.r_max, L0=w.L0, K=w.K, P=w.P, M_iter=w.M_iter,
                          L_sched=w.L_sched, rounds=5, max_shift=w.max_shift, upsample=20)
    for b in range(w.B):
        assert math.degrees(O.rotation_angle(out["R"][b], d["R_true"][b])) < 0.25
        assert np.abs(out["tau"][b] - d["tau_true"][b]).max() < 0.08
        assert np.allclose(out["R"][b] @ out["tau"][b], out["t"][b], atol=1e-12)
