"""Pins for the oracle's gradient of the refined score with respect to the
template: the coefficient gradient at a fixed rotation, the implicit-function
term through the refined rotation, the transpose of the analysis map, and the
whole path (analysis -> search -> Newton -> argmax) against central
differences."""
import numpy as np

import oracle as O
import synth

RNG = np.random.default_rng(77)


def rand_coef(L, S):
    """Coefficients of real shell functions: [S][lm], m >= 0, real for m = 0."""
    a = RNG.normal(size=(S, O.lm_size(L))) + 1j * RNG.normal(size=(S, O.lm_size(L)))
    for l in range(L + 1):
        a[:, O.lm_index(l, 0)] = a[:, O.lm_index(l, 0)].real
    return a


def test_implicit_shift_matches_numpy_solve():
    H = RNG.normal(size=(3, 3))
    H = -(H @ H.T + 0.5 * np.eye(3))
    g = RNG.normal(size=3)
    v, fl = O.implicit_shift(g, H)
    assert fl == 0
    np.testing.assert_allclose(v, np.linalg.solve(H, g), rtol=1e-13, atol=1e-14)
    v0, fl0 = O.implicit_shift(g, np.outer(g, g))  # rank one: no isolated maximum
    assert fl0 == 1 and np.all(v0 == 0)


def test_coef_grad_at_fixed_rotation_matches_central_differences():
    """dC_L(theta)/dh at fixed theta (c linear in conj(h)); the stored n > 0
    coefficient also drives h_{l,-n}, n = 0 drives only itself."""
    L, S, R = 6, 3, 10.0
    f, h = rand_coef(L, S), rand_coef(L, S)
    abg = np.array([0.7, 1.1, 2.3])

    def lam(hh):
        return O.objective(O.correlate(f, hh, S, R, L), L, *abg)[0]

    G = O.coef_grad(f, S, R, L, abg)
    eps = 1e-6
    for (s, l, n) in [(0, 0, 0), (1, 3, 0), (2, 4, 2), (0, 6, 5), (1, 5, 1), (2, 6, 6)]:
        i = O.lm_index(l, n)
        for part in ((1.0,) if n == 0 else (1.0, 1j)):
            hp, hm = h.copy(), h.copy()
            hp[s, i] += eps * part
            hm[s, i] -= eps * part
            fd = (lam(hp) - lam(hm)) / (2 * eps)
            an = G[s, i].real if part == 1.0 else G[s, i].imag
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (s, l, n, part, fd, an)


def test_analysis_adjoint_is_the_transpose():
    """<A vol, G> = <vol, A^T G> with <a, b> = sum Re(conj(a) b): the voxel
    gradient is the exact transpose of sampling + SH analysis."""
    N, S, L = 16, 4, 7
    R = N / 2 - 1
    vol = RNG.normal(size=(N, N, N)).astype(np.float32)
    G = rand_coef(L, S)
    lhs = np.sum((np.conj(G) * O.analyze_volume(vol, S, R, L)).real)
    rhs = np.sum(vol.astype(np.float64) * O.analysis_adjoint(G, N, S, R, L))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _small_pair():
    w = synth.WORKLOADS["small32"]
    b = synth.make_batch(w)
    return w, b["particles"].numpy(), b["templates"].numpy()


def test_implicit_term_is_the_gradient_at_the_maximum_to_second_order():
    """Away from the maximiser by delta, the partial gradient errs by O(delta),
    the gradient with the implicit term -grad^T H^{-1} d grad/dh by
    O(delta^2): it equals the derivative of max_theta C_L to second order."""
    w, parts, temps = _small_pair()
    S, L, R = w.n_shells, w.L_sched[-1], w.N / 2 - 1
    f = O.analyze_volume(parts[0], S, R, L)
    h = O.analyze_volume(temps[0], S, R, L)
    c = O.correlate(f, h, S, R, L)
    res = O.align_batch(parts, temps, S=S, r_max=R, L0=w.L0, K=w.K, P=w.P, M_iter=w.M_iter,
                        L_sched=list(w.L_sched))
    th, _, _ = O.newton_march(c, [L], 20, res["euler"][0], step_tol=0.0, accept_tol=1e-15)
    G_hat = O.coef_grad(f, S, R, L, th)
    nrm = np.linalg.norm(G_hat)
    errs = []
    for dlt in (3e-3, 1e-3):
        th1 = th + np.array([1.0, -2.0, 1.5]) * dlt
        _, g1, H1, _ = O.objective(c, L, *th1, derivs=True)
        v, fl = O.implicit_shift(g1, H1)
        assert fl == 0
        e_impl = np.linalg.norm(O.coef_grad(f, S, R, L, th1, v) - G_hat) / nrm
        e_part = np.linalg.norm(O.coef_grad(f, S, R, L, th1) - G_hat) / nrm
        assert e_impl < 0.1 * e_part
        errs.append(e_impl)
    assert errs[1] < errs[0] / 5  # quadratic: a factor of 9 for delta / 3


def test_refined_score_gradient_matches_central_differences():
    """Lambda = C_{L_J}(theta*) from the whole path (search, Newton march,
    argmax) at template coefficients h + t A v, A the analysis map and v a
    random unit voxel direction; (Lambda(t) - Lambda(-t)) / 2t against
    <dLambda/dvoxel, v>, t = 1e-6 ||template|| (FP64)."""
    w, parts, temps = _small_pair()
    S, R, N = 8, w.N / 2 - 1, w.N
    L_sched = [6, 10, 14]
    L = L_sched[-1]
    kw = dict(S=S, r_max=R, L0=6, K=1, P=4, M_iter=3, L_sched=L_sched, N=N)
    f = O.analyze_volume(parts[0], S, R, L)[None]
    h = O.analyze_volume(temps[0], S, R, L)
    base = O.align_coefs_batch(f, h, **kw)
    G, out4, flags = O.template_grad_batch(f, h, base["euler"], S=S, r_max=R, L_sched=L_sched, N=N)
    assert flags[0] == 0
    assert abs(out4[0, 3] - base["score"][0]) <= 1e-12 * abs(base["score"][0])
    vox_grad = O.analysis_adjoint(G[0], N, S, R, L)
    scale = 1e-6 * float(np.linalg.norm(temps[0].astype(np.float64)))
    fd, an = [], []
    for _ in range(4):
        v = RNG.normal(size=(N, N, N))
        v = (v / np.linalg.norm(v)).astype(np.float32)
        hv = O.analyze_volume(v, S, R, L)
        sp = O.align_coefs_batch(f, h + scale * hv, **kw)["score"][0]
        sm = O.align_coefs_batch(f, h - scale * hv, **kw)["score"][0]
        fd.append((sp - sm) / (2 * scale))
        an.append(float(np.sum(vox_grad * v.astype(np.float64))))
        # the same number through the coefficient gradient
        assert abs(np.sum((np.conj(G[0]) * hv).real) - an[-1]) <= 1e-12 * np.abs(vox_grad).sum()
    fd, an = np.array(fd), np.array(an)
    assert np.max(np.abs(fd - an)) <= 1e-6 * np.max(np.abs(an)), (fd, an)


def test_align_from_coefficients_equals_align_from_volumes():
    """The coefficient-input entry of the oracle's Algorithm 1 is the volume
    entry minus the analysis: same rotations and scores, bit for bit."""
    w, parts, temps = _small_pair()
    S, R, L = w.n_shells, w.N / 2 - 1, w.L_sched[-1]
    kw = dict(S=S, r_max=R, L0=w.L0, K=w.K, P=w.P, M_iter=w.M_iter, L_sched=list(w.L_sched))
    ref = O.align_batch(parts, temps, **kw)
    f = O.analyze_volume(parts[0], S, R, L)[None]
    h = O.analyze_volume(temps[0], S, R, L)[None]
    got = O.align_coefs_batch(f, h, N=w.N, **kw)
    assert np.array_equal(got["euler"], ref["euler"])
    assert np.array_equal(got["score"], ref["score"])
    assert np.array_equal(got["best_p"], ref["best_p"])
