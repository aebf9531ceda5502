"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 plans: SH coefficients and c^l_mn to 1e-12 of their scale, SOFFT grid
to 1e-12, top-P grid indices bit-exact (grid values closer than 1e-12 of the
grid's scale count as ties), refined rotations to 1e-8 rad, scores to 1e-10
relative.  FP32 plans: refined rotations within 0.05 degrees of the oracle.
"""
import dataclasses
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_2603_15285_gb300 as m
import synth
from gpu_helpers import coef_to_complex, corr_to_oracle, oracle_align

pytestmark = pytest.mark.gpu

SMALL = synth.WORKLOADS["small32"]
# ragged case: odd sizes, few shells, short schedule, several particles
RAGGED = dataclasses.replace(SMALL, name="ragged", B=3, N=21, n_blobs=9, ball_radius=7.0,
                             n_shells=5, L_sched=(3, 5, 7), L0=3, K=1, P=5, base_seed=77)
DEG = math.pi / 180


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def gen(w, B=None, start=0):
    d = synth.make_batch(w, B=B, start=start)
    return d, d["particles"].cuda().contiguous(), d["templates"].cuda().contiguous()


@pytest.mark.parametrize("w", [SMALL, RAGGED], ids=lambda w: w.name)
def test_plan_tables_match_oracle(w):
    plan = m.plan_for_workload(w)
    r, wr = O.radial_nodes(w.n_shells, w.r_max)
    x, wx = O.gauss_legendre(w.L_final + 1)
    for which, ref in enumerate([r, wr, x, wx]):
        got = plan.table(which)
        assert np.allclose(got, ref, rtol=1e-14, atol=1e-14 * np.abs(ref).max())


@pytest.mark.parametrize("w", [SMALL, RAGGED], ids=lambda w: w.name)
def test_analyze_fp64_matches_oracle(w):
    d, parts, temps = gen(w)
    plan = m.plan_for_workload(w)
    f = coef_to_complex(m.matcha_analyze(plan, parts))
    h = coef_to_complex(m.matcha_analyze(plan, temps))
    for b in range(parts.shape[0]):
        ref = O.analyze_volume(d["particles"][b].numpy(), w.n_shells, w.r_max, w.L_final)
        assert np.abs(f[b] - ref).max() <= 1e-12 * np.abs(ref).max()
    ref = O.analyze_volume(d["templates"][0].numpy(), w.n_shells, w.r_max, w.L_final)
    assert np.abs(h[0] - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("w", [SMALL, RAGGED], ids=lambda w: w.name)
def test_correlate_fp64_matches_oracle(w):
    d, parts, temps = gen(w)
    plan = m.plan_for_workload(w)
    f = m.matcha_analyze(plan, parts)
    h = m.matcha_analyze(plan, temps)
    c = m.matcha_correlate_coeffs(plan, f, h, 1)
    fc, hc = coef_to_complex(f), coef_to_complex(h)
    for b in range(parts.shape[0]):
        ref = O.correlate(fc[b], hc[b], w.n_shells, w.r_max, w.L_final)
        got = corr_to_oracle(c[b], w.L_final)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def _tie_tolerant_equal(got_idx, ref_idx, grid, tol):
    """Index lists equal, except that positions whose grid values differ by
    less than tol may swap."""
    if list(got_idx) == list(ref_idx):
        return True
    if len(got_idx) != len(ref_idx):
        return False
    for a, b in zip(got_idx, ref_idx):
        if a != b and abs(grid[a] - grid[b]) > tol:
            return False
    return True


@pytest.mark.parametrize("w", [SMALL, RAGGED], ids=lambda w: w.name)
def test_soft_grid_and_top_p_fp64(w):
    d, parts, temps = gen(w)
    plan = m.plan_for_workload(w)
    c = m.matcha_correlate_coeffs(plan, m.matcha_analyze(plan, parts), m.matcha_analyze(plan, temps), 1)
    s = m.matcha_soft_search(plan, c)
    n = plan.info.soft_n
    for b in range(parts.shape[0]):
        cref = corr_to_oracle(c[b], w.L_final)
        gref = O.soft_grid(cref, w.L0, w.K)
        ggot = s["grid"][b].cpu().numpy().ravel()
        scale = np.abs(gref).max()
        assert np.abs(ggot - gref).max() <= 1e-12 * scale
        idx, sc = O.local_maxima_topk(gref, n, w.P)
        nc = int(s["n_cand"][b])
        assert nc == len(idx)
        gidx = s["idx"][b, :nc].cpu().numpy()
        assert _tie_tolerant_equal(gidx, idx, gref, 1e-12 * scale)
        assert np.all(s["idx"][b, nc:].cpu().numpy() == -1)
        e = s["euler"][b, :nc].cpu().numpy()
        for q in range(nc):
            assert np.allclose(e[q], O.soft_angles(n, int(gidx[q])), atol=1e-15)


@pytest.mark.parametrize("w", [SMALL, RAGGED], ids=lambda w: w.name)
def test_newton_fp64_matches_oracle(w):
    d, parts, temps = gen(w)
    plan = m.plan_for_workload(w)
    c = m.matcha_correlate_coeffs(plan, m.matcha_analyze(plan, parts), m.matcha_analyze(plan, temps), 1)
    s = m.matcha_soft_search(plan, c)
    e0 = s["euler"].clone()
    out = m.matcha_newton_march(plan, c, s["n_cand"], s["euler"])
    for b in range(parts.shape[0]):
        cref = corr_to_oracle(c[b], w.L_final)
        for q in range(int(s["n_cand"][b])):
            x, sc, fl = O.newton_march(cref, w.L_sched, w.M_iter, e0[b, q].cpu().numpy(), step_tol=1e-9)
            ge = out["euler"][b, q].cpu().numpy()
            ang = O.rotation_angle(O.euler_to_matrix(*ge), O.euler_to_matrix(*x))
            assert ang < 1e-8, (b, q, ang)
            assert abs(out["score"][b, q].item() - sc) <= 1e-10 * abs(sc)


@pytest.mark.parametrize("w", [SMALL, RAGGED], ids=lambda w: w.name)
def test_align_fp64_end_to_end(w):
    d, parts, temps = gen(w)
    plan = m.plan_for_workload(w)
    out = m.matcha_align(plan, parts, temps)
    ref = oracle_align(w, d["particles"].numpy(), d["templates"].numpy())
    R = out["R"].cpu().numpy()
    for b in range(parts.shape[0]):
        assert O.rotation_angle(R[b], ref["R"][b]) < 1e-8
        assert abs(out["score"][b].item() - ref["score"][b]) <= 1e-10 * abs(ref["score"][b])
        assert int(out["best_p"][b]) == ref["best_p"][b]
        assert np.allclose(R[b], O.euler_to_matrix(*out["euler"][b].cpu().numpy()), atol=1e-14)


@pytest.mark.parametrize("w", [SMALL, RAGGED], ids=lambda w: w.name)
def test_align_fp32_within_005_degrees(w):
    d, parts, temps = gen(w)
    plan = m.plan_for_workload(w, precision=m.FP32)
    out = m.matcha_align(plan, parts, temps)
    ref = oracle_align(w, d["particles"].numpy(), d["templates"].numpy())
    R = out["R"].cpu().numpy()
    for b in range(parts.shape[0]):
        assert O.rotation_angle(R[b], ref["R"][b]) < 0.05 * DEG


def test_shared_template_and_per_particle_P():
    w = dataclasses.replace(SMALL, B=3, shared_template=True, P=6)
    d, parts, temps = gen(w)
    assert temps.shape[0] == 1
    plan = m.plan_for_workload(w)
    P_per = torch.tensor([6, 2, 4], dtype=torch.int32, device="cuda")
    out = m.matcha_align(plan, parts, temps, P_per=P_per)
    ref = oracle_align(w, d["particles"].numpy(), d["templates"].numpy(), P_per=np.array([6, 2, 4]))
    R = out["R"].cpu().numpy()
    for b in range(3):
        assert O.rotation_angle(R[b], ref["R"][b]) < 1e-8
        assert int(out["flags"][b]) & 8 == ref["flags"][b] & 8


def test_empty_batch_and_errors():
    plan = m.plan_for_workload(SMALL)
    z = torch.empty((0, 32, 32, 32), dtype=torch.float32, device="cuda")
    out = m.matcha_align(plan, z, z)
    assert out["euler"].shape == (0, 3)
    d, parts, temps = gen(SMALL)
    small_ws = torch.empty((1024,), dtype=torch.uint8, device="cuda")
    with pytest.raises(m.MatchaError, match="workspace"):
        m.matcha_align(plan, parts, temps, ws=small_ws)
    with pytest.raises(m.MatchaError):
        m.Plan(32, 12, 8, 2, 8, 3, (8, 12, 12))


def test_nan_volume_sets_flag_and_returns():
    d, parts, temps = gen(SMALL)
    bad = parts.clone()
    bad[0, 16, 16, 16] = float("nan")
    plan = m.plan_for_workload(SMALL)
    out = m.matcha_align(plan, bad, temps)
    torch.cuda.synchronize()
    assert int(out["best_p"][0]) == -1 or int(out["flags"][0]) & 1


def test_host_buffers_match_device_path():
    d, parts, temps = gen(SMALL)
    plan = m.plan_for_workload(SMALL)
    dev = m.matcha_align(plan, parts, temps)
    host = m.matcha_align_host(plan, d["particles"].numpy(), d["templates"].numpy())
    assert np.array_equal(host["R"], dev["R"].cpu().numpy())
    assert np.array_equal(host["score"], dev["score"].cpu().numpy())


def _brute_top_p(grid, n, P):
    """Local maxima in (value desc, index asc) order, decided in grid's own dtype."""
    g = grid.reshape(n, n, n)
    out = []
    for i in range(n):
        for k in range(n):
            for j in range(n):
                p = (i * n + k) * n + j
                v = g[i, k, j]
                ok = not np.isnan(v)
                for di in (-1, 0, 1):
                    for dk in (-1, 0, 1):
                        for dj in (-1, 0, 1):
                            if not ok or (di, dk, dj) == (0, 0, 0) or not 0 <= k + dk < n:
                                continue
                            q = (((i + di) % n) * n + k + dk) * n + (j + dj) % n
                            wv = grid[q]
                            ok = v > wv or (v == wv and p < q)
                if ok:
                    out.append((-float(v), p))
    out.sort()
    return [p for _, p in out[:P]]


@pytest.mark.parametrize("w", [SMALL, RAGGED], ids=lambda w: w.name)
def test_soft_grid_and_top_p_fp32(w):
    d, parts, temps = gen(w)
    plan = m.plan_for_workload(w, precision=m.FP32)
    c = m.matcha_correlate_coeffs(plan, m.matcha_analyze(plan, parts), m.matcha_analyze(plan, temps), 1)
    s = m.matcha_soft_search(plan, c)
    n = plan.info.soft_n
    for b in range(parts.shape[0]):
        cref = corr_to_oracle(c[b].double(), w.L_final)
        gref = O.soft_grid(cref, w.L0, w.K)
        ggot = s["grid"][b].cpu().numpy().ravel()
        assert np.abs(ggot - gref).max() <= 1e-5 * np.abs(gref).max()
        nc = int(s["n_cand"][b])
        assert list(s["idx"][b, :nc].cpu().numpy()) == _brute_top_p(ggot, n, w.P)


def test_host_buffers_in_several_chunks_match_device_path():
    """600 particles: the host path copies and aligns them in 3 chunks."""
    w = dataclasses.replace(SMALL, B=600)
    d, parts, temps = gen(w)
    plan = m.plan_for_workload(w, precision=m.FP32)
    dev = m.matcha_align(plan, parts, temps)
    hp = d["particles"].pin_memory()
    ht = d["templates"].pin_memory()
    host = m.matcha_align_host(plan, hp, ht)
    assert np.array_equal(host["R"], dev["R"].cpu().numpy())
    assert np.array_equal(host["best_p"], dev["best_p"].cpu().numpy())


def test_align_replays_in_a_cuda_graph():
    """matcha_align is stream-ordered and allocates nothing, so it can be captured
    into a CUDA graph; replays give the eager results bit for bit."""
    w = synth.WORKLOADS["batch64"]
    B = 8
    d = synth.make_batch(w, B=B, device="cuda")
    parts, temps = d["particles"].contiguous(), d["templates"].contiguous()
    plan = m.plan_for_workload(w, precision=m.FP32)
    ws = m.alloc_workspace(plan, B)
    eager = {k: v.clone() for k, v in m.matcha_align(plan, parts, temps, ws=ws).items()}
    out = {k: torch.empty_like(v) for k, v in eager.items()}
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        m.matcha_align(plan, parts, temps, ws=ws, out=out)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        m.matcha_align(plan, parts, temps, ws=ws, out=out)
    for rep in range(2):
        for v in out.values():
            v.zero_()
        g.replay()
        torch.cuda.synchronize()
        for k in eager:
            assert torch.equal(out[k], eager[k]), (rep, k)


@pytest.mark.parametrize("prec", [m.FP64, m.FP32, m.TF32])
def test_poisoned_workspace_gives_the_same_results(prec):
    """A workspace filled with NaN bit patterns (0xFF bytes) before the call
    gives bit-identical results: no kernel reads workspace it has not written."""
    d, parts, temps = gen(SMALL)
    plan = m.plan_for_workload(SMALL, precision=prec)
    ws = m.alloc_workspace(plan, parts.shape[0])
    ws.zero_()
    ref = {k: v.clone() for k, v in m.matcha_align(plan, parts, temps, ws=ws).items()}
    ws.fill_(255)
    out = m.matcha_align(plan, parts, temps, ws=ws)
    torch.cuda.synchronize()
    for k in ref:
        assert torch.equal(out[k], ref[k]), k
    assert plan.device_status() == 0


def test_c_program_through_the_c_abi_matches_python(tmp_path):
    """A C program that links only the library (and the CUDA runtime for its
    workspace) gives the same results as the Python binding."""
    import os
    import subprocess
    w = synth.WORKLOADS["small32"]
    d = synth.make_batch(w, B=3)
    parts, temps = d["particles"].numpy(), d["templates"].numpy()
    pf, tf = tmp_path / "p.f32", tmp_path / "t.f32"
    parts.astype(np.float32).tofile(pf)
    temps.astype(np.float32).tofile(tf)
    exe = os.path.join(os.path.dirname(m.LIB_PATH), "align_from_c")
    args = [exe, str(w.N), str(w.n_shells), str(w.L0), str(w.K), str(w.P), str(w.M_iter), "3",
            str(pf), str(tf)] + [str(L) for L in w.L_sched[1:]]
    out = subprocess.run(args, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    rows = [line.split() for line in out.stdout.strip().splitlines()]
    plan = m.plan_for_workload(w, precision=m.FP64)
    ref = m.matcha_align_host(plan, parts, temps)
    for b, r in enumerate(rows):
        assert int(r[1]) == int(ref["best_p"][b])
        assert float(r[2]) == ref["score"][b]
        assert [float(x) for x in r[3:6]] == list(ref["euler"][b])


@pytest.mark.parametrize("name", ["batch64", "grad64"])
def test_concurrent_parts_equal_single_passes(name):
    """512 particles in one call run as four concurrent parts; the same
    particles in four calls of 128 run in one pass each: identical results,
    with per-particle candidate counts (batch64) and with one shared template
    analysed once before the parts fork (grad64)."""
    w = synth.WORKLOADS[name]
    B = 512
    d = synth.make_batch(w, B=B, device="cuda")
    parts, temps = d["particles"].contiguous(), d["templates"].contiguous()
    shared = temps.shape[0] == 1
    P_per = None
    if not shared:
        rng = np.random.default_rng(5)
        P_per = torch.from_numpy(rng.integers(4, w.P + 1, size=B).astype(np.int32)).cuda()
    plan = m.plan_for_workload(w, precision=m.FP32)
    whole = {k: v.clone() for k, v in m.matcha_align(plan, parts, temps, P_per=P_per).items()}
    for c in range(4):
        sl = slice(128 * c, 128 * (c + 1))
        t = temps if shared else temps[sl].contiguous()
        pp = None if P_per is None else P_per[sl].contiguous()
        out = m.matcha_align(plan, parts[sl].contiguous(), t, P_per=pp)
        torch.cuda.synchronize()
        for k in whole:
            assert torch.equal(out[k], whole[k][sl]), (name, c, k)
