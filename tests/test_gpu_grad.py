"""Template gradient of the refined scores (the 64^3 shared-template
workload: 512 particles, 32 shells, final L = 32, SNR 0.2).

FP64 gradient against the oracle's adjoint on a sample; against central
differences of the whole GPU path (analysis -> contraction -> SOFFT search
-> Newton march -> argmax) on 64 random voxel directions at the full batch;
per-template and shared-template forms against each other; the autograd
function against the C-ABI call; FP32 against FP64."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_2603_15285_gb300 as m
import synth
from gpu_helpers import coef_to_complex

pytestmark = pytest.mark.gpu
W = synth.WORKLOADS["grad64"]
SAMPLE = 4


@pytest.fixture(scope="module")
def batch():
    import __graft_entry__
    __graft_entry__.build()
    return synth.make_batch(W, device="cuda")


@pytest.fixture(scope="module")
def plan64():
    return m.plan_for_workload(W, precision=m.FP64)


def forward(plan, parts, temp):
    f = m.matcha_analyze(plan, parts)
    h = m.matcha_analyze(plan, temp)
    return f, h, m.align_from_coefs(plan, f, h, 0)


def test_template_grad_matches_oracle_adjoint(batch, plan64):
    parts = batch["particles"][:SAMPLE].contiguous()
    temp = batch["templates"]
    f, h, out = forward(plan64, parts, temp)
    g = m.matcha_template_grad(plan64, f, out["c"], out["euler"])
    torch.cuda.synchronize()

    pn, tn = parts.cpu().numpy(), temp.cpu().numpy()
    S, R, L, N = W.n_shells, W.r_max, W.L_sched[-1], W.N
    ref = O.align_batch(pn, tn, S=S, r_max=R, L0=W.L0, K=W.K, P=W.P, M_iter=W.M_iter,
                        L_sched=list(W.L_sched))
    eu = out["euler"].cpu().numpy()
    for b in range(SAMPLE):
        assert O.rotation_angle(O.euler_to_matrix(*eu[b]), ref["R"][b]) < 1e-8
    fo = np.stack([O.analyze_volume(pn[b], S, R, L) for b in range(SAMPLE)])
    ho = O.analyze_volume(tn[0], S, R, L)
    Go, out4, fl = O.template_grad_batch(fo, ho, ref["euler"], S=S, r_max=R,
                                         L_sched=list(W.L_sched), N=N)
    assert np.all(fl == 0) and np.all(g["flags"].cpu().numpy() == 0)
    sh = g["shift"].cpu().numpy()
    np.testing.assert_allclose(sh[:, 3], out4[:, 3], rtol=1e-10)
    Gsum = Go.sum(axis=0)
    Gg = coef_to_complex(g["coef_grad"][0])
    # element by element: every coefficient (real and imaginary parts, n = 0 and
    # the mirrored n > 0 terms alike) and every voxel within 1e-6 of the largest
    err_c = max(np.abs(Gg.real - Gsum.real).max(), np.abs(Gg.imag - Gsum.imag).max()) / np.abs(Gsum).max()
    vo = O.analysis_adjoint(Gsum, N, S, R, L)
    vg = g["vox_grad"][0].cpu().numpy()
    err_v = np.abs(vg - vo).max() / np.abs(vo).max()
    # the per-particle gradients, each against its own oracle adjoint
    per = m.matcha_template_grad(plan64, f, out["c"], out["euler"], template_batch_stride=1)
    torch.cuda.synchronize()
    err_b = 0.0
    for b in range(SAMPLE):
        Gb = coef_to_complex(per["coef_grad"][b])
        err_b = max(err_b, max(np.abs(Gb.real - Go[b].real).max(), np.abs(Gb.imag - Go[b].imag).max())
                    / np.abs(Go[b]).max())
    print("template grad vs oracle: coef %.2e, voxel %.2e, per particle %.2e (max |diff| / max |G|)"
          % (err_c, err_v, err_b))
    assert err_c < 1e-6 and err_v < 1e-6 and err_b < 1e-6


def test_template_grad_matches_central_differences(batch, plan64):
    """Lambda(t) = sum_b C_{L_J}(theta*_b) for template coefficients h + t A v
    (A the analysis map, linear, so this is the template h + t v), v a random
    unit voxel direction; (Lambda(t) - Lambda(-t)) / 2t with t = 1e-6
    ||template|| against <dLambda/dvoxel, v>, FP64, on the full batch."""
    parts, temp = batch["particles"], batch["templates"]
    f, h, out = forward(plan64, parts, temp)
    g = m.matcha_template_grad(plan64, f, out["c"], out["euler"])
    vg = g["vox_grad"][0]
    t = 1e-6 * float(torch.linalg.vector_norm(temp.double()))
    gen = torch.Generator(device="cuda").manual_seed(515)

    def lam(hc):
        sc = m.align_from_coefs(plan64, f, hc, 0)["score"].cpu().numpy()
        return math.fsum(sc.tolist())

    fd, an = [], []
    for _ in range(64):
        v = torch.randn((1,) + tuple(temp.shape[1:]), generator=gen, device="cuda", dtype=torch.float64)
        v = (v / torch.linalg.vector_norm(v)).float()
        hv = m.matcha_analyze(plan64, v)
        fd.append((lam(h + t * hv) - lam(h - t * hv)) / (2 * t))
        an.append(float((vg * v[0].double()).sum()))
    fd, an = np.array(fd), np.array(an)
    err = np.abs(fd - an).max() / np.abs(an).max()
    print("template grad vs central differences (64 directions, B=%d): max err %.2e of max |<g,v>|"
          % (parts.shape[0], err))
    assert err <= 1e-6


def test_per_template_form_and_weights(batch, plan64):
    B = 8
    parts = batch["particles"][:B].contiguous()
    temp = batch["templates"]
    f, h, out = forward(plan64, parts, temp)
    w = torch.linspace(-1.0, 2.0, B, dtype=torch.float64, device="cuda")
    shared = m.matcha_template_grad(plan64, f, out["c"], out["euler"], weight=w)
    per = m.matcha_template_grad(plan64, f, out["c"], out["euler"], template_batch_stride=1)
    cs = (per["coef_grad"] * w[:, None, None, None]).sum(0)
    vs = (per["vox_grad"] * w[:, None, None, None]).sum(0)
    torch.testing.assert_close(shared["coef_grad"][0], cs, rtol=1e-11, atol=1e-11 * cs.abs().max().item())
    torch.testing.assert_close(shared["vox_grad"][0], vs, rtol=1e-10, atol=1e-11 * vs.abs().max().item())


def test_autograd_function_matches_c_abi(batch, plan64):
    from paper_2603_15285_gb300.autograd import refined_scores, refined_scores_from_coefs
    B = 8
    parts = batch["particles"][:B].contiguous()
    temp = batch["templates"][0].clone().requires_grad_(True)
    scores, euler = refined_scores(temp, parts, plan64)
    w = torch.linspace(0.5, 1.5, B, dtype=torch.float64, device="cuda")
    (scores * w).sum().backward()
    f, h, out = forward(plan64, parts, batch["templates"])
    torch.testing.assert_close(scores.detach(), out["score"], rtol=0, atol=0)
    g = m.matcha_template_grad(plan64, f, out["c"], out["euler"], weight=w)
    torch.testing.assert_close(temp.grad, g["vox_grad"][0].float(), rtol=1e-6, atol=1e-9)
    hc = h[0].clone().requires_grad_(True)
    s2, _ = refined_scores_from_coefs(hc, f, plan64)
    (s2 * w).sum().backward()
    torch.testing.assert_close(hc.grad, g["coef_grad"][0], rtol=0, atol=0)


def test_fp32_template_grad_close_to_fp64(batch, plan64):
    B = 64
    parts = batch["particles"][:B].contiguous()
    temp = batch["templates"]
    f, h, out = forward(plan64, parts, temp)
    g64 = m.matcha_template_grad(plan64, f, out["c"], out["euler"])
    p32 = m.plan_for_workload(W, precision=m.FP32)
    f32, h32, out32 = forward(p32, parts, temp)
    g32 = m.matcha_template_grad(p32, f32, out32["c"], out32["euler"])
    a, b = g64["vox_grad"][0], g32["vox_grad"][0]
    err = float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(a))
    ca, cb = g64["coef_grad"][0], g32["coef_grad"][0].double()
    errc = float(torch.linalg.vector_norm(ca - cb) / torch.linalg.vector_norm(ca))
    print("FP32 template grad vs FP64: voxel %.2e, coef %.2e (relative 2-norm, B=%d)" % (err, errc, B))
    assert err < 1e-3 and errc < 1e-3
