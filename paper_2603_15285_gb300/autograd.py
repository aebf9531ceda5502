"""Differentiable refined scores (torch.autograd over the C ABI).

``refined_scores(template, particles, plan)`` returns C_{L_J}(theta*_b) of
every particle against one shared template (Algorithm 1: analysis, SOFFT
search, Newton march, argmax); its backward is ``matcha_template_grad``:
the gradient with respect to the template voxels, with the implicit-function
term through the refined rotations (Section 2.2).  The ``*_from_coefs``
form takes the template's SH coefficients and differentiates with respect
to them.  All arithmetic runs in the library's kernels.
"""
from __future__ import annotations

from . import (MatchaError, Plan, align_from_coefs, matcha_analyze, matcha_template_grad, _torch)


def _function_classes():
    T = _torch()  # raises without a CUDA device (no CPU path)

    class _Voxels(T.autograd.Function):
        @staticmethod
        def forward(ctx, template, particles, plan):
            f = matcha_analyze(plan, particles)
            h = matcha_analyze(plan, template.reshape(1, *template.shape[-3:]).contiguous())
            out = align_from_coefs(plan, f, h, 0)
            ctx.plan = plan
            ctx.tdtype = template.dtype
            ctx.save_for_backward(f, out["c"], out["euler"])
            ctx.mark_non_differentiable(out["euler"])
            return out["score"], out["euler"]

        @staticmethod
        def backward(ctx, g_score, g_euler):
            f, c, euler = ctx.saved_tensors
            if g_score is None:  # only the (non-differentiable) rotations were used
                return None, None, None
            w = g_score.to(T.float64).contiguous()
            g = matcha_template_grad(ctx.plan, f, c, euler, weight=w, template_batch_stride=0)
            return g["vox_grad"][0].to(ctx.tdtype), None, None

    class _Coefs(T.autograd.Function):
        @staticmethod
        def forward(ctx, h_coef, f_coef, plan):
            out = align_from_coefs(plan, f_coef, h_coef.reshape(1, *h_coef.shape[-3:]).contiguous(), 0)
            ctx.plan = plan
            ctx.save_for_backward(f_coef, out["c"], out["euler"])
            ctx.mark_non_differentiable(out["euler"])
            return out["score"], out["euler"]

        @staticmethod
        def backward(ctx, g_score, g_euler):
            f, c, euler = ctx.saved_tensors
            if g_score is None:
                return None, None, None
            w = g_score.to(T.float64).contiguous()
            g = matcha_template_grad(ctx.plan, f, c, euler, weight=w, template_batch_stride=0,
                                     voxels=False)
            return g["coef_grad"][0], None, None

    return _Voxels, _Coefs


_classes = None


def _cls():
    global _classes
    if _classes is None:
        _classes = _function_classes()
    return _classes


def refined_scores(template, particles, plan: Plan):
    """(scores [B] float64, euler [B][3]) of ``particles`` [B][N][N][N]
    against one ``template`` [N][N][N] (float32, CUDA); differentiable in
    ``template``."""
    if particles.dim() != 4 or template.shape[-3:] != particles.shape[-3:]:
        raise MatchaError("refined_scores: particles [B][N][N][N] and one template [N][N][N]")
    return _cls()[0].apply(template, particles, plan)


def refined_scores_from_coefs(h_coef, f_coef, plan: Plan):
    """As ``refined_scores`` from SH coefficients (``matcha_analyze`` layout):
    ``h_coef`` [S][n_lm][2] of the template, ``f_coef`` [B][S][n_lm][2];
    differentiable in ``h_coef``."""
    return _cls()[1].apply(h_coef, f_coef, plan)
