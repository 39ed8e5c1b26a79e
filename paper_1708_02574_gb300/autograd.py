"""torch.autograd.Function for learning edge weights through TPA (supervised random walks).

Edge weights w_e = exp(theta . f_e) parameterise A~ = w / rowsum.  The loss is
L = sum over triples (s, p, q) of softplus(r_TPA^(s)[q] - r_TPA^(s)[p]), with
r_TPA from Algorithms 2-3 (the stranger chain run for exactly K iterations).
When theta requires a gradient, the forward pass already runs the adjoint
kernels (tpa_loss_grad), because the backward recursions need the forward
iterates, and backward scales the stored dL/dtheta by the incoming gradient;
otherwise the forward pass computes the loss alone.
"""
from __future__ import annotations

import torch

from . import tpa


class TPALinkLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, feat, g, seeds, pos, neg, c=0.15, S=5, T=10, K=None, eps=1e-9):
        w = tpa.edge_weights(feat, theta)
        tpa.set_edge_weights(g, w)
        if K is None:
            # the iteration count of preprocessing on these weights (Algorithm 2's break)
            tpa.preprocess(g, c, T, eps)
            K = max(int(tpa.get_stranger(g)[1]), T)
        want = bool(ctx.needs_input_grad[0])
        loss, gw = tpa.loss_grad(g, seeds, pos, neg, c, S, T, K, want_grad=want)
        gtheta = tpa.theta_grad(feat, w, gw) if want else torch.zeros_like(theta, dtype=torch.float64)
        ctx.save_for_backward(gtheta)
        ctx.theta_dtype = theta.dtype
        ctx.K = K
        return torch.tensor(loss, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        (gtheta,) = ctx.saved_tensors
        return (grad_out * gtheta).to(ctx.theta_dtype), None, None, None, None, None, None, None, None, None, None
