"""Soft-VQ heatmap with gradients (the training path) over the C ABI.

``soft_heatmap(Qf, Tf, C, wf, tau, G)`` is a ``torch.autograd.Function``: the forward is
``vqnnf_soft_forward`` (soft assignment p_j = softmax(-||x - c_j||^2 / tau), soft counts over
the G x G template grid cells, Eq. 2 with the L1 norm), the backward ``vqnnf_soft_backward``
(gradients for the query features, the centroids and the filter weights; the workspace of
the forward keeps the soft assignments and the cell sums for it).  All work runs in the
library's kernels; this module only marshals tensors.
"""
from __future__ import annotations

import torch

from . import _lib
from .api import Workspace, _need, _stream


def soft_workspace_bytes(B, H, W, D, k, th, tw, G=3) -> int:
    return int(_lib.load().vqnnf_soft_workspace_bytes(B, H, W, D, k, th, tw, G))


class SoftHeatmap(torch.autograd.Function):
    """heat = SoftHeatmap.apply(Qf (B,H,W,D), Tf (th,tw,D), C (k,D), wf (G*G,), tau, G)."""

    @staticmethod
    def forward(ctx, Qf, Tf, C, wf, tau, G):
        for t, n in ((Qf, "Qf"), (Tf, "Tf"), (C, "C"), (wf, "wf")):
            _need(t, n, torch.float32)
        B, H, W, D = Qf.shape
        th, tw = Tf.shape[:2]
        k = C.shape[0]
        if Tf.shape[2] != D or C.shape[1] != D or wf.numel() != G * G:
            raise ValueError("inconsistent shapes")
        nb = soft_workspace_bytes(B, H, W, D, k, th, tw, G)
        if nb == 0:
            raise _lib.VqnnfError("vqnnf_soft_forward", _lib.EUNSUPPORTED, "unsupported shape")
        ws = Workspace(nb, Qf.device)
        heat = torch.empty((B, H - th + 1, W - tw + 1), dtype=torch.float32, device=Qf.device)
        st = _lib.load().vqnnf_soft_forward(Qf.data_ptr(), B, H, W, Tf.data_ptr(), th, tw, D, C.data_ptr(), k,
                                            float(tau), int(G), wf.data_ptr(), heat.data_ptr(), ws.ptr, ws.nbytes,
                                            _stream(None))
        _lib.check("vqnnf_soft_forward", st)
        ctx.save_for_backward(Qf, Tf, C, wf)
        ctx.ws, ctx.tau, ctx.G = ws, float(tau), int(G)
        return heat

    @staticmethod
    def backward(ctx, dheat):
        Qf, Tf, C, wf = ctx.saved_tensors
        dheat = dheat.contiguous().float()
        B, H, W, D = Qf.shape
        th, tw = Tf.shape[:2]
        k = C.shape[0]
        dQ = torch.empty_like(Qf)
        dC = torch.empty_like(C)
        dw = torch.empty_like(wf)
        st = _lib.load().vqnnf_soft_backward(Qf.data_ptr(), B, H, W, Tf.data_ptr(), th, tw, D, C.data_ptr(), k,
                                             ctx.tau, ctx.G, wf.data_ptr(), dheat.data_ptr(), dQ.data_ptr(),
                                             dC.data_ptr(), dw.data_ptr(), ctx.ws.ptr, ctx.ws.nbytes,
                                             _stream(None))
        _lib.check("vqnnf_soft_backward", st)
        return dQ, None, dC, dw, None, None


def soft_heatmap(Qf, Tf, C, wf, tau: float = 0.1, G: int = 3):
    """Soft-VQ heatmap (B, H - th + 1, W - tw + 1), differentiable in Qf, C and wf."""
    return SoftHeatmap.apply(Qf, Tf, C, wf, tau, G)
