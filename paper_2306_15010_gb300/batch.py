"""Batched matching over the C ABI: many templates against many queries.

``vqnnf_match_batch(queries, templates, ks)`` fits each template's codebook (k-means, seed +
template index), its NNF and grid-bank responses once, quantises every query against every
codebook (codebooks sharing one tensor-core contraction per group) and returns every pair's
Eq. 2 heatmap and maximum.  ``vqnnf_batch_tune`` times candidate tile plans on the largest
query and returns the fastest.  All work runs in libvqnnf.so; this module only marshals
tensors.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Sequence

import torch

from . import _lib
from .api import Workspace, _keep, _need, _stream


@dataclass
class BatchPlan:
    """Tile choices of the batched contraction (see vqnnf_batch_plan in the header)."""
    group_cols: int = 256
    sf: int = 0
    pf: int = -1
    stationary: int = 1

    def c(self) -> "_lib.VqnnfBatchPlan":
        return _lib.VqnnfBatchPlan(int(self.group_cols), int(self.sf), int(self.pf), int(self.stationary))


def _arrays(queries: Sequence[torch.Tensor], templates: Sequence[torch.Tensor], ks: Sequence[int]):
    if len(templates) != len(ks):
        raise ValueError("one k per template")
    D = None
    qa = (_lib.VqnnfImage * len(queries))()
    for i, X in enumerate(queries):
        _need(X, f"queries[{i}]", torch.float32)
        H, W, d = X.shape
        D = d if D is None else D
        if d != D:
            raise ValueError("every feature map needs the same D")
        qa[i] = _lib.VqnnfImage(X.data_ptr(), H, W)
    ta = (_lib.VqnnfBatchTemplate * len(templates))()
    for j, T in enumerate(templates):
        _need(T, f"templates[{j}]", torch.float32)
        h, w, d = T.shape
        if d != D:
            raise ValueError("every feature map needs the same D")
        ta[j] = _lib.VqnnfBatchTemplate(T.data_ptr(), h, w, int(ks[j]))
    return qa, ta, D


def vqnnf_batch_workspace_bytes(queries, templates, ks, G: int = 3) -> int:
    qa, ta, D = _arrays(queries, templates, ks)
    return int(_lib.load().vqnnf_batch_workspace_bytes(qa, len(qa), ta, len(ta), D, G))


def vqnnf_match_batch(queries: Sequence[torch.Tensor], templates: Sequence[torch.Tensor], ks: Sequence[int],
                      iters: int = 10, seed: int = 0, G: int = 3, plan: BatchPlan | None = None, *,
                      heat: bool | Sequence[torch.Tensor] = True, argmax_yx: torch.Tensor | None = None,
                      ws: Workspace | None = None, stream=None):
    """Heatmaps (list over queries of lists over templates, or None with heat=False) and the
    (nq, nt, 2) int32 tensor of each pair's best window (y, x)."""
    qa, ta, D = _arrays(queries, templates, ks)
    nq, nt = len(qa), len(ta)
    dev = queries[0].device
    if argmax_yx is None:
        argmax_yx = torch.empty((nq, nt, 2), dtype=torch.int32, device=dev)
    _need(argmax_yx, "argmax_yx", torch.int32)
    nb = int(_lib.load().vqnnf_batch_workspace_bytes(qa, nq, ta, nt, D, G))
    p = (plan or BatchPlan()).c()
    if nb == 0:
        # the shapes are refused: the call reports why, before it touches any memory
        st = _lib.load().vqnnf_match_batch(qa, nq, ta, nt, D, int(iters), ctypes.c_uint64(0), int(G),
                                           ctypes.byref(p), None, argmax_yx.data_ptr(), None, 0, _stream(stream))
        _lib.check("vqnnf_match_batch", st if st != _lib.OK else _lib.EUNSUPPORTED)
    heats = None
    hp = None
    if heat is True:
        heats = [[torch.empty((X.shape[0] - T.shape[0] + 1, X.shape[1] - T.shape[1] + 1), dtype=torch.float32,
                              device=dev) for T in templates] for X in queries]
    elif heat is not False:
        heats = [[heat[i * nt + j] for j in range(nt)] for i in range(nq)]
    if heats is not None:
        hp = (ctypes.c_void_p * (nq * nt))()
        for i in range(nq):
            for j in range(nt):
                _need(heats[i][j], f"heat[{i}][{j}]", torch.float32)
                hp[i * nt + j] = heats[i][j].data_ptr()
    ws = Workspace.ensure(ws, nb, dev)
    _keep(stream, ws.tensor, argmax_yx, *(h for row in (heats or []) for h in row))
    st = _lib.load().vqnnf_match_batch(qa, nq, ta, nt, D, int(iters), ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF),
                                       int(G), ctypes.byref(p), hp, argmax_yx.data_ptr(), ws.ptr, ws.nbytes,
                                       _stream(stream))
    _lib.check("vqnnf_match_batch", st)
    return heats, argmax_yx


def vqnnf_batch_tune(queries: Sequence[torch.Tensor], templates: Sequence[torch.Tensor], ks: Sequence[int],
                     iters: int = 10, seed: int = 0, G: int = 3, *, ws: Workspace | None = None,
                     stream=None) -> BatchPlan:
    """Fastest plan for the assignment of the largest query (synchronises the stream)."""
    qa, ta, D = _arrays(queries, templates, ks)
    nb = int(_lib.load().vqnnf_batch_workspace_bytes(qa, len(qa), ta, len(ta), D, G))
    p = _lib.VqnnfBatchPlan(0, 0, 0, 0)
    if nb == 0:
        st = _lib.load().vqnnf_batch_tune(qa, len(qa), ta, len(ta), D, int(iters), ctypes.c_uint64(0), int(G),
                                          ctypes.byref(p), None, 0, _stream(stream))
        _lib.check("vqnnf_batch_tune", st if st != _lib.OK else _lib.EUNSUPPORTED)
    ws = Workspace.ensure(ws, nb, queries[0].device)
    st = _lib.load().vqnnf_batch_tune(qa, len(qa), ta, len(ta), D, int(iters),
                                      ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), int(G), ctypes.byref(p),
                                      ws.ptr, ws.nbytes, _stream(stream))
    _lib.check("vqnnf_batch_tune", st)
    return BatchPlan(p.group_cols, p.sf, p.pf, p.stationary)
