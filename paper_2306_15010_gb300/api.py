"""Torch-tensor binding of the C ABI (same names as include/vqnnf.h).

Argument marshalling only: every step of the path runs in libvqnnf.so.  Tensors must be
CUDA tensors on the current device; work is enqueued on ``torch.cuda.current_stream()``
(or the stream passed in) and nothing synchronises the host, so the calls can be captured
in a CUDA graph when their workspaces are allocated up front (see :class:`Workspace`).
"""
from __future__ import annotations

import ctypes
from typing import Iterable, Sequence

import torch

from . import _lib

_STATS_WORDS = 4


def _stream(stream) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _keep(stream, *tensors) -> None:
    """Tensors allocated here on the current stream but used on another one: tell the
    caching allocator, so their memory is not reused before that stream is done."""
    if stream is None or stream == torch.cuda.current_stream():
        return
    for t in tensors:
        if t is not None:
            t.record_stream(stream)


def _need(t: torch.Tensor, name: str, dtype: torch.dtype) -> None:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _stats_ptr(stats) -> int:
    if stats is None:
        return 0
    _need(stats, "stats", torch.int64)
    if stats.numel() < _STATS_WORDS:
        raise ValueError("stats needs 4 int64 words")
    return stats.data_ptr()


def _prec(prec) -> int:
    if isinstance(prec, str):
        try:
            return _lib.PREC[prec]
        except KeyError:
            raise ValueError(f"unknown precision {prec!r}; use one of {list(_lib.PREC)}")
    return int(prec)


class Bank:
    """A filter bank in the C layout (vqnnf_filter / vqnnf_rect arrays kept alive here).

    ``filters`` is a sequence of dicts with ``rects`` [(x0, y0, x1, y1, weight), ...],
    ``w_f`` and ``area`` (the form produced by ``synth.grid_bank``).
    """

    def __init__(self, filters: Sequence[dict]):
        self.filters = list(filters)
        self._rects = []
        arr = (_lib.VqnnfFilter * len(self.filters))()
        for f, filt in enumerate(self.filters):
            rs = (_lib.VqnnfRect * len(filt["rects"]))()
            for i, (x0, y0, x1, y1, w) in enumerate(filt["rects"]):
                rs[i] = _lib.VqnnfRect(int(x0), int(y0), int(x1), int(y1), int(w))
            self._rects.append(rs)
            arr[f] = _lib.VqnnfFilter(len(filt["rects"]), ctypes.cast(rs, ctypes.POINTER(_lib.VqnnfRect)),
                                      float(filt["w_f"]), float(filt["area"]))
        self._arr = arr

    @property
    def F(self) -> int:
        return len(self.filters)

    @property
    def ptr(self) -> int:
        return ctypes.addressof(self._arr)

    @staticmethod
    def of(bank) -> "Bank":
        return bank if isinstance(bank, Bank) else Bank(bank)


class Workspace:
    """Caller-owned scratch memory for one operation (a uint8 CUDA tensor)."""

    def __init__(self, nbytes: int, device=None):
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        self.tensor = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=dev)

    @property
    def ptr(self) -> int:
        return self.tensor.data_ptr()

    @property
    def nbytes(self) -> int:
        return self.tensor.numel()

    @staticmethod
    def ensure(ws, nbytes: int, device) -> "Workspace":
        if ws is None or ws.nbytes < nbytes:
            return Workspace(nbytes, device)
        return ws


def vqnnf_version() -> int:
    return int(_lib.load().vqnnf_version())


def vqnnf_workspace_bytes(op: int, H: int, W: int, D: int = 0, k: int = 0, th: int = 0,
                          tw: int = 0, F: int = 0, prec="fp32") -> int:
    return int(_lib.load().vqnnf_workspace_bytes(op, H, W, D, k, th, tw, F, _prec(prec)))


def vqnnf_fit_codebook(T: torch.Tensor, k: int, iters: int, seed: int, prec="fp32", *,
                       C: torch.Tensor | None = None, ws: Workspace | None = None,
                       stream=None) -> torch.Tensor:
    """k x D float32 k-means codebook of the template T (h x w x D float32)."""
    _need(T, "T", torch.float32)
    h, w, D = T.shape
    if C is None:
        C = torch.empty((k, D), dtype=torch.float32, device=T.device)
    _need(C, "C", torch.float32)
    p = _prec(prec)
    nb = vqnnf_workspace_bytes(_lib.OP_FIT, h, w, D, k, prec=p)
    if nb == 0:
        raise _lib.VqnnfError("vqnnf_fit_codebook", _lib.EUNSUPPORTED, "unsupported shape")
    ws = Workspace.ensure(ws, nb, T.device)
    _keep(stream, ws.tensor, C)
    st = _lib.load().vqnnf_fit_codebook(T.data_ptr(), h, w, D, k, iters,
                                        ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), p,
                                        C.data_ptr(), ws.ptr, ws.nbytes, _stream(stream))
    _lib.check("vqnnf_fit_codebook", st)
    return C


def vqnnf_assign(X: torch.Tensor, C: torch.Tensor, prec="fp32", *,
                 labels: torch.Tensor | None = None, stats: torch.Tensor | None = None,
                 ws: Workspace | None = None, stream=None) -> torch.Tensor:
    """H x W uint8 nearest-centroid labels of X (H x W x D float32) over C (k x D).

    ``stats``: optional int64 CUDA tensor of 4 words, overwritten with (n_flagged,
    n_candidates, n_deep, 0) of the near-tie re-scoring.
    """
    _need(X, "X", torch.float32)
    _need(C, "C", torch.float32)
    if X.dim() == 2:
        H, W, D = 1, X.shape[0], X.shape[1]
    else:
        H, W, D = X.shape
    k = C.shape[0]
    if C.dim() != 2 or C.shape[1] != D:
        raise ValueError("codebook width differs from the feature depth")
    if labels is None:
        labels = torch.empty(X.shape[:-1], dtype=torch.uint8, device=X.device)
    _need(labels, "labels", torch.uint8)
    if labels.numel() < H * W:
        raise ValueError(f"labels holds {labels.numel()} bytes, the feature map has {H * W} pixels")
    sp = _stats_ptr(stats)
    p = _prec(prec)
    nb = vqnnf_workspace_bytes(_lib.OP_ASSIGN, H, W, D, k, prec=p)
    if nb == 0:
        raise _lib.VqnnfError("vqnnf_assign", _lib.EUNSUPPORTED, "unsupported shape")
    ws = Workspace.ensure(ws, nb, X.device)
    _keep(stream, ws.tensor, labels)
    st = _lib.load().vqnnf_assign(X.data_ptr(), H, W, D, C.data_ptr(), k, p, labels.data_ptr(),
                                  sp, ws.ptr, ws.nbytes, _stream(stream))
    _lib.check("vqnnf_assign", st)
    return labels


def vqnnf_assign_noalloc(X: torch.Tensor, C: torch.Tensor, prec="fp32", *,
                         labels: torch.Tensor, stats: torch.Tensor | None = None,
                         stream=None) -> torch.Tensor:
    """vqnnf_assign without a workspace, for callers that cannot allocate device memory
    themselves (a plug-in whose host application owns every device allocation, or a loop
    that must never wait on the allocator): the library's fixed 16 MiB scratch area is used
    instead.  ``labels`` must be passed in; nothing is allocated here either.  Calls that
    overlap on the GPU share that area and race; requests that need more scratch than it
    holds raise (status VQNNF_ENOMEM).  Every shape check of vqnnf_assign is made here too,
    before anything is enqueued."""
    _need(X, "X", torch.float32)
    _need(C, "C", torch.float32)
    _need(labels, "labels", torch.uint8)
    if X.dim() == 2:
        H, W, D = 1, X.shape[0], X.shape[1]
    else:
        H, W, D = X.shape
    if C.dim() != 2 or C.shape[1] != D:
        raise ValueError("codebook width differs from the feature depth")
    if labels.numel() < H * W:
        raise ValueError(f"labels holds {labels.numel()} bytes, the feature map has {H * W} pixels")
    sp = _stats_ptr(stats)
    st = _lib.load().vqnnf_assign_noalloc(X.data_ptr(), H, W, D, C.data_ptr(), C.shape[0],
                                          _prec(prec), labels.data_ptr(), sp, _stream(stream))
    _lib.check("vqnnf_assign_noalloc", st)
    return labels


def vqnnf_filter_responses(labels: torch.Tensor, k: int, bank, *,
                           counts: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """F x k int32 template representation vectors of the template NNF."""
    _need(labels, "labels", torch.uint8)
    h, w = labels.shape
    b = Bank.of(bank)
    if counts is None:
        counts = torch.empty((b.F, k), dtype=torch.int32, device=labels.device)
    _need(counts, "counts", torch.int32)
    _keep(stream, counts)
    st = _lib.load().vqnnf_filter_responses(labels.data_ptr(), h, w, k, b.ptr, b.F,
                                            counts.data_ptr(), None, 0, _stream(stream))
    _lib.check("vqnnf_filter_responses", st)
    return counts


def vqnnf_score(q_labels: torch.Tensor, k: int, th: int, tw: int, bank, t_counts: torch.Tensor,
                *, heatmap: torch.Tensor | None = None, argmax_yx: torch.Tensor | None = None,
                ws: Workspace | None = None, stream=None):
    """Eq. 2 heatmap ((H-th+1) x (W-tw+1) float32) and the int32 (y, x) of its maximum."""
    _need(q_labels, "q_labels", torch.uint8)
    _need(t_counts, "t_counts", torch.int32)
    H, W = q_labels.shape
    b = Bank.of(bank)
    if heatmap is None:
        heatmap = torch.empty((H - th + 1, W - tw + 1), dtype=torch.float32, device=q_labels.device)
    _need(heatmap, "heatmap", torch.float32)
    if argmax_yx is None:
        argmax_yx = torch.empty(2, dtype=torch.int32, device=q_labels.device)
    _need(argmax_yx, "argmax_yx", torch.int32)
    nb = vqnnf_workspace_bytes(_lib.OP_SCORE, H, W, 0, k, th, tw, b.F)
    if nb == 0:
        raise _lib.VqnnfError("vqnnf_score", _lib.EUNSUPPORTED, "unsupported shape")
    ws = Workspace.ensure(ws, nb, q_labels.device)
    _keep(stream, ws.tensor, heatmap, argmax_yx)
    st = _lib.load().vqnnf_score(q_labels.data_ptr(), H, W, k, th, tw, b.ptr, b.F,
                                 t_counts.data_ptr(), heatmap.data_ptr(), argmax_yx.data_ptr(),
                                 ws.ptr, ws.nbytes, _stream(stream))
    _lib.check("vqnnf_score", st)
    return heatmap, argmax_yx


def _need_host(t: torch.Tensor, name: str, dtype: torch.dtype) -> None:
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a host (CPU) tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def vqnnf_match_host_workspace_bytes(H: int, W: int, D: int, k: int, th: int, tw: int, F: int, prec="bf16") -> int:
    return int(_lib.load().vqnnf_match_host_workspace_bytes(H, W, D, k, th, tw, F, _prec(prec)))


def vqnnf_match_host(X: torch.Tensor, T: torch.Tensor, k: int, iters: int, seed: int, bank, prec="bf16", *,
                     heatmap: torch.Tensor | bool = True, argmax_yx: torch.Tensor | None = None,
                     ws: Workspace | None = None, stream=None, stream2=None):
    """The whole path for one pair with host feature maps (H x W x D and th x tw x D float32 CPU
    tensors, pinned for asynchronous copies): the host heatmap (or None with heatmap=False) and
    the host int32 (y, x) of its maximum, valid once ``stream`` reaches the end of the call's
    work.  ``stream2``: the compute stream (copies and compute overlap), or None."""
    _need_host(X, "X", torch.float32)
    _need_host(T, "T", torch.float32)
    H, W, D = X.shape
    th, tw = T.shape[:2]
    b = Bank.of(bank)
    p = _prec(prec)
    if heatmap is True:
        heatmap = torch.empty((H - th + 1, W - tw + 1), dtype=torch.float32, pin_memory=True)
    if heatmap is not False:
        _need_host(heatmap, "heatmap", torch.float32)
    if argmax_yx is None:
        argmax_yx = torch.empty(2, dtype=torch.int32, pin_memory=True)
    _need_host(argmax_yx, "argmax_yx", torch.int32)
    nb = int(_lib.load().vqnnf_match_host_workspace_bytes(H, W, D, k, th, tw, b.F, p))
    if nb == 0:
        raise _lib.VqnnfError("vqnnf_match_host", _lib.EUNSUPPORTED, "unsupported shape")
    ws = Workspace.ensure(ws, nb, None)
    st = _lib.load().vqnnf_match_host(X.data_ptr(), H, W, D, T.data_ptr(), th, tw, k, iters,
                                      ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), p, b.ptr, b.F,
                                      heatmap.data_ptr() if heatmap is not False else None,
                                      argmax_yx.data_ptr(), ws.ptr, ws.nbytes, _stream(stream),
                                      None if stream2 is None else int(stream2.cuda_stream))
    _lib.check("vqnnf_match_host", st)
    return (heatmap if heatmap is not False else None), argmax_yx


def vqnnf_set_kernel_events(op: int, start=None, stop=None) -> None:
    """Profiling aid: record the torch.cuda.Event pair (start, stop) immediately around the main
    kernel of every later call of ``op`` (OP_ASSIGN: the distance contraction; OP_SCORE: the
    score kernel); None, None switches it off.  The events must have been recorded once (so
    that their CUDA handles exist) and stay alive while set."""
    h0 = 0 if start is None else int(start.cuda_event)
    h1 = 0 if stop is None else int(stop.cuda_event)
    _lib.check("vqnnf_set_kernel_events", _lib.load().vqnnf_set_kernel_events(int(op), h0 or None, h1 or None))


def vqnnf_last_device_error(stream=None) -> int:
    """Synchronise the stream and return (and clear) the device error status code."""
    return int(_lib.load().vqnnf_last_device_error(_stream(stream)))


def vqnnf_selftest_bounded_wait(limit_cycles: int = 2_000_000, stream=None) -> None:
    """Enqueue the bounded-wait self-test: a one-thread kernel whose mbarrier wait (nothing
    completes it) gives up after ``limit_cycles`` SM cycles and records VQNNF_ETIMEOUT, which
    the next :func:`vqnnf_last_device_error` on that stream returns."""
    _lib.check("vqnnf_selftest_bounded_wait",
               _lib.load().vqnnf_selftest_bounded_wait(int(limit_cycles), _stream(stream)))
