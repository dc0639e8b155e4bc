"""Row-band sharding of one query (the data-parallel split of Sec. 3.4: every window is scored
independently).

The valid window rows [0, H - th + 1) are cut into contiguous bands, one per rank (or one after
another on one GPU).  A band of window rows [y0, y1) reads the label rows [y0, y1 + th - 1): its
own rows plus a halo of th - 1 rows.  It assigns those rows itself (the nearest-neighbour field
is per pixel), builds an integral image of them alone, and scores its windows.  Every box count
of Alg. 2 is a difference of integral-image values over rows inside the band, so the local
table gives the same counts as the whole query's, and the band's heatmap rows are exactly rows
y0 .. y1 - 1 of the whole heatmap (Eq. 2).  The template side (codebook, template counts) is the
same for every band: computed once and shared, or recomputed from the same seed on each rank.

The global maximum is the largest band maximum, the lowest row-major (y, x) on ties, as the
single-query argmax.  Across ranks it is one MAX all-reduce of a 64-bit key that orders by the
value and then by the inverted window index (``argmax_key``).

Only argument marshalling and the band bookkeeping live here; every step runs in the library's
kernels through ``vqnnf_assign`` and ``vqnnf_score``.
"""
from __future__ import annotations

import struct

import torch

from .api import vqnnf_assign, vqnnf_score


def band_rows(HO: int, n: int) -> list[tuple[int, int]]:
    """``n`` contiguous ranges [y0, y1) of window rows covering [0, HO), sizes differing by at
    most one (the first HO % n bands one row longer); bands beyond HO rows are empty."""
    if HO < 1 or n < 1:
        raise ValueError("need HO >= 1 and n >= 1")
    base, extra = divmod(HO, n)
    out, y = [], 0
    for b in range(n):
        rows = base + (1 if b < extra else 0)
        out.append((y, y + rows))
        y += rows
    return out


def argmax_key(value: float, y: int, x: int, WO: int) -> int:
    """Signed 64-bit key, larger for a larger value and, on equal values, for a lower row-major
    window index: the FP32 bits mapped to an order-preserving unsigned word in the high half,
    the inverted index in the low half, then the top bit flipped so that signed order agrees."""
    b = struct.unpack("<I", struct.pack("<f", value))[0]
    b = (~b & 0xFFFFFFFF) if b & 0x80000000 else (b | 0x80000000)
    key = (b << 32) | (0xFFFFFFFF - (y * WO + x))
    return key - (1 << 63)


def key_to_yx(key: int, WO: int) -> tuple[int, int]:
    idx = 0xFFFFFFFF - ((key + (1 << 63)) & 0xFFFFFFFF)
    return idx // WO, idx % WO


def combine_maxima(maxima, WO: int) -> tuple[int, int]:
    """Global argmax (y, x) from the bands' (value, y, x) maxima (empty bands left out)."""
    best = max(argmax_key(v, y, x, WO) for (v, y, x) in maxima)
    return key_to_yx(best, WO)


def allreduce_argmax(value: float, y: int, x: int, WO: int, group=None, device="cpu") -> tuple[int, int]:
    """Global argmax over ranks: one MAX all-reduce of the band maxima's keys.  A rank whose
    band is empty passes value = -inf."""
    import torch.distributed as dist
    t = torch.tensor([argmax_key(value, y, x, WO)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return key_to_yx(int(t.item()), WO)


def match_band(X: torch.Tensor, C: torch.Tensor, prec, k: int, th: int, tw: int, bank, t_counts: torch.Tensor,
               y0: int, y1: int, *, heatmap: torch.Tensor | None = None, labels: torch.Tensor | None = None,
               ws_assign=None, ws_score=None, stream=None):
    """Scores window rows [y0, y1) of the query X (H x W x D) against the template side (C,
    t_counts): assigns label rows [y0, y1 + th - 1) and scores them with their own integral
    image.  Returns (the heatmap rows y0 .. y1 - 1, the band's argmax as a device int32[2]
    (y - y0, x), y0)."""
    H, W, _ = X.shape
    if not (0 <= y0 < y1 <= H - th + 1):
        raise ValueError(f"band [{y0}, {y1}) outside the window rows [0, {H - th + 1})")
    rows = X[y0:y1 + th - 1]
    if labels is None:
        labels = torch.empty((y1 + th - 1 - y0, W), dtype=torch.uint8, device=X.device)
    vqnnf_assign(rows, C, prec, labels=labels, ws=ws_assign, stream=stream)
    heat, am = vqnnf_score(labels, k, th, tw, bank, t_counts, heatmap=heatmap, ws=ws_score, stream=stream)
    return heat, am, y0
