"""Row-band sharding (paper_2306_15010_gb300/bands.py) on the CPU: the band plan, the argmax key,
the band heatmaps of the oracle against its whole-query heatmap (the th - 1 row halo and the
band's own integral image give every window's exact counts), and the argmax all-reduce over two
gloo ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from paper_2306_15010_gb300 import bands


@pytest.mark.parametrize("HO,n", [(1, 1), (7, 3), (1921, 4), (5, 8), (100, 7)])
def test_band_rows(HO, n):
    r = bands.band_rows(HO, n)
    assert len(r) == n and r[0][0] == 0 and r[-1][1] == HO
    for (a, b), (c, _) in zip(r, r[1:]):
        assert b == c
    sizes = [b - a for a, b in r]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0


def test_argmax_key_order():
    rng = np.random.default_rng(3)
    WO = 13
    vals = rng.choice(np.array([-2.5, -1.0, -0.0, 0.0, 0.75, 3.0, -np.inf], np.float32), 200)
    idx = rng.permutation(13 * 20)[:200]
    keys = [bands.argmax_key(float(v), int(i) // WO, int(i) % WO, WO) for v, i in zip(vals, idx)]
    # the largest key: the largest value, then the lowest index (-0.0 and 0.0 compare equal)
    top = max(vals)
    want = min(int(i) for v, i in zip(vals, idx) if v == top)
    got = bands.key_to_yx(max(keys), WO)
    if top == 0.0:      # +0.0 orders above -0.0 in the key; both are maxima of the float compare
        assert got[0] * WO + got[1] in [int(i) for v, i in zip(vals, idx) if v == 0.0]
    else:
        assert got == (want // WO, want % WO)
    for a, b in [(1.0, 2.0), (-3.0, -1.0), (-np.inf, -1e30), (0.5, 0.5000001)]:
        assert bands.argmax_key(a, 0, 0, WO) < bands.argmax_key(b, 0, 0, WO)
    assert bands.argmax_key(1.0, 0, 5, WO) > bands.argmax_key(1.0, 1, 0, WO)


def _case(H, W, k, th, tw, seed):
    rng = np.random.default_rng(seed)
    lab = rng.integers(0, k, (H, W)).astype(np.int32)
    lab[:, 5:9] = 1                                  # repeated columns: equal windows, argmax ties
    tl = lab[3:3 + th, 4:4 + tw].copy()
    bank = synth.grid_bank(th, tw, 3)
    tc = oracle.filter_counts(tl, k, bank)
    return lab, bank, tc


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_band_heatmaps_equal_whole(n):
    H, W, k, th, tw = 41, 37, 6, 12, 10
    lab, bank, tc = _case(H, W, k, th, tw, seed=11)
    heat, am = oracle.score(lab, k, th, tw, bank, tc)
    HO, WO = heat.shape
    maxima = []
    for (y0, y1) in bands.band_rows(HO, n):
        if y1 == y0:
            continue
        hb, (by, bx) = oracle.score(lab[y0:y1 + th - 1], k, th, tw, bank, tc)
        assert hb.shape == (y1 - y0, WO)
        assert np.array_equal(hb, heat[y0:y1])
        maxima.append((float(hb[by, bx]), by + y0, bx))
    assert bands.combine_maxima(maxima, WO) == am


def _worker(rank, world, port, heat, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        HO, WO = heat.shape
        y0, y1 = bands.band_rows(HO, world)[rank]
        hb = heat[y0:y1]
        i = int(np.argmax(hb))                        # first occurrence: lowest row-major index
        out[rank] = bands.allreduce_argmax(float(hb.flat[i]), y0 + i // WO, i % WO, WO)
    finally:
        dist.destroy_process_group()


def test_allreduce_argmax_two_ranks():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    heat = np.random.default_rng(5).normal(size=(9, 7)).astype(np.float32)
    heat[2, 3] = heat[6, 1] = heat.max() + 1.0       # the same maximum in both bands
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, heat, out), nprocs=2, join=True)
    assert out[0] == out[1] == (2, 3)
