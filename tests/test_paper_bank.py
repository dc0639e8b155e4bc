"""The paper's filter bank as weighted rectangles (synth.paper_bank), checked on the CPU
against what Sec. 3.2-3.3 and Sec. 4.2 fix: filter counts per set and scale, rectangles inside
the window and on the scale's 3 x 3 bin grid, Haar weights that cancel over each row / column,
w_{s,f} = w_f / s, and the Gaussian filter's response equal to the scale region's histogram
under the equal-weight reading (Algorithm 2's all-ones closed form)."""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("filters,n", [("gauss", 1), ("2-rect", 3), ("3-rect", 3), ("2,3-rect", 5)])
@pytest.mark.parametrize("S", [1, 3, 4])
def test_counts_and_geometry(filters, n, S):
    th, tw = 128, 96
    for gauss in ("equal", "exp"):
        bank = synth.paper_bank(th, tw, filters, S, gauss)
        assert len(bank) == n * S
        for idx, f in enumerate(bank):
            s = idx // n + 1
            ws, hs = tw // s, th // s
            xo, yo = (tw - ws) // 2, (th - hs) // 2
            assert f["area"] == ws * hs
            for (x0, y0, x1, y1, w) in f["rects"]:
                assert xo <= x0 < x1 <= xo + ws and yo <= y0 < y1 <= yo + hs
                assert w != 0


def test_paper_filter_weights():
    bank = synth.paper_bank(90, 90, "2,3-rect", 2, "equal")
    names = ["gauss", "haar2x", "haar2y", "haar3x", "haar3y"]
    for idx, f in enumerate(bank):
        s, name = idx // 5 + 1, names[idx % 5]
        assert f["w_f"] == pytest.approx((1.0 if name == "gauss" else 0.25) / s)
        ws = sum(w for (*_, w) in f["rects"])
        if name == "gauss":
            assert f["rects"] == [((90 - 90 // s) // 2, (90 - 90 // s) // 2,
                                   (90 - 90 // s) // 2 + 90 // s, (90 - 90 // s) // 2 + 90 // s, 1)]
        elif name.endswith("2x") or name.endswith("2y"):
            assert sorted(w for (*_, w) in f["rects"]) == [-1, 1] and ws == 0
        else:
            assert sorted(w for (*_, w) in f["rects"]) == [-2, 1, 1] and ws == 0


def test_exp_gaussian_weights():
    import math
    f = synth.paper_bank(60, 60, "gauss", 1, "exp", quant=4096)[0]
    w = sorted({wt for (*_, wt) in f["rects"]})
    assert w == sorted({round(4096 * math.exp(-(i * i + j * j) / 8.0)) for i in (-1, 0, 1) for j in (-1, 0, 1)})
    assert f["w_f"] == 1.0 / 4096


def test_equal_gaussian_is_region_histogram():
    r = np.random.default_rng(3)
    k, th, tw = 7, 30, 33
    lab = r.integers(0, k, (th, tw)).astype(np.int32)
    bank = synth.paper_bank(th, tw, "gauss", 3, "equal")
    counts = oracle.filter_counts(lab, k, bank)
    for s in range(1, 4):
        ws, hs = tw // s, th // s
        xo, yo = (tw - ws) // 2, (th - hs) // 2
        hist = np.bincount(lab[yo:yo + hs, xo:xo + ws].ravel(), minlength=k)
        assert np.array_equal(counts[s - 1], hist)
