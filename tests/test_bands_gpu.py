"""Row-band sharding on one GPU (paper_2306_15010_gb300/bands.py): the query's window rows split
into bands, each band assigned and scored on its own rows plus the th - 1 row halo with its own
integral image, must give exactly the whole query's heatmap rows (bit for bit: the per-filter
counts are the same integers and the FP32 combination runs in the same order) and, combined,
the same argmax; checked against the whole-query pipeline and, at sampled windows, the oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vq():
    from paper_2306_15010_gb300 import build
    build.build()
    import paper_2306_15010_gb300 as m
    torch.cuda.set_device(0)
    return m


@pytest.mark.parametrize("prec,n", [("bf16", 3), ("fp32", 4), ("bf16", 7)])
def test_bands_equal_whole_query(vq, prec, n):
    from paper_2306_15010_gb300 import bands
    H, W, D, k, th, tw = 1024, 960, 128, 128, 128, 112
    q = synth.query_map(H, W, D, M=64, n_sp=4000, seed=7100, device="cuda")
    T, _ = synth.warped_template(q, th, tw, seed=7200)
    T = T.cuda().contiguous()
    bank = synth.grid_bank(th, tw, 3)
    C = vq.vqnnf_fit_codebook(T, k, 10, 7300, prec)
    tl = vq.vqnnf_assign(T, C, prec)
    tc = vq.vqnnf_filter_responses(tl, k, bank)
    ql = vq.vqnnf_assign(q.X, C, prec)
    heat, am = vq.vqnnf_score(ql, k, th, tw, bank, tc)
    HO, WO = heat.shape
    hb_all = torch.full_like(heat, float("nan"))
    maxima = []
    for (y0, y1) in bands.band_rows(HO, n):
        hb, bam, _ = bands.match_band(q.X, C, prec, k, th, tw, bank, tc, y0, y1, heatmap=hb_all[y0:y1])
        by, bx = (int(v) for v in bam.cpu())
        maxima.append((float(hb[by, bx]), by + y0, bx))
    torch.cuda.synchronize()
    assert torch.equal(hb_all, heat)
    assert bands.combine_maxima(maxima, WO) == tuple(int(v) for v in am.cpu())
    # the band path against the oracle at windows around the band seams and the argmax
    rows = sorted({y for (y0, y1) in bands.band_rows(HO, n) for y in (y0, max(y0, y1 - 1))})
    rng = np.random.default_rng(n)
    win = np.array([(y, int(x)) for y in rows for x in rng.integers(0, WO, 4)] +
                   [(maxima[0][1], maxima[0][2])], np.int32)
    ref = oracle.score_at(ql.cpu().numpy(), k, bank, tc.cpu().numpy(), win)
    got = hb_all.cpu().numpy()[win[:, 0], win[:, 1]].astype(np.float64)
    areas = [f["area"] for f in bank]
    assert np.all(np.abs(got - ref) < 0.5 * min(1.0 / a for a in areas))
