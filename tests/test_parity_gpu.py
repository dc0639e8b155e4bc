"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (from the arithmetic, see the design notes):
* labels: equal to the oracle's wherever the oracle's own relative gap between the two best
  distances is >= 1e-6 (the near-tie band); duplicate centroids must give the lowest index;
* codebook: bit-identical (same FP64 additions in the same order, same roundings);
* counts: exact integers;
* heatmap from identical labels: |H_gpu - H_ref| < min_f(w_f / A_f) / 2 at every window.
  Each per-filter L1 sum of Eq. 2 is an exact integer and the float part is F float32 terms
  (far below that bound here), so one count error in any filter shows.  The wide-row case
  also recovers every per-filter L1 sum as an integer (one run per filter with the other
  weights 0) and compares it with the oracle's;
  heatmap of the whole path: <= 1e-4 * max|H_ref|.
"""
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


def _dev(a):
    return torch.as_tensor(a).cuda()


def _labels_ok(gpu, ref, d1, d2):
    band = oracle.relative_gap(d1, d2) < 1e-6
    bad = (gpu.astype(np.int32) != ref) & ~band
    return int(bad.sum()), int(band.sum())


def _codebook_case(H, W, D, k, seed, iters=3):
    """Query features and a codebook fitted by the oracle on a crop of the query (so that
    near-duplicate centroids and near-ties occur as in real use).  A query with fewer
    pixels than k gets a seeded random codebook instead."""
    q = synth.query_map(H, W, D, M=max(4, k // 2 + 3), n_sp=max(8, H * W // 200), seed=seed)
    if H * W < k:
        r = np.random.default_rng(seed)
        return q, None, r.random((k, D)).astype(np.float32)
    th, tw = min(H, max(4, H // 4)), min(W, max(4, W // 4))
    while th * tw < k:
        th, tw = min(H, th + 1), min(W, tw + 1)
    T, _ = synth.crop_template(q, th, tw, seed=seed + 1000)
    C = oracle.fit_codebook(T.numpy(), k, iters, seed)
    return q, T, C


PRECS = ["fp32", "bf16", "fp8"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("H,W,D,k", [
    (256, 256, 64, 16),      # the small 256 x 256 workload
    (129, 67, 64, 16),       # ragged tail of the 128-pixel tile
    (33, 50, 512, 128),      # headline depth and codebook size
    (21, 38, 1024, 128),     # the precision study's D = 1024 variant
    (40, 41, 16, 8),
    (17, 19, 32, 256),       # largest k (two 128-centroid passes)
    (9, 7, 4, 3),            # D = 4, partial k tile
    (1, 1, 64, 5),           # a single pixel
])
def test_assign_parity(vq, prec, H, W, D, k):
    q, _, C = _codebook_case(H, W, D, k, seed=H * 7 + W)
    if prec != "fp32" and D % 16:
        # the tensor paths need D % 16 == 0: refused on the host, nothing launched
        with pytest.raises(vq.VqnnfError) as e:
            vq.vqnnf_assign(_dev(q.X), _dev(C), prec)
        assert e.value.status == 5
        return
    ref, d1, d2 = oracle.assign(q.X.numpy(), C, return_dist=True)
    stats = torch.zeros(4, dtype=torch.int64, device="cuda")
    lab = vq.vqnnf_assign(_dev(q.X), _dev(C), prec, stats=stats).cpu().numpy()
    bad, inband = _labels_ok(lab, ref, d1, d2)
    assert bad == 0, f"{bad} labels differ outside the near-tie band ({inband} in band)"
    n_flag, n_cand, n_deep, _ = stats.cpu().tolist()
    assert 0 <= n_flag <= H * W and n_cand >= 2 * n_flag and n_deep <= n_flag


def test_assign_fp8_limits_and_wide_range_rows(vq):
    """FP8: a codebook too large to stay in shared memory is refused on the host; rows whose
    values span many binades (most of them quantise to zero or to the subnormal range of e4m3)
    still get exact labels, the bound flagging what the contraction cannot decide."""
    X = torch.zeros((4, 4, 1024), device="cuda")
    C = torch.zeros((129, 1024), device="cuda")
    with pytest.raises(vq.VqnnfError) as e:
        vq.vqnnf_assign(X, C, "fp8")
    assert e.value.status == 5
    r = np.random.default_rng(12)
    Xh = (r.random((33, 29, 128)) * np.exp2(r.integers(-30, 4, (33, 29, 128)))).astype(np.float32)
    Ch = Xh.reshape(-1, 128)[r.choice(33 * 29, 24, replace=False)] * np.float32(1.001)
    ref, d1, d2 = oracle.assign(Xh, Ch, return_dist=True)
    stats = torch.zeros(4, dtype=torch.int64, device="cuda")
    got = vq.vqnnf_assign(_dev(Xh), _dev(Ch), "fp8", stats=stats).cpu().numpy()
    bad, _ = _labels_ok(got, ref, d1, d2)
    assert bad == 0


@pytest.mark.parametrize("prec", PRECS)
def test_assign_k1_and_duplicates_lowest_index(vq, prec):
    r = np.random.default_rng(3)
    X = r.random((37, 45, 32)).astype(np.float32)
    C1 = r.random((1, 32)).astype(np.float32)
    assert int(vq.vqnnf_assign(_dev(X), _dev(C1), prec).max()) == 0
    base = r.random((5, 32)).astype(np.float32)
    C = np.concatenate([base, base[[3, 1]]])          # duplicates at 5 (of 3) and 6 (of 1)
    ref = oracle.assign(X, C)
    got = vq.vqnnf_assign(_dev(X), _dev(C), prec).cpu().numpy()
    assert np.array_equal(got.astype(np.int32), ref)
    assert got.max() <= 4


@pytest.mark.parametrize("prec", PRECS)
def test_assign_points_on_centroids(vq, prec):
    # pixels equal to centroids: distance 0 against a clear second best
    r = np.random.default_rng(4)
    C = r.random((24, 64)).astype(np.float32)
    X = C[r.integers(0, 24, size=(31, 33))]
    got = vq.vqnnf_assign(_dev(X), _dev(C), prec).cpu().numpy()
    assert np.array_equal(got.astype(np.int32), oracle.assign(X, C))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("h,w,D,k,iters", [(32, 32, 64, 16, 10), (48, 40, 128, 32, 6),
                                           (8, 8, 16, 64, 3), (20, 13, 32, 1, 2)])
def test_fit_codebook_bit_exact(vq, prec, h, w, D, k, iters):
    q = synth.query_map(4 * h, 4 * w, D, M=12, n_sp=60, seed=h + w)
    T, _ = synth.crop_template(q, h, w, seed=5)
    ref = oracle.fit_codebook(T.numpy(), k, iters, 99)
    got = vq.vqnnf_fit_codebook(_dev(T), k, iters, 99, prec).cpu().numpy()
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("prec", PRECS)
def test_fit_codebook_exact_sum_edge_values(vq, prec):
    """Centroid sums with values the exact fixed-point route cannot take (below 2^-57,
    spans over 52 bits, subnormals, a column with no value in range, sums too large for the
    128-bit accumulator), negatives and signed zeros: still bit-identical."""
    r = np.random.default_rng(5)
    l, D, k = 700, 64, 6
    T = r.normal(0.5, 0.3, (l, D)).astype(np.float32)
    T[r.random((l, D)) < 0.05] = 0.0
    T[r.random((l, D)) < 0.02] = -0.0
    T[r.random((l, D)) < 0.01] *= np.float32(2.0 ** -50)        # spans over 52 bits
    T[r.random((l, D)) < 0.005] = np.float32(1e-30)             # below the exact range
    T[r.random((l, D)) < 0.002] = np.float32(3e-42)             # subnormal
    T[:, :8] = np.abs(T[:, :8])                                 # some all-positive columns
    T[:, 8] = np.float32(1e-30)                                 # a column entirely below the range
    T[:, 9] = (r.uniform(1, 2, l) * 2.0 ** 44).astype(np.float32)   # sums past 2^127 units
    T[:, 10] = (r.uniform(-2, 2, l) * 2.0 ** 45).astype(np.float32)  # large, both signs
    T = T.reshape(35, 20, D)
    C = vq.vqnnf_fit_codebook(_dev(T), k, 4, 9, prec)
    C_ref = oracle.fit_codebook(T, k, 4, 9)
    assert np.array_equal(C.cpu().numpy().view(np.uint32), C_ref.view(np.uint32))


@pytest.mark.parametrize("prec", PRECS)
def test_fit_codebook_large_clusters_exact(vq, prec):
    """Clusters of more than a thousand members (many chunks, and the block-wide staged route
    of the in-order FP64 sums) with values that force that route: bit-identical to the oracle."""
    r = np.random.default_rng(11)
    l, D, k = 3600, 32, 2
    T = np.abs(r.normal(0.5, 0.3, (l, D))).astype(np.float32)
    T[r.random((l, D)) < 0.01] *= np.float32(2.0 ** -50)        # spans over 52 bits
    T[:, 3] = np.float32(1e-30)                                 # a column with no value in range
    T[:, 5] = (r.uniform(1, 2, l) * 2.0 ** 44).astype(np.float32)   # sums past 2^127 units
    T = T.reshape(60, 60, D)
    C = vq.vqnnf_fit_codebook(_dev(T), k, 3, 21, prec)
    C_ref = oracle.fit_codebook(T, k, 3, 21)
    assert np.array_equal(C.cpu().numpy().view(np.uint32), C_ref.view(np.uint32))


@pytest.mark.parametrize("prec", PRECS)
def test_fit_codebook_mixed_routes_across_chunks(vq, prec):
    """Clusters of many 128-member chunks where a few chunks hold values of 32 or more (outside
    the 64-bit fixed-point range, inside the 128-bit one) and the rest do not: the chunks'
    partial sums come from both routes and are combined; bit-identical to the oracle."""
    r = np.random.default_rng(17)
    l, D, k = 2000, 48, 3
    T = np.abs(r.normal(0.5, 0.3, (l, D))).astype(np.float32)
    big = r.random((l, D)) < 0.0002
    T[big] = r.uniform(32.0, 64.0, big.sum()).astype(np.float32)
    T = T.reshape(40, 50, D)
    C = vq.vqnnf_fit_codebook(_dev(T), k, 3, 5, prec)
    C_ref = oracle.fit_codebook(T, k, 3, 5)
    assert np.array_equal(C.cpu().numpy().view(np.uint32), C_ref.view(np.uint32))


def test_fit_zero_iters_gathers_seeded_init(vq):
    r = np.random.default_rng(6)
    T = r.random((30, 31, 8)).astype(np.float32)
    got = vq.vqnnf_fit_codebook(_dev(T), 40, 0, 2024).cpu().numpy()
    assert np.array_equal(got, T.reshape(-1, 8)[oracle.kmeans_init(30 * 31, 40, 2024)])


def _banks(th, tw):
    weighted = [
        {"rects": [(0, 0, tw, th, 1)], "w_f": 1.0, "area": float(th * tw)},
        {"rects": [(0, 0, tw // 2, th, 1), (tw // 2, 0, tw, th, -1)], "w_f": 0.25,
         "area": float(th * tw)},
        {"rects": [(0, 0, tw, th // 3, 1), (0, th // 3, tw, 2 * th // 3, -2),
                   (0, 2 * th // 3, tw, th, 1)], "w_f": 0.25, "area": float(th * tw)},
        {"rects": [(1, 2, tw - 1, th - 1, 3)], "w_f": 0.5, "area": float((tw - 2) * (th - 3))},
    ]
    return {"grid2": synth.grid_bank(th, tw, 2), "grid3": synth.grid_bank(th, tw, 3),
            "grid3_nofull": synth.grid_bank(th, tw, 3, full=False),
            "grid4": synth.grid_bank(th, tw, 4), "full_only": synth.grid_bank(th, tw, 1, full=False),
            "weighted": weighted}


@pytest.mark.parametrize("bank_name", ["grid2", "grid3", "grid3_nofull", "grid4", "full_only",
                                       "weighted"])
def test_filter_responses_exact(vq, bank_name):
    r = np.random.default_rng(7)
    th, tw, k = 37, 29, 11
    t = r.integers(0, k, size=(th, tw)).astype(np.int32)
    bank = _banks(th, tw)[bank_name]
    got = vq.vqnnf_filter_responses(_dev(t.astype(np.uint8)), k, bank).cpu().numpy()
    assert np.array_equal(got, oracle.filter_counts(t, k, bank))


def _exact_bound(bank):
    """Half the smallest change of H that one count of one rectangle can make:
    w_f / A_f times the rectangle's weight (the filter's L1 sum moves by at least that)."""
    return 0.5 * min(abs(f["w_f"]) / f["area"] * min(abs(r[4]) for r in f["rects"])
                     for f in bank if f["w_f"] != 0)


def _check_heat(got_heat, got_am, ref_heat, rtol, bank=None):
    scale = max(np.abs(ref_heat).max(), 1e-30)
    if bank is not None:
        # identical labels: every per-filter sum is exact
        err = np.abs(got_heat - ref_heat)
        i = int(err.argmax())
        assert err.max() < _exact_bound(bank), \
            f"heatmap error {err.max():.3g} at {divmod(i, got_heat.shape[1])}"
        rtol = _exact_bound(bank) / scale
    else:
        err = np.abs(got_heat - ref_heat).max() / scale
        assert err <= rtol, f"heatmap relative error {err:.3g}"
    y, x = got_am
    # the reported maximum is a maximum of the oracle heatmap up to the tolerance, and the
    # lowest row-major index among the GPU's own maxima
    assert ref_heat[y, x] >= ref_heat.max() - 2 * rtol * scale
    flat = np.flatnonzero(got_heat.ravel() == got_heat.max())[0]
    assert (y, x) == divmod(int(flat), got_heat.shape[1])


@pytest.mark.parametrize("bank_name", ["grid2", "grid3", "grid3_nofull", "grid4", "full_only",
                                       "weighted"])
@pytest.mark.parametrize("H,W,th,tw,k", [(96, 300, 37, 29, 11), (70, 64, 70, 64, 6),
                                         (41, 260, 9, 5, 3),
                                         (80, 200, 20, 24, 45),      # two cluster groups, the second ragged
                                         (66, 130, 16, 16, 256)])    # every label byte in use
def test_score_from_oracle_labels(vq, bank_name, H, W, th, tw, k):
    r = np.random.default_rng(H + W)
    q = synth.query_map(H, W, 4, M=6, n_sp=max(8, H * W // 150), seed=H)
    ql = (q.sp_id.numpy() * 7 % k).astype(np.int32)       # piecewise-constant label field
    ql[r.random(ql.shape) < 0.05] = r.integers(0, k)      # plus salt
    t = ql[3:3 + th, 1:1 + tw].copy() if th < H else ql.copy()
    bank = _banks(th, tw)[bank_name]
    tc = oracle.filter_counts(t, k, bank)
    ref, _ = oracle.score(ql, k, th, tw, bank, tc)
    heat, am = vq.vqnnf_score(_dev(ql.astype(np.uint8)), k, th, tw, bank,
                              _dev(tc.astype(np.int32)))
    _check_heat(heat.cpu().numpy(), tuple(am.cpu().tolist()), ref, 1e-5, bank)


@pytest.mark.parametrize("bank_name", ["grid3", "grid2", "grid4", "full_only", "weighted"])
@pytest.mark.parametrize("k", [3, 45, 256])
def test_score_wide_rows_every_filter_exact(vq, bank_name, k):
    """More than 1,024 windows per row (so every block seam of the score kernels along x is
    crossed) and a ragged last tile; every window element by element, and every per-filter
    L1 sum as an integer: the bank is scored once per filter with that filter's weight 1 and
    the others 0 (same rectangles, so the same kernel), giving H = -(1 / A_f) L1_f."""
    H, W, th, tw = 80, 1200, 24, 24
    r = np.random.default_rng(k + 5)
    q = synth.query_map(H, W, 4, M=6, n_sp=H * W // 120, seed=k)
    ql = (q.sp_id.numpy() * 7 % k).astype(np.int32)
    ql[r.random(ql.shape) < 0.08] = r.integers(0, k)
    t = ql[30:30 + th, 1000:1000 + tw].copy()
    bank = _banks(th, tw)[bank_name]
    tc = oracle.filter_counts(t, k, bank)
    ql_d, tc_d = _dev(ql.astype(np.uint8)), _dev(tc.astype(np.int32))
    ref, _ = oracle.score(ql, k, th, tw, bank, tc)
    heat, am = vq.vqnnf_score(ql_d, k, th, tw, bank, tc_d)
    assert heat.shape[1] > 1024
    _check_heat(heat.cpu().numpy(), tuple(am.cpu().tolist()), ref, 1e-5, bank)
    for f, flt in enumerate(bank):
        unit = [dict(g, w_f=1.0 if i == f else 0.0) for i, g in enumerate(bank)]
        hf, _ = vq.vqnnf_score(ql_d, k, th, tw, unit, tc_d)
        c32 = np.float64(np.float32(1.0 / flt["area"]))
        l1_gpu = np.rint(-hf.cpu().numpy().astype(np.float64) / c32)
        rf, _ = oracle.score(ql, k, th, tw, [dict(flt, w_f=1.0)], tc[f:f + 1])
        l1_ref = np.rint(-rf * flt["area"])
        bad = np.argwhere(l1_gpu != l1_ref)
        assert bad.size == 0, (f, bad[:5])


@pytest.mark.parametrize("th,tw,G", [(127, 129, 1),   # one cell of 16,383 pixels
                                     (128, 128, 1),   # 16,384 pixels
                                     (130, 131, 1),
                                     (200, 240, 2),   # cells of 12,000 pixels, full window 48,000
                                     (255, 257, 1)])  # 65,535 pixels: the largest 16-bit table
def test_score_counts_near_the_table_modulus(vq, th, tw, G):
    """Large grid cells on the 16-bit table (counts mod 2^16): regions of one label make the
    counts reach the cell area, up to the largest template the 16-bit table takes."""
    H, W, k = th + 37, tw + 300, 7
    r = np.random.default_rng(th + tw)
    q = synth.query_map(H, W, 4, M=6, n_sp=H * W // 3000, seed=th)
    ql = (q.sp_id.numpy() * 3 % k).astype(np.int32)
    ql[:, : W // 3] = 2                                     # a large one-label region
    ql[r.random(ql.shape) < 0.01] = r.integers(0, k)
    t = ql[5:5 + th, 11:11 + tw].copy()
    t[: th // 2] = 2
    for full in (True, False):
        bank = synth.grid_bank(th, tw, G, full=full)
        tc = oracle.filter_counts(t, k, bank)
        ref, _ = oracle.score(ql, k, th, tw, bank, tc)
        heat, am = vq.vqnnf_score(_dev(ql.astype(np.uint8)), k, th, tw, bank, _dev(tc.astype(np.int32)))
        _check_heat(heat.cpu().numpy(), tuple(am.cpu().tolist()), ref, 1e-5, bank)


@pytest.mark.parametrize("filters,S,gauss", [("2,3-rect", 3, "equal"), ("2,3-rect", 3, "exp"),
                                             ("2-rect", 2, "exp"), ("gauss", 1, "equal"),
                                             ("3-rect", 4, "equal")])
def test_score_paper_bank(vq, filters, S, gauss):
    """The paper's coarse Gaussian / Haar filters at sub-scales (multi-rectangle, signed
    integer weights) through the generic score kernel, against the oracle's direct counts."""
    H, W, th, tw, k = 90, 150, 36, 44, 9
    r = np.random.default_rng(31)
    q = synth.query_map(H, W, 4, M=6, n_sp=90, seed=7)
    ql = (q.sp_id.numpy() * 5 % k).astype(np.int32)
    ql[r.random(ql.shape) < 0.05] = r.integers(0, k)
    t = ql[20:20 + th, 61:61 + tw].copy()
    bank = synth.paper_bank(th, tw, filters, S, gauss)
    tc = oracle.filter_counts(t, k, bank)
    got_tc = vq.vqnnf_filter_responses(_dev(t.astype(np.uint8)), k, bank)
    assert np.array_equal(got_tc.cpu().numpy(), tc)
    ref, _ = oracle.score(ql, k, th, tw, bank, tc)
    heat, am = vq.vqnnf_score(_dev(ql.astype(np.uint8)), k, th, tw, bank, _dev(tc.astype(np.int32)))
    _check_heat(heat.cpu().numpy(), tuple(am.cpu().tolist()), ref, 1e-5, bank)
    assert tuple(am.cpu().tolist()) == (20, 61) or ref[20, 61] == ref.max()


def test_score_k1_and_whole_query(vq):
    ql = np.zeros((50, 40), np.int32)
    bank = synth.grid_bank(10, 8, 3)
    tc = oracle.filter_counts(ql[:10, :8], 1, bank)
    heat, am = vq.vqnnf_score(_dev(ql.astype(np.uint8)), 1, 10, 8, bank, _dev(tc.astype(np.int32)))
    assert float(heat.abs().max()) == 0.0 and am.cpu().tolist() == [0, 0]
    r = np.random.default_rng(9)
    ql = r.integers(0, 5, size=(23, 31)).astype(np.int32)
    bank = synth.grid_bank(23, 31, 2)
    tc = oracle.filter_counts(ql, 5, bank)
    heat, am = vq.vqnnf_score(_dev(ql.astype(np.uint8)), 5, 23, 31, bank, _dev(tc.astype(np.int32)))
    assert heat.shape == (1, 1) and float(heat[0, 0]) == 0.0


@pytest.mark.parametrize("prec", PRECS)
def test_whole_path_config1(vq, prec):
    """256x256 query, D=64, k=16, 32x32 template, F=5: every step on the GPU vs the oracle."""
    q = synth.query_map(256, 256, 64, M=32, n_sp=200, seed=1000)
    T, (ty, tx) = synth.crop_template(q, 32, 32, seed=2000)
    k, iters, seed = 16, 10, 3000
    bank = synth.grid_bank(32, 32, 2)
    C = vq.vqnnf_fit_codebook(_dev(T), k, iters, seed, prec)
    t_lab = vq.vqnnf_assign(_dev(T), C, prec)
    q_lab = vq.vqnnf_assign(_dev(q.X), C, prec)
    tc = vq.vqnnf_filter_responses(t_lab, k, bank)
    heat, am = vq.vqnnf_score(q_lab, k, 32, 32, bank, tc)
    C_ref = oracle.fit_codebook(T.numpy(), k, iters, seed)
    assert np.array_equal(C.cpu().numpy(), C_ref)
    ql_ref, d1, d2 = oracle.assign(q.X.numpy(), C_ref, return_dist=True)
    bad, _ = _labels_ok(q_lab.cpu().numpy(), ql_ref, d1, d2)
    assert bad == 0
    tl_ref = oracle.assign(T.numpy(), C_ref)
    tc_ref = oracle.filter_counts(tl_ref, k, bank)
    heat_ref, _ = oracle.score(ql_ref, k, 32, 32, bank, tc_ref)
    _check_heat(heat.cpu().numpy(), tuple(am.cpu().tolist()), heat_ref, 1e-4)


def test_whole_path_graph_capture(vq):
    """The calls only enqueue work: the whole path captures into a CUDA graph and replays
    to the same results."""
    q = synth.query_map(128, 96, 32, M=10, n_sp=50, seed=11)
    T, _ = synth.crop_template(q, 20, 16, seed=12)
    k, bank = 12, vq.Bank(synth.grid_bank(20, 16, 3))
    X, Td = _dev(q.X), _dev(T)
    ws_fit = vq.Workspace(vq.vqnnf_workspace_bytes(0, 20, 16, 32, 12))
    ws_a = vq.Workspace(vq.vqnnf_workspace_bytes(1, 128, 96, 32, 12))
    ws_s = vq.Workspace(vq.vqnnf_workspace_bytes(3, 128, 96, 0, 12, 20, 16, bank.F))
    C = torch.empty((k, 32), device="cuda")
    tl = torch.empty((20, 16), dtype=torch.uint8, device="cuda")
    ql = torch.empty((128, 96), dtype=torch.uint8, device="cuda")
    tc = torch.empty((bank.F, k), dtype=torch.int32, device="cuda")
    heat = torch.empty((109, 81), device="cuda")
    am = torch.empty(2, dtype=torch.int32, device="cuda")

    def step(stream=None):
        vq.vqnnf_fit_codebook(Td, k, 5, 1, C=C, ws=ws_fit, stream=stream)
        vq.vqnnf_assign(Td, C, labels=tl, ws=ws_a, stream=stream)
        vq.vqnnf_assign(X, C, labels=ql, ws=ws_a, stream=stream)
        vq.vqnnf_filter_responses(tl, k, bank, counts=tc, stream=stream)
        vq.vqnnf_score(ql, k, 20, 16, bank, tc, heatmap=heat, argmax_yx=am, ws=ws_s, stream=stream)

    step()
    torch.cuda.synchronize()
    want = (C.clone(), ql.clone(), heat.clone(), am.clone())
    for t in (C, ql, heat, am):
        t.zero_()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            step(stream=s)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip((C, ql, heat, am), want):
        assert torch.equal(a, b)


def test_score_large_template_uses_32bit_table(vq):
    """Template area above 65,535 pixels: the integral image is kept in 32 bits."""
    r = np.random.default_rng(21)
    k, th, tw = 5, 260, 260
    q = synth.query_map(300, 290, 4, M=6, n_sp=400, seed=21)
    ql = (q.sp_id.numpy() * 3 % k).astype(np.int32)
    ql[r.random(ql.shape) < 0.02] = r.integers(0, k)
    t = ql[10:10 + th, 7:7 + tw].copy()
    bank = synth.grid_bank(th, tw, 2)
    tc = oracle.filter_counts(t, k, bank)
    ref, _ = oracle.score(ql, k, th, tw, bank, tc)
    heat, am = vq.vqnnf_score(_dev(ql.astype(np.uint8)), k, th, tw, bank, _dev(tc.astype(np.int32)))
    _check_heat(heat.cpu().numpy(), tuple(am.cpu().tolist()), ref, 1e-5, bank)
    assert am.cpu().tolist() == [10, 7]
