"""Pins for the FP64 oracle: checks against things other than the oracle itself.

Exact rational brute force on tiny inputs, an independent summed-area-table route, the
textbook histogram L1, closed forms of Algorithm 2, invariants of the counts and of Eq. 2,
symmetries, the k-means objective, and the published SplitMix64 outputs.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from tests import _brute

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(s):
    return np.random.default_rng(s)


# ---------------------------------------------------------------- SplitMix64 / init
def test_splitmix64_published_outputs():
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    assert oracle.splitmix64(0, 3) == want
    assert _brute.splitmix64(0, 3) == want


@pytest.mark.parametrize("seed", [1, 12345, 2**63 + 7, 2**64 - 1])
def test_splitmix64_matches_definition(seed):
    assert oracle.splitmix64(seed, 20) == _brute.splitmix64(seed, 20)


def test_kmeans_init_k1_closed_form():
    for seed in (0, 5, 99):
        r = _brute.splitmix64(seed, 1)[0]
        assert oracle.kmeans_init(1000, 1, seed)[0] == r % 1000


@pytest.mark.parametrize("l,k", [(10, 10), (100, 7), (16384, 128)])
def test_kmeans_init_distinct(l, k):
    idx = oracle.kmeans_init(l, k, 42)
    assert len(set(idx.tolist())) == k
    assert idx.min() >= 0 and idx.max() < l
    if k == l:
        assert sorted(idx.tolist()) == list(range(l))


def test_kmeans_init_rejects_k_above_l():
    with pytest.raises(ValueError):
        oracle.kmeans_init(3, 4, 0)


# ---------------------------------------------------------------- nearest neighbours
@pytest.mark.parametrize("seed", range(4))
def test_assign_exact_bruteforce(seed):
    r = _rng(seed)
    X = r.normal(size=(60, 5)).astype(np.float32)
    C = r.normal(size=(7, 5)).astype(np.float32)
    assert np.array_equal(oracle.assign(X, C), _brute.nn_exact(X, C))


def test_assign_tie_takes_lowest_index():
    # duplicate centroids and points exactly half-way between two centroids
    C = np.array([[1, 0], [0, 0], [1, 0], [2, 0]], np.float32)
    X = np.array([[1, 0], [0.5, 0], [1.5, 0], [3, 0], [-1, 0]], np.float32)
    lab, d1, d2 = oracle.assign(X, C, return_dist=True)
    assert lab.tolist() == [0, 0, 0, 3, 1]
    assert np.array_equal(lab, _brute.nn_exact(X, C))
    assert d1[0] == 0 and d2[0] == 0          # duplicate centroids -> relative gap 0
    assert oracle.relative_gap(d1, d2)[0] == 0


def test_assign_distances_exact_small_integers():
    X = np.array([[3, 4, 0]], np.float32)
    C = np.array([[0, 0, 0], [3, 4, 1], [6, 8, 0]], np.float32)
    lab, d1, d2 = oracle.assign(X, C, return_dist=True)
    assert lab[0] == 1 and d1[0] == 1.0 and d2[0] == 25.0


def test_assign_permutation_symmetry():
    r = _rng(7)
    X = r.random((500, 16)).astype(np.float32)
    C = r.random((12, 16)).astype(np.float32)
    perm = r.permutation(12)
    lab = oracle.assign(X, C)
    lab_p = oracle.assign(X, C[perm])
    assert np.array_equal(perm[lab_p], lab)


def test_assign_fp64_matches_exact_on_near_ties():
    # centroids a hair apart: FP64 must still order them exactly like rationals
    r = _rng(3)
    c0 = r.random(8).astype(np.float32)
    C = np.stack([c0, np.nextafter(c0, np.float32(2)), c0 + np.float32(1e-3)])
    X = (c0[None] + r.normal(scale=1e-3, size=(200, 8))).astype(np.float32)
    assert np.array_equal(oracle.assign(X, C), _brute.nn_exact(X, C))


# ---------------------------------------------------------------- k-means
@pytest.mark.parametrize("seed", [0, 1])
def test_fit_codebook_equals_exact_lloyd(seed):
    r = _rng(seed)
    T = (r.integers(0, 9, size=(40, 3)) / 8.0 + r.normal(scale=0.05, size=(40, 3))).astype(np.float32)
    k, iters = 4, 5
    init = oracle.kmeans_init(40, k, seed)
    want = _brute.lloyd_exact(T, init, iters)
    got = oracle.fit_codebook(T, k, iters, seed)
    assert np.array_equal(got, want)


def test_fit_zero_iters_is_init():
    r = _rng(2)
    T = r.random((50, 4)).astype(np.float32)
    C = oracle.fit_codebook(T, 6, 0, 77)
    assert np.array_equal(C, T[oracle.kmeans_init(50, 6, 77)])


def test_lloyd_objective_non_increasing():
    q = synth.query_map(48, 48, 8, M=6, n_sp=20, seed=11)
    T = q.X.numpy().reshape(-1, 8)
    obj = [oracle.kmeans_objective(T, oracle.fit_codebook(T, 10, it, 3)) for it in range(8)]
    for a, b in zip(obj, obj[1:]):
        assert b <= a * (1 + 1e-12)
    assert obj[-1] < obj[0]


def test_kmeans_k_equals_l_zero_objective():
    r = _rng(4)
    T = r.random((9, 3)).astype(np.float32)
    C = oracle.fit_codebook(T, 9, 3, 1)
    assert oracle.kmeans_objective(T, C) == 0.0


def test_kmeans_planted_clusters_recovered():
    # four well separated clusters; with seed chosen so that init hits all four, the
    # means come out within noise of the planted centres
    r = _rng(5)
    centres = np.array([[0, 0], [10, 0], [0, 10], [10, 10]], np.float64)
    T = np.concatenate([c + r.normal(scale=0.1, size=(50, 2)) for c in centres]).astype(np.float32)
    for seed in range(50):
        init = oracle.kmeans_init(200, 4, seed)
        if len(set((init // 50).tolist())) == 4:
            break
    C = oracle.fit_codebook(T, 4, 5, seed)
    for c in centres:
        assert np.min(np.linalg.norm(C - c, axis=1)) < 0.05


# ---------------------------------------------------------------- counts / score
def _labels(r, H, W, k):
    return r.integers(0, k, size=(H, W)).astype(np.int32)


def test_counts_match_sat_route_and_invariant():
    r = _rng(8)
    lab = _labels(r, 40, 37, 6)
    bank = synth.grid_bank(12, 15, 3)
    S = _brute.sat(lab, 6)
    for (wy, wx) in [(0, 0), (28, 22), (5, 9), (17, 3)]:
        got = oracle.window_counts(lab, 6, bank, wy, wx)
        assert np.array_equal(got, _brute.counts_via_sat(S, bank, wy, wx))
        for f, filt in enumerate(bank):
            (x0, y0, x1, y1, _), = filt["rects"]
            assert got[f].sum() == (x1 - x0) * (y1 - y0)      # one label per pixel


def test_template_counts_are_window_counts_at_origin():
    r = _rng(9)
    lab = _labels(r, 10, 14, 5)
    bank = synth.grid_bank(10, 14, 2)
    assert np.array_equal(oracle.filter_counts(lab, 5, bank),
                          oracle.window_counts(lab, 5, bank, 0, 0))


def test_score_exact_bruteforce_tiny():
    r = _rng(10)
    k = 3
    q = _labels(r, 6, 5, k)
    t = _labels(r, 3, 2, k)
    bank = [{"rects": [(0, 0, 2, 3, 1)], "w_f": 1.0, "area": 6.0},
            {"rects": [(0, 0, 1, 3, 1)], "w_f": 0.25, "area": 3.0},
            {"rects": [(1, 1, 2, 3, 2), (0, 0, 1, 1, 1)], "w_f": 0.5, "area": 6.0}]
    want, tc = _brute.heatmap_via_sat(q, t, k, bank)
    assert np.array_equal(oracle.filter_counts(t, k, bank), tc)
    heat, am = oracle.score(q, k, 3, 2, bank, tc)
    assert heat.shape == want.shape
    for y in range(heat.shape[0]):
        for x in range(heat.shape[1]):
            assert abs(heat[y, x] - float(want[y, x])) <= 1e-15 * max(1.0, abs(float(want[y, x])))
    wv = np.vectorize(float)(want)
    best = np.flatnonzero(wv.ravel() == wv.max())[0]
    assert am == (best // wv.shape[1], best % wv.shape[1])


def test_score_single_full_filter_is_histogram_l1():
    r = _rng(11)
    k = 7
    q = _labels(r, 30, 26, k)
    t = q[4:13, 6:17].copy()
    t[0, 0] = (t[0, 0] + 1) % k
    bank = synth.grid_bank(9, 11, 1, full=False)       # one filter: the full window
    heat, _ = oracle.score(q, k, 9, 11, bank, oracle.filter_counts(t, k, bank))
    np.testing.assert_allclose(heat, _brute.histogram_score(q, t, k), rtol=0, atol=1e-14)


def test_score_self_match_peaks_at_zero():
    q = synth.query_map(64, 64, 8, M=8, n_sp=40, seed=3)
    T, (y, x) = synth.crop_template(q, 16, 16, seed=4, sigma=0.0)   # cut unaltered
    C = oracle.fit_codebook(T.numpy(), 8, 4, 9)
    ql = oracle.assign(q.X.numpy(), C)
    tl = oracle.assign(T.numpy(), C)
    assert np.array_equal(tl, ql[y:y + 16, x:x + 16])
    bank = synth.grid_bank(16, 16, 3)
    heat, am = oracle.score(ql, 8, 16, 16, bank, oracle.filter_counts(tl, 8, bank))
    assert heat[y, x] == 0.0
    assert heat.max() == 0.0
    assert heat[am] == 0.0 and am <= (y, x)


def test_score_k1_is_identically_zero():
    q = np.zeros((12, 10), np.int32)
    bank = synth.grid_bank(4, 3, 2)
    heat, am = oracle.score(q, 1, 4, 3, bank, oracle.filter_counts(q[:4, :3], 1, bank))
    assert np.all(heat == 0.0) and am == (0, 0)


def test_score_template_is_whole_query():
    r = _rng(12)
    q = _labels(r, 9, 8, 4)
    bank = synth.grid_bank(9, 8, 3)
    heat, am = oracle.score(q, 4, 9, 8, bank, oracle.filter_counts(q, 4, bank))
    assert heat.shape == (1, 1) and heat[0, 0] == 0.0 and am == (0, 0)


def test_score_translation_shifts_heatmap():
    r = _rng(13)
    k = 5
    q = _labels(r, 25, 22, k)
    t = _labels(r, 6, 7, k)
    bank = synth.grid_bank(6, 7, 2)
    tc = oracle.filter_counts(t, k, bank)
    big = _labels(r, 25 + 3, 22 + 4, k)
    big[3:, 4:] = q
    h0, _ = oracle.score(q, k, 6, 7, bank, tc)
    h1, _ = oracle.score(big, k, 6, 7, bank, tc)
    assert np.array_equal(h1[3:, 4:], h0)


def test_score_weight_scaling_and_label_permutation():
    r = _rng(14)
    k = 6
    q = _labels(r, 20, 21, k)
    t = _labels(r, 8, 6, k)
    bank = synth.grid_bank(8, 6, 2)
    tc = oracle.filter_counts(t, k, bank)
    h, _ = oracle.score(q, k, 8, 6, bank, tc)
    bank4 = [dict(f, w_f=4.0 * f["w_f"]) for f in bank]
    h4, _ = oracle.score(q, k, 8, 6, bank4, tc)
    assert np.array_equal(h4, 4.0 * h)
    perm = r.permutation(k)
    hp, _ = oracle.score(perm[q].astype(np.int32), k, 8, 6, bank,
                         oracle.filter_counts(perm[t].astype(np.int32), k, bank))
    assert np.array_equal(hp, h)


def test_score_at_matches_full_heatmap():
    r = _rng(15)
    k = 4
    q = _labels(r, 30, 30, k)
    t = _labels(r, 7, 9, k)
    bank = synth.grid_bank(7, 9, 3)
    tc = oracle.filter_counts(t, k, bank)
    heat, _ = oracle.score(q, k, 7, 9, bank, tc)
    win = np.array([[0, 0], [23, 21], [11, 5], [3, 17]])
    assert np.array_equal(oracle.score_at(q, k, bank, tc, win), heat[win[:, 0], win[:, 1]])


def test_score_rejects_template_larger_than_query():
    q = np.zeros((4, 4), np.int32)
    with pytest.raises(ValueError):
        oracle.score(q, 1, 5, 2, synth.grid_bank(5, 2, 1), np.zeros((2, 1), np.int64))


# ---------------------------------------------------------------- Algorithm 2
def test_alg2_unit_filter_closed_form():
    a = 3.5
    np.testing.assert_array_equal(oracle.coarse_to_dilation([[a]]), a * np.array([[1, -1], [-1, 1]]))


@pytest.mark.parametrize("g", [2, 3, 5])
def test_alg2_all_ones_telescopes_to_outer_corners(g):
    fd = oracle.coarse_to_dilation(np.ones((g, g)))
    want = np.zeros((g + 1, g + 1))
    want[0, 0] = want[g, g] = 1
    want[0, g] = want[g, 0] = -1
    np.testing.assert_array_equal(fd, want)


def test_alg2_dilation_on_integral_image_equals_direct_bins():
    r = _rng(16)
    k, r_w, r_h, d_x, d_y = 4, 3, 2, 4, 5
    lab = _labels(r, 30, 28, k)
    S = _brute.sat(lab, k)
    f_i = r.integers(-3, 4, size=(r_w, r_h)).astype(np.float64)
    fd = oracle.coarse_to_dilation(f_i)
    for (wy, wx) in [(0, 0), (7, 11), (19, 15)]:
        for cls in range(k):
            via_sat = sum(fd[i, j] * S[wy + j * d_y, wx + i * d_x, cls]
                          for i in range(r_w + 1) for j in range(r_h + 1))
            assert via_sat == oracle.coarse_direct(lab, wy, wx, cls, f_i, d_x, d_y)
