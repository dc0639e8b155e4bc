"""Batched matching (many templates of uneven size and k against many queries) on the GPU.

* Every pair equals the single-pair path through the C ABI (codebook with seed + j, BF16
  assignment, grid-bank responses, score) bit for bit: sharing one contraction between
  several codebooks changes no label, count or heatmap value.
* Every pair against the FP64 oracle: labels outside the near-tie band, heatmap within
  1e-4 of max|H| (the whole-path tolerance of the single-pair tests), argmax a maximum.
* Plans (one launch per group with 128 or 256 shared columns, feature boxes in flight, L2
  prefetch; or the stationary launches, features read once per tile for every group) give
  identical results; the tuner returns one of its candidates; the call captures into a CUDA
  graph.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

D, G, ITERS, SEED = 32, 3, 3, 500
QUERIES = [(70, 90), (64, 64), (101, 77)]
# (h, w, k): ten codebooks of 8 (more than the eight segments a group may hold), the
# uneven sizes of the batching workload, and k = 256 (a group of its own)
TEMPLATES = [(16, 20, 8), (24, 18, 16), (30, 30, 40), (17, 23, 64), (20, 16, 100), (22, 25, 8),
             (18, 18, 8), (19, 21, 8), (16, 16, 8), (21, 17, 8), (23, 19, 8), (16, 24, 8), (20, 20, 8),
             (24, 24, 256), (26, 22, 32)]


@pytest.fixture(scope="module")
def vq():
    from paper_2306_15010_gb300 import build
    build.build()
    import paper_2306_15010_gb300 as m
    torch.cuda.set_device(0)
    return m


@pytest.fixture(scope="module")
def case():
    qs = [synth.query_map(H, W, D, M=12, n_sp=max(8, H * W // 150), seed=SEED + i) for i, (H, W) in
          enumerate(QUERIES)]
    ts = []
    for j, (h, w, k) in enumerate(TEMPLATES):
        T, _ = synth.crop_template(qs[j % len(qs)], h, w, seed=SEED + 100 + j)
        ts.append(T)
    return qs, ts, [k for (_, _, k) in TEMPLATES]


@pytest.fixture(scope="module")
def single(vq, case):
    """The single-pair path per pair: heatmaps, maxima, codebooks and query labels."""
    qs, ts, ks = case
    heats, ams, Cs, qlabs = {}, {}, [], {}
    for j, (T, k) in enumerate(zip(ts, ks)):
        h, w = T.shape[:2]
        bank = synth.grid_bank(h, w, G)
        Td = T.cuda()
        C = vq.vqnnf_fit_codebook(Td, k, ITERS, SEED + j, "bf16")
        tl = vq.vqnnf_assign(Td, C, "bf16")
        tc = vq.vqnnf_filter_responses(tl, k, bank)
        Cs.append(C.cpu().numpy())
        for i, q in enumerate(qs):
            ql = vq.vqnnf_assign(q.X.cuda(), C, "bf16")
            heat, am = vq.vqnnf_score(ql, k, h, w, bank, tc)
            heats[i, j], ams[i, j], qlabs[i, j] = heat.cpu(), am.cpu(), ql.cpu().numpy()
    return heats, ams, Cs, qlabs


def _run(vq, case, plan=None, heat=True):
    qs, ts, ks = case
    return vq.vqnnf_match_batch([q.X.cuda() for q in qs], [T.cuda() for T in ts], ks, ITERS, SEED, G, plan,
                                heat=heat)


def test_batch_equals_single_pair_path(vq, case, single):
    heats, ams = _run(vq, case)
    torch.cuda.synchronize()
    s_heat, s_am, _, _ = single
    for i in range(len(QUERIES)):
        for j in range(len(TEMPLATES)):
            assert torch.equal(heats[i][j].cpu(), s_heat[i, j]), (i, j)
            assert ams[i, j].cpu().tolist() == s_am[i, j].tolist(), (i, j)


def test_batch_against_oracle(vq, case, single):
    qs, ts, ks = case
    heats, ams = _run(vq, case)
    _, _, Cs, qlabs = single
    for j, (T, k) in enumerate(zip(ts, ks)):
        h, w = T.shape[:2]
        bank = synth.grid_bank(h, w, G)
        C_ref = oracle.fit_codebook(T.numpy(), k, ITERS, SEED + j)
        assert np.array_equal(Cs[j], C_ref), j
        tl = oracle.assign(T.numpy(), C_ref)
        tc = oracle.filter_counts(tl, k, bank)
        for i, q in enumerate(qs):
            ql, d1, d2 = oracle.assign(q.X.numpy(), C_ref, return_dist=True)
            band = oracle.relative_gap(d1, d2) < 1e-6
            assert not ((qlabs[i, j].astype(np.int32) != ql) & ~band).any(), (i, j)
            ref, _ = oracle.score(ql, k, h, w, bank, tc)
            got = heats[i][j].cpu().numpy()
            scale = max(np.abs(ref).max(), 1e-30)
            assert np.abs(got - ref).max() <= 1e-4 * scale, (i, j)
            y, x = ams[i, j].cpu().tolist()
            assert ref[y, x] >= ref.max() - 2e-4 * scale, (i, j)


@pytest.mark.parametrize("gc,sf,pf,stat", [(128, 0, -1, 0), (256, 4, 0, 0), (256, 8, 8, 0), (128, 6, 0, 0),
                                           (256, 0, -1, 1)])
def test_batch_plans_agree(vq, case, single, gc, sf, pf, stat):
    """One launch per group (any group width, feature stages, prefetch) and the stationary
    launches (every group against features read once per tile) give identical results."""
    heats, ams = _run(vq, case, vq.BatchPlan(gc, sf, pf, stat))
    s_heat, s_am, _, _ = single
    for i in range(len(QUERIES)):
        for j in range(len(TEMPLATES)):
            assert torch.equal(heats[i][j].cpu(), s_heat[i, j]), (gc, sf, pf, stat, i, j)
            assert ams[i, j].cpu().tolist() == s_am[i, j].tolist()


def test_batch_tune_and_maxima_only(vq, case, single):
    qs, ts, ks = case
    plan = vq.vqnnf_batch_tune([q.X.cuda() for q in qs], [T.cuda() for T in ts], ks, ITERS, SEED, G)
    assert plan.stationary == 1 or (plan.group_cols in (128, 256) and plan.sf in (4, 6, 8) and plan.pf in (0, 8))
    heats, ams = _run(vq, case, plan, heat=False)
    assert heats is None
    _, s_am, _, _ = single
    for i in range(len(QUERIES)):
        for j in range(len(TEMPLATES)):
            assert ams[i, j].cpu().tolist() == s_am[i, j].tolist()


def test_batch_graph_capture(vq, case):
    qs, ts, ks = case
    Xs = [q.X.cuda() for q in qs]
    Ts = [T.cuda() for T in ts]
    heats = [torch.empty((X.shape[0] - T.shape[0] + 1, X.shape[1] - T.shape[1] + 1), device="cuda")
             for X in Xs for T in Ts]
    am = torch.empty((len(Xs), len(Ts), 2), dtype=torch.int32, device="cuda")
    ws = vq.Workspace(vq.vqnnf_batch_workspace_bytes(Xs, Ts, ks, G))
    s = torch.cuda.Stream()

    def step(stream=None):
        vq.vqnnf_match_batch(Xs, Ts, ks, ITERS, SEED, G, heat=heats, argmax_yx=am, ws=ws, stream=stream)

    step()
    torch.cuda.synchronize()
    want = [h.clone() for h in heats] + [am.clone()]
    for t in heats + [am]:
        t.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            step(stream=s)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(heats + [am], want):
        assert torch.equal(a, b)


def test_batch_argument_errors(vq, case):
    qs, ts, ks = case
    Xs = [q.X.cuda() for q in qs]
    Ts = [T.cuda() for T in ts]
    big = torch.zeros((80, 95, D), device="cuda")            # larger than the 64 x 64 query
    with pytest.raises(vq.VqnnfError) as e:
        vq.vqnnf_match_batch(Xs, Ts[:2] + [big], ks[:2] + [8], ITERS, SEED, G)
    assert e.value.status == 1
    with pytest.raises(vq.VqnnfError) as e:                  # k > h w
        vq.vqnnf_match_batch(Xs, [Ts[0]], [16 * 20 + 1], ITERS, SEED, G)
    assert e.value.status == 1
    with pytest.raises(vq.VqnnfError) as e:                  # unsupported grid
        vq.vqnnf_match_batch(Xs, [Ts[0]], [8], ITERS, SEED, 5)
    assert e.value.status == 5
    with pytest.raises(vq.VqnnfError) as e:                  # plan outside the candidates
        vq.vqnnf_match_batch(Xs, [Ts[0]], [8], ITERS, SEED, G, vq.BatchPlan(64, 0, -1))
    assert e.value.status == 1


def test_batch_wide_template_and_tiny_query(vq):
    """A template wider than the grid score kernel stages (the generic score kernel) and a
    query that is exactly one template: still bit-identical to the single-pair path."""
    q1 = synth.query_map(60, 420, 32, M=8, n_sp=60, seed=901)
    q2 = synth.query_map(40, 300, 32, M=8, n_sp=40, seed=902)
    T1, _ = synth.crop_template(q1, 20, 300, seed=903)                 # 300 columns wide
    T2 = q2.X[:40, :300].clone()                                       # the whole second query
    Xs, Ts, ks = [q1.X.cuda(), q2.X.cuda()], [T1.cuda(), T2.cuda()], [12, 40]
    heats, ams = vq.vqnnf_match_batch(Xs, Ts, ks, 3, 77, 2)
    for j, (T, k) in enumerate(zip(Ts, ks)):
        h, w = T.shape[:2]
        bank = synth.grid_bank(h, w, 2)
        C = vq.vqnnf_fit_codebook(T, k, 3, 77 + j, "bf16")
        tc = vq.vqnnf_filter_responses(vq.vqnnf_assign(T, C, "bf16"), k, bank)
        for i, X in enumerate(Xs):
            if h > X.shape[0] or w > X.shape[1]:
                continue
            heat, am = vq.vqnnf_score(vq.vqnnf_assign(X, C, "bf16"), k, h, w, bank, tc)
            assert torch.equal(heats[i][j], heat), (i, j)
            assert ams[i, j].tolist() == am.tolist()
