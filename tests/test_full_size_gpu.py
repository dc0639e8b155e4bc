"""The whole path at full size, run the way bench.py times it, against the FP64 oracle on
what the oracle can compute one by one.  Two workloads: the headline one (2048 x 2048
query, D = 512, k = 128, 128 x 128 template, F = 10) and the precision study's D = 1024
variant (1024 x 1024 query, D = 1024, the same generator, codebook size and template).

* codebook: bit-identical to the oracle's fit of the same template (BF16, FP32 and FP8 paths);
* template labels: every pixel against the oracle (outside the 1e-6 near-tie band);
* query labels: BF16 == FP8 == FP32 on every pixel outside the band, and all three against the
  oracle on a seeded sample plus every pixel where the paths disagree;
* template counts: exact;
* heatmap, at every window the score kernel's tiling could get wrong (the four corners, the
  whole first and last valid rows and columns, both sides of every 256-window seam, which
  covers tile widths of 256, 512 and 1024) plus seeded random windows and the maximum,
  against the oracle's Eq. 2 of the GPU labels:
  - |H_gpu - H_ref| < min_f(w_f / A_f) / 2.  Every per-filter L1 sum is an integer and the
    float part is F float32 terms (about 1e-5 here), so a single count error anywhere shows;
  - every per-filter L1 sum exactly: the bank is scored again once per filter with that
    filter's weight 1 and the others 0 (same rectangles, same kernel), which gives
    H = -(1 / A_f) L1_f, and the integer L1_f recovered from it equals the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


# (H = W, D, superpixels): the superpixel count keeps the headline's superpixel size
WORKLOADS = {"d512_2048": (2048, 512, 20000), "d1024_1024": (1024, 1024, 5000)}


@pytest.fixture(scope="module", params=sorted(WORKLOADS))
def run(request):
    from paper_2306_15010_gb300 import build
    build.build()
    import paper_2306_15010_gb300 as vq
    import bench
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    cfg = dict(bench.HEADLINE)
    side, D, n_sp = WORKLOADS[request.param]
    cfg.update(H=side, W=side, D=D, n_sp=n_sp)
    q, T, info, bank = bench.make_workload(dev, cfg)
    s = torch.cuda.Stream(device=dev)
    out = {}
    for prec in ("bf16", "fp32", "fp8"):
        pipe = bench.Pipeline(vq, q.X, T, cfg, bank, prec, s)
        with torch.cuda.stream(s):
            pipe.step()
            pipe.step()
        torch.cuda.synchronize()
        assert vq.vqnnf_last_device_error() == 0
        out[prec] = {k: getattr(pipe, k).clone() for k in ("C", "tl", "ql", "tc", "heat", "am")}
        del pipe
    return cfg, q, T, bank, out


def test_codebook_bit_exact(run):
    cfg, q, T, bank, out = run
    C_ref = oracle.fit_codebook(T.cpu().numpy(), cfg["k"], cfg["iters"], cfg["fit_seed"])
    for prec in ("bf16", "fp32", "fp8"):
        assert np.array_equal(out[prec]["C"].cpu().numpy(), C_ref), prec


def test_template_labels_and_counts(run):
    cfg, q, T, bank, out = run
    C = out["fp32"]["C"].cpu().numpy()
    ref, d1, d2 = oracle.assign(T.cpu().numpy(), C, return_dist=True)
    band = oracle.relative_gap(d1, d2) < 1e-6
    for prec in ("bf16", "fp32", "fp8"):
        got = out[prec]["tl"].cpu().numpy().astype(np.int32)
        assert int(((got != ref) & ~band).sum()) == 0, prec
        tc = oracle.filter_counts(got, cfg["k"], bank)
        assert np.array_equal(out[prec]["tc"].cpu().numpy(), tc), prec


def test_query_labels(run):
    cfg, q, T, bank, out = run
    C = out["fp32"]["C"].cpu().numpy()
    lb = out["bf16"]["ql"].view(-1)
    lf = out["fp32"]["ql"].view(-1)
    l8 = out["fp8"]["ql"].view(-1)
    diff = ((lb != lf) | (l8 != lf)).nonzero().view(-1)
    rng = np.random.default_rng(7)
    sample = torch.as_tensor(rng.choice(lb.numel(), 4096, replace=False), device=lb.device)
    idx = torch.unique(torch.cat([diff[:20000], sample]))
    X = q.X.view(-1, cfg["D"])[idx].cpu().numpy()
    ref, d1, d2 = oracle.assign(X[None], C, return_dist=True)
    ref, band = ref[0], (oracle.relative_gap(d1, d2) < 1e-6)[0]
    for name, lab in (("bf16", lb), ("fp32", lf), ("fp8", l8)):
        got = lab[idx].cpu().numpy().astype(np.int32)
        assert int(((got != ref) & ~band).sum()) == 0, name
    # every disagreement between the paths lies in the near-tie band
    assert diff.numel() <= 20000
    in_diff = torch.isin(idx, diff).cpu().numpy()
    assert bool(band[in_diff].all())


def _windows(HO, WO, am, seed=11, seam=256):
    ys, xs = np.arange(HO), np.arange(WO)
    col = lambda x: np.stack([ys, np.full(HO, x)], 1)
    row = lambda y: np.stack([np.full(WO, y), xs], 1)
    parts = [row(0), row(HO - 1), col(0), col(WO - 1), np.asarray(am)[None]]
    for s0 in range(seam, WO, seam):
        parts += [col(s0 - 1), col(s0)]
    rng = np.random.default_rng(seed)
    parts.append(np.stack([rng.integers(0, HO, 256), rng.integers(0, WO, 256)], 1))
    return np.unique(np.concatenate(parts).astype(np.int32), axis=0)


def _unit_bank(bank, f):
    """The same filters with weight 1 for filter f and 0 for every other one."""
    return [dict(flt, w_f=1.0 if i == f else 0.0) for i, flt in enumerate(bank)]


def test_heatmap_exact_at_edges_and_seams(run):
    import paper_2306_15010_gb300 as vq
    cfg, q, T, bank, out = run
    k, th, tw = cfg["k"], cfg["th"], cfg["tw"]
    coef = np.array([f["w_f"] / f["area"] for f in bank])
    for prec in ("bf16", "fp32", "fp8"):
        ql_d, tc_d = out[prec]["ql"], out[prec]["tc"]
        ql = ql_d.cpu().numpy().astype(np.int32)
        tc = tc_d.cpu().numpy()
        heat = out[prec]["heat"]
        HO, WO = heat.shape
        am = out[prec]["am"].cpu().numpy()
        win = _windows(HO, WO, am)
        wy = torch.as_tensor(win[:, 0], device=heat.device, dtype=torch.long)
        wx = torch.as_tensor(win[:, 1], device=heat.device, dtype=torch.long)
        ref = oracle.score_at(ql, k, bank, tc, win)
        got = heat[wy, wx].cpu().numpy().astype(np.float64)
        err = np.abs(got - ref)
        assert err.max() < 0.5 * coef.min(), (prec, float(err.max()), win[int(err.argmax())])
        assert float(heat[am[0], am[1]]) == float(heat.max()), prec
        # every per-filter L1 sum, as an integer
        for f in range(len(bank)):
            ub = _unit_bank(bank, f)
            hf, _ = vq.vqnnf_score(ql_d, k, th, tw, ub, tc_d)
            c32 = np.float32(coef[f])
            l1_gpu = np.rint(-hf[wy, wx].cpu().numpy().astype(np.float64) / np.float64(c32))
            l1_ref = np.rint(-oracle.score_at(ql, k, [dict(bank[f], w_f=1.0)], tc[f:f + 1], win) *
                             bank[f]["area"])
            bad = np.flatnonzero(l1_gpu != l1_ref)
            assert bad.size == 0, (prec, f, win[bad[:5]], l1_gpu[bad[:5]], l1_ref[bad[:5]])
