"""Pins of the soft-VQ oracle (oracle/soft.py), CPU only:

* gradients against FP64 central differences (every entry on a tiny instance; sampled
  entries on the 64 x 64, D = 16, k = 8 instance of the differentiation workload);
* the tau -> 0 limit equals the hard heatmap of Eq. 2 computed by the hard oracle (labels by
  brute-force nearest neighbour, counts by direct counting);
* soft counts sum to the cell area (sum_j p_j = 1), and the heatmap is linear in w.
"""
import numpy as np
import pytest

import oracle
from oracle import soft


def _instance(B, H, W, D, k, th, tw, seed):
    r = np.random.default_rng(seed)
    C = r.normal(0, 1, (k, D))
    lab = r.integers(0, k, (B, H, W))
    Q = C[lab] + r.normal(0, 0.7, (B, H, W, D))
    T = Q[0, 1:1 + th, 2:2 + tw] + r.normal(0, 0.2, (th, tw, D))
    return Q, T, C


def _loss(Q, T, C, tau, G, wf, Gw):
    return float((soft.soft_forward(Q, T, C, tau, G, wf)["heat"] * Gw).sum())


def test_gradients_match_central_differences_everywhere():
    Q, T, C = _instance(2, 9, 10, 3, 3, 6, 5, seed=1)
    tau, G = 0.7, 3
    r = np.random.default_rng(2)
    wf = r.uniform(0.5, 1.5, G * G)
    Gw = r.normal(0, 1, (2, 9 - 6 + 1, 10 - 5 + 1))
    dQ, dC, dw = soft.soft_backward(Q, T, C, tau, G, wf, Gw)
    eps = 1e-6
    for arr, grad in ((Q, dQ), (C, dC), (wf, dw)):
        num = np.zeros_like(grad)
        for idx in np.ndindex(arr.shape):
            keep = arr[idx]
            arr[idx] = keep + eps
            lp = _loss(Q, T, C, tau, G, wf, Gw)
            arr[idx] = keep - eps
            lm = _loss(Q, T, C, tau, G, wf, Gw)
            arr[idx] = keep
            num[idx] = (lp - lm) / (2 * eps)
        assert np.allclose(grad, num, rtol=1e-5, atol=1e-7 * max(1.0, np.abs(num).max()))


def test_gradients_sampled_on_the_fd_workload():
    # the FD instance of the differentiation workload: 64 x 64 query, D = 16, k = 8
    Q, T, C = _instance(1, 64, 64, 16, 8, 21, 24, seed=3)
    tau, G = 0.1, 3
    r = np.random.default_rng(4)
    wf = np.ones(G * G)
    Gw = r.normal(0, 1, (1, 64 - 21 + 1, 64 - 24 + 1))
    dQ, dC, dw = soft.soft_backward(Q, T, C, tau, G, wf, Gw)
    eps = 1e-6
    picks = [(Q, dQ, tuple(r.integers(0, s) for s in Q.shape)) for _ in range(25)]
    picks += [(C, dC, tuple(r.integers(0, s) for s in C.shape)) for _ in range(15)]
    picks += [(wf, dw, (i,)) for i in range(G * G)]
    for arr, grad, idx in picks:
        keep = arr[idx]
        arr[idx] = keep + eps
        lp = _loss(Q, T, C, tau, G, wf, Gw)
        arr[idx] = keep - eps
        lm = _loss(Q, T, C, tau, G, wf, Gw)
        arr[idx] = keep
        num = (lp - lm) / (2 * eps)
        assert abs(grad[idx] - num) <= 1e-5 * max(1.0, abs(num)), (idx, grad[idx], num)


def test_zero_temperature_limit_is_the_hard_heatmap():
    r = np.random.default_rng(5)
    k, D, G = 5, 4, 3
    C = r.normal(0, 3, (k, D))
    lab = (np.arange(40 * 37).reshape(40, 37) // 7 + r.integers(0, 3, (40, 37))) % k
    Q = C[lab] + r.normal(0, 0.01, (40, 37, D))
    th, tw = 12, 10
    T = Q[5:5 + th, 9:9 + tw].copy()
    wf = r.uniform(0.5, 2.0, G * G)
    heat = soft.soft_forward(Q[None], T, C, 1e-4, G, wf)["heat"][0]
    ql = oracle.assign(Q.astype(np.float32), C.astype(np.float32))
    tl = oracle.assign(T.astype(np.float32), C.astype(np.float32))
    bank = [{"rects": [(x0, y0, x1, y1, 1)], "w_f": float(wf[i]), "area": float((y1 - y0) * (x1 - x0))}
            for i, (y0, y1, x0, x1) in enumerate(soft.grid_cells(th, tw, G))]
    ref, _ = oracle.score(ql, k, th, tw, bank, oracle.filter_counts(tl, k, bank))
    assert np.allclose(heat, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def test_soft_counts_sum_to_areas_and_linear_in_weights():
    Q, T, C = _instance(2, 12, 13, 3, 4, 7, 8, seed=6)
    f = soft.soft_forward(Q, T, C, 0.3, 3, np.ones(9))
    assert np.allclose(f["T"].sum(-1), f["area"])
    assert np.allclose(f["Qc"].sum(-1), f["area"][:, None, None, None])
    w = np.random.default_rng(7).uniform(0, 2, 9)
    h1 = soft.soft_forward(Q, T, C, 0.3, 3, w)["heat"]
    h2 = soft.soft_forward(Q, T, C, 0.3, 3, 2.5 * w)["heat"]
    assert np.allclose(h2, 2.5 * h1)
