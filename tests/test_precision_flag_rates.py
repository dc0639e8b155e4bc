"""Why the assignment contraction is BF16 with three products and not FP8 (CPU only).

On a sample of the headline workload (the 2048-wide query generator, D = 512, k = 128 codebook
fitted by the oracle on the warped 128 x 128 template), the proven interval test of the
assignment (a pixel keeps every centroid j with s_j - B_j <= s_min + B_min, where B_j bounds
the contraction error of s_j = ||c_j'||^2 - 2 x'.c_j' on the centred vectors) flags a pixel for
exact re-scoring when more than one centroid survives.  With the per-product rounding error
((1 + u)^2 - 1) sum_i |x'_i| |c'_ji| of the contraction:

* FP8 e4m3 with per-row scales (u = 2^-4): most pixels are flagged, so the FP32 re-scoring
  would do most of the work, and without it many labels would be wrong;
* BF16, one product (u = 2^-8): a fifth of the pixels;
* BF16 with the three-product split x_hi c_hi + x_hi c_lo + x_lo c_hi (residual ~2^-16): about
  one pixel in a hundred, which is what the library runs.
"""
import numpy as np
import pytest
import torch

import oracle
import synth


@pytest.fixture(scope="module")
def sample():
    Hs, W, D, k = 128, 2048, 512, 128
    q = synth.query_map(Hs, W, D, M=128, n_sp=20000 * Hs // 2048, seed=1000)
    T, _ = synth.warped_template(q, 128, 128, seed=2000)
    C = oracle.fit_codebook(T.numpy(), k, 10, 3000).astype(np.float64)
    X = q.X.numpy().reshape(-1, D).astype(np.float64)[::16]          # 16384 pixels
    m = C.mean(0)
    return X - m, C - m


def _flag_rate(Xc, Cc, u):
    s = -2.0 * Xc @ Cc.T + (Cc ** 2).sum(1)[None, :]
    B = 2.0 * ((1.0 + u) ** 2 - 1.0) * (np.abs(Xc) @ np.abs(Cc).T)
    lab = s.argmin(1)
    U = s[np.arange(len(s)), lab] + B[np.arange(len(s)), lab]
    return float((((s - B) <= U[:, None]).sum(1) > 1).mean()), lab


def _fp8_rows(A):
    t = torch.tensor(A, dtype=torch.float32)
    sc = t.abs().amax(1, keepdim=True).clamp_min(1e-30) / 448.0      # per-row scale: absmax -> 448
    return ((t / sc).to(torch.float8_e4m3fn).to(torch.float32) * sc).double().numpy()


def test_flag_rates_by_contraction_precision(sample):
    Xc, Cc = sample
    fp8, lab = _flag_rate(Xc, Cc, 2.0 ** -4)
    bf1, _ = _flag_rate(Xc, Cc, 2.0 ** -8)
    bf3, _ = _flag_rate(Xc, Cc, 2.0 ** -16)
    assert fp8 > 0.5, fp8
    assert 0.05 < bf1 < 0.5, bf1
    assert bf3 < 0.03, bf3
    # the FP8 contraction itself, per-row scaled on both sides: its labels are wrong for a
    # sizeable fraction of the pixels, so the re-scoring could not be skipped
    Xq, Cq = _fp8_rows(Xc), _fp8_rows(Cc)
    s8 = -2.0 * Xq @ Cq.T + (Cc ** 2).sum(1)[None, :]
    wrong = float((s8.argmin(1) != lab).mean())
    assert wrong > 0.01, wrong
