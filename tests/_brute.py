"""Independent exact re-derivations used to pin the oracle on tiny inputs.

Nothing here is imported by the oracle or by the CUDA path.  Each routine reaches the
same quantity as the oracle by a different route or in exact arithmetic:

* nearest neighbours and k-means in exact rational arithmetic (``fractions.Fraction``),
* window counts through a numpy summed-area table (the oracle counts pixel by pixel),
* the single-filter score as the textbook L1 distance of two label histograms.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(seed: int, n: int) -> list[int]:
    """SplitMix64 written from its published definition (Steele, Lea & Flood 2014)."""
    out = []
    s = seed & MASK64
    for _ in range(n):
        s = (s + 0x9E3779B97F4A7C15) & MASK64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        out.append(z ^ (z >> 31))
    return out


def nn_exact(X: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Exact nearest centroid of every row (rational arithmetic, lowest index on ties)."""
    Xf = [[Fraction(float(v)) for v in row] for row in X.reshape(-1, X.shape[-1])]
    Cf = [[Fraction(float(v)) for v in row] for row in C]
    lab = []
    for x in Xf:
        best, arg = None, -1
        for j, c in enumerate(Cf):
            d = sum((a - b) * (a - b) for a, b in zip(x, c))
            if best is None or d < best:
                best, arg = d, j
        lab.append(arg)
    return np.array(lab, np.int32).reshape(X.shape[:-1])


def lloyd_exact(T: np.ndarray, init_idx, iters: int) -> np.ndarray:
    """Lloyd iterations with exact means, each mean rounded to float32 like a codebook."""
    T2 = T.reshape(-1, T.shape[-1]).astype(np.float32)
    C = T2[np.asarray(init_idx)].copy()
    for _ in range(iters):
        lab = nn_exact(T2, C)
        for j in range(C.shape[0]):
            members = T2[lab == j]
            if len(members) == 0:
                continue
            for i in range(C.shape[1]):
                m = sum((Fraction(float(v)) for v in members[:, i]), Fraction(0)) / len(members)
                C[j, i] = np.float32(float(m))
    return C


def sat(labels: np.ndarray, k: int) -> np.ndarray:
    """Exclusive-prefix integral image of the one-hot NNF: (H+1) x (W+1) x k int64."""
    H, W = labels.shape
    onehot = np.zeros((H, W, k), np.int64)
    onehot[np.arange(H)[:, None], np.arange(W)[None, :], labels] = 1
    S = np.zeros((H + 1, W + 1, k), np.int64)
    S[1:, 1:] = onehot.cumsum(0).cumsum(1)
    return S


def counts_via_sat(S: np.ndarray, bank, wy: int, wx: int) -> np.ndarray:
    k = S.shape[2]
    out = np.zeros((len(bank), k), np.int64)
    for f, filt in enumerate(bank):
        for (x0, y0, x1, y1, wgt) in filt["rects"]:
            X0, X1, Y0, Y1 = wx + x0, wx + x1, wy + y0, wy + y1
            out[f] += wgt * (S[Y1, X1] - S[Y0, X1] - S[Y1, X0] + S[Y0, X0])
    return out


def heatmap_via_sat(q_labels, t_labels, k, bank):
    """Eq. 2 heatmap with every count taken from summed-area tables, weights exact."""
    H, W = q_labels.shape
    th, tw = t_labels.shape
    Sq, St = sat(q_labels, k), sat(t_labels, k)
    tc = counts_via_sat(St, bank, 0, 0)
    heat = np.empty((H - th + 1, W - tw + 1), object)
    for y in range(H - th + 1):
        for x in range(W - tw + 1):
            qc = counts_via_sat(Sq, bank, y, x)
            s = Fraction(0)
            for f, filt in enumerate(bank):
                s -= Fraction(filt["w_f"]) / Fraction(filt["area"]) * int(np.abs(tc[f] - qc[f]).sum())
            heat[y, x] = s
    return heat, tc


def histogram_score(q_labels, t_labels, k):
    """Textbook: -(1/A) * L1(hist(template) - hist(window)) for every valid window."""
    H, W = q_labels.shape
    th, tw = t_labels.shape
    ht = np.bincount(t_labels.ravel(), minlength=k)
    out = np.empty((H - th + 1, W - tw + 1))
    for y in range(H - th + 1):
        for x in range(W - tw + 1):
            hq = np.bincount(q_labels[y:y + th, x:x + tw].ravel(), minlength=k)
            out[y, x] = -np.abs(ht - hq).sum() / float(th * tw)
    return out
