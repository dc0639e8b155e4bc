"""Soft vector-quantised heatmap and its gradients -- FP64 oracle.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``): the tests, the smoke run and
bench.py's CPU baseline may use it; the product path never does.

The differentiable reading of the method: the hard nearest-neighbour field of Algorithm 1 is
replaced by a soft assignment p_j(x) = softmax_j(-||x - c_j||^2 / tau) of every pixel, the
per-cluster filter responses of Eq. 1 by the same box sums of p (soft counts), and Eq. 2 is
kept as written, with |.| the L1 norm over clusters (subgradient sign(0) = 0):

    T_fj      = sum over template pixels v in cell f of p_j(v)
    Q_fj(y,x) = sum over query pixels u in cell f + (y, x) of p_j(u)
    H(y,x)    = - sum_f (w_f / A_f) sum_j | T_fj - Q_fj(y, x) |

The filters are the G x G grid cells of the template window (floor boundaries, Sec. 3.2.1),
A_f the cell area, w_f learnable weights.  For L = sum_{b,y,x} Gw(b,y,x) H(b,y,x) the
gradients with respect to the query features, the centroids and the filter weights follow
the chain rule step by step (functions below); as tau -> 0 the soft heatmap tends to the
hard one of Eq. 2 (pinned in the tests).
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np


def grid_cells(th: int, tw: int, G: int):
    """Cells (y0, y1, x0, x1) of the G x G grid over a th x tw window, row-major,
    boundaries floor(i * side / G)."""
    bx = [(i * tw) // G for i in range(G + 1)]
    by = [(i * th) // G for i in range(G + 1)]
    return [(by[r], by[r + 1], bx[c], bx[c + 1]) for r in range(G) for c in range(G)]


def soft_assign(X, C, tau: float):
    """p (..., k): softmax over centroids of -||x - c_j||^2 / tau, in FP64 (direct differences,
    the largest logit subtracted before exponentiation)."""
    X = np.asarray(X, np.float64)
    C = np.asarray(C, np.float64)
    shape = X.shape[:-1]
    X = X.reshape(-1, X.shape[-1])
    p = np.empty((X.shape[0], C.shape[0]))
    step = 2048                       # pixels per pass, to bound the (pixels, k, D) temporary

    def rows(i):
        d = ((X[i:i + step, None, :] - C) ** 2).sum(-1)
        z = -d / tau
        z -= z.max(-1, keepdims=True)
        e = np.exp(z)
        p[i:i + step] = e / e.sum(-1, keepdims=True)

    # independent pixel blocks (numpy releases the GIL inside each array operation)
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(rows, range(0, X.shape[0], step)))
    return p.reshape(shape + (C.shape[0],))


def _box_all(p, y0, y1, x0, x1, HO, WO):
    """Soft counts of the cell [y0, y1) x [x0, x1) for every window top-left (y, x):
    (B, HO, WO, k), from an FP64 integral image of p (B, H, W, k)."""
    B, H, W, k = p.shape
    S = np.zeros((B, H + 1, W + 1, k))
    S[:, 1:, 1:] = p.cumsum(1).cumsum(2)
    return (S[:, y1:y1 + HO, x1:x1 + WO] - S[:, y0:y0 + HO, x1:x1 + WO]
            - S[:, y1:y1 + HO, x0:x0 + WO] + S[:, y0:y0 + HO, x0:x0 + WO])


def soft_forward(Qf, Tf, C, tau: float, G: int, wf):
    """Qf (B, H, W, D), Tf (th, tw, D), C (k, D), wf (G*G,) -> dict with heat (B, HO, WO) and
    the intermediates: pq, pt, T (F, k), Qc (F, B, HO, WO, k), L1 (F, B, HO, WO), cells."""
    Qf = np.asarray(Qf, np.float64)
    Tf = np.asarray(Tf, np.float64)
    B, H, W, _ = Qf.shape
    th, tw = Tf.shape[:2]
    HO, WO = H - th + 1, W - tw + 1
    cells = grid_cells(th, tw, G)
    pq = soft_assign(Qf, C, tau)
    pt = soft_assign(Tf, C, tau)
    T = np.stack([pt[y0:y1, x0:x1].sum((0, 1)) for (y0, y1, x0, x1) in cells])
    Qc = np.stack([_box_all(pq, *c, HO, WO) for c in cells])
    L1 = np.abs(T[:, None, None, None, :] - Qc).sum(-1)
    area = np.array([(y1 - y0) * (x1 - x0) for (y0, y1, x0, x1) in cells], np.float64)
    heat = -(np.asarray(wf, np.float64)[:, None, None, None] / area[:, None, None, None] * L1).sum(0)
    return {"heat": heat, "pq": pq, "pt": pt, "T": T, "Qc": Qc, "L1": L1, "cells": cells,
            "area": area}


def _softmax_back(p, g, tau: float):
    """dL/dd_j for p = softmax(-d / tau) and g = dL/dp: -(1/tau) p_j (g_j - sum_i p_i g_i)."""
    return -(p * (g - (p * g).sum(-1, keepdims=True))) / tau


def soft_backward(Qf, Tf, C, tau: float, G: int, wf, Gw, forward=None):
    """Gradients of L = sum Gw * H: dQf (B, H, W, D), dC (k, D), dwf (F,).  ``forward``: the
    result of soft_forward for the same arguments, if already computed."""
    Qf = np.asarray(Qf, np.float64)
    Tf = np.asarray(Tf, np.float64)
    C = np.asarray(C, np.float64)
    wf = np.asarray(wf, np.float64)
    Gw = np.asarray(Gw, np.float64)
    f = soft_forward(Qf, Tf, C, tau, G, wf) if forward is None else forward
    B, H, W, _ = Qf.shape
    HO, WO = Gw.shape[1:]
    k = C.shape[0]
    # dL/dw_f = - sum G L1_f / A_f
    dwf = -(Gw[None] * f["L1"]).sum((1, 2, 3)) / f["area"]
    # dL/dQc_fj(y,x) = -(w_f / A_f) G(y,x) sign(Qc - T)
    M = -(wf / f["area"])[:, None, None, None, None] * Gw[None, ..., None] * np.sign(
        f["Qc"] - f["T"][:, None, None, None, :])
    dT = -M.sum((1, 2, 3))                                           # (F, k)
    # query pixels: every window's cell passes its gradient to the pixels it covers
    # (adjoint of the box sums, through a 2D difference array)
    Dq = np.zeros((B, H + 1, W + 1, k))
    for fi, (y0, y1, x0, x1) in enumerate(f["cells"]):
        Dq[:, y0:y0 + HO, x0:x0 + WO] += M[fi]
        Dq[:, y0:y0 + HO, x1:x1 + WO] -= M[fi]
        Dq[:, y1:y1 + HO, x0:x0 + WO] -= M[fi]
        Dq[:, y1:y1 + HO, x1:x1 + WO] += M[fi]
    gq = Dq.cumsum(1).cumsum(2)[:, :H, :W]
    gt = np.zeros(f["pt"].shape)
    for fi, (y0, y1, x0, x1) in enumerate(f["cells"]):
        gt[y0:y1, x0:x1] += dT[fi]
    aq = _softmax_back(f["pq"], gq, tau)                             # dL/dd (B, H, W, k)
    at = _softmax_back(f["pt"], gt, tau)
    # d = ||x - c||^2:  dd/dx = 2 (x - c),  dd/dc = -2 (x - c)
    dQf = 2.0 * aq.sum(-1, keepdims=True) * Qf - 2.0 * aq @ C
    dC = (-2.0 * np.einsum("bhwj,bhwi->ji", aq, Qf) + 2.0 * aq.sum((0, 1, 2))[:, None] * C
          - 2.0 * np.einsum("hwj,hwi->ji", at, Tf) + 2.0 * at.sum((0, 1))[:, None] * C)
    return dQf, dC, dwf
