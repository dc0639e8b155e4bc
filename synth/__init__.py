"""Seeded synthetic feature maps shaped like the VQ-NNF template-matching workloads.

This module only produces inputs. It holds none of the matching method's arithmetic
(no distances, no codebook, no counting), so that the independent CPU oracle and the
CUDA path can both be fed the same bytes from it without sharing any of the method.

The recipe stands in for the paper's feature maps (colour patches or ResNet-18 stages,
Sec. 4.2 "Feature Extraction"), which need datasets and trained weights that are not
available. It reproduces their structure: a feature map that is piecewise constant over
superpixel-like regions, drawn from a small set of mixture components, plus per-pixel
noise and a ReLU so that every feature is non-negative.

* ``M`` component means ``mu_m ~ U[0,1]^D``.
* About ``n_sp`` Voronoi superpixels; their seeds sit on a jittered grid and every pixel
  joins the nearest seed among the 3x3 grid cells around its own cell.
* Each superpixel draws a component ``m ~ U{0..M-1}`` and ONE vector
  ``v_s = mu_m + N(0, sigma_sp^2 I)`` (sigma_sp = 0.05).
* Pixel feature ``= ReLU(v_s + N(0, sigma_px^2 I))`` (sigma_px = 0.02).

Templates are either a plain crop plus noise, or a rotated / scaled bilinear resample of
the query with a rectangular occluder of random features (see :func:`warped_template`).

All randomness comes from ``torch.Generator`` objects seeded explicitly, so a map is a
pure function of (seed, shape, device type).  CPU and CUDA generators produce different
streams; a parity check therefore always generates once and hands the same tensor to both
sides.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

__all__ = [
    "QueryMap",
    "query_map",
    "crop_template",
    "warped_template",
    "grid_bank",
]


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed))
    return g


@dataclass
class QueryMap:
    """A synthetic query feature map and the latent structure it was drawn from."""

    X: torch.Tensor          # (H, W, D) float32, HWC row-major
    mu: torch.Tensor         # (M, D) component means
    sp_vec: torch.Tensor     # (S, D) per-superpixel vector v_s (before pixel noise)
    sp_comp: torch.Tensor    # (S,) component index of every superpixel
    sp_id: torch.Tensor      # (H, W) superpixel index of every pixel


def _superpixel_ids(H: int, W: int, n_sp: int, g: torch.Generator, device) -> torch.Tensor:
    """Voronoi superpixels from jittered-grid seeds (nearest seed among 3x3 cells)."""
    cell = math.sqrt(H * W / max(1, n_sp))
    gy = max(1, math.ceil(H / cell))
    gx = max(1, math.ceil(W / cell))
    jit = torch.rand((gy, gx, 2), generator=g, device=device, dtype=torch.float32)
    cy = (torch.arange(gy, device=device, dtype=torch.float32)[:, None] + jit[..., 0]) * cell
    cx = (torch.arange(gx, device=device, dtype=torch.float32)[None, :] + jit[..., 1]) * cell
    out = torch.empty((H, W), dtype=torch.int64, device=device)
    xs = torch.arange(W, device=device, dtype=torch.float32) + 0.5
    rows_per_chunk = max(1, (1 << 22) // max(1, W))
    for y0 in range(0, H, rows_per_chunk):
        y1 = min(H, y0 + rows_per_chunk)
        ys = torch.arange(y0, y1, device=device, dtype=torch.float32) + 0.5
        py = ys[:, None].expand(-1, W)
        px = xs[None, :].expand(y1 - y0, -1)
        icy = torch.clamp((py / cell).long(), 0, gy - 1)
        icx = torch.clamp((px / cell).long(), 0, gx - 1)
        best_d = torch.full(py.shape, float("inf"), device=device)
        best_i = torch.zeros(py.shape, dtype=torch.int64, device=device)
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                ny = icy + dy
                nx = icx + dx
                ok = (ny >= 0) & (ny < gy) & (nx >= 0) & (nx < gx)
                nyc = ny.clamp(0, gy - 1)
                nxc = nx.clamp(0, gx - 1)
                d = (cy[nyc, nxc] - py) ** 2 + (cx[nyc, nxc] - px) ** 2
                d = torch.where(ok, d, torch.full_like(d, float("inf")))
                better = d < best_d
                best_d = torch.where(better, d, best_d)
                best_i = torch.where(better, nyc * gx + nxc, best_i)
        out[y0:y1] = best_i
    return out


def query_map(H: int, W: int, D: int, *, M: int, n_sp: int, seed: int,
              device="cpu", sigma_sp: float = 0.05, sigma_px: float = 0.02) -> QueryMap:
    """Query feature map (H, W, D) float32 following the recipe in the module docstring."""
    g = _gen(seed, device)
    mu = torch.rand((M, D), generator=g, device=device, dtype=torch.float32)
    sp_id = _superpixel_ids(H, W, n_sp, g, device)
    S = int(sp_id.max().item()) + 1
    sp_comp = torch.randint(0, M, (S,), generator=g, device=device)
    sp_vec = mu[sp_comp] + sigma_sp * torch.randn((S, D), generator=g, device=device)
    X = torch.empty((H, W, D), dtype=torch.float32, device=device)
    rows_per_chunk = max(1, (1 << 26) // max(1, W * D))
    for y0 in range(0, H, rows_per_chunk):
        y1 = min(H, y0 + rows_per_chunk)
        blk = sp_vec[sp_id[y0:y1]]
        blk.add_(torch.randn(blk.shape, generator=g, device=device), alpha=sigma_px)
        X[y0:y1] = torch.relu_(blk)
    return QueryMap(X=X, mu=mu, sp_vec=sp_vec, sp_comp=sp_comp, sp_id=sp_id)


def crop_template(q: QueryMap, th: int, tw: int, *, seed: int, sigma: float = 0.02,
                  relu: bool = False):
    """A th x tw crop of the query at a seeded location, plus N(0, sigma^2) noise.

    ``sigma = 0`` gives a template cut unaltered from the query.
    Returns (template (th, tw, D) float32, (y, x) top-left of the crop).
    """
    H, W, D = q.X.shape
    dev = q.X.device
    g = _gen(seed, dev)
    y = int(torch.randint(0, H - th + 1, (1,), generator=g, device=dev).item())
    x = int(torch.randint(0, W - tw + 1, (1,), generator=g, device=dev).item())
    T = q.X[y:y + th, x:x + tw].clone()
    if sigma > 0:
        T.add_(torch.randn(T.shape, generator=g, device=dev), alpha=sigma)
    if relu:
        T.relu_()
    return T.contiguous(), (y, x)


def warped_template(q: QueryMap, th: int, tw: int, *, seed: int,
                    rot_deg: float = 30.0, scale_lo: float = 0.8, scale_hi: float = 1.25,
                    occl_frac: float = 0.25, sigma: float = 0.05, sigma_sp: float = 0.05):
    """A th x tw template resampled bilinearly from the query around a seeded centre.

    Rotation theta ~ U[-rot_deg, rot_deg] degrees and scale s ~ U[scale_lo, scale_hi];
    then a seeded rectangle covering ``occl_frac`` of the area is replaced by i.i.d.
    features of one random component (mu_m' + N(0, sigma_sp^2), ReLU); then N(0, sigma^2)
    noise is added to the whole template and a ReLU keeps features non-negative.

    Returns (template (th, tw, D) float32, info dict with the planted top-left (y, x),
    theta, scale and the occluder rectangle).
    """
    H, W, D = q.X.shape
    dev = q.X.device
    g = _gen(seed, dev)
    u = torch.rand((6,), generator=g, device=dev, dtype=torch.float64).cpu().tolist()
    theta = math.radians((2.0 * u[0] - 1.0) * rot_deg)
    s = scale_lo + (scale_hi - scale_lo) * u[1]
    half = 0.5 * math.hypot(th, tw) * scale_hi + 2.0
    cy = half + (H - 2 * half) * u[2]
    cx = half + (W - 2 * half) * u[3]
    # template pixel (i, j) centre relative to the template centre, rotated and scaled
    ii = torch.arange(th, device=dev, dtype=torch.float32) - (th - 1) / 2.0
    jj = torch.arange(tw, device=dev, dtype=torch.float32) - (tw - 1) / 2.0
    di = ii[:, None].expand(th, tw)
    dj = jj[None, :].expand(th, tw)
    c, sn = math.cos(theta), math.sin(theta)
    sy = cy - 0.5 + s * (c * di - sn * dj)
    sx = cx - 0.5 + s * (sn * di + c * dj)
    y0 = torch.floor(sy).long().clamp(0, H - 2)
    x0 = torch.floor(sx).long().clamp(0, W - 2)
    fy = (sy - y0.float()).clamp(0, 1)[..., None]
    fx = (sx - x0.float()).clamp(0, 1)[..., None]
    X = q.X
    T = ((1 - fy) * (1 - fx) * X[y0, x0] + (1 - fy) * fx * X[y0, x0 + 1]
         + fy * (1 - fx) * X[y0 + 1, x0] + fy * fx * X[y0 + 1, x0 + 1])
    # occluder: a rectangle of area occl_frac * th * tw at a seeded place
    area = occl_frac * th * tw
    ow_lo = max(1, int(math.ceil(area / th)))
    ow_hi = min(tw, int(area))
    ow = int(round(ow_lo + (ow_hi - ow_lo) * u[4])) if ow_hi >= ow_lo else tw
    oh = min(th, max(1, int(round(area / ow))))
    oy = int(torch.randint(0, th - oh + 1, (1,), generator=g, device=dev).item())
    ox = int(torch.randint(0, tw - ow + 1, (1,), generator=g, device=dev).item())
    m = int(torch.randint(0, q.mu.shape[0], (1,), generator=g, device=dev).item())
    occ = q.mu[m] + sigma_sp * torch.randn((oh, ow, D), generator=g, device=dev)
    T[oy:oy + oh, ox:ox + ow] = torch.relu(occ)
    T.add_(torch.randn(T.shape, generator=g, device=dev), alpha=sigma)
    T.relu_()
    info = {
        "top_left": (int(round(cy - th / 2.0)), int(round(cx - tw / 2.0))),
        "theta_deg": math.degrees(theta), "scale": s,
        "occluder": (oy, ox, oh, ow), "occluder_component": m,
    }
    return T.contiguous(), info


def grid_bank(th: int, tw: int, g: int, *, full: bool = True):
    """Filter bank of single rectangles: the full window plus a g x g grid of sub-windows.

    Sub-window boundaries are floor(i * side / g). Every filter has weight w_f = 1 and is
    normalised by its own area. Returned as a list of filters, each a dict with a list of
    half-open window-relative rectangles (x0, y0, x1, y1, weight), w_f and area.
    """
    bank = []
    if full:
        bank.append({"rects": [(0, 0, tw, th, 1)], "w_f": 1.0, "area": float(th * tw)})
    bx = [(i * tw) // g for i in range(g + 1)]
    by = [(i * th) // g for i in range(g + 1)]
    for r in range(g):
        for c in range(g):
            x0, x1, y0, y1 = bx[c], bx[c + 1], by[r], by[r + 1]
            bank.append({"rects": [(x0, y0, x1, y1, 1)], "w_f": 1.0,
                         "area": float((x1 - x0) * (y1 - y0))})
    return bank


def paper_bank(th: int, tw: int, filters: str = "2,3-rect", S: int = 3, gauss: str = "equal",
               quant: int = 4096):
    """The coarse filter bank of the paper's experiments (Sec. 3.2.2, Sec. 4.2 "Filtering",
    Supp. "Modulating Filter Response Granularity" c): 3 x 3 coarse filters at sub-scales
    s = 1..S, each a weighted sum of its 9 bin boxes, as integer-weighted rectangles.

    Scale s covers the central (tw // s) x (th // s) region of the window, cut into 3 x 3 bins
    with floor boundaries.  Filter sets: "gauss" = {Gaussian}, "2-rect" = {Gaussian, Haar-2x,
    Haar-2y}, "3-rect" = {Gaussian, Haar-3x, Haar-3y}, "2,3-rect" = all five.  Haar kernels on
    the 3 x 3 bin grid (a reading; the paper prints no layout): 2x = columns (+1, 0, -1),
    3x = columns (+1, -2, +1), 2y / 3y the same over rows, each multiplied by the Gaussian.
    Weights w_{s,f} = w_f / s with w_f = 1 (Gaussian) and 0.25 (Haar); the normalising area is
    the scale's region (Eq. 1: the receptive field).

    gauss = "equal": the paper's stated intent for its sigma = 2 kernel ("equal weights to all
    the bins"), so every bin weight is the Haar sign pattern; gauss = "exp": the kernel
    exp(-(i^2 + j^2) / (2 sigma^2)), sigma = 2, at bin offsets i, j in {-1, 0, 1}, with the bin
    weights rounded to integers at scale `quant` (the filter's w_f is divided by `quant`).
    """
    import math
    sets = {"gauss": ["gauss"], "2-rect": ["gauss", "haar2x", "haar2y"],
            "3-rect": ["gauss", "haar3x", "haar3y"],
            "2,3-rect": ["gauss", "haar2x", "haar2y", "haar3x", "haar3y"]}
    names = sets[filters]
    pat = {"gauss": lambda i, j: 1, "haar2x": lambda i, j: -j, "haar2y": lambda i, j: -i,
           "haar3x": lambda i, j: 1 if j else -2, "haar3y": lambda i, j: 1 if i else -2}
    bank = []
    for s in range(1, S + 1):
        ws, hs = tw // s, th // s
        xo, yo = (tw - ws) // 2, (th - hs) // 2
        bx = [xo + (q * ws) // 3 for q in range(4)]
        by = [yo + (q * hs) // 3 for q in range(4)]
        for name in names:
            wgt = {}
            for i in (-1, 0, 1):
                for j in (-1, 0, 1):
                    h = pat[name](i, j)
                    if gauss == "exp":
                        wgt[(i, j)] = int(round(quant * h * math.exp(-(i * i + j * j) / 8.0)))
                    else:
                        wgt[(i, j)] = h
            rects = []
            cols_equal = all(wgt[(-1, j)] == wgt[(0, j)] == wgt[(1, j)] for j in (-1, 0, 1))
            rows_equal = all(wgt[(i, -1)] == wgt[(i, 0)] == wgt[(i, 1)] for i in (-1, 0, 1))
            if cols_equal and rows_equal:
                rects.append((bx[0], by[0], bx[3], by[3], wgt[(0, 0)]))
            elif cols_equal:
                for j in (-1, 0, 1):
                    if wgt[(0, j)]:
                        rects.append((bx[j + 1], by[0], bx[j + 2], by[3], wgt[(0, j)]))
            elif rows_equal:
                for i in (-1, 0, 1):
                    if wgt[(i, 0)]:
                        rects.append((bx[0], by[i + 1], bx[3], by[i + 2], wgt[(i, 0)]))
            else:
                for i in (-1, 0, 1):
                    for j in (-1, 0, 1):
                        if wgt[(i, j)]:
                            rects.append((bx[j + 1], by[i + 1], bx[j + 2], by[i + 2], wgt[(i, j)]))
            w_f = (1.0 if name == "gauss" else 0.25) / s
            if gauss == "exp":
                w_f /= quant
            bank.append({"rects": rects, "w_f": w_f, "area": float(ws * hs)})
    return bank

