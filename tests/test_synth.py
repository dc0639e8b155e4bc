"""The seeded input generator (`synth/`) follows the recipe its docstring states (CPU only):
piecewise-constant features over Voronoi-like superpixels drawn from a mixture, per-pixel
noise of the stated size, non-negative after the ReLU; warped templates inside the stated
rotation, scale and occluder ranges; crops that are crops; the grid bank's floor boundaries;
and every map a pure function of its seed."""
import pytest
import torch

import synth


def test_query_map_recipe():
    q = synth.query_map(96, 128, 16, M=8, n_sp=60, seed=5)
    X = q.X
    assert X.shape == (96, 128, 16) and X.dtype == torch.float32
    assert float(X.min()) >= 0.0                                   # ReLU
    assert 0.0 <= float(q.mu.min()) and float(q.mu.max()) <= 1.0   # means ~ U[0, 1]^D
    assert 0.6 * 60 <= len(torch.unique(q.sp_id)) <= 1.6 * 60      # about n_sp superpixels
    # one vector per superpixel: its component's mean plus N(0, 0.05^2)
    dev = (q.sp_vec - q.mu[q.sp_comp]).flatten()
    assert abs(float(dev.std()) - 0.05) < 0.01 and abs(float(dev.mean())) < 0.01
    # pixel = ReLU(v_s + N(0, 0.02^2)): where v_s is far above zero the residual is the noise
    v = q.sp_vec[q.sp_id]
    keep = v > 0.2
    r = (X - v)[keep]
    assert abs(float(r.std()) - 0.02) < 0.003 and abs(float(r.mean())) < 0.003
    # superpixels are spatially coherent regions, not scattered labels
    assert float((q.sp_id[:, 1:] == q.sp_id[:, :-1]).float().mean()) > 0.8
    assert float((q.sp_id[1:, :] == q.sp_id[:-1, :]).float().mean()) > 0.8


def test_maps_are_pure_functions_of_their_seeds():
    a = synth.query_map(40, 50, 8, M=4, n_sp=20, seed=3)
    b = synth.query_map(40, 50, 8, M=4, n_sp=20, seed=3)
    c = synth.query_map(40, 50, 8, M=4, n_sp=20, seed=4)
    assert torch.equal(a.X, b.X) and not torch.equal(a.X, c.X)
    Ta, ia = synth.warped_template(a, 16, 12, seed=9)
    Tb, ib = synth.warped_template(b, 16, 12, seed=9)
    assert torch.equal(Ta, Tb) and ia == ib


@pytest.mark.parametrize("seed", range(6))
def test_warped_template_ranges(seed):
    H, W, th, tw = 200, 220, 40, 48
    q = synth.query_map(H, W, 8, M=6, n_sp=80, seed=100 + seed)
    T, info = synth.warped_template(q, th, tw, seed=seed)
    assert T.shape == (th, tw, 8) and float(T.min()) >= 0.0
    assert -30.0 <= info["theta_deg"] <= 30.0 and 0.8 <= info["scale"] <= 1.25
    y, x = info["top_left"]
    assert 0 <= y <= H - th and 0 <= x <= W - tw                  # a valid window
    oy, ox, oh, ow = info["occluder"]
    assert 0 <= oy and oy + oh <= th and 0 <= ox and ox + ow <= tw
    assert abs(oh * ow - 0.25 * th * tw) <= 0.1 * th * tw          # about a quarter of the area
    # the occluder holds features of one component: its mean is that component's mean
    mu = q.mu[info["occluder_component"]]
    mean = T[oy:oy + oh, ox:ox + ow].reshape(-1, 8).mean(0)
    big = mu > 0.3                                                 # away from the ReLU's clip
    if bool(big.any()):
        assert float((mean - mu)[big].abs().max()) < 0.03


def test_crop_template_is_a_crop():
    q = synth.query_map(30, 40, 4, M=3, n_sp=12, seed=1)
    T, (y, x) = synth.crop_template(q, 10, 12, seed=2, sigma=0.0)
    assert torch.equal(T, q.X[y:y + 10, x:x + 12])
    Tn, (yn, xn) = synth.crop_template(q, 10, 12, seed=2)
    assert (yn, xn) == (y, x) and not torch.equal(Tn, T)           # same place, plus noise


def test_grid_bank_floor_boundaries():
    bank = synth.grid_bank(128, 128, 3)
    assert len(bank) == 10 and bank[0]["rects"] == [(0, 0, 128, 128, 1)]   # full window first
    cols = sorted({v for f in bank[1:] for (x0, _, x1, _, _) in f["rects"] for v in (x0, x1)})
    assert cols == [0, 42, 85, 128]                                # floor(i * 128 / 3)
    assert sum(f["area"] for f in bank[1:]) == 128 * 128           # the cells tile the window
    assert all(f["w_f"] == 1.0 for f in bank)
    assert all(f["area"] == (x1 - x0) * (y1 - y0) for f in bank for (x0, y0, x1, y1, _) in f["rects"])
    assert len(synth.grid_bank(30, 20, 2, full=False)) == 4
