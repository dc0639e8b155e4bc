"""The whole path with host buffers (vqnnf_match_host) equals the device-pointer path call for
call: the same codebook, labels, counts and therefore a bit-identical heatmap and the same
maximum, whether the inputs are pinned or pageable and whether a second stream overlaps the
compute with the copies."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vq():
    from paper_2306_15010_gb300 import build
    build.build()
    import paper_2306_15010_gb300 as m
    torch.cuda.set_device(0)
    return m


@pytest.fixture(scope="module")
def case(vq):
    q = synth.query_map(203, 190, 64, M=14, n_sp=120, seed=71)
    T, _ = synth.crop_template(q, 40, 36, seed=72)
    k, iters, seed = 24, 5, 73
    bank = synth.grid_bank(40, 36, 3)
    Xd, Td = q.X.cuda(), T.cuda()
    C = vq.vqnnf_fit_codebook(Td, k, iters, seed, "bf16")
    tl = vq.vqnnf_assign(Td, C, "bf16")
    ql = vq.vqnnf_assign(Xd, C, "bf16")
    tc = vq.vqnnf_filter_responses(tl, k, bank)
    heat, am = vq.vqnnf_score(ql, k, 40, 36, bank, tc)
    torch.cuda.synchronize()
    return q.X, T, k, iters, seed, bank, heat.cpu(), am.cpu()


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("two_streams", [True, False])
def test_match_host_equals_device_path(vq, case, pinned, two_streams):
    X, T, k, iters, seed, bank, heat_ref, am_ref = case
    if pinned:
        X, T = X.pin_memory(), T.pin_memory()
    s = torch.cuda.Stream()
    s2 = torch.cuda.Stream() if two_streams else None
    heat, am = vq.vqnnf_match_host(X, T, k, iters, seed, bank, "bf16", stream=s, stream2=s2)
    s.synchronize()
    assert torch.equal(heat, heat_ref)
    assert am.tolist() == am_ref.tolist()


def test_match_host_maximum_only_and_refusals(vq, case):
    X, T, k, iters, seed, bank, _, am_ref = case
    heat, am = vq.vqnnf_match_host(X, T, k, iters, seed, bank, "bf16", heatmap=False)
    torch.cuda.synchronize()
    assert heat is None and am.tolist() == am_ref.tolist()
    with pytest.raises(TypeError):
        vq.vqnnf_match_host(X.cuda(), T, k, iters, seed, bank)
    with pytest.raises(vq.VqnnfError):                      # k larger than the template
        vq.vqnnf_match_host(X, T, 40 * 36 + 1, iters, seed, bank)


def test_match_host_fewer_rows_than_bands(vq):
    """A query of 5 rows (fewer than the copy bands) and a template of its full height."""
    q = synth.query_map(5, 90, 16, M=4, n_sp=6, seed=81)
    T = q.X[:, 10:30].clone()
    bank = synth.grid_bank(5, 20, 1)
    C = vq.vqnnf_fit_codebook(T.cuda(), 6, 2, 82, "bf16")
    tc = vq.vqnnf_filter_responses(vq.vqnnf_assign(T.cuda(), C, "bf16"), 6, bank)
    heat_ref, am_ref = vq.vqnnf_score(vq.vqnnf_assign(q.X.cuda(), C, "bf16"), 6, 5, 20, bank, tc)
    heat, am = vq.vqnnf_match_host(q.X, T, 6, 2, 82, bank, "bf16", stream2=torch.cuda.Stream())
    torch.cuda.synchronize()
    assert torch.equal(heat, heat_ref.cpu()) and am.tolist() == am_ref.cpu().tolist()
    assert float(heat[0, 10]) == 0.0                                   # the template's own place
