"""Failure detection on the GPU without a fault.

A bounded device wait that nothing completes (the self-test kernel: an mbarrier with no
arrivals and no copy in flight) gives up after its cycle limit.  The host then reads
VQNNF_ETIMEOUT through vqnnf_last_device_error, which also clears the word.  The context
stays usable: an assignment and a score on the same stream afterwards are correct and leave
the word clear.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vq():
    from paper_2306_15010_gb300 import build
    build.build()
    import paper_2306_15010_gb300 as m
    torch.cuda.set_device(0)
    return m


def test_bounded_wait_gives_up_and_reports(vq):
    from paper_2306_15010_gb300 import _lib
    s = torch.cuda.Stream()
    assert vq.vqnnf_last_device_error(s) == _lib.OK         # nothing left over
    limit = 2_000_000                                       # about 1 ms at 2 GHz
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    vq.vqnnf_selftest_bounded_wait(limit, stream=s)
    e1.record(s)
    assert vq.vqnnf_last_device_error(s) == _lib.ETIMEOUT
    # the SM clock never exceeds 2.07 GHz, so giving up took at least limit / 2.07e9 s
    assert e0.elapsed_time(e1) >= 0.9 * limit / 2.07e6
    assert vq.vqnnf_last_device_error(s) == _lib.OK         # read and cleared

    # the context is still usable: an assignment and a score on the same stream
    q = synth.query_map(40, 52, 64, M=8, n_sp=24, seed=31)
    T, _ = synth.crop_template(q, 16, 20, seed=32)
    C = oracle.fit_codebook(T.numpy(), 8, 2, 33)
    with torch.cuda.stream(s):
        Cd = torch.from_numpy(C).cuda()
        lab = vq.vqnnf_assign(q.X.cuda(), Cd, "bf16", stream=s)
        tl = vq.vqnnf_assign(T.cuda(), Cd, "bf16", stream=s)
        bank = synth.grid_bank(16, 20, 3)
        tc = vq.vqnnf_filter_responses(tl, 8, bank, stream=s)
        heat, _ = vq.vqnnf_score(lab, 8, 16, 20, bank, tc, stream=s)
    assert vq.vqnnf_last_device_error(s) == _lib.OK
    ref, d1, d2 = oracle.assign(q.X.numpy(), C, return_dist=True)
    band = oracle.relative_gap(d1, d2) < 1e-6
    got = lab.cpu().numpy().astype(np.int32)
    assert not ((got != ref) & ~band).any()
    # the heatmap from the GPU's own labels (the label parity above is the oracle's check)
    tl_np = tl.cpu().numpy().astype(np.int32)
    href, _ = oracle.score(got, 8, 16, 20, bank, oracle.filter_counts(tl_np, 8, bank))
    scale = max(np.abs(href).max(), 1e-30)
    assert np.abs(heat.cpu().numpy() - href).max() <= 1e-5 * scale
