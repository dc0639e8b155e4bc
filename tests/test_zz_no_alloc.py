"""The allocation-free assignment entry point (vqnnf_assign_noalloc).

It serves callers that cannot allocate device memory themselves -- a plug-in whose host
application owns every device allocation, or a loop that must never wait on the allocator --
by using the library's fixed scratch area instead of a caller workspace.  Its labels and
counters must equal those of vqnnf_assign on the same inputs, call after call, in both
contraction precisions (the area keeps the previous call's contents, which must not leak into
the next result); the BF16 tensor-core route, whose tensor maps point into that area, is also
checked against the FP64 oracle outside the near-tie band.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2306_15010_gb300 import build, _lib
    build.build()
    torch.cuda.set_device(0)
    return _lib.load()


def _case(H, W, D, k, seed):
    q = synth.query_map(H, W, D, M=k // 2 + 3, n_sp=max(8, H * W // 200), seed=seed)
    T, _ = synth.crop_template(q, max(8, H // 4), max(8, W // 4), seed=seed + 1)
    C = oracle.fit_codebook(T.numpy(), k, 3, seed)
    return q.X.cuda(), torch.as_tensor(C).cuda()


def _reference(lib, X, C, prec):
    H, W, D = X.shape
    k = C.shape[0]
    nb = lib.vqnnf_workspace_bytes(1, H, W, D, k, 0, 0, 0, prec)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    lab = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    st = torch.zeros(4, dtype=torch.int64, device="cuda")
    assert lib.vqnnf_assign(X.data_ptr(), H, W, D, C.data_ptr(), k, prec, lab.data_ptr(),
                            st.data_ptr(), ws.data_ptr(), nb, None) == 0
    torch.cuda.synchronize()
    return lab, st


def _noalloc(lib, X, C, prec):
    H, W, D = X.shape
    k = C.shape[0]
    lab = torch.full((H, W), 255, dtype=torch.uint8, device="cuda")
    st = torch.full((4,), -1, dtype=torch.int64, device="cuda")
    assert lib.vqnnf_assign_noalloc(X.data_ptr(), H, W, D, C.data_ptr(), k, prec,
                                    lab.data_ptr(), st.data_ptr(), None) == 0
    torch.cuda.synchronize()
    return lab, st


@pytest.mark.parametrize("prec", [0, 1, 2])  # FP32 SIMT / BF16 / FP8 tcgen05 contraction, re-scored
def test_noalloc_matches_assign_on_consecutive_calls(lib, prec):
    cases = [_case(200, 180, 64, 16, 11), _case(97, 131, 128, 32, 12)]
    for X, C in cases + cases[:1]:       # three calls in a row, the first input repeated
        want_lab, want_st = _reference(lib, X, C, prec)
        got_lab, got_st = _noalloc(lib, X, C, prec)
        assert torch.equal(got_lab, want_lab)
        assert torch.equal(got_st, want_st)
        # and against the FP64 oracle, outside its near-tie band
        ref, d1, d2 = oracle.assign(X.cpu().numpy(), C.cpu().numpy(), return_dist=True)
        band = oracle.relative_gap(d1, d2) < 1e-6
        got = got_lab.cpu().numpy().astype(np.int32)
        assert int(((got != ref) & ~band).sum()) == 0


def test_noalloc_binding_refuses_mis_sized_arguments(lib):
    """The binding checks every size the kernels would trust, before anything is enqueued."""
    import paper_2306_15010_gb300 as vq
    X, C = _case(40, 30, 64, 16, 13)
    lab = torch.empty((40, 30), dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):                                    # codebook width != D
        vq.vqnnf_assign_noalloc(X, C[:, :32].contiguous(), labels=lab)
    with pytest.raises(ValueError):                                    # labels too short
        vq.vqnnf_assign_noalloc(X, C, labels=lab[:20])
    with pytest.raises(ValueError):                                    # stats too short
        vq.vqnnf_assign_noalloc(X, C, labels=lab, stats=torch.zeros(2, dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):                                    # the same checks in vqnnf_assign
        vq.vqnnf_assign(X, C, labels=lab[:20])
    with pytest.raises(ValueError):
        vq.vqnnf_assign(X, C, stats=torch.zeros(3, dtype=torch.int64, device="cuda"))
    vq.vqnnf_assign_noalloc(X, C, labels=lab)                          # well-formed: accepted
    torch.cuda.synchronize()
    assert torch.equal(lab, vq.vqnnf_assign(X, C))


def test_noalloc_rejects_requests_beyond_its_scratch(lib):
    from paper_2306_15010_gb300 import _lib
    X = torch.zeros((1, 4, 64), device="cuda")
    C = torch.zeros((16, 64), device="cuda")
    lab = torch.empty((1, 4), dtype=torch.uint8, device="cuda")
    H, W = 1024, 1024          # needs far more than the fixed area; nothing is launched
    assert lib.vqnnf_workspace_bytes(1, H, W, 64, 16, 0, 0, 0, 0) > _lib.NOALLOC_SCRATCH_BYTES
    assert lib.vqnnf_assign_noalloc(X.data_ptr(), H, W, 64, C.data_ptr(), 16, 0, lab.data_ptr(),
                                    None, None) == _lib.ENOMEM
