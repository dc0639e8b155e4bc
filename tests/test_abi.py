"""The C ABI library: it loads, exports every entry point the header declares, and checks
its arguments on the host (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vqnnf.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2306_15010_gb300 import build, _lib
    build.build()
    return _lib.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vqnnf_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["vqnnf_fit_codebook", "vqnnf_assign", "vqnnf_filter_responses", "vqnnf_score",
                 "vqnnf_workspace_bytes", "vqnnf_status_str", "vqnnf_last_device_error"]:
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2306_15010_gb300 import _lib
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"


def test_version_and_status_strings(lib):
    assert lib.vqnnf_version() == 100
    assert lib.vqnnf_status_str(0) == b"ok"
    assert lib.vqnnf_status_str(2) == b"workspace too small"
    assert lib.vqnnf_status_str(99) == b"unknown status"


def test_workspace_sizes(lib):
    from paper_2306_15010_gb300 import _lib
    a = lib.vqnnf_workspace_bytes(_lib.OP_ASSIGN, 2048, 2048, 512, 128, 0, 0, 0, 1)
    assert a % 256 == 0 and a > 2048 * 2048 * 36
    assert lib.vqnnf_workspace_bytes(_lib.OP_ASSIGN, 2048, 2048, 512, 257, 0, 0, 0, 1) == 0
    # 16-bit integral image while the template area is below 65,536 pixels, 32-bit beyond
    s = lib.vqnnf_workspace_bytes(_lib.OP_SCORE, 256, 256, 0, 16, 32, 32, 5, 0)
    assert s >= 257 * 16 * 264 * 2
    big = lib.vqnnf_workspace_bytes(_lib.OP_SCORE, 600, 600, 0, 16, 300, 300, 5, 0)
    assert big >= 601 * 16 * 608 * 4
    assert lib.vqnnf_workspace_bytes(_lib.OP_SCORE, 256, 256, 0, 16, 300, 32, 5, 0) == 0
    assert lib.vqnnf_workspace_bytes(99, 1, 1, 1, 1, 1, 1, 1, 0) == 0
    f = lib.vqnnf_workspace_bytes(_lib.OP_FIT, 128, 128, 512, 128, 0, 0, 0, 0)
    assert f > lib.vqnnf_workspace_bytes(_lib.OP_ASSIGN, 128, 128, 512, 128, 0, 0, 0, 0)


FAKE = 1 << 20          # a non-null, 256-aligned pointer value never dereferenced


def test_assign_argument_errors(lib):
    from paper_2306_15010_gb300 import _lib
    ws = lib.vqnnf_workspace_bytes(_lib.OP_ASSIGN, 4, 4, 16, 3, 0, 0, 0, 0)
    call = lambda **kw: lib.vqnnf_assign(*[kw.get(n, d) for n, d in [
        ("X", FAKE), ("H", 4), ("W", 4), ("D", 16), ("C", FAKE), ("k", 3), ("prec", 0),
        ("labels", FAKE), ("stats", None), ("ws", FAKE), ("ws_bytes", ws), ("stream", None)]])
    assert call(X=None) == _lib.EINVAL
    assert call(labels=None) == _lib.EINVAL
    assert call(H=0) == _lib.EINVAL
    assert call(k=0) == _lib.EINVAL
    assert call(k=300) == _lib.EUNSUPPORTED
    assert call(X=FAKE + 4) == _lib.EINVAL           # misaligned features
    assert call(prec=7) == _lib.EINVAL
    assert call(D=18, prec=0) == _lib.EUNSUPPORTED    # FP32 path wants D % 4 == 0
    assert call(D=20, prec=1) == _lib.EUNSUPPORTED    # tensor path wants D % 16 == 0
    assert call(ws_bytes=ws - 1) == _lib.ENOMEM


def test_fit_argument_errors(lib):
    from paper_2306_15010_gb300 import _lib
    ws = lib.vqnnf_workspace_bytes(_lib.OP_FIT, 4, 4, 8, 3, 0, 0, 0, 0)
    def call(**kw):
        a = dict(T=FAKE, h=4, w=4, D=8, k=3, iters=2, seed=ctypes.c_uint64(1), prec=0, C=FAKE,
                 ws=FAKE, ws_bytes=ws, stream=None)
        a.update(kw)
        return lib.vqnnf_fit_codebook(*a.values())
    assert call(k=17) == _lib.EINVAL                  # more clusters than pixels
    assert call(iters=-1) == _lib.EINVAL
    assert call(C=None) == _lib.EINVAL
    assert call(ws_bytes=16) == _lib.ENOMEM


def _bank(rects, w_f=1.0, area=None):
    from paper_2306_15010_gb300 import Bank
    area = area if area is not None else float(sum((r[2] - r[0]) * (r[3] - r[1]) for r in rects))
    return Bank([{"rects": rects, "w_f": w_f, "area": area}])


def test_score_rejects_bad_banks_and_shapes(lib):
    from paper_2306_15010_gb300 import _lib
    ws = lib.vqnnf_workspace_bytes(_lib.OP_SCORE, 16, 16, 0, 4, 4, 4, 1, 0)
    def call(bank, **kw):
        a = dict(q=FAKE, H=16, W=16, k=4, th=4, tw=4, bank=bank.ptr, F=bank.F, tc=FAKE,
                 heat=FAKE, am=None, ws=FAKE, ws_bytes=ws, stream=None)
        a.update(kw)
        return lib.vqnnf_score(*a.values())
    good = _bank([(0, 0, 4, 4, 1)])
    assert call(good, th=17) == _lib.EINVAL           # template taller than the query
    assert call(good, F=0) == _lib.EINVAL
    assert call(good, ws_bytes=100) == _lib.ENOMEM
    assert call(_bank([(0, 0, 5, 4, 1)])) == _lib.EINVAL    # rectangle outside the window
    assert call(_bank([(2, 0, 2, 4, 1)])) == _lib.EINVAL    # empty rectangle
    assert call(_bank([(0, 0, 4, 4, 1)], area=0.0)) == _lib.EINVAL
    assert call(_bank([(0, 0, 4, 4, 1)], w_f=float("nan"))) == _lib.EINVAL


def test_filter_responses_rejects_bad_banks(lib):
    from paper_2306_15010_gb300 import _lib
    b = _bank([(0, 0, 9, 4, 1)])
    assert lib.vqnnf_filter_responses(FAKE, 4, 8, 4, b.ptr, 1, FAKE, None, 0, None) == _lib.EINVAL
    assert lib.vqnnf_filter_responses(None, 4, 8, 4, b.ptr, 1, FAKE, None, 0, None) == _lib.EINVAL


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2306_15010_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        _lib.load()


def _batch_arrays(qshapes, tshapes):
    from paper_2306_15010_gb300 import _lib
    qa = (_lib.VqnnfImage * len(qshapes))(*[_lib.VqnnfImage(FAKE, H, W) for H, W in qshapes])
    ta = (_lib.VqnnfBatchTemplate * len(tshapes))(*[_lib.VqnnfBatchTemplate(FAKE, h, w, k) for h, w, k in tshapes])
    return qa, ta


def test_batch_workspace_and_refusals(lib):
    """Batched matching: workspace sizes and the host-side checks (no kernel is launched)."""
    from paper_2306_15010_gb300 import _lib
    qa, ta = _batch_arrays([(512, 700), (300, 256)], [(16, 20, 8), (64, 64, 256), (40, 33, 100)])
    nb = lib.vqnnf_batch_workspace_bytes(qa, 2, ta, 3, 256, 3)
    # at least: the NNF of the largest query under every codebook, flag lists of eight codebooks,
    # one 16-bit integral image of the largest pair
    assert nb % 256 == 0 and nb > 3 * 512 * 700 + 8 * 512 * 700 * 36 + 513 * 256 * 700 * 2
    for q, t, D, G in [([(512, 700)], [(16, 20, 8), (600, 20, 8)], 256, 3),    # template taller than a query
                       ([(512, 700)], [(16, 20, 321)], 256, 3),                 # k > h w
                       ([(512, 700)], [(16, 20, 8)], 250, 3),                   # D % 16
                       ([(512, 700)], [(16, 20, 8)], 256, 5),                   # G > 4
                       ([(512, 700)], [(3, 20, 8)], 256, 4),                    # cells thinner than G
                       ([(512, 700)], [(64, 64, 257)], 256, 3)]:               # k > 256
        qa, ta = _batch_arrays(q, t)
        assert lib.vqnnf_batch_workspace_bytes(qa, len(q), ta, len(t), D, G) == 0
    qa, ta = _batch_arrays([(512, 700)], [(16, 20, 8)])
    plan = _lib.VqnnfBatchPlan(256, 0, -1, 0)
    call = lambda **kw: lib.vqnnf_match_batch(
        qa, 1, ta, 1, 256, 3, ctypes.c_uint64(1), kw.get("G", 3), ctypes.byref(kw.get("plan", plan)), None,
        kw.get("am", FAKE), kw.get("ws", FAKE), kw.get("wsb", 1 << 40), None)
    assert call(am=None) == _lib.EINVAL
    assert call(ws=None) == _lib.EINVAL
    assert call(wsb=1024) == _lib.ENOMEM
    assert call(G=0) == _lib.EUNSUPPORTED
    assert call(plan=_lib.VqnnfBatchPlan(64, 0, -1, 0)) == _lib.EINVAL
    assert call(plan=_lib.VqnnfBatchPlan(256, 3, -1, 0)) == _lib.EINVAL
    assert lib.vqnnf_batch_tune(qa, 1, ta, 1, 256, 3, ctypes.c_uint64(1), 3, None, FAKE, 1 << 40, None) == _lib.EINVAL


def test_match_host_workspace_and_refusals(lib):
    """Whole path with host buffers: workspace size and host-side argument checks only."""
    from paper_2306_15010_gb300 import _lib
    nb = lib.vqnnf_match_host_workspace_bytes(2048, 2048, 512, 128, 128, 128, 10, 1)
    # at least the device copy of the query's features and the 16-bit integral image
    assert nb % 256 == 0 and nb > 2048 * 2048 * 512 * 4 + 2049 * 128 * 2056 * 2
    for args in [(64, 64, 16, 8, 65, 8, 5, 1),       # template taller than the query
                 (64, 64, 16, 257, 32, 32, 5, 1),    # k > 256
                 (64, 64, 16, 100, 8, 8, 5, 1),      # k > template pixels
                 (64, 64, 10, 8, 8, 8, 5, 1),        # D % 16 on the tensor path
                 (64, 64, 16, 8, 8, 8, 0, 1)]:       # empty bank
        assert lib.vqnnf_match_host_workspace_bytes(*args) == 0
    rect = _lib.VqnnfRect(0, 0, 8, 8, 1)
    filt = (_lib.VqnnfFilter * 1)(_lib.VqnnfFilter(1, ctypes.pointer(rect), 1.0, 64.0))
    am = (ctypes.c_int32 * 2)()
    call = lambda **kw: lib.vqnnf_match_host(
        kw.get("X", FAKE), 64, 64, 16, kw.get("T", FAKE), 8, 8, 8, 3, ctypes.c_uint64(1), 1, filt, 1, None,
        kw.get("am", ctypes.addressof(am)), kw.get("ws", FAKE), kw.get("wsb", 1 << 40), None, None)
    assert call(X=None) == _lib.EINVAL
    assert call(T=None) == _lib.EINVAL
    assert call(am=None) == _lib.EINVAL
    assert call(ws=None) == _lib.EINVAL
    assert call(wsb=256) == _lib.ENOMEM


def test_soft_workspace_and_refusals(lib):
    """Soft-VQ heatmap: workspace sizes and the host-side checks of both calls (nothing is
    launched: every case below is refused before the stream is touched)."""
    from paper_2306_15010_gb300 import _lib
    nb = lib.vqnnf_soft_workspace_bytes(8, 512, 512, 256, 64, 64, 64, 3)
    # at least the per-filter L1 maps of the backward pass: B x HO x WO x F float32
    assert nb % 256 == 0 and nb >= 8 * 449 * 449 * 9 * 4
    for args in [(0, 64, 64, 16, 8, 8, 8, 3),      # no query
                 (1, 64, 64, 16, 8, 65, 8, 3),     # template taller than the query
                 (1, 64, 64, 16, 0, 8, 8, 3),      # k = 0
                 (1, 64, 64, 16, 8, 8, 8, 0),      # G = 0
                 (1, 64, 64, 16, 8, 2, 8, 3)]:     # cells thinner than G
        assert lib.vqnnf_soft_workspace_bytes(*args) == 0
    fwd = lambda **kw: lib.vqnnf_soft_forward(
        kw.get("Q", FAKE), kw.get("B", 2), 64, 64, kw.get("T", FAKE), 16, 16, kw.get("D", 32), FAKE,
        kw.get("k", 16), ctypes.c_float(kw.get("tau", 0.1)), kw.get("G", 3), kw.get("wf", FAKE),
        kw.get("heat", FAKE), kw.get("ws", FAKE), kw.get("wsb", 1 << 40), None)
    assert fwd(Q=None) == _lib.EINVAL
    assert fwd(T=None) == _lib.EINVAL
    assert fwd(wf=None) == _lib.EINVAL
    assert fwd(heat=None) == _lib.EINVAL
    assert fwd(ws=FAKE + 16) == _lib.EINVAL           # misaligned workspace
    assert fwd(tau=0.0) == _lib.EINVAL
    assert fwd(tau=float("nan")) == _lib.EINVAL
    assert fwd(tau=float("inf")) == _lib.EINVAL
    assert fwd(wsb=256) == _lib.ENOMEM
    assert fwd(k=129) == _lib.EUNSUPPORTED            # k > 128
    assert fwd(D=513) == _lib.EUNSUPPORTED            # D > 512
    assert fwd(k=128, D=512) == _lib.EUNSUPPORTED     # k D > 32768
    assert fwd(G=5) == _lib.EUNSUPPORTED              # G > 4
    bwd = lambda **kw: lib.vqnnf_soft_backward(
        FAKE, 2, 64, 64, FAKE, 16, 16, 32, FAKE, 16, ctypes.c_float(kw.get("tau", 0.1)), 3, FAKE,
        kw.get("dheat", FAKE), kw.get("dQ", FAKE), kw.get("dC", FAKE), kw.get("dwf", FAKE), FAKE,
        kw.get("wsb", 1 << 40), None)
    assert bwd(dheat=None) == _lib.EINVAL
    assert bwd(dQ=None) == _lib.EINVAL
    assert bwd(dC=None) == _lib.EINVAL
    assert bwd(dwf=None) == _lib.EINVAL
    assert bwd(tau=-1.0) == _lib.EINVAL
    assert bwd(wsb=256) == _lib.ENOMEM


def test_selftest_wait_limit_refusals(lib):
    """The bounded-wait self-test refuses limits outside 1 .. the kernels' own limit on the
    host (nothing is enqueued)."""
    from paper_2306_15010_gb300 import _lib
    for bad in (0, -5, 4_000_000_001):
        assert lib.vqnnf_selftest_bounded_wait(bad, None) == _lib.EINVAL
