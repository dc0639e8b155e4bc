"""VQ-NNF oracle: plain FP64 CPU implementation of the template-matching hot path.

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this package; the product path never does, and this
package imports nothing from it.

Every function follows a passage of Gupta & Sintorn, "Efficient High-Resolution Template
Matching with Vector Quantized Nearest Neighbour Fields":

* :func:`kmeans_init`, :func:`fit_codebook` -- the k-means codebook of Sec. 3.1 (the paper
  names only a library, Sec. 4.2; the seeded init and fixed Lloyd count are this
  project's reading).
* :func:`assign` -- the nearest-neighbour field of Algorithm 1 with the exact L2 nearest
  neighbour of Sec. 4.2.
* :func:`filter_counts`, :func:`window_counts` -- filter responses (Eq. 1 counts, Sec. 3.2)
  by direct counting of labels inside each rectangle.
* :func:`score`, :func:`score_at` -- the similarity heatmap of Eq. 2 (L1 norm) and its
  maximum (Sec. 4 "Target Localization").
* :func:`coarse_to_dilation`, :func:`coarse_direct` -- Algorithm 2 (dilation filter on the
  integral image) and the direct bin-weighted count it must reproduce.

Every function above is pinned in ``tests/test_oracle_pins.py`` against exact brute force,
closed forms and invariants.  One input is not: the layouts of the Haar coarse filters in the
paper's bank (Sec. 4.2 "Filtering", supplementary c) are a reading, because the paper prints
neither their signs nor their values.  For those banks the direct counts here are pinned, but
parity of the bank itself is unpinned against the paper.

The C source is compiled on first use (``gcc -O2 -fopenmp``) into ``oracle/liboracle.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vqnnf_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent).  Returns its path."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_splitmix64_next.argtypes = [_u64p]
            lib.oracle_splitmix64_next.restype = ctypes.c_uint64
            lib.oracle_kmeans_init.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, _i64p]
            lib.oracle_kmeans_init.restype = ctypes.c_int
            lib.oracle_assign.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int, _f32p, ctypes.c_int,
                                          _i32p, _f64p, _f64p]
            lib.oracle_assign.restype = None
            lib.oracle_fit_codebook.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_uint64, _f32p]
            lib.oracle_fit_codebook.restype = ctypes.c_int
            lib.oracle_kmeans_objective.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int, _f32p,
                                                    ctypes.c_int]
            lib.oracle_kmeans_objective.restype = ctypes.c_double
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_set_threads.restype = ctypes.c_int
            lib.oracle_filter_counts.argtypes = [_i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, _i32p, _i32p, _i64p]
            lib.oracle_filter_counts.restype = None
            lib.oracle_window_counts.argtypes = [_i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_int, ctypes.c_int, _i32p,
                                                 _i32p, _i64p]
            lib.oracle_window_counts.restype = None
            lib.oracle_score.argtypes = [_i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, _i32p, _i32p,
                                         _f64p, _f64p, _i64p, _f64p, _i32p]
            lib.oracle_score.restype = ctypes.c_int
            lib.oracle_score_at.argtypes = [_i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, _i32p, _i32p, _f64p, _f64p, _i64p,
                                            ctypes.c_int64, _i32p, _f64p]
            lib.oracle_score_at.restype = None
            lib.oracle_coarse_to_dilation.argtypes = [_f64p, ctypes.c_int, ctypes.c_int, _f64p]
            lib.oracle_coarse_to_dilation.restype = None
            lib.oracle_coarse_direct.argtypes = [_i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, _f64p, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_int]
            lib.oracle_coarse_direct.restype = ctypes.c_double
            _lib = lib
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _c(a, dtype):
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


# ----------------------------------------------------------------------------------------
def splitmix64(seed: int, n: int) -> list[int]:
    """First n SplitMix64 outputs from state ``seed``."""
    lib = _load()
    st = ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF)
    return [int(lib.oracle_splitmix64_next(ctypes.byref(st))) for _ in range(n)]


def kmeans_init(l: int, k: int, seed: int) -> np.ndarray:
    """k distinct initial pixel indices in [0, l) (partial Fisher-Yates, SplitMix64)."""
    out = np.empty(k, np.int64)
    if _load().oracle_kmeans_init(l, k, seed & 0xFFFFFFFFFFFFFFFF, _p(out, _i64p)) != 0:
        raise ValueError("kmeans_init: need 1 <= k <= l")
    return out


def assign(X, C, *, return_dist: bool = False):
    """Nearest centroid of every row of X (n x D float32) among C (k x D float32).

    Returns int32 labels (lowest index on ties); with ``return_dist`` also the FP64
    smallest and second-smallest squared distances.
    """
    X = _c(X, np.float32)
    C = _c(C, np.float32)
    D = X.shape[-1]
    X2 = X.reshape(-1, D)
    n, k = X2.shape[0], C.shape[0]
    lab = np.empty(n, np.int32)
    d1 = np.empty(n, np.float64)
    d2 = np.empty(n, np.float64)
    _load().oracle_assign(_p(X2, _f32p), n, D, _p(C, _f32p), k, _p(lab, _i32p),
                          _p(d1, _f64p), _p(d2, _f64p))
    shape = X.shape[:-1]
    if return_dist:
        return lab.reshape(shape), d1.reshape(shape), d2.reshape(shape)
    return lab.reshape(shape)


def relative_gap(d1: np.ndarray, d2: np.ndarray) -> np.ndarray:
    """g = (d2 - d1) / max(d2, tiny): the oracle's own near-tie measure per pixel."""
    return (d2 - d1) / np.maximum(d2, 1e-300)


def fit_codebook(T, k: int, iters: int, seed: int) -> np.ndarray:
    """k-means codebook (k x D float32) of the template features T (... x D float32)."""
    T = _c(T, np.float32)
    D = T.shape[-1]
    T2 = T.reshape(-1, D)
    C = np.empty((k, D), np.float32)
    if _load().oracle_fit_codebook(_p(T2, _f32p), T2.shape[0], D, k, iters,
                                   seed & 0xFFFFFFFFFFFFFFFF, _p(C, _f32p)) != 0:
        raise ValueError("fit_codebook: need 1 <= k <= number of template pixels")
    return C


def kmeans_objective(T, C) -> float:
    T = _c(T, np.float32)
    C = _c(C, np.float32)
    D = T.shape[-1]
    T2 = T.reshape(-1, D)
    return float(_load().oracle_kmeans_objective(_p(T2, _f32p), T2.shape[0], D, _p(C, _f32p),
                                                 C.shape[0]))


def flatten_bank(bank):
    """(n_rects int32[F], rects int32[R,5], w_f float64[F], area float64[F])."""
    n_rects = np.array([len(f["rects"]) for f in bank], np.int32)
    rects = np.array([list(r) for f in bank for r in f["rects"]], np.int32).reshape(-1, 5)
    w_f = np.array([f["w_f"] for f in bank], np.float64)
    area = np.array([f["area"] for f in bank], np.float64)
    return n_rects, np.ascontiguousarray(rects), w_f, area


def filter_counts(labels, k: int, bank) -> np.ndarray:
    """Template representation vectors: F x k int64 weighted label counts."""
    lab = _c(labels, np.int32)
    h, w = lab.shape
    n_rects, rects, _, _ = flatten_bank(bank)
    out = np.empty((len(bank), k), np.int64)
    _load().oracle_filter_counts(_p(lab, _i32p), h, w, k, len(bank), _p(n_rects, _i32p),
                                 _p(rects, _i32p), _p(out, _i64p))
    return out


def window_counts(labels, k: int, bank, wy: int, wx: int) -> np.ndarray:
    lab = _c(labels, np.int32)
    H, W = lab.shape
    n_rects, rects, _, _ = flatten_bank(bank)
    out = np.empty((len(bank), k), np.int64)
    _load().oracle_window_counts(_p(lab, _i32p), H, W, k, wy, wx, len(bank),
                                 _p(n_rects, _i32p), _p(rects, _i32p), _p(out, _i64p))
    return out


def score(q_labels, k: int, th: int, tw: int, bank, t_counts):
    """Eq. 2 heatmap ((H-th+1) x (W-tw+1) float64) and its argmax (y, x)."""
    lab = _c(q_labels, np.int32)
    H, W = lab.shape
    n_rects, rects, w_f, area = flatten_bank(bank)
    tc = _c(t_counts, np.int64)
    heat = np.empty((H - th + 1, W - tw + 1), np.float64)
    am = np.empty(2, np.int32)
    rc = _load().oracle_score(_p(lab, _i32p), H, W, k, th, tw, len(bank), _p(n_rects, _i32p),
                              _p(rects, _i32p), _p(w_f, _f64p), _p(area, _f64p),
                              _p(tc, _i64p), _p(heat, _f64p), _p(am, _i32p))
    if rc != 0:
        raise ValueError("score: template larger than query")
    return heat, (int(am[0]), int(am[1]))


def score_at(q_labels, k: int, bank, t_counts, windows) -> np.ndarray:
    """Eq. 2 at the given window top-left corners (n x 2 int (y, x))."""
    lab = _c(q_labels, np.int32)
    H, W = lab.shape
    n_rects, rects, w_f, area = flatten_bank(bank)
    tc = _c(t_counts, np.int64)
    win = _c(windows, np.int32).reshape(-1, 2)
    out = np.empty(win.shape[0], np.float64)
    _load().oracle_score_at(_p(lab, _i32p), H, W, k, len(bank), _p(n_rects, _i32p),
                            _p(rects, _i32p), _p(w_f, _f64p), _p(area, _f64p), _p(tc, _i64p),
                            win.shape[0], _p(win, _i32p), _p(out, _f64p))
    return out


def coarse_to_dilation(f_i) -> np.ndarray:
    """Algorithm 2: (r_w x r_h) coarse filter -> ((r_w+1) x (r_h+1)) dilation filter."""
    f = _c(f_i, np.float64)
    r_w, r_h = f.shape
    out = np.empty((r_w + 1, r_h + 1), np.float64)
    _load().oracle_coarse_to_dilation(_p(f, _f64p), r_w, r_h, _p(out, _f64p))
    return out


def coarse_direct(labels, wy: int, wx: int, cls: int, f_i, d_x: int, d_y: int) -> float:
    """Direct bin-weighted count of label ``cls`` for a coarse filter over one window."""
    lab = _c(labels, np.int32)
    f = _c(f_i, np.float64)
    r_w, r_h = f.shape
    return float(_load().oracle_coarse_direct(_p(lab, _i32p), lab.shape[1], wy, wx, cls,
                                              _p(f, _f64p), r_w, r_h, d_x, d_y))


def set_threads(n: int) -> int:
    """Threads of the oracle's parallel loops (timing only: results do not depend on it);
    returns the previous count."""
    return int(_load().oracle_set_threads(int(n)))
