"""Oracle for the block-sparse x dense product (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` / reference leg may import this package.  The product path
(the CUDA library and its Python binding) never imports it, and this package
imports nothing from the product.

Contents
--------
* ``spmm(...)`` -- the FP64 definition of Section 3 (C, single thread), over
  the inputs exactly as supplied (values widened to FP64 without rounding).
* ``spmm_t(...)`` -- the transposed product W^T.Y on the same blocks, written
  out from its own definition (not through ``spmm``).
* ``sddmm(...)`` -- dW = (dY.X^T) on the block mask (the product's gradient
  with respect to the stored blocks), from its definition.
* ``e4m3_to_f64`` -- FP8 E4M3 decoding from the format definition.
* ``e4m3_block_values`` -- effective FP64 values of E4M3 blocks, one FP32
  scale per block (pattern order).
* ``normwise_err`` -- ||Y - Y_o||_F / (||W||_F ||X||_F), the acceptance metric.
* ``relative_err`` -- ||Y - Y_o||_F / ||Y_o||_F, the bar that still bites at
  large k (the normwise metric shrinks like 1/sqrt(k) for random data).
* ``componentwise_ratio`` -- max_ij |Y - Y_o|_ij / (|W| |X|)_ij, the
  componentwise diagnostic of the error analysis of a sum of products.
* ``oracle.plan`` -- the integer plan / partition rules (Section 3.2, 3.3,
  Appendix A.2, and this library's GPU work decomposition), plain Python.

Parity pins: see tests/test_oracle_pins.py and tests/test_oracle_plan.py.
Paper values: the paper prints no Y values and no worked plans (its Fig. 1
and Fig. 7 images are missing), so no golden value comes from the paper
itself except the App. A.2 partition formula's closed forms.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = _bind(ctypes.CDLL(path))
    return _lib


def _bind(lib):
    i64, i32p = ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_spmm_f64.restype = ctypes.c_int
    lib.oracle_spmm_f64.argtypes = [i64, i64, i64, i64, i64, i32p, i32p, dp, dp,
                                    i64, dp, i64]
    lib.oracle_spmm_t_f64.restype = ctypes.c_int
    lib.oracle_spmm_t_f64.argtypes = [i64, i64, i64, i64, i64, i32p, i32p, dp, dp,
                                      i64, dp, i64]
    lib.oracle_sddmm_f64.restype = ctypes.c_int
    lib.oracle_sddmm_f64.argtypes = [i64, i64, i64, i64, i64, i32p, i32p, dp, i64, dp, i64,
                                     dp]
    lib.oracle_e4m3_to_f64.restype = ctypes.c_int64
    lib.oracle_e4m3_to_f64.argtypes = [ctypes.POINTER(ctypes.c_uint8), i64, dp]
    return lib


def load_variant(path):
    """Loads a separately built copy of the oracle (mutation tests)."""
    return _bind(ctypes.CDLL(path))


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def to_f64(a):
    """Widens a numpy array or torch CPU tensor (f16/bf16/f32/f64) to FP64
    exactly; FP8 E4M3 bytes go through ``e4m3_to_f64``."""
    if hasattr(a, "detach"):  # torch tensor: bf16 has no numpy dtype
        import torch
        t = a.detach().cpu()
        if t.dtype == torch.float8_e4m3fn:
            return e4m3_to_f64(t.view(torch.uint8).numpy())
        return t.to(torch.float64).numpy()
    return np.asarray(a, dtype=np.float64)


def spmm(m, k, b, brow, bcol, vals, X, lib=None):
    """Y = W.X in FP64 per Section 3.

    brow, bcol: int arrays of length nnzb (block coordinates, user order).
    vals: (nnzb, b, b) values, any float dtype, widened exactly to FP64.
    X: (k, n).  Returns Y (m, n) float64.
    """
    lib = lib or _load()
    brow = np.ascontiguousarray(brow, dtype=np.int32)
    bcol = np.ascontiguousarray(bcol, dtype=np.int32)
    nnzb = brow.shape[0]
    v = np.ascontiguousarray(to_f64(vals)).reshape(nnzb * b * b)
    x = np.ascontiguousarray(to_f64(X))
    assert x.shape[0] == k
    n = x.shape[1]
    y = np.empty((m, n), dtype=np.float64)
    rc = lib.oracle_spmm_f64(m, k, n, b, nnzb, _ptr(brow, ctypes.c_int32),
                             _ptr(bcol, ctypes.c_int32), _ptr(v, ctypes.c_double),
                             _ptr(x, ctypes.c_double), n, _ptr(y, ctypes.c_double), n)
    if rc != 0:
        raise ValueError("oracle_spmm_f64: pattern or sizes invalid (rc=%d)" % rc)
    return y


def spmm_t(m, k, b, brow, bcol, vals, Y, lib=None):
    """Z = W^T.Y in FP64 (the transposed product on the same blocks).

    W is m x k given by brow, bcol, vals (user order, blocks row-major);
    Y: (m, n).  Returns Z (k, n) float64.
    """
    lib = lib or _load()
    brow = np.ascontiguousarray(brow, dtype=np.int32)
    bcol = np.ascontiguousarray(bcol, dtype=np.int32)
    nnzb = brow.shape[0]
    v = np.ascontiguousarray(to_f64(vals)).reshape(nnzb * b * b)
    y = np.ascontiguousarray(to_f64(Y))
    assert y.shape[0] == m
    n = y.shape[1]
    z = np.empty((k, n), dtype=np.float64)
    rc = lib.oracle_spmm_t_f64(m, k, n, b, nnzb, _ptr(brow, ctypes.c_int32),
                               _ptr(bcol, ctypes.c_int32), _ptr(v, ctypes.c_double),
                               _ptr(y, ctypes.c_double), n, _ptr(z, ctypes.c_double), n)
    if rc != 0:
        raise ValueError("oracle_spmm_t_f64: pattern or sizes invalid (rc=%d)" % rc)
    return z


def sddmm(m, k, b, brow, bcol, dY, X, lib=None):
    """dW = (dY.X^T) on the block mask in FP64: for every block p (user
    order), dW[p][ii][l] = sum_j dY[brow*b+ii, j] * X[bcol*b+l, j] (Section 3's
    product differentiated with respect to the stored blocks).

    dY: (m, n), X: (k, n).  Returns dW (nnzb, b, b) float64.
    """
    lib = lib or _load()
    brow = np.ascontiguousarray(brow, dtype=np.int32)
    bcol = np.ascontiguousarray(bcol, dtype=np.int32)
    nnzb = brow.shape[0]
    dy = np.ascontiguousarray(to_f64(dY))
    x = np.ascontiguousarray(to_f64(X))
    assert dy.shape[0] == m and x.shape[0] == k and dy.shape[1] == x.shape[1]
    n = x.shape[1]
    out = np.empty((nnzb, b, b), dtype=np.float64)
    rc = lib.oracle_sddmm_f64(m, k, n, b, nnzb, _ptr(brow, ctypes.c_int32),
                              _ptr(bcol, ctypes.c_int32), _ptr(dy, ctypes.c_double), n,
                              _ptr(x, ctypes.c_double), n, _ptr(out, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle_sddmm_f64: pattern or sizes invalid (rc=%d)" % rc)
    return out


def e4m3_to_f64(codes, lib=None):
    """Decodes uint8 E4M3 codes to FP64 from the format definition."""
    lib = lib or _load()
    c = np.ascontiguousarray(codes, dtype=np.uint8)
    out = np.empty(c.shape, dtype=np.float64)
    lib.oracle_e4m3_to_f64(_ptr(c.reshape(-1), ctypes.c_uint8), c.size,
                           _ptr(out.reshape(-1), ctypes.c_double))
    return out


def e4m3_block_values(codes, scales):
    """Effective FP64 values of E4M3 blocks with one FP32 scale per block:
    v(p, i, l) = decode(code(p, i, l)) * scale[p], codes (nnzb, b, b) and
    scales (nnzb,) both in the pattern's order (block p of the pattern)."""
    d = e4m3_to_f64(codes)
    if d.ndim != 3:
        raise ValueError("codes must be (nnzb, b, b)")
    s = np.asarray(scales, dtype=np.float64).reshape(-1)
    if s.shape[0] != d.shape[0]:
        raise ValueError("one scale per block required")
    return d * s[:, None, None]


def normwise_err(Y, Y_o, W_fro, X):
    """||Y - Y_o||_F / (||W||_F * ||X||_F), all in FP64 on the host.

    ``W_fro`` is ||W||_F (= || |W| ||_F).  When the denominator is 0 the
    metric is defined as 0 if Y == 0 exactly and +inf otherwise."""
    Y = to_f64(Y)
    d = float(W_fro) * float(np.linalg.norm(to_f64(X)))
    num = float(np.linalg.norm(Y - Y_o))
    if d == 0.0:
        return 0.0 if not np.any(Y) else float("inf")
    return num / d


def relative_err(Y, Y_o):
    """||Y - Y_o||_F / ||Y_o||_F in FP64 (0 when both are 0, +inf when only
    Y_o is).  For N(0, 1) data ||Y||_F is about ||W||_F ||X||_F / sqrt(k),
    so a bar on this ratio sees a dropped block that the normwise metric
    would admit at large k."""
    Y = to_f64(Y)
    Y_o = to_f64(Y_o)
    num = float(np.linalg.norm(Y - Y_o))
    den = float(np.linalg.norm(Y_o))
    if den == 0.0:
        return 0.0 if num == 0.0 else float("inf")
    return num / den


def componentwise_ratio(Y, Y_o, absWX):
    """max_ij |Y - Y_o|_ij / (|W| |X|)_ij over the entries where the
    denominator is positive; an entry with (|W| |X|)_ij = 0 must match
    exactly (else +inf).  ``absWX`` is the product of the absolute values,
    e.g. ``spmm(m, k, b, brow, bcol, |vals|, |X|)``.  Rounding the FP32
    accumulation of s terms and then the output to unit roundoff u bounds it
    by about u + s * 2^-24."""
    Y = to_f64(Y)
    Y_o = to_f64(Y_o)
    A = to_f64(absWX)
    diff = np.abs(Y - Y_o)
    pos = A > 0
    if np.any(diff[~pos] != 0):
        return float("inf")
    if not np.any(pos):
        return 0.0
    return float(np.max(diff[pos] / A[pos]))


def block_fro(vals):
    """||W||_F from the block values (FP64)."""
    return float(np.linalg.norm(to_f64(vals)))
