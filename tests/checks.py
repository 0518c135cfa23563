"""Parity checks shared by the GPU tests (test infrastructure).

Three bars on a floating-point result Y against the FP64 oracle's Y_o:

* normwise  ||Y - Y_o||_F / (||W||_F ||X||_F) <= the stated tolerance
  (1e-6 FP32, 4e-3 FP16/BF16 inputs with FP32 accumulation);
* relative  ||Y - Y_o||_F / ||Y_o||_F <= 1e-2 for 16-bit outputs (1e-5 for
  FP32): for N(0, 1) data ||Y||_F is about ||W||_F ||X||_F / sqrt(k), so
  only this bar still sees a dropped block or interval at k = 4096;
* componentwise  max |Y - Y_o| / (|W| |X|) <= 2 (u_out + u_w + s 2^-24):
  rounding an FP32 sum of s products, then the output to unit roundoff
  u_out (and, for E4M3 weights, code x scale to the 16-bit operand type,
  u_w), bounds the error of each entry by that fraction of (|W| |X|)_ij.

And exact identities for integer-valued operands, which hold for every row
and column of Y at any size: Y c = W (X c) and r^T Y = (W^T r)^T X for
random +-1 vectors c and r, with every quantity an integer computed
exactly in FP64 (by the oracle's product and transposed product).
"""
import numpy as np

import oracle

try:
    import torch
    UNIT = {torch.float32: 2.0 ** -24, torch.float16: 2.0 ** -11, torch.bfloat16: 2.0 ** -8}
    TOL = {torch.float32: 1e-6, torch.float16: 4e-3, torch.bfloat16: 4e-3}
    REL = {torch.float32: 1e-5, torch.float16: 1e-2, torch.bfloat16: 1e-2}
except ImportError:  # CPU-only environments without torch never call these
    UNIT = TOL = REL = {}


def max_terms(brow, b):
    """Largest number of products summed into one entry of Y: b times the
    largest block count of a block row."""
    brow = np.asarray(brow)
    if brow.size == 0:
        return 0
    return int(np.bincount(brow).max()) * b


def assert_parity(Y, Y_o, W_fro, X, absWX, dt, terms, tol=None, u_w=0.0):
    """The normwise, relative and componentwise bars (see the module text).
    Returns the three measured values."""
    tol = TOL[dt] if tol is None else tol
    nw = oracle.normwise_err(Y, Y_o, W_fro, X)
    rel = oracle.relative_err(Y, Y_o)
    cw = oracle.componentwise_ratio(Y, Y_o, absWX)
    bound = 2.0 * (UNIT[dt] + u_w + terms * 2.0 ** -24)
    assert nw <= tol, ("normwise", nw, tol)
    assert rel <= REL[dt], ("relative", rel, REL[dt])
    assert cw <= bound, ("componentwise", cw, bound)
    return nw, rel, cw


def sub_rows(brow, bcol, vals, rows_blk):
    """The blocks of the chosen block rows, renumbered 0, 1, ... in the
    order given (for an oracle product over those rows only)."""
    brow = np.asarray(brow)
    sel = np.isin(brow, rows_blk)
    remap = {int(r): i for i, r in enumerate(rows_blk)}
    br = np.array([remap[int(r)] for r in brow[sel]], np.int32)
    return br, np.asarray(bcol)[sel], vals[sel], sel


def check_rows(Y, rows_blk, m, k, b, brow, bcol, vals, X, dt, tol=None, u_w=0.0):
    """Sampled block rows of Y against the oracle, with all three bars."""
    br, bc, v, _ = sub_rows(brow, bcol, vals, rows_blk)
    mr = len(rows_blk) * b
    Yo = oracle.spmm(mr, k, b, br, bc, v, X)
    A = oracle.spmm(mr, k, b, br, bc, np.abs(oracle.to_f64(v)), np.abs(oracle.to_f64(X)))
    Ys = np.concatenate([oracle.to_f64(Y[r * b:(r + 1) * b]) for r in rows_blk])
    return assert_parity(Ys, Yo, oracle.block_fro(v), X, A, dt, max_terms(br, b), tol, u_w)


def exact_identities(Y, m, k, b, brow, bcol, vals, X, seed=0, reps=2):
    """Integer operands: every row and column of Y through Y c = W (X c)
    and r^T Y = (W^T r)^T X, exactly (see the module text)."""
    Yf = oracle.to_f64(Y)
    Xf = oracle.to_f64(X)
    assert np.all(np.isfinite(Yf)) and np.array_equal(Yf, np.round(Yf * 2) / 2), \
        "integer-valued operands must give a result on the half-integer grid"
    rng = np.random.default_rng(seed)
    for _ in range(reps):
        c = rng.choice([-1.0, 1.0], size=Xf.shape[1])
        want = oracle.spmm(m, k, b, brow, bcol, vals, (Xf @ c)[:, None])[:, 0]
        assert np.array_equal(Yf @ c, want), "some row of Y differs (Y c != W X c)"
        r = rng.choice([-1.0, 1.0], size=m)
        wr = oracle.spmm_t(m, k, b, brow, bcol, vals, r[:, None])[:, 0]
        assert np.array_equal(r @ Yf, wr @ Xf), "some column of Y differs (r^T Y != r^T W X)"


def exact_rows(Y, rows_blk, k, b, brow, bcol, vals, X, dt):
    """Sampled block rows of Y bit for bit equal to the oracle's result
    rounded once to the output type (integer operands)."""
    br, bc, v, _ = sub_rows(brow, bcol, vals, rows_blk)
    Yo = oracle.spmm(len(rows_blk) * b, k, b, br, bc, v, X)
    Ys = torch.cat([Y[r * b:(r + 1) * b].cpu() for r in rows_blk])
    assert torch.equal(Ys, torch.from_numpy(Yo).to(dt))
