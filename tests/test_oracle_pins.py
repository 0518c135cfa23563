"""Pins of the FP64 oracle against what the paper and mathematics fix.

Section 3 defines Y = (M (.) W) * X with M_ij = Mhat_{floor(i/b), floor(j/b)}.
Each ``check_*`` takes the oracle's C library handle so that the mutation
tests (test_oracle_mutants.py) can re-run the same checks against copies of
the oracle with a planted mistake.
"""
import numpy as np
import pytest

import oracle
from paper_2303_16999_gb300 import workloads as wl


def _blocks_from_dense(W, Mhat, b):
    """Turns a dense W and a block mask Mhat (Section 3 notation) into the
    user block list, padding edge blocks with zeros beyond m x k."""
    m, k = W.shape
    rows, cols = np.nonzero(Mhat)
    vals = np.zeros((len(rows), b, b))
    for p, (r, c) in enumerate(zip(rows, cols)):
        blk = W[r * b:(r + 1) * b, c * b:(c + 1) * b]
        vals[p, :blk.shape[0], :blk.shape[1]] = blk
    return rows.astype(np.int32), cols.astype(np.int32), vals


def _masked_product(W, Mhat, b, X):
    """Y = (M (.) W) X exactly as written in Section 3, with numpy."""
    m, k = W.shape
    i = np.arange(m)[:, None] // b
    j = np.arange(k)[None, :] // b
    M = Mhat[i, j]
    return (M * W) @ X


def check_definition_brute_force(lib):
    rng = np.random.default_rng(11)
    for b in (1, 2, 3, 4, 8, 16):
        for (m, k, n) in ((16, 16, 5), (40, 24, 7), (10, 13, 3), (64, 48, 9)):
            mb, kb = -(-m // b), -(-k // b)
            Mhat = rng.random((mb, kb)) < 0.35
            W = rng.standard_normal((m, k))
            X = rng.standard_normal((k, n))
            brow, bcol, vals = _blocks_from_dense(W, Mhat, b)
            # shuffle the user order: the definition does not depend on it
            o = rng.permutation(len(brow))
            Y = oracle.spmm(m, k, b, brow[o], bcol[o], vals[o], X, lib=lib)
            Yr = _masked_product(W, Mhat, b, X)
            assert np.allclose(Y, Yr, rtol=1e-12, atol=1e-12), (b, m, k, n)


def check_hand_example(lib):
    # 4 x 4 W with two 2 x 2 blocks (b = 2): blocks at (0, 1) and (1, 0).
    #   W = [[0, 0, 1, 2],
    #        [0, 0, 3, 4],
    #        [5, 6, 0, 0],
    #        [7, 8, 0, 0]]
    brow = np.array([0, 1], np.int32)
    bcol = np.array([1, 0], np.int32)
    vals = np.array([[[1, 2], [3, 4]], [[5, 6], [7, 8]]], np.float64)
    X = np.array([[1, 0], [0, 1], [2, 0], [0, 3]], np.float64)
    # row 0: 1*2 + 2*0 = 2 ; 1*0 + 2*3 = 6
    # row 1: 3*2 + 4*0 = 6 ; 3*0 + 4*3 = 12
    # row 2: 5*1 + 6*0 = 5 ; 5*0 + 6*1 = 6
    # row 3: 7*1 + 8*0 = 7 ; 7*0 + 8*1 = 8
    want = np.array([[2, 6], [6, 12], [5, 6], [7, 8]], np.float64)
    Y = oracle.spmm(4, 4, 2, brow, bcol, vals, X, lib=lib)
    assert np.array_equal(Y, want)


def check_exact_integers(lib):
    """Values and X in {-3..3}: every product and partial sum is an integer
    far below 2^53, so the FP64 oracle must equal exact integer arithmetic."""
    rng = np.random.default_rng(5)
    for b in (1, 4, 8, 16):
        m, k, n = 64, 96, 11
        mb, kb = m // b, k // b
        nnzb = max(1, (mb * kb) // 3)
        idx = rng.choice(mb * kb, nnzb, replace=False)
        brow, bcol = (idx // kb).astype(np.int32), (idx % kb).astype(np.int32)
        vals = rng.integers(-3, 4, size=(nnzb, b, b))
        X = rng.integers(-3, 4, size=(k, n))
        W = np.zeros((m, k), dtype=np.int64)
        for p in range(nnzb):
            W[brow[p] * b:(brow[p] + 1) * b, bcol[p] * b:(bcol[p] + 1) * b] = vals[p]
        want = W @ X  # int64 matmul: exact
        Y = oracle.spmm(m, k, b, brow, bcol, vals.astype(np.float64), X.astype(np.float64), lib=lib)
        assert np.array_equal(Y, want.astype(np.float64)), b


def check_density_one_is_dense(lib):
    import torch
    rng = np.random.default_rng(7)
    for b in (1, 4, 8, 16):
        m, k, n = 48, 32, 6
        mb, kb = m // b, k // b
        W = rng.standard_normal((m, k))
        X = rng.standard_normal((k, n))
        brow, bcol, vals = _blocks_from_dense(W, np.ones((mb, kb), bool), b)
        Y = oracle.spmm(m, k, b, brow, bcol, vals, X, lib=lib)
        ref = torch.matmul(torch.from_numpy(W), torch.from_numpy(X)).numpy()
        assert np.allclose(Y, ref, rtol=1e-12, atol=1e-12)


def check_block_identity(lib):
    rng = np.random.default_rng(3)
    for b in (1, 4, 8, 16):
        m = 64
        brow = np.arange(m // b, dtype=np.int32)
        bcol = brow.copy()
        vals = np.broadcast_to(np.eye(b), (m // b, b, b)).copy()
        X = rng.standard_normal((m, 5))
        Y = oracle.spmm(m, m, b, brow, bcol, vals, X, lib=lib)
        assert np.array_equal(Y, X)


def check_empty_pattern(lib):
    X = np.ones((32, 4))
    Y = oracle.spmm(48, 32, 4, np.zeros(0, np.int32), np.zeros(0, np.int32),
                    np.zeros((0, 4, 4)), X, lib=lib)
    assert Y.shape == (48, 4) and not np.any(Y)


def check_linearity(lib):
    rng = np.random.default_rng(9)
    b, m, k, n = 4, 32, 40, 6
    mb, kb = m // b, k // b
    idx = rng.choice(mb * kb, 20, replace=False)
    brow, bcol = (idx // kb).astype(np.int32), (idx % kb).astype(np.int32)
    V1 = rng.standard_normal((20, b, b))
    V2 = rng.standard_normal((20, b, b))
    X = rng.standard_normal((k, n))
    a, c = 0.75, -2.5
    Y = oracle.spmm(m, k, b, brow, bcol, a * V1 + c * V2, X, lib=lib)
    Y1 = oracle.spmm(m, k, b, brow, bcol, V1, X, lib=lib)
    Y2 = oracle.spmm(m, k, b, brow, bcol, V2, X, lib=lib)
    assert np.allclose(Y, a * Y1 + c * Y2, rtol=1e-12, atol=1e-12)


def check_permutation_equivariance(lib):
    rng = np.random.default_rng(13)
    for b in (1, 4, 8):
        m, k, n = 48, 64, 5
        mb, kb = m // b, k // b
        nnzb = (mb * kb) // 4
        idx = rng.choice(mb * kb, nnzb, replace=False)
        brow, bcol = (idx // kb).astype(np.int32), (idx % kb).astype(np.int32)
        V = rng.standard_normal((nnzb, b, b))
        X = rng.standard_normal((k, n))
        Y = oracle.spmm(m, k, b, brow, bcol, V, X, lib=lib)
        # block-row permutation pi: block row r moves to pi[r]
        pi = rng.permutation(mb)
        Yp = oracle.spmm(m, k, b, pi[brow].astype(np.int32), bcol, V, X, lib=lib)
        for r in range(mb):
            assert np.array_equal(Yp[pi[r] * b:(pi[r] + 1) * b], Y[r * b:(r + 1) * b])
        # block-column permutation sigma on bcol and on X's row blocks
        sg = rng.permutation(kb)
        Xs = np.empty_like(X)
        for c in range(kb):
            Xs[sg[c] * b:(sg[c] + 1) * b] = X[c * b:(c + 1) * b]
        Ys = oracle.spmm(m, k, b, brow, sg[bcol].astype(np.int32), V, Xs, lib=lib)
        assert np.allclose(Ys, Y, rtol=1e-12, atol=1e-12)


ALL_CHECKS = [check_definition_brute_force, check_hand_example, check_exact_integers,
              check_density_one_is_dense, check_block_identity, check_empty_pattern,
              check_linearity, check_permutation_equivariance]


@pytest.mark.parametrize("check", ALL_CHECKS, ids=lambda f: f.__name__)
def test_oracle_pin(check):
    check(oracle._load())


def test_oracle_rejects_out_of_range():
    with pytest.raises(ValueError):
        oracle.spmm(16, 16, 4, np.array([4], np.int32), np.array([0], np.int32),
                    np.zeros((1, 4, 4)), np.zeros((16, 2)))


# ------------------------------------------------------------- E4M3 --------
def test_e4m3_closed_forms():
    codes = np.array([0x00, 0x80, 0x38, 0xB8, 0x7E, 0xFE, 0x01, 0x08, 0x07, 0x40, 0x3C], np.uint8)
    want = [0.0, -0.0, 1.0, -1.0, 448.0, -448.0, 2.0 ** -9, 2.0 ** -6, 7 * 2.0 ** -9, 2.0, 1.5]
    got = oracle.e4m3_to_f64(codes)
    assert list(got) == want
    assert np.isnan(oracle.e4m3_to_f64(np.array([0x7F, 0xFF], np.uint8))).all()


def test_e4m3_matches_library_decoder():
    import torch
    codes = np.arange(256, dtype=np.uint8)
    ours = oracle.e4m3_to_f64(codes)
    lib = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    both_nan = np.isnan(ours) & np.isnan(lib)
    assert np.array_equal(ours[~both_nan], lib[~both_nan])
    assert both_nan.sum() == 2


# E4M3 blocks with one FP32 scale each.  Codes are sign | 4 exponent bits
# (bias 7) | 3 mantissa bits, decoded here by hand:
#   0x38 = +1.0, 0x40 = +2.0, 0xB8 = -1.0, 0x3C = +1.5,
#   0x7E = +448 (1.75 * 2^8), 0x01 = 2^-9 (smallest subnormal), 0xC0 = -2.0,
#   0x44 = +3.0.
# As many blocks as a block has rows, so that a scale broadcast along the
# wrong axis still has the right shape and must be caught by value.
E4M3_CODES = np.array([[[0x38, 0x40], [0xB8, 0x3C]],
                       [[0x7E, 0x01], [0xC0, 0x44]]], np.uint8)
E4M3_SCALES = np.array([0.5, 3.0], np.float32)
E4M3_WANT = np.array([[[0.5, 1.0], [-0.5, 0.75]],
                      [[1344.0, 3.0 * 2.0 ** -9], [-6.0, 9.0]]])


def check_e4m3_block_values(fn):
    """Block p scaled by its own scale, every element of the block alike."""
    got = fn(E4M3_CODES, E4M3_SCALES)
    assert got.shape == E4M3_WANT.shape
    assert np.array_equal(got, E4M3_WANT)


def check_e4m3_pattern_order(fn):
    """Scales follow the pattern's order, not the block-CSR order: with the
    pattern listing block rows 1, 0 (b = 2, m = 4, k = 2) and X = I, Y's
    block row r is the block whose pattern entry names row r."""
    brow = np.array([1, 0], np.int32)
    bcol = np.zeros(2, np.int32)
    v = fn(E4M3_CODES, E4M3_SCALES)
    Y = oracle.spmm(4, 2, 2, brow, bcol, v, np.eye(2))
    want = np.concatenate([E4M3_WANT[1], E4M3_WANT[0]])
    assert np.array_equal(Y, want)


E4M3_CHECKS = [check_e4m3_block_values, check_e4m3_pattern_order]


@pytest.mark.parametrize("check", E4M3_CHECKS, ids=lambda f: f.__name__)
def test_e4m3_block_values_pin(check):
    check(oracle.e4m3_block_values)


def test_e4m3_block_values_rejects_bad_shapes():
    with pytest.raises(ValueError):
        oracle.e4m3_block_values(E4M3_CODES, E4M3_SCALES[:1])
    with pytest.raises(ValueError):
        oracle.e4m3_block_values(E4M3_CODES.reshape(2, 4), E4M3_SCALES)


# ------------------------------------------------------- error metric ------
def test_normwise_err_closed_form():
    Yo = np.zeros((3, 4))
    Y = Yo.copy()
    Y[0, 0], Y[2, 3] = 3.0, 4.0          # ||Y - Yo||_F = 5
    X = np.zeros((2, 4))
    X[1, 1] = 2.0                        # ||X||_F = 2
    assert oracle.normwise_err(Y, Yo, 10.0, X) == 5.0 / 20.0
    assert oracle.normwise_err(Yo, Yo, 0.0, X) == 0.0
    assert oracle.normwise_err(Y, Yo, 0.0, X) == float("inf")


def test_relative_err_closed_form():
    Yo = np.zeros((2, 2))
    Yo[0, 0], Yo[1, 1] = 3.0, 4.0        # ||Yo||_F = 5
    Y = Yo.copy()
    Y[0, 1] = 1.0                        # ||Y - Yo||_F = 1
    assert oracle.relative_err(Y, Yo) == 0.2
    assert oracle.relative_err(np.zeros(3), np.zeros(3)) == 0.0
    assert oracle.relative_err(np.ones(3), np.zeros(3)) == float("inf")


def test_componentwise_ratio_closed_form():
    Yo = np.array([[1.0, 2.0], [0.0, 5.0]])
    A = np.array([[4.0, 8.0], [0.0, 10.0]])
    Y = np.array([[1.5, 2.0], [0.0, 4.0]])     # |dY| / A = 0.125, 0, -, 0.1
    assert oracle.componentwise_ratio(Y, Yo, A) == 0.125
    Y[1, 0] = 1e-30                             # a nonzero where |W||X| = 0
    assert oracle.componentwise_ratio(Y, Yo, A) == float("inf")


def test_componentwise_ratio_sees_a_dropped_block():
    """At large k a dropped block moves ||Y - Y_o||_F / (||W||_F ||X||_F)
    by about 1/sqrt(k * nnz_row) only, but the relative and componentwise
    ratios by far more than any 16-bit rounding (u = 2^-8 for BF16)."""
    rng = np.random.default_rng(3)
    m, k, n, b = 64, 4096, 16, 16
    c = wl.problem(5, m, k, n, b, wl.nnzb_for(m, k, b, 1 / 4))
    Yo = oracle.spmm(m, k, b, c["brow"], c["bcol"], c["vals"], c["X"])
    keep = np.ones(len(c["brow"]), bool)
    keep[rng.integers(len(keep))] = False
    Yd = oracle.spmm(m, k, b, c["brow"][keep], c["bcol"][keep], c["vals"][keep], c["X"])
    A = oracle.spmm(m, k, b, c["brow"], c["bcol"], np.abs(c["vals"]), np.abs(c["X"]))
    assert oracle.normwise_err(Yd, Yo, oracle.block_fro(c["vals"]), c["X"]) < 4e-3
    assert oracle.relative_err(Yd, Yo) > 1e-2
    assert oracle.componentwise_ratio(Yd, Yo, A) > 2 * 2.0 ** -8 + 4096 * 2.0 ** -24


def test_workload_recipe_shapes():
    c = wl.smoke_case()
    assert c["vals"].shape == (512, 4, 4) and c["X"].shape == (256, 64)
    assert len(set(zip(c["brow"].tolist(), c["bcol"].tolist()))) == 512
    s = wl.sweep_case(16, 1 / 32, m=256, k=256, n=8)
    assert s["vals"].shape[0] == (256 // 16) ** 2 // 32
    assert wl.sweep_seed(16, 1 / 32) == 16005 and wl.sweep_seed(1, 1 / 4) == 1002
    d = wl.dynamic_call(3, m=512, k=512, n=4)
    assert d["nnzb_max"] // 2 <= len(d["brow"]) <= d["nnzb_max"]


# ---- the transposed product W^T.Y (oracle.spmm_t) ------------------------
@pytest.mark.parametrize("b", [1, 2, 4, 8])
def test_transposed_matches_dense_transpose(b):
    """W^T.Y equals the dense W^T @ Y computed by numpy in FP64."""
    rng = np.random.default_rng(40 + b)
    m, k, n = 8 * b, 12 * b, 5
    mb, kb = m // b, k // b
    idx = rng.choice(mb * kb, size=mb * kb // 3, replace=False)
    brow, bcol = (idx // kb).astype(np.int32), (idx % kb).astype(np.int32)
    vals = rng.standard_normal((len(idx), b, b))
    Y = rng.standard_normal((m, n))
    W = np.zeros((m, k))
    for p in range(len(idx)):
        W[brow[p] * b:(brow[p] + 1) * b, bcol[p] * b:(bcol[p] + 1) * b] = vals[p]
    np.testing.assert_allclose(oracle.spmm_t(m, k, b, brow, bcol, vals, Y), W.T @ Y,
                               rtol=1e-13, atol=1e-13)


def test_transposed_is_the_adjoint():
    """<W x, y> = <x, W^T y> for the oracle's own forward and transposed
    products (a wrong transpose, row index or sign in either breaks it)."""
    rng = np.random.default_rng(7)
    b, m, k, n = 4, 32, 48, 3
    mb, kb = m // b, k // b
    idx = rng.choice(mb * kb, size=30, replace=False)
    brow, bcol = (idx // kb).astype(np.int32), (idx % kb).astype(np.int32)
    vals = rng.standard_normal((30, b, b))
    X = rng.standard_normal((k, n))
    Y = rng.standard_normal((m, n))
    lhs = np.sum(oracle.spmm(m, k, b, brow, bcol, vals, X) * Y)
    rhs = np.sum(X * oracle.spmm_t(m, k, b, brow, bcol, vals, Y))
    assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + 1)


def test_transposed_exact_integers_and_truncation():
    """Integer blocks give an exact result; a block over the bottom edge is
    truncated as in the forward product (rows >= m of W do not exist)."""
    b, m, k = 4, 6, 8                       # the second block row hangs over m = 6
    brow = np.array([0, 1], np.int32)
    bcol = np.array([1, 0], np.int32)
    vals = np.arange(2 * 16, dtype=np.float64).reshape(2, 4, 4) - 10
    Y = np.arange(6 * 2, dtype=np.float64).reshape(6, 2)
    Z = oracle.spmm_t(m, k, b, brow, bcol, vals, Y)
    Wfull = np.zeros((8, k))                # the untruncated block grid, then cut to m rows
    for p in range(2):
        Wfull[brow[p] * b:(brow[p] + 1) * b, bcol[p] * b:(bcol[p] + 1) * b] = vals[p]
    assert np.array_equal(Z, Wfull[:m].T @ Y)


# ------------------------------------------------------------- SDDMM -------
def _sddmm_case(rng, b, mb, kb, frac, n):
    idx = rng.choice(mb * kb, size=max(1, int(mb * kb * frac)), replace=False)
    brow, bcol = (idx // kb).astype(np.int32), (idx % kb).astype(np.int32)
    return brow, bcol, rng.standard_normal((mb * b, n)), rng.standard_normal((kb * b, n))


def check_sddmm_masked_dense(lib):
    """Every block equals the matching b x b window of numpy's dense dY @ X^T."""
    rng = np.random.default_rng(11)
    for b in (1, 2, 4, 8):
        mb, kb, n = 6, 5, 7
        brow, bcol, dY, X = _sddmm_case(rng, b, mb, kb, 0.4, n)
        dW = oracle.sddmm(mb * b, kb * b, b, brow, bcol, dY, X, lib=lib)
        G = dY @ X.T
        for p in range(len(brow)):
            want = G[brow[p] * b:(brow[p] + 1) * b, bcol[p] * b:(bcol[p] + 1) * b]
            np.testing.assert_allclose(dW[p], want, rtol=1e-12, atol=1e-12)


def check_sddmm_is_the_gradient(lib):
    """<dW, V> = <dY, (M . V) X> for any V on the pattern: dW is the gradient
    of <dY, Y> with respect to the stored blocks, checked through the forward
    oracle (a transposed block, a wrong row or a lost term breaks it)."""
    rng = np.random.default_rng(12)
    b, mb, kb, n = 4, 7, 9, 6
    brow, bcol, dY, X = _sddmm_case(rng, b, mb, kb, 0.3, n)
    V = rng.standard_normal((len(brow), b, b))
    dW = oracle.sddmm(mb * b, kb * b, b, brow, bcol, dY, X, lib=lib)
    lhs = float(np.sum(dW * V))
    rhs = float(np.sum(dY * oracle.spmm(mb * b, kb * b, b, brow, bcol, V, X, lib=lib)))
    assert abs(lhs - rhs) <= 1e-10 * (abs(rhs) + 1)


def check_sddmm_exact_integers_and_truncation(lib):
    """Small integers give exact sums; a block hanging over both edges keeps
    only the entries inside m x k and is zero elsewhere."""
    b, m, k, n = 4, 6, 10, 3                # block row 1 and block column 2 hang over
    brow = np.array([0, 1, 1], np.int32)
    bcol = np.array([2, 0, 2], np.int32)
    dY = (np.arange(m * n).reshape(m, n) % 7 - 3).astype(np.float64)
    X = (np.arange(k * n).reshape(k, n) % 5 - 2).astype(np.float64)
    dW = oracle.sddmm(m, k, b, brow, bcol, dY, X, lib=lib)
    G = np.zeros((8, 12))
    G[:m, :k] = dY @ X.T
    for p in range(3):
        assert np.array_equal(dW[p], G[brow[p] * b:(brow[p] + 1) * b,
                                       bcol[p] * b:(bcol[p] + 1) * b])
    assert not np.any(dW[1][2:]) and not np.any(dW[2][:, 2:])


def check_sddmm_hand_example(lib):
    """b = 2, one block at (0, 1) of a 2 x 4 W, n = 2, worked by hand:
    dY = [[1, 2], [3, 4]], X rows 2, 3 = [5, 6], [7, 8] give
    [[1*5+2*6, 1*7+2*8], [3*5+4*6, 3*7+4*8]] = [[17, 23], [39, 53]]."""
    dY = np.array([[1.0, 2.0], [3.0, 4.0]])
    X = np.array([[0.0, 0.0], [0.0, 0.0], [5.0, 6.0], [7.0, 8.0]])
    dW = oracle.sddmm(2, 4, 2, np.array([0], np.int32), np.array([1], np.int32), dY, X,
                      lib=lib)
    assert np.array_equal(dW[0], np.array([[17.0, 23.0], [39.0, 53.0]]))


SDDMM_CHECKS = [check_sddmm_masked_dense, check_sddmm_is_the_gradient,
                check_sddmm_exact_integers_and_truncation, check_sddmm_hand_example]


@pytest.mark.parametrize("check", SDDMM_CHECKS, ids=lambda f: f.__name__)
def test_sddmm_pin(check):
    check(oracle._load())


def test_sddmm_empty_and_rejects_out_of_range():
    out = oracle.sddmm(8, 8, 4, np.zeros(0, np.int32), np.zeros(0, np.int32),
                       np.ones((8, 3)), np.ones((8, 3)))
    assert out.shape == (0, 4, 4)
    with pytest.raises(ValueError):
        oracle.sddmm(8, 8, 4, np.array([0], np.int32), np.array([2], np.int32),
                     np.ones((8, 3)), np.ones((8, 3)))
