"""Seeded synthetic inputs shaped like the paper's sweeps (Section 4, Table 2).

This module draws random numbers and nothing else: it holds none of the
method's arithmetic, so both the CUDA path's tests/benchmark and the oracle
can take their inputs from it.  The paper generates "random sparsity pattern
and values" without naming a generator (Section 4); the recipe here is
numpy ``Generator(PCG64(seed))`` with draws in this order: block positions
(uniform without replacement over the block grid), then values, then X.
Values and X are N(0, 1), drawn in FP32 and rounded to the working dtype by
the caller (``torch`` round-to-nearest-even).
"""
import math

import numpy as np


def rng_for(seed):
    return np.random.Generator(np.random.PCG64(seed))


def pattern(rng, mb, kb, nnzb):
    """nnzb distinct block positions, uniform over the mb x kb block grid."""
    idx = rng.choice(mb * kb, size=nnzb, replace=False)
    return (idx // kb).astype(np.int32), (idx % kb).astype(np.int32)


def problem(seed, m, k, n, b, nnzb):
    """One SpMM problem: returns dict(m, k, n, b, brow, bcol, vals f32 (nnzb,b,b), X f32 (k,n))."""
    rng = rng_for(seed)
    brow, bcol = pattern(rng, m // b, k // b, nnzb)
    vals = rng.standard_normal((nnzb, b, b), dtype=np.float32)
    X = rng.standard_normal((k, n), dtype=np.float32)
    return dict(m=m, k=k, n=n, b=b, brow=brow, bcol=bcol, vals=vals, X=X, seed=seed)


def transposed_problem(seed, m, k, n, b, nnzb):
    """Operands of Z = W^T.Y: W's pattern and values as in problem() (W is
    m x k), then Y f32 (m, n) in place of X."""
    rng = rng_for(seed)
    brow, bcol = pattern(rng, m // b, k // b, nnzb)
    vals = rng.standard_normal((nnzb, b, b), dtype=np.float32)
    Y = rng.standard_normal((m, n), dtype=np.float32)
    return dict(m=m, k=k, n=n, b=b, brow=brow, bcol=bcol, vals=vals, Y=Y, seed=seed)


def sddmm_problem(seed, m, k, n, b, nnzb):
    """Operands of dW = (dY.X^T) on W's mask: the pattern as in problem()
    (W is m x k), then dY f32 (m, n) and X f32 (k, n)."""
    rng = rng_for(seed)
    brow, bcol = pattern(rng, m // b, k // b, nnzb)
    dY = rng.standard_normal((m, n), dtype=np.float32)
    X = rng.standard_normal((k, n), dtype=np.float32)
    return dict(m=m, k=k, n=n, b=b, brow=brow, bcol=bcol, dY=dY, X=X, seed=seed)


def to_ell(brow, bcol, mb, width=None):
    """Blocked-ELL layout of a block pattern: cols (mb, E) int32 with each
    row's block columns ascending and -1 padding, and src (mb, E) int64, the
    pattern index of each slot (-1 for padding).  E = the largest row count
    unless a larger width is given."""
    brow = np.asarray(brow, np.int64)
    bcol = np.asarray(bcol, np.int64)
    counts = np.bincount(brow, minlength=mb) if len(brow) else np.zeros(mb, np.int64)
    E = int(counts.max()) if len(brow) else 0
    E = E if width is None else int(width)
    cols = np.full((mb, E), -1, np.int32)
    src = np.full((mb, E), -1, np.int64)
    order = np.lexsort((bcol, brow))
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    for i, p in enumerate(order):
        r = brow[p]
        e = i - starts[r]
        cols[r, e] = bcol[p]
        src[r, e] = p
    return cols, src


def nnzb_for(m, k, b, d):
    """nnzb = d * (m/b) * (k/b); Section 3 defines d over the element mask,
    which for b x b blocks is the same fraction of the block grid."""
    v = d * (m // b) * (k // b)
    if abs(v - round(v)) > 1e-9:
        raise ValueError("density does not give a whole number of blocks")
    return int(round(v))


# ---- static FP32 smoke case: 256 x 256, b = 4, d = 1/8, n = 64, seed 0 -----
def smoke_case():
    return problem(0, 256, 256, 64, 4, nnzb_for(256, 256, 4, 1 / 8))


# ---- static sweep: m = k = 4096, n = 2048, b x d grid (Table 2 subset) -----
SWEEP_B = (1, 4, 8, 16)
SWEEP_D = (1 / 32, 1 / 16, 1 / 8, 1 / 4)


def sweep_seed(b, d):
    return 1000 * b + int(round(math.log2(1 / d)))


def sweep_case(b, d, m=4096, k=4096, n=2048):
    return problem(sweep_seed(b, d), m, k, n, b, nnzb_for(m, k, b, d))


# ---- dynamic: m = k = 8192, n = 1024, b = 16, d_max = 1/16 -----------------
def dynamic_call(call, m=8192, k=8192, n=1024, b=16, d_max=1 / 16):
    """Call ``call`` draws nnzb uniform in [ceil(nnzb_max / 2), nnzb_max]."""
    nmax = nnzb_for(m, k, b, d_max)
    rng = rng_for(call)
    nnzb = int(rng.integers(-(-nmax // 2), nmax, endpoint=True))
    brow, bcol = pattern(rng, m // b, k // b, nnzb)
    vals = rng.standard_normal((nnzb, b, b), dtype=np.float32)
    X = rng.standard_normal((k, n), dtype=np.float32)
    return dict(m=m, k=k, n=n, b=b, brow=brow, bcol=bcol, vals=vals, X=X,
                nnzb_max=nmax, seed=call)


# ---- batched: 48 uneven FFN-like problems -----------------------------------
def batched_spec(i, count=48):
    """Shape of problem i: W 4096 x 16384 if i even else 16384 x 4096,
    b = (8, 16)[(i >> 1) & 1], d = (1/16, 1/8)[(i >> 2) & 1],
    n = round(exp(U(0, ln 512))) clipped to [1, 512], seed 3000 + i."""
    m, k = (4096, 16384) if i % 2 == 0 else (16384, 4096)
    b = (8, 16)[(i >> 1) & 1]
    d = (1 / 16, 1 / 8)[(i >> 2) & 1]
    rng = rng_for(3000 + i)
    n = int(min(512, max(1, round(math.exp(rng.uniform(0.0, math.log(512)))))))
    return dict(m=m, k=k, b=b, d=d, n=n, seed=3000 + i, nnzb=nnzb_for(m, k, b, d))


def batched_case(i, scale_shapes=1):
    """Full inputs of batched problem i (positions, values, X), drawn after n
    from the same generator.  ``scale_shapes`` divides m and k (tests only)."""
    s = batched_spec(i)
    m, k = s["m"] // scale_shapes, s["k"] // scale_shapes
    nnzb = nnzb_for(m, k, s["b"], s["d"])
    rng = rng_for(s["seed"])
    rng.uniform(0.0, 1.0)  # the n draw
    brow, bcol = pattern(rng, m // s["b"], k // s["b"], nnzb)
    vals = rng.standard_normal((nnzb, s["b"], s["b"]), dtype=np.float32)
    X = rng.standard_normal((k, s["n"]), dtype=np.float32)
    return dict(m=m, k=k, n=s["n"], b=s["b"], brow=brow, bcol=bcol, vals=vals,
                X=X, seed=s["seed"])


# ---- serving: 12 resident weights, Poisson request stream -------------------
SERVE_SIZES = (2048, 4096, 8192)
SERVE_B = (8, 16)


def serve_weights():
    """12 weights: m = k in {2048, 4096, 8192} x b in {8, 16} x 2 seeds, d = 1/16."""
    out = []
    for mi, m in enumerate(SERVE_SIZES):
        for bi, b in enumerate(SERVE_B):
            for s in range(2):
                seed = 4100 + 10 * mi + 2 * bi + s
                rng = rng_for(seed)
                nnzb = nnzb_for(m, m, b, 1 / 16)
                brow, bcol = pattern(rng, m // b, m // b, nnzb)
                vals = rng.standard_normal((nnzb, b, b), dtype=np.float32)
                out.append(dict(m=m, k=m, b=b, brow=brow, bcol=bcol, vals=vals, seed=seed))
    return out


def serve_requests(count, rate_per_s, n_weights, seed, n_max=256):
    """Poisson arrivals at ``rate_per_s``: exponential gaps, uniform weight
    choice, n = round(exp(U(0, ln n_max))).  Returns arrays (t_arrive_s, weight, n)."""
    rng = rng_for(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps)
    w = rng.integers(0, n_weights, size=count)
    n = np.clip(np.rint(np.exp(rng.uniform(0.0, math.log(n_max), size=count))), 1, n_max)
    return t, w.astype(np.int32), n.astype(np.int64)


def request_x(seed, k, n):
    return rng_for(seed).standard_normal((k, n), dtype=np.float32)


# ---- integer-valued operands (exact-arithmetic parity cases) ----------------
def integer_problem(seed, m, k, n, b, nnzb, vals_range=(-2, 2), x_range=(-1, 1)):
    """The pattern recipe of problem(), then integer values uniform in
    ``vals_range`` and integer X uniform in ``x_range`` (inclusive), as FP32.
    Small integers are exact in every input type, and their sums of
    products are exact in FP32 accumulation."""
    rng = rng_for(seed)
    brow, bcol = pattern(rng, m // b, k // b, nnzb)
    vals = rng.integers(vals_range[0], vals_range[1], size=(nnzb, b, b),
                        endpoint=True).astype(np.float32)
    X = rng.integers(x_range[0], x_range[1], size=(k, n), endpoint=True).astype(np.float32)
    return dict(m=m, k=k, n=n, b=b, brow=brow, bcol=bcol, vals=vals, X=X, seed=seed)
