"""GPU parity of the sampled product dW = (dY.X^T) on the block mask (the
gradient of Section 3's product with respect to the stored blocks) against
the FP64 oracle's ``sddmm``.

Blocks of 16 below a density of 1/13 take the gathered kernel, every other
case the dense-tile kernel; the cases below cover both.

Bars: FP32 output within 1e-5 of the oracle relative to ||dW_o||_F (16-bit
inputs are exact in FP32 products; only the FP32 accumulation order
differs), 16-bit output within 4e-3 normwise (||dW - dW_o||_F /
(||dY||_F ||X||_F), one rounding of each output); small-integer inputs with
FP32 output bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_2303_16999_gb300 import spmm as S
from paper_2303_16999_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2303_16999_gb300 import build
    build.build()


def _dev_rows(A, dt):
    """A (rows x n) on the device with the leading dimension padded to 8."""
    rows, n = A.shape
    ld = max(((n + 7) // 8) * 8, 8)
    buf = torch.zeros((rows, ld), dtype=dt, device="cuda")
    buf[:, :n] = A.to(dt).cuda()
    return buf[:, :n]


def _check(dW, dWo, dY, X, out_dt):
    dW = oracle.to_f64(dW.cpu())
    assert not np.isnan(dW).any()
    if out_dt == torch.float32:
        den = float(np.linalg.norm(dWo))
        assert float(np.linalg.norm(dW - dWo)) <= 1e-5 * max(den, 1e-30)
    else:
        assert oracle.normwise_err(dW, dWo, float(np.linalg.norm(oracle.to_f64(dY))), X) <= 4e-3


def run_case(m, k, n, b, d, dt, out_dt, seed):
    c = wl.sddmm_problem(seed, m, k, n, b, wl.nnzb_for(m, k, b, d))
    dY = torch.from_numpy(c["dY"]).to(dt)
    X = torch.from_numpy(c["X"]).to(dt)
    plan = S.Plan(m, k, max(n, 1), b, w_dtype=S.dtype_code(dt), brow=c["brow"], bcol=c["bcol"])
    assert plan.info()["sddmm_form"] == (1 if b == 16 and d * 13 < 1 else 0)
    dW = torch.full((len(c["brow"]), b, b), float("nan"), dtype=out_dt, device="cuda")
    plan.sddmm(_dev_rows(dY, dt), _dev_rows(X, dt), dW)
    torch.cuda.synchronize()
    assert plan.status() == 0
    dWo = oracle.sddmm(m, k, b, c["brow"], c["bcol"], dY, X)
    return dW, dWo, dY, X


CASES = [
    # m, k, n, b, density: ragged m (not a multiple of 128), k (of 256) and n (of 64)
    (256, 512, 200, 16, 1 / 4),
    (384, 640, 130, 8, 1 / 8),
    (208, 304, 64, 4, 1 / 8),
    (520, 700, 33, 1, 1 / 16),
    (2048, 4096, 64, 16, 1 / 16),    # 256 tiles: CTAs span several rows of tiles
    (256, 256, 1000, 8, 1 / 4),      # 16 steps along n
    (512, 512, 130, 16, 1 / 4),      # b = 16 above density 1/13: dense tiles
    (1024, 768, 200, 16, 1 / 16),    # b = 16 below it: gathered blocks, rows of 1 to 8+ blocks
]


@pytest.mark.parametrize("out", ["f32", "x"])
@pytest.mark.parametrize("dt", [torch.float16, torch.bfloat16])
@pytest.mark.parametrize("case", CASES)
def test_sddmm_parity(case, dt, out):
    m, k, n, b, d = case
    out_dt = torch.float32 if out == "f32" else dt
    dW, dWo, dY, X = run_case(m, k, n, b, d, dt, out_dt, seed=m + k + n + b)
    _check(dW, dWo, dY, X, out_dt)


@pytest.mark.parametrize("d", [1 / 16, 1 / 4])
@pytest.mark.parametrize("n", [1, 7, 8])
def test_sddmm_small_n(n, d):
    dW, dWo, dY, X = run_case(256, 384, n, 16, d, torch.bfloat16, torch.float32, seed=3 + n)
    _check(dW, dWo, dY, X, torch.float32)


@pytest.mark.parametrize("b,nnzb,form", [(16, 16, 1), (16, 64, 0), (4, 64, 0)])
def test_sddmm_n_zero_writes_zero_blocks(b, nnzb, form):
    c = wl.sddmm_problem(5, 256, 256, 8, b, nnzb)
    plan = S.Plan(256, 256, 8, b, w_dtype=S.F16, brow=c["brow"], bcol=c["bcol"])
    assert plan.info()["sddmm_form"] == form
    dY = torch.zeros((256, 8), dtype=torch.float16, device="cuda")[:, :0]
    dW = torch.full((nnzb, b, b), 7.0, dtype=torch.float32, device="cuda")
    plan.sddmm(dY, dY, dW)
    torch.cuda.synchronize()
    assert plan.status() == 0 and not torch.any(dW)


@pytest.mark.parametrize("b", [16, 8, 4, 1])
def test_sddmm_integers_bit_exact(b):
    """Small integers: products and sums are exact in FP32, so dW equals the
    oracle's value exactly."""
    m, k, n = 256, 512, 136
    c = wl.sddmm_problem(60 + b, m, k, n, b, wl.nnzb_for(m, k, b, 1 / 8))
    dY = torch.from_numpy(np.rint(c["dY"] * 2).clip(-4, 4)).half()
    X = torch.from_numpy(np.rint(c["X"] * 2).clip(-4, 4)).half()
    plan = S.Plan(m, k, n, b, w_dtype=S.F16, brow=c["brow"], bcol=c["bcol"])
    dW = plan.sddmm(_dev_rows(dY, torch.float16), _dev_rows(X, torch.float16))
    torch.cuda.synchronize()
    assert plan.status() == 0
    dWo = oracle.sddmm(m, k, b, c["brow"], c["bcol"], dY, X)
    assert np.array_equal(dW.cpu().double().numpy(), dWo)


def _dev_pattern(brow, bcol, cap, nnzb=None):
    n = len(brow) if nnzb is None else nnzb
    br = torch.zeros(cap, dtype=torch.int32)
    bc = torch.zeros(cap, dtype=torch.int32)
    br[:len(brow)] = torch.from_numpy(np.asarray(brow, np.int32))
    bc[:len(bcol)] = torch.from_numpy(np.asarray(bcol, np.int32))
    return (torch.tensor([n], dtype=torch.int32, device="cuda"), br.cuda(), bc.cuda())


@pytest.mark.parametrize("b", [16, 1])
def test_sddmm_dynamic_calls(b):
    """A fresh pattern every call through one dynamic plan (the step of
    dynamic sparse training); the forward product runs on the same plan in
    between, so the two share the rebuilt block CSR correctly."""
    m, k, n = 512, 768, 96
    cap = wl.nnzb_for(m, k, b, 1 / 16)
    plan = S.Plan(m, k, n, b, w_dtype=S.BF16, mode=S.DYNAMIC, nnzb_max=cap)
    for call in range(3):
        nnz = cap - 11 * call
        c = wl.sddmm_problem(200 + 10 * b + call, m, k, n, b, nnz)
        dY = torch.from_numpy(c["dY"]).bfloat16()
        X = torch.from_numpy(c["X"]).bfloat16()
        pat = _dev_pattern(c["brow"], c["bcol"], cap)
        vd = torch.zeros((cap, b, b), dtype=torch.bfloat16, device="cuda")
        plan.run(_dev_rows(X, torch.bfloat16), values=vd, pattern=pat)
        dW = plan.sddmm(_dev_rows(dY, torch.bfloat16), _dev_rows(X, torch.bfloat16), pattern=pat)
        torch.cuda.synchronize()
        assert plan.status() == 0
        dWo = oracle.sddmm(m, k, b, c["brow"], c["bcol"], dY, X)
        _check(dW[:nnz], dWo, dY, X, torch.float32)


@pytest.mark.parametrize("bad", ["duplicate", "col_range", "over_capacity"])
def test_sddmm_dynamic_rejects_bad_patterns(bad):
    m = k = 256
    b, n, cap = 16, 32, 16
    brow = np.arange(6, dtype=np.int32) % (m // b)
    bcol = (np.arange(6, dtype=np.int32) * 3) % (k // b)
    nnzb = 6
    if bad == "duplicate":
        brow[4], bcol[4] = brow[1], bcol[1]
    elif bad == "col_range":
        bcol[2] = k // b
    else:
        nnzb = cap + 1
    plan = S.Plan(m, k, n, b, w_dtype=S.F16, mode=S.DYNAMIC, nnzb_max=cap)
    ones = torch.ones((m, n), dtype=torch.float16, device="cuda")
    dW = torch.full((cap, b, b), 5.0, dtype=torch.float32, device="cuda")
    plan.sddmm(ones, ones, dW, pattern=_dev_pattern(brow, bcol, cap, nnzb))
    torch.cuda.synchronize()
    want = S.ERR_CAPACITY if bad == "over_capacity" else S.ERR_PATTERN
    assert plan.status() == want
    assert torch.all(dW == 5.0), "dW must be left unwritten"


@pytest.mark.parametrize("b,d", [(16, 1 / 16), (1, 1 / 16)])
def test_sddmm_full_size_sampled(b, d):
    """m = k = 4096, n = 2048, BF16 in, FP32 out (the size the benchmark
    times): 96 sampled blocks against the oracle, which computes each block
    on its own."""
    m = k = 4096
    n = 2048
    c = wl.sddmm_problem(4343 + b, m, k, n, b, wl.nnzb_for(m, k, b, d))
    dY = torch.from_numpy(c["dY"]).bfloat16()
    X = torch.from_numpy(c["X"]).bfloat16()
    plan = S.Plan(m, k, n, b, w_dtype=S.BF16, brow=c["brow"], bcol=c["bcol"])
    dW = plan.sddmm(dY.cuda(), X.cuda())
    torch.cuda.synchronize()
    assert plan.status() == 0
    sel = np.random.default_rng(9).choice(len(c["brow"]), size=96, replace=False)
    dWo = oracle.sddmm(m, k, b, c["brow"][sel], c["bcol"][sel], dY, X)
    dWs = dW[torch.from_numpy(sel)]
    _check(dWs, dWo, dY, X, torch.float32)
    # componentwise: an FP32 sum of n products, rounded once, stays within
    # 2 (u + n 2^-24) of sum |dY| |X| for every element of every block
    A = oracle.sddmm(m, k, b, c["brow"][sel], c["bcol"][sel], np.abs(oracle.to_f64(dY)),
                     np.abs(oracle.to_f64(X)))
    assert oracle.componentwise_ratio(dWs.cpu(), dWo, A) <= 2 * (2.0 ** -24 + n * 2.0 ** -24)
