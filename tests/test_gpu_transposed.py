"""GPU parity of the transposed product Z = W^T.Y (W's pattern and values as
given for Y = W.X; Section 3's operands with the roles of rows and columns
exchanged) against the FP64 oracle's ``spmm_t``.

A transposed plan is the plan of W^T: the pattern is swapped on the host, the
values are transposed block by block while packing, and a dynamic call's
pattern is swapped on the device before the re-partition.  Every kernel
(tensor-core, gather, plain) and both modes run through it here.  Bars as for
Y = W.X: 1e-6 normwise for FP32, 4e-3 for FP16 / BF16 / E4M3 weights with FP32
accumulation, bit-exact on integer-valued inputs.
"""
import numpy as np
import pytest

import checks
import oracle
from oracle import plan as P
from paper_2303_16999_gb300 import spmm as S
from paper_2303_16999_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {torch.float32: 1e-6, torch.float16: 4e-3, torch.bfloat16: 4e-3}


@pytest.fixture(scope="module", autouse=True)
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2303_16999_gb300 import build
    build.build()


def _y_dev(Y, dt):
    """Y on the device with a leading dimension padded to 8 elements."""
    m, n = Y.shape
    ld = max(((n + 7) // 8) * 8, 8)
    buf = torch.zeros((m, ld), dtype=dt, device="cuda")
    buf[:, :n] = Y.to(dt).cuda()
    return buf[:, :n]


def run_t(m, k, n, b, d, dt, kernel, seed, **kw):
    c = wl.transposed_problem(seed, m, k, n, b, wl.nnzb_for(m, k, b, d))
    vals = torch.from_numpy(c["vals"]).to(dt)
    Y = torch.from_numpy(c["Y"]).to(dt)
    plan = S.Plan(m, k, max(n, 1), b, w_dtype=S.dtype_code(dt), brow=c["brow"],
                  bcol=c["bcol"], kernel=kernel, transposed=True, **kw)
    assert (plan.m, plan.k) == (k, m)
    plan.pack(vals.cuda())
    Z = torch.full((k, n), float("nan"), dtype=dt, device="cuda")
    plan.run(_y_dev(Y, dt), Z)
    torch.cuda.synchronize()
    assert plan.status() == 0
    Zo = oracle.spmm_t(m, k, b, c["brow"], c["bcol"], vals, Y)
    return oracle.normwise_err(Z.cpu(), Zo, oracle.block_fro(vals), Y), Z, Zo, c


TC_CASES = [
    # m, k, n, b, density: m != k throughout so a swapped shape would show
    (512, 384, 200, 16, 1 / 4),
    (384, 512, 130, 8, 1 / 8),
    (256, 512, 1, 16, 1 / 4),
    (512, 256, 257, 4, 1 / 32),
    (2048, 1024, 384, 16, 1 / 16),
    (512, 768, 200, 1, 1 / 8),
]


@pytest.mark.parametrize("dt", [torch.float16, torch.bfloat16])
@pytest.mark.parametrize("case", TC_CASES)
def test_tc_transposed_parity(case, dt):
    m, k, n, b, d = case
    err, Z, _, _ = run_t(m, k, n, b, d, dt, "tc", seed=m + 3 * n + b)
    assert not torch.isnan(Z).any()
    assert err <= TOL[dt], err


@pytest.mark.parametrize("b", [1, 4, 8, 16])
def test_plain_transposed_parity(b):
    m, k = 48 * b, 20 * b
    err, Z, _, _ = run_t(m, k, 37, b, 1 / 4, torch.float32, "plain", seed=5 + b)
    assert not torch.isnan(Z).any()
    assert err <= TOL[torch.float32], err


@pytest.mark.parametrize("dt", [torch.float32, torch.float16, torch.bfloat16])
@pytest.mark.parametrize("n", [1, 2, 4, 8, 33])
def test_gather_transposed_parity(n, dt):
    err, Z, _, _ = run_t(600, 344, n, 1, 1 / 8, dt, "gather", seed=40 + n)
    assert not torch.isnan(Z).any()
    assert err <= TOL[dt], err


@pytest.mark.parametrize("b,kernel", [(16, "tc"), (8, "tc"), (4, "tc"), (1, "tc"),
                                      (1, "gather"), (4, "plain")])
def test_transposed_integers_bit_exact(b, kernel):
    """Small integers: every product and partial sum is exact in FP32, so Z
    is the oracle's value rounded once to the output type."""
    m, k, n = 256, 128, 72
    dt = torch.float32 if kernel == "plain" else torch.float16
    c = wl.transposed_problem(77 + b, m, k, n, b, wl.nnzb_for(m, k, b, 1 / 4))
    vals = torch.from_numpy(np.rint(c["vals"] * 2).clip(-4, 4)).to(dt)
    Y = torch.from_numpy(np.rint(c["Y"] * 2).clip(-4, 4)).to(dt)
    plan = S.Plan(m, k, n, b, w_dtype=S.dtype_code(dt), brow=c["brow"], bcol=c["bcol"],
                  kernel=kernel, transposed=True)
    plan.pack(vals.cuda())
    Z = plan.run(_y_dev(Y, dt))
    torch.cuda.synchronize()
    assert plan.status() == 0
    Zo = oracle.spmm_t(m, k, b, c["brow"], c["bcol"], vals, Y)
    assert torch.equal(Z.cpu(), torch.from_numpy(Zo).to(dt))


@pytest.mark.parametrize("b,d,n", [(16, 1 / 8, 200), (8, 1 / 16, 64), (4, 1 / 16, 9)])
def test_e4m3_transposed_parity(b, d, n):
    """E4M3 codes with one scale per block: the scale is a property of the
    block, so it moves with the block; the codes are transposed in packing."""
    m, k = 1024, 512
    c = wl.transposed_problem(90 + b, m, k, n, b, wl.nnzb_for(m, k, b, d))
    xdt = torch.bfloat16
    codes, scales = S.quantize_e4m3(torch.from_numpy(c["vals"]).to(xdt).cuda())
    plan = S.Plan(m, k, n, b, w_dtype=S.E4M3, x_dtype=S.dtype_code(xdt), brow=c["brow"],
                  bcol=c["bcol"], transposed=True)
    plan.pack(codes.view(torch.uint8), scales)
    Y = torch.from_numpy(c["Y"]).to(xdt)
    Z = plan.run(_y_dev(Y, xdt))
    torch.cuda.synchronize()
    assert plan.status() == 0
    v = oracle.e4m3_block_values(codes.cpu().view(torch.uint8).numpy(), scales.cpu().numpy())
    Zo = oracle.spmm_t(m, k, b, c["brow"], c["bcol"], v, Y)
    assert oracle.normwise_err(Z.cpu(), Zo, oracle.block_fro(v), Y) <= 4e-3


def _dev_pattern(brow, bcol, cap, nnzb=None):
    n = len(brow) if nnzb is None else nnzb
    br = torch.zeros(cap, dtype=torch.int32)
    bc = torch.zeros(cap, dtype=torch.int32)
    br[:len(brow)] = torch.from_numpy(np.asarray(brow, np.int32))
    bc[:len(bcol)] = torch.from_numpy(np.asarray(bcol, np.int32))
    return (torch.tensor([n], dtype=torch.int32, device="cuda"), br.cuda(), bc.cuda())


@pytest.mark.parametrize("b,dt", [(16, torch.bfloat16), (8, torch.float16), (1, torch.float16)])
def test_dynamic_transposed_calls(b, dt):
    """Three calls with fresh patterns through one transposed dynamic plan;
    the device-built CSR is that of W^T (the oracle's CSR of the swapped
    pattern), bit for bit."""
    m, k, n = (1024, 512, 136) if b > 1 else (512, 256, 136)
    cap = wl.nnzb_for(m, k, b, 1 / 16)
    plan = S.Plan(m, k, n, b, w_dtype=S.dtype_code(dt), mode=S.DYNAMIC, nnzb_max=cap,
                  transposed=True)
    for call in range(3):
        nnz = cap - 7 * call
        c = wl.transposed_problem(300 + 10 * b + call, m, k, n, b, nnz)
        vals = torch.from_numpy(c["vals"]).to(dt)
        Y = torch.from_numpy(c["Y"]).to(dt)
        vd = torch.zeros((cap, b, b), dtype=dt)
        vd[:nnz] = vals
        Z = plan.run(Y.cuda(), values=vd.cuda(), pattern=_dev_pattern(c["brow"], c["bcol"], cap))
        torch.cuda.synchronize()
        assert plan.status() == 0
        Zo = oracle.spmm_t(m, k, b, c["brow"], c["bcol"], vals, Y)
        assert oracle.normwise_err(Z.cpu(), Zo, oracle.block_fro(vals), Y) <= 4e-3
        rp, ci, pm = P.csr(k // b, c["bcol"], c["brow"])
        assert np.array_equal(plan.array("row_ptr"), rp)
        assert np.array_equal(plan.array("col_idx"), ci)
        assert np.array_equal(plan.array("perm"), pm)


def test_dynamic_transposed_rejects_column_out_of_range():
    """A column index >= k/b is a row index out of range of W^T: the call sets
    the status word and leaves Z unwritten."""
    m, k, b, n, cap = 256, 128, 16, 32, 16
    brow = np.arange(4, dtype=np.int32)
    bcol = np.array([0, 1, k // b, 2], np.int32)
    plan = S.Plan(m, k, n, b, w_dtype=S.F16, mode=S.DYNAMIC, nnzb_max=cap, transposed=True)
    Z = torch.full((k, n), 5.0, dtype=torch.float16, device="cuda")
    vals = torch.ones((cap, b, b), dtype=torch.float16, device="cuda")
    plan.run(torch.ones((m, n), dtype=torch.float16, device="cuda"), Z, values=vals,
             pattern=_dev_pattern(brow, bcol, cap))
    torch.cuda.synchronize()
    assert plan.status() == S.ERR_PATTERN
    assert torch.all(Z == 5.0)


def test_transposed_full_size_sampled():
    """m = k = 4096, n = 2048, b = 16, d = 1/16, BF16 (the size the benchmark
    times): sampled columns of Z against the oracle (columns of Z = W^T.Y
    depend only on the same columns of Y)."""
    m = k = 4096
    n, b, dt = 2048, 16, torch.bfloat16
    c = wl.transposed_problem(4242, m, k, n, b, wl.nnzb_for(m, k, b, 1 / 16))
    vals = torch.from_numpy(c["vals"]).to(dt)
    Y = torch.from_numpy(c["Y"]).to(dt)
    plan = S.Plan(m, k, n, b, w_dtype=S.BF16, brow=c["brow"], bcol=c["bcol"], transposed=True)
    plan.pack(vals.cuda())
    Z = plan.run(Y.cuda())
    torch.cuda.synchronize()
    assert plan.status() == 0
    cols = [0, 1, 63, 64, 127, 128, 1000, 1535, 2046, 2047]
    Zo = oracle.spmm_t(m, k, b, c["brow"], c["bcol"], vals, Y[:, cols])
    A = oracle.spmm_t(m, k, b, c["brow"], c["bcol"], np.abs(oracle.to_f64(vals)),
                      np.abs(oracle.to_f64(Y[:, cols])))
    checks.assert_parity(Z[:, cols].cpu(), Zo, oracle.block_fro(vals), Y[:, cols], A, dt,
                         checks.max_terms(c["bcol"], b))
