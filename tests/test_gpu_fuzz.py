"""Seeded random configurations through every entry point, against the FP64
oracle: shapes (multiples of 16 up to 1024, so tiles are ragged against the
128 / 256-row and 128-column tiles), n from 1 to 300 (ragged against 64 and
128), block size, density, dtype and the kernel the library picks.  Each
case is small enough for the oracle to finish in well under a second; the
bars are those of the targeted tests (1e-6 FP32, 4e-3 16-bit normwise,
1e-5 relative for the sampled product's FP32 output)."""
import numpy as np
import pytest

import oracle
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


def _draw(seed):
    """(m, k, n, b, nnzb, dtype) for one case."""
    rng = np.random.default_rng(seed)
    b = int(rng.choice([1, 4, 8, 16]))
    m = 16 * int(rng.integers(1, 65))
    k = 16 * int(rng.integers(1, 65))
    n = int(rng.integers(1, 301))
    grid = (m // b) * (k // b)
    d = float(rng.choice([1 / 32, 1 / 16, 1 / 8, 1 / 4, 1 / 2]))
    nnzb = max(1, min(grid, int(round(d * grid))))
    dt = [torch.float16, torch.bfloat16][int(rng.integers(0, 2))]
    return m, k, n, b, nnzb, dt


def _dev_rows(A, dt):
    rows, n = A.shape
    ld = max(((n + 7) // 8) * 8, 8)
    buf = torch.zeros((rows, ld), dtype=dt, device="cuda")
    buf[:, :n] = A.to(dt).cuda()
    return buf[:, :n]


@pytest.mark.parametrize("seed", range(24))
def test_fuzz_forward_static(seed):
    m, k, n, b, nnzb, dt = _draw(1000 + seed)
    if seed % 6 == 5:
        dt = torch.float32                      # FP32 goes to the plain kernel
    c = wl.problem(1000 + seed, m, k, n, b, nnzb)
    vals = torch.from_numpy(c["vals"]).to(dt)
    X = torch.from_numpy(c["X"]).to(dt)
    plan = S.Plan(m, k, n, b, w_dtype=S.dtype_code(dt), brow=c["brow"], bcol=c["bcol"])
    plan.pack(vals.cuda())
    Y = torch.full((m, n), float("nan"), dtype=dt, device="cuda")
    plan.run(_dev_rows(X, dt), Y)
    torch.cuda.synchronize()
    assert plan.status() == 0
    Yo = oracle.spmm(m, k, b, c["brow"], c["bcol"], vals, X)
    err = oracle.normwise_err(Y.cpu(), Yo, oracle.block_fro(vals), X)
    assert err <= TOL[dt], (m, k, n, b, nnzb, dt, err)


@pytest.mark.parametrize("seed", range(10))
def test_fuzz_transposed(seed):
    m, k, n, b, nnzb, dt = _draw(2000 + seed)
    c = wl.transposed_problem(2000 + seed, m, k, n, b, nnzb)
    vals = torch.from_numpy(c["vals"]).to(dt)
    Y = torch.from_numpy(c["Y"]).to(dt)
    plan = S.Plan(m, k, n, b, w_dtype=S.dtype_code(dt), brow=c["brow"], bcol=c["bcol"],
                  transposed=True)
    plan.pack(vals.cuda())
    Z = plan.run(_dev_rows(Y, dt))
    torch.cuda.synchronize()
    assert plan.status() == 0
    Zo = oracle.spmm_t(m, k, b, c["brow"], c["bcol"], vals, Y)
    err = oracle.normwise_err(Z.cpu(), Zo, oracle.block_fro(vals), Y)
    assert err <= TOL[dt], (m, k, n, b, nnzb, dt, err)


@pytest.mark.parametrize("seed", range(12))
def test_fuzz_sddmm(seed):
    m, k, n, b, nnzb, dt = _draw(3000 + seed)
    c = wl.sddmm_problem(3000 + seed, m, k, n, b, nnzb)
    dY = torch.from_numpy(c["dY"]).to(dt)
    X = torch.from_numpy(c["X"]).to(dt)
    plan = S.Plan(m, k, n, b, w_dtype=S.dtype_code(dt), brow=c["brow"], bcol=c["bcol"])
    dW = plan.sddmm(_dev_rows(dY, dt), _dev_rows(X, dt))
    torch.cuda.synchronize()
    assert plan.status() == 0
    dWo = oracle.sddmm(m, k, b, c["brow"], c["bcol"], dY, X)
    got = dW.cpu().double().numpy()
    assert np.linalg.norm(got - dWo) <= 1e-5 * max(np.linalg.norm(dWo), 1e-30), \
        (m, k, n, b, nnzb, plan.info()["sddmm_form"])


def _dev_pattern(brow, bcol, cap):
    br = torch.zeros(cap, dtype=torch.int32)
    bc = torch.zeros(cap, dtype=torch.int32)
    br[:len(brow)] = torch.from_numpy(np.asarray(brow, np.int32))
    bc[:len(bcol)] = torch.from_numpy(np.asarray(bcol, np.int32))
    return (torch.tensor([len(brow)], dtype=torch.int32, device="cuda"), br.cuda(), bc.cuda())


@pytest.mark.parametrize("seed", range(6))
def test_fuzz_dynamic(seed):
    """One dynamic plan, three calls with nnzb drawn in [0, nnzb_max]."""
    m, k, n, b, nnzb, dt = _draw(4000 + seed)
    cap = nnzb
    plan = S.Plan(m, k, n, b, w_dtype=S.dtype_code(dt), mode=S.DYNAMIC, nnzb_max=cap)
    rng = np.random.default_rng(4000 + seed)
    for call in range(3):
        nz = int(rng.integers(0, cap + 1))
        c = wl.problem(4100 + 10 * seed + call, m, k, n, b, nz)
        vals = torch.from_numpy(c["vals"]).to(dt)
        X = torch.from_numpy(c["X"]).to(dt)
        vd = torch.zeros((cap, b, b), dtype=dt)
        vd[:nz] = vals
        Y = plan.run(_dev_rows(X, dt), values=vd.cuda(),
                     pattern=_dev_pattern(c["brow"], c["bcol"], cap))
        torch.cuda.synchronize()
        assert plan.status() == 0
        Yo = oracle.spmm(m, k, b, c["brow"], c["bcol"], vals, X)
        err = oracle.normwise_err(Y.cpu(), Yo, oracle.block_fro(vals), X)
        assert err <= TOL[dt], (m, k, n, b, nz, dt, err)


@pytest.mark.parametrize("seed", range(8))
def test_fuzz_ell(seed):
    m, k, n, _, _, dt = _draw(5000 + seed)
    b = 16
    grid = (m // b) * (k // b)
    nnzb = max(1, grid // int(np.random.default_rng(seed).choice([2, 4, 8, 16])))
    c = wl.problem(5000 + seed, m, k, n, b, nnzb)
    cols, src = wl.to_ell(c["brow"], c["bcol"], m // b)
    vals = torch.from_numpy(c["vals"]).to(dt)
    ev = torch.zeros((m // b, cols.shape[1], b, b), dtype=dt)
    sel = src >= 0
    ev[torch.from_numpy(sel)] = vals[torch.from_numpy(src[sel])]
    X = torch.from_numpy(c["X"]).to(dt)
    plan = S.Plan(m, k, n, b, w_dtype=S.dtype_code(dt), mode=S.DYNAMIC, nnzb_max=nnzb)
    Y = plan.run_ell(torch.from_numpy(cols).cuda(), ev.cuda(), _dev_rows(X, dt))
    torch.cuda.synchronize()
    assert plan.status() == 0
    Yo = oracle.spmm(m, k, b, c["brow"], c["bcol"], vals, X)
    err = oracle.normwise_err(Y.cpu(), Yo, oracle.block_fro(vals), X)
    assert err <= TOL[dt], (m, k, n, nnzb, dt, err)
