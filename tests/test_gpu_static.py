"""GPU parity of the static path through the C ABI against the FP64 oracle.

Bars (normwise ||Y - Y_o||_F / (||W||_F ||X||_F)): 1e-6 for FP32, 4e-3 for
FP16 / BF16 inputs with FP32 accumulation.  Integer-valued inputs are exact
in FP32 accumulation, so there the output must equal the oracle's value
rounded once to the output type, bit for bit.
"""
import numpy as np
import pytest

import checks
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
    return torch.device("cuda:0")


def _x_dev(X, dt, ld=None):
    """X on the device, optionally with leading dimension ld > n."""
    k, n = X.shape
    if ld is None or ld == n:
        return X.to(dt).cuda()
    buf = torch.zeros((k, ld), dtype=dt, device="cuda")
    buf[:, :n] = X.to(dt).cuda()
    return buf[:, :n]


def run_case(m, k, n, b, nnzb, dt, kernel, seed, ldx=None, **kw):
    c = wl.problem(seed, m, k, n, b, nnzb)
    vals = torch.from_numpy(c["vals"]).to(dt)
    X = torch.from_numpy(c["X"]).to(dt)
    plan = S.Plan(m, k, max(n, 1), b, w_dtype=S.dtype_code(dt), brow=c["brow"], bcol=c["bcol"],
                  kernel=kernel, **kw)
    plan.pack(vals.cuda())
    Xd = _x_dev(X, dt, ldx)
    Y = torch.full((m, n), float("nan"), dtype=dt, device="cuda")
    plan.run(Xd, Y)
    torch.cuda.synchronize()
    assert plan.status() == 0
    Yo = oracle.spmm(m, k, b, c["brow"], c["bcol"], vals, X)
    err = oracle.normwise_err(Y.cpu(), Yo, oracle.block_fro(vals), X)
    return err, Y, Yo, plan


CASES = [
    # m, k, n, b, density
    (256, 256, 64, 4, 1 / 8),
    (512, 384, 200, 16, 1 / 4),
    (384, 512, 130, 8, 1 / 8),
    (256, 256, 1, 16, 1 / 4),
    (512, 512, 257, 4, 1 / 32),
    (2048, 1024, 384, 16, 1 / 16),
    (512, 768, 200, 1, 1 / 8),
    (256, 512, 33, 1, 1 / 32),
]


@pytest.mark.parametrize("dt", [torch.float16, torch.bfloat16])
@pytest.mark.parametrize("case", CASES)
def test_tc_parity(case, dt):
    m, k, n, b, d = case
    err, Y, _, _ = run_case(m, k, n, b, wl.nnzb_for(m, k, b, d), dt, "tc", seed=m + n + b,
                            ldx=((n + 7) // 8) * 8)
    assert not torch.isnan(Y).any()
    assert err <= TOL[dt], err


@pytest.mark.parametrize("dt", [torch.float32, torch.float16, torch.bfloat16])
@pytest.mark.parametrize("n", [1, 4, 16, 33, 64, 2048])
def test_gather_parity(n, dt):
    m, k = 512, 768
    err, Y, _, _ = run_case(m, k, n, 1, wl.nnzb_for(m, k, 1, 1 / 16), dt, "gather", seed=n)
    assert not torch.isnan(Y).any()
    assert err <= TOL[dt], err


@pytest.mark.parametrize("b", [1, 4, 8, 16])
def test_plain_parity(b):
    m, k, n = 256, 512, 80
    err, Y, _, _ = run_case(m, k, n, b, wl.nnzb_for(m, k, b, 1 / 8), torch.float32, "plain", seed=b)
    assert err <= 1e-6, err


def test_smoke_config_fp32():
    c = wl.smoke_case()
    vals = torch.from_numpy(c["vals"])
    X = torch.from_numpy(c["X"])
    plan = S.Plan(256, 256, 64, 4, w_dtype=S.F32, brow=c["brow"], bcol=c["bcol"])
    plan.pack(vals.cuda())
    Y = plan.run(X.cuda())
    Yo = oracle.spmm(256, 256, 4, c["brow"], c["bcol"], vals, X)
    assert oracle.normwise_err(Y.cpu(), Yo, oracle.block_fro(vals), X) <= 1e-6


def _int_case(m, k, n, b, nnzb, seed):
    rng = np.random.default_rng(seed)
    mb, kb = m // b, k // b
    idx = rng.choice(mb * kb, nnzb, replace=False)
    brow, bcol = (idx // kb).astype(np.int32), (idx % kb).astype(np.int32)
    vals = rng.integers(-3, 4, size=(nnzb, b, b)).astype(np.float32)
    X = rng.integers(-3, 4, size=(k, n)).astype(np.float32)
    return brow, bcol, vals, X


@pytest.mark.parametrize("kernel,b,dt", [("tc", 16, torch.float16), ("tc", 8, torch.bfloat16),
                                         ("tc", 4, torch.float16), ("tc", 1, torch.bfloat16),
                                         ("gather", 1, torch.float16),
                                         ("gather", 1, torch.bfloat16), ("gather", 1, torch.float32),
                                         ("plain", 4, torch.float32)])
def test_exact_integer_inputs(kernel, b, dt):
    m, k, n = 256, 512, 136
    brow, bcol, vals, X = _int_case(m, k, n, b, (m // b) * (k // b) // 4, seed=7 * b)
    plan = S.Plan(m, k, n, b, w_dtype=S.dtype_code(dt), brow=brow, bcol=bcol, kernel=kernel)
    plan.pack(torch.from_numpy(vals).to(dt).cuda())
    Y = plan.run(_x_dev(torch.from_numpy(X), dt, 136)).cpu()
    Yo = oracle.spmm(m, k, b, brow, bcol, vals, X)
    want = torch.from_numpy(Yo).to(dt)
    assert torch.equal(Y, want)


@pytest.mark.parametrize("kernel,b", [("tc", 16), ("tc", 4), ("gather", 1)])
def test_split_rows_worst_case(kernel, b):
    """Appendix A.2's worst case: every block in one block row.  The row is
    split over several work items and reduced in chunk order."""
    m, k, n = 512, 2048, 160
    kb = k // b
    nnz = min(kb, 96)
    brow = np.zeros(nnz, np.int32)
    bcol = np.arange(nnz, dtype=np.int32) * (kb // nnz)
    rng = np.random.default_rng(1)
    vals = rng.standard_normal((nnz, b, b)).astype(np.float32)
    X = rng.standard_normal((k, n)).astype(np.float32)
    dt = torch.float16
    plan = S.Plan(m, k, n, b, w_dtype=S.F16, brow=brow, bcol=bcol, kernel=kernel, max_per_item=8)
    assert plan.info()["n_reductions"] == 1
    vt = torch.from_numpy(vals).to(dt)
    plan.pack(vt.cuda())
    Y = plan.run(_x_dev(torch.from_numpy(X), dt)).cpu()
    Yo = oracle.spmm(m, k, b, brow, bcol, vt, torch.from_numpy(X).to(dt))
    err = oracle.normwise_err(Y, Yo, oracle.block_fro(vt), torch.from_numpy(X).to(dt))
    assert err <= 4e-3
    assert not torch.any(Y[b:]), "rows outside the single block row must be zero"


@pytest.mark.parametrize("kernel,b,dt", [("tc", 16, torch.float16), ("gather", 1, torch.float16),
                                         ("plain", 8, torch.float32)])
def test_empty_pattern_zero_fill(kernel, b, dt):
    m, k, n = 256, 256, 72
    plan = S.Plan(m, k, n, b, w_dtype=S.dtype_code(dt), brow=[], bcol=[], kernel=kernel)
    plan.pack(torch.zeros(1, dtype=dt, device="cuda"))
    Y = torch.full((m, n), 7.0, dtype=dt, device="cuda")
    plan.run(_x_dev(torch.ones(k, n), dt, 72), Y)
    assert not torch.any(Y.cpu())


def test_deterministic_repeat():
    m, k, n, b = 1024, 1024, 256, 16
    err, Y1, _, plan = run_case(m, k, n, b, wl.nnzb_for(m, k, b, 1 / 8), torch.float16, "tc", 3)
    c = wl.problem(3, m, k, n, b, wl.nnzb_for(m, k, b, 1 / 8))
    X = torch.from_numpy(c["X"]).half().cuda()
    for _ in range(3):
        assert torch.equal(plan.run(X), Y1)


def test_run_host_buffers():
    m, k, n, b = 512, 512, 96, 16
    c = wl.problem(9, m, k, n, b, wl.nnzb_for(m, k, b, 1 / 8))
    vals = torch.from_numpy(c["vals"]).half()
    X = torch.from_numpy(c["X"]).half().pin_memory()
    plan = S.Plan(m, k, n, b, w_dtype=S.F16, brow=c["brow"], bcol=c["bcol"])
    plan.pack(vals.cuda())
    Y = torch.empty((m, n), dtype=torch.float16).pin_memory()
    plan.run_host(X, Y)
    Yo = oracle.spmm(m, k, b, c["brow"], c["bcol"], vals, X)
    assert oracle.normwise_err(Y, Yo, oracle.block_fro(vals), X) <= 4e-3


@pytest.mark.parametrize("n", [82, 5])
def test_tc_unaligned_x_rows(n):
    """Tensor-core plans read X by TMA, which needs 16-byte aligned rows: a
    device X with ldx not a multiple of 8 is refused up front with a clear
    status, while spmm_run_host (which stages X itself, rows padded) takes
    the same X and matches the oracle."""
    m, k, b = 256, 1024, 16
    c = wl.problem(40 + n, m, k, n, b, wl.nnzb_for(m, k, b, 1 / 8))
    vals = torch.from_numpy(c["vals"]).half()
    plan = S.Plan(m, k, n, b, w_dtype=S.F16, brow=c["brow"], bcol=c["bcol"], kernel="tc")
    plan.pack(vals.cuda())
    X = torch.from_numpy(c["X"]).half()
    with pytest.raises(S.SpmmError) as e:
        plan.run(X.cuda())
    assert e.value.status == S.ERR_UNSUPPORTED and "ldx" in str(e.value)
    Y = torch.empty((m, n), dtype=torch.float16).pin_memory()
    plan.run_host(X.pin_memory(), Y)
    Yo = oracle.spmm(m, k, b, c["brow"], c["bcol"], vals, X)
    assert oracle.normwise_err(Y, Yo, oracle.block_fro(vals), X) <= 4e-3


def test_not_packed_and_bad_n():
    plan = S.Plan(256, 256, 64, 16, w_dtype=S.F16, brow=[0], bcol=[0])
    X = torch.zeros(256, 64, dtype=torch.float16, device="cuda")
    with pytest.raises(S.SpmmError) as e:
        plan.run(X)
    assert e.value.status == S.ERR_NOT_PACKED
    plan.pack(torch.zeros(256, dtype=torch.float16, device="cuda"))
    with pytest.raises(S.SpmmError) as e:
        plan.run(torch.zeros(256, 65, dtype=torch.float16, device="cuda"))
    assert e.value.status == S.ERR_SHAPE


@pytest.mark.parametrize("b", [1, 4, 8, 16])
def test_full_size_sweep_sampled(b):
    """m = k = 4096, n = 2048 FP16 at d = 1/4, in the launch configuration the
    benchmark times; 8 sampled block rows checked against the oracle with the
    normwise, relative and componentwise bars."""
    d = 1 / 4
    c = wl.sweep_case(b, d)
    dt = torch.float16
    plan = S.Plan(4096, 4096, 2048, b, w_dtype=S.F16, brow=c["brow"], bcol=c["bcol"])
    plan.pack(torch.from_numpy(c["vals"]).to(dt).cuda())
    Y = plan.run(torch.from_numpy(c["X"]).to(dt).cuda()).cpu()
    mb = 4096 // b
    rows = [0, 17, mb // 3, mb // 2, mb // 2 + 1, 2 * mb // 3 + 5, mb - 2, mb - 1]
    checks.check_rows(Y, rows, 4096, 4096, b, c["brow"], c["bcol"],
                      torch.from_numpy(c["vals"]).to(dt), torch.from_numpy(c["X"]).to(dt), dt)


@pytest.mark.parametrize("b,d", [(1, 1 / 4), (4, 1 / 16), (8, 1 / 8), (16, 1 / 4), (16, 1 / 32)])
def test_full_size_sweep_integers_exact(b, d):
    """The sweep's shape (m = k = 4096, n = 2048, FP16) with integer values in
    [-2, 2] and X in [-1, 1]: every sum is exact in FP32 and every result
    fits FP16 exactly, so Y must equal the oracle bit for bit.  Every row and
    column of Y is checked through exact identities (Y c = W X c, r^T Y =
    r^T W X), and 12 block rows element by element.  The points cover both
    stage geometries and both launch widths the benchmark uses."""
    m = k = 4096
    n = 2048
    c = wl.integer_problem(8800 + b, m, k, n, b, wl.nnzb_for(m, k, b, d))
    dt = torch.float16
    plan = S.Plan(m, k, n, b, w_dtype=S.F16, brow=c["brow"], bcol=c["bcol"])
    plan.pack(torch.from_numpy(c["vals"]).to(dt).cuda())
    Y = plan.run(torch.from_numpy(c["X"]).to(dt).cuda())
    torch.cuda.synchronize()
    assert plan.status() == 0
    Y = Y.cpu()
    checks.exact_identities(Y, m, k, b, c["brow"], c["bcol"], c["vals"], c["X"], seed=b)
    mb = m // b
    rows = sorted(set([0, 1, mb // 4, mb // 3, mb // 2, mb // 2 + 1, 2 * mb // 3, 3 * mb // 4,
                       mb - 3, mb - 2, mb - 1, 7 % mb]))
    checks.exact_rows(Y, rows, k, b, c["brow"], c["bcol"], c["vals"], c["X"], dt)


@pytest.mark.parametrize("n", [1, 4, 32])
def test_gather_large_small_n_sampled(n):
    """The configuration the benchmark's small-n gather section times:
    m = k = 16384, d = 1/16, FP16; sampled rows against the oracle (n = 4:
    X fills the five-stage ring's shared memory)."""
    m = k = 16384
    c = wl.problem(7, m, k, 32, 1, wl.nnzb_for(m, k, 1, 1 / 16))
    dt = torch.float16
    plan = S.Plan(m, k, 32, 1, w_dtype=S.F16, brow=c["brow"], bcol=c["bcol"], kernel="gather")
    plan.pack(torch.from_numpy(c["vals"].reshape(-1)).to(dt).cuda())
    Xn = torch.from_numpy(c["X"][:, :n].copy()).to(dt)
    Y = plan.run(Xn.cuda()).cpu()
    rows = [0, 4097, 9000, 12000, m - 2, m - 1]
    checks.check_rows(Y, rows, m, k, 1, c["brow"], c["bcol"],
                      torch.from_numpy(c["vals"]).to(dt), Xn, dt)


@pytest.mark.parametrize("b,d,n,geo", [(16, 1 / 32, 200, 1), (1, 1 / 4, 136, 0), (8, 1 / 4, 256, 0),
                                       (16, 1 / 16, 130, 1), (4, 1 / 8, 64, 0)])
def test_both_stage_geometries(b, d, n, geo):
    """Plans choose dense-tile or sparse-tile stages by tiles per entry (at
    least 8: dense); both geometries stay within the bound against the
    oracle.  Groups of 16 tile rows, so that entries can hold many tiles."""
    m, k = 1024, 2048
    err, Y, _, plan = run_case(m, k, n, b, wl.nnzb_for(m, k, b, d), torch.float16, "tc",
                               seed=11 * b + n, ldx=((n + 7) // 8) * 8, rows_per_group=16)
    info = plan.info()
    assert (info["n_tiles"] >= 8 * info["n_entries"]) == (geo == 0)
    assert info["stage_geometry"] == geo
    assert not torch.isnan(Y).any()
    assert err <= 4e-3, err


@pytest.mark.parametrize("b,d,n,geo", [(1, 1 / 4, 192, 0), (1, 1 / 8, 256, 0), (8, 1 / 4, 320, 0),
                                       (4, 1 / 4, 640, 0), (1, 1 / 4, 384, 0), (8, 1 / 4, 200, 0),
                                       (16, 1 / 16, 256, 1), (16, 1 / 4, 448, 1),
                                       (8, 1 / 32, 192, 1), (16, 1 / 32, 130, 1)])
@pytest.mark.parametrize("dt", [torch.float16, torch.bfloat16])
def test_two_column_tiles_per_cta(b, d, n, geo, dt):
    """Plans of either stage geometry whose CTAs cover two 128-column tiles
    of n (the two share each stage's W tiles; the second tile's slabs,
    accumulators and MMA warps are separate).  n = 192: the second tile is
    partly past n; 320, 448 and 640: the last CTA has one tile only; 200 and
    130: not multiples of 64, so X is read through a 2-D map, two 64-column
    boxes per slab (130: the second tile's upper half lies past n and is not
    fetched).  Within the bound against the oracle, and bit for bit equal to
    one tile per CTA (every accumulator column sees the same MMAs in the
    same order)."""
    m, k = 1024, 1024
    nnzb = wl.nnzb_for(m, k, b, d)
    err, Y2, _, plan = run_case(m, k, n, b, nnzb, dt, "tc", seed=5 * b + n,
                                ldx=((n + 7) // 8) * 8, rows_per_group=16, col_tiles=2)
    assert plan.info()["stage_geometry"] == geo
    assert not torch.isnan(Y2).any()
    assert err <= TOL[dt], err
    _, Y1, _, _ = run_case(m, k, n, b, nnzb, dt, "tc", seed=5 * b + n,
                           ldx=((n + 7) // 8) * 8, rows_per_group=16, col_tiles=1)
    assert torch.equal(Y1, Y2)


def test_two_column_tiles_split_rows():
    """Two column tiles per CTA with rows split across work items (partials
    through the FP32 workspace and the reduction)."""
    m, k, n, b = 512, 4096, 384, 1
    err, Y, _, plan = run_case(m, k, n, b, wl.nnzb_for(m, k, b, 1 / 4), torch.float16, "tc",
                               seed=77, rows_per_group=16, max_per_item=32, col_tiles=2)
    info = plan.info()
    assert info["stage_geometry"] == 0 and info["n_reductions"] > 0
    assert err <= 4e-3, err


def test_two_column_tiles_integers_bit_exact():
    m, k, n, b = 256, 512, 256, 1
    brow, bcol, vals, X = _int_case(m, k, n, b, (m // b) * (k // b) // 4, seed=99)
    plan = S.Plan(m, k, n, b, w_dtype=S.F16, brow=brow, bcol=bcol, kernel="tc",
                  rows_per_group=16, col_tiles=2)
    assert plan.info()["stage_geometry"] == 0
    plan.pack(torch.from_numpy(vals).half().cuda())
    Y = plan.run(torch.from_numpy(X).half().cuda()).cpu()
    Yo = oracle.spmm(m, k, b, brow, bcol, vals, X)
    assert torch.equal(Y, torch.from_numpy(Yo).half())


@pytest.mark.parametrize("b,d,n,ct", [(1, 1 / 4, 256, 2), (16, 1 / 16, 256, 0), (4, 1 / 8, 192, 2),
                                      (8, 1 / 4, 130, 0), (16, 1 / 4, 384, 2)])
def test_near_equal_groups(b, d, n, ct):
    """Tile rows in 19 near-equal groups (3 or 4 rows each here) instead of the
    planner's equal partition: within the bound against the oracle, and,
    where no row is split across items in either plan, bit for bit equal to
    the default grouping (every row of Y sums its tiles in ascending column
    order either way)."""
    m, k = 1024, 1024
    nnzb = wl.nnzb_for(m, k, b, d)
    ld = ((n + 7) // 8) * 8
    err, Yq, _, pq = run_case(m, k, n, b, nnzb, torch.float16, "tc", seed=9 * b + n, ldx=ld,
                              groups=19, col_tiles=ct)
    assert pq.info()["n_groups"] == 19 and pq.info()["rows_per_group"] == 0
    assert err <= 4e-3, err
    _, Y0, _, p0 = run_case(m, k, n, b, nnzb, torch.float16, "tc", seed=9 * b + n, ldx=ld,
                            col_tiles=ct)
    if pq.info()["n_reductions"] == 0 and p0.info()["n_reductions"] == 0:
        assert torch.equal(Yq, Y0)


@pytest.mark.parametrize("b,d,n,s", [(8, 1 / 8, 82, 19), (16, 1 / 16, 40, 7), (4, 1 / 16, 136, 3),
                                     (8, 1 / 16, 256, 38)])
def test_k_splits_integers_exact_and_bars(b, d, n, s):
    """16-row groups split along k into about s work items each (k_splits,
    the tuner's choice for tall-k problems at small n): integer inputs give
    the oracle's Y exactly (one rounding of exact sums), and N(0,1) inputs
    stay within the bars."""
    m, k = 512, 8192
    nnzb = wl.nnzb_for(m, k, b, d)
    brow, bcol, vals, X = _int_case(m, k, n, b, nnzb, seed=300 + s)
    plan = S.Plan(m, k, n, b, w_dtype=S.F16, brow=brow, bcol=bcol, kernel="tc",
                  rows_per_group=16, k_splits=s)
    info = plan.info()
    assert info["n_reductions"] == info["n_groups"] and info["n_items"] >= info["n_groups"] * (s // 2)
    plan.pack(torch.from_numpy(vals).half().cuda())
    ld = ((n + 7) // 8) * 8
    Y = plan.run(_x_dev(torch.from_numpy(X).half(), torch.float16, ld)).cpu()
    assert plan.status() == 0
    Yo = oracle.spmm(m, k, b, brow, bcol, vals, X)
    assert torch.equal(Y, torch.from_numpy(Yo).half())
    err, Yn, _, _ = run_case(m, k, n, b, nnzb, torch.bfloat16, "tc", seed=310 + s,
                             ldx=((n + 7) // 8) * 8, rows_per_group=16, k_splits=s)
    assert not torch.isnan(Yn).any()
    assert err <= 4e-3, err


@pytest.mark.parametrize("b,d,n,ct", [(16, 1 / 4, 512, 1), (1, 1 / 4, 512, 2), (8, 1 / 16, 200, 0)])
def test_device_wait_times_out_and_recovers(b, d, n, ct):
    """Failure detection on the device: with the test hook on, the MMA warps
    of every CTA wait on a barrier nothing arrives on; the wait runs out after
    its 200 us limit, the CTA records SPMM_ERR_TIMEOUT, lets its copies and
    MMAs land, frees its tensor memory and exits.  The context stays usable:
    the next call, with the default limit, is correct against the oracle.
    Covers one and two column tiles per CTA and both stage geometries."""
    m = k = 1024
    c = wl.problem(6100 + b, m, k, n, b, wl.nnzb_for(m, k, b, d))
    dt = torch.float16
    vals = torch.from_numpy(c["vals"]).to(dt)
    X = torch.from_numpy(c["X"]).to(dt)
    plan = S.Plan(m, k, n, b, w_dtype=S.F16, brow=c["brow"], bcol=c["bcol"], kernel="tc",
                  col_tiles=ct)
    plan.pack(vals.cuda())
    Xd = _x_dev(X, dt, ((n + 7) // 8) * 8)
    plan.set_wait(200_000, stall=True)
    Y = torch.zeros((m, n), dtype=dt, device="cuda")
    plan.run(Xd, Y)
    torch.cuda.synchronize()
    assert plan.status() == S.ERR_TIMEOUT
    plan.set_wait(0, stall=False)
    Y = plan.run(Xd)
    torch.cuda.synchronize()
    assert plan.status() == 0
    Yo = oracle.spmm(m, k, b, c["brow"], c["bcol"], vals, X)
    assert oracle.normwise_err(Y.cpu(), Yo, oracle.block_fro(vals), X) <= 4e-3


@pytest.mark.parametrize("dt", [torch.float16, torch.bfloat16])
@pytest.mark.parametrize("n", [1, 4, 8])
def test_gather_index_widths(n, dt):
    """The shared-memory gather reads a static plan's 16-bit copy of the
    column indices and a dynamic plan's int32 indices: on the same pattern
    (same CSR and items) both give the same Y bit for bit, within the bar
    against the oracle; k spans several 16-bit index ranges' worth of bank
    patterns (k = 3000)."""
    m, k = 640, 3000
    nnzb = wl.nnzb_for(m, k, 1, 1 / 16)
    c = wl.problem(900 + n, m, k, n, 1, nnzb)
    wd = S.dtype_code(dt)
    sp = S.Plan(m, k, n, 1, w_dtype=wd, brow=c["brow"], bcol=c["bcol"], kernel="gather")
    assert sp.info()["index_bytes"] == 2
    vals = torch.from_numpy(c["vals"].reshape(-1)).to(dt)
    sp.pack(vals.cuda())
    X = torch.from_numpy(c["X"]).to(dt).cuda()
    Ys = sp.run(X)
    dp = S.Plan(m, k, n, 1, w_dtype=wd, mode=S.DYNAMIC, nnzb_max=nnzb)
    assert dp.info()["index_bytes"] == 4
    pat = (torch.tensor([nnzb], dtype=torch.int32, device="cuda"),
           torch.from_numpy(np.asarray(c["brow"], np.int32)).cuda(),
           torch.from_numpy(np.asarray(c["bcol"], np.int32)).cuda())
    Yd = dp.run(X, values=vals.reshape(-1, 1, 1).cuda(), pattern=pat)
    torch.cuda.synchronize()
    assert dp.status() == 0
    assert torch.equal(Ys.cpu(), Yd.cpu())
    Yo = oracle.spmm(m, k, 1, c["brow"], c["bcol"], vals.reshape(-1, 1, 1), X.cpu())
    assert oracle.normwise_err(Ys.cpu(), Yo, oracle.block_fro(vals.reshape(-1, 1, 1)),
                               X.cpu()) <= TOL[dt]
