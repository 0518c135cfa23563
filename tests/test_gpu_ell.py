"""GPU parity of the Blocked-ELL product (b = 16, dynamic plans) against the
FP64 oracle: the ELL rows are the same blocks as the pattern the oracle
takes, so Y must match oracle.spmm on that pattern.  Bars as for the other
16-bit products: 4e-3 normwise, bit-exact on small integers.  Layouts that
break the ELL rules set the status word and leave Y unwritten."""
import numpy as np
import pytest

import checks
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


def _x_dev(X, dt):
    k, n = X.shape
    ld = max(((n + 7) // 8) * 8, 8)
    buf = torch.zeros((k, ld), dtype=dt, device="cuda")
    buf[:, :n] = X.to(dt).cuda()
    return buf[:, :n]


def _ell_operands(c, dt, width=None):
    mb = c["m"] // 16
    cols, src = wl.to_ell(c["brow"], c["bcol"], mb, width)
    E = cols.shape[1]
    vals = torch.from_numpy(c["vals"]).to(dt)
    ev = torch.zeros((mb, E, 16, 16), dtype=dt)
    sel = src >= 0
    ev[torch.from_numpy(sel)] = vals[torch.from_numpy(src[sel])]
    return torch.from_numpy(cols).cuda(), ev.cuda(), vals


def run_ell(m, k, n, d, dt, seed, width=None, plan=None):
    c = wl.problem(seed, m, k, n, 16, wl.nnzb_for(m, k, 16, d))
    cols, ev, vals = _ell_operands(c, dt, width)
    if plan is None:
        plan = S.Plan(m, k, max(n, 1), 16, w_dtype=S.dtype_code(dt), mode=S.DYNAMIC,
                      nnzb_max=max(1, len(c["brow"])))
    X = torch.from_numpy(c["X"]).to(dt)
    Y = torch.full((m, n), float("nan"), dtype=dt, device="cuda")
    plan.run_ell(cols, ev, _x_dev(X, dt), Y)
    torch.cuda.synchronize()
    assert plan.status() == 0
    Yo = oracle.spmm(m, k, 16, c["brow"], c["bcol"], vals, X)
    return oracle.normwise_err(Y.cpu(), Yo, oracle.block_fro(vals), X), Y


CASES = [
    # m, k, n, density (ELL width = the longest row; n ragged against 128 and 64)
    (512, 768, 200, 1 / 8),
    (1024, 512, 130, 1 / 16),
    (256, 256, 1, 1 / 4),
    (2048, 2048, 384, 1 / 16),
    (256, 8192, 64, 1 / 4),        # rows longer than 64 slots: the producer loads the rest
    (4096, 256, 256, 1 / 4),       # many short rows, some empty
]


@pytest.mark.parametrize("dt", [torch.float16, torch.bfloat16])
@pytest.mark.parametrize("case", CASES)
def test_ell_parity(case, dt):
    m, k, n, d = case
    err, Y = run_ell(m, k, n, d, dt, seed=m + k + n)
    assert not torch.isnan(Y).any()
    assert err <= 4e-3, err


def test_ell_wider_than_rows_and_width_zero():
    err, _ = run_ell(512, 512, 96, 1 / 16, torch.bfloat16, seed=8, width=32)
    assert err <= 4e-3
    plan = S.Plan(256, 256, 64, 16, w_dtype=S.F16, mode=S.DYNAMIC, nnzb_max=16)
    Y = torch.full((256, 64), 3.0, dtype=torch.float16, device="cuda")
    plan.run_ell(torch.zeros((16, 0), dtype=torch.int32, device="cuda"),
                 torch.zeros((16, 0, 16, 16), dtype=torch.float16, device="cuda"),
                 torch.ones((256, 64), dtype=torch.float16, device="cuda"), Y)
    torch.cuda.synchronize()
    assert plan.status() == 0 and not torch.any(Y)


def test_ell_integers_bit_exact():
    m, k, n = 512, 1024, 136
    c = wl.problem(31, m, k, n, 16, wl.nnzb_for(m, k, 16, 1 / 8))
    c["vals"] = np.rint(c["vals"] * 2).clip(-4, 4).astype(np.float32)
    c["X"] = np.rint(c["X"] * 2).clip(-4, 4).astype(np.float32)
    cols, ev, vals = _ell_operands(c, torch.float16)
    plan = S.Plan(m, k, n, 16, w_dtype=S.F16, mode=S.DYNAMIC, nnzb_max=len(c["brow"]))
    X = torch.from_numpy(c["X"]).half()
    Y = plan.run_ell(cols, ev, _x_dev(X, torch.float16))
    torch.cuda.synchronize()
    assert plan.status() == 0
    Yo = oracle.spmm(m, k, 16, c["brow"], c["bcol"], vals, X)
    assert torch.equal(Y.cpu(), torch.from_numpy(Yo).half())


@pytest.mark.parametrize("bad", ["unsorted", "col_range", "pad_before_block", "negative"])
def test_ell_rejects_bad_layouts(bad):
    m = k = 256
    n = 32
    cols = np.full((16, 4), -1, np.int32)
    cols[:, 0] = np.arange(16) % 16
    cols[:, 1] = (np.arange(16) + 3) % 16
    cols[:, :2].sort(axis=1)
    if bad == "unsorted":
        cols[5, :2] = cols[5, 1::-1]
    elif bad == "col_range":
        cols[7, 1] = 16
    elif bad == "pad_before_block":
        cols[9, 2] = -1
        cols[9, 3] = 15
    else:
        cols[2, 0] = -5
    plan = S.Plan(m, k, n, 16, w_dtype=S.F16, mode=S.DYNAMIC, nnzb_max=64)
    Y = torch.full((m, n), 5.0, dtype=torch.float16, device="cuda")
    plan.run_ell(torch.from_numpy(cols).cuda(),
                 torch.ones((16, 4, 16, 16), dtype=torch.float16, device="cuda"),
                 torch.ones((k, n), dtype=torch.float16, device="cuda"), Y)
    torch.cuda.synchronize()
    assert plan.status() == S.ERR_PATTERN
    assert torch.all(Y == 5.0), "Y must be left unwritten"
    # the next calls' validation writes their status itself: a rejected call
    # left unread, then a valid one, reads back 0 and a full Y
    plan.run_ell(torch.from_numpy(cols).cuda(),
                 torch.ones((16, 4, 16, 16), dtype=torch.float16, device="cuda"),
                 torch.ones((k, n), dtype=torch.float16, device="cuda"), Y)
    good = np.full((16, 4), -1, np.int32)
    good[:, 0] = np.arange(16) % 16
    good[:, 1] = (np.arange(16) + 3) % 16
    good[:, :2].sort(axis=1)
    Y2 = plan.run_ell(torch.from_numpy(good).cuda(),
                      torch.ones((16, 4, 16, 16), dtype=torch.float16, device="cuda"),
                      torch.ones((k, n), dtype=torch.float16, device="cuda"))
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert torch.all(Y2 == 32.0)   # two all-ones blocks per block row, 16 terms each


def test_ell_and_csr_calls_share_a_plan():
    """The same dynamic plan serves CSR-pattern calls (device re-partition)
    and ELL calls in turn; each matches the oracle."""
    m = k = 1024
    n = 128
    cap = wl.nnzb_for(m, k, 16, 1 / 16)
    plan = S.Plan(m, k, n, 16, w_dtype=S.BF16, mode=S.DYNAMIC, nnzb_max=cap)
    for call in range(2):
        c = wl.dynamic_call(call, m=m, k=k, n=n, b=16, d_max=1 / 16)
        vals = torch.from_numpy(c["vals"]).bfloat16()
        X = torch.from_numpy(c["X"]).bfloat16()
        Yo = oracle.spmm(m, k, 16, c["brow"], c["bcol"], vals, X)
        nnz = len(c["brow"])
        br = torch.zeros(cap, dtype=torch.int32)
        bc = torch.zeros(cap, dtype=torch.int32)
        br[:nnz] = torch.from_numpy(c["brow"])
        bc[:nnz] = torch.from_numpy(c["bcol"])
        vd = torch.zeros((cap, 16, 16), dtype=torch.bfloat16)
        vd[:nnz] = vals
        pat = (torch.tensor([nnz], dtype=torch.int32, device="cuda"), br.cuda(), bc.cuda())
        Y1 = plan.run(X.cuda(), values=vd.cuda(), pattern=pat)
        cols, ev, _ = _ell_operands(c, torch.bfloat16)
        Y2 = plan.run_ell(cols, ev, X.cuda())
        torch.cuda.synchronize()
        assert plan.status() == 0
        for Y in (Y1, Y2):
            assert oracle.normwise_err(Y.cpu(), Yo, oracle.block_fro(vals), X) <= 4e-3


def test_ell_full_size_sampled():
    """m = k = 8192, n = 1024, d = 1/16, BF16 (the dynamic benchmark's size):
    sampled block rows against the oracle."""
    m = k = 8192
    n = 1024
    c = wl.dynamic_call(0)
    cols, ev, vals = _ell_operands(c, torch.bfloat16)
    plan = S.Plan(m, k, n, 16, w_dtype=S.BF16, mode=S.DYNAMIC, nnzb_max=16384)
    X = torch.from_numpy(c["X"]).bfloat16()
    Y = plan.run_ell(cols, ev, X.cuda())
    torch.cuda.synchronize()
    assert plan.status() == 0
    rows = [0, 77, 128, 255, 300, 411, 510, 511]
    checks.check_rows(Y.cpu(), rows, m, k, 16, c["brow"], c["bcol"], vals, X, torch.bfloat16)
