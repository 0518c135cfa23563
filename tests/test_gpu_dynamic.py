"""GPU tests of dynamic mode: the partition is rebuilt on the device every call
(Section 3.3 / Appendix A.2).  Y is compared with the FP64 oracle; every
integer array the device builds is compared bit for bit with the oracle's
dynamic-plan rules (CSR, items in (group, chunk) order, unpadded slots).
Invalid patterns must set the status word and leave Y untouched."""
import numpy as np
import pytest

import checks
import oracle
from oracle import plan as P
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


def _dev_pattern(brow, bcol, cap, nnzb=None):
    n = len(brow) if nnzb is None else nnzb
    br = torch.zeros(cap, dtype=torch.int32)
    bc = torch.zeros(cap, dtype=torch.int32)
    br[:len(brow)] = torch.from_numpy(np.asarray(brow, np.int32))
    bc[:len(bcol)] = torch.from_numpy(np.asarray(bcol, np.int32))
    return (torch.tensor([n], dtype=torch.int32, device="cuda"), br.cuda(), bc.cuda())


def _check_arrays(plan, m, k, b, brow, bcol):
    info = plan.info()
    mb = m // b
    rp, ci, pm = P.csr(mb, brow, bcol)
    assert np.array_equal(plan.array("row_ptr"), rp)
    assert np.array_equal(plan.array("col_idx"), ci)
    assert np.array_equal(plan.array("perm"), pm)
    if b == 1:
        want = P.row_plan(mb, rp, info["max_per_item"], sort_items=False)
    else:
        want = P.tc_plan(m, k, b, brow, bcol, info["rows_per_group"], info["max_per_item"],
                         sort_items=False, pad=False, groups=info["n_groups"])
        for key in ("grp_ebeg", "ent_col", "ent_tbeg", "ent_cover", "tile_row", "blk_slot",
                    "blk_off"):
            assert np.array_equal(plan.array(key), want[key]), key
    assert np.array_equal(plan.array("items").reshape(-1, 6), want["items"])
    assert np.array_equal(plan.array("ws_row0"), want["ws_row0"])
    assert np.array_equal(plan.array("red").reshape(-1, 3), want["red"])
    assert info["ws_rows"] == want["ws_rows"]


@pytest.mark.parametrize("b,dt", [(16, torch.bfloat16), (8, torch.float16), (4, torch.bfloat16),
                                  (1, torch.float16)])
def test_dynamic_calls_parity_and_plans(b, dt):
    m = k = 1024 if b > 1 else 512
    n = 136
    cap = wl.nnzb_for(m, k, b, 1 / 16)
    plan = S.Plan(m, k, n, b, w_dtype=S.dtype_code(dt), mode=S.DYNAMIC, nnzb_max=cap)
    for call in range(3):
        c = wl.dynamic_call(call + 10 * b, m=m, k=k, n=n, b=b, d_max=1 / 16)
        vals = torch.from_numpy(c["vals"]).to(dt)
        X = torch.from_numpy(c["X"]).to(dt)
        pat = _dev_pattern(c["brow"], c["bcol"], cap)
        vd = torch.zeros((cap, b, b), dtype=dt)
        vd[:len(vals)] = vals
        Y = plan.run(X.cuda(), values=vd.cuda(), pattern=pat)
        torch.cuda.synchronize()
        assert plan.status() == 0
        Yo = oracle.spmm(m, k, b, c["brow"], c["bcol"], vals, X)
        assert oracle.normwise_err(Y.cpu(), Yo, oracle.block_fro(vals), X) <= 4e-3
        _check_arrays(plan, m, k, b, c["brow"], c["bcol"])


@pytest.mark.parametrize("b", [16, 1])
def test_dynamic_worst_case_single_row(b):
    """Appendix A.2's worst case: every block in one partition.  The group
    (or row) is split into chunks and reduced."""
    m, k, n = 512, 4096, 64
    kb = k // b
    nnz = min(kb, 256)
    brow = np.zeros(nnz, np.int32)
    bcol = (np.arange(nnz) * (kb // nnz)).astype(np.int32)
    cap = nnz + 64
    dt = torch.float16
    rng = np.random.default_rng(4)
    vals = torch.from_numpy(rng.standard_normal((nnz, b, b)).astype(np.float32)).to(dt)
    X = torch.from_numpy(rng.standard_normal((k, n)).astype(np.float32)).to(dt)
    plan = S.Plan(m, k, n, b, w_dtype=S.F16, mode=S.DYNAMIC, nnzb_max=cap)
    vd = torch.zeros((cap, b, b), dtype=dt)
    vd[:nnz] = vals
    Y = plan.run(X.cuda(), values=vd.cuda(), pattern=_dev_pattern(brow, bcol, cap))
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert plan.info()["n_reductions"] == 1
    Yo = oracle.spmm(m, k, b, brow, bcol, vals, X)
    assert oracle.normwise_err(Y.cpu(), Yo, oracle.block_fro(vals), X) <= 4e-3
    _check_arrays(plan, m, k, b, brow, bcol)


@pytest.mark.parametrize("b", [16, 1])
@pytest.mark.parametrize("bad", ["duplicate", "row_range", "col_range", "over_capacity",
                                 "negative"])
def test_dynamic_rejects_bad_patterns(b, bad):
    m = k = 256
    n = 32
    cap = 64
    brow = np.arange(8, dtype=np.int32) % (m // b)
    bcol = (np.arange(8, dtype=np.int32) * 3) % (k // b)
    nnzb = 8
    if bad == "duplicate":
        brow[5], bcol[5] = brow[2], bcol[2]
    elif bad == "row_range":
        brow[3] = m // b
    elif bad == "col_range":
        bcol[7] = -1
    elif bad == "over_capacity":
        nnzb = cap + 1
    elif bad == "negative":
        nnzb = -3
    plan = S.Plan(m, k, n, b, w_dtype=S.F16, mode=S.DYNAMIC, nnzb_max=cap)
    X = torch.ones((k, n), dtype=torch.float16, device="cuda")
    Y = torch.full((m, n), 5.0, dtype=torch.float16, device="cuda")
    vals = torch.ones((cap, b, b), dtype=torch.float16, device="cuda")
    plan.run(X, Y, values=vals, pattern=_dev_pattern(brow, bcol, cap, nnzb))
    torch.cuda.synchronize()
    want = S.ERR_CAPACITY if bad in ("over_capacity", "negative") else S.ERR_PATTERN
    assert plan.status() == want
    assert torch.all(Y == 5.0), "Y must be left unwritten"
    # the plan recovers on the next valid call
    Y2 = plan.run(X, values=vals, pattern=_dev_pattern(brow[:1] * 0, bcol[:1] * 0, cap))
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert torch.all(Y2[:b] == b) and not torch.any(Y2[b:])


def test_dynamic_empty_pattern():
    plan = S.Plan(512, 512, 64, 16, w_dtype=S.BF16, mode=S.DYNAMIC, nnzb_max=32)
    Y = torch.full((512, 64), 3.0, dtype=torch.bfloat16, device="cuda")
    vals = torch.zeros((32, 16, 16), dtype=torch.bfloat16, device="cuda")
    plan.run(torch.ones((512, 64), dtype=torch.bfloat16, device="cuda"), Y, values=vals,
             pattern=_dev_pattern([], [], 32, 0))
    torch.cuda.synchronize()
    assert plan.status() == 0 and not torch.any(Y)


def test_dynamic_full_size_sampled():
    """m = k = 8192, n = 1024, b = 16, d_max = 1/16 (nnzb_max = 16384): two
    calls with fresh patterns; 8 sampled block rows against the oracle with
    the normwise, relative and componentwise bars; every device-built array
    bit for bit."""
    m = k = 8192
    n = 1024
    cap = 16384
    plan = S.Plan(m, k, n, 16, w_dtype=S.BF16, mode=S.DYNAMIC, nnzb_max=cap)
    for call in range(2):
        c = wl.dynamic_call(call)
        vals = torch.from_numpy(c["vals"]).to(torch.bfloat16)
        X = torch.from_numpy(c["X"]).to(torch.bfloat16)
        vd = torch.zeros((cap, 16, 16), dtype=torch.bfloat16)
        vd[:len(vals)] = vals
        Y = plan.run(X.cuda(), values=vd.cuda(), pattern=_dev_pattern(c["brow"], c["bcol"], cap))
        torch.cuda.synchronize()
        assert plan.status() == 0
        rows = [0, 101, 170, 255, 256, 340, 510, 511]
        checks.check_rows(Y.cpu(), rows, m, k, 16, c["brow"], c["bcol"], vals, X, torch.bfloat16)
        _check_arrays(plan, m, k, 16, c["brow"], c["bcol"])


def test_dynamic_full_size_integers_exact():
    """The dynamic benchmark's shape (m = k = 8192, n = 1024, b = 16, BF16,
    nnzb_max = 16384) with integer values in [-2, 2] and X in [-1, 1]: sums
    are exact in FP32 and the results fit BF16 exactly, so every row and
    column of Y is checked through exact identities and 8 block rows bit
    for bit, on two calls with different patterns and block counts."""
    m = k = 8192
    n = 1024
    cap = 16384
    plan = S.Plan(m, k, n, 16, w_dtype=S.BF16, mode=S.DYNAMIC, nnzb_max=cap)
    for call, nnz in enumerate((cap, 9001)):
        c = wl.integer_problem(8900 + call, m, k, n, 16, nnz)
        vd = torch.zeros((cap, 16, 16), dtype=torch.bfloat16)
        vd[:nnz] = torch.from_numpy(c["vals"]).to(torch.bfloat16)
        X = torch.from_numpy(c["X"]).to(torch.bfloat16)
        Y = plan.run(X.cuda(), values=vd.cuda(), pattern=_dev_pattern(c["brow"], c["bcol"], cap))
        torch.cuda.synchronize()
        assert plan.status() == 0
        Y = Y.cpu()
        checks.exact_identities(Y, m, k, 16, c["brow"], c["bcol"], c["vals"], c["X"], seed=call)
        checks.exact_rows(Y, [0, 3, 100, 255, 256, 400, 510, 511], k, 16, c["brow"], c["bcol"],
                          c["vals"], c["X"], torch.bfloat16)


@pytest.mark.parametrize("b", [4, 8, 16])
def test_dynamic_near_equal_groups(b):
    """Dynamic tensor-core plans with an explicit count of near-equal
    tile-row groups (11 groups of 5 or 6 tile rows at m = 1024): the device
    re-partition over groups of unequal size (group offsets, chunking,
    workspace rows) equals the oracle's plan of the same groups bit for bit,
    and Y is within the bars, on three calls."""
    m = k = 1024
    n = 136
    cap = wl.nnzb_for(m, k, b, 1 / 16)
    dt = torch.bfloat16
    plan = S.Plan(m, k, n, b, w_dtype=S.BF16, mode=S.DYNAMIC, nnzb_max=cap, groups=11)
    info = plan.info()
    assert info["n_groups"] == 11 and info["rows_per_group"] == 0
    for call in range(3):
        c = wl.dynamic_call(call + 40 * b, m=m, k=k, n=n, b=b, d_max=1 / 16)
        if call == 2:
            # one crowded block row (for b = 16 its group is split over
            # several items and reduced)
            keep = c["brow"] != 3
            extra = np.arange(0, k // b, 2, dtype=np.int32)[:cap - int(keep.sum())]
            c["brow"] = np.concatenate([c["brow"][keep], np.full(len(extra), 3, np.int32)])
            c["bcol"] = np.concatenate([c["bcol"][keep], extra])
            c["vals"] = np.concatenate([c["vals"][keep],
                                        np.ones((len(extra), b, b), np.float32)])
        vals = torch.from_numpy(c["vals"]).to(dt)
        X = torch.from_numpy(c["X"]).to(dt)
        vd = torch.zeros((cap, b, b), dtype=dt)
        vd[:len(vals)] = vals
        Y = plan.run(X.cuda(), values=vd.cuda(), pattern=_dev_pattern(c["brow"], c["bcol"], cap))
        torch.cuda.synchronize()
        assert plan.status() == 0
        info = plan.info()
        assert info["n_groups"] == 11 and info["rows_per_group"] == 0
        Yo = oracle.spmm(m, k, b, c["brow"], c["bcol"], vals, X)
        A = oracle.spmm(m, k, b, c["brow"], c["bcol"], np.abs(oracle.to_f64(vals)),
                        np.abs(oracle.to_f64(X)))
        checks.assert_parity(Y.cpu(), Yo, oracle.block_fro(vals), X, A, dt,
                             checks.max_terms(c["brow"], b))
        _check_arrays(plan, m, k, b, c["brow"], c["bcol"])
        if call == 2 and b == 16:
            assert info["n_reductions"] > 0


@pytest.mark.parametrize("b,dt,w8", [(16, torch.bfloat16, False), (8, torch.float16, False),
                                     (4, torch.bfloat16, False), (16, torch.bfloat16, True),
                                     (8, torch.bfloat16, True)])
def test_fused_repartition_equals_launch_chain(b, dt, w8):
    """Dynamic tensor-core plans re-partition, pack and cut their stages in
    one cooperative launch; the same calls through the launch chain
    (dyn_chain) must give the same device-built arrays and the same Y bit
    for bit, on consecutive calls with different block counts (E4M3 values
    too, where the fused launch clears and fills the tiles' scales)."""
    m, k, n = 1024, 1024, 136
    cap = wl.nnzb_for(m, k, b, 1 / 16)
    wd = S.E4M3 if w8 else S.dtype_code(dt)
    plans = [S.Plan(m, k, n, b, w_dtype=wd, x_dtype=S.dtype_code(dt), mode=S.DYNAMIC,
                    nnzb_max=cap, dyn_chain=ch) for ch in (False, True)]
    for call in range(3):
        c = wl.dynamic_call(call + 60 * b, m=m, k=k, n=n, b=b, d_max=1 / 16)
        X = torch.from_numpy(c["X"]).to(dt).cuda()
        vd = torch.zeros((cap, b, b), dtype=dt)
        vd[:len(c["vals"])] = torch.from_numpy(c["vals"]).to(dt)
        vd = vd.cuda()
        pat = _dev_pattern(c["brow"], c["bcol"], cap)
        outs = []
        for p in plans:
            if w8:
                codes, scales = S.quantize_e4m3(vd)
                Y = p.run(X, values=codes.view(torch.uint8), scales=scales, pattern=pat)
            else:
                Y = p.run(X, values=vd, pattern=pat)
            torch.cuda.synchronize()
            assert p.status() == 0
            outs.append(Y.cpu())
        assert torch.equal(outs[0], outs[1])
        for key in ("row_ptr", "col_idx", "perm", "items", "grp_ebeg", "ent_col", "ent_tbeg",
                    "ent_cover", "tile_row", "blk_slot", "blk_off", "ws_row0", "red"):
            assert np.array_equal(plans[0].array(key), plans[1].array(key)), key
        if not w8:
            vals = torch.from_numpy(c["vals"]).to(dt)
            Yo = oracle.spmm(m, k, b, c["brow"], c["bcol"], vals, X.cpu())
            assert oracle.normwise_err(outs[0], Yo, oracle.block_fro(vals), X.cpu()) <= 4e-3


@pytest.mark.parametrize("b,m,k,groups", [(16, 208, 640, 0), (8, 80, 48, 0), (4, 4096, 4096, 0),
                                          (4, 4096, 2048, 0), (16, 2048, 1024, 100),
                                          (16, 41600, 128, 2600)])
def test_fused_repartition_scan_paths(b, m, k, groups):
    """The fused launch's scans and stage-record paths: a bitmap whose word
    count is not a multiple of four (b = 16, 13 block rows of two words;
    b = 8, 10 block rows of one word), runs longer than the words a thread
    keeps in registers, scanned by every CTA for itself (b = 4, m = 4096,
    k = 2048: 16384 words) and by CTA 0 alone (b = 4, m = k = 4096: 32768
    words, past the per-CTA limit); 100 near-equal groups of one or two
    tile rows; and more groups than the per-CTA group scan takes (2600
    one-row groups: CTA 0 scans).  Arrays and Y equal the launch chain's
    bit for bit; the CSR equals the oracle's; Y is within the normwise
    bar."""
    n = 72
    dt = torch.bfloat16
    cap = max(wl.nnzb_for(m, k, b, 1 / 4), 1)
    plans = [S.Plan(m, k, n, b, w_dtype=S.BF16, mode=S.DYNAMIC, nnzb_max=cap, dyn_chain=ch,
                    groups=groups) for ch in (False, True)]
    if groups:
        assert plans[0].info()["n_groups"] == groups
    for call in range(2):
        c = wl.dynamic_call(call + 70 * b, m=m, k=k, n=n, b=b, d_max=1 / 4)
        X = torch.from_numpy(c["X"]).to(dt).cuda()
        vals = torch.from_numpy(c["vals"]).to(dt)
        vd = torch.zeros((cap, b, b), dtype=dt)
        vd[:len(vals)] = vals
        vd = vd.cuda()
        pat = _dev_pattern(c["brow"], c["bcol"], cap)
        outs = []
        for p in plans:
            Y = p.run(X, values=vd, pattern=pat)
            torch.cuda.synchronize()
            assert p.status() == 0
            outs.append(Y.cpu())
        assert torch.equal(outs[0], outs[1])
        for key in ("row_ptr", "col_idx", "perm", "items", "grp_ebeg", "ent_col", "ent_tbeg",
                    "ent_cover", "tile_row", "blk_slot", "blk_off", "ws_row0", "red"):
            assert np.array_equal(plans[0].array(key), plans[1].array(key)), key
        rp, ci, pm = P.csr(m // b, c["brow"], c["bcol"])
        assert np.array_equal(plans[0].array("row_ptr"), rp)
        assert np.array_equal(plans[0].array("col_idx"), ci)
        assert np.array_equal(plans[0].array("perm"), pm)
        Yo = oracle.spmm(m, k, b, c["brow"], c["bcol"], vals, X.cpu())
        assert oracle.normwise_err(outs[0], Yo, oracle.block_fro(vals), X.cpu()) <= 4e-3


def test_fused_repartition_wait_times_out_and_recovers():
    """Failure detection in the fused re-partition: with the test hook on, one
    CTA skips its arrival at the first grid barrier; every CTA's bounded wait
    runs out (200 us), the status word reads SPMM_ERR_TIMEOUT, the product
    launch skips (Y keeps its contents) and the context stays usable: the
    next call, with the default limit, is correct against the oracle."""
    m = k = 1024
    n = 64
    b = 16
    cap = wl.nnzb_for(m, k, b, 1 / 16)
    plan = S.Plan(m, k, n, b, w_dtype=S.BF16, mode=S.DYNAMIC, nnzb_max=cap)
    c = wl.dynamic_call(7100, m=m, k=k, n=n, b=b, d_max=1 / 16)
    X = torch.from_numpy(c["X"]).to(torch.bfloat16)
    vals = torch.from_numpy(c["vals"]).to(torch.bfloat16)
    vd = torch.zeros((cap, b, b), dtype=torch.bfloat16)
    vd[:len(vals)] = vals
    pat = _dev_pattern(c["brow"], c["bcol"], cap)
    plan.set_wait(200_000, stall=True)
    Y = torch.full((m, n), 5.0, dtype=torch.bfloat16, device="cuda")
    plan.run(X.cuda(), Y, values=vd.cuda(), pattern=pat)
    torch.cuda.synchronize()
    assert plan.status() == S.ERR_TIMEOUT
    assert torch.all(Y == 5.0)
    plan.set_wait(0, stall=False)
    Y = plan.run(X.cuda(), values=vd.cuda(), pattern=pat)
    torch.cuda.synchronize()
    assert plan.status() == 0
    Yo = oracle.spmm(m, k, b, c["brow"], c["bcol"], vals, X)
    assert oracle.normwise_err(Y.cpu(), Yo, oracle.block_fro(vals), X) <= 4e-3
    _check_arrays(plan, m, k, b, c["brow"], c["bcol"])


def test_fused_barrier_words_across_calls_and_graph_replays():
    """The fused re-partition's barrier words are cleared by the previous
    call (its reduction launch, or a memset after a call without a
    product) instead of before each launch.  Calls with and without a
    product in any order, and a captured call replayed between eager calls,
    all give the oracle's Y and plan arrays."""
    m = k = 1024
    n = 64
    b = 16
    cap = wl.nnzb_for(m, k, b, 1 / 16)
    dt = torch.bfloat16
    plan = S.Plan(m, k, n, b, w_dtype=S.BF16, mode=S.DYNAMIC, nnzb_max=cap)
    cases = []
    for call in range(3):
        c = wl.dynamic_call(7300 + call, m=m, k=k, n=n, b=b, d_max=1 / 16)
        vals = torch.from_numpy(c["vals"]).to(dt)
        vd = torch.zeros((cap, b, b), dtype=dt)
        vd[:len(vals)] = vals
        cases.append(dict(c=c, vals=vals, vd=vd.cuda(), X=torch.from_numpy(c["X"]).to(dt),
                          pat=_dev_pattern(c["brow"], c["bcol"], cap)))

    def check(Y, q):
        Yo = oracle.spmm(m, k, b, q["c"]["brow"], q["c"]["bcol"], q["vals"], q["X"])
        assert oracle.normwise_err(Y.cpu(), Yo, oracle.block_fro(q["vals"]), q["X"]) <= 4e-3
        _check_arrays(plan, m, k, b, q["c"]["brow"], q["c"]["bcol"])

    Xe = torch.empty((k, 0), dtype=dt, device="cuda")
    Ye = torch.empty((m, 0), dtype=dt, device="cuda")
    for q in (cases[0], cases[1], cases[1], cases[2]):
        plan.run(Xe, Ye, values=q["vd"], pattern=q["pat"])         # no product
        Y = plan.run(q["X"].cuda(), values=q["vd"], pattern=q["pat"])
        torch.cuda.synchronize()
        assert plan.status() == 0
        check(Y, q)
    # a captured call, replayed with eager calls (with and without a product) between
    q = cases[0]
    Xd = q["X"].cuda()
    Yg = torch.empty((m, n), dtype=dt, device="cuda")
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        plan.run(Xd, Yg, values=q["vd"], pattern=q["pat"], stream=st)
        st.synchronize()
        with torch.cuda.graph(g, stream=st):
            plan.run(Xd, Yg, values=q["vd"], pattern=q["pat"], stream=st)
    torch.cuda.synchronize()
    for other in (cases[1], cases[2], cases[1]):
        plan.run(Xe, Ye, values=other["vd"], pattern=other["pat"])
        Y = plan.run(other["X"].cuda(), values=other["vd"], pattern=other["pat"])
        torch.cuda.synchronize()
        assert plan.status() == 0
        check(Y, other)
        Yg.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert plan.status() == 0
        check(Yg, q)
