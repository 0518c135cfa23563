"""GPU test of spmm_gather_noalloc, the entry point for callers that cannot
allocate device memory (code running inside someone else's CUDA graph
capture, frameworks that own every device allocation, fixed-budget loops):
it keeps its scratch in a fixed device array instead of plan-owned buffers.
Its output must match the dynamic-plan spmm_run on the same inputs and the
FP64 oracle, on two calls in a row with different patterns (the shared
scratch keeps the previous call's contents); it must run inside a CUDA
graph captured in global mode (where any allocation would abort the
capture); and sizes beyond its limits must be refused.  This file is
collected last on purpose."""
import ctypes

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


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _call(m, k, dt, pat, cap, vals, X, Y, status):
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)  # the capturing stream, if any
    S.spmm_gather_noalloc(m, k, S.dtype_code(dt), _p(pat[0]), _p(pat[1]), _p(pat[2]), cap,
                          _p(vals), _p(X), X.shape[1], X.stride(0), _p(Y), Y.stride(0),
                          _p(status), s)


@pytest.mark.parametrize("dt", [torch.float16, torch.float32])
def test_noalloc_matches_dynamic_plan_twice(dt):
    m, k, n = 2048, 4096, 200
    cap = 140000
    plan = S.Plan(m, k, n, 1, w_dtype=S.dtype_code(dt), mode=S.DYNAMIC, nnzb_max=cap)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for call, dens in ((0, 1 / 64), (1, 1 / 80)):
        rng = np.random.default_rng(500 + call)
        brow, bcol = wl.pattern(rng, m, k, int(m * k * dens))
        if call == 1:
            # one long row: exercises the split-row workspace
            keep = brow != 7
            brow = np.concatenate([brow[keep], np.full(600, 7, np.int32)])
            bcol = np.concatenate([bcol[keep], np.arange(600, dtype=np.int32) * 6])
        nnzb = len(brow)
        vals = torch.from_numpy(rng.standard_normal(nnzb).astype(np.float32)).to(dt)
        X = torch.from_numpy(rng.standard_normal((k, n)).astype(np.float32)).to(dt).cuda()
        br = torch.zeros(cap, dtype=torch.int32)
        bc = torch.zeros(cap, dtype=torch.int32)
        br[:nnzb] = torch.from_numpy(brow)
        bc[:nnzb] = torch.from_numpy(bcol)
        vd = torch.zeros(cap, dtype=dt)
        vd[:nnzb] = vals
        pat = (torch.tensor([nnzb], dtype=torch.int32, device="cuda"), br.cuda(), bc.cuda())
        vd = vd.cuda()
        Y_ref = plan.run(X, values=vd, pattern=pat)
        Y = torch.full((m, n), float("nan"), dtype=dt, device="cuda")
        _call(m, k, dt, pat, cap, vd, X, Y, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0 and plan.status() == 0
        tol = 1e-6 if dt == torch.float32 else 4e-3
        Wf = oracle.block_fro(vals)
        assert oracle.normwise_err(Y.cpu(), oracle.to_f64(Y_ref.cpu()), Wf, X.cpu()) <= tol
        assert not torch.isnan(Y).any()
        # and both against the oracle itself
        Yo = oracle.spmm(m, k, 1, brow, bcol, vals, X.cpu())
        A = oracle.spmm(m, k, 1, brow, bcol, np.abs(oracle.to_f64(vals)),
                        np.abs(oracle.to_f64(X.cpu())))
        for out in (Y, Y_ref):
            checks.assert_parity(out.cpu(), Yo, Wf, X.cpu(), A, dt, checks.max_terms(brow, 1))


def test_noalloc_inside_graph_capture():
    """A call captured into a CUDA graph in global capture mode (any
    cudaMalloc there would abort the capture), after one uncaptured call on
    the device; the graph replayed twice, with new values written into the
    same buffers before the second replay, each against the oracle."""
    m, k, n, dt = 1024, 2048, 64, torch.float16
    cap = 40000
    rng = np.random.default_rng(77)
    brow, bcol = wl.pattern(rng, m, k, 30000)
    nnzb = len(brow)
    pat = (torch.tensor([nnzb], dtype=torch.int32, device="cuda"),
           torch.zeros(cap, dtype=torch.int32, device="cuda"),
           torch.zeros(cap, dtype=torch.int32, device="cuda"))
    pat[1][:nnzb] = torch.from_numpy(brow).cuda()
    pat[2][:nnzb] = torch.from_numpy(bcol).cuda()
    vd = torch.zeros(cap, dtype=dt, device="cuda")
    X = torch.from_numpy(rng.standard_normal((k, n)).astype(np.float32)).to(dt).cuda()
    Y = torch.empty((m, n), dtype=dt, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    _call(m, k, dt, pat, cap, vd, X, Y, status)     # uncaptured: looks up the scratch
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="global"):
        _call(m, k, dt, pat, cap, vd, X, Y, status)
    for rep in range(2):
        vals = torch.from_numpy(rng.standard_normal(nnzb).astype(np.float32)).to(dt)
        vd[:nnzb] = vals.cuda()
        Y.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        Yo = oracle.spmm(m, k, 1, brow, bcol, vals, X.cpu())
        A = oracle.spmm(m, k, 1, brow, bcol, np.abs(oracle.to_f64(vals)),
                        np.abs(oracle.to_f64(X.cpu())))
        checks.assert_parity(Y.cpu(), Yo, oracle.block_fro(vals), X.cpu(), A, dt,
                             checks.max_terms(brow, 1))


def test_noalloc_refuses_oversize_and_reports_pattern_errors():
    m, k, n = 512, 512, 16
    X = torch.ones((k, n), dtype=torch.float16, device="cuda")
    Y = torch.full((m, n), 2.0, dtype=torch.float16, device="cuda")
    vals = torch.ones(8, dtype=torch.float16, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    pat = (torch.tensor([2], dtype=torch.int32, device="cuda"),
           torch.tensor([3, 3] + [0] * 6, dtype=torch.int32, device="cuda"),
           torch.tensor([5, 5] + [0] * 6, dtype=torch.int32, device="cuda"))
    with pytest.raises(S.SpmmError) as e:
        _call(8193, k, torch.float16, pat, 8, vals, X, Y, status)
    assert e.value.status == S.ERR_SHAPE
    with pytest.raises(S.SpmmError) as e:
        _call(m, k, torch.float16, pat, 262145, vals, X, Y, status)
    assert e.value.status == S.ERR_SHAPE
    Xw = torch.ones((k, 257), dtype=torch.float16, device="cuda")
    with pytest.raises(S.SpmmError) as e:
        _call(m, k, torch.float16, pat, 8, vals, Xw, torch.empty((m, 257), dtype=torch.float16,
                                                                  device="cuda"), status)
    assert e.value.status == S.ERR_SHAPE
    # a repeated block: status set on the device, Y left as it was
    _call(m, k, torch.float16, pat, 8, vals, X, Y, status)
    torch.cuda.synchronize()
    assert int(status.item()) == S.ERR_PATTERN
    assert torch.all(Y == 2.0)
