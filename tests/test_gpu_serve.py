"""GPU tests of the serving loop (include/spmm_serve.h).

* Each result is the same alone and in a mix of concurrent requests aimed at
  several resident weights (bit-identical here; the stated tolerance is the
  acceptance bar), and matches the FP64 oracle.
* Admission by HBM budget: a budget that holds one request at a time still
  serves everything; a request larger than the budget is refused.
* Host-side fault injection: a delayed batcher makes serve_wait time out
  (and the request completes later); failing staging allocations surface as
  an error on the ticket.
* A weight of the plain FP32 kernel is served one request per launch.
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


WEIGHTS = [(1024, 8), (2048, 16), (1024, 16), (2048, 8)]


def _weights(dt=torch.float16):
    out = []
    for i, (m, b) in enumerate(WEIGHTS):
        c = wl.problem(7000 + i, m, m, 1, b, wl.nnzb_for(m, m, b, 1 / 16))
        plan = S.Plan(m, m, 256, b, w_dtype=S.dtype_code(dt), brow=c["brow"], bcol=c["bcol"])
        vals = torch.from_numpy(c["vals"]).to(dt)
        plan.pack(vals.cuda())
        out.append(dict(c=c, plan=plan, vals=vals, m=m))
    torch.cuda.synchronize()
    return out


def _requests(ws, count, seed, dt=torch.float16):
    rng = np.random.default_rng(seed)
    reqs = []
    for r in range(count):
        w = int(rng.integers(0, len(ws)))
        n = int(min(256, max(1, round(float(np.exp(rng.uniform(0, np.log(256))))))))
        X = torch.from_numpy(wl.request_x(seed * 1000 + r, ws[w]["m"], n)).to(dt).pin_memory()
        reqs.append((w, X))
    return reqs


def test_same_alone_and_in_mix():
    ws = _weights()
    srv = S.Server(hbm_budget_bytes=64 << 20, max_inflight=3)
    ids = [srv.register(w["plan"]) for w in ws]
    reqs = _requests(ws, 24, 1)
    alone = []
    for w, X in reqs:
        Y = torch.empty((ws[w]["m"], X.shape[1]), dtype=torch.float16).pin_memory()
        srv.wait(srv.submit(ids[w], X, Y))
        alone.append(Y)
    mix = [torch.empty_like(a).pin_memory() for a in alone]
    tickets = [srv.submit(ids[w], X, Y) for (w, X), Y in zip(reqs, mix)]
    for t in tickets:
        srv.wait(t)
    st = srv.stats()
    assert st["completed"] == 48 and st["failed"] == 0
    assert st["mean_requests_per_launch"] > 1.0, "concurrent requests should share launches"
    for (w, X), a, b in zip(reqs, alone, mix):
        Wf = oracle.block_fro(ws[w]["vals"])
        assert oracle.normwise_err(b, oracle.to_f64(a), Wf, X) <= 4e-3
        assert torch.equal(a, b)
    for (w, X), a in list(zip(reqs, alone))[:4]:
        c = ws[w]["c"]
        Yo = oracle.spmm(ws[w]["m"], ws[w]["m"], c["b"], c["brow"], c["bcol"], ws[w]["vals"], X)
        assert oracle.normwise_err(a, Yo, oracle.block_fro(ws[w]["vals"]), X) <= 4e-3
    assert st["p50_us"] <= st["p99_us"]
    srv.close()


def test_budget_admission_and_refusal():
    ws = _weights()
    big = ws[1]["m"] * 256 * 2 * 2           # largest request: X and Y at n = 256
    srv = S.Server(hbm_budget_bytes=big + 4096, max_inflight=2)
    ids = [srv.register(w["plan"]) for w in ws]
    reqs = _requests(ws, 12, 2)
    outs = []
    tickets = []
    for w, X in reqs:
        Y = torch.empty((ws[w]["m"], X.shape[1]), dtype=torch.float16).pin_memory()
        tickets.append(srv.submit(ids[w], X, Y))
        outs.append(Y)
    for t in tickets:
        srv.wait(t)
    for (w, X), Y in zip(reqs, outs):
        c = ws[w]["c"]
        Yo = oracle.spmm(ws[w]["m"], ws[w]["m"], c["b"], c["brow"], c["bcol"], ws[w]["vals"], X)
        assert oracle.normwise_err(Y, Yo, oracle.block_fro(ws[w]["vals"]), X) <= 4e-3
    srv.close()
    tiny = S.Server(hbm_budget_bytes=1 << 16, max_inflight=1)
    wid = tiny.register(ws[0]["plan"])
    X = torch.zeros((ws[0]["m"], 64), dtype=torch.float16)
    Y = torch.empty((ws[0]["m"], 64), dtype=torch.float16)
    with pytest.raises(S.SpmmError) as e:
        tiny.submit(wid, X, Y)
    assert e.value.status == S.ERR_CAPACITY
    assert tiny.stats()["rejected"] == 1
    tiny.close()


def test_wait_timeout_with_delayed_batcher():
    ws = _weights()
    srv = S.Server(hbm_budget_bytes=16 << 20, max_inflight=1, inject_delay_us=300000)
    wid = srv.register(ws[0]["plan"])
    X = torch.ones((ws[0]["m"], 16), dtype=torch.float16).pin_memory()
    Y = torch.empty((ws[0]["m"], 16), dtype=torch.float16).pin_memory()
    t = srv.submit(wid, X, Y)
    with pytest.raises(S.SpmmError) as e:
        srv.wait(t, timeout_ms=10)
    assert e.value.status == S.ERR_TIMEOUT
    srv.wait(t, timeout_ms=10000)
    c = ws[0]["c"]
    Yo = oracle.spmm(ws[0]["m"], ws[0]["m"], c["b"], c["brow"], c["bcol"], ws[0]["vals"], X)
    assert oracle.normwise_err(Y, Yo, oracle.block_fro(ws[0]["vals"]), X) <= 4e-3
    srv.close()


def test_failing_staging_allocation():
    ws = _weights()
    srv = S.Server(hbm_budget_bytes=16 << 20, max_inflight=1, inject_alloc_fail=1)
    wid = srv.register(ws[0]["plan"])
    X = torch.ones((ws[0]["m"], 8), dtype=torch.float16)
    Y = torch.empty((ws[0]["m"], 8), dtype=torch.float16)
    t = srv.submit(wid, X, Y)
    with pytest.raises(S.SpmmError) as e:
        srv.wait(t, timeout_ms=10000)
    assert e.value.status == S.ERR_OOM
    assert srv.stats()["failed"] == 1
    srv.close()


def test_plain_fp32_weight_one_per_launch():
    m, b = 512, 8
    c = wl.problem(7100, m, m, 1, b, wl.nnzb_for(m, m, b, 1 / 16))
    plan = S.Plan(m, m, 128, b, w_dtype=S.F32, brow=c["brow"], bcol=c["bcol"], kernel="plain")
    vals = torch.from_numpy(c["vals"])
    plan.pack(vals.cuda())
    srv = S.Server(hbm_budget_bytes=16 << 20, max_inflight=2)
    wid = srv.register(plan)
    outs, tickets, xs = [], [], []
    for r in range(5):
        X = torch.from_numpy(wl.request_x(r, m, 40 + r)).pin_memory()
        Y = torch.empty((m, X.shape[1]), dtype=torch.float32).pin_memory()
        tickets.append(srv.submit(wid, X, Y))
        outs.append(Y)
        xs.append(X)
    for t in tickets:
        srv.wait(t)
    st = srv.stats()
    assert st["launches"] == 5 and st["mean_requests_per_launch"] == 1.0
    for X, Y in zip(xs, outs):
        Yo = oracle.spmm(m, m, b, c["brow"], c["bcol"], vals, X)
        assert oracle.normwise_err(Y, Yo, oracle.block_fro(vals), X) <= 1e-6
    srv.close()


def test_native_replay_matches_submissions():
    ws = _weights()
    srv = S.Server(hbm_budget_bytes=64 << 20, max_inflight=4)
    ids = [srv.register(w["plan"]) for w in ws]
    reqs = _requests(ws, 40, 3)
    outs = [torch.empty((ws[w]["m"], X.shape[1]), dtype=torch.float16).pin_memory()
            for w, X in reqs]
    t_arr = np.linspace(0.0, 0.01, len(reqs))
    st = srv.replay(t_arr, [ids[w] for w, _ in reqs], [X.shape[1] for _, X in reqs],
                    [X.data_ptr() for _, X in reqs], [Y.data_ptr() for Y in outs])
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["p99_us"] > 0
    for (w, X), Y in zip(reqs, outs):
        c = ws[w]["c"]
        Yo = oracle.spmm(ws[w]["m"], ws[w]["m"], c["b"], c["brow"], c["bcol"], ws[w]["vals"], X)
        assert oracle.normwise_err(Y, Yo, oracle.block_fro(ws[w]["vals"]), X) <= 4e-3
    srv.close()
