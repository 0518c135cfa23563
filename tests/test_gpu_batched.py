"""GPU tests of the low-precision and batched forms.

* The E4M3 quantiser (one FP32 scale per block, scale = max|w| / 448) against
  an independent torch quantisation of the same blocks (bit-exact codes).
* E4M3 plans: Y against the FP64 oracle evaluated on decode(code) * scale,
  bound 3e-2 normwise.
* spmm_batch_run: uneven problems in one persistent launch, each against
  the oracle, and each equal to the same plan run alone (the batch changes
  only where and when a work unit runs, never its arithmetic order).
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


@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16, torch.float16])
@pytest.mark.parametrize("b", [4, 16])
def test_quantizer_matches_torch(dt, b):
    rng = np.random.default_rng(b)
    v = torch.from_numpy(rng.standard_normal((300, b, b)).astype(np.float32) * 3).to(dt)
    v[7] = 0                                      # all-zero block: scale 1, codes 0
    codes, scales = S.quantize_e4m3(v.cuda())
    vf = v.float()
    amax = vf.abs().amax(dim=(1, 2))
    want_s = torch.where(amax > 0, amax / 448.0, torch.ones_like(amax))
    assert torch.equal(scales.cpu(), want_s)
    want_c = (vf / want_s.view(-1, 1, 1)).clamp(-448, 448).to(torch.float8_e4m3fn)
    assert torch.equal(codes.cpu().view(torch.uint8), want_c.view(torch.uint8))


def _problem(seed, m, k, n, b, d):
    c = wl.problem(seed, m, k, n, b, wl.nnzb_for(m, k, b, d))
    return c


def _e4m3_plan(c, xdt=torch.bfloat16, **kw):
    vals = torch.from_numpy(c["vals"]).to(xdt).cuda()
    codes, scales = S.quantize_e4m3(vals)
    plan = S.Plan(c["m"], c["k"], max(c["n"], 1), c["b"], w_dtype=S.E4M3,
                  x_dtype=S.dtype_code(xdt), brow=c["brow"], bcol=c["bcol"], **kw)
    plan.pack(codes.view(torch.uint8), scales)
    return plan, codes.cpu(), scales.cpu()


def _x(c, dt):
    k, n = c["X"].shape
    ld = ((n + 7) // 8) * 8
    buf = torch.zeros((k, ld), dtype=dt, device="cuda")
    buf[:, :n] = torch.from_numpy(c["X"]).to(dt).cuda()
    return buf[:, :n]


@pytest.mark.parametrize("b,d,n", [(16, 1 / 8, 200), (8, 1 / 16, 64), (4, 1 / 16, 9),
                                   (16, 1 / 4, 1)])
def test_e4m3_parity(b, d, n):
    c = _problem(70 + b, 1024, 2048, n, b, d)
    plan, codes, scales = _e4m3_plan(c)
    X = _x(c, torch.bfloat16)
    Y = plan.run(X)
    torch.cuda.synchronize()
    v = oracle.e4m3_block_values(codes.view(torch.uint8).numpy(), scales.numpy())
    Yo = oracle.spmm(c["m"], c["k"], b, c["brow"], c["bcol"], v, X.cpu())
    err = oracle.normwise_err(Y.cpu(), Yo, oracle.block_fro(v), X.cpu())
    assert err <= 3e-2, err
    # and the quantised product stays close to the unquantised definition
    Yq = oracle.spmm(c["m"], c["k"], b, c["brow"], c["bcol"], c["vals"], X.cpu())
    assert oracle.normwise_err(Y.cpu(), Yq, oracle.block_fro(c["vals"]), X.cpu()) <= 3e-2


SHAPES = [  # m, k, n, b, d  (FFN-like uneven problems, scaled down)
    (1024, 4096, 77, 8, 1 / 16), (4096, 1024, 130, 16, 1 / 16), (1024, 4096, 1, 16, 1 / 8),
    (4096, 1024, 512, 8, 1 / 8), (2048, 2048, 33, 16, 1 / 16), (1024, 1024, 256, 16, 1 / 4),
]


@pytest.mark.parametrize("fp8", [True, False])
def test_batch_matches_oracle_and_alone(fp8):
    cases = [_problem(900 + i, *s) for i, s in enumerate(SHAPES)]
    plans, Xs, Ys, vals = [], [], [], []
    for c in cases:
        if fp8:
            plan, codes, scales = _e4m3_plan(c)
            vals.append(oracle.e4m3_block_values(codes.view(torch.uint8).numpy(), scales.numpy()))
        else:
            v = torch.from_numpy(c["vals"]).to(torch.bfloat16)
            plan = S.Plan(c["m"], c["k"], c["n"], c["b"], w_dtype=S.BF16, brow=c["brow"],
                          bcol=c["bcol"])
            plan.pack(v.cuda())
            vals.append(v)
        plans.append(plan)
        Xs.append(_x(c, torch.bfloat16))
        Ys.append(torch.full((c["m"], c["n"]), float("nan"), dtype=torch.bfloat16, device="cuda"))
    for _ in range(2):                   # the second launch reuses the cached schedule
        S.spmm_batch_run(plans, Xs, Ys)
    torch.cuda.synchronize()
    tol = 3e-2 if fp8 else 4e-3
    for c, plan, X, Y, v in zip(cases, plans, Xs, Ys, vals):
        Yo = oracle.spmm(c["m"], c["k"], c["b"], c["brow"], c["bcol"], v, X.cpu())
        assert oracle.normwise_err(Y.cpu(), Yo, oracle.block_fro(v), X.cpu()) <= tol
        alone = plan.run(X)
        torch.cuda.synchronize()
        assert torch.equal(alone, Y), "batched result differs from the same plan run alone"
        assert plan.status() == 0


def test_batch_rejects_mixed_or_dynamic():
    c = _problem(5, 512, 512, 64, 16, 1 / 8)
    p1 = S.Plan(512, 512, 64, 16, w_dtype=S.F16, brow=c["brow"], bcol=c["bcol"])
    p1.pack(torch.from_numpy(c["vals"]).half().cuda())
    p2 = S.Plan(512, 512, 64, 16, w_dtype=S.BF16, brow=c["brow"], bcol=c["bcol"])
    p2.pack(torch.from_numpy(c["vals"]).bfloat16().cuda())
    X = torch.zeros((512, 64), dtype=torch.float16, device="cuda")
    with pytest.raises(S.SpmmError) as e:
        S.spmm_batch_run([p1, p2], [X, X.bfloat16()], [torch.empty_like(X)] * 2)
    assert e.value.status == S.ERR_UNSUPPORTED
    p3 = S.Plan(512, 512, 64, 16, w_dtype=S.F16, mode=S.DYNAMIC, nnzb_max=64)
    with pytest.raises(S.SpmmError) as e:
        S.spmm_batch_run([p1, p3], [X, X], [torch.empty_like(X)] * 2)
    assert e.value.status == S.ERR_UNSUPPORTED


@pytest.mark.parametrize("b,d,geo", [(8, 1 / 4, 0), (16, 1 / 32, 1)])
def test_e4m3_both_stage_geometries(b, d, geo):
    """E4M3 plans also choose dense- or sparse-tile stages; both within the
    FP8 bound against the oracle on the decoded values."""
    c = _problem(90 + b, 1024, 2048, 136, b, d)
    plan, codes, scales = _e4m3_plan(c, rows_per_group=16)
    assert plan.info()["stage_geometry"] == geo
    X = _x(c, torch.bfloat16)
    Y = plan.run(X)
    torch.cuda.synchronize()
    v = oracle.e4m3_block_values(codes.view(torch.uint8).numpy(), scales.numpy())
    Yo = oracle.spmm(c["m"], c["k"], b, c["brow"], c["bcol"], v, X.cpu())
    assert oracle.normwise_err(Y.cpu(), Yo, oracle.block_fro(v), X.cpu()) <= 3e-2
