"""GPU tests of the low-precision and batched forms.

* The E4M3 quantiser (one FP32 scale per block, scale = max|w| / 448) against
  an independent torch quantisation of the same blocks (bit-exact codes).
* E4M3 plans: Y against the FP64 oracle evaluated on decode(code) * scale
  with the 16-bit bars (4e-3 normwise, 1e-2 relative, componentwise): the
  only roundings left are code x scale to the 16-bit operand type, the FP32
  accumulation and the output; against the unquantised values, the FP8
  bound 3e-2.
* spmm_batch_run: uneven problems in one persistent launch, each against
  the oracle, and each equal to the same plan run alone (the batch changes
  only where and when a work unit runs, never its arithmetic order).
"""
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
    A = oracle.spmm(c["m"], c["k"], b, c["brow"], c["bcol"], np.abs(v), np.abs(oracle.to_f64(X.cpu())))
    checks.assert_parity(Y.cpu(), Yo, oracle.block_fro(v), X.cpu(), A, torch.bfloat16,
                         checks.max_terms(c["brow"], b), u_w=2.0 ** -8)
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
    for c, plan, X, Y, v in zip(cases, plans, Xs, Ys, vals):
        Yo = oracle.spmm(c["m"], c["k"], c["b"], c["brow"], c["bcol"], v, X.cpu())
        A = oracle.spmm(c["m"], c["k"], c["b"], c["brow"], c["bcol"], np.abs(oracle.to_f64(v)),
                        np.abs(oracle.to_f64(X.cpu())))
        checks.assert_parity(Y.cpu(), Yo, oracle.block_fro(v), X.cpu(), A, torch.bfloat16,
                             checks.max_terms(c["brow"], c["b"]), u_w=2.0 ** -8 if fp8 else 0.0)
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
    A = oracle.spmm(c["m"], c["k"], b, c["brow"], c["bcol"], np.abs(v), np.abs(oracle.to_f64(X.cpu())))
    checks.assert_parity(Y.cpu(), Yo, oracle.block_fro(v), X.cpu(), A, torch.bfloat16,
                         checks.max_terms(c["brow"], b), u_w=2.0 ** -8)


def _e4m3_full(i):
    """Problem i of the benchmark's batched configuration at full size, its
    weights quantised on the device; the codes and scales come back to the
    host for the oracle."""
    c = wl.batched_case(i)
    v = torch.from_numpy(c["vals"]).to(torch.bfloat16).cuda()
    codes, scales = S.quantize_e4m3(v)
    plan = S.Plan(c["m"], c["k"], c["n"], c["b"], w_dtype=S.E4M3, x_dtype=S.BF16,
                  brow=c["brow"], bcol=c["bcol"])
    plan.pack(codes.view(torch.uint8), scales)
    return c, plan, codes.view(torch.uint8).cpu().numpy(), scales.cpu().numpy()


def test_batched_config_sampled():
    """The benchmark's batched configuration itself: 48 FFN-like problems
    (W 4096 x 16384 or 16384 x 4096, b in {8, 16}, d in {1/16, 1/8}, n
    log-uniform in [1, 512]), E4M3 weights with per-block FP32 scales, BF16
    X, in one spmm_batch_run as the benchmark times it.  Three block rows of
    every problem against the oracle on the decoded values (all 16-bit
    bars), and against the unquantised values within the FP8 bound."""
    plans, Xs, Ys, kept = [], [], [], []
    for i in range(48):
        c, plan, codes, scales = _e4m3_full(i)
        mb = c["m"] // c["b"]
        rows = [0, mb // 2 + i, mb - 1]
        br, bc, cs, sel = checks.sub_rows(c["brow"], c["bcol"], codes, rows)
        kept.append(dict(c=c, rows=rows, br=br, bc=bc,
                         v=oracle.e4m3_block_values(cs, scales[sel]), raw=c["vals"][sel]))
        plans.append(plan)
        Xs.append(_x(c, torch.bfloat16))
        Ys.append(torch.full((c["m"], c["n"]), float("nan"), dtype=torch.bfloat16,
                             device="cuda"))
        del c["vals"]
    S.spmm_batch_run(plans, Xs, Ys)
    torch.cuda.synchronize()
    for plan, X, Y, kp in zip(plans, Xs, Ys, kept):
        assert plan.status() == 0
        c, rows, b = kp["c"], kp["rows"], kp["c"]["b"]
        Xc = X.cpu()
        mr = len(rows) * b
        Ys_ = torch.cat([Y[r * b:(r + 1) * b].cpu() for r in rows])
        Yo = oracle.spmm(mr, c["k"], b, kp["br"], kp["bc"], kp["v"], Xc)
        A = oracle.spmm(mr, c["k"], b, kp["br"], kp["bc"], np.abs(kp["v"]),
                        np.abs(oracle.to_f64(Xc)))
        checks.assert_parity(Ys_, Yo, oracle.block_fro(kp["v"]), Xc, A, torch.bfloat16,
                             checks.max_terms(kp["br"], b), u_w=2.0 ** -8)
        Yq = oracle.spmm(mr, c["k"], b, kp["br"], kp["bc"], kp["raw"], Xc)
        assert oracle.normwise_err(Ys_, Yq, oracle.block_fro(kp["raw"]), Xc) <= 3e-2
        plan.close()


def test_batched_full_size_integers_exact():
    """Two problems of the batched configuration at full size (problem 0:
    4096 x 16384, b = 8; problem 3: 16384 x 4096, b = 16) with E4M3 codes of
    -1, 0, 1 and power-of-two block scales (1/2 or 1), X in [-1, 1]: code x
    scale is exact in BF16, sums are exact in FP32 and results fit BF16, so
    every row and column of each Y is checked through exact identities and
    sampled block rows bit for bit, after one spmm_batch_run of both."""
    e4m3 = np.array([0xB8, 0x00, 0x38], np.uint8)          # -1, 0, +1
    plans, Xs, Ys, cases = [], [], [], []
    for i in (0, 3):
        sp = wl.batched_spec(i)
        c = wl.integer_problem(9100 + i, sp["m"], sp["k"], sp["n"], sp["b"], sp["nnzb"],
                               vals_range=(-1, 1))
        rng = np.random.default_rng(9200 + i)
        codes = e4m3[(c["vals"] + 1).astype(np.int64)]
        scales = rng.choice([0.5, 1.0], size=len(c["brow"])).astype(np.float32)
        c["v"] = oracle.e4m3_block_values(codes, scales)
        plan = S.Plan(c["m"], c["k"], c["n"], c["b"], w_dtype=S.E4M3, x_dtype=S.BF16,
                      brow=c["brow"], bcol=c["bcol"])
        plan.pack(torch.from_numpy(codes).cuda(), torch.from_numpy(scales).cuda())
        plans.append(plan)
        Xs.append(_x(c, torch.bfloat16))
        Ys.append(torch.full((c["m"], c["n"]), float("nan"), dtype=torch.bfloat16,
                             device="cuda"))
        cases.append(c)
    S.spmm_batch_run(plans, Xs, Ys)
    torch.cuda.synchronize()
    for plan, Y, c in zip(plans, Ys, cases):
        assert plan.status() == 0
        Y = Y.cpu()
        checks.exact_identities(Y, c["m"], c["k"], c["b"], c["brow"], c["bcol"], c["v"],
                                c["X"], seed=c["seed"])
        mb = c["m"] // c["b"]
        checks.exact_rows(Y, [0, 1, mb // 2, mb - 1], c["k"], c["b"], c["brow"], c["bcol"],
                          c["v"], c["X"], torch.bfloat16)
        plan.close()


def test_batch_mixed_geometries_one_launch_equals_alone():
    """Plans forced to different stage geometries run in one tensor-core
    launch (the minority plan on stage records cut for the other geometry):
    each result bit for bit equal to the plan run alone, and within the
    bars against the oracle."""
    cases = [_problem(950 + i, 1024, 2048, n, b, d)
             for i, (b, d, n) in enumerate(((16, 1 / 16, 130), (8, 1 / 4, 200), (16, 1 / 4, 256)))]
    plans, Xs, Ys = [], [], []
    for c, geo in zip(cases, (1, 2, 1)):
        v = torch.from_numpy(c["vals"]).to(torch.bfloat16)
        p = S.Plan(c["m"], c["k"], c["n"], c["b"], w_dtype=S.BF16, brow=c["brow"], bcol=c["bcol"],
                   kernel="tc", stage_geometry=geo)
        assert p.info()["stage_geometry"] == geo - 1
        p.pack(v.cuda())
        plans.append(p)
        Xs.append(_x(c, torch.bfloat16))
        Ys.append(torch.full((c["m"], c["n"]), float("nan"), dtype=torch.bfloat16, device="cuda"))
    for _ in range(2):
        S.spmm_batch_run(plans, Xs, Ys)
    torch.cuda.synchronize()
    for c, p, X, Y in zip(cases, plans, Xs, Ys):
        assert p.status() == 0
        alone = p.run(X)
        torch.cuda.synchronize()
        assert torch.equal(alone, Y)
        v = torch.from_numpy(c["vals"]).to(torch.bfloat16)
        Yo = oracle.spmm(c["m"], c["k"], c["b"], c["brow"], c["bcol"], v, X.cpu())
        A = oracle.spmm(c["m"], c["k"], c["b"], c["brow"], c["bcol"], np.abs(oracle.to_f64(v)),
                        np.abs(oracle.to_f64(X.cpu())))
        checks.assert_parity(Y.cpu(), Yo, oracle.block_fro(v), X.cpu(), A, torch.bfloat16,
                             checks.max_terms(c["brow"], c["b"]))


@pytest.mark.parametrize("b,d,n,geo", [(8, 1 / 8, 331, 2), (16, 1 / 16, 257, 2), (8, 1 / 16, 200, 1),
                                       (16, 1 / 4, 384, 1), (4, 1 / 8, 136, 2)])
def test_e4m3_two_column_tiles_equal_one(b, d, n, geo):
    """E4M3 plans whose CTAs cover two column tiles (col_tiles = 2: each
    stage's W tiles expanded once for both), with 3-D X maps (n a multiple of
    64) and 2-D ones (331, 257, 200, 136): bit for bit equal to one column
    tile per CTA (each accumulator column sees the same MMAs in the same
    order), and within the bars against the oracle."""
    c = _problem(990 + n, 1024, 4096, n, b, d)
    p2, codes, scales = _e4m3_plan(c, kernel="tc", stage_geometry=geo, col_tiles=2)
    p1, _, _ = _e4m3_plan(c, kernel="tc", stage_geometry=geo, col_tiles=1)
    assert p2.info()["col_tiles"] == 2 and p1.info()["col_tiles"] == 1
    X = _x(c, torch.bfloat16)
    Y2 = torch.full((c["m"], n), float("nan"), dtype=torch.bfloat16, device="cuda")
    p2.run(X, Y2)
    Y1 = p1.run(X)
    torch.cuda.synchronize()
    assert p2.status() == 0 and p1.status() == 0
    assert torch.equal(Y1, Y2)
    v = oracle.e4m3_block_values(codes.view(torch.uint8).numpy(), scales.numpy())
    Yo = oracle.spmm(c["m"], c["k"], b, c["brow"], c["bcol"], v, X.cpu())
    A = oracle.spmm(c["m"], c["k"], b, c["brow"], c["bcol"], np.abs(v), np.abs(oracle.to_f64(X.cpu())))
    checks.assert_parity(Y2.cpu(), Yo, oracle.block_fro(v), X.cpu(), A, torch.bfloat16,
                         checks.max_terms(c["brow"], b), u_w=2.0 ** -8)


def test_batch_with_two_column_tile_plans_equals_alone():
    """A batch mixing plans with two column tiles per CTA (n > 128), plans
    asking for two with n <= 128 (they run with one) and default plans: the
    two kinds run as two tensor-core launches, and each result is bit for
    bit the plan run alone."""
    spec = ((8, 1 / 8, 331, 2), (16, 1 / 16, 90, 2), (8, 1 / 16, 257, 0), (16, 1 / 8, 200, 2),
            (16, 1 / 16, 40, 0))
    cases = [_problem(1100 + i, 1024, 2048, n, b, d) for i, (b, d, n, _) in enumerate(spec)]
    plans, Xs, Ys, keep = [], [], [], []
    for c, (_, _, n, ct) in zip(cases, spec):
        p, codes, scales = _e4m3_plan(c, kernel="tc", col_tiles=ct)
        plans.append(p)
        keep.append((codes, scales))
        Xs.append(_x(c, torch.bfloat16))
        Ys.append(torch.full((c["m"], n), float("nan"), dtype=torch.bfloat16, device="cuda"))
    for _ in range(2):
        S.spmm_batch_run(plans, Xs, Ys)
    torch.cuda.synchronize()
    for c, p, X, Y, (codes, scales) in zip(cases, plans, Xs, Ys, keep):
        assert p.status() == 0
        alone = p.run(X)
        torch.cuda.synchronize()
        assert torch.equal(alone, Y)
        v = oracle.e4m3_block_values(codes.view(torch.uint8).numpy(), scales.numpy())
        Yo = oracle.spmm(c["m"], c["k"], c["b"], c["brow"], c["bcol"], v, X.cpu())
        A = oracle.spmm(c["m"], c["k"], c["b"], c["brow"], c["bcol"], np.abs(v),
                        np.abs(oracle.to_f64(X.cpu())))
        checks.assert_parity(Y.cpu(), Yo, oracle.block_fro(v), X.cpu(), A, torch.bfloat16,
                             checks.max_terms(c["brow"], c["b"]), u_w=2.0 ** -8)


def test_tuner_choice_applies_to_auto_plans():
    """spmm_tune times the candidates of a product's bucket and AUTO plans of
    that bucket then take the fastest; the tuned plan is still within the
    bars against the oracle."""
    S.spmm_tune_clear()
    assert S.spmm_tune_size() == 0
    c = _problem(970, 2048, 4096, 6, 8, 1 / 8)
    v = torch.from_numpy(c["vals"]).to(torch.bfloat16).cuda()
    codes, scales = S.quantize_e4m3(v)
    X = _x(c, torch.bfloat16)
    r = S.spmm_tune(c["m"], c["k"], c["b"], c["brow"], c["bcol"], codes.view(torch.uint8), X,
                    w_dtype=S.E4M3, x_dtype=S.BF16, scales=scales, reps=5)
    assert S.spmm_tune_size() == 1
    kinds = {q["kernel"] for q in r["candidates"]}
    # both stage geometries with the default groups and (m / 16 = 128 tile
    # rows: 8 groups of 16, too few for the SMs) with 16-row groups split
    # along k, and the block gather
    assert kinds == {"tc", "bgather"} and len(r["candidates"]) == 5
    split = [q for q in r["candidates"] if q["rows_per_group"] == 16]
    assert len(split) == 2 and all(q["k_splits"] >= 2 for q in split)
    ok = [q for q in r["candidates"] if q["us"] > 0]
    best = min(ok, key=lambda q: q["us"])
    assert r["kernel"] == best["kernel"] and r["best_us"] == best["us"]
    assert (r["rows_per_group"], r["k_splits"]) == (best["rows_per_group"], best["k_splits"])
    # a fresh AUTO plan in the same bucket (other values) takes the choice
    c2 = _problem(971, 2048, 4096, 5, 8, 1 / 8)
    p, codes2, scales2 = _e4m3_plan(c2)
    info = p.info()
    assert info["kernel"] == {"tc": 3, "bgather": 4}[r["kernel"]]
    if r["kernel"] == "tc":
        assert info["stage_geometry"] == r["stage_geometry"] - 1
        if r["rows_per_group"]:
            assert info["rows_per_group"] == 16 and info["n_reductions"] > 0
    X2 = _x(c2, torch.bfloat16)
    Y = p.run(X2)
    torch.cuda.synchronize()
    v2 = oracle.e4m3_block_values(codes2.view(torch.uint8).numpy(), scales2.numpy())
    Yo = oracle.spmm(c2["m"], c2["k"], 8, c2["brow"], c2["bcol"], v2, X2.cpu())
    assert oracle.normwise_err(Y.cpu(), Yo, oracle.block_fro(v2), X2.cpu()) <= 4e-3
    S.spmm_tune_clear()
    assert S.spmm_tune_size() == 0
