"""GPU parity of the CUDA-core block gather (BGATHER: small n, b in {4, 8,
16}, 16-bit or E4M3 weights) against the FP64 oracle, with the three bars
of checks.py; bit-exact on integer operands; the kernel choice of AUTO at
small n; its limits."""
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


def _x(X, dt, n):
    ld = max(((n + 7) // 8) * 8, 8)
    buf = torch.zeros((X.shape[0], ld), dtype=dt, device="cuda")
    buf[:, :n] = X.to(dt).cuda()
    return buf[:, :n]


@pytest.mark.parametrize("w8", [False, True])
@pytest.mark.parametrize("dt", [torch.float16, torch.bfloat16])
@pytest.mark.parametrize("b,n", [(16, 1), (16, 3), (16, 9), (16, 16), (8, 2), (8, 8), (8, 13),
                                 (4, 1), (4, 9), (4, 16)])
def test_bgather_parity(b, n, dt, w8):
    m, k = 528, 784                  # ragged against 128 (and, for b = 4 and 8, against 16)
    m, k = (m // b) * b, (k // b) * b
    c = wl.problem(3100 + b + n, m, k, n, b, (m // b) * (k // b) // 8)
    X = torch.from_numpy(c["X"]).to(dt)
    if w8:
        codes, scales = S.quantize_e4m3(torch.from_numpy(c["vals"]).to(dt).cuda())
        plan = S.Plan(m, k, n, b, w_dtype=S.E4M3, x_dtype=S.dtype_code(dt), brow=c["brow"],
                      bcol=c["bcol"], kernel="bgather")
        plan.pack(codes.view(torch.uint8), scales)
        v = oracle.e4m3_block_values(codes.cpu().view(torch.uint8).numpy(), scales.cpu().numpy())
    else:
        vt = torch.from_numpy(c["vals"]).to(dt)
        plan = S.Plan(m, k, n, b, w_dtype=S.dtype_code(dt), brow=c["brow"], bcol=c["bcol"],
                      kernel="bgather")
        plan.pack(vt.cuda())
        v = vt
    assert plan.info()["kernel"] == 4
    Y = torch.full((m, n), float("nan"), dtype=dt, device="cuda")
    plan.run(_x(X, dt, n), Y)
    torch.cuda.synchronize()
    assert plan.status() == 0
    Yo = oracle.spmm(m, k, b, c["brow"], c["bcol"], v, X)
    A = oracle.spmm(m, k, b, c["brow"], c["bcol"], np.abs(oracle.to_f64(v)),
                    np.abs(oracle.to_f64(X)))
    # E4M3 values are decoded and scaled in FP32 here (no 16-bit rounding of
    # code x scale): one FP32 rounding per value
    checks.assert_parity(Y.cpu(), Yo, oracle.block_fro(v), X, A, dt,
                         checks.max_terms(c["brow"], b), u_w=2.0 ** -24 if w8 else 0.0)


@pytest.mark.parametrize("b,dt", [(16, torch.float16), (8, torch.bfloat16), (4, torch.float16)])
def test_bgather_integers_exact_and_empty_rows(b, dt):
    """Integer operands: bit for bit; block rows without blocks are zero;
    X with a leading dimension that is not a multiple of 8 (the unaligned
    staging path)."""
    m, k, n = 512, 1024, 13
    c = wl.integer_problem(3200 + b, m, k, n, b, wl.nnzb_for(m, k, b, 1 / 8))
    keep = c["brow"] % 3 != 1                      # a third of the block rows empty
    brow, bcol, vals = c["brow"][keep], c["bcol"][keep], c["vals"][keep]
    plan = S.Plan(m, k, n, b, w_dtype=S.dtype_code(dt), brow=brow, bcol=bcol, kernel="bgather")
    assert plan.info()["kernel"] == 4
    plan.pack(torch.from_numpy(vals).to(dt).cuda())
    Y = torch.full((m, n), float("nan"), dtype=dt, device="cuda")
    Xd = torch.from_numpy(c["X"]).to(dt).cuda().contiguous()     # ldx = 13
    plan.run(Xd, Y)
    torch.cuda.synchronize()
    Yo = oracle.spmm(m, k, b, brow, bcol, vals, c["X"])
    assert torch.equal(Y.cpu(), torch.from_numpy(Yo).to(dt))


def test_bgather_transposed_and_row_slices():
    m, k, n, b = 256, 512, 12, 8   # n_max 12: AUTO picks BGATHER
    c = wl.integer_problem(3300, m, k, n, b, wl.nnzb_for(m, k, b, 1 / 4))
    vals = torch.from_numpy(c["vals"]).half().cuda()
    Yin = torch.from_numpy(c["X"][:m]).half().cuda()
    Z = torch.full((k, n), float("nan"), dtype=torch.float16, device="cuda")
    for rb, re in ((0, 256), (256, 512)):
        p = S.Plan(m, k, n, b, w_dtype=S.F16, brow=c["brow"], bcol=c["bcol"], transposed=True,
                   rows=(rb, re))
        assert p.info()["kernel"] == 4
        p.pack(vals)   # (the mixed batch of test_gpu_batched covers BGATHER beside TC)
        p.run(Yin, Z[rb:re])
    torch.cuda.synchronize()
    Zo = oracle.spmm_t(m, k, b, c["brow"], c["bcol"], c["vals"], c["X"][:m])
    assert torch.equal(Z.cpu(), torch.from_numpy(Zo).half())


def test_bgather_limits():
    with pytest.raises(S.SpmmError) as e:
        S.Plan(256, 256, 17, 16, w_dtype=S.F16, brow=[0], bcol=[0], kernel="bgather")
    assert e.value.status == S.ERR_UNSUPPORTED
    with pytest.raises(S.SpmmError) as e:
        S.Plan(256, 256, 16, 16, w_dtype=S.F16, mode=S.DYNAMIC, nnzb_max=8, kernel="bgather")
    assert e.value.status == S.ERR_UNSUPPORTED
    with pytest.raises(S.SpmmError) as e:
        S.Plan(256, 256, 16, 1, w_dtype=S.F16, brow=[0], bcol=[0], kernel="bgather")
    assert e.value.status == S.ERR_UNSUPPORTED
    # AUTO: the gather up to n_max = 16 for b = 8 (8 for b = 16), then the
    # tensor cores
    for b, n, kern in ((8, 16, 4), (8, 17, 3), (16, 8, 4), (16, 9, 3)):
        p = S.Plan(256, 256, n, b, w_dtype=S.F16, brow=[0], bcol=[0])
        assert p.info()["kernel"] == kern, (b, n)
