"""GPU parity of row-slice plans (the per-GPU share of a product split by
rows of W, X replicated): one GPU runs every slice's plan in turn, each
writing its rows of one Y, and the whole Y must equal the oracle's product
bit for bit on integer operands (and within the bars on random ones).  The
slices get the whole W's pattern and values; each plan keeps its blocks and
gathers their values."""
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


@pytest.mark.parametrize("b,kernel,dt", [(16, "auto", torch.float16), (8, "auto", torch.bfloat16),
                                         (4, "tc", torch.float16), (1, "gather", torch.float16),
                                         (1, "tc", torch.bfloat16), (4, "plain", torch.float32)])
@pytest.mark.parametrize("workers", [2, 3])
def test_row_slices_integers_exact(b, kernel, dt, workers):
    m, k, n = 1024, 768, 136
    c = wl.integer_problem(7700 + b, m, k, n, b, wl.nnzb_for(m, k, b, 1 / 8))
    vals = torch.from_numpy(c["vals"]).to(dt).cuda()
    X = torch.from_numpy(c["X"]).to(dt).cuda()
    Y = torch.full((m, n), float("nan"), dtype=dt, device="cuda")
    plans = []
    for rb, re in P.row_split(m, b, workers):
        p = S.Plan(m, k, n, b, w_dtype=S.dtype_code(dt), brow=c["brow"], bcol=c["bcol"],
                   kernel=kernel, rows=(rb, re))
        p.pack(vals)
        p.run(X, Y[rb:re])
        plans.append(p)
    torch.cuda.synchronize()
    for p in plans:
        assert p.status() == 0
    Yo = oracle.spmm(m, k, b, c["brow"], c["bcol"], c["vals"], c["X"])
    assert torch.equal(Y.cpu(), torch.from_numpy(Yo).to(dt))


def test_row_slices_e4m3_and_values_at_run():
    """E4M3 weights with per-block scales: each slice gathers its blocks'
    codes and scales from the whole arrays; values passed to run() (not
    packed beforehand) take the same path."""
    m, k, n, b = 2048, 1024, 96, 16
    c = wl.problem(7800, m, k, n, b, wl.nnzb_for(m, k, b, 1 / 8))
    codes, scales = S.quantize_e4m3(torch.from_numpy(c["vals"]).bfloat16().cuda())
    X = torch.from_numpy(c["X"]).bfloat16().cuda()
    Y = torch.full((m, n), float("nan"), dtype=torch.bfloat16, device="cuda")
    for rb, re in P.row_split(m, b, 2):
        p = S.Plan(m, k, n, b, w_dtype=S.E4M3, x_dtype=S.BF16, brow=c["brow"], bcol=c["bcol"],
                   rows=(rb, re))
        p.run(X, Y[rb:re], values=codes.view(torch.uint8), scales=scales)
        torch.cuda.synchronize()
        assert p.status() == 0
        p.close()
    v = oracle.e4m3_block_values(codes.cpu().view(torch.uint8).numpy(), scales.cpu().numpy())
    Yo = oracle.spmm(m, k, b, c["brow"], c["bcol"], v, X.cpu())
    A = oracle.spmm(m, k, b, c["brow"], c["bcol"], np.abs(v), np.abs(oracle.to_f64(X.cpu())))
    checks.assert_parity(Y.cpu(), Yo, oracle.block_fro(v), X.cpu(), A, torch.bfloat16,
                         checks.max_terms(c["brow"], b), u_w=2.0 ** -8)


def test_row_slices_transposed():
    """A transposed plan's slice is a slice of Z = W^T.Y's rows (columns of W)."""
    m, k, n, b = 512, 1024, 64, 8
    c = wl.integer_problem(7900, m, k, n, b, wl.nnzb_for(m, k, b, 1 / 8))
    vals = torch.from_numpy(c["vals"]).half().cuda()
    Yin = torch.from_numpy(c["X"][:m]).half().cuda()          # any m x n integer operand
    Z = torch.full((k, n), float("nan"), dtype=torch.float16, device="cuda")
    for rb, re in P.row_split(k, b, 2):
        p = S.Plan(m, k, n, b, w_dtype=S.F16, brow=c["brow"], bcol=c["bcol"], transposed=True,
                   rows=(rb, re))
        p.pack(vals)
        p.run(Yin, Z[rb:re])
        torch.cuda.synchronize()
        assert p.status() == 0
    Zo = oracle.spmm_t(m, k, b, c["brow"], c["bcol"], c["vals"], c["X"][:m])
    assert torch.equal(Z.cpu(), torch.from_numpy(Zo).half())
