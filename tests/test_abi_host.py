"""C-ABI checks that need no GPU: the library loads and exports every entry
point of include/spmm.h, argument / shape / pattern errors come back as
status codes, and host-only static plans reproduce the oracle's integer plan
arrays bit for bit."""
import re

import numpy as np
import pytest

from oracle import plan as P
from paper_2303_16999_gb300 import spmm as S


@pytest.fixture(scope="module", autouse=True)
def native():
    from paper_2303_16999_gb300 import build
    build.build()
    return S.lib()


def test_exports_match_header():
    import os
    hdr = open(os.path.join(os.path.dirname(S.HERE), "include", "spmm.h")).read()
    declared = set(re.findall(r"\b(spmm_[a-z_0-9]+)\s*\(", hdr))
    declared = {d for d in declared if not d.endswith("_t")}
    assert declared == set(S.EXPORTS), declared ^ set(S.EXPORTS)
    L = S.lib()
    for name in declared:
        assert hasattr(L, name)
    assert "sm_103a" in S.spmm_version()
    shdr = open(os.path.join(os.path.dirname(S.HERE), "include", "spmm_serve.h")).read()
    sdecl = set(re.findall(r"\b(serve_[a-z_0-9]+)\s*\(", shdr))
    assert sdecl == set(S.SERVE_EXPORTS), sdecl ^ set(S.SERVE_EXPORTS)
    for name in sdecl:
        assert hasattr(L, name)


def test_appendix_formulas_match_oracle():
    for e, q in ((4096, 3), (4096, 4096), (9, 3), (10, 4), (7, 1), (0, 5)):
        assert S.spmm_equal_partition(e, q) == P.equal_partition(e, q)
    from fractions import Fraction
    for m, k, d, qm, qk in ((4096, 4096, Fraction(1, 16), 4, 4), (9, 9, Fraction(1, 3), 1, 3),
                            (10, 10, Fraction(1, 3), 1, 1), (8192, 8192, Fraction(1, 16), 7, 3)):
        assert S.spmm_bucket_size(m, k, d.numerator, d.denominator, qm, qk) == \
            P.bucket_size(m, k, d, qm, qk)


def _plan(m, k, b, brow, bcol, **kw):
    return S.Plan(m, k, kw.pop("n_max", 64), b, w_dtype=kw.pop("w_dtype", S.F16),
                  brow=brow, bcol=bcol, host_only=True, **kw)


def test_errors():
    with pytest.raises(S.SpmmError) as e:
        _plan(16, 16, 4, [4], [0])
    assert e.value.status == S.ERR_PATTERN
    with pytest.raises(S.SpmmError) as e:
        _plan(16, 16, 4, [1, 1], [2, 2])
    assert e.value.status == S.ERR_PATTERN
    with pytest.raises(S.SpmmError) as e:
        _plan(18, 16, 4, [0], [0])
    assert e.value.status == S.ERR_SHAPE
    with pytest.raises(S.SpmmError) as e:
        _plan(16, 16, 2, [0], [0])
    assert e.value.status == S.ERR_SHAPE
    with pytest.raises(S.SpmmError) as e:
        _plan(16, 16, 4, [0], [0], w_dtype=S.F16, kernel="plain")
    assert e.value.status == S.ERR_UNSUPPORTED
    with pytest.raises(S.SpmmError) as e:
        _plan(16, 16, 4, [0], [0], kernel="gather")
    assert e.value.status == S.ERR_UNSUPPORTED
    with pytest.raises(S.SpmmError) as e:
        _plan(24, 24, 4, [0], [0], kernel="tc")     # m, k not multiples of 16
    assert e.value.status == S.ERR_UNSUPPORTED
    for bad in (-1, 3):
        with pytest.raises(S.SpmmError) as e:
            _plan(16, 16, 4, [0], [0], col_tiles=bad)
        assert e.value.status == S.ERR_ARG
    for bad in (-1, 1025):
        with pytest.raises(S.SpmmError) as e:
            _plan(16, 16, 4, [0], [0], kernel="tc", k_splits=bad)
        assert e.value.status == S.ERR_ARG and "k_splits" in str(e.value)
    # the options a plan runs with are reported back
    q = _plan(64, 64, 4, [0, 5], [1, 3], kernel="tc", col_tiles=2, n_max=256)
    assert q.info()["col_tiles"] == 2
    assert _plan(64, 64, 4, [0], [1], kernel="tc").info()["col_tiles"] == 0
    # static b = 1 gather plans read 16-bit column indices while k <= 65536
    assert _plan(64, 65536, 1, [0, 3], [65535, 7], kernel="gather").info()["index_bytes"] == 2
    assert _plan(64, 65552, 1, [0], [65551], kernel="gather").info()["index_bytes"] == 4
    assert _plan(64, 64, 4, [0], [1], kernel="tc").info()["index_bytes"] == 4
    p = _plan(16, 16, 4, [], [])
    assert p.info()["nnzb"] == 0
    # the sampled product refuses host-only plans before touching the device
    with pytest.raises(S.SpmmError) as e:
        S.spmm_sddmm(p.h, None, 16, 8, 16, 8, 4, 16, S.F32, None)
    assert e.value.status == S.ERR_ARG


def test_int32_index_range_is_enforced():
    """Block indices, block-CSR offsets and tile slots are int32 on the
    device: shapes and block counts beyond that range are refused before any
    pattern array is read or any memory is allocated."""
    import ctypes
    big = 1 << 31
    opts = S.PlanOpts(host_only=1)
    tiny = np.zeros(1, np.int32)
    ptr = tiny.ctypes.data_as(ctypes.c_void_p)
    for m, k, nnzb in ((big, 16, 1), (16, big, 1), (16, 16, big)):
        with pytest.raises(S.SpmmError) as e:
            S.spmm_plan_create(m, k, 8, 1, S.STATIC, S.F16, S.F16,
                               S.Pattern(nnzb, ptr, ptr), 0, opts)
        assert e.value.status == S.ERR_SHAPE, (m, k, nnzb)
    with pytest.raises(S.SpmmError) as e:
        S.spmm_plan_create(256, 256, 8, 16, S.DYNAMIC, S.F16, S.F16, None, big, None)
    assert e.value.status == S.ERR_ARG


def test_sddmm_form_follows_density():
    """spmm_sddmm gathers blocks of 16 below a density of 1/13 and computes
    dense tiles otherwise (reported in the plan info)."""
    rng = np.random.default_rng(3)
    for b, d, form in ((16, 1 / 16, 1), (16, 1 / 8, 0), (16, 1 / 4, 0), (8, 1 / 32, 0), (1, 1 / 64, 0)):
        mb = kb = 512 // b
        brow, bcol = _rand(rng, mb, kb, int(d * mb * kb))
        assert _plan(512, 512, b, brow, bcol).info()["sddmm_form"] == form, (b, d)


def _rand(rng, mb, kb, nnzb):
    idx = rng.choice(mb * kb, nnzb, replace=False)
    o = rng.permutation(nnzb)
    return (idx // kb).astype(np.int32)[o], (idx % kb).astype(np.int32)[o]


@pytest.mark.parametrize("b", [1, 4, 8, 16])
def test_csr_bit_exact(b):
    rng = np.random.default_rng(20 + b)
    m = k = 256
    mb, kb = m // b, k // b
    for d in (0.0, 1 / 32, 1 / 4, 1.0):
        brow, bcol = _rand(rng, mb, kb, int(d * mb * kb))
        p = _plan(m, k, b, brow, bcol)
        rp, ci, pm = P.csr(mb, brow, bcol)
        assert np.array_equal(p.array("row_ptr"), rp)
        assert np.array_equal(p.array("col_idx"), ci)
        assert np.array_equal(p.array("perm"), pm)


def test_row_plan_bit_exact():
    rng = np.random.default_rng(3)
    for m, k, nnzb, C in ((512, 512, 9000, 0), (64, 4096, 30000, 50), (300, 300, 0, 0)):
        brow, bcol = _rand(rng, m, k, nnzb)
        p = _plan(m, k, 1, brow, bcol, max_per_item=C)
        info = p.info()
        rp, _, _ = P.csr(m, brow, bcol)
        want = P.row_plan(m, rp, info["max_per_item"], sort_items=True)
        assert np.array_equal(p.array("items").reshape(-1, 6), want["items"])
        assert np.array_equal(p.array("ws_row0"), want["ws_row0"])
        assert np.array_equal(p.array("red").reshape(-1, 3), want["red"])
        assert info["ws_rows"] == want["ws_rows"]


TC_KEYS = ["grp_row0", "grp_rows", "grp_ebeg", "ent_col", "ent_tbeg", "ent_cover", "tile_row",
           "blk_slot", "blk_off", "ws_row0"]


@pytest.mark.parametrize("b", [4, 8, 16])
def test_tc_plan_bit_exact(b):
    rng = np.random.default_rng(50 + b)
    cases = [(256, 256, 1 / 8, 0, 0, 64), (512, 256, 1 / 4, 5, 7, 300), (1024, 512, 1 / 32, 16, 0, 2048),
             (160, 96, 1 / 2, 3, 2, 16), (64, 64, 0.0, 0, 0, 8)]
    for m, k, d, R, C, nmax in cases:
        mb, kb = m // b, k // b
        brow, bcol = _rand(rng, mb, kb, int(d * mb * kb))
        p = _plan(m, k, b, brow, bcol, rows_per_group=R, max_per_item=C, n_max=nmax, kernel="tc")
        info = p.info()
        want = P.tc_plan(m, k, b, brow, bcol, info["rows_per_group"], info["max_per_item"],
                         groups=info["n_groups"])
        for key in TC_KEYS:
            assert np.array_equal(p.array(key), want[key]), key
        assert np.array_equal(p.array("items").reshape(-1, 6), want["items"])
        assert np.array_equal(p.array("red").reshape(-1, 3), want["red"])
        assert info["ws_rows"] == want["ws_rows"]
        assert info["n_tiles"] == len(want["tile_row"])


@pytest.mark.parametrize("b", [4, 8, 16])
def test_tc_plan_k_splits_bit_exact(b):
    """k_splits: every group's entries in about k_splits items of at most
    ceil(E / (G k_splits)) entries (E entries, G groups), every group with
    more entries than that split; the arrays bit for bit against the
    oracle's plan with that chunk size."""
    rng = np.random.default_rng(90 + b)
    for m, k, d, s in ((1024, 8192, 1 / 8, 19), (512, 4096, 1 / 16, 4), (256, 2048, 1 / 4, 1)):
        mb, kb = m // b, k // b
        brow, bcol = _rand(rng, mb, kb, int(d * mb * kb))
        p0 = _plan(m, k, b, brow, bcol, rows_per_group=16, kernel="tc")
        E, G = p0.info()["n_entries"], p0.info()["n_groups"]
        p = _plan(m, k, b, brow, bcol, rows_per_group=16, k_splits=s, kernel="tc")
        info = p.info()
        C = -(-E // (G * s))
        assert info["max_per_item"] == C and info["n_entries"] == E and info["n_groups"] == G
        want = P.tc_plan(m, k, b, brow, bcol, 16, C)
        for key in TC_KEYS:
            assert np.array_equal(p.array(key), want[key]), key
        assert np.array_equal(p.array("items").reshape(-1, 6), want["items"])
        assert np.array_equal(p.array("red").reshape(-1, 3), want["red"])
        ents = np.diff(p.array("grp_ebeg"))
        assert info["n_items"] == sum(-(-int(e) // C) if e > C else 1 for e in ents)


@pytest.mark.parametrize("b", [1, 4, 16])
def test_tc_plan_near_equal_groups_bit_exact(b):
    """Plans with an explicit group count: the tile rows in near-equal groups
    (the shape that fills the SMs with whole units), bit for bit against
    the oracle's plan, with and without split items."""
    rng = np.random.default_rng(70 + b)
    for m, k, d, q, C in ((4096, 512, 1 / 8, 19, 0), (1024, 768, 1 / 4, 5, 9), (272, 256, 1 / 4, 17, 0),
                          (528, 320, 1 / 16, 3, 0)):
        mb, kb = m // b, k // b
        brow, bcol = _rand(rng, mb, kb, int(d * mb * kb))
        p = _plan(m, k, b, brow, bcol, groups=q, max_per_item=C, kernel="tc")
        info = p.info()
        assert info["rows_per_group"] == 0 and info["n_groups"] == q
        rows = p.array("grp_rows")
        assert rows.sum() == m // 16 and rows.max() - rows.min() <= 1 and rows.max() <= 16
        want = P.tc_plan(m, k, b, brow, bcol, 0, info["max_per_item"], groups=q)
        for key in TC_KEYS:
            assert np.array_equal(p.array(key), want[key]), key
        assert np.array_equal(p.array("items").reshape(-1, 6), want["items"])
        assert np.array_equal(p.array("red").reshape(-1, 3), want["red"])


def test_groups_option_errors():
    brow, bcol = [0], [0]
    for q, extra in ((1, {}), (65, {}), (-1, {}), (8, {"rows_per_group": 4})):
        with pytest.raises(S.SpmmError) as e:
            _plan(1024, 64, 16, brow, bcol, groups=q, kernel="tc", **extra)
        assert e.value.status == S.ERR_ARG, q


def test_tc_plan_worst_case_splits():
    # Appendix A.2 worst case: every block in one tile row -> that group splits
    m = k = 1024
    b = 16
    brow = np.zeros(64, np.int32)
    bcol = np.arange(64, dtype=np.int32)
    p = _plan(m, k, b, brow, bcol, n_max=256)
    info = p.info()
    want = P.tc_plan(m, k, b, brow, bcol, info["rows_per_group"], info["max_per_item"],
                         groups=info["n_groups"])
    assert np.array_equal(p.array("items").reshape(-1, 6), want["items"])
    assert info["n_reductions"] == 1 and info["ws_rows"] > 0


def test_auto_kernel_choice_for_b1():
    """b = 1 with 16-bit values: the tensor-core kernel when n_max >= 128 and
    the tiles hold at least 4 non-zeros on average, else the gather kernel."""
    rng = np.random.default_rng(0)
    brow, bcol = _rand(rng, 512, 512, 512 * 512 // 8)        # ~32 per 16 x 16 tile
    p = _plan(512, 512, 1, brow, bcol, n_max=256)
    assert p.info()["kernel"] == S.KERNEL_TC
    p = _plan(512, 512, 1, brow, bcol, n_max=64)
    assert p.info()["kernel"] == S.KERNEL_GATHER
    brow, bcol = _rand(rng, 512, 512, 300)                     # about one per tile
    p = _plan(512, 512, 1, brow, bcol, n_max=256)
    assert p.info()["kernel"] == S.KERNEL_GATHER
    p = _plan(512, 512, 1, brow, bcol, n_max=256, kernel="tc")
    assert p.info()["kernel"] == S.KERNEL_TC
    want = P.tc_plan(512, 512, 1, brow, bcol, p.info()["rows_per_group"], p.info()["max_per_item"],
                     groups=p.info()["n_groups"])
    assert np.array_equal(p.array("ent_cover"), want["ent_cover"])
    assert np.array_equal(p.array("blk_slot"), want["blk_slot"])


@pytest.mark.parametrize("b", [1, 8, 16])
def test_transposed_plan_is_the_plan_of_w_transpose(b):
    """A transposed plan of W (m x k) is the plan of W^T (k x m): its CSR and
    tile plan equal the oracle's for the swapped pattern, and it reports the
    swapped shape."""
    rng = np.random.default_rng(70 + b)
    m, k = 512, 256
    brow, bcol = _rand(rng, m // b, k // b, (m // b) * (k // b) // 8)
    p = _plan(m, k, b, brow, bcol, n_max=256, transposed=True, kernel="tc")
    info = p.info()
    assert (info["m"], info["k"], p.m, p.k) == (k, m, k, m)
    rp, ci, pm = P.csr(k // b, bcol, brow)
    assert np.array_equal(p.array("row_ptr"), rp)
    assert np.array_equal(p.array("col_idx"), ci)
    assert np.array_equal(p.array("perm"), pm)
    want = P.tc_plan(k, m, b, bcol, brow, info["rows_per_group"], info["max_per_item"],
                     groups=info["n_groups"])
    for key in TC_KEYS:
        assert np.array_equal(p.array(key), want[key]), key
    assert np.array_equal(p.array("items").reshape(-1, 6), want["items"])


@pytest.mark.parametrize("b", [4, 16])
def test_transposed_plan_with_near_equal_groups(b):
    """A transposed plan with an explicit group count splits W^T's tile rows
    (W's tile columns) into near-equal groups, as the oracle's plan of W^T."""
    rng = np.random.default_rng(90 + b)
    m, k, q = 256, 1024, 11
    brow, bcol = _rand(rng, m // b, k // b, (m // b) * (k // b) // 8)
    p = _plan(m, k, b, brow, bcol, n_max=256, transposed=True, kernel="tc", groups=q)
    info = p.info()
    assert info["n_groups"] == q and info["rows_per_group"] == 0
    want = P.tc_plan(k, m, b, bcol, brow, 0, info["max_per_item"], groups=q)
    for key in TC_KEYS:
        assert np.array_equal(p.array(key), want[key]), key
    assert np.array_equal(p.array("items").reshape(-1, 6), want["items"])


def test_ell_layout_of_a_pattern():
    """workloads.to_ell, the Blocked-ELL layout the ELL tests and benchmark
    feed spmm_run_ell: every block appears once in its row, columns ascend,
    -1 padding follows the blocks, src maps each slot back to the pattern."""
    from paper_2303_16999_gb300 import workloads as wl
    rng = np.random.default_rng(12)
    mb, kb = 40, 30
    brow, bcol = _rand(rng, mb, kb, 300)
    cols, src = wl.to_ell(brow, bcol, mb)
    counts = np.bincount(brow, minlength=mb)
    assert cols.shape == (mb, counts.max())
    for r in range(mb):
        c = cols[r]
        nv = counts[r]
        assert np.all(c[nv:] == -1) and np.all(c[:nv] >= 0)
        assert np.all(np.diff(c[:nv]) > 0)
        assert np.array_equal(np.sort(bcol[brow == r]), c[:nv])
        assert np.all(brow[src[r, :nv]] == r) and np.array_equal(bcol[src[r, :nv]], c[:nv])
        assert np.all(src[r, nv:] == -1)
    wide, _ = wl.to_ell(brow, bcol, mb, width=counts.max() + 3)
    assert wide.shape[1] == counts.max() + 3 and np.all(wide[:, -3:] == -1)
