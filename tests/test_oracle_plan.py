"""Pins of the oracle's integer plan rules (CPU only).

Closed forms from Appendix A.2's equal partition, brute force on small
patterns (dense masks), invariants, and the two extreme cases Appendix A.2
describes (balanced, and everything in one partition).
"""
import math

import numpy as np
import pytest

from oracle import plan as P


def _rand_pattern(rng, mb, kb, nnzb):
    idx = rng.choice(mb * kb, nnzb, replace=False)
    return (idx // kb).astype(np.int32), (idx % kb).astype(np.int32)


# ------------------------------------------------------ Appendix A.2 -------
def test_equal_partition_closed_forms():
    assert P.equal_partition(4096, 3) == [1365, 1365, 1366]
    assert P.equal_partition(4096, 4096) == [1] * 4096
    assert P.equal_partition(9, 3) == [3, 3, 3]          # Fig. 1: m = k = 9, q^k = 3
    assert P.equal_partition(10, 4) == [2, 2, 2, 4]
    assert P.equal_partition(7, 1) == [7]


def test_bucket_size_closed_forms():
    # N_nz = m k d_max / (q^m q^k)
    assert P.bucket_size(4096, 4096, 1 / 16, 4, 4) == 65536
    assert P.bucket_size(9, 9, 1 / 3, 1, 3) == 9
    assert P.bucket_size(10, 10, 1 / 3, 1, 1) == 34       # 33.3.. rounded up


def test_group_partition_brute_force():
    for mt in range(1, 80):
        for R in range(1, 34):
            sizes = P.group_partition(mt, R)
            assert sum(sizes) == mt and max(sizes) <= R and min(sizes) >= 1
            # the smallest q >= ceil(mt/R) whose equal partition fits
            q = next(q for q in range(-(-mt // R), mt + 1)
                     if max(P.equal_partition(mt, q)) <= R)
            assert sizes == P.equal_partition(mt, q)


def test_chunk_sizes():
    assert P.chunk_sizes(0, 4) == [0]
    assert P.chunk_sizes(4, 4) == [4]
    assert P.chunk_sizes(5, 4) == [3, 2]
    assert P.chunk_sizes(10, 3) == [3, 3, 2, 2]
    for L in range(0, 60):
        for C in range(1, 12):
            s = P.chunk_sizes(L, C)
            assert sum(s) == L and max(s) <= max(C, 0 if L == 0 else 1) or L == 0
            assert max(s) - min(s) <= 1 and len(s) == max(1, math.ceil(L / C))


# ---------------------------------------------------------- checks ---------
def test_validate():
    assert P.validate(16, 16, 4, [0, 3], [3, 0]) == P.OK
    assert P.validate(16, 16, 4, [4], [0]) == P.ERR_PATTERN
    assert P.validate(16, 16, 4, [0], [-1]) == P.ERR_PATTERN
    assert P.validate(16, 16, 4, [1, 1], [2, 2]) == P.ERR_PATTERN
    assert P.validate(18, 16, 4, [0], [0]) == P.ERR_SHAPE
    assert P.validate(16, 16, 2, [0], [0]) == P.ERR_SHAPE
    assert P.validate(16, 16, 4, [], []) == P.OK


# ------------------------------------------------------------- CSR ---------
def test_csr_brute_force():
    rng = np.random.default_rng(1)
    for mb, kb, nnzb in ((8, 8, 20), (17, 5, 40), (3, 30, 0), (1, 64, 64)):
        brow, bcol = _rand_pattern(rng, mb, kb, nnzb)
        row_ptr, col_idx, perm = P.csr(mb, brow, bcol)
        mask = np.zeros((mb, kb), bool)
        mask[brow, bcol] = True
        assert row_ptr[0] == 0 and row_ptr[-1] == nnzb
        for r in range(mb):
            cols = col_idx[row_ptr[r]:row_ptr[r + 1]]
            assert list(cols) == list(np.nonzero(mask[r])[0])
        assert np.array_equal(brow[perm], np.repeat(np.arange(mb), np.diff(row_ptr)))
        assert np.array_equal(bcol[perm], col_idx)


def test_csr_order_invariance():
    rng = np.random.default_rng(2)
    brow, bcol = _rand_pattern(rng, 12, 9, 50)
    a = P.csr(12, brow, bcol)
    o = rng.permutation(50)
    b = P.csr(12, brow[o], bcol[o])
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(o[b[2]], a[2])  # perm re-mapped through the shuffle


# ------------------------------------------------- b = 1 row items ---------
def _check_row_plan(mb, row_ptr, C1, pl, sort_items):
    items = pl["items"]
    covered = np.zeros(row_ptr[-1], int)
    rows_seen = set()
    for g, beg, end, ch, nch, ws in items:
        rows_seen.add(g)
        assert row_ptr[g] <= beg <= end <= row_ptr[g + 1]
        assert end - beg <= max(C1, 0)
        covered[beg:end] += 1
        assert (ws >= 0) == (nch > 1)
    assert rows_seen == set(range(mb))
    assert np.all(covered == 1)
    # chunks of a row are contiguous and in order
    for r in range(mb):
        its = sorted((it for it in items if it[0] == r), key=lambda it: it[3])
        assert its[0][1] == row_ptr[r] and its[-1][2] == row_ptr[r + 1]
        for a, b in zip(its, its[1:]):
            assert a[2] == b[1]
    cost = items[:, 2] - items[:, 1]
    if sort_items:
        keys = list(zip(-cost, items[:, 0], items[:, 3]))
        assert keys == sorted(keys)
    else:
        keys = list(zip(items[:, 0], items[:, 3]))
        assert keys == sorted(keys)


@pytest.mark.parametrize("sort_items", [True, False])
def test_row_plan_invariants(sort_items):
    rng = np.random.default_rng(4)
    for mb, kb, nnzb, C1 in ((16, 64, 300, 8), (40, 40, 0, 4), (5, 100, 400, 30)):
        brow, bcol = _rand_pattern(rng, mb, kb, nnzb)
        row_ptr, _, _ = P.csr(mb, brow, bcol)
        pl = P.row_plan(mb, row_ptr, C1, sort_items)
        _check_row_plan(mb, row_ptr, C1, pl, sort_items)


def test_row_plan_extremes():
    # balanced (Appendix A.2 best case): every row holds the same count <= C1
    mb, kb = 8, 8
    brow = np.repeat(np.arange(mb), 2).astype(np.int32)
    bcol = np.tile([1, 5], mb).astype(np.int32)
    row_ptr, _, _ = P.csr(mb, brow, bcol)
    pl = P.row_plan(mb, row_ptr, 4)
    assert len(pl["items"]) == mb and pl["ws_rows"] == 0
    # worst case: everything in one row, which must be split
    brow = np.zeros(64, np.int32)
    bcol = np.arange(64, dtype=np.int32)
    row_ptr, _, _ = P.csr(4, brow, bcol)
    pl = P.row_plan(4, row_ptr, 10)
    assert len(pl["items"]) == 7 + 3
    assert pl["ws_rows"] == 7 and pl["red"].tolist() == [[0, 0, 7]]
    _check_row_plan(4, row_ptr, 10, pl, True)


# --------------------------------------------- tensor-core tile plan -------
def _brute_tc(m, k, b, brow, bcol, R):
    """Distinct tiles and per-group distinct tile columns from a dense mask."""
    mt, kt = m // 16, k // 16
    tmask = np.zeros((mt, kt), bool)
    for r, c in zip(brow, bcol):
        tmask[r * b // 16, c * b // 16] = True
    sizes = P.group_partition(mt, R)
    starts = np.cumsum([0] + sizes)
    ents = []
    for g in range(len(sizes)):
        sub = tmask[starts[g]:starts[g + 1]]
        ents.append(list(np.nonzero(sub.any(axis=0))[0]))
    return tmask, sizes, ents


def _check_tc_plan(m, k, b, brow, bcol, R, C, pl, sort_items, pad=None):
    pad = sort_items if pad is None else pad
    tmask, sizes, ents = _brute_tc(m, k, b, brow, bcol, R)
    assert list(pl["grp_rows"]) == sizes
    assert list(pl["grp_row0"]) == list(np.cumsum([0] + sizes)[:-1])
    flat = [c for e in ents for c in e]
    assert list(pl["ent_col"]) == flat
    assert list(np.diff(pl["grp_ebeg"])) == [len(e) for e in ents]
    assert pl["ent_tbeg"][-1] == len(pl["tile_row"])
    # each entry's slots: its real tile rows, plus (padded plans only) the
    # rows inside each covering interval, ascending, one slot per row
    for g in range(len(sizes)):
        for e in range(pl["grp_ebeg"][g], pl["grp_ebeg"][g + 1]):
            rows = list(pl["tile_row"][pl["ent_tbeg"][e]:pl["ent_tbeg"][e + 1]])
            col = pl["ent_col"][e]
            real = list(np.nonzero(tmask[pl["grp_row0"][g]:pl["grp_row0"][g] + sizes[g], col])[0])
            cov = pl["ent_cover"][e] & 0xFFFF
            starts = (pl["ent_cover"][e] >> 16) & 0xFFFF
            assert rows == sorted(rows) and len(set(rows)) == len(rows)
            assert set(real) <= set(rows) and cov == sum(1 << int(r) for r in rows)
            if not pad:
                assert rows == real and starts == cov
            # intervals: maximal runs split at start bits; each starts and ends on a real row
            ivs = []
            for r in rows:
                if (starts >> r) & 1:
                    ivs.append([r, r])
                else:
                    assert ivs and ivs[-1][1] == r - 1
                    ivs[-1][1] = r
            for a, z in ivs:
                assert a in real and z in real
            assert sum(P.mma_cost(z - a + 1) for a, z in ivs) == \
                _best_cover_cost(real) if pad else True
    # items cover every entry exactly once, every group has an item
    cover = np.zeros(len(flat), int)
    for g, beg, end, ch, nch, ws in pl["items"]:
        assert pl["grp_ebeg"][g] <= beg <= end <= pl["grp_ebeg"][g + 1]
        assert end - beg <= C or (nch == 1 and end - beg <= C)
        cover[beg:end] += 1
        assert (ws >= 0) == (nch > 1)
    assert np.all(cover == 1)
    assert set(pl["items"][:, 0]) == set(range(len(sizes)))
    # every block lands in the slot of its entry and row, at its offset
    for p in range(len(brow)):
        s = pl["blk_slot"][p]
        tr = brow[p] * b // 16
        g = int(np.searchsorted(pl["grp_row0"], tr, side="right") - 1)
        assert pl["tile_row"][s] == tr - pl["grp_row0"][g]
        e = int(np.searchsorted(pl["ent_tbeg"], s, side="right") - 1)
        assert pl["ent_col"][e] == bcol[p] * b // 16
        assert pl["blk_off"][p] == (brow[p] * b % 16) * 16 + bcol[p] * b % 16
    cost = [pl["ent_tbeg"][it[2]] - pl["ent_tbeg"][it[1]] + it[2] - it[1] for it in pl["items"]]
    if sort_items:
        keys = list(zip([-c for c in cost], pl["items"][:, 0], pl["items"][:, 3]))
    else:
        keys = list(zip(pl["items"][:, 0], pl["items"][:, 3]))
    assert keys == sorted(keys)


def _best_cover_cost(rows):
    """Brute force over every split of the sorted rows into consecutive runs."""
    n = len(rows)
    best = None
    for cuts in range(1 << max(n - 1, 0)):
        c, a = 0, 0
        for i in range(1, n + 1):
            if i == n or (cuts >> (i - 1)) & 1:
                c += P.mma_cost(rows[i - 1] - rows[a] + 1)
                a = i
        best = c if best is None else min(best, c)
    return best


def test_cover_intervals_brute_force():
    rng = np.random.default_rng(8)
    assert P.cover_intervals([3]) == [(3, 1)]
    assert P.cover_intervals([0, 15]) == [(0, 1), (15, 1)]       # 42 < mma_cost(16) = 80
    assert P.cover_intervals([0, 1, 2, 3]) == [(0, 4)]           # 24 < 4 * 21
    for _ in range(400):
        rows = sorted(rng.choice(16, size=rng.integers(1, 17), replace=False).tolist())
        ivs = P.cover_intervals(rows)
        assert sum(P.mma_cost(L) for _, L in ivs) == _best_cover_cost(rows)
        covered = [r for a, L in ivs for r in range(a, a + L)]
        assert set(rows) <= set(covered) and covered == sorted(covered)


@pytest.mark.parametrize("b", [4, 8, 16])
@pytest.mark.parametrize("sort_items", [True, False])
def test_tc_plan_invariants(b, sort_items):
    rng = np.random.default_rng(100 + b)
    for m, k, d, R, C in ((256, 256, 1 / 8, 4, 5), (512, 256, 1 / 4, 16, 1000),
                          (160, 96, 1 / 2, 3, 2), (64, 64, 0.0, 2, 3)):
        mb, kb = m // b, k // b
        brow, bcol = _rand_pattern(rng, mb, kb, int(d * mb * kb))
        pl = P.tc_plan(m, k, b, brow, bcol, R, C, sort_items)
        _check_tc_plan(m, k, b, brow, bcol, R, C, pl, sort_items)
        pl = P.tc_plan(m, k, b, brow, bcol, R, C, sort_items, pad=not sort_items)
        _check_tc_plan(m, k, b, brow, bcol, R, C, pl, sort_items, pad=not sort_items)


def test_tc_plan_extremes():
    # everything in one tile row (Appendix A.2 worst case): that group splits
    m = k = 512
    b = 16
    brow = np.zeros(32, np.int32)
    bcol = np.arange(32, dtype=np.int32)
    pl = P.tc_plan(m, k, b, brow, bcol, R=8, C=5)
    _check_tc_plan(m, k, b, brow, bcol, 8, 5, pl, True)
    assert pl["red"].tolist() == [[0, 0, 7]]
    assert pl["ws_rows"] == 7 * 8 * 16
    # balanced: each group holds the same number of entries, no split
    brow = np.repeat(np.arange(32), 2).astype(np.int32)
    bcol = np.tile([0, 17], 32).astype(np.int32)
    pl = P.tc_plan(m, k, b, brow, bcol, R=8, C=5)
    assert pl["ws_rows"] == 0 and len(pl["items"]) == 4


def test_tile_values():
    brow = np.array([0, 3], np.int32)
    bcol = np.array([1, 2], np.int32)
    vals = np.arange(2 * 16, dtype=np.float32).reshape(2, 4, 4)
    pl = P.tc_plan(16, 16, 4, brow, bcol, 1, 4)
    t = P.tile_values(4, 1, pl["blk_slot"], pl["blk_off"], vals)
    assert np.array_equal(t[0, 0:4, 4:8], vals[0])
    assert np.array_equal(t[0, 12:16, 8:12], vals[1])
    assert t[0].sum() == vals.sum()


@pytest.mark.parametrize("mt,q", [(256, 19), (256, 16), (17, 17), (100, 7), (5, 1)])
def test_near_equal_groups(mt, q):
    """q groups covering every tile row once, sizes within one of each
    other, larger groups first."""
    g = P.near_equal_groups(mt, q)
    assert len(g) == q and sum(g) == mt
    assert max(g) - min(g) <= 1
    assert g == sorted(g, reverse=True)
