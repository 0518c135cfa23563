"""Integer plan and partition rules, written plainly (test infrastructure only).

This module states, in slow obvious Python, every integer array the GPU
library builds: the pattern checks, the canonical block-CSR, the equal
partition of Appendix A.2, and the work decomposition that the library uses
in place of the paper's tile partitions (Section 3.2 balances non-zeros over
unequal splits; Section 3.3 / Appendix A.2 uses equal splits with fixed
buckets).  The library's host planner (static mode) and its device
re-partition kernels (dynamic mode) must reproduce these arrays bit for bit.

All arrays are returned as numpy int32 (int64 where noted).

Readings of the paper that these rules rest on (the paper is silent here):
* pattern entries must be in range and unique; anything else is an error;
* m and k must be multiples of b;
* the tensor-core decomposition works on a 16 x 16 tile grid: a b x b block
  (b in {4, 8, 16}) lies inside exactly one 16 x 16 tile;
* long rows / long tile-row groups are split into near-equal chunks, the
  analogue of the unequal k-splits of Section 3.2, and the chunks' partial
  results are summed in chunk order (the cross-tile reduction of Section 3.2
  and the reduction over q^k of Appendix A.2).
"""
from fractions import Fraction
import math

import numpy as np

TILE = 16
BLOCK_SIZES = (1, 4, 8, 16)

OK, ERR_SHAPE, ERR_PATTERN = "ok", "shape", "pattern"


# ---------------------------------------------------------------- checks ----
def validate(m, k, b, brow, bcol):
    """Section 3: Mhat is a ceil(m/b) x ceil(k/b) block mask; this library
    requires b in {1, 4, 8, 16} (Section 3.1) and m, k multiples of b.
    Returns OK, ERR_SHAPE or ERR_PATTERN (out-of-range or repeated block)."""
    if b not in BLOCK_SIZES or m <= 0 or k <= 0 or m % b or k % b:
        return ERR_SHAPE
    mb, kb = m // b, k // b
    seen = set()
    for r, c in zip(list(brow), list(bcol)):
        r, c = int(r), int(c)
        if not (0 <= r < mb and 0 <= c < kb):
            return ERR_PATTERN
        if (r, c) in seen:
            return ERR_PATTERN
        seen.add((r, c))
    return OK


# ------------------------------------------------------------------- CSR ----
def csr(mb, brow, bcol):
    """Canonical block-CSR: slots ordered by (block row, block column).

    row_ptr[r] = number of blocks with block row < r (length mb + 1);
    col_idx[s] = block column of slot s; perm[s] = user index of slot s."""
    nnzb = len(brow)
    order = sorted(range(nnzb), key=lambda p: (int(brow[p]), int(bcol[p])))
    row_ptr = np.zeros(mb + 1, dtype=np.int32)
    for p in range(nnzb):
        row_ptr[int(brow[p]) + 1] += 1
    for r in range(mb):
        row_ptr[r + 1] += row_ptr[r]
    col_idx = np.array([int(bcol[p]) for p in order], dtype=np.int32)
    perm = np.array(order, dtype=np.int32)
    return row_ptr, col_idx, perm


# ------------------------------------------------------- Appendix A.2 ------
def equal_partition(m, q):
    """Appendix A.2: q - 1 parts of floor(m / q) and a last part of
    m - (q - 1) * floor(m / q)."""
    if q <= 0:
        raise ValueError("q must be positive")
    base = m // q
    return [base] * (q - 1) + [m - (q - 1) * base]


def bucket_size(m, k, d_max, q_m, q_k):
    """Appendix A.2: N_nz = m * k * d_max / (q^m * q^k), rounded up to an
    integer (the paper does not say how a fractional bucket is rounded)."""
    return math.ceil(Fraction(m) * k * Fraction(d_max) / (q_m * q_k))


def group_partition(mt, R):
    """Tile-row groups: the equal partition of Appendix A.2 applied to the mt
    tile rows, with the smallest q >= ceil(mt / R) whose largest (last) part
    holds at most R tile rows."""
    if mt == 0:
        return []
    q = -(-mt // R)
    while mt - (q - 1) * (mt // q) > R:
        q += 1
    return equal_partition(mt, q)


def near_equal_groups(mt, q):
    """Tile-row groups of a plan built with an explicit group count q: mt
    rows in q groups whose sizes differ by at most one, the larger first."""
    base, rem = divmod(mt, q)
    return [base + (1 if i < rem else 0) for i in range(q)]


def chunk_sizes(L, C):
    """Splits a list of L work units into ceil(L / C) near-equal chunks (one
    chunk when L <= C); the first L mod q chunks get one unit more."""
    q = 1 if L <= C else -(-L // C)
    base, rem = divmod(L, q)
    return [base + (1 if i < rem else 0) for i in range(q)]


def _assign_ws(items, rows_of):
    """Partial-result workspace slots for split items: in (group, chunk)
    order, slot s starts at row ws_row0[s] (rows counted in Y rows)."""
    split = sorted((it for it in items if it["nch"] > 1),
                   key=lambda it: (it["grp"], it["chunk"]))
    row = 0
    ws_row0 = []
    for s, it in enumerate(split):
        it["ws"] = s
        ws_row0.append(row)
        row += rows_of(it["grp"])
    for it in items:
        it.setdefault("ws", -1)
    return np.array(ws_row0, dtype=np.int64), row


def _items_array(items):
    a = np.zeros((len(items), 6), dtype=np.int32)
    for i, it in enumerate(items):
        a[i] = (it["grp"], it["beg"], it["end"], it["chunk"], it["nch"], it["ws"])
    return a


def _reductions(items):
    """Split groups to reduce: (group, first ws slot, number of chunks)."""
    red = {}
    for it in items:
        if it["nch"] > 1:
            g = it["grp"]
            s0, n = red.get(g, (1 << 30, 0))
            red[g] = (min(s0, it["ws"]), n + 1)
    return np.array([(g, s0, n) for g, (s0, n) in sorted(red.items())],
                    dtype=np.int32).reshape(-1, 3)


# ------------------------------------------------- b = 1 row work items ----
def row_plan(mb, row_ptr, C1, sort_items=True):
    """Work items of the b = 1 gather kernel: one item per block row, a row
    longer than C1 blocks split by ``chunk_sizes``; an empty row is one
    zero-fill item.  Static plans order items by cost (blocks) descending,
    ties by (row, chunk); dynamic plans keep (row, chunk) order."""
    items = []
    for r in range(mb):
        beg, end = int(row_ptr[r]), int(row_ptr[r + 1])
        sizes = chunk_sizes(end - beg, C1)
        s = beg
        for ci, sz in enumerate(sizes):
            items.append(dict(grp=r, beg=s, end=s + sz, chunk=ci,
                              nch=len(sizes), cost=sz))
            s += sz
    if sort_items:
        items.sort(key=lambda it: (-it["cost"], it["grp"], it["chunk"]))
    ws_row0, ws_rows = _assign_ws(items, lambda g: 1)
    return dict(items=_items_array(items), ws_row0=ws_row0, ws_rows=ws_rows,
                red=_reductions(items))


# ---------------------------------------- b >= 4 tensor-core work items ----
def mma_cost(L):
    """Cost, in units of two SM cycles, of one tensor-core product covering L
    consecutive tile rows (N = 16 L): at least 40 cycles to issue, 8 cycles per
    16 rows, plus one unit per tile slot moved through shared memory."""
    return max(20, 4 * L) + L


def cover_intervals(rows):
    """Cheapest cover of an entry's tile rows (ascending) by intervals of
    consecutive rows under ``mma_cost``; rows inside an interval without a
    tile become zero tiles.  Exact DP over the rows; on ties the earliest
    split point wins.  Returns [(start row, length), ...] ascending."""
    n = len(rows)
    dp = [0] + [None] * n
    arg = [0] * (n + 1)
    for j in range(1, n + 1):
        for i in range(j):
            c = dp[i] + mma_cost(rows[j - 1] - rows[i] + 1)
            if dp[j] is None or c < dp[j]:
                dp[j], arg[j] = c, i
    out, j = [], n
    while j > 0:
        i = arg[j]
        out.append((rows[i], rows[j - 1] - rows[i] + 1))
        j = i
    return out[::-1]


def tc_plan(m, k, b, brow, bcol, R, C, sort_items=True, pad=None, groups=None):
    """Decomposition of the tensor-core kernel.

    * Each b x b block lies in 16 x 16 tile (tr, tc) = (brow*b // 16,
      bcol*b // 16) at offset (brow*b % 16, bcol*b % 16).
    * Tile rows form groups by ``group_partition(m // 16, R)``; with R = 0,
      ``near_equal_groups(m // 16, groups)`` instead.
    * A group's entries are the distinct tile columns of its tiles, ascending;
      entries of all groups are concatenated in group order.
    * Each entry's rows are covered by intervals, one MMA each:
      ``cover_intervals`` when ``pad`` (static plans), else one interval per
      row (dynamic plans).  The entry owns one tile slot per covered row, in
      interval order; ent_tbeg[e] is the first slot of entry e (length
      E + 1); ent_cover[e] holds the covered-row mask in bits 0-15 and the
      interval-start mask in bits 16-31; tile_row[s] is the group row of slot s.
    * Items: a group with L entries becomes ``chunk_sizes(L, C)`` chunks of
      consecutive entries; a group with no entries is one zero-fill item.
      cost = slots in the chunk + entries in the chunk.  Static plans order
      items by (-cost, group, chunk); dynamic plans by (group, chunk).
    """
    if pad is None:
        pad = sort_items
    mt = m // TILE
    nnzb = len(brow)
    tr = [int(brow[p]) * b // TILE for p in range(nnzb)]
    tcol = [int(bcol[p]) * b // TILE for p in range(nnzb)]
    sizes = near_equal_groups(mt, groups) if R == 0 else group_partition(mt, R)
    grp_row0 = np.zeros(len(sizes), dtype=np.int32)
    acc = 0
    group_of = {}
    for g, sz in enumerate(sizes):
        grp_row0[g] = acc
        for t in range(acc, acc + sz):
            group_of[t] = g
        acc += sz
    grp_rows = np.array(sizes, dtype=np.int32)

    # entries: (group, tile column) -> sorted group rows holding a tile
    ent_rows = {}
    for t in set(zip(tr, tcol)):
        g = group_of[t[0]]
        ent_rows.setdefault((g, t[1]), []).append(t[0] - int(grp_row0[g]))
    keys = sorted(ent_rows)
    ent_col, ent_tbeg, ent_cover, tile_row = [], [], [], []
    grp_ebeg = [0] * (len(sizes) + 1)
    slot_of = {}
    for (g, c) in keys:
        rows = sorted(ent_rows[(g, c)])
        ivs = cover_intervals(rows) if pad else [(r, 1) for r in rows]
        ent_col.append(c)
        ent_tbeg.append(len(tile_row))
        cov = starts = 0
        for (r0, L) in ivs:
            starts |= 1 << r0
            for r in range(r0, r0 + L):
                cov |= 1 << r
                slot_of[(int(grp_row0[g]) + r, c)] = len(tile_row)
                tile_row.append(r)
        ent_cover.append(cov | (starts << 16))
        grp_ebeg[g + 1] += 1
    for g in range(len(sizes)):
        grp_ebeg[g + 1] += grp_ebeg[g]
    ent_tbeg.append(len(tile_row))

    items = []
    for g in range(len(sizes)):
        e0, e1 = grp_ebeg[g], grp_ebeg[g + 1]
        csz = chunk_sizes(e1 - e0, C)
        e = e0
        for ci, sz in enumerate(csz):
            nslot = ent_tbeg[e + sz] - ent_tbeg[e]
            items.append(dict(grp=g, beg=e, end=e + sz, chunk=ci, nch=len(csz),
                              cost=nslot + sz))
            e += sz
    if sort_items:
        items.sort(key=lambda it: (-it["cost"], it["grp"], it["chunk"]))
    ws_row0, ws_rows = _assign_ws(items, lambda g: int(grp_rows[g]) * TILE)

    blk_slot = np.array([slot_of[(tr[p], tcol[p])] for p in range(nnzb)], dtype=np.int32)
    blk_off = np.array([(int(brow[p]) * b % TILE) * TILE + int(bcol[p]) * b % TILE
                        for p in range(nnzb)], dtype=np.int32)
    return dict(
        grp_row0=grp_row0, grp_rows=grp_rows,
        grp_ebeg=np.array(grp_ebeg, dtype=np.int32),
        ent_col=np.array(ent_col, dtype=np.int32),
        ent_tbeg=np.array(ent_tbeg, dtype=np.int32),
        ent_cover=np.array(ent_cover, dtype=np.uint32).view(np.int32),
        tile_row=np.array(tile_row, dtype=np.int32),
        items=_items_array(items), ws_row0=ws_row0, ws_rows=ws_rows,
        red=_reductions(items),
        blk_slot=blk_slot, blk_off=blk_off,
    )


def tile_values(b, ntiles, blk_slot, blk_off, vals):
    """Dense 16 x 16 tiles in slot order, built from user-order blocks:
    tile[s][i][j] for i, j < 16; positions not covered by a block are zero.
    (Value layout only; the byte swizzle the kernel wants is not part of the
    method and is checked through the product, not here.)"""
    v = np.asarray(vals)
    out = np.zeros((ntiles, TILE, TILE), dtype=v.dtype)
    for p in range(len(blk_slot)):
        i0, j0 = divmod(int(blk_off[p]), TILE)
        out[blk_slot[p], i0:i0 + b, j0:j0 + b] = v[p]
    return out


# ------------------------------------------------------------ row slices ----
def row_slice(brow, bcol, b, row_begin, row_end):
    """One worker's share of a product split by rows of W (Section 3.2
    distributes W's non-zeros over workers; here each worker owns whole rows
    and X is replicated): the blocks whose rows lie in [row_begin, row_end),
    kept in the pattern's order with their block rows counted from
    row_begin, and the pattern index of each kept block.  Returns
    (brow_slice, bcol_slice, src_index) as int32 arrays."""
    if row_begin % b or row_end % b or not 0 <= row_begin < row_end:
        raise ValueError("slice bounds must be multiples of b with row_begin < row_end")
    r0, r1 = row_begin // b, row_end // b
    keep = [p for p in range(len(brow)) if r0 <= int(brow[p]) < r1]
    return (np.array([int(brow[p]) - r0 for p in keep], np.int32),
            np.array([int(bcol[p]) for p in keep], np.int32),
            np.array(keep, np.int32))


def row_split(m, b, workers, align=TILE):
    """Row ranges of ``workers`` near-equal slices of m rows, each boundary a
    multiple of ``align`` (and of b): the first m_a % workers slices get one
    more unit of ``align`` rows than the rest, m_a = m / align."""
    unit = max(align, b)
    if m % unit:
        raise ValueError("m must be a multiple of the alignment")
    units = m // unit
    sizes = [units // workers + (1 if w < units % workers else 0) for w in range(workers)]
    out, acc = [], 0
    for s in sizes:
        out.append((acc * unit, (acc + s) * unit))
        acc += s
    return out
