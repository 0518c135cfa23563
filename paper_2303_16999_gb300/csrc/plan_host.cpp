// Host planner for static mode (Section 3.2: the pattern is known when the
// plan is built, so the partition is chosen once, balanced by non-zero
// count).  Builds the canonical block-CSR, the b = 1 row items and the
// tensor-core tile-group items.  The rules are the library's own GPU
// decomposition; they are stated independently, in plain Python, by the
// test oracle, and the two must agree bit for bit.
#include <algorithm>
#include <cstdint>
#include <numeric>
#include <vector>

#include "spmm_internal.h"

namespace spmm {

spmm_status validate_pattern(int64_t m, int64_t k, int b, int64_t nnzb, const int32_t *brow,
                             const int32_t *bcol) {
    if (!(b == 1 || b == 4 || b == 8 || b == 16) || m <= 0 || k <= 0 || m % b || k % b) {
        set_error("shape: b=%d m=%lld k=%lld (b in {1,4,8,16}, m and k multiples of b)", b,
                  (long long)m, (long long)k);
        return SPMM_ERR_SHAPE;
    }
    // block indices, block-CSR offsets and tile slots are int32 on the device
    if (m / b > INT32_MAX || k / b > INT32_MAX || nnzb > INT32_MAX) {
        set_error("shape: %lld x %lld blocks or nnzb=%lld outside the int32 index range",
                  (long long)(m / b), (long long)(k / b), (long long)nnzb);
        return SPMM_ERR_SHAPE;
    }
    if (nnzb < 0 || (nnzb > 0 && (!brow || !bcol))) {
        set_error("pattern: nnzb=%lld with null arrays", (long long)nnzb);
        return SPMM_ERR_ARG;
    }
    const int64_t mb = m / b, kb = k / b;
    for (int64_t p = 0; p < nnzb; ++p) {
        if (brow[p] < 0 || brow[p] >= mb || bcol[p] < 0 || bcol[p] >= kb) {
            set_error("pattern: block %lld at (%d, %d) outside the %lld x %lld block grid",
                      (long long)p, brow[p], bcol[p], (long long)mb, (long long)kb);
            return SPMM_ERR_PATTERN;
        }
    }
    return SPMM_OK;
}

// Canonical block-CSR by (block row, block column); also detects repeated
// blocks (returns false and sets the error message).
static bool csr_impl(int64_t mb, int64_t nnzb, const int32_t *brow, const int32_t *bcol,
                     HostPlan &hp) {
    hp.row_ptr.assign(mb + 1, 0);
    for (int64_t p = 0; p < nnzb; ++p) hp.row_ptr[brow[p] + 1]++;
    for (int64_t r = 0; r < mb; ++r) hp.row_ptr[r + 1] += hp.row_ptr[r];
    std::vector<int32_t> cur(hp.row_ptr.begin(), hp.row_ptr.end() - 1);
    hp.perm.assign(nnzb, 0);
    for (int64_t p = 0; p < nnzb; ++p) hp.perm[cur[brow[p]]++] = (int32_t)p;
    hp.col_idx.assign(nnzb, 0);
    for (int64_t r = 0; r < mb; ++r) {
        auto b0 = hp.perm.begin() + hp.row_ptr[r], b1 = hp.perm.begin() + hp.row_ptr[r + 1];
        std::sort(b0, b1, [&](int32_t x, int32_t y) { return bcol[x] < bcol[y]; });
        for (int64_t s = hp.row_ptr[r]; s < hp.row_ptr[r + 1]; ++s) {
            hp.col_idx[s] = bcol[hp.perm[s]];
            if (s > hp.row_ptr[r] && hp.col_idx[s] == hp.col_idx[s - 1]) {
                set_error("pattern: block (%lld, %d) given twice", (long long)r, hp.col_idx[s]);
                return false;
            }
        }
    }
    return true;
}

void build_csr(int64_t mb, int64_t nnzb, const int32_t *brow, const int32_t *bcol, HostPlan &hp) {
    csr_impl(mb, nnzb, brow, bcol, hp);
}

bool build_csr_checked(int64_t mb, int64_t nnzb, const int32_t *brow, const int32_t *bcol,
                       HostPlan &hp) {
    return csr_impl(mb, nnzb, brow, bcol, hp);
}

// Appendix A.2 equal partition: q - 1 parts of floor(e/q), the last the rest.
static std::vector<int64_t> equal_partition(int64_t e, int64_t q) {
    std::vector<int64_t> s(q, e / q);
    s[q - 1] = e - (q - 1) * (e / q);
    return s;
}

std::vector<int64_t> group_partition(int64_t mt, int64_t R) {
    if (mt == 0) return {};
    int64_t q = (mt + R - 1) / R;
    while (mt - (q - 1) * (mt / q) > R) ++q;
    return equal_partition(mt, q);
}

std::vector<int64_t> near_equal_partition(int64_t mt, int64_t q) {
    std::vector<int64_t> out;
    if (mt == 0 || q <= 0) return out;
    out.assign(q, mt / q);
    for (int64_t i = 0; i < mt % q; ++i) out[i]++;
    return out;
}

static void chunk_sizes(int64_t L, int64_t C, std::vector<int64_t> &out) {
    const int64_t q = (L <= C) ? 1 : (L + C - 1) / C;
    out.assign(q, L / q);
    for (int64_t i = 0; i < L % q; ++i) out[i]++;
}

struct Item {
    int32_t grp, beg, end, chunk, nch, ws;
    int64_t cost;
};

static void finish_items(std::vector<Item> &items, bool sort_items,
                         const std::vector<int64_t> &rows_of_grp, HostPlan &hp) {
    if (sort_items)
        std::sort(items.begin(), items.end(), [](const Item &a, const Item &b) {
            if (a.cost != b.cost) return a.cost > b.cost;
            if (a.grp != b.grp) return a.grp < b.grp;
            return a.chunk < b.chunk;
        });
    // workspace slots for split items, in (group, chunk) order
    std::vector<int32_t> idx;
    for (int32_t i = 0; i < (int32_t)items.size(); ++i)
        if (items[i].nch > 1) idx.push_back(i);
    std::sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) {
        if (items[a].grp != items[b].grp) return items[a].grp < items[b].grp;
        return items[a].chunk < items[b].chunk;
    });
    hp.ws_row0.clear();
    hp.red.clear();
    int64_t row = 0;
    for (size_t s = 0; s < idx.size(); ++s) {
        Item &it = items[idx[s]];
        it.ws = (int32_t)s;
        hp.ws_row0.push_back(row);
        row += rows_of_grp[it.grp];
        if (it.chunk == 0) {
            hp.red.push_back(it.grp);
            hp.red.push_back((int32_t)s);
            hp.red.push_back(it.nch);
        }
    }
    hp.ws_rows = row;
    hp.items.resize(items.size() * kItemFields);
    for (size_t i = 0; i < items.size(); ++i) {
        int32_t *d = &hp.items[i * kItemFields];
        d[0] = items[i].grp;
        d[1] = items[i].beg;
        d[2] = items[i].end;
        d[3] = items[i].chunk;
        d[4] = items[i].nch;
        d[5] = items[i].ws;
    }
}

void build_row_plan(int64_t mb, int64_t C1, bool sort_items, HostPlan &hp) {
    std::vector<Item> items;
    items.reserve(mb);
    std::vector<int64_t> cs;
    for (int64_t r = 0; r < mb; ++r) {
        const int64_t beg = hp.row_ptr[r], end = hp.row_ptr[r + 1];
        chunk_sizes(end - beg, C1, cs);
        int64_t s = beg;
        for (size_t c = 0; c < cs.size(); ++c) {
            items.push_back(Item{(int32_t)r, (int32_t)s, (int32_t)(s + cs[c]), (int32_t)c,
                                 (int32_t)cs.size(), -1, cs[c]});
            s += cs[c];
        }
    }
    std::vector<int64_t> one(mb, 1);
    finish_items(items, sort_items, one, hp);
}

// Cost, in units of two SM cycles, of one MMA over L consecutive tile rows
// (N = 16 L): at least 40 cycles to issue, 8 cycles per 16 rows, plus one
// unit per tile slot moved through shared memory.
static int mma_cost(int L) { return std::max(20, 4 * L) + L; }

// Cheapest cover of ascending rows by runs of consecutive rows (exact DP,
// earliest split point on ties); rows inside a run without a tile are
// zero tiles.
static void cover_intervals(const std::vector<int> &rows, std::vector<std::pair<int, int>> &out) {
    const int n = (int)rows.size();
    int dp[kMaxGroupRows + 1], arg[kMaxGroupRows + 1];
    dp[0] = 0;
    for (int j = 1; j <= n; ++j) {
        dp[j] = -1;
        for (int i = 0; i < j; ++i) {
            const int c = dp[i] + mma_cost(rows[j - 1] - rows[i] + 1);
            if (dp[j] < 0 || c < dp[j]) {
                dp[j] = c;
                arg[j] = i;
            }
        }
    }
    out.clear();
    for (int j = n; j > 0; j = arg[j]) out.push_back({rows[arg[j]], rows[j - 1] - rows[arg[j]] + 1});
    std::reverse(out.begin(), out.end());
}

void build_tc_plan(int64_t m, int64_t k, int b, int64_t nnzb, const int32_t *brow,
                   const int32_t *bcol, int64_t R, int64_t C, bool sort_items, bool pad,
                   HostPlan &hp, int64_t groups) {
    const int64_t mt = m / kTile;
    (void)k;
    const std::vector<int64_t> sizes =
        groups > 0 ? near_equal_partition(mt, groups) : group_partition(mt, R);
    const int64_t G = (int64_t)sizes.size();
    hp.grp_row0.assign(G, 0);
    hp.grp_rows.assign(G, 0);
    std::vector<int32_t> group_of(mt, 0);
    int64_t acc = 0;
    for (int64_t g = 0; g < G; ++g) {
        hp.grp_row0[g] = (int32_t)acc;
        hp.grp_rows[g] = (int32_t)sizes[g];
        for (int64_t t = acc; t < acc + sizes[g]; ++t) group_of[t] = (int32_t)g;
        acc += sizes[g];
    }
    // distinct tiles per group, ordered by (tile column, tile row)
    std::vector<std::vector<int64_t>> keys(G);  // key = tc * mt + tr
    std::vector<int64_t> bkey(nnzb);
    for (int64_t p = 0; p < nnzb; ++p) {
        const int64_t tr = (int64_t)brow[p] * b / kTile, tc = (int64_t)bcol[p] * b / kTile;
        bkey[p] = tc * mt + tr;
        keys[group_of[tr]].push_back(bkey[p]);
    }
    std::vector<int64_t> slot_base(G + 1, 0);
    for (int64_t g = 0; g < G; ++g) {
        auto &v = keys[g];
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        slot_base[g + 1] = slot_base[g] + (int64_t)v.size();
    }
    // entries: runs of one tile column within a group's sorted keys; each
    // entry's rows are covered by MMA intervals and get one slot per row
    hp.tile_row.clear();
    hp.ent_col.clear();
    hp.ent_tbeg.clear();
    hp.ent_cover.clear();
    hp.grp_ebeg.assign(G + 1, 0);
    std::vector<int32_t> key_slot(slot_base[G]);
    std::vector<int> rows;
    std::vector<std::pair<int, int>> ivs;
    for (int64_t g = 0; g < G; ++g) {
        const auto &v = keys[g];
        size_t i = 0;
        while (i < v.size()) {
            const int64_t tc = v[i] / mt;
            size_t j = i;
            rows.clear();
            while (j < v.size() && v[j] / mt == tc) {
                rows.push_back((int)(v[j] % mt - hp.grp_row0[g]));
                ++j;
            }
            if (pad) {
                cover_intervals(rows, ivs);
            } else {
                ivs.clear();
                for (int r : rows) ivs.push_back({r, 1});
            }
            hp.ent_col.push_back((int32_t)tc);
            hp.ent_tbeg.push_back((int32_t)hp.tile_row.size());
            uint32_t cov = 0, starts = 0;
            size_t q = i;
            for (const auto &iv : ivs) {
                starts |= 1u << iv.first;
                for (int r = iv.first; r < iv.first + iv.second; ++r) {
                    cov |= 1u << r;
                    if (q < j && (int)(v[q] % mt - hp.grp_row0[g]) == r) key_slot[slot_base[g] + q++] = (int32_t)hp.tile_row.size();
                    hp.tile_row.push_back(r);
                }
            }
            hp.ent_cover.push_back((int32_t)(cov | (starts << 16)));
            i = j;
        }
        hp.grp_ebeg[g + 1] = (int32_t)hp.ent_col.size();
    }
    hp.ent_tbeg.push_back((int32_t)hp.tile_row.size());
    hp.blk_slot.assign(nnzb, 0);
    hp.blk_off.assign(nnzb, 0);
    for (int64_t p = 0; p < nnzb; ++p) {
        const int64_t tr = (int64_t)brow[p] * b / kTile;
        const int g = group_of[tr];
        const auto &v = keys[g];
        const int64_t i = std::lower_bound(v.begin(), v.end(), bkey[p]) - v.begin();
        hp.blk_slot[p] = key_slot[slot_base[g] + i];
        hp.blk_off[p] = (int32_t)(((int64_t)brow[p] * b % kTile) * kTile + (int64_t)bcol[p] * b % kTile);
    }
    // items: near-equal chunks of each group's entries
    std::vector<Item> items;
    std::vector<int64_t> cs;
    for (int64_t g = 0; g < G; ++g) {
        const int64_t e0 = hp.grp_ebeg[g], e1 = hp.grp_ebeg[g + 1];
        chunk_sizes(e1 - e0, C, cs);
        int64_t e = e0;
        for (size_t c = 0; c < cs.size(); ++c) {
            const int64_t nt = hp.ent_tbeg[e + cs[c]] - hp.ent_tbeg[e];
            items.push_back(Item{(int32_t)g, (int32_t)e, (int32_t)(e + cs[c]), (int32_t)c,
                                 (int32_t)cs.size(), -1, nt + cs[c]});
            e += cs[c];
        }
    }
    std::vector<int64_t> grows(G);
    for (int64_t g = 0; g < G; ++g) grows[g] = (int64_t)hp.grp_rows[g] * kTile;
    finish_items(items, sort_items, grows, hp);
}

}  // namespace spmm
