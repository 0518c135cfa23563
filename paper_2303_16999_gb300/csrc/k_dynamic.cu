// Dynamic mode: the partition is rebuilt on the device on every call
// (Section 3.3 / Appendix A.2: only the maximum non-zero count is fixed when
// the plan is made; the pattern arrives at run time and is distributed then).
//
// The paper's host utility encodes metaInfo buckets and the device walks
// distribution and propagation phases; here the whole re-partition runs on
// the device in a handful of stream-ordered kernels with no host round trip:
//   1. validate + histogram of block rows, then (the last block to finish)
//      the exclusive scan -> row_ptr (and b = 1 items) (grid over the pattern)
//   2. scatter into rows                            (grid over the pattern)
//   3. per-row rank sort by column, duplicate check (one warp per row)
//   4. tensor-core plans: per-group column bitmap -> entry / slot counts,
//      then (the last block) the group scan (chunk size, item / workspace
//      offsets), and a per-group fill of entries, slots, items and
//      block -> slot maps.
// A scan runs in the last block of the kernel before it (a ticket counter,
// with fences on both sides) rather than as its own launch: each launch of
// this latency-bound chain costs a few microseconds.
// The arrays equal the oracle's dynamic-plan rules bit for bit (no item
// reordering, no zero-padded intervals).  A rejected pattern sets the plan's
// status word; the product kernels then skip, leaving Y unwritten.
#include <cuda_runtime.h>

#include "pdl.cuh"
#include "spmm_internal.h"

namespace spmm {
namespace {

__device__ __forceinline__ void flag(int32_t *status, int32_t code) { atomicCAS(status, 0, code); }

__device__ __forceinline__ int64_t clamp_nnzb(const int32_t *d_nnzb, int64_t cap) {
    const int64_t n = *d_nnzb;
    return n < 0 ? 0 : (n > cap ? cap : n);
}

// True in the one block that finishes last: every block fences its writes
// and takes a ticket; the block that draws the last ticket fences again
// before it reads what the others wrote.
__device__ bool last_block_done(int32_t *ticket) {
    __shared__ int is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(ticket, 1) == (int)(gridDim.x - 1) ? 1 : 0;
    __syncthreads();
    if (is_last) __threadfence();
    return is_last != 0;
}

__device__ void scan_rows(const int32_t *d_nnzb, int64_t cap, int32_t mb, const int32_t *row_cnt,
                          int32_t *row_ptr, int32_t *cursor, int32_t *row_ibeg, int32_t *row_wbeg,
                          int32_t *row_rbeg, int32_t *counts, int rows_items);

// 1. range check and block-row histogram; the last block scans the rows
__global__ void __launch_bounds__(1024) dyn_validate_scan(
    const int32_t *d_nnzb, const int32_t *brow, const int32_t *bcol, int64_t cap, int32_t mb,
    int32_t kb, int32_t *row_cnt, int32_t *status, int32_t *row_ptr, int32_t *cursor,
    int32_t *row_ibeg, int32_t *row_wbeg, int32_t *row_rbeg, int32_t *counts, int rows_items) {
    pdl_enter();
    const int64_t raw = *d_nnzb;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (raw < 0 || raw > cap)) flag(status, kDevCapacity);
    const int64_t n = raw < 0 ? 0 : (raw > cap ? cap : raw);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = brow[p], c = bcol[p];
        if (r < 0 || r >= mb || c < 0 || c >= kb) {
            flag(status, kDevPattern);
            continue;
        }
        atomicAdd(&row_cnt[r], 1);
    }
    if (!last_block_done(counts + kCntTicketRows)) return;
    scan_rows(d_nnzb, cap, mb, row_cnt, row_ptr, cursor, row_ibeg, row_wbeg, row_rbeg, counts,
              rows_items);
}

// Block-wide exclusive scan of one value per thread (blockDim.x == 1024).
__device__ int64_t block_scan(int64_t v, int64_t *total) {
    __shared__ int64_t warp_sums[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t s = warp_sums[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    const int64_t excl = x - v + (w > 0 ? warp_sums[w - 1] : 0);
    *total = warp_sums[31];
    __syncthreads();
    return excl;
}

__device__ __forceinline__ int32_t nchunks(int64_t L, int64_t C) {
    return (int32_t)(L <= C ? 1 : (L + C - 1) / C);
}

// row_ptr / cursor; for b = 1 also the row-item, workspace and reduction
// offsets (C1 = max(64, 2 * ceil(nnzb / mb)), the static default).  One
// block of 1024 threads (the histogram's last).
__device__ void scan_rows(const int32_t *d_nnzb, int64_t cap, int32_t mb, const int32_t *row_cnt,
                          int32_t *row_ptr, int32_t *cursor, int32_t *row_ibeg, int32_t *row_wbeg,
                          int32_t *row_rbeg, int32_t *counts, int rows_items) {
    const int64_t nnzb = clamp_nnzb(d_nnzb, cap);
    const int64_t avg = mb ? (nnzb + mb - 1) / mb : 0;
    const int64_t C1 = avg * 2 > 64 ? avg * 2 : 64;
    int64_t base = 0, ibase = 0, wbase = 0, rbase = 0;
    for (int32_t r0 = 0; r0 < mb; r0 += 1024) {
        const int32_t r = r0 + threadIdx.x;
        const int64_t L = r < mb ? __ldcg(row_cnt + r) : 0;
        const int32_t nch = r < mb ? nchunks(L, C1) : 0;
        int64_t t0, t1, t2, t3;
        const int64_t e0 = block_scan(L, &t0);
        const int64_t e1 = block_scan(nch, &t1);
        const int64_t e2 = block_scan(nch > 1 ? nch : 0, &t2);
        const int64_t e3 = block_scan(nch > 1 ? 1 : 0, &t3);
        if (r < mb) {
            row_ptr[r] = (int32_t)(base + e0);
            cursor[r] = (int32_t)(base + e0);
            if (rows_items) {
                row_ibeg[r] = (int32_t)(ibase + e1);
                row_wbeg[r] = (int32_t)(wbase + e2);
                row_rbeg[r] = (int32_t)(rbase + e3);
            }
        }
        base += t0;
        ibase += t1;
        wbase += t2;
        rbase += t3;
    }
    if (threadIdx.x == 0) {
        row_ptr[mb] = (int32_t)base;
        counts[kCntNnzb] = (int32_t)base;
        if (rows_items) {
            counts[kCntItems] = (int32_t)ibase;
            counts[kCntWsRows] = (int32_t)wbase;
            counts[kCntRed] = (int32_t)rbase;
            counts[kCntChunk] = (int32_t)C1;
        }
    }
}

// 2. scatter into rows (order within a row fixed by step 3)
__global__ void dyn_scatter(const int32_t *d_nnzb, const int32_t *brow, const int32_t *bcol,
                            int64_t cap, int32_t mb, int32_t kb, int32_t *cursor, int32_t *tmp_col,
                            int32_t *tmp_perm) {
    pdl_enter();
    const int64_t n = clamp_nnzb(d_nnzb, cap);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = brow[p], c = bcol[p];
        if (r < 0 || r >= mb || c < 0 || c >= kb) continue;
        const int32_t pos = atomicAdd(&cursor[r], 1);
        tmp_col[pos] = c;
        tmp_perm[pos] = (int32_t)p;
    }
}

// 3. one warp per row: rank of each element among the row's columns (keys
// are unique unless the pattern repeats a block, which is flagged); for
// b = 1 the warp also writes its row's items.
__global__ void dyn_sort_rows(int32_t mb, const int32_t *row_ptr, const int32_t *tmp_col,
                              const int32_t *tmp_perm, int32_t *col_idx, int32_t *perm,
                              int32_t *status, int rows_items, const int32_t *row_ibeg,
                              const int32_t *row_wbeg, const int32_t *row_rbeg,
                              const int32_t *counts, int32_t *items, int64_t *ws_row0,
                              int32_t *red) {
    pdl_enter();
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= mb) return;
    const int32_t r = (int32_t)wid, beg = row_ptr[r], end = row_ptr[r + 1];
    for (int32_t i = beg + lane; i < end; i += 32) {
        const int32_t ci = tmp_col[i];
        int32_t rank = 0;
        bool dup = false;
        for (int32_t j = beg; j < end; ++j) {
            const int32_t cj = tmp_col[j];
            rank += cj < ci;
            dup |= (cj == ci) && (j != i);
            if (cj == ci && j < i) ++rank;   // keeps ranks distinct when duplicated
        }
        if (dup) flag(status, kDevPattern);
        col_idx[beg + rank] = ci;
        perm[beg + rank] = tmp_perm[i];
    }
    if (!rows_items || lane != 0) return;
    const int64_t C1 = counts[kCntChunk];
    const int32_t L = end - beg, nch = nchunks(L, C1);
    const int32_t base = L / nch, rem = L % nch;
    int32_t s = beg;
    for (int32_t c = 0; c < nch; ++c) {
        const int32_t sz = base + (c < rem ? 1 : 0);
        int32_t *it = items + (int64_t)(row_ibeg[r] + c) * kItemFields;
        const int32_t ws = nch > 1 ? row_wbeg[r] + c : -1;
        it[0] = r;
        it[1] = s;
        it[2] = s + sz;
        it[3] = c;
        it[4] = nch;
        it[5] = ws;
        if (ws >= 0) ws_row0[ws] = ws;   // one Y row per b = 1 chunk
        s += sz;
    }
    if (nch > 1) {
        int32_t *rd = red + (int64_t)row_rbeg[r] * 3;
        rd[0] = r;
        rd[1] = row_wbeg[r];
        rd[2] = nch;
    }
}

__device__ void group_scan(int32_t G, const int32_t *grp_rows, const int32_t *grp_cnt,
                           int32_t *grp_ebeg, int32_t *grp_sbeg, int32_t *grp_ibeg,
                           int32_t *grp_wbeg, int64_t *grp_wrow, int32_t *grp_rbeg,
                           int32_t *ent_tbeg, int32_t *counts);

// 4a. per group: bitmap of group rows per tile column -> entry and slot
// counts; the last block scans the groups
__global__ void __launch_bounds__(1024) dyn_group_count_scan(
    int32_t kt, int32_t T, const int32_t *grp_row0, const int32_t *grp_rows,
    const int32_t *row_ptr, const int32_t *col_idx, int32_t *grp_cnt, int32_t *grp_ebeg,
    int32_t *grp_sbeg, int32_t *grp_ibeg, int32_t *grp_wbeg, int64_t *grp_wrow,
    int32_t *grp_rbeg, int32_t *ent_tbeg, int32_t *counts) {
    pdl_enter();
    extern __shared__ uint32_t colmask[];
    const int g = blockIdx.x;
    for (int32_t c = threadIdx.x; c < kt; c += blockDim.x) colmask[c] = 0;
    __syncthreads();
    const int32_t t0 = grp_row0[g], nrows = grp_rows[g];
    const int32_t s0 = row_ptr[t0 * T], s1 = row_ptr[(t0 + nrows) * T];
    for (int32_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        // block row of slot s: search the group's rows
        int32_t lo = t0 * T, hi = (t0 + nrows) * T;
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (row_ptr[mid] <= s) lo = mid; else hi = mid;
        }
        atomicOr(&colmask[col_idx[s] / T], 1u << (lo / T - t0));
    }
    __syncthreads();
    int32_t ne = 0, ns = 0;
    for (int32_t c = threadIdx.x; c < kt; c += blockDim.x) {
        ne += colmask[c] != 0;
        ns += __popc(colmask[c]);
    }
    ne = __reduce_add_sync(0xffffffffu, ne);
    ns = __reduce_add_sync(0xffffffffu, ns);
    __shared__ int32_t acc[2];
    if (threadIdx.x == 0) acc[0] = acc[1] = 0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc[0], ne);
        atomicAdd(&acc[1], ns);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        grp_cnt[g * 2] = acc[0];
        grp_cnt[g * 2 + 1] = acc[1];
    }
    if (!last_block_done(counts + kCntTicketGroups)) return;
    group_scan((int32_t)gridDim.x, grp_rows, grp_cnt, grp_ebeg, grp_sbeg, grp_ibeg, grp_wbeg,
               grp_wrow, grp_rbeg, ent_tbeg, counts);
}

// 4b. group offsets and the chunk size C = max(16, ceil(5E / 4G)); one block
// of 1024 threads (the group counts' last).
__device__ void group_scan(int32_t G, const int32_t *grp_rows, const int32_t *grp_cnt,
                           int32_t *grp_ebeg, int32_t *grp_sbeg, int32_t *grp_ibeg,
                           int32_t *grp_wbeg, int64_t *grp_wrow, int32_t *grp_rbeg,
                           int32_t *ent_tbeg, int32_t *counts) {
    __shared__ int64_t sE;
    int64_t tot;
    {
        int64_t part = 0;
        for (int32_t g = threadIdx.x; g < G; g += 1024) part += __ldcg(grp_cnt + g * 2);
        block_scan(part, &tot);
        if (threadIdx.x == 0) sE = tot;
        __syncthreads();
    }
    const int64_t E = sE;
    const int64_t Cq = G ? (5 * E + 4 * G - 1) / (4 * G) : 16;
    const int64_t C = Cq > 16 ? Cq : 16;
    int64_t be = 0, bs = 0, bi = 0, bw = 0, bwr = 0, br = 0;
    for (int32_t g0 = 0; g0 < G; g0 += 1024) {
        const int32_t g = g0 + threadIdx.x;
        const int64_t L = g < G ? __ldcg(grp_cnt + g * 2) : 0;
        const int64_t S = g < G ? __ldcg(grp_cnt + g * 2 + 1) : 0;
        const int32_t nch = g < G ? nchunks(L, C) : 0;
        const int64_t rows = g < G ? (int64_t)grp_rows[g] * kTile : 0;
        int64_t t0, t1, t2, t3, t4, t5;
        const int64_t e0 = block_scan(L, &t0);
        const int64_t e1 = block_scan(S, &t1);
        const int64_t e2 = block_scan(nch, &t2);
        const int64_t e3 = block_scan(nch > 1 ? nch : 0, &t3);
        const int64_t e4 = block_scan(nch > 1 ? nch * rows : 0, &t4);
        const int64_t e5 = block_scan(nch > 1 ? 1 : 0, &t5);
        if (g < G) {
            grp_ebeg[g] = (int32_t)(be + e0);
            grp_sbeg[g] = (int32_t)(bs + e1);
            grp_ibeg[g] = (int32_t)(bi + e2);
            grp_wbeg[g] = (int32_t)(bw + e3);
            grp_wrow[g] = bwr + e4;
            grp_rbeg[g] = (int32_t)(br + e5);
        }
        be += t0;
        bs += t1;
        bi += t2;
        bw += t3;
        bwr += t4;
        br += t5;
    }
    if (threadIdx.x == 0) {
        grp_ebeg[G] = (int32_t)be;
        ent_tbeg[be] = (int32_t)bs;
        counts[kCntEntries] = (int32_t)be;
        counts[kCntSlots] = (int32_t)bs;
        counts[kCntItems] = (int32_t)bi;
        counts[kCntWsSlots] = (int32_t)bw;
        counts[kCntWsRows] = (int32_t)bwr;
        counts[kCntRed] = (int32_t)br;
        counts[kCntChunk] = (int32_t)C;
    }
}

// 4c. per group: entries (ascending tile column), slots (ascending rows, one
// per tile), block -> slot / offset, items and workspace / reduction records
__global__ void dyn_group_fill(int32_t kt, int32_t T, int32_t b, const int32_t *grp_row0,
                               const int32_t *grp_rows, const int32_t *row_ptr,
                               const int32_t *col_idx, const int32_t *perm, const int32_t *grp_ebeg,
                               const int32_t *grp_sbeg, const int32_t *grp_ibeg,
                               const int32_t *grp_wbeg, const int64_t *grp_wrow,
                               const int32_t *grp_rbeg, const int32_t *counts, int32_t *ent_col,
                               int32_t *ent_tbeg, int32_t *ent_cover, int32_t *tile_row,
                               int32_t *blk_slot, int32_t *blk_off, int32_t *items,
                               int64_t *ws_row0, int32_t *red) {
    pdl_enter();
    extern __shared__ uint32_t sm[];
    uint32_t *colmask = sm;                 // kt
    int32_t *ent_of = (int32_t *)(sm + kt); // kt: entry index of each column, slot base in ent_tbeg
    int32_t *slot_of = ent_of + kt;         // kt: first slot of the column's entry
    const int g = blockIdx.x;
    for (int32_t c = threadIdx.x; c < kt; c += blockDim.x) colmask[c] = 0;
    __syncthreads();
    const int32_t t0 = grp_row0[g], nrows = grp_rows[g];
    const int32_t s0 = row_ptr[t0 * T], s1 = row_ptr[(t0 + nrows) * T];
    for (int32_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        int32_t lo = t0 * T, hi = (t0 + nrows) * T;
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (row_ptr[mid] <= s) lo = mid; else hi = mid;
        }
        atomicOr(&colmask[col_idx[s] / T], 1u << (lo / T - t0));
    }
    __syncthreads();
    // column prefix over entries and slots, in chunks of blockDim (1024)
    int64_t eb = grp_ebeg[g], sb = grp_sbeg[g];
    for (int32_t c0 = 0; c0 < kt; c0 += 1024) {
        const int32_t c = c0 + threadIdx.x;
        const uint32_t mk = c < kt ? colmask[c] : 0u;
        int64_t te, ts;
        const int64_t xe = block_scan(mk != 0, &te);
        const int64_t xs = block_scan(__popc(mk), &ts);
        if (c < kt && mk) {
            const int32_t e = (int32_t)(eb + xe);
            ent_of[c] = e;
            slot_of[c] = (int32_t)(sb + xs);
            ent_col[e] = c;
            ent_tbeg[e] = (int32_t)(sb + xs);
            ent_cover[e] = (int32_t)(mk | (mk << 16));
            uint32_t m = mk;
            int32_t q = (int32_t)(sb + xs);
            while (m) {
                tile_row[q++] = __ffs(m) - 1;
                m &= m - 1;
            }
        }
        eb += te;
        sb += ts;
    }
    __syncthreads();
    // blocks of the group -> slot and offset (indexed by user position)
    for (int32_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        int32_t lo = t0 * T, hi = (t0 + nrows) * T;
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (row_ptr[mid] <= s) lo = mid; else hi = mid;
        }
        const int32_t br = lo, bc = col_idx[s];
        const int32_t tc = bc / T, trow = br / T - t0;
        const uint32_t mk = colmask[tc];
        const int32_t slot = slot_of[tc] + __popc(mk & ((1u << trow) - 1u));
        const int32_t p = perm[s];
        blk_slot[p] = slot;
        blk_off[p] = ((br * b) % kTile) * kTile + (bc * b) % kTile;
    }
    if (threadIdx.x != 0) return;
    // items: near-equal chunks of the group's entries
    const int64_t C = counts[kCntChunk];
    const int32_t e0 = grp_ebeg[g], L = grp_ebeg[g + 1] - e0, nch = nchunks(L, C);
    const int32_t base = L / nch, rem = L % nch;
    int32_t e = e0;
    for (int32_t c = 0; c < nch; ++c) {
        const int32_t sz = base + (c < rem ? 1 : 0);
        int32_t *it = items + (int64_t)(grp_ibeg[g] + c) * kItemFields;
        const int32_t ws = nch > 1 ? grp_wbeg[g] + c : -1;
        it[0] = g;
        it[1] = e;
        it[2] = e + sz;
        it[3] = c;
        it[4] = nch;
        it[5] = ws;
        if (ws >= 0) ws_row0[ws] = grp_wrow[g] + (int64_t)c * nrows * kTile;
        e += sz;
    }
    if (nch > 1) {
        int32_t *rd = red + (int64_t)grp_rbeg[g] * 3;
        rd[0] = g;
        rd[1] = grp_wbeg[g];
        rd[2] = nch;
    }
}

inline unsigned grid_for(int64_t n, int threads, unsigned cap) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    return (unsigned)(g > cap ? cap : g);
}

}  // namespace

cudaError_t launch_dynamic_csr(spmm_plan *p, const spmm_dpattern *dp, cudaStream_t s) {
    DynBufs &d = p->dyn;
    const int32_t mb = (int32_t)(p->m / p->b), kb = (int32_t)(p->k / p->b);
    const int64_t cap = p->nnzb_max;
    cudaError_t e = cudaMemsetAsync(p->d_status, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.row_cnt, 0, sizeof(int32_t) * mb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_counts, 0, sizeof(int32_t) * kCntCount, s);
    if (e != cudaSuccess) return e;
    const unsigned gp = grid_for(cap, 256, 4096);
    pdl_launch(dyn_validate_scan, dim3(grid_for(cap, 1024, 1024)), dim3(1024), 0, s, dp->d_nnzb,
        dp->d_brow, dp->d_bcol, cap, mb, kb, d.row_cnt, p->d_status, p->d_row_ptr, d.cursor,
        d.row_ibeg, d.row_wbeg, d.row_rbeg, p->d_counts, 0);
    pdl_launch(dyn_scatter, dim3(gp), dim3(256), 0, s, dp->d_nnzb, dp->d_brow, dp->d_bcol, cap, mb,
        kb, d.cursor, d.tmp_col, d.tmp_perm);
    pdl_launch(dyn_sort_rows, dim3(grid_for((int64_t)mb * 32, 256, 1u << 30)), dim3(256), 0, s, mb,
        p->d_row_ptr, d.tmp_col, d.tmp_perm, p->d_col_idx, p->d_perm, p->d_status, 0,
        d.row_ibeg, d.row_wbeg, d.row_rbeg, p->d_counts, p->d_items, p->d_ws_row0, p->d_red);
    return cudaGetLastError();
}

cudaError_t launch_dynamic_partition(spmm_plan *p, const spmm_dpattern *dp, cudaStream_t s) {
    DynBufs &d = p->dyn;
    const int32_t mb = (int32_t)(p->m / p->b), kb = (int32_t)(p->k / p->b);
    const int64_t cap = p->nnzb_max;
    const bool tc = p->kernel == SPMM_KERNEL_TC;
    cudaError_t e = cudaMemsetAsync(p->d_status, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.row_cnt, 0, sizeof(int32_t) * mb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_counts, 0, sizeof(int32_t) * kCntCount, s);
    if (e != cudaSuccess) return e;
    const unsigned gp = grid_for(cap, 256, 4096);
    pdl_launch(dyn_validate_scan, dim3(grid_for(cap, 1024, 1024)), dim3(1024), 0, s, dp->d_nnzb,
        dp->d_brow, dp->d_bcol, cap, mb, kb, d.row_cnt, p->d_status, p->d_row_ptr, d.cursor,
        d.row_ibeg, d.row_wbeg, d.row_rbeg, p->d_counts, tc ? 0 : 1);
    pdl_launch(dyn_scatter, dim3(gp), dim3(256), 0, s, dp->d_nnzb, dp->d_brow, dp->d_bcol, cap, mb,
        kb, d.cursor, d.tmp_col, d.tmp_perm);
    pdl_launch(dyn_sort_rows, dim3(grid_for((int64_t)mb * 32, 256, 1u << 30)), dim3(256), 0, s, mb,
        p->d_row_ptr, d.tmp_col, d.tmp_perm, p->d_col_idx, p->d_perm, p->d_status, tc ? 0 : 1,
        d.row_ibeg, d.row_wbeg, d.row_rbeg, p->d_counts, p->d_items, p->d_ws_row0, p->d_red);
    if (tc) {
        const int32_t kt = (int32_t)(p->k / kTile), T = kTile / p->b, G = (int32_t)p->n_groups;
        pdl_launch(dyn_group_count_scan, dim3(G), dim3(1024), sizeof(uint32_t) * kt, s, kt, T,
            p->d_grp_row0, p->d_grp_rows, p->d_row_ptr, p->d_col_idx, d.grp_cnt, p->d_grp_ebeg,
            d.grp_sbeg, d.grp_ibeg, d.grp_wbeg, d.grp_wrow, d.grp_rbeg, p->d_ent_tbeg,
            p->d_counts);
        pdl_launch(dyn_group_fill, dim3(G), dim3(1024), sizeof(uint32_t) * 3 * kt, s, kt, T, p->b,
            p->d_grp_row0, p->d_grp_rows, p->d_row_ptr, p->d_col_idx, p->d_perm, p->d_grp_ebeg,
            d.grp_sbeg, d.grp_ibeg, d.grp_wbeg, d.grp_wrow, d.grp_rbeg, p->d_counts, p->d_ent_col,
            p->d_ent_tbeg, p->d_ent_cover, p->d_tile_row, p->d_blk_slot, p->d_blk_off, p->d_items,
            p->d_ws_row0, p->d_red);
    }
    return cudaGetLastError();
}

}  // namespace spmm
