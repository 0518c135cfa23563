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
// this latency-bound chain costs a few microseconds.  Dynamic tensor-core
// plans run all of it, with the packing and the stage records, in one
// cooperative launch instead (see "fused" below); the chain remains for the
// b = 1 gather plans, the sampled product's block CSR, devices without
// cooperative launches and spmm_plan_opts.dyn_chain.  The whole job is a
// chain of dependent steps over a few megabytes: its time goes to memory
// round trips, CTA barriers and the grid barriers between steps, not to
// bytes or arithmetic (a kernel boundary of the chain costs a few
// microseconds, a grid barrier of the fused launch about one).
// The arrays equal the oracle's dynamic-plan rules bit for bit (no item
// reordering, no zero-padded intervals).  A rejected pattern sets the plan's
// status word; the product kernels then skip, leaving Y unwritten.
#include <cuda_runtime.h>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>

#include "pdl.cuh"
#include "spmm_internal.h"
#include "tc_stage.cuh"

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
// The last block also puts the ticket back to zero for the next launch.
__device__ bool last_block_done(int32_t *ticket) {
    __shared__ int is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(ticket, 1) == (int)(gridDim.x - 1) ? 1 : 0;
    __syncthreads();
    if (is_last) {
        __threadfence();
        if (threadIdx.x == 0) *ticket = 0;
    }
    return is_last != 0;
}

__device__ void scan_rows(const int32_t *d_nnzb, int64_t cap, int32_t mb, int32_t *row_cnt,
                          int32_t *row_ptr, int32_t *cursor, int32_t *row_ibeg, int32_t *row_wbeg,
                          int32_t *row_rbeg, int32_t *counts, int rows_items);

// 1. range check and block-row histogram; the last block scans the rows.
// The blocks record what they find in counts[kCntFlags]; the last block
// stores the call's status from it (capacity first, then pattern, else 0)
// and leaves the flags, the ticket and the row counts zero for the next
// call, so that the chain needs no memsets once they start out zero.
__global__ void __launch_bounds__(1024) dyn_validate_scan(
    const int32_t *d_nnzb, const int32_t *brow, const int32_t *bcol, int64_t cap, int32_t mb,
    int32_t kb, int32_t *row_cnt, int32_t *status, int32_t *row_ptr, int32_t *cursor,
    int32_t *row_ibeg, int32_t *row_wbeg, int32_t *row_rbeg, int32_t *counts, int rows_items) {
    pdl_enter();
    const int64_t raw = *d_nnzb;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (raw < 0 || raw > cap))
        atomicOr(counts + kCntFlags, 1);
    const int64_t n = raw < 0 ? 0 : (raw > cap ? cap : raw);
    bool bad = false;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = brow[p], c = bcol[p];
        if (r < 0 || r >= mb || c < 0 || c >= kb) {
            bad = true;
            continue;
        }
        atomicAdd(&row_cnt[r], 1);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(counts + kCntFlags, 2);
    if (!last_block_done(counts + kCntTicketRows)) return;
    if (threadIdx.x == 0) {
        const int32_t f = atomicExch(counts + kCntFlags, 0);
        *status = (f & 1) ? (int32_t)kDevCapacity : (f & 2) ? (int32_t)kDevPattern : 0;
    }
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

// N block-wide exclusive scans at once (blockDim.x == 1024): v[i] in,
// the exclusive prefix in v[i], the block's total in tot[i].
template <int N>
__device__ void block_scan_n(int64_t (&v)[N], int64_t (&tot)[N]) {
    __shared__ int64_t warp_sums[N][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        x[i] = v[i];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x[i], o);
            if (lane >= o) x[i] += y;
        }
        if (lane == 31) warp_sums[i][w] = x[i];
    }
    __syncthreads();
    if (w < N) {
        int64_t t = warp_sums[w][lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_sums[w][lane] = t;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) {
        v[i] = x[i] - v[i] + (w > 0 ? warp_sums[i][w - 1] : 0);
        tot[i] = warp_sums[i][31];
    }
    __syncthreads();
}

__device__ __forceinline__ int32_t nchunks(int64_t L, int64_t C) {
    return (int32_t)(L <= C ? 1 : (L + C - 1) / C);
}

// row_ptr / cursor; for b = 1 also the row-item, workspace and reduction
// offsets (C1 = max(64, 2 * ceil(nnzb / mb)), the static default).  One
// block of 1024 threads (the histogram's last).
__device__ void scan_rows(const int32_t *d_nnzb, int64_t cap, int32_t mb, int32_t *row_cnt,
                          int32_t *row_ptr, int32_t *cursor, int32_t *row_ibeg, int32_t *row_wbeg,
                          int32_t *row_rbeg, int32_t *counts, int rows_items) {
    const int64_t nnzb = clamp_nnzb(d_nnzb, cap);
    const int64_t avg = mb ? (nnzb + mb - 1) / mb : 0;
    const int64_t C1 = avg * 2 > 64 ? avg * 2 : 64;
    int64_t base = 0, ibase = 0, wbase = 0, rbase = 0;
    for (int32_t r0 = 0; r0 < mb; r0 += 1024) {
        const int32_t r = r0 + threadIdx.x;
        const int64_t L = r < mb ? __ldcg(row_cnt + r) : 0;
        if (r < mb) row_cnt[r] = 0;   // for the next call
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

// One warp orders one row's slots by column: the rank of each element among
// the row's columns (keys are unique unless the pattern repeats a block,
// which is flagged).
__device__ void sort_row(int32_t beg, int32_t end, int lane, const int32_t *tmp_col,
                         const int32_t *tmp_perm, int32_t *col_idx, int32_t *perm,
                         int32_t *status) {
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
    sort_row(beg, end, lane, tmp_col, tmp_perm, col_idx, perm, status);
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

// Group g's offsets from the group scan.
struct GroupOff {
    int32_t row0, rows;          // first tile row, tile rows
    int32_t ebeg, eend;          // entries [ebeg, eend)
    int32_t sbeg, send;          // slots [sbeg, send)
    int32_t ibeg, wbeg, rbeg;    // first item, workspace slot, reduction
    int64_t wrow, C;             // first workspace row, chunk size
};

__device__ void group_scan(int32_t G, const int32_t *grp_rows, const int32_t *grp_cnt,
                           int32_t *grp_ebeg, int32_t *grp_sbeg, int32_t *grp_ibeg,
                           int32_t *grp_wbeg, int64_t *grp_wrow, int32_t *grp_rbeg,
                           int32_t *ent_tbeg, int32_t *counts, bool write_global = true,
                           GroupOff *own = nullptr, const int32_t *grp_row0 = nullptr);

// The column masks of group g in shared memory (colmask[kt], whole CTA):
// bit r of colmask[c] is set when tile row r of the group holds a block in
// tile column c.  [*s0, *s1) receives the group's CSR slots.
__device__ void group_colmask(int g, int32_t kt, int32_t T, const int32_t *grp_row0,
                              const int32_t *grp_rows, const int32_t *row_ptr,
                              const int32_t *col_idx, uint32_t *colmask, int32_t *s0_out,
                              int32_t *s1_out) {
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
    *s0_out = s0;
    *s1_out = s1;
}

// Entries (non-empty tile columns) and slots (non-empty tiles) of group g
// from its column masks -> grp_cnt[2g], grp_cnt[2g + 1] (whole CTA).
__device__ void group_counts(int g, int32_t kt, const uint32_t *colmask, int32_t *grp_cnt) {
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
    __syncthreads();
}

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
    int32_t s0, s1;
    group_colmask(g, kt, T, grp_row0, grp_rows, row_ptr, col_idx, colmask, &s0, &s1);
    group_counts(g, kt, colmask, grp_cnt);
    if (!last_block_done(counts + kCntTicketGroups)) return;
    group_scan((int32_t)gridDim.x, grp_rows, grp_cnt, grp_ebeg, grp_sbeg, grp_ibeg, grp_wbeg,
               grp_wrow, grp_rbeg, ent_tbeg, counts);
}

// 4b. group offsets and the chunk size C = max(16, ceil(5E / 4G)); one block
// of 1024 threads (the group counts' last).  write_global: store the
// offsets and counts (else only `own`); own: the offsets of the groups
// g = blockIdx.x + i * gridDim.x at own[i] (with grp_row0), for a CTA that
// runs the scan for itself.
__device__ void group_scan(int32_t G, const int32_t *grp_rows, const int32_t *grp_cnt,
                           int32_t *grp_ebeg, int32_t *grp_sbeg, int32_t *grp_ibeg,
                           int32_t *grp_wbeg, int64_t *grp_wrow, int32_t *grp_rbeg,
                           int32_t *ent_tbeg, int32_t *counts, bool write_global,
                           GroupOff *own, const int32_t *grp_row0) {
    __shared__ int64_t sE;
    int64_t tot;
    // this thread's group among the first 1024, read once for both passes
    int64_t L0 = 0, S0 = 0, R0 = 0;
    int32_t Q0 = 0;
    {
        int64_t part = 0;
        for (int32_t g = threadIdx.x; g < G; g += 1024) {
            const int64_t L = __ldcg(grp_cnt + g * 2);
            if (g < 1024) {
                L0 = L;
                S0 = __ldcg(grp_cnt + g * 2 + 1);
                R0 = grp_rows[g];
                if (own) Q0 = grp_row0[g];
            }
            part += L;
        }
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
        const int64_t L = g < G ? (g0 == 0 ? L0 : __ldcg(grp_cnt + g * 2)) : 0;
        const int64_t S = g < G ? (g0 == 0 ? S0 : __ldcg(grp_cnt + g * 2 + 1)) : 0;
        const int32_t nch = g < G ? nchunks(L, C) : 0;
        const int64_t rows = g < G ? (g0 == 0 ? R0 : (int64_t)grp_rows[g]) * kTile : 0;
        int64_t v[6] = {L, S, nch, nch > 1 ? nch : 0, nch > 1 ? nch * rows : 0, nch > 1 ? 1 : 0};
        int64_t t[6];
        block_scan_n<6>(v, t);
        if (g < G && write_global) {
            grp_ebeg[g] = (int32_t)(be + v[0]);
            grp_sbeg[g] = (int32_t)(bs + v[1]);
            grp_ibeg[g] = (int32_t)(bi + v[2]);
            grp_wbeg[g] = (int32_t)(bw + v[3]);
            grp_wrow[g] = bwr + v[4];
            grp_rbeg[g] = (int32_t)(br + v[5]);
        }
        if (g < G && own && g % (int32_t)gridDim.x == (int32_t)blockIdx.x) {
            GroupOff &o = own[g / (int32_t)gridDim.x];
            o.row0 = g0 == 0 ? Q0 : grp_row0[g];
            o.rows = (int32_t)(rows / kTile);
            o.ebeg = (int32_t)(be + v[0]);
            o.eend = (int32_t)(be + v[0] + L);
            o.sbeg = (int32_t)(bs + v[1]);
            o.send = (int32_t)(bs + v[1] + S);
            o.ibeg = (int32_t)(bi + v[2]);
            o.wbeg = (int32_t)(bw + v[3]);
            o.wrow = bwr + v[4];
            o.rbeg = (int32_t)(br + v[5]);
            o.C = C;
        }
        be += t[0];
        bs += t[1];
        bi += t[2];
        bw += t[3];
        bwr += t[4];
        br += t[5];
    }
    if (threadIdx.x == 0 && write_global) {
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

__device__ __forceinline__ GroupOff load_group_off(int g, const int32_t *grp_row0,
                                                   const int32_t *grp_rows,
                                                   const int32_t *grp_ebeg,
                                                   const int32_t *grp_sbeg,
                                                   const int32_t *grp_ibeg,
                                                   const int32_t *grp_wbeg,
                                                   const int64_t *grp_wrow,
                                                   const int32_t *grp_rbeg,
                                                   const int32_t *counts, int32_t G) {
    GroupOff o;
    o.row0 = grp_row0[g];
    o.rows = grp_rows[g];
    o.ebeg = grp_ebeg[g];
    o.eend = grp_ebeg[g + 1];
    o.sbeg = grp_sbeg[g];
    o.send = g + 1 < G ? grp_sbeg[g + 1] : counts[kCntSlots];
    o.ibeg = grp_ibeg[g];
    o.wbeg = grp_wbeg[g];
    o.rbeg = grp_rbeg[g];
    o.wrow = grp_wrow[g];
    o.C = counts[kCntChunk];
    return o;
}

// Group g's fill, in three parts (whole CTA of 1024 threads for the first;
// slot_of[kt] in shared memory; [s0, s1) the group's CSR slots; o its
// offsets):
//  * group_fill_entries: entries (ascending tile column), slots (ascending
//    rows, one per tile) and slot_of from its column masks; with ent_s, the
//    entries' columns, first tiles and covers again, in three arrays of kt
//    in shared memory, from the group's first entry;
//  * group_fill_slots: block -> slot / offset (indexed by user position),
//    by threads [t0, t0 + nt) of the CTA; rp_s: the group's row pointers in
//    shared memory, rp_s[i] = row_ptr of block row row0 * T + i; pk: per
//    slot of the group, the block's user index, tile slot and offset;
//  * group_fill_items (one thread): items (near-equal chunks of the
//    group's entries) and workspace / reduction records.
__device__ void group_fill_entries(const GroupOff &o, int32_t kt, const uint32_t *colmask,
                                   int32_t *slot_of, int32_t *ent_col, int32_t *ent_tbeg,
                                   int32_t *ent_cover, int32_t *tile_row, int32_t *ent_s) {
    // column prefix over entries and slots, in chunks of blockDim (1024)
    int64_t eb = o.ebeg, sb = o.sbeg;
    for (int32_t c0 = 0; c0 < kt; c0 += 1024) {
        const int32_t c = c0 + threadIdx.x;
        const uint32_t mk = c < kt ? colmask[c] : 0u;
        int64_t te, ts;
        const int64_t xe = block_scan(mk != 0, &te);
        const int64_t xs = block_scan(__popc(mk), &ts);
        if (c < kt && mk) {
            const int32_t e = (int32_t)(eb + xe);
            slot_of[c] = (int32_t)(sb + xs);
            ent_col[e] = c;
            ent_tbeg[e] = (int32_t)(sb + xs);
            ent_cover[e] = (int32_t)(mk | (mk << 16));
            if (ent_s) {
                ent_s[e - o.ebeg] = c;
                ent_s[kt + e - o.ebeg] = (int32_t)(sb + xs);
                ent_s[2 * kt + e - o.ebeg] = (int32_t)(mk | (mk << 16));
            }
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
}

__device__ void group_fill_slots(const GroupOff &o, int32_t T, int32_t b, const int32_t *row_ptr,
                                 const int32_t *col_idx, const int32_t *perm,
                                 const uint32_t *colmask, const int32_t *slot_of, int32_t s0,
                                 int32_t s1, int32_t *blk_slot, int32_t *blk_off,
                                 const int32_t *rp_s, int32_t *pk, int t0n, int nt) {
    const int32_t t0 = o.row0, nrows = o.rows;
    for (int32_t s = s0 + (int32_t)threadIdx.x - t0n; s < s1; s += nt) {
        int32_t lo = t0 * T, hi = (t0 + nrows) * T;
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if ((rp_s ? rp_s[mid - t0 * T] : row_ptr[mid]) <= s) lo = mid; else hi = mid;
        }
        const int32_t br = lo, bc = col_idx[s];
        const int32_t tc = bc / T, trow = br / T - t0;
        const uint32_t mk = colmask[tc];
        const int32_t slot = slot_of[tc] + __popc(mk & ((1u << trow) - 1u));
        const int32_t p = perm[s];
        const int32_t off = ((br * b) % kTile) * kTile + (bc * b) % kTile;
        blk_slot[p] = slot;
        blk_off[p] = off;
        if (pk) {
            pk[3 * (s - s0)] = p;
            pk[3 * (s - s0) + 1] = slot;
            pk[3 * (s - s0) + 2] = off;
        }
    }
}

__device__ void group_fill_items(int g, const GroupOff &o, int32_t *items, int64_t *ws_row0,
                                 int32_t *red) {
    const int32_t e0 = o.ebeg, L = o.eend - e0, nch = nchunks(L, o.C);
    const int32_t base = L / nch, rem = L % nch;
    int32_t e = e0;
    for (int32_t c = 0; c < nch; ++c) {
        const int32_t sz = base + (c < rem ? 1 : 0);
        int32_t *it = items + (int64_t)(o.ibeg + c) * kItemFields;
        const int32_t ws = nch > 1 ? o.wbeg + c : -1;
        it[0] = g;
        it[1] = e;
        it[2] = e + sz;
        it[3] = c;
        it[4] = nch;
        it[5] = ws;
        if (ws >= 0) ws_row0[ws] = o.wrow + (int64_t)c * o.rows * kTile;
        e += sz;
    }
    if (nch > 1) {
        int32_t *rd = red + (int64_t)o.rbeg * 3;
        rd[0] = g;
        rd[1] = o.wbeg;
        rd[2] = nch;
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
    int32_t *slot_of = (int32_t *)(sm + kt); // kt: first slot of the column's entry
    const int g = blockIdx.x;
    const GroupOff o = load_group_off(g, grp_row0, grp_rows, grp_ebeg, grp_sbeg, grp_ibeg,
                                      grp_wbeg, grp_wrow, grp_rbeg, counts, (int32_t)gridDim.x);
    int32_t s0, s1;
    group_colmask(g, kt, T, grp_row0, grp_rows, row_ptr, col_idx, colmask, &s0, &s1);
    group_fill_entries(o, kt, colmask, slot_of, ent_col, ent_tbeg, ent_cover, tile_row, nullptr);
    __syncthreads();
    group_fill_slots(o, T, b, row_ptr, col_idx, perm, colmask, slot_of, s0, s1, blk_slot, blk_off,
                     nullptr, nullptr, 0, (int)blockDim.x);
    if (threadIdx.x == 0) group_fill_items(g, o, items, ws_row0, red);
}

// ------------------------------------------------ fused (cooperative) ---
// Dynamic tensor-core plans run the re-partition, the value packing and the
// stage records in ONE cooperative launch: every CTA is resident and the
// steps are separated by three grid barriers instead of seven kernel
// boundaries (each costs a few microseconds).  The arrays are the same as
// the launch chain's, bit for bit; the block CSR is built from a bitmap of
// each block row's block columns instead of a scatter and a row sort:
//   A. clear the bitmap, the count words and the status word      | barrier
//   B. validate; set each block's bit (a bit already set is a
//      repeated block)                                              | barrier,
//      then CTA 0 scans the bitmap's popcounts (row_ptr, and the
//      blocks before each bitmap word)
//      (a rejected pattern ends the launch here: nothing else is written)
//   C. place each block in the CSR after the set bits before it; per
//      group, the column masks (from the bitmap) and the entry / slot
//      counts                                                       | barrier,
//      then CTA 0 scans the groups (offsets, chunk size)
//   D. per group: the group's tiles cleared where blocks do not fill
//      them, its entries and slots (the chain's fill); then, side by side,
//      the stage records of the group's items (12 warps; an item's entries
//      are its group's, so no barrier is needed) and, on the other 20
//      warps, block -> slot, the items, and the blocks' values packed, a
//      warp per block (the group's row pointers and its blocks' slots in
//      shared memory).
// Barrier: each CTA counts its arrival on one counter.  Where no step
// follows, every CTA waits for the count; where one does (a scan), CTA 0
// waits, runs it and publishes the barrier's generation, which the other
// CTAs wait for.  Every wait is bounded; on expiry the status word records
// SPMM_ERR_TIMEOUT and the launch ends (the product launch then skips).
struct DynFusedArgs {
    const int32_t *d_nnzb, *brow, *bcol;
    int64_t cap;
    int32_t mb, kb, kw, kt, T, b, G;
    uint32_t *bits, *gmask;
    int32_t *wpre;           // per bitmap word: blocks in the CSR before it
    int32_t *bar;
    int32_t *row_cnt, *status, *row_ptr, *cursor, *counts, *col_idx, *perm;
    const int32_t *grp_row0, *grp_rows;
    int32_t *grp_cnt, *grp_ebeg, *grp_sbeg, *grp_ibeg, *grp_wbeg;
    int64_t *grp_wrow;
    int32_t *grp_rbeg;
    int32_t *ent_col, *ent_tbeg, *ent_cover, *tile_row, *blk_slot, *blk_off, *items;
    int64_t *ws_row0;
    int32_t *red;
    const void *values;      // user-order values (16-bit) or E4M3 codes
    const float *scales;     // E4M3 block scales
    void *packed;            // tiles
    float *tile_scale;       // E4M3 tile scales
    int32_t w8, tr, seg;     // E4M3 weights; transposed plan; 16-bit vector width (8, 4 or 1)
    int32_t ent_cap, tiles_cap;
    int64_t items_cap;
    uint32_t *srec, *sprog;
    unsigned long long wait_ns;
    int32_t stall;           // test hook: CTA 0 skips its first arrival
};

__device__ __forceinline__ unsigned long long dyn_timer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The grid barrier described above.  Each CTA adds one to the arrival
// counter bar[0] with a release reduction after a CTA barrier, so barrier
// `epoch` (1, 2, ...) is complete once the counter reaches epoch * grid; an
// acquire load that reads that value orders every CTA's writes before it.
// grid_sync: every CTA waits on the counter itself.  grid_sync_step: CTA 0
// waits, reads the status word, runs `step` (all its threads) and
// publishes the generation bar[1] = epoch (bit 30 set when the status word
// was not zero once every CTA had arrived), which the other CTAs wait for;
// all return false on a set status so that every CTA takes the same
// branch.  Both return false when a wait ran out (the status word then
// says so).
__device__ __forceinline__ void st_release(int32_t *p, int32_t v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_release_add(int32_t *p, int32_t v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int32_t ld_acquire(const int32_t *p) {
    int32_t v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int32_t ld_relaxed(const int32_t *p) {
    int32_t v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
constexpr int32_t kGenError = 1 << 30;

// Thread 0: waits until *word (masked) reaches `target`; false on expiry.
__device__ __forceinline__ bool wait_at_least(const int32_t *word, int32_t target, int32_t mask,
                                              unsigned long long lim, int32_t *seen) {
    const unsigned long long t0 = dyn_timer();
    int32_t v;
    while (((v = ld_acquire(word)) & mask) < target)
        if (dyn_timer() - t0 > lim) return false;
    *seen = v;
    return true;
}

__device__ bool grid_sync(int32_t *bar, int32_t epoch, int32_t *status, unsigned long long lim,
                          bool arrive = true) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (arrive) red_release_add(bar, 1);
        int32_t v;
        const bool ok = wait_at_least(bar, epoch * (int32_t)gridDim.x, 0x7fffffff, lim, &v);
        if (!ok) flag(status, kDevTimeout);
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

template <typename Step>
__device__ bool grid_sync_step(int32_t *bar, int32_t epoch, int32_t *status,
                               unsigned long long lim, Step step) {
    __shared__ int ok_s, err_s;
    __syncthreads();
    int32_t st = 0;   // CTA 0, thread 0: the status word once every CTA arrived
    if (threadIdx.x == 0) {
        red_release_add(bar, 1);
        int32_t v = 0;
        bool ok;
        if (blockIdx.x == 0) {
            ok = wait_at_least(bar, epoch * (int32_t)gridDim.x, 0x7fffffff, lim, &v);
            // ordered after the acquire above; read now, used after the step
            st = ld_relaxed(status);
        } else {
            ok = wait_at_least(bar + 1, epoch, kGenError - 1, lim, &v);
            err_s = (v & kGenError) != 0;
        }
        if (!ok) flag(status, kDevTimeout);
        ok_s = ok;
    }
    __syncthreads();
    if (!ok_s) return false;
    if (blockIdx.x != 0) return err_s == 0;
    step();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int32_t err = st != 0;
        st_release(bar + 1, epoch | (err ? kGenError : 0));
        err_s = err;
    }
    __syncthreads();
    return err_s == 0;
}

// After the bitmap is set: the exclusive prefix of the bitmap words'
// popcounts in row-major order into `wpre` (global or shared memory, 16-byte
// aligned), with write_rows row_ptr[r] = wpre[r * kw] and the block count,
// and with bits_out a copy of the bitmap (shared memory, 16-byte aligned)
// (1024 threads, each a contiguous run of whole 16-byte vectors of words;
// the bitmap is a 256-byte aligned allocation).
// Runs of up to kScanKeep words stay in registers between the count and
// the prefix; longer runs read the bitmap twice.
constexpr int kScanKeep = 8;

__device__ __forceinline__ void scan_bits_put(const DynFusedArgs &a, int64_t i, int32_t run,
                                              int64_t &nbnd, int32_t &r, bool write_rows) {
    if (write_rows && i == nbnd) {   // first word of block row r
        a.row_ptr[r] = run;
        ++r;
        nbnd += a.kw;
    }
}

__device__ __noinline__ void scan_bits(const DynFusedArgs &a, int32_t *wpre, bool write_rows,
                                       uint32_t *bits_out) {
    const int64_t W = (int64_t)a.mb * a.kw;
    int64_t q = (W + blockDim.x - 1) / blockDim.x;
    q = (q + 3) & ~(int64_t)3;                           // whole uint4 per thread
    const int64_t lo = min(W, (int64_t)threadIdx.x * q), hi = min(W, lo + q);
    const bool keep = q <= kScanKeep;
    uint32_t w[kScanKeep];
    int64_t local = 0;
    if (keep) {
#pragma unroll
        for (int u = 0; u < kScanKeep; u += 4) {
            const int64_t i = lo + u;
            if (i + 4 <= hi) {
                const uint4 v = __ldcg((const uint4 *)(a.bits + i));
                w[u] = v.x;
                w[u + 1] = v.y;
                w[u + 2] = v.z;
                w[u + 3] = v.w;
                if (bits_out) *(uint4 *)(bits_out + i) = v;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    w[u + j] = i + j < hi ? __ldcg(a.bits + i + j) : 0u;
                    if (bits_out && i + j < hi) bits_out[i + j] = w[u + j];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kScanKeep; ++u) local += __popc(w[u]);
    } else {
        for (int64_t i = lo; i < hi; i += 4) {
            if (i + 4 <= hi) {
                const uint4 v = __ldcg((const uint4 *)(a.bits + i));
                local += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
                if (bits_out) *(uint4 *)(bits_out + i) = v;
            } else {
                for (int64_t j = i; j < hi; ++j) {
                    const uint32_t v = __ldcg(a.bits + j);
                    local += __popc(v);
                    if (bits_out) bits_out[j] = v;
                }
            }
        }
    }
    int64_t total;
    int64_t run = block_scan(local, &total);
    // the first block row starting in [lo, hi) and its first word
    int32_t r = (int32_t)((lo + a.kw - 1) / a.kw);
    int64_t nbnd = (int64_t)r * a.kw;
    if (keep) {
#pragma unroll
        for (int u = 0; u < kScanKeep; u += 4) {
            const int64_t i = lo + u;
            if (i + 4 <= hi) {
                int4 o;
                o.x = (int32_t)run;
                scan_bits_put(a, i, o.x, nbnd, r, write_rows);
                run += __popc(w[u]);
                o.y = (int32_t)run;
                scan_bits_put(a, i + 1, o.y, nbnd, r, write_rows);
                run += __popc(w[u + 1]);
                o.z = (int32_t)run;
                scan_bits_put(a, i + 2, o.z, nbnd, r, write_rows);
                run += __popc(w[u + 2]);
                o.w = (int32_t)run;
                scan_bits_put(a, i + 3, o.w, nbnd, r, write_rows);
                run += __popc(w[u + 3]);
                *(int4 *)(wpre + i) = o;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (i + j < hi) {
                        wpre[i + j] = (int32_t)run;
                        scan_bits_put(a, i + j, (int32_t)run, nbnd, r, write_rows);
                        run += __popc(w[u + j]);
                    }
                }
            }
        }
    } else {
        for (int64_t i = lo; i < hi; ++i) {
            wpre[i] = (int32_t)run;
            scan_bits_put(a, i, (int32_t)run, nbnd, r, write_rows);
            run += __popc(__ldcg(a.bits + i));
        }
    }
    if (threadIdx.x == 0 && write_rows) {
        a.row_ptr[a.mb] = (int32_t)total;
        a.counts[kCntNnzb] = (int32_t)total;
    }
}

// The column masks of the group of tile rows [t0, t0 + nrows) from the
// bitmap (global, or its copy in shared memory) (bit r of colmask[c]: tile
// row r of the group holds a block in tile column c), into shared memory.
__device__ void group_colmask_bits(const DynFusedArgs &a, const uint32_t *bits, int32_t t0,
                                   int32_t nrows, uint32_t *colmask) {
    const uint32_t tmask = a.T >= 32 ? 0xffffffffu : ((1u << a.T) - 1u);
    const int32_t nb = nrows * a.T;                       // block rows of the group
    const uint32_t *base = bits + (int64_t)t0 * a.T * a.kw;
    for (int32_t c = threadIdx.x; c < a.kt; c += blockDim.x) {
        const int32_t bc = c * a.T;                       // first block column of tile column c
        const int32_t w = bc >> 5, sh = bc & 31;
        uint32_t mk = 0;
#pragma unroll 16
        for (int32_t j = 0; j < nb; ++j)
            if ((base[(int64_t)j * a.kw + w] >> sh) & tmask) mk |= 1u << (j / a.T);
        colmask[c] = mk;
    }
    __syncthreads();
}

// Shared memory of the fused launch: colmask[kt], slot_of[kt], the group's
// row pointers (at most 16 * 16 + 1), kFusedPk (user index, slot, offset)
// triples, the group's entries (three arrays of kt) and, from a 16-byte
// boundary, the packing warps' staging pieces (before step D: the bitmap
// prefix and the bitmap).
constexpr int kFusedPk = 4096;
constexpr int kStageWarps = 12;  // warps cutting stage records in step D
constexpr int kPackDepth = 8;    // blocks in flight per packing warp
constexpr int kMaxOwnGroups = 16;  // groups per CTA for the per-CTA group scan
// bitmap words whose prefix fits the packing staging area (per-CTA scan)
constexpr int64_t kLocalWords = (int64_t)(32 - kStageWarps) * kPackDepth * 512 / 4;
constexpr int kFusedRp = 16 * 16 + 1;
__host__ __device__ inline size_t fused_pack_buf_offset(int32_t kt) {
    return (sizeof(int32_t) * (5 * (size_t)kt + kFusedRp + 3 * (size_t)kFusedPk) + 15) / 16 * 16;
}
inline size_t fused_smem(int32_t kt) {
    return fused_pack_buf_offset(kt) + (size_t)(32 - kStageWarps) * kPackDepth * 512;
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

// Packs the blocks of CSR slots [s0, s1), a warp per block, on warps
// [w0, w0 + nw) of the CTA: their user index, slot and offset from `pk`
// (shared memory) when given, else read through perm / blk_slot / blk_off.
// `buf`: kPackDepth * 32 16-byte pieces of shared memory per packing warp.
__device__ void pack_group(const DynFusedArgs &a, int32_t s0, int32_t s1, const int32_t *pk,
                           int w0, int nw, uint4 *buf) {
    const int lane = threadIdx.x & 31, warp = (threadIdx.x >> 5) - w0;
    int32_t q0 = s0 + warp;
    if (pk && !a.w8 && a.b == 16 && a.seg == 8 && !a.tr) {
        // 16 x 16 blocks, 16-byte pieces: kPackDepth blocks per round copied
        // into shared memory (cp.async, all in flight together), then
        // stored (the block's 512 B is one piece per lane, row lane / 2,
        // half lane % 2, placed as pack_block_warp places it)
        const uint4 *v = (const uint4 *)a.values;
        uint16_t *o = (uint16_t *)a.packed;
        uint4 *wb = buf + (size_t)warp * kPackDepth * 32 + lane;
        const int i = lane >> 1, seg = lane & 1;
        const int toff = (i >> 3) * 128 + seg * 64 + (i & 7) * 8;
        for (; q0 < s1; q0 += kPackDepth * nw) {
            int32_t sl[kPackDepth];
#pragma unroll
            for (int u = 0; u < kPackDepth; ++u) {
                const int32_t qq = q0 + u * nw - s0;
                if (q0 + u * nw < s1) {
                    cp_async16(wb + u * 32, v + (int64_t)pk[3 * qq] * 32 + lane);
                    sl[u] = pk[3 * qq + 1];
                }
            }
            cp_async_wait_all();   // this lane's pieces
#pragma unroll
            for (int u = 0; u < kPackDepth; ++u)
                if (q0 + u * nw < s1)
                    *(uint4 *)(o + (int64_t)sl[u] * (kTile * kTile) + toff) = wb[u * 32];
        }
        return;
    }
    for (int32_t q = q0; q < s1; q += nw) {
        int64_t p;
        int32_t slot, off;
        if (pk) {
            p = pk[3 * (q - s0)];
            slot = pk[3 * (q - s0) + 1];
            off = pk[3 * (q - s0) + 2];
        } else {
            p = a.perm[q];
            slot = a.blk_slot[p];
            off = a.blk_off[p];
        }
        if (a.w8) {
            pack_block_e4m3_warp((const uint8_t *)a.values, a.scales, p, a.b, slot, off, a.tr,
                                 (uint8_t *)a.packed, a.tile_scale, lane);
            continue;
        }
        const uint16_t *v = (const uint16_t *)a.values;
        uint16_t *o = (uint16_t *)a.packed;
        switch (a.b * 16 + a.seg) {
            case 16 * 16 + 8: pack_block_warp<uint16_t, 16, 8>(v, p, slot, off, a.tr, o, lane); break;
            case 16 * 16 + 1: pack_block_warp<uint16_t, 16, 1>(v, p, slot, off, a.tr, o, lane); break;
            case 8 * 16 + 8: pack_block_warp<uint16_t, 8, 8>(v, p, slot, off, a.tr, o, lane); break;
            case 8 * 16 + 1: pack_block_warp<uint16_t, 8, 1>(v, p, slot, off, a.tr, o, lane); break;
            case 4 * 16 + 4: pack_block_warp<uint16_t, 4, 4>(v, p, slot, off, a.tr, o, lane); break;
            case 4 * 16 + 1: pack_block_warp<uint16_t, 4, 1>(v, p, slot, off, a.tr, o, lane); break;
            default: pack_block_warp<uint16_t, 1, 1>(v, p, slot, off, a.tr, o, lane); break;
        }
    }
}

// Named barrier 1 over the first n threads of the CTA (the stage warps),
// named barrier 2 over the packing warps (n threads).
__device__ __forceinline__ void sync_first(int n) {
    asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory");
}
__device__ __forceinline__ void sync_pack(int n) {
    asm volatile("bar.sync 2, %0;" ::"r"(n) : "memory");
}

// The stage records of group g's work items (the near-equal chunks of its
// entries, as group_fill writes them; read from its copy in shared memory,
// ent_s), cut by warps [0, nbw) of the CTA
// exactly as a CTA per item cuts them (32 entries per warp, the cut, a
// prefix of the stage counts, the write pass), with named barrier 1 between
// the passes; items at or past the items' capacity are skipped.
__device__ void build_group_stages(const DynFusedArgs &a, const GroupOff &o, int nbw,
                                   int32_t *bcounts, const int32_t *ent_s) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t L = o.eend - o.ebeg, nch = nchunks(L, o.C);
    const int32_t base = L / nch, rem = L % nch;
    int32_t e = o.ebeg;
    for (int32_t c = 0; c < nch; ++c) {
        const int32_t sz = base + (c < rem ? 1 : 0), e1 = e + sz;
        if ((int64_t)o.ibeg + c < a.items_cap) {
            const int32_t nb = (sz + 31) / 32;
            int32_t rec = e;
            for (int32_t b0 = 0; b0 < nb; b0 += nbw) {
                const int32_t bi = b0 + warp;
                const bool active = bi < nb;
                const int32_t eb = e + 32 * bi;
                BatchCut cut;
                if (active)   // entries indexed from the group's first
                    cut = cut_batch(eb - o.ebeg, e1 - o.ebeg, a.ent_cap, a.tiles_cap, ent_s,
                                    ent_s + a.kt, ent_s + 2 * a.kt);
                if (lane == 0) bcounts[warp] = active ? cut.nst : 0;
                sync_first(nbw * 32);
                int32_t off = rec, tot = 0;
                for (int w = 0; w < nbw; ++w) {
                    if (w < warp) off += bcounts[w];
                    tot += bcounts[w];
                }
                if (active) write_batch(cut, bi == nb - 1, off, a.srec, a.sprog);
                rec += tot;
                sync_first(nbw * 32);
            }
        }
        e = e1;
    }
}

__global__ void __launch_bounds__(1024, 1) dyn_tc_fused_kernel(const __grid_constant__ DynFusedArgs a) {
    pdl_enter();
    extern __shared__ uint32_t dsm[];   // see fused_smem
    __shared__ int32_t bcounts[32];
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    const unsigned long long lim = a.wait_ns;
    uint32_t *colmask = dsm;
    int32_t *slot_of = (int32_t *)(dsm + a.kt);
    int32_t *rp_s = slot_of + a.kt;
    int32_t *pk = rp_s + kFusedRp;
    int32_t *ent_s = pk + 3 * kFusedPk;
    uint4 *pack_buf = (uint4 *)((uint8_t *)dsm + fused_pack_buf_offset(a.kt));
    // the first group's rows (plan constants), read while A runs
    __shared__ int32_t row0_s, rows_s, err_s;
    __shared__ GroupOff go_s, own_s[kMaxOwnGroups];
    if (threadIdx.x == 0 && (int)blockIdx.x < a.G) {
        row0_s = a.grp_row0[blockIdx.x];
        rows_s = a.grp_rows[blockIdx.x];
    }
    // A.
    for (int64_t i = gt; i < (int64_t)a.mb * a.kw; i += gs) a.bits[i] = 0;
    if (gt < kCntCount) a.counts[gt] = 0;
    if (gt == 0) *a.status = 0;
    // (with the test hook on, CTA 0 does not arrive: every wait runs out)
    if (!grid_sync(a.bar, 1, a.status, lim, !(a.stall && blockIdx.x == 0))) return;
    // B.
    const int64_t raw = *a.d_nnzb;
    if (gt == 0 && (raw < 0 || raw > a.cap)) flag(a.status, kDevCapacity);
    const int64_t n = raw < 0 ? 0 : (raw > a.cap ? a.cap : raw);
    for (int64_t p = gt; p < n; p += gs) {
        const int32_t r = a.brow[p], c = a.bcol[p];
        if (r < 0 || r >= a.mb || c < 0 || c >= a.kb) {
            flag(a.status, kDevPattern);
            continue;
        }
        const uint32_t bit = 1u << (c & 31);
        if (atomicOr(&a.bits[(int64_t)r * a.kw + (c >> 5)], bit) & bit) flag(a.status, kDevPattern);
    }
    // The bitmap scan: run by every CTA for itself into shared memory (the
    // packing staging area, free until step D) when the prefix fits there,
    // else by CTA 0 between the barrier's arrivals and its release.  CTA 0
    // writes row_ptr either way.  A rejected pattern ends the launch here,
    // in every CTA.
    const int64_t W = (int64_t)a.mb * a.kw;
    const bool local_bits = W <= kLocalWords;
    // the bitmap's copy too where both fit (after the prefix, 16-byte aligned)
    const bool local_copy = ((W + 3) & ~(int64_t)3) + W <= kLocalWords;
    const int32_t *wpre = local_bits ? (const int32_t *)pack_buf : a.wpre;
    uint32_t *bits_s = (uint32_t *)pack_buf + ((W + 3) & ~(int64_t)3);
    const uint32_t *bits_c = local_copy ? bits_s : a.bits;
    if (local_bits) {
        if (!grid_sync(a.bar, 2, a.status, lim)) return;
        int32_t st = 0;
        if (threadIdx.x == 0) st = ld_relaxed(a.status);   // ordered after the barrier's acquire
        scan_bits(a, (int32_t *)pack_buf, blockIdx.x == 0, local_copy ? bits_s : nullptr);
        if (threadIdx.x == 0) err_s = st;
        __syncthreads();
        if (err_s != 0) return;
    } else if (!grid_sync_step(a.bar, 2, a.status, lim,
                               [&] { scan_bits(a, a.wpre, true, nullptr); })) {
        return;
    }
    // C.
    for (int64_t p = gt; p < n; p += gs) {
        const int32_t r = a.brow[p], c = a.bcol[p];
        const int64_t wi = (int64_t)r * a.kw + (c >> 5);
        const int32_t pos = wpre[wi] + __popc(bits_c[wi] & ((1u << (c & 31)) - 1u));
        a.col_idx[pos] = c;
        a.perm[pos] = (int32_t)p;
    }
    for (int g = blockIdx.x; g < a.G; g += gridDim.x) {
        const bool first = g == (int)blockIdx.x;
        group_colmask_bits(a, bits_c, first ? row0_s : a.grp_row0[g],
                           first ? rows_s : a.grp_rows[g], colmask);
        for (int32_t c = threadIdx.x; c < a.kt; c += blockDim.x)
            a.gmask[(int64_t)g * a.kt + c] = colmask[c];
        group_counts(g, a.kt, colmask, a.grp_cnt);
    }
    // The group scan: every CTA for itself (its own groups' offsets into
    // shared memory; CTA 0 also stores all of them) while each CTA has at
    // most kMaxOwnGroups groups, else CTA 0 between arrivals and release.
    const bool local_groups = a.G <= kMaxOwnGroups * (int)gridDim.x;
    if (local_groups) {
        if (!grid_sync(a.bar, 3, a.status, lim)) return;
        group_scan(a.G, a.grp_rows, a.grp_cnt, a.grp_ebeg, a.grp_sbeg, a.grp_ibeg, a.grp_wbeg,
                   a.grp_wrow, a.grp_rbeg, a.ent_tbeg, a.counts, blockIdx.x == 0, own_s,
                   a.grp_row0);
    } else if (!grid_sync_step(a.bar, 3, a.status, lim, [&] {
                   group_scan(a.G, a.grp_rows, a.grp_cnt, a.grp_ebeg, a.grp_sbeg, a.grp_ibeg,
                              a.grp_wbeg, a.grp_wrow, a.grp_rbeg, a.ent_tbeg, a.counts);
               })) {
        return;
    }
    // D.  Per group: the fill, then the group's stage records on warps
    // [0, kStageWarps) beside the value packing on the others.
    const int64_t tile_bytes = a.w8 ? kTile * kTile : kTile * kTile * 2;
    const int warp = threadIdx.x >> 5;
    for (int g = blockIdx.x; g < a.G; g += gridDim.x) {
        const bool first = g == (int)blockIdx.x;
        const int32_t t0 = first ? row0_s : a.grp_row0[g], nrows = first ? rows_s : a.grp_rows[g];
        if (threadIdx.x == 0)
            go_s = local_groups
                       ? own_s[(g - (int)blockIdx.x) / (int)gridDim.x]
                       : load_group_off(g, a.grp_row0, a.grp_rows, a.grp_ebeg, a.grp_sbeg,
                                        a.grp_ibeg, a.grp_wbeg, a.grp_wrow, a.grp_rbeg, a.counts,
                                        a.G);
        for (int32_t c = threadIdx.x; c < a.kt; c += blockDim.x)
            colmask[c] = a.gmask[(int64_t)g * a.kt + c];
        for (int32_t i = threadIdx.x; i <= nrows * a.T; i += blockDim.x)
            rp_s[i] = a.row_ptr[t0 * a.T + i];
        __syncthreads();
        const GroupOff go = go_s;
        if (a.b < 16) {
            // tiles hold several blocks: clear the group's tiles (and E4M3
            // scales); 16 x 16 blocks fill their tile and every scale
            const int64_t sb = go.sbeg, se = go.send;
            uint4 *t = (uint4 *)((uint8_t *)a.packed + sb * tile_bytes);
            const int64_t nv = (se - sb) * tile_bytes / 16;
            for (int64_t i = threadIdx.x; i < nv; i += blockDim.x) t[i] = make_uint4(0, 0, 0, 0);
            if (a.w8) {
                float *ts = a.tile_scale + sb * 16;
                for (int64_t i = threadIdx.x; i < (se - sb) * 16; i += blockDim.x) ts[i] = 0.f;
            }
        }
        const int32_t s0 = rp_s[0], s1 = rp_s[nrows * a.T];
        const bool stage = s1 - s0 <= kFusedPk;
        group_fill_entries(go, a.kt, colmask, slot_of, a.ent_col, a.ent_tbeg, a.ent_cover,
                           a.tile_row, ent_s);
        __syncthreads();   // the group's entries and slot_of, and the cleared tiles
        if (warp < kStageWarps) {
            build_group_stages(a, go, kStageWarps, bcounts, ent_s);
        } else {
            // the packing warps map the group's blocks to their slots, then pack
            const int t0n = kStageWarps * 32, nt = (32 - kStageWarps) * 32;
            group_fill_slots(go, a.T, a.b, a.row_ptr, a.col_idx, a.perm, colmask, slot_of, s0, s1,
                             a.blk_slot, a.blk_off, rp_s, stage ? pk : nullptr, t0n, nt);
            if ((int)threadIdx.x == t0n) group_fill_items(g, go, a.items, a.ws_row0, a.red);
            sync_pack(nt);
            pack_group(a, s0, s1, stage ? pk : nullptr, kStageWarps, 32 - kStageWarps,
                       pack_buf);
        }
        __syncthreads();
    }
}

inline unsigned grid_for(int64_t n, int threads, unsigned cap) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    return (unsigned)(g > cap ? cap : g);
}

}  // namespace

// The chain's row counts, tickets and error flags start out zero and its
// launches leave them so (the status word is written by the first launch):
// memsets only for a plan's first chain call, or after one that failed to
// enqueue.
static cudaError_t chain_prepare(spmm_plan *p, int32_t mb, cudaStream_t s) {
    DynBufs &d = p->dyn;
    cudaError_t e = cudaSuccess;
    if (!d.chain_clean) {
        e = cudaMemsetAsync(d.row_cnt, 0, sizeof(int32_t) * mb, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(p->d_counts, 0, sizeof(int32_t) * kCntCount, s);
    }
    d.chain_clean = false;   // until this call's launches are enqueued
    return e;
}

cudaError_t launch_dynamic_csr(spmm_plan *p, const spmm_dpattern *dp, cudaStream_t s) {
    DynBufs &d = p->dyn;
    const int32_t mb = (int32_t)(p->m / p->b), kb = (int32_t)(p->k / p->b);
    const int64_t cap = p->nnzb_max;
    cudaError_t e = chain_prepare(p, mb, s);
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
    e = cudaGetLastError();
    d.chain_clean = e == cudaSuccess;
    return e;
}

cudaError_t launch_dynamic_partition(spmm_plan *p, const spmm_dpattern *dp, cudaStream_t s) {
    DynBufs &d = p->dyn;
    const int32_t mb = (int32_t)(p->m / p->b), kb = (int32_t)(p->k / p->b);
    const int64_t cap = p->nnzb_max;
    const bool tc = p->kernel == SPMM_KERNEL_TC;
    cudaError_t e = chain_prepare(p, mb, s);
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
    e = cudaGetLastError();
    d.chain_clean = e == cudaSuccess;
    return e;
}


bool dyn_fused_supported(int dev) {
    int coop = 0;
    return cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop;
}

cudaError_t launch_dynamic_tc_fused(spmm_plan *p, const spmm_dpattern *dp, const void *d_values,
                                    const float *d_scales, cudaStream_t s) {
    DynBufs &d = p->dyn;
    DynFusedArgs a;
    a.d_nnzb = dp->d_nnzb;
    a.brow = dp->d_brow;
    a.bcol = dp->d_bcol;
    a.cap = p->nnzb_max;
    a.mb = (int32_t)(p->m / p->b);
    a.kb = (int32_t)(p->k / p->b);
    a.kw = (a.kb + 31) / 32;
    a.kt = (int32_t)(p->k / kTile);
    a.T = kTile / p->b;
    a.b = p->b;
    a.G = (int32_t)p->n_groups;
    a.bits = d.bits;
    a.gmask = d.gmask;
    a.wpre = d.wpre;
    a.bar = d.bar;
    a.row_cnt = d.row_cnt;
    a.status = p->d_status;
    a.row_ptr = p->d_row_ptr;
    a.cursor = d.cursor;
    a.counts = p->d_counts;
    a.col_idx = p->d_col_idx;
    a.perm = p->d_perm;
    a.grp_row0 = p->d_grp_row0;
    a.grp_rows = p->d_grp_rows;
    a.grp_cnt = d.grp_cnt;
    a.grp_ebeg = p->d_grp_ebeg;
    a.grp_sbeg = d.grp_sbeg;
    a.grp_ibeg = d.grp_ibeg;
    a.grp_wbeg = d.grp_wbeg;
    a.grp_wrow = d.grp_wrow;
    a.grp_rbeg = d.grp_rbeg;
    a.ent_col = p->d_ent_col;
    a.ent_tbeg = p->d_ent_tbeg;
    a.ent_cover = p->d_ent_cover;
    a.tile_row = p->d_tile_row;
    a.blk_slot = p->d_blk_slot;
    a.blk_off = p->d_blk_off;
    a.items = p->d_items;
    a.ws_row0 = p->d_ws_row0;
    a.red = p->d_red;
    a.values = d_values;
    a.scales = d_scales;
    a.packed = p->d_packed;
    a.tile_scale = p->d_tile_scale;
    a.w8 = p->wdt == SPMM_E4M3 ? 1 : 0;
    a.tr = p->transposed ? 1 : 0;
    // vector copies need aligned values and untransposed blocks
    const bool al = ((uintptr_t)d_values % 16) == 0 && !p->transposed;
    a.seg = al ? (p->b >= 8 ? 8 : (p->b == 4 ? 4 : 1)) : 1;
    stage_caps(p, &a.ent_cap, &a.tiles_cap);
    a.items_cap = d.items_cap;
    a.srec = p->d_srec;
    a.sprog = p->d_sprog;
    a.wait_ns = p->wait_ns ? p->wait_ns : 2000000000ull;
    a.stall = p->stall;
    // the kernel's shared-memory limit is set once per device for the
    // largest k of a dynamic TC plan (k / 16 <= kDynMaxTileCols)
    const size_t smem = fused_smem(a.kt);
    static std::atomic<uint64_t> attrs{0};
    cudaError_t e = set_smem_attrs_once(attrs, dyn_tc_fused_kernel,
                                        (int)fused_smem(kDynMaxTileCols), false);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dyn_tc_fused_kernel, 1024, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    const int grid = std::min(per_sm * std::max(p->sm_count, 1), kFusedMaxCtas);
    // the counts are cleared by the launch itself (step A); the barrier's
    // counter and generation here, unless the plan's last call left them
    // zero (its reduction launch, or a memset after a call without a
    // product, clears them)
    if (!d.bar_clean) e = cudaMemsetAsync(d.bar, 0, sizeof(int32_t) * 2, s);
    d.bar_clean = false;
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, dyn_tc_fused_kernel, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace spmm
