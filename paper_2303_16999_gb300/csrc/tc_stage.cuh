// Stage records and value packing of the tensor-core plans, shared by the
// product launches (k_tc.cu) and the fused dynamic re-partition
// (k_dynamic.cu): one statement of each rule, run by either.  No pointer
// here is __restrict__: in the fused launch these functions read arrays
// that other CTAs of the same launch wrote, which the read-only data path
// must not serve.
#ifndef SPMM_TC_STAGE_CUH
#define SPMM_TC_STAGE_CUH

#include <cuda_runtime.h>

#include <cstdint>

#include "spmm_internal.h"

namespace spmm {
namespace {

constexpr int kRecWords = 16;           // words per stage record
constexpr int kMmaStage = 32;           // MMAs per stage and row half (one per lane)
constexpr int kJointSlabs = 4;          // slabs of a joint X box
// A stage whose entries are 2 to 4 consecutive tile columns (record info
// bit 20) gets its X slabs in one TMA box of kJointSlabs slabs when X's map
// is 3-D; the slabs then lie 2048 B apart inside each 64-column half, the
// halves 8192 B apart.
constexpr uint32_t kJointBit = 1u << 20;
constexpr int kBuildWarps = 16;         // warps of a stage_build_kernel CTA

// Stages never span two 32-entry batches of an item, so the batches are cut
// independently: one CTA per work item, one warp per batch.  A warp cuts
// its batch exactly as the producers consume it (consecutive entries while
// the stage holds at most `ent_cap` X slabs, `tiles_cap` W tiles and
// kMmaStage MMAs per row half; one entry always fits), counts its stages,
// and after a CTA-wide prefix of the counts writes its records at
// e0 + (stages of earlier batches) + i, expanding every entry's row
// intervals (runs of covered rows cut at interval starts) into MMA words:
// slab | first W tile in the stage << 4 | first tile row << 12 | rows << 16,
// one list per row half (an interval across row 8 is cut there).  Dynamic
// plans read the item count and the status word on the device (a rejected
// pattern builds nothing).

// One batch of entries, cut: the per-lane state (lane i = entry eb + i)
// that the write pass needs.  The cut itself is the one serial part: from
// stage start j, the stage takes the longest run of entries that fits.
struct BatchCut {
    int32_t mcol, mtb;      // entry's tile column and first tile
    uint32_t mcov;          // covered rows | interval starts << 16
    int S, L, H;            // inclusive prefixes: tiles, MMAs of each half
    int nlo, nhi, mslots;   // this entry's MMAs per half and tiles
    int my_j, my_stage;     // start lane and index of this entry's stage
    int kst;                // lane k: start lane of stage k
    int cnt, nst;           // entries in the batch, stages
};

__device__ BatchCut cut_batch(int32_t eb, int32_t e1, int ent_cap, int tiles_cap,
                              const int32_t *ent_col, const int32_t *ent_tbeg,
                              const int32_t *ent_cover) {
    const int lane = threadIdx.x & 31;
    BatchCut c;
    const int32_t e = eb + lane;
    const bool valid = e < e1;
    c.mcol = valid ? ent_col[e] : 0;
    c.mtb = valid ? ent_tbeg[e] : 0;
    c.mcov = valid ? (uint32_t)ent_cover[e] : 0u;
    const uint32_t cov = c.mcov & 0xFFFFu;
    // this entry's MMAs per row half: intervals below / above row 8, an
    // interval across it counting in both
    int nlo = 0, nhi = 0;
    for (uint32_t st = c.mcov >> 16; st; st &= st - 1) {
        const uint32_t r0 = __ffs(st) - 1;
        const uint32_t rest = st & (st - 1);
        const uint32_t next = rest ? (uint32_t)(__ffs(rest) - 1) : 16u;
        uint32_t len = (uint32_t)__ffs(~(cov >> r0)) - 1;   // run of covered rows
        len = len < next - r0 ? len : next - r0;
        nlo += r0 < 8;
        nhi += r0 + len > 8;
    }
    c.nlo = nlo;
    c.nhi = nhi;
    c.mslots = __popc(cov);
    // inclusive prefix sums over the batch: tiles, MMAs of each half
    int S = c.mslots, L = nlo, H = nhi;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int s2 = __shfl_up_sync(0xffffffffu, S, o);
        const int l2 = __shfl_up_sync(0xffffffffu, L, o);
        const int h2 = __shfl_up_sync(0xffffffffu, H, o);
        if (lane >= o) {
            S += s2;
            L += l2;
            H += h2;
        }
    }
    c.S = S;
    c.L = L;
    c.H = H;
    c.cnt = min(32, e1 - eb);
    c.my_j = 0;
    c.my_stage = 0;
    c.kst = 0;
    int nst = 0;
    for (int j = 0; j < c.cnt; ++nst) {
        // sums are monotone: the fitting lanes are contiguous from j
        const int Sb = j ? __shfl_sync(0xffffffffu, S, j - 1) : 0;
        const int Lb = j ? __shfl_sync(0xffffffffu, L, j - 1) : 0;
        const int Hb = j ? __shfl_sync(0xffffffffu, H, j - 1) : 0;
        const bool fits = lane >= j && lane < j + ent_cap && lane < c.cnt &&
                          S - Sb <= tiles_cap && L - Lb <= kMmaStage && H - Hb <= kMmaStage;
        const int nent = __popc(__ballot_sync(0xffffffffu, fits));
        if (lane >= j && lane < j + nent) {
            c.my_j = j;
            c.my_stage = nst;
        }
        if (lane == nst) c.kst = j;
        j += nent;
    }
    c.nst = nst;
    return c;
}

// The write pass of a cut batch, every stage at once: stores its records
// from record index `rec`, expanding every entry's row intervals (runs of
// covered rows cut at interval starts) into MMA words: slab | first W tile
// in the stage << 4 | first tile row << 12 | rows << 16, one list per row
// half (an interval across row 8 is cut there).
__device__ void write_batch(const BatchCut &c, bool last_batch, int32_t rec, uint32_t *srec,
                            uint32_t *sprog) {
    const int lane = threadIdx.x & 31;
    const bool in = lane < c.cnt;
    // the prefixes before this entry's stage
    const int src = in && c.my_j > 0 ? c.my_j - 1 : 0;
    const int Sp = __shfl_sync(0xffffffffu, c.S, src);
    const int Lp = __shfl_sync(0xffffffffu, c.L, src);
    const int Hp = __shfl_sync(0xffffffffu, c.H, src);
    if (in) {
        const bool first = c.my_j == 0;
        uint32_t klo = (uint32_t)(c.L - c.nlo - (first ? 0 : Lp));
        uint32_t khi = (uint32_t)(c.H - c.nhi - (first ? 0 : Hp));
        uint32_t toff = (uint32_t)(c.S - c.mslots - (first ? 0 : Sp));
        const uint32_t slab = (uint32_t)(lane - c.my_j);
        const uint32_t cov = c.mcov & 0xFFFFu;
        uint32_t *pr = sprog + (int64_t)(rec + c.my_stage) * 2 * kMmaStage;
        for (uint32_t st = c.mcov >> 16; st; st &= st - 1) {
            const uint32_t r0 = __ffs(st) - 1;
            const uint32_t rest = st & (st - 1);
            const uint32_t next = rest ? (uint32_t)(__ffs(rest) - 1) : 16u;
            uint32_t len = (uint32_t)__ffs(~(cov >> r0)) - 1;
            len = len < next - r0 ? len : next - r0;
            if (r0 < 8) {
                const uint32_t l0 = r0 + len > 8 ? 8 - r0 : len;
                pr[2 * klo++] = slab | toff << 4 | r0 << 12 | l0 << 16;
            }
            if (r0 + len > 8) {
                const uint32_t a = r0 < 8 ? 8u : r0;   // first row at or above 8
                pr[2 * khi++ + 1] = slab | (toff + (a - r0)) << 4 | a << 12 | (r0 + len - a) << 16;
            }
            toff += len;
        }
    }
    // bit i: entry i is not one tile column past entry i - 1
    const int32_t pcol = __shfl_up_sync(0xffffffffu, c.mcol, 1);
    const uint32_t brk = __ballot_sync(0xffffffffu, lane > 0 && c.mcol != pcol + 1);
    // records, kRecWords words per stage: word 0 the MMA counts, entry
    // count and flags, 1 the stage's tiles, 2 its first tile, 3 + i the X
    // column of its entry i
    for (int w0 = 0; w0 < c.nst * kRecWords; w0 += 32) {
        const int w = w0 + lane;
        const int k = min(w / kRecWords, c.nst - 1), i = w % kRecWords;
        const int j = __shfl_sync(0xffffffffu, c.kst, k);
        const int jn0 = __shfl_sync(0xffffffffu, c.kst, min(k + 1, 31));
        const int jn = k + 1 < c.nst ? jn0 : c.cnt;
        const int nent = jn - j;
        const int Se = __shfl_sync(0xffffffffu, c.S, jn - 1);
        const int Le = __shfl_sync(0xffffffffu, c.L, jn - 1);
        const int He = __shfl_sync(0xffffffffu, c.H, jn - 1);
        const int Sb0 = __shfl_sync(0xffffffffu, c.S, max(j - 1, 0));
        const int Lb0 = __shfl_sync(0xffffffffu, c.L, max(j - 1, 0));
        const int Hb0 = __shfl_sync(0xffffffffu, c.H, max(j - 1, 0));
        const int32_t stb = __shfl_sync(0xffffffffu, c.mtb, j);
        const int32_t xc = __shfl_sync(0xffffffffu, c.mcol, min(j + max(i - 3, 0), 31));
        if (w < c.nst * kRecWords) {
            const int Sb = j ? Sb0 : 0, Lb = j ? Lb0 : 0, Hb = j ? Hb0 : 0;
            const bool joint = nent >= 2 && nent <= kJointSlabs &&
                               ((brk >> (j + 1)) & ((1u << (nent - 1)) - 1u)) == 0;
            const bool last = last_batch && jn == c.cnt;
            uint32_t v = 0;
            if (i == 0)
                v = (uint32_t)(Le - Lb) | (uint32_t)(He - Hb) << 6 | (uint32_t)nent << 12 |
                    (joint ? kJointBit : 0u) | (last ? 0x80000000u : 0u);
            else if (i == 1) v = (uint32_t)(Se - Sb);
            else if (i == 2) v = (uint32_t)stb;
            else if (i - 3 < nent) v = (uint32_t)xc;
            srec[(int64_t)(rec + k) * kRecWords + i] = v;
        }
    }
}

// The stage records of one work item (fields as in the items array), cut by
// all warps of the calling CTA, 32 entries per warp at a time; `counts`
// holds one int per warp of the CTA (shared memory).
__device__ void build_item_stages(const int32_t *it, int ent_cap, int tiles_cap,
                                  const int32_t *ent_col,
                                  const int32_t *ent_tbeg,
                                  const int32_t *ent_cover,
                                  uint32_t *srec, uint32_t *sprog,
                                  int32_t *counts) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = (int)(blockDim.x >> 5);
    const int32_t e0 = it[1], e1 = it[2];
    const int32_t nb = (e1 - e0 + 31) / 32;
    int32_t base = e0;
    for (int32_t b0 = 0; b0 < nb; b0 += nwarps) {
        const int32_t b = b0 + warp;
        const bool active = b < nb;
        const int32_t eb = e0 + 32 * b;
        BatchCut cut;
        if (active) cut = cut_batch(eb, e1, ent_cap, tiles_cap, ent_col, ent_tbeg, ent_cover);
        if (lane == 0) counts[warp] = active ? cut.nst : 0;
        __syncthreads();
        int32_t off = base, tot = 0;
        for (int w = 0; w < nwarps; ++w) {
            if (w < warp) off += counts[w];
            tot += counts[w];
        }
        if (active) write_batch(cut, b == nb - 1, off, srec, sprog);
        base += tot;
        __syncthreads();
    }
}

// Tile layout of the MMA B operand, K-major without swizzle: 8 x 8 core
// matrices of 128 contiguous bytes; element (i = row of W in the tile,
// j = column) at byte (i/8)*256 + (j/8)*128 + (i%8)*16 + (j%8)*2.
// One thread per (block, row, segment of SEG columns): it reads SEG
// consecutive values of the block row and writes them as one piece of an
// 8 x 8 core-matrix row (SEG = min(b, 8): 8 or 16 bytes of 16-bit values;
// SEG = 1 for values not aligned to a segment).
template <typename U, int B, int SEG>
__device__ __forceinline__ void pack_tiles_range(const U *vals,
                                                 const int32_t *blk_slot,
                                                 const int32_t *blk_off,
                                                 int64_t nnzb, int tr, U *out,
                                                 int64_t t0, int64_t stride) {
    constexpr int kSeg = SEG;                           // values per thread
    constexpr int kPer = B * (B / kSeg);                // threads per block
    const int64_t total = nnzb * kPer;
    for (int64_t t = t0; t < total; t += stride) {
        const int64_t p = t / kPer;
        const int r = (int)(t - p * kPer);
        const int i = r / (B / kSeg), seg = r % (B / kSeg);   // block row, segment
        const int off = blk_off[p];
        const int ti = off / kTile + i, tj = off % kTile + seg * kSeg;
        // transposed plans (SEG = 1 only): element (i, j) is W's (j, i)
        const U *src = vals + p * (B * B) + (tr ? seg * B + i : i * B + seg * kSeg);
        U *dst = out + (int64_t)blk_slot[p] * (kTile * kTile) + (ti >> 3) * 128 + (tj >> 3) * 64 +
                 (ti & 7) * 8 + (tj & 7);
        if constexpr (kSeg == 8) {
            *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(src);
        } else if constexpr (kSeg == 4) {
            *reinterpret_cast<uint2 *>(dst) = *reinterpret_cast<const uint2 *>(src);
        } else {
            *dst = *src;
        }
    }
}

// E4M3 tiles: codes row-major (16 x 16 bytes per slot) and, per slot, the
// scale of each 4 x 4 sub-square (the block covering it: one scale for
// b = 16, four for b = 8, sixteen for b = 4).
__device__ __forceinline__ void pack_tiles_e4m3_range(const uint8_t *codes,
                                                      const float *scales,
                                                      const int32_t *blk_slot,
                                                      const int32_t *blk_off,
                                                      int64_t nnzb, int b, int tr,
                                                      uint8_t *out,
                                                      float *tile_scale, int64_t t0,
                                                      int64_t stride) {
    const int bb = b * b;
    const int64_t total = nnzb * bb;
    for (int64_t t = t0; t < total; t += stride) {
        const int64_t p = t / bb;
        const int e = (int)(t - p * bb);
        const int off = blk_off[p];
        const int ti = off / kTile + e / b, tj = off % kTile + e % b;
        const int64_t s = blk_slot[p];
        // transposed plans: element (i, j) is W's (j, i); a block's scale is
        // the same either way
        out[s * (kTile * kTile) + ti * kTile + tj] = codes[tr ? p * bb + (e % b) * b + e / b : t];
        if ((ti & 3) == 0 && (tj & 3) == 0) tile_scale[s * 16 + (ti >> 2) * 4 + (tj >> 2)] = scales[p];
    }
}

// One block's values into its tile by the 32 lanes of a warp, with the
// element placement of pack_tiles_range (block p of the user order, tile
// slot `slot`, offset `off` = row * 16 + column of the block in the tile).
template <typename U, int B, int SEG>
__device__ __forceinline__ void pack_block_warp(const U *vals, int64_t p, int32_t slot,
                                                int32_t off, int tr, U *out, int lane) {
    constexpr int kSeg = SEG;
    constexpr int kPer = B * (B / kSeg);
    for (int r = lane; r < kPer; r += 32) {
        const int i = r / (B / kSeg), seg = r % (B / kSeg);
        const int ti = off / kTile + i, tj = off % kTile + seg * kSeg;
        const U *src = vals + p * (B * B) + (tr ? seg * B + i : i * B + seg * kSeg);
        U *dst = out + (int64_t)slot * (kTile * kTile) + (ti >> 3) * 128 + (tj >> 3) * 64 +
                 (ti & 7) * 8 + (tj & 7);
        if constexpr (kSeg == 8) {
            *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(src);
        } else if constexpr (kSeg == 4) {
            *reinterpret_cast<uint2 *>(dst) = *reinterpret_cast<const uint2 *>(src);
        } else {
            *dst = *src;
        }
    }
}

// The same for E4M3 codes and the block's scale (pack_tiles_e4m3_range's
// placement).
__device__ __forceinline__ void pack_block_e4m3_warp(const uint8_t *codes, const float *scales,
                                                     int64_t p, int b, int32_t slot, int32_t off,
                                                     int tr, uint8_t *out, float *tile_scale,
                                                     int lane) {
    const int bb = b * b;
    for (int e = lane; e < bb; e += 32) {
        const int ti = off / kTile + e / b, tj = off % kTile + e % b;
        const int64_t s = slot;
        out[s * (kTile * kTile) + ti * kTile + tj] =
            codes[tr ? p * bb + (e % b) * b + e / b : p * bb + e];
        if ((ti & 3) == 0 && (tj & 3) == 0) tile_scale[s * 16 + (ti >> 2) * 4 + (tj >> 2)] = scales[p];
    }
}

}  // namespace
}  // namespace spmm

#endif
