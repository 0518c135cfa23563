// Tensor-core block-sparse kernel for b in {4, 8, 16}, and for b = 1 where
// tiles fill (Section 3.1: b x b blocks hold all non-zeros; b = 16 is one
// 16 x 16 tile, smaller blocks are packed into 16 x 16 tiles with zero fill).
//
// The product is computed transposed, Y^T = X^T W^T, so one MMA is
//   D[128 n x 16 m] += A[128 n x 16 k] * B[16 k x 16 m]
// with A = a 16-row slab of X (read by TMA straight from X's row-major
// layout, i.e. MN-major), B = one packed W tile (K-major), D = FP32 in TMEM.
// A CTA owns a group of up to 16 tile rows (256 rows of Y) and 128 columns
// of n; it walks the union of the group's tile columns ("entries"), loading
// each X slab once and applying it to every tile of that column, with one
// TMEM accumulator (16 columns) per tile row.  The planner covers each
// entry's rows by intervals of consecutive rows (zero tiles fill the gaps);
// one MMA with N = 16 x (interval length) serves an interval, since below
// N = 128 an MMA costs about the reads of its 4 KB A operand.  Accumulators
// start at zero in TMEM (the epilogue clears what it reads), so every MMA
// accumulates.
//
// Pipeline: a stage holds up to StageGeom::ent entries (X slabs) and up to
// StageGeom::tiles W tiles, in one of two geometries the plan picks (dense
// or sparse tiles).  How a work item's entries fall into stages, and the
// MMAs of each stage (one word per MMA: slab, first W tile, first tile row,
// rows; one list per half of the tile rows), is fixed by the plan, so
// stage_build_kernel writes it once per plan (every call for dynamic plans)
// as stage records.  Three producer warps follow the records with three in
// flight: warp 0 copies the stage's W tiles (contiguous in the packed array,
// one bulk copy) and its MMA program into shared memory, warps 6 and 7
// request the two halves of its X slabs (one TMA per slab, both 64-column
// halves in one 3-D box when n is a multiple of 64).  Issuing a copy costs
// its warp a few hundred cycles, so they run side by side.  Two MMA warps
// (1: tile rows 0-7, 8: rows 8-15) stay converged: each lane loads one
// program word and the warp walks them with one shuffle per MMA, issuing
// through elect.sync; each owns its accumulator columns, so the order of
// accumulation into every column is fixed.  With two stages the ring is
// bound by the copy latency (a stage is refilled only after its MMAs
// complete): each role spends about a third of a stage waiting.
//
// Wide launches (stage geometries 2 and 3): one CTA per SM covers two
// 128-column tiles of n with all 512 TMEM columns; each stage holds both
// tiles' X slabs and one set of W tiles, and every MMA word is issued once
// per tile, so each W tile is read from L2 once per 256 columns.  Four MMA
// warps (row half x column tile) keep the issue rate of two narrow CTAs.
//
// Warp roles (288 threads; wide: 352, wide sparse-tile: 416): warp 0 = W
// producer, warps 1 and 8 = MMA issuers (warp 1 owns TMEM; wide: 9 and 10
// issue the second column tile's MMAs), warps 2..5 = epilogue (TMEM ->
// registers -> Y or workspace) and, for E4M3 weights, converters, warps 6
// and 7 = X producers (wide: one column tile each; wide sparse-tile: warps
// 11 and 12 take a share of each tile's slabs).
// Every mbarrier wait is bounded (globaltimer); on expiry the CTA records
// SPMM_ERR_TIMEOUT in the plan's status word, stops, frees TMEM and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "pdl.cuh"
#include "spmm_internal.h"
#include "tc_ptx.cuh"
#include "tc_stage.cuh"

namespace spmm {
namespace {

// Launch geometry (compile-time; overridable for experiments)
#ifndef SPMM_TC_CTAS
#define SPMM_TC_CTAS 2      // CTAs per SM
#endif
#ifndef SPMM_TC_RCAP
#define SPMM_TC_RCAP 16     // tile rows per group (accumulator columns / 16)
#endif
#ifndef SPMM_TC_ACCBUFS
#define SPMM_TC_ACCBUFS 1   // accumulator sets per CTA (2 needs one CTA per SM)
#endif
// Stage geometries (stages, X slabs and W tiles per stage, all in about
// 110 KB of shared memory per CTA), for 16-bit and for E4M3 weights.  The plan picks one
// by its tiles per entry: few-tile entries (sparse tiles) need many slabs
// per stage to amortise the stage's fixed costs, many-tile entries need
// room for their tiles.  Measured on m = k = 4096, n = 2048: the dense
// geometry takes b=1 d=1/4 from 70 to 58 us, the sparse one b=16 d=1/32
// from 25 to 21 us, against one geometry of 4 slabs x 32 tiles x 3 stages.
#ifndef SPMM_TC_STAGES_D
#define SPMM_TC_STAGES_D 2  // dense: 4 slabs, 64 tiles
#endif
#ifndef SPMM_TC_ENT_D
#define SPMM_TC_ENT_D 4
#endif
#ifndef SPMM_TC_TILES_D
#define SPMM_TC_TILES_D 64
#endif
// Two column tiles per CTA (one CTA per SM), dense tiles: 2 x 4 slabs and
// 64 tiles in each of 3 stages.  Measured at b = 1 against smaller stages
// in the same shared memory: 2 x 3 slabs, 48 tiles, 4 stages 65 us; 2 x 2
// slabs, 32 tiles, 6 stages 80 us; this one 59 us (each stage's fixed
// costs, not the bytes in flight, set the pace).
#ifndef SPMM_TC_STAGES_W
#define SPMM_TC_STAGES_W 3
#endif
#ifndef SPMM_TC_STAGES_WS
#define SPMM_TC_STAGES_WS 2  // sparse tiles, two column tiles: 2 x 8 slabs, 44 tiles
#endif
#ifndef SPMM_TC_WIDE_MIN
#define SPMM_TC_WIDE_MIN 3  // wide launches need work units >= this x SMs / 2
#endif
#ifndef SPMM_TC_STAGES_S
#define SPMM_TC_STAGES_S 2  // sparse: 8 slabs, 44 tiles
#endif
#ifndef SPMM_TC_ENT_S
#define SPMM_TC_ENT_S 8
#endif
#ifndef SPMM_TC_TILES_S
#define SPMM_TC_TILES_S 44
#endif
#ifndef SPMM_TC_STAGES8
#define SPMM_TC_STAGES8 3   // E4M3 weights, dense: 4 slabs, 24 tiles
#endif
#ifndef SPMM_TC_ENT8
#define SPMM_TC_ENT8 4
#endif
#ifndef SPMM_TC_TILES8
#define SPMM_TC_TILES8 24
#endif
#ifndef SPMM_TC_STAGES8_S
#define SPMM_TC_STAGES8_S 2 // E4M3 weights, sparse: 8 slabs, 26 tiles
#endif
#ifndef SPMM_TC_ENT8_S
#define SPMM_TC_ENT8_S 8
#endif
#ifndef SPMM_TC_TILES8_S
#define SPMM_TC_TILES8_S 26 // the most that leaves two CTAs per SM
#endif
constexpr int kSlabBytes = kTile * kNTile * 2;                    // 4096: 16 k x 128 n, 16-bit
constexpr int kTileBytes8 = kTile * kTile;                        // 256: E4M3 tile, row-major
constexpr int kScaleBytes = 16 * 4;                               // per slot: 4 x 4 sub-square scales
constexpr int kStagesMax = 8;                                     // >= every geometry's stages
constexpr int kRowCap = SPMM_TC_RCAP;
constexpr int kAccCols = kRowCap * kTile;                         // TMEM columns per buffer
constexpr int kMaxBatch = 64;                                     // problems per launch

// Stage layout: X slabs (of each column tile the CTA covers) | 16-bit W
// tiles (MMA B operand) | (E4M3 only) the FP8 codes and their scales as
// loaded, which the converter warps expand into the 16-bit area.
// GEO: 0 = dense, 1 = sparse; 2 and 3 = the same over two column tiles per
// CTA ("wide": one CTA per SM, each W tile serves 256 columns of n; the
// same entry and tile caps, hence the same stage records, as GEO - 2).
template <bool W8, int GEO> struct StageGeom {
    static constexpr int base = GEO & 1;            // dense (0) or sparse (1) tiles
    static constexpr int sets = GEO >= 2 ? 2 : 1;   // column tiles per CTA
    // X producer warps per column tile in wide CTAs: sparse-tile stages
    // carry up to 2 x 8 separate slab copies, so two warps share each tile's
    static constexpr int xprod = GEO == 3 ? 2 : 1;
    static constexpr int producers = sets > 1 ? 1 + sets * xprod : 3;   // W + X warps
    static constexpr int threads = GEO == 3 ? 416 : sets > 1 ? 352 : 288;
    static constexpr int mma_warps = 2 * sets;      // one per row half and column tile
    // E4M3 weights: the same stage shapes whether a CTA covers one column
    // tile or two (its W tiles, codes and scales serve both)
    static constexpr int stages = W8 ? (base ? SPMM_TC_STAGES8_S : SPMM_TC_STAGES8)
                                     : GEO == 3   ? SPMM_TC_STAGES_WS
                                       : GEO == 2 ? SPMM_TC_STAGES_W
                                       : GEO      ? SPMM_TC_STAGES_S
                                                  : SPMM_TC_STAGES_D;
    static constexpr int ent = W8 ? (base ? SPMM_TC_ENT8_S : SPMM_TC_ENT8)
                                  : (base ? SPMM_TC_ENT_S : SPMM_TC_ENT_D);   // X slabs
    static constexpr int tiles = W8 ? (base ? SPMM_TC_TILES8_S : SPMM_TC_TILES8)
                                    : (base ? SPMM_TC_TILES_S : SPMM_TC_TILES_D);
    static_assert(stages <= kStagesMax && ent <= 12 && tiles >= 16, "stage geometry");
    // a joint box of consecutive slabs must fit one column tile's slab area
    static_assert(sets == 1 || ent >= kJointSlabs, "wide stage entries");
    static constexpr int xset = ent * kSlabBytes;    // X bytes of one column tile
    static constexpr int w16 = sets * xset;
    static constexpr int w8 = w16 + tiles * kTileBytes16;
    static constexpr int sc = w8 + tiles * kTileBytes8;
    // every stage starts on a 1024-byte boundary: the 128-byte-swizzled X
    // slabs (TMA destinations and MMA A operands) need it
    static constexpr int bytes = ((W8 ? sc + tiles * kScaleBytes : w8) + 1023) / 1024 * 1024;
    static_assert(bytes % 1024 == 0 && xset % 1024 == 0, "swizzle-aligned stages");
};
// Two CTAs share an SM: each holds one accumulator set (256 of the SM's 512
// TMEM columns) and half the shared memory, so the two CTAs' producer / MMA
// pipelines run side by side and one CTA's epilogue overlaps the other's MMAs.
// (A single warp cannot issue its copies and MMAs faster than its own
// dependent scalar work allows; a second pipeline per SM doubles that rate.)
constexpr int kAccBufs = SPMM_TC_ACCBUFS;
static_assert(kAccBufs * SPMM_TC_CTAS * SPMM_TC_RCAP * 16 <= 512, "TMEM columns per SM");
constexpr int kCtasPerSm = SPMM_TC_CTAS;
static_assert(kRowCap <= kMaxGroupRows && kRowCap <= 16, "a stage must hold a full entry");
constexpr int kThreads = 288;                                     // one column tile per CTA
constexpr int kMmaWarpsMax = 4;
constexpr int kXWarp0 = 6, kXWarp1 = 7;                           // X-slab producers (two halves)
constexpr int kXWarp2 = 11;                                       // wide sparse: warps 11, 12 as well
constexpr int kMmaWarpHi = 8;                                     // MMAs of tile rows 8-15
constexpr int kProducersMax = 5;                                  // W + up to four X
constexpr unsigned long long kWaitNs = 2000000000ull;             // 2 s: default per wait, and
                                                                  // every wait of the abort drain

// A stage's MMA program: one word per MMA (slab index in the stage | first
// W tile in the stage << 4 | first tile row << 12 | rows << 16), so the MMA
// warps decode nothing on their critical path.  Two MMA warps split the
// accumulator by tile rows (0-7 and 8-15; an interval crossing row 8 becomes
// two MMAs), so each TMEM column is written by one warp in a fixed order.
// (StageGeom checks that a stage record's 12 X columns suffice)
// Stage record (built before the launch; a work item's stages are records
// e0, e0 + 1, ... where e0 is its first entry, since every stage holds at
// least one entry): info (MMAs of rows 0-7 | MMAs of rows 8-15 << 6 |
// entries << 12 | last << 31), W tiles, first W tile, the X column of each
// entry; the stage's MMA program lives in a parallel array of 2 x kMmaStage
// words per record, (rows 0-7 word, rows 8-15 word) pairs.
struct StageMeta {
    uint32_t info;                 // as in the stage record
    uint32_t nslots;               // W tiles in the stage
    uint32_t prog[2][kMmaStage];   // MMA words of rows 0-7 and of rows 8-15
};

// Control block after the stages; S = the geometry's stage count.
template <int S> struct __align__(8) SmemT {
    uint64_t full[S], empty[S], conv[S], accf[kAccBufs], acce[kAccBufs];
    uint64_t drain;                // abort: one tcgen05.commit per MMA warp
    uint64_t never;                // failure-detection tests: nothing arrives here
    StageMeta meta[S];
    uint32_t tmem_base;
    volatile int32_t abort_flag;
    int32_t issued[kProducersMax], consumed[kMmaWarpsMax];   // per producer / per MMA warp
    int64_t nunits;
    int32_t epi_ok[2];             // accumulator-ready outcome, per unit parity
};

// ------------------------------------------------------------ PTX helpers
// (generic ones in tc_ptx.cuh)
// Bounded wait: false after the launch's wait limit (`lim`, read from the
// kernel's parameters: reading it from shared memory in every wait cost
// about a fifth of the two-column-tile kernel's time) or once another role
// has aborted.
template <class SM>
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, SM *sm,
                                          unsigned long long lim) {
    return mbar_wait_bounded(b, parity, &sm->abort_flag, lim);
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and B
// format (bits 7-9 / 10-12: 0 = F16, 1 = BF16), A MN-major (bit 15),
// B K-major (bit 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, uint32_t M, uint32_t N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | (1u << 15) | ((N >> 3) << 17) |
           ((M >> 4) << 24);
}


// One product of a launch (a single spmm_run is a batch of one).
struct TcProb {
    const int32_t *items, *grp_row0, *grp_rows, *ent_col, *ent_tbeg, *ent_cover;
    const uint8_t *packed;       // 16-bit tiles (512 B, MMA B layout) or E4M3 tiles (256 B)
    const float *tile_scale;     // E4M3: 16 scales per slot (4 x 4 sub-squares of 4 x 4)
    void *Y;
    float *ws;
    const int64_t *ws_row0;
    const uint32_t *srec, *sprog;  // stage records and MMA programs
    int64_t ldy, n;
    int64_t unit_base;           // first unit of this problem in launch order
    int32_t ntn, x3d;            // n tiles of 128; X map is 3-D (64, k, n/64)
};

// A stage whose entries are 2 to 4 consecutive tile columns (record info
// bit 20) gets its X slabs in one TMA box of 4 slabs when X's map is 3-D;
// the slabs then lie 2048 B apart inside each 64-column half, the halves
// 8192 B apart.

struct TcBatch {
    CUtensorMap maps[kMaxBatch]; // X of each problem
    CUtensorMap maps4[kMaxBatch];// the same X, boxes of kJointSlabs slabs
    TcProb prob[kMaxBatch];
    const int32_t *units;        // optional schedule: (problem, unit) pairs, costliest first
    int64_t total_units;
    int32_t nprob;
    const int32_t *n_items_dev;  // dynamic single problem: item count on the device
    int32_t *status;
    unsigned long long wait_ns;  // limit of each pipeline wait, never 0 (the abort drain waits kWaitNs)
    int32_t stall;               // failure-detection tests: after their first stage the MMA
                                 // warps wait on a barrier nothing arrives on, so that wait
                                 // runs out and the CTA takes its abort path
};

static_assert(sizeof(TcBatch) <= 32764, "kernel parameter space");

__device__ __forceinline__ void record(int32_t *status, int32_t code) {
    atomicCAS(status, 0, code);
}

// A-operand descriptor: X slab, MN-major, 128-byte swizzle; the two 64-column
// halves of the slab are 2048 B apart (leading offset), the two 8-row k
// groups 1024 B apart (stride offset).
__device__ __forceinline__ uint64_t a_desc(uint32_t addr) { return smem_desc(addr, 2048, 1024, 2); }
// The same for a stage loaded as one box of kJointSlabs slabs.
__device__ __forceinline__ uint64_t a_desc_joint(uint32_t addr) {
    return smem_desc(addr, kJointSlabs * 2048, 1024, 2);
}
// B-operand descriptor: one W tile, K-major, no swizzle; 8 x 8 core matrices,
// k-adjacent ones 128 B apart (leading), row-adjacent ones 256 B (stride).
__device__ __forceinline__ uint64_t b_desc(uint32_t addr) { return smem_desc(addr, 128, 256, 0); }

// Unit u of the launch -> (problem, item, n tile).
struct Unit {
    int p;
    int64_t item;
    int t;
};
__device__ __forceinline__ Unit decode_unit(const TcBatch &B, int64_t u) {
    Unit r;
    int64_t lu;
    if (B.units) {
        r.p = B.units[2 * u];
        lu = B.units[2 * u + 1];
    } else {
        int p = 0;
        while (p + 1 < B.nprob && B.prob[p + 1].unit_base <= u) ++p;
        r.p = p;
        lu = u - B.prob[p].unit_base;
    }
    const int ntn = B.prob[r.p].ntn;
    r.item = lu / ntn;
    r.t = (int)(lu - r.item * ntn);
    return r;
}

template <typename T, bool W8, int GEO>
__global__ void __launch_bounds__(GEO == 3 ? 416 : GEO == 2 ? 352 : kThreads, GEO >= 2 ? 1 : kCtasPerSm)
    tc_kernel(const __grid_constant__ TcBatch B) {
    pdl_enter();
    using G = StageGeom<W8, GEO>;
    // wide CTAs hold one accumulator set per column tile (all 512 columns)
    constexpr int kBufs = G::sets > 1 ? 1 : kAccBufs;
    constexpr int kTmemCols = kBufs * G::sets * kAccCols;
    static_assert(G::sets == 1 || kAccCols * G::sets <= 512, "TMEM columns");
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *stages = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int kStages = G::stages;
    using Smem = SmemT<kStages>;
    Smem *sm = (Smem *)(stages + kStages * G::bytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        int64_t nu = B.total_units;
        if (B.n_items_dev) {
            // dynamic plans: item count from the device; a rejected pattern
            // leaves Y unwritten
            const int64_t cap = B.total_units / B.prob[0].ntn;
            const int64_t ni = min(cap, (int64_t)max(*B.n_items_dev, 0));
            nu = (*(volatile int32_t *)B.status != 0) ? 0 : ni * B.prob[0].ntn;
        }
        sm->nunits = nu;
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&sm->full[s], G::producers);
            mbar_init(&sm->empty[s], G::mma_warps);   // every MMA warp
            mbar_init(&sm->conv[s], 4);    // E4M3: one arrival per converter warp
        }
        for (int b = 0; b < kBufs; ++b) {
            mbar_init(&sm->accf[b], G::mma_warps);    // MMA completion, every MMA warp
            mbar_init(&sm->acce[b], 128);  // every epilogue thread
        }
        mbar_init(&sm->drain, G::mma_warps);
        mbar_init(&sm->never, 1);
        sm->abort_flag = 0;
        for (int i = 0; i < kProducersMax; ++i) sm->issued[i] = 0;
        for (int i = 0; i < kMmaWarpsMax; ++i) sm->consumed[i] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int64_t nunits = sm->nunits;
    if (nunits == 0) return;
    if (warp == 1) {
        tmem_alloc(&sm->tmem_base, kTmemCols);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm->tmem_base;
    if (warp >= 2 && warp < 6) {
        // accumulators start at zero: each epilogue warp clears its lane quarter
        const uint32_t lq = (uint32_t)((warp & 3) * 32) << 16;
        for (int c = 0; c < kTmemCols; c += 16) tmem_zero16(tmem + lq + c);
        tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    if (warp == 0 || warp == kXWarp0 || warp == kXWarp1 || warp >= kXWarp2) {
        // ------------------------------------------------ TMA producers
        // Warp 0 copies each stage's W tiles and its MMA program; warp 6
        // requests its X slabs.  Both follow the stage records of the unit
        // (built ahead of the launch) with three records in flight, so
        // neither waits on a global load or decodes anything per stage.
        const bool wprod = warp == 0;
        const int pid = wprod ? 0 : warp == kXWarp0 ? 1 : warp == kXWarp1 ? 2 : warp - kXWarp2 + 3;

        int stage = 0;
        uint32_t phase = 0;
        int32_t issued = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x; ok && u < nunits; u += gridDim.x) {
            const Unit un = decode_unit(B, u);
            const TcProb &P = B.prob[un.p];
            const int32_t *it = P.items + un.item * kItemFields;
            const int32_t e0 = it[1], e1 = it[2];
            if (e0 >= e1) continue;
            const int n0 = un.t * kNTile * G::sets;
            // wide: the second column tile, unless it lies wholly past n
            const bool two = G::sets > 1 && n0 + kNTile < P.n;
            // lane l: word (l & 7) of the record, and (W producer) program word l
            auto ld_rec = [&](int32_t r) -> uint32_t {
                return r < e1 ? __ldg(P.srec + (int64_t)r * kRecWords + (lane & (kRecWords - 1))) : 0u;
            };
            auto ld_prog = [&](int32_t r) -> uint2 {
                return (wprod && r < e1)
                           ? __ldg((const uint2 *)(P.sprog + (int64_t)r * 2 * kMmaStage) + lane)
                           : make_uint2(0u, 0u);
            };
            // one stage from its record word (lane l: word l & 7) and program
            // word; 1 after the unit's last stage, -1 on a failed wait
            auto stage_step = [&](uint32_t rc, uint2 pc) -> int {
                const uint32_t info = __shfl_sync(0xffffffffu, rc, 0);
                const uint32_t nslots = __shfl_sync(0xffffffffu, rc, 1);
                const uint32_t stb = __shfl_sync(0xffffffffu, rc, 2);
                const int nent = (int)((info >> 12) & 0xfu);
                // X producer 1 requests slabs [0, h), producer 2 slabs [h, nent)
                const int h = (nent + 1) >> 1;
                const int xlo = pid == 2 ? h : 0, mine = pid == 2 ? nent - h : h;
                const uint32_t col = __shfl_sync(0xffffffffu, rc, min(3 + xlo + lane, kRecWords - 1));
                int w = 1;
                if (lane == 0) w = mbar_wait(&sm->empty[stage], phase ^ 1, sm, B.wait_ns) ? 1 : 0;
                if (!__shfl_sync(0xffffffffu, w, 0)) return -1;
                uint8_t *st = stages + stage * G::bytes;
                if (wprod) {
                    sm->meta[stage].prog[0][lane] = pc.x;
                    sm->meta[stage].prog[1][lane] = pc.y;
                    if (lane == 0) {
                        sm->meta[stage].info = info;
                        sm->meta[stage].nslots = nslots;
                    }
                    __syncwarp();
                    if (lane == 0 && nslots) {
                        if (W8) {
                            mbar_arrive_tx(&sm->full[stage], nslots * (kTileBytes8 + kScaleBytes));
                            bulk_load(st + G::w8, P.packed + (int64_t)stb * kTileBytes8,
                                      nslots * kTileBytes8, &sm->full[stage]);
                            bulk_load(st + G::sc, P.tile_scale + (int64_t)stb * 16,
                                      nslots * kScaleBytes, &sm->full[stage]);
                        } else {
                            mbar_arrive_tx(&sm->full[stage], nslots * kTileBytes16);
                            bulk_load(st + G::w16, P.packed + (int64_t)stb * kTileBytes16,
                                      nslots * kTileBytes16, &sm->full[stage]);
                        }
                    } else if (lane == 0) {
                        mbar_arrive(&sm->full[stage]);
                    }
                } else if (G::sets > 1) {
                    // wide: producers 1 and 3 bring the stage's slabs of the
                    // first column tile, 2 and 4 those of the second
                    // (G::xprod warps per tile, each a share of the slabs):
                    // with a 3-D X map as one box of consecutive slabs (the
                    // first warp of the tile) or one box per slab, with a 2-D
                    // map as two 64-column boxes per slab (the lower one only
                    // when the upper 64 columns lie past n)
                    const bool joint = (info & kJointBit) && P.x3d;
                    const int tset = (pid - 1) & 1, part = (pid - 1) >> 1;
                    const bool act = tset == 0 || two;
                    const int per = (nent + G::xprod - 1) / G::xprod;
                    const int lo = part * per;
                    const int cnt = joint ? (part == 0 ? kJointSlabs : 0) : max(0, min(nent, lo + per) - lo);
                    const uint32_t xc =
                        __shfl_sync(0xffffffffu, rc, min(3 + (joint ? 0 : lo) + lane, kRecWords - 1));
                    const int64_t ncol = n0 + (int64_t)tset * kNTile;     // this tile's first column
                    const bool half = !P.x3d && ncol + kNTile / 2 >= P.n;
                    // (a joint box always lands all kJointSlabs slabs)
                    if (lane == 0)
                        mbar_arrive_tx(&sm->full[stage],
                                       act ? cnt * (half ? kSlabBytes / 2 : kSlabBytes) : 0);
                    __syncwarp();
                    uint8_t *xs = st + tset * G::xset;
                    const int nh = n0 / (kNTile / 2) + tset * 2;
                    if (P.x3d) {
                        if (act && joint && cnt && lane == 0)
                            tma_load_3d(xs, &B.maps4[un.p], 0, (int)xc * kTile, nh, &sm->full[stage]);
                        if (act && !joint && lane < cnt)
                            tma_load_3d(xs + (lo + lane) * kSlabBytes, &B.maps[un.p], 0,
                                        (int)xc * kTile, nh, &sm->full[stage]);
                    } else if (act && lane < cnt) {
                        uint8_t *slab = xs + (lo + lane) * kSlabBytes;
                        tma_load_2d(slab, &B.maps[un.p], (int)ncol, (int)xc * kTile, &sm->full[stage]);
                        if (!half)
                            tma_load_2d(slab + kSlabBytes / 2, &B.maps[un.p], (int)ncol + kNTile / 2,
                                        (int)xc * kTile, &sm->full[stage]);
                    }
                } else if ((info & kJointBit) && P.x3d) {
                    // consecutive columns: X producer 1 requests all slabs in one box
                    if (lane == 0) {
                        if (pid == 1) {
                            mbar_arrive_tx(&sm->full[stage], kJointSlabs * kSlabBytes);
                            tma_load_3d(st, &B.maps4[un.p], 0, (int)col * kTile, n0 / (kNTile / 2),
                                        &sm->full[stage]);
                        } else {
                            mbar_arrive(&sm->full[stage]);
                        }
                    }
                } else {
                    // a column tile whose upper 64 columns lie past n (small n)
                    // fetches its lower halves only: the upper half of the
                    // accumulator then holds rows of Y that are never stored
                    const bool half = !P.x3d && n0 + kNTile / 2 >= P.n;
                    if (lane == 0)
                        mbar_arrive_tx(&sm->full[stage],
                                       mine * (half ? kSlabBytes / 2 : kSlabBytes));
                    __syncwarp();
                    if (lane < mine) {
                        const CUtensorMap *xmap = &B.maps[un.p];
                        uint8_t *slab = st + (xlo + lane) * kSlabBytes;
                        if (P.x3d) {
                            tma_load_3d(slab, xmap, 0, (int)col * kTile, n0 / (kNTile / 2),
                                        &sm->full[stage]);
                        } else {
                            tma_load_2d(slab, xmap, n0, (int)col * kTile, &sm->full[stage]);
                            if (!half)
                                tma_load_2d(slab + kSlabBytes / 2, xmap, n0 + kNTile / 2,
                                            (int)col * kTile, &sm->full[stage]);
                        }
                    }
                }
                __syncwarp();
                ++issued;
                if (++stage == kStages) {
                    stage = 0;
                    phase ^= 1;
                }
                return (info >> 31) ? 1 : 0;
            };
            // three records in flight, in three registers that are only ever
            // reloaded (never moved: a move would wait for the load)
            uint32_t ra = ld_rec(e0), rb = ld_rec(e0 + 1), rd = ld_rec(e0 + 2);
            uint2 pa = ld_prog(e0), pb = ld_prog(e0 + 1), pd = ld_prog(e0 + 2);
            bool done = false;   // a unit's stages never outnumber its entries
            for (int32_t r = e0; ok && !done && r < e1; r += 3) {
                int v = stage_step(ra, pa);
                ra = ld_rec(r + 3);
                pa = ld_prog(r + 3);
                if (v == 0 && r + 1 < e1) {
                    v = stage_step(rb, pb);
                    rb = ld_rec(r + 4);
                    pb = ld_prog(r + 4);
                    if (v == 0 && r + 2 < e1) {
                        v = stage_step(rd, pd);
                        rd = ld_rec(r + 5);
                        pd = ld_prog(r + 5);
                    }
                }
                if (v < 0) ok = false;
                if (v > 0) done = true;
            }
            if (ok && !done) {
                record(B.status, kDevBadPlan);
                ok = false;
            }
        }
        if (!ok && lane == 0) {
            record(B.status, kDevTimeout);   // no effect if a bad plan was recorded first
            sm->abort_flag = 1;
        }
        if (lane == 0) sm->issued[pid] = issued;
    } else if (warp == 1 || (warp >= kMmaWarpHi && warp <= kMmaWarpHi + 2)) {
        // ------------------------------- MMA issuers (converged warps)
        // warps 1 / 8: tile rows 0-7 / 8-15 of the first column tile; wide
        // CTAs: warps 9 / 10 the same rows of the second column tile
        const int mw = warp == 1 ? 0 : warp - kMmaWarpHi + 1;   // 0..3
        const int half = mw & 1;              // tile rows 0-7 / 8-15
        const int tset = mw >> 1;             // column tile
        constexpr uint32_t idesc0 = make_idesc(Cvt<T>::fmt, kNTile, 0);
        int stage = 0;
        uint32_t phase = 0;
        int32_t consumed = 0;
        bool ok = true;
        int local = 0;
        for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x, ++local) {
            const Unit un = decode_unit(B, u);
            const int32_t *it = B.prob[un.p].items + un.item * kItemFields;
            const bool has_entries = it[2] > it[1];
            const bool two = G::sets > 1 && (int64_t)un.t * kNTile * G::sets + kNTile < B.prob[un.p].n;
            const int ab = local % kBufs;
            const uint32_t aphase = (local / kBufs) & 1;
            int w = 1;
            if (lane == 0) w = mbar_wait(&sm->acce[ab], aphase ^ 1, sm, B.wait_ns) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, w, 0) != 0;
            tc_fence_after();
            const uint32_t dbase = tmem + ab * G::sets * kAccCols;
            bool last = !has_entries;
            while (ok && !last) {
                if (lane == 0)
                    w = mbar_wait(W8 ? &sm->conv[stage] : &sm->full[stage], phase, sm, B.wait_ns) ? 1 : 0;
                if (!__shfl_sync(0xffffffffu, w, 0)) {
                    ok = false;
                    break;
                }
                __syncwarp();   // orders lane 0's acquire before every lane's reads
                tc_fence_after();
                ++consumed;
                // every lane reads the stage header and one program word
                const uint32_t info = sm->meta[stage].info;
                // (a second column tile wholly past n gets no MMAs)
                const int nmma = (tset && !two) ? 0 : (int)((info >> (6 * half)) & 63u);
                last = (info >> 31) != 0;
                const uint32_t myword = sm->meta[stage].prog[half][lane];   // words >= nmma unused
                const uint32_t sbase = smem_u32(stages + stage * G::bytes);
                const bool joint = (info & kJointBit) && B.prob[un.p].x3d;
                const uint64_t adesc0 = joint ? a_desc_joint(sbase) : a_desc(sbase);
                const uint32_t astep = joint ? (kSlabBytes / 2) >> 4 : kSlabBytes >> 4;
                const uint64_t bdesc0 = b_desc(sbase + G::w16);
                for (int i = 0; i < nmma; ++i) {
                    const uint32_t wd = __shfl_sync(0xffffffffu, myword, i);
                    const uint32_t slab = wd & 15u, toff = (wd >> 4) & 255u;
                    const uint32_t r0 = (wd >> 12) & 15u, len = (wd >> 16) & 31u;
                    // descriptor start addresses are in 16-byte units (bits 0-13)
                    // wide, second column tile: the same W tiles against that
                    // tile's slabs, into the second accumulator set
                    tc_mma_elect(dbase + tset * kAccCols + r0 * kTile,
                                 adesc0 + tset * (G::xset >> 4) + slab * astep,
                                 bdesc0 + toff * (kTileBytes16 >> 4),
                                 idesc0 | ((len * kTile) >> 3) << 17, 1u);
                }
                if (lane == 0) tc_commit(&sm->empty[stage]);
                __syncwarp();
                if (++stage == kStages) {
                    stage = 0;
                    phase ^= 1;
                }
                if (B.stall) {
                    // failure-detection tests: a wait that nothing ends
                    if (lane == 0) w = mbar_wait(&sm->never, 0, sm, B.wait_ns) ? 1 : 0;
                    if (!__shfl_sync(0xffffffffu, w, 0)) {
                        ok = false;
                        break;
                    }
                }
            }
            if (!ok) break;
            if (lane == 0) tc_commit(&sm->accf[ab]);
            __syncwarp();
        }
        if (lane == 0) {
            if (!ok) {
                record(B.status, kDevTimeout);
                sm->abort_flag = 1;
            }
            sm->consumed[mw] = consumed;
        }
    } else {
        // ------------------------- converters (E4M3) and epilogue
        const int q = warp & 3;              // TMEM lane quarter of this warp
        const int nl = q * 32 + lane;        // D row = column of Y within the tile
        const int et = threadIdx.x - 64;     // 0..127 among the four warps
        int local = 0;
        int cstage = 0;
        uint32_t cphase = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x; ok && u < nunits; u += gridDim.x, ++local) {
            const Unit un = decode_unit(B, u);
            const TcProb &P = B.prob[un.p];
            const int32_t *it = P.items + un.item * kItemFields;
            if (W8 && it[2] > it[1]) {
                // expand this unit's E4M3 tiles to 16-bit MMA tiles, stage by stage
                bool last = false;
                while (!last) {
                    int w = 1;
                    if (lane == 0) w = mbar_wait(&sm->full[cstage], cphase, sm, B.wait_ns) ? 1 : 0;
                    if (!__shfl_sync(0xffffffffu, w, 0)) {
                        // every epilogue warp still meets the named barrier
                        // below, where the poller sees the abort
                        if (lane == 0) {
                            record(B.status, kDevTimeout);
                            sm->abort_flag = 1;
                        }
                        break;
                    }
                    const uint32_t mnent = sm->meta[cstage].info;
                    last = (mnent >> 31) != 0;
                    const int nslots = (int)sm->meta[cstage].nslots;
                    uint8_t *st = stages + cstage * G::bytes;
                    const uint8_t *w8 = st + G::w8;
                    const float *sc = (const float *)(st + G::sc);
                    // thread -> (slot, tile row i): 16 codes of one row per step
                    for (int r = et; r < nslots * kTile; r += 128) {
                        const int slot = r >> 4, i = r & 15;
                        const uint4 codes = *(const uint4 *)(w8 + slot * kTileBytes8 + i * kTile);
                        const float *s4 = sc + slot * 16 + (i >> 2) * 4;
                        const uint32_t cw[4] = {codes.x, codes.y, codes.z, codes.w};
                        uint32_t outw[8];
#pragma unroll
                        for (int qd = 0; qd < 4; ++qd) {          // columns 4qd .. 4qd+3
                            const float scl = s4[qd];
                            const __half2_raw h01 = __nv_cvt_fp8x2_to_halfraw2(
                                (__nv_fp8x2_storage_t)(cw[qd] & 0xFFFFu), __NV_E4M3);
                            const __half2_raw h23 = __nv_cvt_fp8x2_to_halfraw2(
                                (__nv_fp8x2_storage_t)(cw[qd] >> 16), __NV_E4M3);
                            const float2 f01 = __half22float2(*(const __half2 *)&h01);
                            const float2 f23 = __half22float2(*(const __half2 *)&h23);
                            // code x scale in FP32, rounded once; a pair per multiply
                            // and per conversion
                            const float2 p01 = mul2_rn(f01, scl), p23 = mul2_rn(f23, scl);
                            outw[qd * 2] = pack2_rn<T>(p01.x, p01.y);
                            outw[qd * 2 + 1] = pack2_rn<T>(p23.x, p23.y);
                        }
                        // columns 0-7 and 8-15 land in two core matrices
                        uint8_t *dst = st + G::w16 + slot * kTileBytes16 + (i >> 3) * 256 + (i & 7) * 16;
                        *(uint4 *)dst = make_uint4(outw[0], outw[1], outw[2], outw[3]);
                        *(uint4 *)(dst + 128) = make_uint4(outw[4], outw[5], outw[6], outw[7]);
                    }
                    // make the generic-proxy writes visible to the tensor core
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sm->conv[cstage]);
                    if (++cstage == kStages) {
                        cstage = 0;
                        cphase ^= 1;
                    }
                }
            }
            const int ab = local % kBufs;
            const uint32_t aphase = (local / kBufs) & 1;
            // one thread polls the accumulator barrier, sleeping between polls
            // (the mbarrier unit is shared with the copy and MMA pipelines of
            // both CTAs of the SM); the other epilogue threads block on a
            // named barrier, which costs the mbarrier unit nothing
            if (warp == 2 && lane == 0) {
                const unsigned long long t0 = gtimer();
                int okp = 1;
                while (!mbar_try(&sm->accf[ab], aphase)) {
                    __nanosleep(400);
                    if (sm->abort_flag || gtimer() - t0 > B.wait_ns) {
                        okp = 0;
                        break;
                    }
                }
                sm->epi_ok[local & 1] = okp;
            }
            asm volatile("bar.sync 1, 128;" ::: "memory");
            const int okw = sm->epi_ok[local & 1];
            if (!okw) {
                ok = false;
                break;
            }
            tc_fence_after();
            const int32_t g = it[0], slot = it[5];
            const int rows = P.grp_rows[g];
            const int64_t yrow0 = (int64_t)P.grp_row0[g] * kTile;
            const int64_t wrow0 = slot >= 0 ? P.ws_row0[slot] : 0;
            T *Y = (T *)P.Y;
            // one pass per column tile of the unit (wide CTAs: two, the second
            // skipped when it lies wholly past n: its MMAs were never issued)
            for (int h = 0; h < G::sets; ++h) {
                const int64_t cbase = ((int64_t)un.t * G::sets + h) * kNTile;
                if (h > 0 && cbase >= P.n) break;
                const int64_t col = cbase + nl;
                const bool in = col < P.n;
                const uint32_t acc = (uint32_t)((ab * G::sets + h) * kAccCols);
                // four tile rows (64 accumulator columns) per TMEM load and wait
                int r = 0;
                for (; r + 4 <= rows; r += 4) {
                    float v[64];
                    const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + acc + r * kTile;
                    tmem_ld64(ta, v);
                    tmem_zero64(ta);
                    if (!in) continue;
                    if (slot >= 0) {
                        float *dst = P.ws + (wrow0 + r * kTile) * P.n + col;
#pragma unroll
                        for (int i = 0; i < 64; ++i) dst[i * P.n] = v[i];
                    } else {
                        T *dst = Y + (yrow0 + r * kTile) * P.ldy + col;
#pragma unroll
                        for (int i = 0; i < 64; ++i) dst[i * P.ldy] = Cvt<T>::f(v[i]);
                    }
                }
                for (; r < rows; ++r) {
                    float v[16];
                    const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + acc + r * kTile;
                    tmem_ld16(ta, v);
                    tmem_zero16(ta);
                    if (!in) continue;
                    // (staging through shared memory for 16-byte row stores measured slower)
                    if (slot >= 0) {
                        float *dst = P.ws + (wrow0 + r * kTile) * P.n + col;
#pragma unroll
                        for (int i = 0; i < 16; ++i) dst[i * P.n] = v[i];
                    } else {
                        T *dst = Y + (yrow0 + r * kTile) * P.ldy + col;
#pragma unroll
                        for (int i = 0; i < 16; ++i) dst[i * P.ldy] = Cvt<T>::f(v[i]);
                    }
                }
            }
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(&sm->acce[ab]);
        }
        if (!ok && lane == 0) {
            record(B.status, kDevTimeout);
            sm->abort_flag = 1;
        }
    }

    __syncthreads();
    // after an abort, let copies and MMAs still in flight land before TMEM
    // and shared memory are released (every wait here is bounded by kWaitNs)
    if (sm->abort_flag) {
        if (threadIdx.x == 0) {
            int32_t hi = 0;
            for (int i = 0; i < G::producers; ++i) hi = max(hi, sm->issued[i]);
            int32_t lo = sm->consumed[0];
            for (int i = 1; i < G::mma_warps; ++i) lo = min(lo, sm->consumed[i]);
            for (int32_t c = lo; c < hi; ++c) {
                const int s = c % kStages;
                const uint32_t par = (uint32_t)((c / kStages) & 1);   // kStages = G::stages
                // stand in for the arrivals of producers that stopped before stage c
                for (int i = 0; i < G::producers; ++i)
                    if (c >= sm->issued[i]) mbar_arrive(&sm->full[s]);
                const unsigned long long t0 = gtimer();
                while (!mbar_try(&sm->full[s], par) && gtimer() - t0 < kWaitNs) {
                }
            }
        }
        // each MMA warp's issuing lane commits once more: the drain barrier
        // completes when every MMA any of them issued has completed
        const bool mma_warp = warp == 1 || (warp >= kMmaWarpHi && warp < kMmaWarpHi + G::mma_warps - 1);
        if (mma_warp && lane == 0) tc_commit(&sm->drain);
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned long long t0 = gtimer();
            while (!mbar_try(&sm->drain, 0) && gtimer() - t0 < kWaitNs) {
            }
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// ------------------------------------------------------- stage records ---
// (the cutting of stages, build_item_stages, is in tc_stage.cuh: the fused
// dynamic re-partition runs it too)
__global__ void __launch_bounds__(kBuildWarps * 32)
    stage_build_kernel(const int32_t *__restrict__ items, int64_t n_items,
                       const int32_t *__restrict__ n_items_dev, const int32_t *__restrict__ status,
                       const int32_t *__restrict__ ent_col, const int32_t *__restrict__ ent_tbeg,
                       const int32_t *__restrict__ ent_cover, int ent_cap, int tiles_cap,
                       uint32_t *__restrict__ srec, uint32_t *__restrict__ sprog) {
    pdl_enter();
    __shared__ int32_t counts[kBuildWarps];
    int64_t ni = n_items;
    if (n_items_dev) {
        if (*status != 0) return;
        ni = min(ni, (int64_t)max(*n_items_dev, 0));
    }
    const int64_t item = blockIdx.x;
    if (item >= ni) return;
    build_item_stages(items + item * kItemFields, ent_cap, tiles_cap, ent_col, ent_tbeg, ent_cover,
                      srec, sprog, counts);
}

// ------------------------------------------------------------- packing ---
// (the per-element packing, pack_tiles_range / pack_tiles_e4m3_range, is in
// tc_stage.cuh)
template <typename U, int B, int SEG>
__global__ void pack_tiles_kernel(const U *__restrict__ vals, const int32_t *__restrict__ blk_slot,
                                  const int32_t *__restrict__ blk_off, int64_t nnzb, int tr,
                                  const int32_t *__restrict__ nnzb_dev,
                                  const int32_t *__restrict__ status, U *__restrict__ out) {
    pdl_enter();
    // dynamic plans: a rejected pattern leaves blk_slot / blk_off incomplete
    if (status && *status != 0) return;
    if (nnzb_dev) nnzb = min((int64_t)max(*nnzb_dev, 0), nnzb);
    pack_tiles_range<U, B, SEG>(vals, blk_slot, blk_off, nnzb, tr, out,
                                blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                                (int64_t)gridDim.x * blockDim.x);
}

__global__ void pack_tiles_e4m3_kernel(const uint8_t *__restrict__ codes,
                                       const float *__restrict__ scales,
                                       const int32_t *__restrict__ blk_slot,
                                       const int32_t *__restrict__ blk_off, int64_t nnzb, int b,
                                       int tr, const int32_t *__restrict__ nnzb_dev,
                                       const int32_t *__restrict__ status, uint8_t *__restrict__ out,
                                       float *__restrict__ tile_scale) {
    pdl_enter();
    if (status && *status != 0) return;   // rejected dynamic pattern
    if (nnzb_dev) nnzb = min((int64_t)max(*nnzb_dev, 0), nnzb);
    pack_tiles_e4m3_range(codes, scales, blk_slot, blk_off, nnzb, b, tr, out, tile_scale,
                          blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                          (int64_t)gridDim.x * blockDim.x);
}

// Per block: scale = max|w| / 448 (1 for an all-zero block), code = the E4M3
// value nearest w / scale (round to nearest even, saturating).
template <typename U>
__global__ void quantize_e4m3_kernel(const U *__restrict__ src, int64_t nnzb, int b,
                                     uint8_t *__restrict__ codes, float *__restrict__ scales) {
    pdl_enter();
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= nnzb) return;
    const int bb = b * b;
    const U *v = src + wid * bb;
    float amax = 0.f;
    for (int e = lane; e < bb; e += 32) amax = fmaxf(amax, fabsf((float)v[e]));
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    const float scale = amax > 0.f ? amax / 448.f : 1.f;
    if (lane == 0) scales[wid] = scale;
    for (int e = lane; e < bb; e += 32)
        codes[wid * bb + e] =
            (uint8_t)__nv_cvt_float_to_fp8((float)v[e] / scale, __NV_SATFINITE, __NV_E4M3);
}

// Wide launches (two column tiles per CTA, one CTA per SM, each W tile read
// once per 256 columns of n): static 16-bit plans over a 3-D X map (n a
// multiple of 64) with n > 128.  Automatically for dense-tile plans with
// enough work units that halving them still fills the SMs (a wide CTA does
// the work of two narrow ones, which share an SM otherwise).  Measured at
// m = k = 4096, n = 2048, every dense-tile point of the sweep ran 5-11 %
// faster wide; every sparse-tile point 6-11 % slower (two 86 KB stages per
// CTA, against two narrow CTAs whose stages interleave).
bool use_wide(const spmm_plan *p, int64_t n, int x3d) {
    if (p->col_tiles == 1 || p->mode != SPMM_STATIC || n <= kNTile) return false;
    // forced: any n > 128 (2-D X maps included) and E4M3 weights as well
    if (p->col_tiles == 2) return true;
    if (!x3d || p->wdt == SPMM_E4M3) return false;
    const int64_t units = p->n_items * ((n + kNTile - 1) / kNTile);
    return p->tc_geo == 0 && 2 * units >= (int64_t)SPMM_TC_WIDE_MIN * p->sm_count;
}

void fill_prob(TcProb &P, const spmm_plan *p, void *Y, int64_t n, int64_t ldy, int x3d,
               bool alt = false) {
    P.items = p->d_items;
    P.grp_row0 = p->d_grp_row0;
    P.grp_rows = p->d_grp_rows;
    P.ent_col = p->d_ent_col;
    P.ent_tbeg = p->d_ent_tbeg;
    P.ent_cover = p->d_ent_cover;
    P.packed = (const uint8_t *)p->d_packed;
    P.tile_scale = p->d_tile_scale;
    P.Y = Y;
    P.ws = p->d_ws;
    P.ws_row0 = p->d_ws_row0;
    P.srec = alt ? p->d_srec_alt : p->d_srec;
    P.sprog = alt ? p->d_sprog_alt : p->d_sprog;
    P.ldy = ldy;
    P.n = n;
    P.ntn = (int)((n + kNTile - 1) / kNTile);
    P.x3d = x3d;
}

// Shared memory of one CTA of a geometry; one-column-tile geometries must
// leave room for two CTAs per SM (228 KB, 1 KB of it reserved per CTA).
template <bool W8, int GEO> constexpr size_t tc_smem_bytes() {
    using G = StageGeom<W8, GEO>;
    return 1024 + (size_t)G::stages * G::bytes + sizeof(SmemT<G::stages>);
}
static_assert(kCtasPerSm * (tc_smem_bytes<false, 0>() + 1024) <= 228 * 1024 &&
                  kCtasPerSm * (tc_smem_bytes<false, 1>() + 1024) <= 228 * 1024 &&
                  kCtasPerSm * (tc_smem_bytes<true, 0>() + 1024) <= 228 * 1024 &&
                  kCtasPerSm * (tc_smem_bytes<true, 1>() + 1024) <= 228 * 1024,
              "two CTAs per SM");

template <typename T, bool W8, int GEO>
cudaError_t launch_batch(const TcBatch &B, int sm_count, cudaStream_t s) {
    if (B.total_units == 0) return cudaSuccess;
    const int64_t slots = (int64_t)sm_count * (GEO >= 2 ? 1 : kCtasPerSm);
    const int grid = (int)(B.total_units < slots ? B.total_units : slots);
    using G = StageGeom<W8, GEO>;
    const size_t smem = tc_smem_bytes<W8, GEO>();
    static std::atomic<uint64_t> attrs{0};
    const cudaError_t e = set_smem_attrs_once(attrs, tc_kernel<T, W8, GEO>, (int)smem, GEO >= 2);
    if (e != cudaSuccess) return e;
    pdl_launch(tc_kernel<T, W8, GEO>, dim3(grid), dim3(G::threads), smem, s, B);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_geo(const TcBatch &B, int geo, bool w8, int sm_count, cudaStream_t s) {
    if (w8) {
        if (geo == 3) return launch_batch<T, true, 3>(B, sm_count, s);
        if (geo == 2) return launch_batch<T, true, 2>(B, sm_count, s);
        return geo ? launch_batch<T, true, 1>(B, sm_count, s) : launch_batch<T, true, 0>(B, sm_count, s);
    }
    if (geo == 3) return launch_batch<T, false, 3>(B, sm_count, s);
    if (geo == 2) return launch_batch<T, false, 2>(B, sm_count, s);
    return geo ? launch_batch<T, false, 1>(B, sm_count, s) : launch_batch<T, false, 0>(B, sm_count, s);
}
cudaError_t dispatch_batch(const TcBatch &B, int geo, bool bf16, bool w8, int sm_count,
                           cudaStream_t s) {
    return bf16 ? launch_geo<__nv_bfloat16>(B, geo, w8, sm_count, s)
                : launch_geo<__half>(B, geo, w8, sm_count, s);
}

// Cached launch schedules of batches: (problem, unit) pairs of all problems,
// costliest first (item cost = tile slots + entries, as the planner defines
// it), then by problem and unit.  Keyed by the plans and each problem's n.
struct SchedKey {
    std::vector<const void *> plans;
    std::vector<int64_t> n;
    bool operator<(const SchedKey &o) const {
        return plans != o.plans ? plans < o.plans : n < o.n;
    }
};
std::mutex g_sched_mu;
std::map<SchedKey, int32_t *> g_sched;

}  // namespace

cudaError_t launch_tc(const spmm_plan *p, const void *X, int64_t n, int64_t ldx, void *Y,
                      int64_t ldy, cudaStream_t s) {
    if (p->R > kRowCap) return cudaErrorInvalidConfiguration;
    TcBatch B;  // the launch parameter (copied at launch)
    int x3d = 0;
    cudaError_t e = encode_x(&B.maps[0], &x3d, p->xdt == SPMM_BF16, X, p->k, n, ldx);
    if (e != cudaSuccess) return e;
    const bool wide = use_wide(p, n, x3d);
    e = encode_x(&B.maps4[0], &x3d, p->xdt == SPMM_BF16, X, p->k, n, ldx, kJointSlabs);
    if (e != cudaSuccess) return e;
    fill_prob(B.prob[0], p, Y, n, ldy, x3d);
    B.prob[0].unit_base = 0;
    B.nprob = 1;
    B.units = nullptr;
    B.status = p->d_status;
    B.wait_ns = p->wait_ns ? p->wait_ns : kWaitNs;
    B.stall = p->stall;
    const bool dyn = p->mode == SPMM_DYNAMIC;
    if (wide) B.prob[0].ntn = (B.prob[0].ntn + 1) / 2;   // units of two column tiles
    B.n_items_dev = dyn ? p->d_counts + kCntItems : nullptr;
    B.total_units = (dyn ? p->dyn.items_cap : p->n_items) * B.prob[0].ntn;
    if (dyn && !p->dyn_fused) {
        // this call's plan was built on the device: cut its stages now (the
        // fused re-partition has cut them already)
        e = launch_stage_build(p, s);
        if (e != cudaSuccess) return e;
    }
    return dispatch_batch(B, p->tc_geo + (wide ? 2 : 0), p->xdt == SPMM_BF16,
                          p->wdt == SPMM_E4M3, p->sm_count, s);
}

namespace {
cudaError_t launch_tc_group(int count, spmm_plan *const *plans, const void *const *X,
                            const int64_t *n, const int64_t *ldx, void *const *Y,
                            const int64_t *ldy, cudaStream_t s, bool schedule, int geo);
cudaError_t ensure_alt_records(spmm_plan *p, int geo, cudaStream_t s);
}

// Plans of both stage geometries in one launch, in the geometry that holds
// most of its work units; plans of the other geometry use stage records cut
// for it (built once per plan, on first use).  Only the stage shapes differ,
// never the arithmetic of a unit, so every result is the same as in its own
// geometry.  Plans that ask for two column tiles per CTA (col_tiles = 2,
// n > 128) run in a second launch of the two-column-tile kernel.
cudaError_t launch_tc_batch(int count, spmm_plan *const *plans, const void *const *X,
                            const int64_t *n, const int64_t *ldx, void *const *Y,
                            const int64_t *ldy, cudaStream_t s, bool schedule) {
    if (count <= 0 || count > kMaxBatch) return cudaErrorInvalidValue;
    for (int wide = 0; wide < 2; ++wide) {
        spmm_plan *gp[kMaxBatch];
        const void *gx[kMaxBatch];
        void *gy[kMaxBatch];
        int64_t gn[kMaxBatch], glx[kMaxBatch], gly[kMaxBatch];
        int c = 0;
        int64_t units[2] = {0, 0};
        for (int i = 0; i < count; ++i) {
            const bool w = plans[i]->col_tiles == 2 && n[i] > kNTile;
            if (w != (wide != 0)) continue;
            gp[c] = plans[i];
            gx[c] = X[i];
            gy[c] = Y[i];
            gn[c] = n[i];
            glx[c] = ldx ? ldx[i] : n[i];
            gly[c] = ldy ? ldy[i] : n[i];
            units[plans[i]->tc_geo & 1] += plans[i]->n_items * ((n[i] + kNTile - 1) / kNTile);
            ++c;
        }
        if (!c) continue;
        const int geo = units[1] > units[0] ? 1 : 0;
        for (int i = 0; i < c; ++i) {
            if (gp[i]->tc_geo == geo) continue;
            cudaError_t e = ensure_alt_records(gp[i], geo, s);
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = launch_tc_group(c, gp, gx, gn, glx, gy, gly, s, schedule, geo + 2 * wide);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

namespace {
// Stage records of plan p cut for stage geometry `geo` (not its own) into
// d_srec_alt / d_sprog_alt, allocated on first use (outside any stream
// capture: the first batched launch of a plan set allocates).
cudaError_t ensure_alt_records(spmm_plan *p, int geo, cudaStream_t s) {
    if (p->alt_geo == geo) return cudaSuccess;
    const int64_t E = std::max<int64_t>(p->n_entries, 1);
    if (!p->d_srec_alt) {
        void *a = nullptr, *b = nullptr;
        cudaError_t e = cudaMalloc(&a, (size_t)E * kRecWords * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc(&b, (size_t)E * 2 * kMmaStage * sizeof(uint32_t));
        if (e != cudaSuccess) {
            if (a) cudaFree(a);
            return e;
        }
        p->allocations.push_back(a);
        p->allocations.push_back(b);
        p->device_bytes += E * (kRecWords + 2 * kMmaStage) * (int64_t)sizeof(uint32_t);
        p->d_srec_alt = (uint32_t *)a;
        p->d_sprog_alt = (uint32_t *)b;
    }
    const bool w8 = p->wdt == SPMM_E4M3;
    const int tiles_cap = w8 ? (geo ? StageGeom<true, 1>::tiles : StageGeom<true, 0>::tiles)
                             : (geo ? StageGeom<false, 1>::tiles : StageGeom<false, 0>::tiles);
    const int ent_cap = w8 ? (geo ? StageGeom<true, 1>::ent : StageGeom<true, 0>::ent)
                           : (geo ? StageGeom<false, 1>::ent : StageGeom<false, 0>::ent);
    if (p->n_items > 0)
        pdl_launch(stage_build_kernel, dim3((unsigned)p->n_items), dim3(kBuildWarps * 32), 0, s,
            p->d_items, p->n_items, (const int32_t *)nullptr, p->d_status, p->d_ent_col,
            p->d_ent_tbeg, p->d_ent_cover, ent_cap, tiles_cap, p->d_srec_alt, p->d_sprog_alt);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) p->alt_geo = geo;
    return e;
}

cudaError_t launch_tc_group(int count, spmm_plan *const *plans, const void *const *X,
                            const int64_t *n, const int64_t *ldx, void *const *Y,
                            const int64_t *ldy, cudaStream_t s, bool schedule, int geo) {
    TcBatch B;
    std::lock_guard<std::mutex> lk(g_sched_mu);
    SchedKey key;
    int64_t base = 0;
    for (int i = 0; i < count; ++i) {
        const spmm_plan *p = plans[i];
        if (p->R > kRowCap) return cudaErrorInvalidConfiguration;
        int x3d = 0;
        const int64_t lx = ldx ? ldx[i] : n[i], ly = ldy ? ldy[i] : n[i];
        cudaError_t e = encode_x(&B.maps[i], &x3d, p->xdt == SPMM_BF16, X[i], p->k, n[i], lx);
        if (e == cudaSuccess)
            e = encode_x(&B.maps4[i], &x3d, p->xdt == SPMM_BF16, X[i], p->k, n[i], lx,
                         kJointSlabs);
        if (e != cudaSuccess) return e;
        fill_prob(B.prob[i], p, Y[i], n[i], ly, x3d, p->tc_geo != (geo & 1));
        if (geo >= 2) B.prob[i].ntn = (B.prob[i].ntn + 1) / 2;   // units of two column tiles
        B.prob[i].unit_base = base;
        base += p->n_items * B.prob[i].ntn;
        key.plans.push_back(p);
        key.n.push_back(n[i]);
    }
    key.n.push_back(geo);   // the same plans may run in either kind of launch
    B.nprob = count;
    B.total_units = base;
    B.status = plans[0]->d_status;
    B.n_items_dev = nullptr;
    B.units = nullptr;
    B.wait_ns = plans[0]->wait_ns ? plans[0]->wait_ns : kWaitNs;
    B.stall = plans[0]->stall;
    if (!schedule) {
        // problems in submission order (serving: every launch is a new mix)
        const bool bf16 = plans[0]->xdt == SPMM_BF16, w8 = plans[0]->wdt == SPMM_E4M3;
        return dispatch_batch(B, geo, bf16, w8, plans[0]->sm_count, s);
    }
    auto it = g_sched.find(key);
    if (it == g_sched.end()) {
        // the first launch of a plan set builds its schedule (this allocates:
        // make it outside any stream capture)
        struct U { int64_t cost; int32_t p, u; };
        std::vector<U> us;
        us.reserve(base);
        for (int i = 0; i < count; ++i) {
            const spmm_plan *p = plans[i];
            const int ntn = B.prob[i].ntn;
            for (int64_t item = 0; item < p->n_items; ++item) {
                const int32_t *f = &p->hp.items[item * kItemFields];
                const int64_t cost = (int64_t)(p->hp.ent_tbeg[f[2]] - p->hp.ent_tbeg[f[1]]) +
                                     (f[2] - f[1]);
                for (int t = 0; t < ntn; ++t) us.push_back({cost, i, (int32_t)(item * ntn + t)});
            }
        }
        std::stable_sort(us.begin(), us.end(), [](const U &a, const U &b) {
            if (a.cost != b.cost) return a.cost > b.cost;
            if (a.p != b.p) return a.p < b.p;
            return a.u < b.u;
        });
        std::vector<int32_t> flat(2 * us.size());
        for (size_t j = 0; j < us.size(); ++j) {
            flat[2 * j] = us[j].p;
            flat[2 * j + 1] = us[j].u;
        }
        int32_t *d = nullptr;
        if (!flat.empty()) {
            cudaError_t e = cudaMalloc(&d, flat.size() * sizeof(int32_t));
            if (e == cudaSuccess)
                e = cudaMemcpy(d, flat.data(), flat.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return e;
        }
        it = g_sched.emplace(key, d).first;
    }
    B.units = it->second;
    const bool bf16 = plans[0]->xdt == SPMM_BF16, w8 = plans[0]->wdt == SPMM_E4M3;
    return dispatch_batch(B, geo, bf16, w8, plans[0]->sm_count, s);
}
}  // namespace

void stage_caps(const spmm_plan *p, int *ent_cap, int *tiles_cap) {
    const bool w8 = p->wdt == SPMM_E4M3;
    // (wide launches use these records too: their caps are the base geometry's)
    *tiles_cap = w8 ? (p->tc_geo ? StageGeom<true, 1>::tiles : StageGeom<true, 0>::tiles)
                    : (p->tc_geo ? StageGeom<false, 1>::tiles : StageGeom<false, 0>::tiles);
    *ent_cap = w8 ? (p->tc_geo ? StageGeom<true, 1>::ent : StageGeom<true, 0>::ent)
                  : (p->tc_geo ? StageGeom<false, 1>::ent : StageGeom<false, 0>::ent);
}

cudaError_t launch_stage_build(const spmm_plan *p, cudaStream_t s) {
    const bool dyn = p->mode == SPMM_DYNAMIC;
    const int64_t ni = dyn ? p->dyn.items_cap : p->n_items;
    if (ni == 0 || !p->d_srec) return cudaSuccess;
    int ent_cap = 0, tiles_cap = 0;
    stage_caps(p, &ent_cap, &tiles_cap);
    pdl_launch(stage_build_kernel, dim3((unsigned)ni), dim3(kBuildWarps * 32), 0, s, p->d_items, ni,
        dyn ? p->d_counts + kCntItems : nullptr, p->d_status, p->d_ent_col, p->d_ent_tbeg,
        p->d_ent_cover, ent_cap, tiles_cap, p->d_srec, p->d_sprog);
    return cudaGetLastError();
}

int64_t stage_record_words() { return kRecWords; }
int tc_geometry(double tiles_per_entry) { return tiles_per_entry >= 8.0 ? 0 : 1; }
int64_t stage_prog_words() { return 2 * kMmaStage; }

cudaError_t launch_pack_tiles(const spmm_plan *p, const void *d_values, const float *d_scales,
                              const int32_t *d_nnzb, cudaStream_t s) {
    if (p->packed_bytes == 0) return cudaSuccess;
    // tiles hold several smaller blocks, static plans have zero tiles that
    // join intervals, and E4M3 tiles carry scales: clear them first; in a
    // dynamic plan (no joining tiles) a 16-bit 16 x 16 block fills its tile
    cudaError_t e = cudaSuccess;
    if (p->b < kTile || p->wdt == SPMM_E4M3 || p->mode == SPMM_STATIC)
        e = cudaMemsetAsync(p->d_packed, 0, p->packed_bytes, s);
    if (e != cudaSuccess) return e;
    const int64_t nmax = d_nnzb ? p->nnzb_max : p->nnzb;
    const int64_t total = nmax * p->b * p->b;
    if (total == 0) return cudaSuccess;
    int64_t g = (total + 255) / 256;
    if (g > 8192) g = 8192;
    if (p->wdt == SPMM_E4M3) {
        const int64_t slots = p->mode == SPMM_STATIC ? p->n_tiles : p->nnzb_max;
        e = cudaMemsetAsync(p->d_tile_scale, 0, sizeof(float) * 16 * slots, s);
        if (e != cudaSuccess) return e;
        pdl_launch(pack_tiles_e4m3_kernel, dim3((unsigned)g), dim3(256), 0, s,
            (const uint8_t *)d_values, d_scales, p->d_blk_slot, p->d_blk_off, nmax, p->b,
            p->transposed ? 1 : 0, d_nnzb, d_nnzb ? p->d_status : nullptr, (uint8_t *)p->d_packed,
            p->d_tile_scale);
        return cudaGetLastError();
    }
    if (p->wdt != SPMM_F16 && p->wdt != SPMM_BF16) return cudaErrorNotSupported;
    const uint16_t *v = (const uint16_t *)d_values;
    uint16_t *o = (uint16_t *)p->d_packed;
    // vector loads need the values aligned to a block row segment
    // vector copies need aligned values and untransposed blocks
    const bool al = ((uintptr_t)v % 16) == 0 && !p->transposed;
    const int tr = p->transposed ? 1 : 0;
    const unsigned gb = (unsigned)std::min<int64_t>(8192, (nmax * p->b * 2 + 255) / 256);
    const unsigned g1 = (unsigned)std::min<int64_t>(8192, (total + 255) / 256);
    const int32_t *bs = p->d_blk_slot, *bo = p->d_blk_off;
    const int32_t *st = d_nnzb ? p->d_status : nullptr;
    switch (p->b) {
        case 16:
            if (al) pdl_launch(pack_tiles_kernel<uint16_t, 16, 8>, dim3(gb), dim3(256), 0, s, v, bs,
                bo, nmax, tr, d_nnzb, st, o);
            else pdl_launch(pack_tiles_kernel<uint16_t, 16, 1>, dim3(g1), dim3(256), 0, s, v, bs,
                bo, nmax, tr, d_nnzb, st, o);
            break;
        case 8:
            if (al) pdl_launch(pack_tiles_kernel<uint16_t, 8, 8>, dim3(gb), dim3(256), 0, s, v, bs,
                bo, nmax, tr, d_nnzb, st, o);
            else pdl_launch(pack_tiles_kernel<uint16_t, 8, 1>, dim3(g1), dim3(256), 0, s, v, bs, bo,
                nmax, tr, d_nnzb, st, o);
            break;
        case 4:
            if (al) pdl_launch(pack_tiles_kernel<uint16_t, 4, 4>, dim3(gb), dim3(256), 0, s, v, bs,
                bo, nmax, tr, d_nnzb, st, o);
            else pdl_launch(pack_tiles_kernel<uint16_t, 4, 1>, dim3(g1), dim3(256), 0, s, v, bs, bo,
                nmax, tr, d_nnzb, st, o);
            break;
        default:
            pdl_launch(pack_tiles_kernel<uint16_t, 1, 1>, dim3(g1), dim3(256), 0, s, v, bs, bo,
                nmax, tr, d_nnzb, st, o);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_quantize_e4m3(int64_t nnzb, int b, spmm_dtype src, const void *d_src,
                                 uint8_t *d_codes, float *d_scales, cudaStream_t s) {
    if (nnzb == 0) return cudaSuccess;
    const int64_t threads = nnzb * 32;
    const unsigned grid = (unsigned)((threads + 255) / 256);
    switch (src) {
        case SPMM_F32:
            pdl_launch(quantize_e4m3_kernel<float>, dim3(grid), dim3(256), 0, s,
                (const float *)d_src, nnzb, b, d_codes, d_scales);
            break;
        case SPMM_F16:
            pdl_launch(quantize_e4m3_kernel<__half>, dim3(grid), dim3(256), 0, s,
                (const __half *)d_src, nnzb, b, d_codes, d_scales);
            break;
        case SPMM_BF16:
            pdl_launch(quantize_e4m3_kernel<__nv_bfloat16>, dim3(grid), dim3(256), 0, s,
                (const __nv_bfloat16 *)d_src, nnzb, b, d_codes, d_scales);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace spmm
