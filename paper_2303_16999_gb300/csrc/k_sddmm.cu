// Sampled dense-dense product on the block mask (SDDMM) on the tensor cores:
//   dW[p][ii][l] = sum_j dY[brow_p*b + ii, j] * X[bcol_p*b + l, j]
// for every stored block p -- the gradient of Section 3's product
// Y = (M . W) X with respect to the stored blocks, the weight-gradient step
// of the sparse training regimes of Section 1.  The contraction runs over n.
//
// Dense-tile form: the m x k output space is cut into 128 x 256 tiles, and a
// tile's D = dY[128 rows] . X[256 rows]^T is accumulated in TMEM over n by
// tcgen05.mma (M = 128, N = 256, K = 16; both operands K-major with 128-byte
// swizzle, exactly as the rows of dY and X lie in memory), fed by TMA in
// 64-element steps of n (16 KB of dY + 32 KB of X per stage, four stages).
// The epilogue keeps only the stored blocks: each epilogue thread owns one dY
// row (one TMEM lane), walks its block row's CSR entries inside the tile's
// columns (sorted by column, so the cursor carries from one tile to the
// next) and writes row ii of each block p, in the pattern's order.  A warp
// reads a 32-column slice of the accumulator only when one of its rows has a
// stored block there.  Every tile costs the same, so the kernel is
// persistent: one CTA per SM owning all 512 TMEM columns (two accumulators,
// so the epilogue of one tile overlaps the MMAs of the next), each CTA taking
// a contiguous run of tiles in row-major order.
//
// Gathered form (b = 16, low density): a work item is up to eight blocks of
// one block row r.  Their X rows (8 x 16 = 128 rows) are gathered by TMA as
// the MMA's A operand and the 16 rows of dY at r as its B operand, so
// D[128 x 16] = X rows . dY rows^T holds the eight blocks, transposed, in
// TMEM (M = 128, N = 16).  Only the stored blocks' rows move: about
// nnzb * 1.125 * 16 * n * 2 bytes from L2, against the dense form's whole
// tiles, which wins below a density of about 1/7.
//
// Warp roles (192 threads) in both kernels: warp 0 = TMA producer, warp 1 =
// MMA issuer and TMEM owner, warps 2..5 = epilogue (warp w reads TMEM lanes
// 32 (w % 4) on).  Every mbarrier wait is bounded; on expiry the CTA records
// SPMM_ERR_TIMEOUT in the plan's status word, lets its copies and MMAs in
// flight finish, frees TMEM and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <climits>

#include "pdl.cuh"
#include "spmm_internal.h"
#include "tc_ptx.cuh"

namespace spmm {
namespace {

constexpr int kSdBM = 128;        // tile rows (rows of dY, TMEM lanes)
constexpr int kSdBN = 256;        // tile columns (rows of X, accumulator columns)
constexpr int kSdBK = 64;         // elements of n per stage (one 128-byte swizzle row)
constexpr int kSdStages = 4;
constexpr int kSdThreads = 192;
constexpr int kSdChunk = 32;      // accumulator columns per epilogue read
constexpr int kSdRing = 24;       // CSR entries (column, block) staged per epilogue thread
constexpr uint32_t kSdABytes = kSdBM * kSdBK * 2;
constexpr uint32_t kSdBBytes = kSdBN * kSdBK * 2;
constexpr uint32_t kSdStageBytes = kSdABytes + kSdBBytes;
constexpr unsigned long long kSdWaitNs = 2000000000ull;   // 2 s per wait

struct __align__(8) SdSmem {
    uint64_t full[kSdStages], empty[kSdStages], accf[2], acce[2], drain;
    uint32_t tmem_base;
    volatile int32_t abort_flag;
    int32_t issued, consumed;      // stages issued by the producer / consumed by the MMA warp
    int32_t issued2[4];            // gathered form: next stage index of each of its producers
};

struct SdArgs {
    const int32_t *row_ptr, *col_idx, *perm;   // block CSR of the pattern (perm: CSR -> pattern order)
    void *dW;
    int32_t *status;
    const int32_t *skip_if;        // dynamic plans: the status word (a rejected pattern writes nothing)
    int64_t m;
    int32_t ntn, ksteps, fmt;      // tiles along k, stages along n, operand format (0 F16, 1 BF16)
    int64_t ntiles;
};

// Bounded wait (lane 0 waits, the warp learns the outcome).
__device__ __forceinline__ bool sd_wait_warp(uint64_t *bar, uint32_t parity, SdSmem *sm,
                                             int lane) {
    return mbar_wait_warp(bar, parity, &sm->abort_flag, kSdWaitNs, lane);
}
__device__ __forceinline__ void sd_abort(SdSmem *sm, int32_t *status) {
    sm->abort_flag = 1;
    atomicCAS(status, 0, (int32_t)kDevTimeout);
}

// K-major operand with 128-byte swizzle: rows of 128 B, 8-row groups 1024 B
// apart (stride offset); the leading offset is unused for this layout.
__device__ __forceinline__ uint64_t sd_desc(uint32_t addr) { return smem_desc(addr, 16, 1024, 2); }

// kind::f16 instruction descriptor with both operands K-major: FP32
// accumulator (bits 4-5 = 1), A / B format in bits 7-9 / 10-12, N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
__device__ __forceinline__ uint32_t sd_idesc(uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kSdBN >> 3) << 17) |
           ((uint32_t)(kSdBM >> 4) << 24);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Output element types: OUT 0 = F32, 1 = F16, 2 = BF16.
template <int OUT> struct SdOut;
template <> struct SdOut<0> {
    using T = float;
    static __device__ __forceinline__ void put(float *d, const float *v, int cnt) {
        if (cnt % 4 == 0) {
            for (int i = 0; i < cnt; i += 4)
                *reinterpret_cast<float4 *>(d + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        } else {
            for (int i = 0; i < cnt; ++i) d[i] = v[i];
        }
    }
};
template <typename H> struct SdOut16 {
    using T = H;
    static __device__ __forceinline__ void put(H *d, const float *v, int cnt) {
        if (cnt % 8 == 0) {
            for (int i = 0; i < cnt; i += 8) {
                uint4 u;
                uint32_t *w = reinterpret_cast<uint32_t *>(&u);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    H lo = Cvt<H>::f(v[i + 2 * j]), hi = Cvt<H>::f(v[i + 2 * j + 1]);
                    w[j] = (uint32_t)*reinterpret_cast<uint16_t *>(&lo) |
                           ((uint32_t)*reinterpret_cast<uint16_t *>(&hi) << 16);
                }
                *reinterpret_cast<uint4 *>(d + i) = u;
            }
        } else {
            for (int i = 0; i < cnt; ++i) d[i] = Cvt<H>::f(v[i]);
        }
    }
};
template <> struct SdOut<1> : SdOut16<__half> {};
template <> struct SdOut<2> : SdOut16<__nv_bfloat16> {};

// Row ii of block p from accumulator columns off .. off + B - 1 of the
// 32-column slice v (off a multiple of B; static indices only).
template <int B, int OUT>
__device__ __forceinline__ void sd_put_row(void *dW, int64_t p, int ii, const float *v, int off) {
    using O = SdOut<OUT>;
    typename O::T *dst = reinterpret_cast<typename O::T *>(dW) + (p * B * B + (int64_t)ii * B);
    if (B == 1) {
        float x = v[0];
#pragma unroll
        for (int q = 1; q < kSdChunk; ++q) x = off == q ? v[q] : x;
        O::put(dst, &x, 1);
    } else {
#pragma unroll
        for (int q = 0; q < kSdChunk / B; ++q)
            if (off == q * B) O::put(dst, v + q * B, B);
    }
}

// A thread's CSR cursor: entries [head, tail) of its block row are staged in
// a ring of kSdRing (column, block) pairs in shared memory (slot i of thread
// t at ring[i * 128 + t]); top_up() refills the free slots with independent
// loads, so one L2 round trip serves up to kSdRing entries.
struct SdCursor {
    int2 *ring;
    int32_t head, tail, end;
    __device__ __forceinline__ void top_up(const int32_t *col_idx, const int32_t *perm) {
        const int32_t cnt = min(kSdRing - (tail - head), end - tail);
        int32_t cv[kSdRing], pv[kSdRing];
#pragma unroll
        for (int i = 0; i < kSdRing; ++i) {
            cv[i] = i < cnt ? __ldg(col_idx + tail + i) : 0;
            pv[i] = i < cnt ? __ldg(perm + tail + i) : 0;
        }
#pragma unroll
        for (int i = 0; i < kSdRing; ++i)
            if (i < cnt) ring[((tail + i) % kSdRing) * 128] = make_int2(cv[i], pv[i]);
        tail += cnt > 0 ? cnt : 0;
    }
    __device__ __forceinline__ int2 front() const { return ring[(head % kSdRing) * 128]; }
};

template <int B, int OUT>
__global__ void __launch_bounds__(kSdThreads, 1)
    sddmm_dense_kernel(const __grid_constant__ CUtensorMap map_dy,
                       const __grid_constant__ CUtensorMap map_x, const SdArgs args) {
    pdl_enter();
    if (args.skip_if && *args.skip_if != 0) return;
    extern __shared__ __align__(1024) uint8_t sm_raw[];
    uint8_t *stages = (uint8_t *)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
    int2 *rings = reinterpret_cast<int2 *>(stages + kSdStages * kSdStageBytes);
    SdSmem *sm = reinterpret_cast<SdSmem *>(rings + kSdRing * 128);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t tb = (int64_t)blockIdx.x * args.ntiles / gridDim.x;
    const int64_t te = (int64_t)(blockIdx.x + 1) * args.ntiles / gridDim.x;
    if (tb >= te) return;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kSdStages; ++s) {
            mbar_init(&sm->full[s], 1);
            mbar_init(&sm->empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&sm->accf[a], 1);
            mbar_init(&sm->acce[a], 128);
        }
        mbar_init(&sm->drain, 1);
        sm->abort_flag = 0;
        sm->issued = sm->consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == 1) {
        tmem_alloc(&sm->tmem_base, 2 * kSdBN);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm->tmem_base;
    const int ntn = args.ntn, ksteps = args.ksteps;

    if (warp == 0) {
        // ---- TMA producer
        if (lane == 0) {
            int32_t it = 0;
            bool ok = true;
            for (int64_t t = tb; t < te && ok; ++t) {
                const int tm = (int)(t / ntn), tn = (int)(t % ntn);
                for (int ks = 0; ks < ksteps; ++ks, ++it) {
                    const int s = it % kSdStages;
                    const uint32_t ph = (uint32_t)((it / kSdStages) & 1);
                    if (!mbar_wait_bounded(&sm->empty[s], ph ^ 1u, &sm->abort_flag, kSdWaitNs)) {
                        sd_abort(sm, args.status);
                        ok = false;
                        break;
                    }
                    uint8_t *a = stages + s * kSdStageBytes;
                    mbar_arrive_tx(&sm->full[s], kSdStageBytes);
                    tma_load_2d(a, &map_dy, ks * kSdBK, tm * kSdBM, &sm->full[s]);
                    tma_load_2d(a + kSdABytes, &map_x, ks * kSdBK, tn * kSdBN, &sm->full[s]);
                }
            }
            sm->issued = it;
        }
    } else if (warp == 1) {
        // ---- MMA issuer (converged warp; one elected lane issues)
        const uint32_t idesc = sd_idesc((uint32_t)args.fmt);
        int32_t it = 0;
        bool ok = true;
        for (int64_t t = tb, lt = 0; t < te && ok; ++t, ++lt) {
            const uint32_t a = (uint32_t)(lt & 1), aph = (uint32_t)((lt >> 1) & 1);
            if (!sd_wait_warp(&sm->acce[a], aph ^ 1u, sm, lane)) {
                if (lane == 0) sd_abort(sm, args.status);
                break;
            }
            tc_fence_after();
            const uint32_t d = tmem + a * kSdBN;
            for (int ks = 0; ks < ksteps; ++ks, ++it) {
                const int s = it % kSdStages;
                const uint32_t ph = (uint32_t)((it / kSdStages) & 1);
                if (!sd_wait_warp(&sm->full[s], ph, sm, lane)) {
                    if (lane == 0) sd_abort(sm, args.status);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t abase = smem_u32(stages + s * kSdStageBytes);
                const uint32_t bbase = abase + kSdABytes;
#pragma unroll
                for (int kk = 0; kk < kSdBK / 16; ++kk)
                    tc_mma_elect(d, sd_desc(abase + kk * 32), sd_desc(bbase + kk * 32), idesc,
                                 (ks | kk) ? 1u : 0u);
                __syncwarp();
                if (lane == 0) tc_commit(&sm->empty[s]);
            }
            if (!ok) break;
            __syncwarp();
            if (lane == 0) {
                if (ksteps > 0) tc_commit(&sm->accf[a]);
                else mbar_arrive(&sm->accf[a]);   // n = 0: nothing accumulated
            }
        }
        if (lane == 0) sm->consumed = it;
    } else {
        // ---- epilogue: one dY row per thread
        const int q = warp & 3;
        const int row_local = q * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        SdCursor cur;
        cur.ring = rings + row_local;
        cur.head = cur.tail = cur.end = 0;
        int cur_tm = -1, ii = 0;
        for (int64_t t = tb, lt = 0; t < te; ++t, ++lt) {
            const int tm = (int)(t / ntn), tn = (int)(t % ntn);
            if (tm != cur_tm) {
                // a new row of tiles: find the first entry at or after the tile's columns
                cur_tm = tm;
                const int64_t r = (int64_t)tm * kSdBM + row_local;
                cur.head = cur.tail = cur.end = 0;
                if (r < args.m) {
                    const int32_t R = (int32_t)(r / B);
                    ii = (int)(r % B);
                    int32_t lo = __ldg(args.row_ptr + R), hi = __ldg(args.row_ptr + R + 1);
                    cur.end = hi;
                    const int32_t cmin = (int32_t)((int64_t)tn * kSdBN / B);
                    while (lo < hi) {
                        const int32_t mid = (lo + hi) >> 1;
                        if (__ldg(args.col_idx + mid) < cmin) lo = mid + 1;
                        else hi = mid;
                    }
                    cur.head = cur.tail = lo;
                }
            }
            cur.top_up(args.col_idx, args.perm);   // before the wait: its loads overlap the MMAs
            const uint32_t a = (uint32_t)(lt & 1), aph = (uint32_t)((lt >> 1) & 1);
            if (!sd_wait_warp(&sm->accf[a], aph, sm, lane)) {
                if (lane == 0) sd_abort(sm, args.status);
                break;
            }
            tc_fence_after();
            int2 e = cur.head < cur.tail ? cur.front() : make_int2(INT_MAX, 0);
            for (int j = 0; j < kSdBN / kSdChunk; ++j) {
                const int32_t cb = tn * kSdBN + j * kSdChunk;       // first column of the slice
                const int32_t cend = (cb + kSdChunk) / B;           // block columns below the slice end
                bool need = e.x < cend;
                if (!__any_sync(0xffffffffu, need)) continue;
                float v[kSdChunk];
                tmem_ld32(tmem + lane_addr + a * kSdBN + j * kSdChunk, v);
                if (ksteps == 0) {
#pragma unroll
                    for (int i = 0; i < kSdChunk; ++i) v[i] = 0.f;
                }
                while (need) {
                    sd_put_row<B, OUT>(args.dW, e.y, ii, v, e.x * B - cb);
                    ++cur.head;
                    if (cur.head == cur.tail && cur.tail < cur.end)
                        cur.top_up(args.col_idx, args.perm);
                    e = cur.head < cur.tail ? cur.front() : make_int2(INT_MAX, 0);
                    need = e.x < cend;
                }
            }
            tc_fence_before();
            mbar_arrive(&sm->acce[a]);
        }
    }

    __syncthreads();
    if (sm->abort_flag) {
        // let copies and MMAs still in flight land before TMEM and shared memory go
        if (threadIdx.x == 0) {
            for (int32_t c = sm->consumed; c < sm->issued; ++c) {
                const int s = c % kSdStages;
                const uint32_t par = (uint32_t)((c / kSdStages) & 1);
                const unsigned long long t0 = gtimer();
                while (!mbar_try(&sm->full[s], par) && gtimer() - t0 < kSdWaitNs) {
                }
            }
        }
        if (warp == 1) {
            if (lane == 0) {
                tc_commit(&sm->drain);
                const unsigned long long t0 = gtimer();
                while (!mbar_try(&sm->drain, 0) && gtimer() - t0 < kSdWaitNs) {
                }
            }
            __syncwarp();
        }
        __syncthreads();
    }
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * kSdBN);
    }
}

// ------------------------------------------------------ gathered form ----
constexpr int kSgBlocks = 8;                      // blocks per work item (A = 128 rows)
constexpr int kSgStages = 4;
constexpr int kSgCtasPerSm = 3;
#ifndef SPMM_SG_PRODUCERS
#define SPMM_SG_PRODUCERS 2
#endif
constexpr int kSgProducers = SPMM_SG_PRODUCERS;   // warp 0 and warps 6, 7, ...
static_assert(kSgProducers >= 1 && kSgProducers <= 4, "producer warps");
constexpr int kSgThreads = kSdThreads + 32 * (kSgProducers - 1);
constexpr uint32_t kSgBox = 16 * kSdBK * 2;       // 2048: 16 rows x 64 elements
constexpr uint32_t kSgStageBytes = (kSgBlocks + 1) * kSgBox;
static_assert(kSgStages <= kSdStages, "the barrier arrays of SdSmem hold kSdStages stages");

// Work items of the gathered form from the block CSR: row r gives
// ceil(count / 8) items (r, first entry, end entry); items[0] = the count.
// One CTA; rows in chunks of 1024, an exclusive scan of the item counts.
__global__ void __launch_bounds__(1024)
    sddmm_items_kernel(const int32_t *row_ptr, int32_t mb, const int32_t *skip_if,
                       int32_t *items) {
    pdl_enter();
    __shared__ int32_t warp_sum[32];
    __shared__ int32_t base_s;
    if (threadIdx.x == 0) base_s = 0;
    __syncthreads();
    const bool skip = skip_if && *skip_if != 0;    // a rejected pattern: no items
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int32_t r0 = 0; r0 < mb && !skip; r0 += 1024) {
        const int32_t r = r0 + threadIdx.x;
        const int32_t beg = r < mb ? row_ptr[r] : 0, end = r < mb ? row_ptr[r + 1] : 0;
        const int32_t ni = (end - beg + kSgBlocks - 1) / kSgBlocks;
        int32_t incl = ni;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) warp_sum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int32_t ws = warp_sum[lane], wi = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t v = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += v;
            }
            warp_sum[lane] = wi - ws;              // exclusive prefix of the warp sums
        }
        __syncthreads();
        const int32_t first = base_s + warp_sum[wid] + incl - ni;
        for (int32_t j = 0; j < ni; ++j) {
            int32_t *it = items + 1 + 3 * (int64_t)(first + j);
            it[0] = r;
            it[1] = beg + j * kSgBlocks;
            it[2] = min(beg + (j + 1) * kSgBlocks, end);
        }
        __syncthreads();
        if (threadIdx.x == 1023) base_s = first + ni;
        __syncthreads();
    }
    if (threadIdx.x == 0) items[0] = skip ? 0 : base_s;
}

// K-major, 128-byte swizzle, N = 16: D[128 x 16] fp32.
__device__ __forceinline__ uint32_t sg_idesc(uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
}

struct SgArgs {
    const int32_t *items, *col_idx, *perm;
    void *dW;
    int32_t *status;
    int32_t ksteps, fmt;
};

template <int OUT>
__global__ void __launch_bounds__(kSgThreads, kSgCtasPerSm)
    sddmm_gather_kernel(const __grid_constant__ CUtensorMap map_dy,
                        const __grid_constant__ CUtensorMap map_x, const SgArgs args) {
    pdl_enter();
    const int32_t nitems = *args.items;            // 0 for a rejected dynamic pattern
    if ((int32_t)blockIdx.x >= nitems) return;
    extern __shared__ __align__(1024) uint8_t sm_raw[];
    uint8_t *stages = (uint8_t *)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
    SdSmem *sm = reinterpret_cast<SdSmem *>(stages + kSgStages * kSgStageBytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kSgStages; ++s) {
            mbar_init(&sm->full[s], 1);
            mbar_init(&sm->empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&sm->accf[a], 1);
            mbar_init(&sm->acce[a], 128);
        }
        mbar_init(&sm->drain, 1);
        sm->abort_flag = 0;
        sm->issued = sm->consumed = 0;
        for (int i = 0; i < 4; ++i) sm->issued2[i] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == 1) {
        tmem_alloc(&sm->tmem_base, 32);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm->tmem_base;
    const int ksteps = args.ksteps;
    const int32_t *items = args.items + 1;

    if (warp == 0 || warp >= 6) {
        // ---- producers: producer j fills stages it with it % kSgProducers
        // == j (each issue costs its warp time, so warps issue side by side);
        // lane i < 8 copies block i's X rows, lane 8 the dY rows
        const int pid = warp == 0 ? 0 : warp - 5;
        int32_t it = 0, mine = 0;
        bool ok = true;
        int32_t nx = (int32_t)blockIdx.x;
        int32_t ncol = 0;
        {
            const int32_t e0 = items[3 * nx + 1], e1 = items[3 * nx + 2];
            ncol = lane < e1 - e0 ? __ldg(args.col_idx + e0 + lane) : 0;
        }
        for (int32_t w = (int32_t)blockIdx.x; w < nitems && ok; w += gridDim.x) {
            const int32_t r = items[3 * w], nb = items[3 * w + 2] - items[3 * w + 1];
            const int32_t col = ncol;
            const int32_t wn = w + (int32_t)gridDim.x;
            if (wn < nitems) {   // the next item's columns, loaded while this one is issued
                const int32_t e0 = items[3 * wn + 1], e1 = items[3 * wn + 2];
                ncol = lane < e1 - e0 ? __ldg(args.col_idx + e0 + lane) : 0;
            }
            for (int ks = 0; ks < ksteps; ++ks, ++it) {
                if (it % kSgProducers != pid) continue;
                const int s = it % kSgStages;
                const uint32_t ph = (uint32_t)((it / kSgStages) & 1);
                if (!sd_wait_warp(&sm->empty[s], ph ^ 1u, sm, lane)) {
                    if (lane == 0) sd_abort(sm, args.status);
                    ok = false;
                    break;
                }
                mine = it + 1;
                uint8_t *base = stages + s * kSgStageBytes;
                if (lane == 0) mbar_arrive_tx(&sm->full[s], (uint32_t)(nb + 1) * kSgBox);
                __syncwarp();
                if (lane < nb)
                    tma_load_2d(base + lane * kSgBox, &map_x, ks * kSdBK, col * 16, &sm->full[s]);
                else if (lane == kSgBlocks)
                    tma_load_2d(base + kSgBlocks * kSgBox, &map_dy, ks * kSdBK, r * 16,
                                &sm->full[s]);
                __syncwarp();
            }
        }
        if (lane == 0) sm->issued2[pid] = mine;
    } else if (warp == 1) {
        // ---- MMA issuer
        const uint32_t idesc = sg_idesc((uint32_t)args.fmt);
        int32_t it = 0;
        bool ok = true;
        int32_t lt = 0;
        for (int32_t w = (int32_t)blockIdx.x; w < nitems && ok; w += gridDim.x, ++lt) {
            const uint32_t a = (uint32_t)(lt & 1), aph = (uint32_t)((lt >> 1) & 1);
            if (!sd_wait_warp(&sm->acce[a], aph ^ 1u, sm, lane)) {
                if (lane == 0) sd_abort(sm, args.status);
                break;
            }
            tc_fence_after();
            const uint32_t d = tmem + a * 16;
            for (int ks = 0; ks < ksteps; ++ks, ++it) {
                const int s = it % kSgStages;
                const uint32_t ph = (uint32_t)((it / kSgStages) & 1);
                if (!sd_wait_warp(&sm->full[s], ph, sm, lane)) {
                    if (lane == 0) sd_abort(sm, args.status);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t abase = smem_u32(stages + s * kSgStageBytes);
                const uint32_t bbase = abase + kSgBlocks * kSgBox;
#pragma unroll
                for (int kk = 0; kk < kSdBK / 16; ++kk)
                    tc_mma_elect(d, sd_desc(abase + kk * 32), sd_desc(bbase + kk * 32), idesc,
                                 (ks | kk) ? 1u : 0u);
                __syncwarp();
                if (lane == 0) tc_commit(&sm->empty[s]);
            }
            if (!ok) break;
            __syncwarp();
            if (lane == 0) {
                if (ksteps > 0) tc_commit(&sm->accf[a]);
                else mbar_arrive(&sm->accf[a]);   // n = 0: nothing accumulated
            }
        }
        if (lane == 0) sm->consumed = it;
    } else {
        // ---- epilogue: TMEM lane t = 16 e + l holds row l of block e, transposed
        const int q = warp & 3;
        const int t = q * 32 + lane, e = t >> 4, l = t & 15;
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        using O = SdOut<OUT>;
        typename O::T *dW = reinterpret_cast<typename O::T *>(args.dW);
        int32_t lt = 0;
        for (int32_t w = (int32_t)blockIdx.x; w < nitems; w += gridDim.x, ++lt) {
            const int32_t e0 = items[3 * w + 1], nb = items[3 * w + 2] - e0;
            const int32_t p = e < nb ? __ldg(args.perm + e0 + e) : 0;
            const uint32_t a = (uint32_t)(lt & 1), aph = (uint32_t)((lt >> 1) & 1);
            if (!sd_wait_warp(&sm->accf[a], aph, sm, lane)) {
                if (lane == 0) sd_abort(sm, args.status);
                break;
            }
            tc_fence_after();
            float v[16];
            tmem_ld16(tmem + lane_addr + a * 16, v);
            if (e < nb) {
                typename O::T *dst = dW + (int64_t)p * 256 + l;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float x = ksteps > 0 ? v[i] : 0.f;
                    O::put(dst + i * 16, &x, 1);
                }
            }
            tc_fence_before();
            mbar_arrive(&sm->acce[a]);
        }
    }

    __syncthreads();
    if (sm->abort_flag) {
        if (threadIdx.x == 0) {
            // stages each producer issued and the MMA warp did not consume
            int32_t hi = 0;
            for (int i = 0; i < kSgProducers; ++i) hi = max(hi, sm->issued2[i]);
            for (int32_t c = sm->consumed; c < hi; ++c) {
                if (c >= sm->issued2[c % kSgProducers]) continue;
                const int s = c % kSgStages;
                const uint32_t par = (uint32_t)((c / kSgStages) & 1);
                const unsigned long long t0 = gtimer();
                while (!mbar_try(&sm->full[s], par) && gtimer() - t0 < kSdWaitNs) {
                }
            }
        }
        if (warp == 1) {
            if (lane == 0) {
                tc_commit(&sm->drain);
                const unsigned long long t0 = gtimer();
                while (!mbar_try(&sm->drain, 0) && gtimer() - t0 < kSdWaitNs) {
                }
            }
            __syncwarp();
        }
        __syncthreads();
    }
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 32);
    }
}

cudaError_t encode_rows(CUtensorMap *map, bool bf16, const void *base, int64_t rows, int64_t n,
                        int64_t ld, uint32_t box_rows) {
    auto enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    const cuuint32_t box[2] = {(cuuint32_t)kSdBK, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                           2, const_cast<void *>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int B, int OUT>
cudaError_t launch_dense(const CUtensorMap &mdy, const CUtensorMap &mx, const SdArgs &a, int grid,
                         cudaStream_t s) {
    const size_t smem = 1024 + (size_t)kSdStages * kSdStageBytes +
                        sizeof(int2) * kSdRing * 128 + sizeof(SdSmem);
    static std::atomic<uint64_t> attrs{0};
    const cudaError_t e = set_smem_attrs_once(attrs, sddmm_dense_kernel<B, OUT>, (int)smem, false);
    if (e != cudaSuccess) return e;
    pdl_launch(sddmm_dense_kernel<B, OUT>, dim3(grid), dim3(kSdThreads), smem, s, mdy, mx, a);
    return cudaGetLastError();
}

template <int OUT>
cudaError_t launch_gather(const CUtensorMap &mdy, const CUtensorMap &mx, const SgArgs &a, int grid,
                          cudaStream_t s) {
    const size_t smem = 1024 + (size_t)kSgStages * kSgStageBytes + sizeof(SdSmem);
    static std::atomic<uint64_t> attrs{0};
    const cudaError_t e = set_smem_attrs_once(attrs, sddmm_gather_kernel<OUT>, (int)smem, true);
    if (e != cudaSuccess) return e;
    pdl_launch(sddmm_gather_kernel<OUT>, dim3(grid), dim3(kSgThreads), smem, s, mdy, mx, a);
    return cudaGetLastError();
}

template <int B>
cudaError_t launch_dense_b(int out, const CUtensorMap &mdy, const CUtensorMap &mx, const SdArgs &a,
                           int grid, cudaStream_t s) {
    switch (out) {
        case 0: return launch_dense<B, 0>(mdy, mx, a, grid, s);
        case 1: return launch_dense<B, 1>(mdy, mx, a, grid, s);
        default: return launch_dense<B, 2>(mdy, mx, a, grid, s);
    }
}

}  // namespace

// The gathered form moves about 1.125 x 16 rows x 2 n bytes per stored
// block, issued as nine 2 KB boxes per step (measured ~7.6 TB/s from L2 at
// m = k = 4096, n = 2048, d = 1/16: 41 us against 49 us of dense tiles at
// ~1.4 PFLOP/s); the times cross near d = 1/13, so blocks of 16 below that
// density (nnzb_max for dynamic plans) take the gathered form.
bool sddmm_gathers(const spmm_plan *p) {
    // (host-only plans report the choice a device plan of theirs would make)
    if (p->b != 16 || (!p->host_only && !p->d_sd_items)) return false;
    const double nb = (double)(p->mode == SPMM_STATIC ? p->nnzb : p->nnzb_max);
    return nb * 256.0 * 13.0 < (double)p->m * (double)p->k;
}

cudaError_t launch_sddmm(const spmm_plan *p, const void *d_dY, int64_t lddy, const void *d_X,
                         int64_t ldx, int64_t n, void *d_dW, spmm_dtype dw_dtype, cudaStream_t s) {
    const bool bf16 = p->xdt == SPMM_BF16;
    CUtensorMap mdy, mx;
    // n = 0 still runs and writes every stored block as zero; no copy is
    // issued then, so the maps only have to encode (over dW's first bytes)
    cudaError_t e = n > 0 ? encode_rows(&mdy, bf16, d_dY, p->m, n, lddy, kSdBM)
                          : encode_rows(&mdy, bf16, d_dW, 1, 8, 8, kSdBM);
    if (e == cudaSuccess)
        e = n > 0 ? encode_rows(&mx, bf16, d_X, p->k, n, ldx, kSdBN)
                  : encode_rows(&mx, bf16, d_dW, 1, 8, 8, kSdBN);
    if (e != cudaSuccess) return e;
    SdArgs a{};
    a.row_ptr = p->d_row_ptr;
    a.col_idx = p->d_col_idx;
    a.perm = p->d_perm;
    a.dW = d_dW;
    a.status = p->d_status;
    a.skip_if = p->mode == SPMM_DYNAMIC ? p->d_status : nullptr;
    a.m = p->m;
    const int64_t ntm = (p->m + kSdBM - 1) / kSdBM;
    a.ntn = (int32_t)((p->k + kSdBN - 1) / kSdBN);
    a.ksteps = (int32_t)((n + kSdBK - 1) / kSdBK);
    a.fmt = bf16 ? 1 : 0;
    a.ntiles = ntm * a.ntn;
    const int grid = (int)(a.ntiles < p->sm_count ? a.ntiles : p->sm_count);
    const int out = dw_dtype == SPMM_F32 ? 0 : (dw_dtype == SPMM_F16 ? 1 : 2);
    if (sddmm_gathers(p)) {
        // dY rows of one block row: a 16-row box (the dense form's map has 128)
        if (n > 0) e = encode_rows(&mdy, bf16, d_dY, p->m, n, lddy, 16);
        if (n > 0 && e == cudaSuccess) e = encode_rows(&mx, bf16, d_X, p->k, n, ldx, 16);
        if (n == 0) {
            e = encode_rows(&mdy, bf16, d_dW, 1, 8, 8, 16);
            if (e == cudaSuccess) e = encode_rows(&mx, bf16, d_dW, 1, 8, 8, 16);
        }
        if (e != cudaSuccess) return e;
        const int32_t mb = (int32_t)(p->m / 16);
        pdl_launch(sddmm_items_kernel, dim3(1), dim3(1024), 0, s, p->d_row_ptr, mb, a.skip_if,
                   p->d_sd_items);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        SgArgs g{};
        g.items = p->d_sd_items;
        g.col_idx = p->d_col_idx;
        g.perm = p->d_perm;
        g.dW = d_dW;
        g.status = p->d_status;
        g.ksteps = a.ksteps;
        g.fmt = a.fmt;
        // the item count is known on the device only: one CTA per item up to three per SM
        const int64_t cap = p->sd_items_cap, slots = (int64_t)p->sm_count * kSgCtasPerSm;
        const int ggrid = (int)(cap < slots ? cap : slots);
        switch (out) {
            case 0: return launch_gather<0>(mdy, mx, g, ggrid, s);
            case 1: return launch_gather<1>(mdy, mx, g, ggrid, s);
            default: return launch_gather<2>(mdy, mx, g, ggrid, s);
        }
    }
    switch (p->b) {
        case 1: return launch_dense_b<1>(out, mdy, mx, a, grid, s);
        case 4: return launch_dense_b<4>(out, mdy, mx, a, grid, s);
        case 8: return launch_dense_b<8>(out, mdy, mx, a, grid, s);
        default: return launch_dense_b<16>(out, mdy, mx, a, grid, s);
    }
}

}  // namespace spmm
