// Blocked-ELL product for b = 16 (dynamic sparsity without re-partition).
//
// W arrives as a padded list of blocks per block row -- the Blocked-ELL
// layout that Section 5 names as the FP16 block-sparse format of the GPU
// library it compares against: ell_cols[r * E + e] is the block column of
// slot e of block row r (columns strictly increasing, then -1 padding up to
// the width E), and values[r * E + e] is that block, 16 x 16 row-major.  The
// layout itself is the work list, so a call with a new pattern needs no
// device re-partition (Section 3.3's dynamic mode re-plans every call): one
// validation launch, one product launch.
//
// One work unit = (block row r, 128 columns of n).  Its accumulator is
// D[128 n x 16 rows] in TMEM; for each block (r, c) of the row one
// tcgen05.mma (M = 128, N = 16, K = 16) adds X slab(c) . W(r, c)^T, with
// the X slab (16 rows of X, 128 columns, MN-major, 128-byte swizzle) and
// the block (K-major, 32-byte swizzle) both loaded by TMA: the block is
// read straight from the caller's row-major values, so nothing is packed.
// A stage holds kEllSlots consecutive slots of one row (their X slabs, one
// TMA each, issued by separate lanes, and one TMA for the slots' blocks).
// Units go to CTAs in contiguous runs (persistent, three CTAs per SM); the
// epilogue of one unit overlaps the MMAs of the next (two accumulators).
//
// Warp roles (224 threads): warps 0 and 6 = TMA producers (alternate
// stages; one warp alone issued too slowly: 52.9 against 48.6 us per call
// at m = k = 8192, n = 1024, d = 1/16), warp 1 = MMA issuer and TMEM owner,
// warps 2..5 = epilogue (TMEM -> Y, 16-bit).  Every mbarrier
// wait is bounded; on expiry the CTA records SPMM_ERR_TIMEOUT in the
// status word, lets its copies and MMAs in flight land and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "pdl.cuh"
#include "spmm_internal.h"
#include "tc_ptx.cuh"

namespace spmm {
namespace {

constexpr int kEllSlots = 4;          // ELL slots per stage
constexpr int kEllStages = 4;
#ifndef SPMM_ELL_PRODUCERS
#define SPMM_ELL_PRODUCERS 2
#endif
constexpr int kEllProducers = SPMM_ELL_PRODUCERS;   // warp 0 and warps 6, 7, ...
static_assert(kEllProducers >= 1 && kEllProducers <= 4, "producer warps");
constexpr int kEllThreads = 192 + 32 * (kEllProducers - 1);
constexpr int kEllCtasPerSm = 3;
constexpr uint32_t kEllSlab = kSlabRows * kSlabHalf * 2 * 2;   // 4096: X slab, 16 x 128
constexpr uint32_t kEllBlock = 16 * 16 * 2;                     // 512: one W block
constexpr uint32_t kEllStageBytes = kEllSlots * (kEllSlab + kEllBlock);
constexpr unsigned long long kEllWaitNs = 2000000000ull;        // 2 s per wait

struct __align__(8) EllSmem {
    uint64_t full[kEllStages], empty[kEllStages], accf[2], acce[2], drain;
    uint32_t mask[kEllStages];        // per stage: valid slots (bits 0-3) | last stage of unit << 8
    uint32_t tmem_base;
    volatile int32_t abort_flag;
    int32_t issued[4], consumed;      // next stage index of each producer / stages consumed
};

struct EllArgs {
    const int32_t *cols;              // ell_cols, mb x E
    void *Y;
    int32_t *status;
    int64_t ldy, n;
    int32_t mb, E, ntn, x3d, fmt;
    int64_t units;
};

// Bounded wait (lane 0 waits, the warp learns the outcome).
__device__ __forceinline__ bool ell_wait_warp(uint64_t *bar, uint32_t parity, EllSmem *sm,
                                              int lane) {
    return mbar_wait_warp(bar, parity, &sm->abort_flag, kEllWaitNs, lane);
}
__device__ __forceinline__ void ell_abort(EllSmem *sm, int32_t *status) {
    sm->abort_flag = 1;
    atomicCAS(status, 0, (int32_t)kDevTimeout);
}

// X slab: MN-major, 128-byte swizzle, the 64-column halves 2048 B apart
// (leading offset), the 8-row k groups 1024 B apart (stride offset).
__device__ __forceinline__ uint64_t ell_a_desc(uint32_t addr) {
    return smem_desc(addr, 2048, 1024, 2);
}
// W block: K-major rows of 32 B with 32-byte swizzle (layout code 6), 8-row
// groups 256 B apart.
__device__ __forceinline__ uint64_t ell_b_desc(uint32_t addr) {
    return smem_desc(addr, 16, 256, 6);
}
// kind::f16, FP32 accumulator, A MN-major (bit 15), B K-major, N = 16, M = 128.
__device__ __forceinline__ uint32_t ell_idesc(uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | (1u << 15) | ((16u >> 3) << 17) |
           ((128u >> 4) << 24);
}

// One warp per block row: 32 slots per step, ascending order checked
// against the previous slot (a shuffle, and the last slot of the step before).
// words (when given): two words, zero between calls; each block ORs its
// finding into words[0] and takes a ticket from words[1], and the last
// block stores the call's status (0 or the pattern error) and zeroes both
// words, so that no memset has to clear the status before the launch.
// Without words the status must be zero already and only errors are set.
__global__ void ell_validate_kernel(const int32_t *cols, int32_t mb, int32_t E, int32_t kb,
                                    int32_t *status, int32_t *words) {
    pdl_enter();
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    bool bad = false;
    if (r < mb) {
        const int32_t *c = cols + r * E;
        int32_t carry = -1;          // the previous slot's value (-1 before the first)
        for (int32_t e0 = 0; e0 < E; e0 += 32) {
            const int32_t v = e0 + lane < E ? __ldg(c + e0 + lane) : -1;
            int32_t prev = __shfl_up_sync(0xffffffffu, v, 1);
            if (lane == 0) prev = carry;
            const bool in = e0 + lane < E;
            // a block must follow a block with a smaller column; padding is -1 only
            bad |= in && (v < -1 || v >= kb || (v >= 0 && (e0 + lane > 0) && prev >= v) ||
                          (v >= 0 && e0 + lane > 0 && prev == -1));
            carry = __shfl_sync(0xffffffffu, v, 31);
        }
    }
    const bool warp_bad = __any_sync(0xffffffffu, bad);
    if (!words) {
        if (warp_bad && lane == 0) atomicCAS(status, 0, (int32_t)kDevPattern);
        return;
    }
    __shared__ int blk_bad;
    if (threadIdx.x == 0) blk_bad = 0;
    __syncthreads();
    if (warp_bad && lane == 0) atomicOr(&blk_bad, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (blk_bad) atomicOr(&words[0], 1);
        __threadfence();
        if (atomicAdd(&words[1], 1) == (int)gridDim.x - 1) {
            __threadfence();
            const int any_bad = atomicExch(&words[0], 0);
            *status = any_bad ? (int32_t)kDevPattern : 0;
            words[1] = 0;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kEllThreads, kEllCtasPerSm)
    ell_kernel(const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_w,
               const EllArgs args) {
    pdl_enter();
    if (*args.status != 0) return;                  // a rejected pattern writes nothing
    extern __shared__ __align__(1024) uint8_t sm_raw[];
    uint8_t *stages = (uint8_t *)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
    EllSmem *sm = reinterpret_cast<EllSmem *>(stages + kEllStages * kEllStageBytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ub = (int64_t)blockIdx.x * args.units / gridDim.x;
    const int64_t ue = (int64_t)(blockIdx.x + 1) * args.units / gridDim.x;
    if (ub >= ue) return;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kEllStages; ++s) {
            mbar_init(&sm->full[s], 1);
            mbar_init(&sm->empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&sm->accf[a], 1);
            mbar_init(&sm->acce[a], 128);
        }
        mbar_init(&sm->drain, 1);
        sm->abort_flag = 0;
        for (int i = 0; i < 4; ++i) sm->issued[i] = 0;
        sm->consumed = 0;
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
    const int32_t mb = args.mb, E = args.E;   // E >= 1 (the host handles width 0)

    if (warp == 0 || warp >= 6) {
        // ---- producers: lanes 0..3 copy the stage's X slabs, lane 4 its blocks;
        // producer j (warp 0, then warps 6, 7, ...) fills the stages it with
        // it % kEllProducers == j.  The first 64 slots of the next unit's row
        // are loaded while this unit's copies are issued (slot lane and
        // 32 + lane in c0 / c1).
        const int pid = warp == 0 ? 0 : warp - 5;
        int32_t mine = 0;
        const int32_t *rn = args.cols + (int64_t)(ub % mb) * E;
        int32_t n0c = lane < E ? __ldg(rn + lane) : -1;
        int32_t n1c = 32 + lane < E ? __ldg(rn + 32 + lane) : -1;
        int32_t it = 0;
        bool ok = true;
        for (int64_t u = ub; u < ue && ok; ++u) {
            const int32_t r = (int32_t)(u % mb);
            const int n0 = (int)(u / mb) * 128;
            const int32_t *rc = args.cols + (int64_t)r * E;
            const int32_t c0 = n0c, c1 = n1c;
            if (u + 1 < ue) {
                rn = args.cols + (int64_t)((u + 1) % mb) * E;
                n0c = lane < E ? __ldg(rn + lane) : -1;
                n1c = 32 + lane < E ? __ldg(rn + 32 + lane) : -1;
            }
            // valid slots form a prefix of the row (validated)
            int32_t nvalid = __popc(__ballot_sync(0xffffffffu, c0 >= 0)) +
                             __popc(__ballot_sync(0xffffffffu, c1 >= 0));
            for (int32_t e0 = 64; e0 < E && nvalid == e0; e0 += 32) {
                const bool v = e0 + lane < E && __ldg(rc + e0 + lane) >= 0;
                nvalid += __popc(__ballot_sync(0xffffffffu, v));
            }
            const int32_t nst = nvalid > 0 ? (nvalid + kEllSlots - 1) / kEllSlots : 1;
            for (int32_t st = 0; st < nst; ++st, ++it) {
                if (it % kEllProducers != pid) continue;
                const int s = it % kEllStages;
                const uint32_t ph = (uint32_t)((it / kEllStages) & 1);
                if (!ell_wait_warp(&sm->empty[s], ph ^ 1u, sm, lane)) {
                    if (lane == 0) ell_abort(sm, args.status);
                    ok = false;
                    break;
                }
                mine = it + 1;
                const int32_t e0 = st * kEllSlots;
                const int nv = min(kEllSlots, nvalid - e0);
                // column of slot e0 + lane (lanes below nv use it)
                const int32_t e = e0 + (lane & (kEllSlots - 1));
                const int32_t ca = __shfl_sync(0xffffffffu, c0, e & 31);
                const int32_t cb = __shfl_sync(0xffffffffu, c1, e & 31);
                uint8_t *base = stages + s * kEllStageBytes;
                if (lane == 0) {
                    sm->mask[s] = (nv > 0 ? (1u << nv) - 1u : 0u) | (st == nst - 1 ? 0x100u : 0u);
                    mbar_arrive_tx(&sm->full[s], nv > 0 ? nv * kEllSlab + kEllSlots * kEllBlock : 0);
                }
                __syncwarp();
                if (lane < nv) {
                    const int32_t c = e < 32 ? ca : (e < 64 ? cb : __ldg(rc + e));
                    uint8_t *slab = base + lane * kEllSlab;
                    if (args.x3d) {
                        tma_load_3d(slab, &map_x, 0, c * kSlabRows, n0 / kSlabHalf, &sm->full[s]);
                    } else {
                        tma_load_2d(slab, &map_x, n0, c * kSlabRows, &sm->full[s]);
                        tma_load_2d(slab + kEllSlab / 2, &map_x, n0 + kSlabHalf, c * kSlabRows,
                                    &sm->full[s]);
                    }
                } else if (lane == kEllSlots && nv > 0) {
                    tma_load_2d(base + kEllSlots * kEllSlab, &map_w, 0,
                                (int)(((int64_t)r * E + e0) * 16), &sm->full[s]);
                }
                __syncwarp();
            }
        }
        if (lane == 0) sm->issued[pid] = mine;
    } else if (warp == 1) {
        // ---- MMA issuer
        const uint32_t idesc = ell_idesc((uint32_t)args.fmt);
        int32_t it = 0;
        bool ok = true;
        for (int64_t u = ub, lu = 0; u < ue && ok; ++u, ++lu) {
            const uint32_t a = (uint32_t)(lu & 1), aph = (uint32_t)((lu >> 1) & 1);
            if (!ell_wait_warp(&sm->acce[a], aph ^ 1u, sm, lane)) {
                if (lane == 0) ell_abort(sm, args.status);
                break;
            }
            tc_fence_after();
            const uint32_t d = tmem + a * 16;
            bool started = false;
            while (true) {
                const int s = it % kEllStages;
                const uint32_t ph = (uint32_t)((it / kEllStages) & 1);
                if (!ell_wait_warp(&sm->full[s], ph, sm, lane)) {
                    if (lane == 0) ell_abort(sm, args.status);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t mk = sm->mask[s];
                const uint32_t base = smem_u32(stages + s * kEllStageBytes);
#pragma unroll
                for (int q = 0; q < kEllSlots; ++q) {
                    if (mk & (1u << q)) {
                        tc_mma_elect(d, ell_a_desc(base + q * kEllSlab),
                                     ell_b_desc(base + kEllSlots * kEllSlab + q * kEllBlock), idesc,
                                     started ? 1u : 0u);
                        started = true;
                    }
                }
                __syncwarp();
                if (lane == 0) tc_commit(&sm->empty[s]);
                ++it;
                if (mk & 0x100u) break;
            }
            if (!ok) break;
            __syncwarp();
            if (lane == 0) {
                if (started) tc_commit(&sm->accf[a]);
                else mbar_arrive(&sm->accf[a]);   // a row without blocks: nothing accumulated
            }
        }
        if (lane == 0) sm->consumed = it;
    } else {
        // ---- epilogue: lane = one of the unit's 128 columns of n
        const int q = warp & 3;
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        T *Y = reinterpret_cast<T *>(args.Y);
        for (int64_t u = ub, lu = 0; u < ue; ++u, ++lu) {
            const uint32_t a = (uint32_t)(lu & 1), aph = (uint32_t)((lu >> 1) & 1);
            if (!ell_wait_warp(&sm->accf[a], aph, sm, lane)) {
                if (lane == 0) ell_abort(sm, args.status);
                break;
            }
            tc_fence_after();
            const int32_t r = (int32_t)(u % mb);
            const int64_t col = (u / mb) * 128 + q * 32 + lane;
            float v[16];
            tmem_ld16(tmem + lane_addr + a * 16, v);
            // valid slots form a prefix, so a row has blocks iff its first slot is one
            const bool zero = __ldg(args.cols + (int64_t)r * E) < 0;
            if (col < args.n) {
                T *y = Y + (int64_t)r * 16 * args.ldy + col;
#pragma unroll
                for (int i = 0; i < 16; ++i) y[i * args.ldy] = Cvt<T>::f(zero ? 0.f : v[i]);
            }
            tc_fence_before();
            mbar_arrive(&sm->acce[a]);
        }
    }

    __syncthreads();
    if (sm->abort_flag) {
        if (threadIdx.x == 0) {
            int32_t hi = 0;
            for (int i = 0; i < kEllProducers; ++i) hi = max(hi, sm->issued[i]);
            for (int32_t c = sm->consumed; c < hi; ++c) {
                if (c >= sm->issued[c % kEllProducers]) continue;
                const int s = c % kEllStages;
                const uint32_t par = (uint32_t)((c / kEllStages) & 1);
                const unsigned long long t0 = gtimer();
                while (!mbar_try(&sm->full[s], par) && gtimer() - t0 < kEllWaitNs) {
                }
            }
        }
        if (warp == 1) {
            if (lane == 0) {
                tc_commit(&sm->drain);
                const unsigned long long t0 = gtimer();
                while (!mbar_try(&sm->drain, 0) && gtimer() - t0 < kEllWaitNs) {
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

// The values seen as (mb * E * 16) rows of 16 elements; one box = the
// kEllSlots blocks of a stage, 32-byte swizzled (the MMA's K-major B layout).
cudaError_t encode_w(CUtensorMap *map, bool bf16, const void *values, int64_t blocks) {
    auto enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {16, (cuuint64_t)(blocks * 16)};
    const cuuint64_t strides[1] = {32};
    const cuuint32_t box[2] = {16, (cuuint32_t)(kEllSlots * 16)};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                           2, const_cast<void *>(values), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_ell_t(const CUtensorMap &mx, const CUtensorMap &mw, const EllArgs &a, int sms,
                         cudaStream_t s) {
    const size_t smem = 1024 + (size_t)kEllStages * kEllStageBytes + sizeof(EllSmem);
    // all of the unified L1 / shared memory as shared: three CTAs per SM
    static std::atomic<uint64_t> attrs{0};
    const cudaError_t e = set_smem_attrs_once(attrs, ell_kernel<T>, (int)smem, true);
    if (e != cudaSuccess) return e;
    const int per_sm = kEllCtasPerSm;
    const int64_t slots = (int64_t)sms * per_sm;
    const int grid = (int)(a.units < slots ? a.units : slots);
    pdl_launch(ell_kernel<T>, dim3(grid), dim3(kEllThreads), smem, s, mx, mw, a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ell(spmm_plan *p, const int32_t *d_cols, int32_t E, const void *d_values,
                       const void *d_X, int64_t n, int64_t ldx, void *d_Y, int64_t ldy,
                       cudaStream_t s) {
    const bool bf16 = p->xdt == SPMM_BF16;
    const int32_t mb = (int32_t)(p->m / 16), kb = (int32_t)(p->k / 16);
    // the status word is written by the validation launch itself (its last
    // block) through two words of the fused re-partition's barrier area,
    // which stay zero between calls; plans without that area clear the
    // status first
    int32_t *words = p->dyn.bar ? p->dyn.bar + 2 : nullptr;
    cudaError_t e = cudaSuccess;
    if (!words) {
        e = cudaMemsetAsync(p->d_status, 0, sizeof(int32_t), s);
    } else if (!p->dyn.ell_clean) {
        e = cudaMemsetAsync(words, 0, 2 * sizeof(int32_t), s);
        p->dyn.ell_clean = true;
    }
    if (e != cudaSuccess) return e;
    pdl_launch(ell_validate_kernel, dim3((unsigned)((mb + 7) / 8)), dim3(256), 0, s, d_cols, mb, E,
               kb, p->d_status, words);
    e = cudaGetLastError();
    if (e != cudaSuccess || n == 0 || p->m == 0) return e;
    if (E == 0)   // no blocks at all: Y = 0
        return cudaMemset2DAsync(d_Y, (size_t)ldy * 2, 0, (size_t)n * 2, (size_t)p->m, s);
    CUtensorMap mx, mw;
    EllArgs a{};
    e = encode_x(&mx, &a.x3d, bf16, d_X, p->k, n, ldx);
    if (e == cudaSuccess) e = encode_w(&mw, bf16, d_values, (int64_t)mb * E);
    if (e != cudaSuccess) return e;
    a.cols = d_cols;
    a.Y = d_Y;
    a.status = p->d_status;
    a.ldy = ldy;
    a.n = n;
    a.mb = mb;
    a.E = E;
    a.ntn = (int32_t)((n + 127) / 128);
    a.fmt = bf16 ? 1 : 0;
    a.units = (int64_t)mb * a.ntn;
    return bf16 ? launch_ell_t<__nv_bfloat16>(mx, mw, a, p->sm_count, s)
                : launch_ell_t<__half>(mx, mw, a, p->sm_count, s);
}

}  // namespace spmm
