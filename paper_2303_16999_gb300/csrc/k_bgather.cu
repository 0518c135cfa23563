// CUDA-core block-sparse product for small n (the BGATHER kernel family):
// Y = W.X for W in b x b blocks, b in {4, 8, 16}, with at most 16 columns
// of X (Section 3's product; the batched and served forms of the hot path
// run many such products with small n).
//
// At small n the tensor-core kernel's 16 x 16 tiles, 128-column MMA tiles
// and X slabs cost far more than the product: a block of 16 x 16 E4M3 values
// is 256 bytes, while the X slab it is multiplied with is 4 KB.  Here every
// block is read once from its CSR-order copy and multiplied on the CUDA
// cores with FP32 accumulation:
//   * a warp's lanes are (block group g, block row i): b lanes per block,
//     32 / b blocks at once; lane (g, i) owns row i of its block and every
//     column of Y, so each stored value is decoded once;
//   * the b rows of X a block needs are staged in the warp's shared memory
//     by the block's lanes (row i by lane i, 16-byte pieces) and read back
//     in 16-byte pieces, 8 columns per read, by all the block's lanes;
//   * wpr warps share a block row (1 to 8, chosen per problem from its
//     blocks per row) and a CTA of 8 warps takes 8 / wpr block rows;
//   * the block groups of a warp are summed by a fixed shuffle butterfly,
//     the warps of a row by thread in warp order, so the result does not
//     depend on how problems are batched together.
// E4M3 blocks are decoded and scaled in FP32 (decode(code) * scale, the
// oracle's value up to one FP32 rounding).  Outputs are rounded once to the
// 16-bit output type.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "pdl.cuh"
#include "spmm_internal.h"

namespace spmm {
namespace {

constexpr int kBgWarps = 8;
constexpr int kBgThreads = kBgWarps * 32;

struct BgProb {
    const int32_t *row_ptr, *col_idx;
    const uint8_t *vals;     // CSR-order blocks, b x b row-major (16-bit values or E4M3 codes)
    const float *scales;     // E4M3: CSR-order block scales
    const void *X;
    void *Y;
    int64_t ldx, ldy, unit_base;
    int32_t n, b, mb, w8, wpr, xvec;   // wpr: warps per block row; xvec: X rows 16-byte aligned
};

struct BgBatch {
    BgProb prob[kBgMaxBatch];
    int32_t nprob;
    int64_t total_units;
};
static_assert(sizeof(BgBatch) <= 32764, "kernel parameter space");

template <typename T> struct Cv;
template <> struct Cv<__half> {
    static __device__ __forceinline__ uint32_t bits(__half v) { return __half_as_ushort(v); }
    static __device__ __forceinline__ float f(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half t(float v) { return __float2half_rn(v); }
    static __device__ __forceinline__ float2 f2(uint32_t w) {
        return __half22float2(*reinterpret_cast<const __half2 *>(&w));
    }
};
template <> struct Cv<__nv_bfloat16> {
    static __device__ __forceinline__ uint32_t bits(__nv_bfloat16 v) { return __bfloat16_as_ushort(v); }
    static __device__ __forceinline__ float f(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 t(float v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ float2 f2(uint32_t w) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w));
    }
};

// Four E4M3 codes (one 32-bit word, lowest byte first) -> floats x scale.
__device__ __forceinline__ void e4m3x4(uint32_t w, float sc, float *o) {
    const __half2_raw h01 = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xFFFFu), __NV_E4M3);
    const __half2_raw h23 = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3);
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&h01));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&h23));
    o[0] = a.x * sc;
    o[1] = a.y * sc;
    o[2] = b.x * sc;
    o[3] = b.y * sc;
}

// A 16-byte shared-memory read kept in program order (an asm volatile: the
// compiler must not hoist a block's 16 rows of X reads ahead of their use,
// which would hold them all in registers at once).
__device__ __forceinline__ uint4 lds128(const uint4 *p) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"((uint32_t)__cvta_generic_to_shared(p)));
    return v;
}

// 8 consecutive 16-bit values (one 16-byte piece) -> floats.
template <typename T>
__device__ __forceinline__ void unpack8(const uint4 v, float *x) {
    const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 f = Cv<T>::f2(u[k]);
        x[2 * k] = f.x;
        x[2 * k + 1] = f.y;
    }
}

// Shared memory: per warp, 32 staged X rows of up to kBgMaxN 16-bit values
// (block group g's row l at g * B + l), reused after the main loop for the
// warps' FP32 partials (B x n per warp).
constexpr int kBgStageBytes = 32 * kBgMaxN * 2;
static_assert(kBgStageBytes >= 16 * kBgMaxN * 4, "partials fit the staging area");

// Raw bytes of one block row of W: B values of 16 bits (B / 2 words) or B
// E4M3 codes (B / 4 words).
template <int B, bool W8> struct RawRow {
    static constexpr int kWords = W8 ? B / 4 : B / 2;
    uint32_t w[kWords];
};
template <int B, bool W8>
__device__ __forceinline__ void fetch_row(const BgProb &P, int64_t q, int i, RawRow<B, W8> &r) {
    const uint8_t *src = P.vals + (q * (B * B) + i * B) * (W8 ? 1 : 2);
    if constexpr (RawRow<B, W8>::kWords == 8) {
        const uint4 v0 = *reinterpret_cast<const uint4 *>(src);
        const uint4 v1 = *reinterpret_cast<const uint4 *>(src + 16);
        r.w[0] = v0.x, r.w[1] = v0.y, r.w[2] = v0.z, r.w[3] = v0.w;
        r.w[4] = v1.x, r.w[5] = v1.y, r.w[6] = v1.z, r.w[7] = v1.w;
    } else if constexpr (RawRow<B, W8>::kWords == 4) {
        const uint4 v = *reinterpret_cast<const uint4 *>(src);
        r.w[0] = v.x, r.w[1] = v.y, r.w[2] = v.z, r.w[3] = v.w;
    } else if constexpr (RawRow<B, W8>::kWords == 2) {
        const uint2 v = *reinterpret_cast<const uint2 *>(src);
        r.w[0] = v.x, r.w[1] = v.y;
    } else {
        r.w[0] = *reinterpret_cast<const uint32_t *>(src);
    }
}
template <typename T, int B, bool W8>
__device__ __forceinline__ void decode_row(const RawRow<B, W8> &r, float sc, float *w) {
    if constexpr (W8) {
#pragma unroll
        for (int k = 0; k < B / 4; ++k) e4m3x4(r.w[k], sc, w + 4 * k);
    } else {
#pragma unroll
        for (int k = 0; k < B / 2; ++k) {
            const float2 f = Cv<T>::f2(r.w[k]);
            w[2 * k] = f.x;
            w[2 * k + 1] = f.y;
        }
    }
}

// Block row r of problem P, this warp's share `part` of its wpr warps.
// NC: columns kept per lane (n rounded up to a multiple of 8, at most 16).
// The warp's blocks are taken in rounds of NB (one per block group); the
// column indices of 32 / NB rounds come in one coalesced load, so a round's
// W row and X rows are requested together.
template <typename T, int B, bool W8, int NC>
__device__ __forceinline__ void bg_row(const BgProb &P, int32_t r, int part, uint8_t *stage) {
    constexpr int NB = 32 / B;                      // blocks per warp round
    constexpr int NV = NC / 8;                      // 16-byte pieces of an X row
    const int lane = threadIdx.x & 31;
    const int i = lane % B, g = lane / B;
    const int n = P.n;
    uint4 *srow = reinterpret_cast<uint4 *>(stage) + (g * B + i) * (kBgMaxN / 8);
    const uint4 *sblk = reinterpret_cast<const uint4 *>(stage) + (g * B) * (kBgMaxN / 8);
    float acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.f;
    const int32_t beg = (r < P.mb) ? P.row_ptr[r] : 0;
    const int32_t end = (r < P.mb) ? P.row_ptr[r + 1] : 0;
    const int32_t first = beg + part * NB;          // slot of round 0, block group 0
    const int32_t stride = P.wpr * NB;              // slots between rounds
    const int32_t rounds = end > first ? (end - first + stride - 1) / stride : 0;
    for (int32_t t0 = 0; t0 < rounds; t0 += 32 / NB) {
        // column of round t0 + l / NB, block group l % NB, in lane l
        int32_t cols;
        {
            const int32_t q = first + (t0 + lane / NB) * stride + lane % NB;
            cols = q < end ? P.col_idx[q] : 0;
        }
        const int32_t tn = min(rounds - t0, 32 / NB);
        for (int32_t u = 0; u < tn; ++u) {
            const int32_t q = first + (t0 + u) * stride + g;
            const int64_t col = __shfl_sync(0xffffffffu, cols, u * NB + g);
            const bool ok = q < end;
            RawRow<B, W8> wr;
            float sc = 1.f;
            if (ok) {
                fetch_row<B, W8>(P, q, i, wr);
                if (W8) sc = P.scales[q];
                const T *src = reinterpret_cast<const T *>(P.X) + (col * B + i) * P.ldx;
                if (P.xvec) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) srow[v] = reinterpret_cast<const uint4 *>(src)[v];
                } else {
                    uint16_t *dst = reinterpret_cast<uint16_t *>(srow);
                    for (int j = 0; j < NC; ++j) dst[j] = j < n ? (uint16_t)Cv<T>::bits(src[j]) : 0;
                }
            }
            __syncwarp();
            if (ok) {
                float w[B];
                decode_row<T, B, W8>(wr, sc, w);
#pragma unroll
                for (int l = 0; l < B; ++l) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        float x[8];
                        unpack8<T>(lds128(sblk + l * (kBgMaxN / 8) + v), x);
#pragma unroll
                        for (int e = 0; e < 8; ++e) acc[v * 8 + e] = fmaf(w[l], x[e], acc[v * 8 + e]);
                    }
                }
            }
            __syncwarp();
        }
    }
    // the warp's block groups: fixed butterfly over the lane bits above B
#pragma unroll
    for (int o = B; o < 32; o <<= 1) {
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    }
    __syncwarp();
    float *part_out = reinterpret_cast<float *>(stage);   // B x n partials of this warp
    if (g == 0) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
            if (c < n) part_out[i * n + c] = acc[c];
    }
}

template <typename T, int B, bool W8>
__device__ __forceinline__ void bg_row_n(const BgProb &P, int32_t r, int part, uint8_t *stage) {
    if (P.n > 8) bg_row<T, B, W8, 16>(P, r, part, stage);
    else bg_row<T, B, W8, 8>(P, r, part, stage);
}

template <typename T>
__global__ void __launch_bounds__(kBgThreads, 3) bgather_kernel(const __grid_constant__ BgBatch Bt) {
    pdl_enter();
    __shared__ __align__(16) uint8_t stage_all[kBgWarps * kBgStageBytes];
    const int warp = threadIdx.x >> 5;
    uint8_t *stage = stage_all + warp * kBgStageBytes;
    for (int64_t u = blockIdx.x; u < Bt.total_units; u += gridDim.x) {
        int pi = 0;
        while (pi + 1 < Bt.nprob && Bt.prob[pi + 1].unit_base <= u) ++pi;
        const BgProb &P = Bt.prob[pi];
        const int rows = kBgWarps / P.wpr;              // block rows of this CTA
        const int32_t r = (int32_t)((u - P.unit_base) * rows) + warp / P.wpr;
        const int part = warp % P.wpr;
        if (P.w8) {
            switch (P.b) {
                case 16: bg_row_n<T, 16, true>(P, r, part, stage); break;
                case 8: bg_row_n<T, 8, true>(P, r, part, stage); break;
                default: bg_row_n<T, 4, true>(P, r, part, stage); break;
            }
        } else {
            switch (P.b) {
                case 16: bg_row_n<T, 16, false>(P, r, part, stage); break;
                case 8: bg_row_n<T, 8, false>(P, r, part, stage); break;
                default: bg_row_n<T, 4, false>(P, r, part, stage); break;
            }
        }
        __syncthreads();
        // each row's warps summed in warp order, rounded once
        T *Y = reinterpret_cast<T *>(P.Y);
        const int bn = P.b * P.n;
        for (int e = threadIdx.x; e < rows * bn; e += kBgThreads) {
            const int rs = e / bn, k = e - rs * bn;
            const int32_t rr = (int32_t)((u - P.unit_base) * rows) + rs;
            if (rr >= P.mb) continue;
            float sum = 0.f;
            for (int w = 0; w < P.wpr; ++w)
                sum += reinterpret_cast<const float *>(stage_all + (rs * P.wpr + w) * kBgStageBytes)[k];
            const int ii = k / P.n, jj = k - ii * P.n;
            Y[((int64_t)rr * P.b + ii) * P.ldy + jj] = Cv<T>::t(sum);
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_bgather_batch(int count, spmm_plan *const *plans, const void *const *X,
                                 const int64_t *n, const int64_t *ldx, void *const *Y,
                                 const int64_t *ldy, cudaStream_t s) {
    if (count <= 0 || count > kBgMaxBatch) return cudaErrorInvalidValue;
    BgBatch Bt;
    int64_t base = 0;
    int c = 0;
    for (int i = 0; i < count; ++i) {
        const spmm_plan *p = plans[i];
        if (n[i] == 0) continue;
        BgProb &P = Bt.prob[c++];
        P.row_ptr = p->d_row_ptr;
        P.col_idx = p->d_col_idx;
        P.vals = (const uint8_t *)p->d_packed;
        P.scales = p->d_tile_scale;
        P.X = X[i];
        P.Y = Y[i];
        P.ldx = ldx ? ldx[i] : n[i];
        P.ldy = ldy ? ldy[i] : n[i];
        P.unit_base = base;
        P.n = (int32_t)n[i];
        P.b = p->b;
        P.mb = (int32_t)(p->m / p->b);
        P.w8 = p->wdt == SPMM_E4M3 ? 1 : 0;
        // warps per block row: about two rounds (of 32 / b blocks) per
        // warp, at most the CTA's 8 warps (the rounds are latency-bound, so
        // more warps in flight beat longer warps)
        const int64_t per_row = P.mb ? (p->nnzb + P.mb - 1) / P.mb : 0;
        const int64_t per_warp = 2 * (32 / p->b);
        int wpr = 1;
        while (wpr < kBgWarps && per_row > (int64_t)wpr * per_warp) wpr <<= 1;
        P.wpr = wpr;
        P.xvec = ((uintptr_t)X[i] % 16 == 0 && (P.ldx * 2) % 16 == 0) ? 1 : 0;
        const int rows = kBgWarps / wpr;
        base += (P.mb + rows - 1) / rows;
    }
    if (c == 0 || base == 0) return cudaSuccess;
    Bt.nprob = c;
    Bt.total_units = base;
    const unsigned grid = (unsigned)(base < (1 << 30) ? base : (1 << 30));
    if (plans[0]->xdt == SPMM_BF16)
        pdl_launch(bgather_kernel<__nv_bfloat16>, dim3(grid), dim3(kBgThreads), 0, s, Bt);
    else
        pdl_launch(bgather_kernel<__half>, dim3(grid), dim3(kBgThreads), 0, s, Bt);
    return cudaGetLastError();
}

cudaError_t launch_bgather(const spmm_plan *p, const void *X, int64_t n, int64_t ldx, void *Y,
                           int64_t ldy, cudaStream_t s) {
    spmm_plan *pp = const_cast<spmm_plan *>(p);
    return launch_bgather_batch(1, &pp, &X, &n, &ldx, &Y, &ldy, s);
}

}  // namespace spmm
