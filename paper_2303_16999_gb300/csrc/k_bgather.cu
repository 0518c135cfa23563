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
#include <atomic>

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

// (a0, a1) += w (x0, x1), each lane's FMA rounded as a scalar fmaf would be:
// one packed FP32 FMA for the pair.
__device__ __forceinline__ void fma2_rn(float &a0, float &a1, float w, float x0, float x1) {
    unsigned long long av, wv, xv, d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(av) : "f"(a0), "f"(a1));
    asm("mov.b64 %0, {%1, %1};" : "=l"(wv) : "f"(w));
    asm("mov.b64 %0, {%1, %2};" : "=l"(xv) : "f"(x0), "f"(x1));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(wv), "l"(xv), "l"(av));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a0), "=f"(a1) : "l"(d));
}

// (a.x s, a.y s), each product rounded to nearest as a scalar multiply
// would be: one packed FP32 multiply for the pair.
__device__ __forceinline__ float2 mul2_rn(float2 a, float s) {
    unsigned long long av, sv, d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(av) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %1};" : "=l"(sv) : "f"(s));
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(av), "l"(sv));
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(d));
    return r;
}

// Four E4M3 codes (one 32-bit word, lowest byte first) -> floats x scale.
__device__ __forceinline__ void e4m3x4(uint32_t w, float sc, float *o) {
    const __half2_raw h01 = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xFFFFu), __NV_E4M3);
    const __half2_raw h23 = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3);
    const float2 a = mul2_rn(__half22float2(*reinterpret_cast<const __half2 *>(&h01)), sc);
    const float2 b = mul2_rn(__half22float2(*reinterpret_cast<const __half2 *>(&h23)), sc);
    o[0] = a.x;
    o[1] = a.y;
    o[2] = b.x;
    o[3] = b.y;
}

// A 16-byte shared-memory read kept in program order (an asm volatile: the
// compiler must not hoist a block's 16 rows of X reads ahead of their use,
// which would hold them all in registers at once).
__device__ __forceinline__ uint4 lds128(const uint8_t *p) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"((uint32_t)__cvta_generic_to_shared(p)));
    return v;
}

// Asynchronous global -> shared copies (cp.async): the bytes land in shared
// memory without passing through registers, so a warp keeps several rounds
// of W rows and X rows in flight at no register cost.
__device__ __forceinline__ uint32_t saddr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
template <int N>
__device__ __forceinline__ void cp_async(void *dst, const void *src) {
    if constexpr (N == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr(dst)), "l"(src)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(saddr(dst)), "l"(src),
                     "n"(N)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
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

// The first NC 16-bit values of an X row slot -> floats.
template <typename T, int NC>
__device__ __forceinline__ void unpack_row(const uint8_t *slot, float *x) {
    if constexpr (NC >= 8) {
#pragma unroll
        for (int v = 0; v < NC / 8; ++v) unpack8<T>(lds128(slot + 16 * v), x + 8 * v);
    } else if constexpr (NC == 4) {
        const uint2 u = *reinterpret_cast<const uint2 *>(slot);
        const float2 a = Cv<T>::f2(u.x), b = Cv<T>::f2(u.y);
        x[0] = a.x, x[1] = a.y, x[2] = b.x, x[3] = b.y;
    } else if constexpr (NC == 2) {
        const float2 a = Cv<T>::f2(*reinterpret_cast<const uint32_t *>(slot));
        x[0] = a.x, x[1] = a.y;
    } else {
        x[0] = Cv<T>::f(*reinterpret_cast<const T *>(slot));
    }
}
// Shared memory: per warp a ring of kBgStages rounds.  One round holds the
// 32 X rows of the warp's blocks (block group g's row l at g * B + l, up to
// kBgMaxN 16-bit values, 32 bytes a row), each lane's W row (up to 32
// bytes) and each lane's block scale (E4M3).  After the main loop the ring
// holds the warp's FP32 partials (B x n).
constexpr int kBgStages = 4;
constexpr int kBgXBytes = 32 * 32;
constexpr int kBgWBytes = 32 * 32;
constexpr int kBgStageBytes = kBgXBytes + kBgWBytes + 32 * 4;
constexpr int kBgRingBytes = kBgStages * kBgStageBytes;
constexpr int kBgSmemBytes = kBgWarps * kBgRingBytes;
static_assert(kBgMaxN * 2 <= 32, "an X row fits its 32-byte slot");
static_assert(kBgRingBytes >= 16 * kBgMaxN * 4, "partials fit the ring");
static_assert(kBgStageBytes % 16 == 0 && kBgRingBytes % 16 == 0, "16-byte aligned stages");

// Raw bytes of one block row of W: B values of 16 bits (B / 2 words) or B
// E4M3 codes (B / 4 words), read back from the lane's shared-memory slot.
template <int B, bool W8> struct RawRow {
    static constexpr int kWords = W8 ? B / 4 : B / 2;
    uint32_t w[kWords];
};
template <int B, bool W8>
__device__ __forceinline__ void read_row(const uint8_t *slot, RawRow<B, W8> &r) {
    if constexpr (RawRow<B, W8>::kWords == 8) {
        const uint4 v0 = lds128(slot), v1 = lds128(slot + 16);
        r.w[0] = v0.x, r.w[1] = v0.y, r.w[2] = v0.z, r.w[3] = v0.w;
        r.w[4] = v1.x, r.w[5] = v1.y, r.w[6] = v1.z, r.w[7] = v1.w;
    } else if constexpr (RawRow<B, W8>::kWords == 4) {
        const uint4 v = lds128(slot);
        r.w[0] = v.x, r.w[1] = v.y, r.w[2] = v.z, r.w[3] = v.w;
    } else if constexpr (RawRow<B, W8>::kWords == 2) {
        const uint2 v = *reinterpret_cast<const uint2 *>(slot);
        r.w[0] = v.x, r.w[1] = v.y;
    } else {
        r.w[0] = *reinterpret_cast<const uint32_t *>(slot);
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

// Requests round u of a warp's share of a block row into ring stage
// u % kBgStages: lane (g, i) copies row i of block group g's W block (and
// its scale) and row i of the X rows that block multiplies.  X rows go by
// cp.async when they are 16-byte aligned, else by plain loads (n values,
// zero-filled to NC).  Called by the whole warp; always commits one group.
template <typename T, int B, bool W8, int NC>
__device__ __forceinline__ void bg_issue(const BgProb &P, int32_t q, int32_t end, int64_t col,
                                         uint8_t *st, int lane, int g, int i) {
    constexpr int WB = W8 ? B : 2 * B;             // bytes of one W row
    if (q < end) {
        const uint8_t *wsrc = P.vals + (int64_t)q * (B * B) * (W8 ? 1 : 2) + i * WB;
        uint8_t *wdst = st + kBgXBytes + lane * 32;
        if constexpr (WB == 32) {
            cp_async<16>(wdst, wsrc);
            cp_async<16>(wdst + 16, wsrc + 16);
        } else {
            cp_async<WB>(wdst, wsrc);
        }
        if (W8) cp_async<4>(st + kBgXBytes + kBgWBytes + lane * 4, P.scales + q);
        const T *xsrc = reinterpret_cast<const T *>(P.X) + (col * B + i) * P.ldx;
        uint8_t *xdst = st + (g * B + i) * 32;
        if (P.xvec) {
            // NC values (at least 4 bytes); the row is 16-byte aligned and
            // its first value is in range, so the piece stays in bounds
            if constexpr (NC >= 8) {
#pragma unroll
                for (int v = 0; v < NC / 8; ++v) cp_async<16>(xdst + 16 * v, xsrc + 8 * v);
            } else {
                cp_async<(NC * 2 > 4 ? NC * 2 : 4)>(xdst, xsrc);
            }
        } else {
            uint16_t *d = reinterpret_cast<uint16_t *>(xdst);
            for (int j = 0; j < NC; ++j) d[j] = j < P.n ? (uint16_t)Cv<T>::bits(xsrc[j]) : 0;
        }
    }
    cp_async_commit();
}

// Block row r of problem P, this warp's share `part` of its wpr warps.
// NC: columns kept per lane (n rounded up to 1, 2, 4, 8 or 16).
// The warp's blocks are taken in rounds of NB (one per block group); the
// column indices of 32 / NB rounds come in one coalesced load (the next
// batch's is requested one batch ahead), and kBgStages rounds of W rows and
// X rows are in flight while the oldest one is multiplied.
template <typename T, int B, bool W8, int NC>
__device__ __forceinline__ void bg_row(const BgProb &P, int32_t r, int part, uint8_t *ring) {
    constexpr int NB = 32 / B;                      // blocks per warp round
    constexpr int RB = 32 / NB;                     // rounds per column batch
    const int lane = threadIdx.x & 31;
    const int i = lane % B, g = lane / B;
    float acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.f;
    const int32_t beg = (r < P.mb) ? P.row_ptr[r] : 0;
    const int32_t end = (r < P.mb) ? P.row_ptr[r + 1] : 0;
    const int32_t first = beg + part * NB;          // slot of round 0, block group 0
    const int32_t stride = P.wpr * NB;              // slots between rounds
    const int32_t rounds = end > first ? (end - first + stride - 1) / stride : 0;
    // column of round (batch * RB + l / NB), block group l % NB, in lane l
    int32_t cols = 0, cols_next = 0;
    {
        const int32_t q0 = first + (lane / NB) * stride + lane % NB;
        const int32_t q1 = q0 + RB * stride;
        if (q0 < end) cols = P.col_idx[q0];
        if (q1 < end) cols_next = P.col_idx[q1];
    }
    int32_t u = 0;                                  // next round to request
    auto issue_next = [&]() {
        if (u < rounds) {
            if (u > 0 && u % RB == 0) {
                cols = cols_next;
                const int32_t q2 = first + (u + RB + lane / NB) * stride + lane % NB;
                cols_next = q2 < end ? P.col_idx[q2] : 0;
            }
            const int64_t col = __shfl_sync(0xffffffffu, cols, (u % RB) * NB + g);
            bg_issue<T, B, W8, NC>(P, first + u * stride + g, end, col,
                                   ring + (u % kBgStages) * kBgStageBytes, lane, g, i);
        } else {
            cp_async_commit();
        }
        ++u;
    };
#pragma unroll
    for (int s = 0; s < kBgStages; ++s) issue_next();
    for (int32_t t = 0; t < rounds; ++t) {
        cp_async_wait<kBgStages - 1>();             // this lane's copies of round t
        __syncwarp();                               // ... and every lane's
        const uint8_t *st = ring + (t % kBgStages) * kBgStageBytes;
        if (first + t * stride + g < end) {
            RawRow<B, W8> wr;
            read_row<B, W8>(st + kBgXBytes + lane * 32, wr);
            const float sc =
                W8 ? *reinterpret_cast<const float *>(st + kBgXBytes + kBgWBytes + lane * 4) : 1.f;
            float w[B];
            decode_row<T, B, W8>(wr, sc, w);
#pragma unroll
            for (int l = 0; l < B; ++l) {
                float x[NC];
                unpack_row<T, NC>(st + (g * B + l) * 32, x);
                if constexpr (NC == 1) {
                    acc[0] = fmaf(w[l], x[0], acc[0]);
                } else {
#pragma unroll
                    for (int c = 0; c < NC; c += 2) fma2_rn(acc[c], acc[c + 1], w[l], x[c], x[c + 1]);
                }
            }
        }
        __syncwarp();                               // stage t % S is free again
        issue_next();
    }
    cp_async_wait<0>();
    __syncwarp();
    // the warp's block groups: fixed butterfly over the lane bits above B
#pragma unroll
    for (int o = B; o < 32; o <<= 1) {
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    }
    float *part_out = reinterpret_cast<float *>(ring);   // B x n partials of this warp
    if (g == 0) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
            if (c < P.n) part_out[i * P.n + c] = acc[c];
    }
}

template <typename T, int B, bool W8>
__device__ __forceinline__ void bg_row_n(const BgProb &P, int32_t r, int part, uint8_t *ring) {
    if (P.n > 8) bg_row<T, B, W8, 16>(P, r, part, ring);
    else if (P.n > 4) bg_row<T, B, W8, 8>(P, r, part, ring);
    else if (P.n > 2) bg_row<T, B, W8, 4>(P, r, part, ring);
    else if (P.n > 1) bg_row<T, B, W8, 2>(P, r, part, ring);
    else bg_row<T, B, W8, 1>(P, r, part, ring);
}

template <typename T>
__global__ void __launch_bounds__(kBgThreads, 3) bgather_kernel(const __grid_constant__ BgBatch Bt) {
    pdl_enter();
    extern __shared__ __align__(128) uint8_t bg_smem[];
    const int warp = threadIdx.x >> 5;
    uint8_t *ring = bg_smem + warp * kBgRingBytes;
    for (int64_t u = blockIdx.x; u < Bt.total_units; u += gridDim.x) {
        int pi = 0;
        while (pi + 1 < Bt.nprob && Bt.prob[pi + 1].unit_base <= u) ++pi;
        const BgProb &P = Bt.prob[pi];
        const int rows = kBgWarps / P.wpr;              // block rows of this CTA
        const int32_t r = (int32_t)((u - P.unit_base) * rows) + warp / P.wpr;
        const int part = warp % P.wpr;
        if (P.w8) {
            switch (P.b) {
                case 16: bg_row_n<T, 16, true>(P, r, part, ring); break;
                case 8: bg_row_n<T, 8, true>(P, r, part, ring); break;
                default: bg_row_n<T, 4, true>(P, r, part, ring); break;
            }
        } else {
            switch (P.b) {
                case 16: bg_row_n<T, 16, false>(P, r, part, ring); break;
                case 8: bg_row_n<T, 8, false>(P, r, part, ring); break;
                default: bg_row_n<T, 4, false>(P, r, part, ring); break;
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
                sum += reinterpret_cast<const float *>(bg_smem + (rs * P.wpr + w) * kBgRingBytes)[k];
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
        // warps per block row: about one ring of rounds (of 32 / b blocks)
        // per warp, so a warp's whole share is requested at once, at most
        // the CTA's 8 warps
        const int64_t per_row = P.mb ? (p->nnzb + P.mb - 1) / P.mb : 0;
        const int64_t per_warp = kBgStages * (32 / p->b);
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
    if (plans[0]->xdt == SPMM_BF16) {
        static std::atomic<uint64_t> attrs{0};
        const cudaError_t e =
            set_smem_attrs_once(attrs, bgather_kernel<__nv_bfloat16>, kBgSmemBytes, false);
        if (e != cudaSuccess) return e;
        pdl_launch(bgather_kernel<__nv_bfloat16>, dim3(grid), dim3(kBgThreads), kBgSmemBytes, s,
                   Bt);
    } else {
        static std::atomic<uint64_t> attrs{0};
        const cudaError_t e = set_smem_attrs_once(attrs, bgather_kernel<__half>, kBgSmemBytes, false);
        if (e != cudaSuccess) return e;
        pdl_launch(bgather_kernel<__half>, dim3(grid), dim3(kBgThreads), kBgSmemBytes, s, Bt);
    }
    return cudaGetLastError();
}

cudaError_t launch_bgather(const spmm_plan *p, const void *X, int64_t n, int64_t ldx, void *Y,
                           int64_t ldy, cudaStream_t s) {
    spmm_plan *pp = const_cast<spmm_plan *>(p);
    return launch_bgather_batch(1, &pp, &X, &n, &ldx, &Y, &ldy, s);
}

}  // namespace spmm
