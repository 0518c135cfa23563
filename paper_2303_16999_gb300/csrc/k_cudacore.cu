// CUDA-core kernels: value packing into CSR order, the plain FP32 kernel,
// the b = 1 gather kernel and the split-row reduction.
//
// Y[i, :] = sum over blocks (r, c) in block row r = i / b of
//           sum_l W_blk[i % b, l] * X[c*b + l, :]           (Section 3)
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "pdl.cuh"
#include "spmm_internal.h"

namespace spmm {
namespace {

// ------------------------------------------------------------- packing ----
// Static values are re-ordered once into CSR slot order (Section 3.2: the
// host-supplied values are re-ordered to match the fixed distribution).
template <typename U>
__global__ void pack_csr_kernel(const U *__restrict__ vals, const int32_t *__restrict__ perm,
                                int64_t nnzb, int b, int tr, const int32_t *__restrict__ nnzb_dev,
                                const int32_t *__restrict__ status, U *__restrict__ out) {
    pdl_enter();
    // dynamic plans: a rejected pattern leaves perm incomplete; pack nothing
    if (status && *status != 0) return;
    if (nnzb_dev) nnzb = min((int64_t)max(*nnzb_dev, 0), nnzb);
    const int bb = b * b;
    const int64_t total = nnzb * bb;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = t / bb, e = t - s * bb;
        // transposed plans: element (i, j) of the packed block is W's (j, i)
        const int64_t src = tr ? (e % b) * b + e / b : e;
        out[t] = vals[(int64_t)perm[s] * bb + src];
    }
}

// ------------------------------------------------------- plain FP32 ------
// One thread per (row i, column j); FP32 throughout.  The deliberately plain
// baseline kernel.
__global__ void plain_f32_kernel(const int32_t *__restrict__ row_ptr,
                                 const int32_t *__restrict__ col_idx,
                                 const float *__restrict__ vals, const float *__restrict__ X,
                                 int64_t ldx, float *__restrict__ Y, int64_t ldy, int64_t m,
                                 int64_t n, int b) {
    pdl_enter();
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    for (int64_t i = blockIdx.y; i < m; i += gridDim.y) {
        const int64_t r = i / b, ii = i - r * b;
        float acc = 0.f;
        for (int32_t s = row_ptr[r]; s < row_ptr[r + 1]; ++s) {
            const int64_t c = col_idx[s];
            const float *v = vals + ((int64_t)s * b + ii) * b;
            const float *x = X + c * b * ldx + j;
            for (int l = 0; l < b; ++l) acc = fmaf(v[l], x[l * ldx], acc);
        }
        Y[i * ldy + j] = acc;
    }
}

// ---------------------------------------------------------- b = 1 gather --
template <typename T> struct Vec;
template <> struct Vec<float> {
    static __device__ __forceinline__ float to_f(float v) { return v; }
    static __device__ __forceinline__ float from_f(float v) { return v; }
};
template <> struct Vec<__half> {
    static __device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half from_f(float v) { return __float2half_rn(v); }
};
template <> struct Vec<__nv_bfloat16> {
    static __device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 from_f(float v) { return __float2bfloat16_rn(v); }
};

// V elements of T per lane, loaded as one vector (16 B when V * sizeof(T) == 16).
template <typename T, int V> struct alignas(V * sizeof(T)) Pack {
    T v[V];
};

// One warp per (row item, column chunk).  Lanes form G = 32 / LN sub-groups
// along the row's non-zeros and LN lanes along n (V columns each).  Indices
// and values of 32 non-zeros are read coalesced once and broadcast by
// shuffles; every sub-group accumulates its share in FP32, and a butterfly
// of shuffles sums the sub-groups at the end (fixed order: deterministic).
template <typename T, int V>
__global__ void __launch_bounds__(256) gather_kernel(
    const int32_t *__restrict__ items, int64_t n_items, int nchunk, int LN,
    const int32_t *__restrict__ col_idx, const T *__restrict__ vals, const T *__restrict__ X,
    int64_t ldx, T *__restrict__ Y, int64_t ldy, int64_t n, float *__restrict__ ws,
    const int64_t *__restrict__ ws_row0, const int32_t *__restrict__ n_items_dev,
    const int32_t *__restrict__ status) {
    pdl_enter();
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (n_items_dev) {
        // dynamic plans: item count from the device; a rejected pattern writes nothing
        if (*status != 0) return;
        n_items = min(n_items, (int64_t)*n_items_dev);
    }
    if (wid >= n_items * nchunk) return;
    const int64_t item = wid / nchunk;
    const int chunk = (int)(wid - item * nchunk);
    const int32_t *it = items + item * kItemFields;
    const int32_t row = it[0], beg = it[1], end = it[2], slot = it[5];
    const int G = 32 / LN;
    const int sg = lane / LN;
    const int64_t c0 = (int64_t)chunk * LN * V + (int64_t)(lane % LN) * V;
    const bool active = c0 < n;
    float acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0.f;
    const T *xcol = X + (active ? c0 : 0);
    // kChunks chunks of 32 non-zeros per round: their indices and values are
    // requested together, so a warp keeps several loads in flight
    constexpr int kChunks = 8;
    __shared__ int2 stage_cw[8][kChunks * 32];   // per warp: (column, weight bits) of a round
    int2 *mine = stage_cw[threadIdx.x >> 5];
    for (int32_t base0 = beg; base0 < end; base0 += 32 * kChunks) {
        int32_t mycol[kChunks];
        float myw[kChunks];
#pragma unroll
        for (int q = 0; q < kChunks; ++q) {
            const int32_t idx = base0 + 32 * q + lane;
            mycol[q] = idx < end ? col_idx[idx] : 0;
            myw[q] = idx < end ? Vec<T>::to_f(vals[idx]) : 0.f;
        }
        // sub-groups of LN lanes share non-zeros: stage the round's (column,
        // weight) pairs in shared memory; sub-group sg takes non-zeros
        // j = sg, sg + G, ... of every chunk, eight X loads in flight per lane
        __syncwarp();
#pragma unroll
        for (int q = 0; q < kChunks; ++q) mine[q * 32 + lane] = make_int2(mycol[q], __float_as_int(myw[q]));
        __syncwarp();
        const int nround = min(32 * kChunks, end - base0);
        const int slots = (nround + G - 1) / G;   // non-zeros per sub-group this round
        for (int f0 = 0; f0 < slots; f0 += 8) {
            float ww[8];
            Pack<T, V> xv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = (f0 + u) * G + sg;
                const bool ok = f0 + u < slots && j < nround && active;
                const int2 cw = mine[ok ? j : 0];
                ww[u] = ok ? __int_as_float(cw.y) : 0.f;
                if (ok) {
                    xv[u] = *reinterpret_cast<const Pack<T, V> *>(xcol + (int64_t)cw.x * ldx);
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v) xv[u].v[v] = Vec<T>::from_f(0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] = fmaf(ww[u], Vec<T>::to_f(xv[u].v[v]), acc[v]);
        }
    }
    for (int off = LN; off < 32; off <<= 1)
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], off);
    if (sg != 0 || !active) return;
    if (slot >= 0) {
        float *dst = ws + ws_row0[slot] * n + c0;
#pragma unroll
        for (int v = 0; v < V; ++v) dst[v] = acc[v];
    } else {
        Pack<T, V> out;
#pragma unroll
        for (int v = 0; v < V; ++v) out.v[v] = Vec<T>::from_f(acc[v]);
        *reinterpret_cast<Pack<T, V> *>(Y + (int64_t)row * ldy + c0) = out;
    }
}

// n <= V (one vector per X row): the HBM-bound case, 4 + sizeof(T) bytes
// per non-zero.  Each warp streams the column indices and values of its
// items (rows or row chunks, taken with a grid stride) through a ring of
// kG1Stages chunks of 256 non-zeros in shared memory: every lane requests 8
// indices and 8 values per chunk with cp.async, so about kG1Stages chunks
// per warp are in flight without holding registers, and the stream runs on
// across item boundaries with no drain.  A chunk starts at a multiple of 8
// non-zeros (16-byte aligned indices and values); non-zeros outside the
// item are masked, and copies stop at the end of the arrays.  Each lane
// adds its own non-zeros in order and the lanes meet in a fixed butterfly
// (deterministic).  X (k x n, up to the shared memory the ring leaves: 79 KB
// of 16-bit values, 31 KB of FP32) is copied into shared memory once per CTA
// (by cp.async when its rows are contiguous), so the X gathers are
// shared-memory reads.
constexpr int kG1Stages = 6;                         // ring stages per warp (a 5-stage
                                                     // variant leaves X 16 KB more)
constexpr int kG1Warps = 16;
constexpr int kG1Chunk = 256;                        // non-zeros per chunk, 8 per lane
// one stage: the chunk's indices (I: int32, or the 16-bit copy of static
// plans), then its values
template <typename T, typename I> __host__ __device__ constexpr int g1_stage_bytes() {
    return kG1Chunk * ((int)sizeof(I) + (int)sizeof(T));
}
template <typename T, typename I, int S = kG1Stages>
__host__ __device__ constexpr int g1_ring_bytes() {
    return S * g1_stage_bytes<T, I>();
}

struct G1Meta {
    int32_t beg, end, row, slot, base, last, pad0, pad1;
};
template <int S = kG1Stages> __host__ __device__ constexpr int g1_meta_bytes() {
    return kG1Warps * S * (int)sizeof(G1Meta);
}
template <typename T, typename I, int S = kG1Stages>
__host__ __device__ constexpr int g1_fixed_smem() {
    return kG1Warps * g1_ring_bytes<T, I, S>() + g1_meta_bytes<S>();
}
// shared memory left for X (of the 227 KB a CTA may hold, 1 KB spare)
template <typename T, typename I, int S = kG1Stages>
__host__ __device__ constexpr int g1_x_budget() {
    return 226 * 1024 - g1_fixed_smem<T, I, S>();
}
static_assert(g1_x_budget<float, int32_t>() >= 16 * 1024, "room for X");

// cp.async of 16 bytes of which the first src_bytes come from src and the
// rest are zero-filled.
__device__ __forceinline__ void cp_async16_zfill(void *dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}

template <typename T, int V, typename I, int S>
__global__ void __launch_bounds__(kG1Warps * 32, 1) gather1_kernel(
    const int32_t *__restrict__ items, int64_t n_items, const I *__restrict__ col_idx,
    const T *__restrict__ vals, int64_t cap, const T *__restrict__ X, int64_t ldx, int64_t k,
    T *__restrict__ Y, int64_t ldy, float *__restrict__ ws, const int64_t *__restrict__ ws_row0,
    const int32_t *__restrict__ n_items_dev, const int32_t *__restrict__ status) {
    pdl_enter();
    constexpr int VB = 8 * (int)sizeof(T);          // value bytes per lane per chunk (16 or 32)
    constexpr int IB = 8 * (int)sizeof(I);          // index bytes per lane per chunk (16 or 32)
    constexpr int kStage = g1_stage_bytes<T, I>(), kRing = g1_ring_bytes<T, I, S>();
    extern __shared__ __align__(128) uint8_t g1_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (n_items_dev) {
        if (*status != 0) return;
        n_items = min(n_items, (int64_t)*n_items_dev);
    }
    uint8_t *ring = g1_smem + warp * kRing;
    G1Meta *meta = reinterpret_cast<G1Meta *>(g1_smem + kG1Warps * kRing) + warp * S;
    const int64_t W = (int64_t)gridDim.x * kG1Warps;
    // the item being requested (c_*) and the next one's header (x_*), read
    // one item ahead so the request stream never waits on a header
    int64_t it = (int64_t)blockIdx.x * kG1Warps + warp;
    int32_t c_beg = 0, c_end = 0, c_row = 0, c_slot = -1, c_pos = 0;
    int32_t x_beg = 0, x_end = 0, x_row = 0, x_slot = -1;
    if (it < n_items) {
        const int32_t *d = items + it * kItemFields;
        c_row = d[0], c_beg = d[1], c_end = d[2], c_slot = d[5];
        c_pos = c_beg & ~7;
    }
    if (it + W < n_items) {
        const int32_t *d = items + (it + W) * kItemFields;
        x_row = d[0], x_beg = d[1], x_end = d[2], x_slot = d[5];
    }
    // X first (its own cp.async group, so it can be waited for alone)
    T *xs = reinterpret_cast<T *>(g1_smem + g1_fixed_smem<T, I, S>());
    const int64_t xbytes = k * V * (int64_t)sizeof(T);
    const bool xbulk = ldx == V && ((uintptr_t)X % 16) == 0;
    if (xbulk) {
        const int64_t pieces = xbytes / 16;
        for (int64_t i = threadIdx.x; i < pieces; i += blockDim.x)
            cp_async16_zfill(reinterpret_cast<uint8_t *>(xs) + 16 * i,
                             reinterpret_cast<const uint8_t *>(X) + 16 * i, 16);
        for (int64_t i = pieces * 16 / (int64_t)sizeof(T) + threadIdx.x; i < k * V; i += blockDim.x)
            xs[i] = X[i];
    } else {
#pragma unroll 8
        for (int64_t i = threadIdx.x; i < k; i += blockDim.x)
            *reinterpret_cast<Pack<T, V> *>(xs + i * V) =
                *reinterpret_cast<const Pack<T, V> *>(X + i * ldx);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    int32_t issued = 0;
    int is = 0;                                       // ring stage of the next request
    const int32_t cap32 = (int32_t)min(cap, (int64_t)INT32_MAX);
    auto issue_next = [&]() {
        if (it < n_items) {
            const int s = is;
            is = is + 1 == S ? 0 : is + 1;
            uint8_t *st = ring + s * kStage;
            const int32_t pos = c_pos + 8 * lane;
            // entries of this lane's 8 that the arrays hold; the others lie
            // past every item's end and are masked, so nothing is read there
            const int ne = max(0, min(8, cap32 - pos));
            if (ne > 0) {
                const uint8_t *is_ = reinterpret_cast<const uint8_t *>(col_idx + pos);
                const int ibytes = ne * (int)sizeof(I);
                cp_async16_zfill(st + lane * IB, is_, min(ibytes, 16));
                if (IB == 32 && ibytes > 16) cp_async16_zfill(st + lane * IB + 16, is_ + 16, ibytes - 16);
                uint8_t *vd = st + kG1Chunk * (int)sizeof(I) + lane * VB;
                const uint8_t *vs = reinterpret_cast<const uint8_t *>(vals + pos);
                const int vbytes = ne * (int)sizeof(T);
                cp_async16_zfill(vd, vs, min(vbytes, 16));
                if (VB == 32 && vbytes > 16) cp_async16_zfill(vd + 16, vs + 16, vbytes - 16);
            }
            const bool last = c_pos + kG1Chunk >= c_end;
            if (lane == 0) meta[s] = G1Meta{c_beg, c_end, c_row, c_slot, c_pos, last ? 1 : 0, 0, 0};
            c_pos += kG1Chunk;
            if (last) {
                it += W;
                c_beg = x_beg, c_end = x_end, c_row = x_row, c_slot = x_slot;
                c_pos = c_beg & ~7;
                if (it + W < n_items) {
                    const int32_t *d = items + (it + W) * kItemFields;
                    x_row = d[0], x_beg = d[1], x_end = d[2], x_slot = d[5];
                }
            }
            ++issued;
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
#pragma unroll 1
    for (int q = 0; q < S; ++q) issue_next();
    // X landed (every thread's share), the ring's chunks may still be in flight
    asm volatile("cp.async.wait_group %0;" ::"n"(S) : "memory");
    __syncthreads();
    float acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0.f;
    int cs = 0;                                       // ring stage of chunk t
#pragma unroll 1
    for (int32_t t = 0; t < issued; ++t) {
        asm volatile("cp.async.wait_group %0;" ::"n"(S - 1) : "memory");
        __syncwarp();
        const uint8_t *st = ring + cs * kStage;
        const G1Meta m = meta[cs];
        cs = cs + 1 == S ? 0 : cs + 1;
        int32_t cq[8];
        if constexpr (sizeof(I) == 4) {
            const int4 c0 = *reinterpret_cast<const int4 *>(st + lane * IB);
            const int4 c1 = *reinterpret_cast<const int4 *>(st + lane * IB + 16);
            cq[0] = c0.x, cq[1] = c0.y, cq[2] = c0.z, cq[3] = c0.w;
            cq[4] = c1.x, cq[5] = c1.y, cq[6] = c1.z, cq[7] = c1.w;
        } else {
            const uint4 c = *reinterpret_cast<const uint4 *>(st + lane * IB);
            const uint32_t h[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                cq[2 * q] = (int32_t)(h[q] & 0xFFFFu);
                cq[2 * q + 1] = (int32_t)(h[q] >> 16);
            }
        }
        const Pack<T, 8> w =
            *reinterpret_cast<const Pack<T, 8> *>(st + kG1Chunk * (int)sizeof(I) + lane * VB);
        if (m.base >= m.beg && m.base + kG1Chunk <= m.end) {
            // a chunk wholly inside its item (all but an item's first and
            // last): no masks
            Pack<T, V> x[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) x[e] = *reinterpret_cast<const Pack<T, V> *>(xs + cq[e] * V);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const float wf = Vec<T>::to_f(w.v[e]);
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] = fmaf(wf, Vec<T>::to_f(x[e].v[v]), acc[v]);
            }
        } else {
            const int32_t p0 = m.base + 8 * lane;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                if (p0 + e >= m.beg && p0 + e < m.end) {
                    const Pack<T, V> x = *reinterpret_cast<const Pack<T, V> *>(xs + cq[e] * V);
                    const float wf = Vec<T>::to_f(w.v[e]);
#pragma unroll
                    for (int v = 0; v < V; ++v) acc[v] = fmaf(wf, Vec<T>::to_f(x.v[v]), acc[v]);
                }
            }
        }
        if (m.last) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], off);
            if (lane == 0) {
                if (m.slot >= 0) {
                    float *dst = ws + ws_row0[m.slot] * (int64_t)V;   // n == V here
#pragma unroll
                    for (int v = 0; v < V; ++v) dst[v] = acc[v];
                } else {
                    Pack<T, V> out;
#pragma unroll
                    for (int v = 0; v < V; ++v) out.v[v] = Vec<T>::from_f(acc[v]);
                    *reinterpret_cast<Pack<T, V> *>(Y + (int64_t)m.row * ldy) = out;
                }
            }
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = 0.f;
        }
        __syncwarp();                                 // stage s is free again
        issue_next();
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// n <= V with X too large for shared memory: the row's indices and values
// stream in as 16-byte / 8-byte vectors, four non-zeros per lane per load
// and kRounds loads per lane in flight, and every lane gathers the X rows of
// its own non-zeros from global memory (L2), up to 4 kRounds gathers in
// flight per lane.  The lanes' sums meet in a fixed butterfly
// (deterministic).
#ifndef SPMM_G1_ROUNDS
#define SPMM_G1_ROUNDS 4    // 16-byte index loads in flight per lane per pass
#endif
#ifndef SPMM_G1_BLOCKS
#define SPMM_G1_BLOCKS 2    // resident 512-thread blocks per SM (bounds registers)
#endif
template <typename T, int V>
__global__ void __launch_bounds__(512, SPMM_G1_BLOCKS) gather1g_kernel(
    const int32_t *__restrict__ items, int64_t n_items, const int32_t *__restrict__ col_idx,
    const T *__restrict__ vals, const T *__restrict__ X, int64_t ldx, T *__restrict__ Y,
    int64_t ldy, float *__restrict__ ws, const int64_t *__restrict__ ws_row0,
    const int32_t *__restrict__ n_items_dev, const int32_t *__restrict__ status) {
    pdl_enter();
    constexpr int kRounds = SPMM_G1_ROUNDS;   // kRounds x 4 non-zeros per lane per pass
    const int lane = threadIdx.x & 31;
    if (n_items_dev) {
        if (*status != 0) return;
        n_items = min(n_items, (int64_t)*n_items_dev);
    }
    const T *xb = X;
    const int64_t lx = ldx;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t item = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; item < n_items;
         item += nwarps) {
        const int32_t *it = items + item * kItemFields;
        const int32_t row = it[0], beg = it[1], end = it[2], slot = it[5];
        float acc[V];
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = 0.f;
        auto add = [&](int32_t c, float w) {
            const Pack<T, V> x = *reinterpret_cast<const Pack<T, V> *>(xb + (int64_t)c * lx);
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = fmaf(w, Vec<T>::to_f(x.v[v]), acc[v]);
        };
        // head up to a multiple of 4 (vector alignment), one non-zero per lane
        const int32_t h = min(end, (beg + 3) & ~3);
        if (beg + lane < h) add(col_idx[beg + lane], Vec<T>::to_f(vals[beg + lane]));
        // full passes: no bounds checks
        int32_t base = h;
        for (; base + 128 * kRounds <= end; base += 128 * kRounds) {
            int4 c[kRounds];
            Pack<T, 4> w[kRounds];
#pragma unroll
            for (int q = 0; q < kRounds; ++q) {
                const int32_t i0 = base + 128 * q + 4 * lane;
                c[q] = *reinterpret_cast<const int4 *>(col_idx + i0);
                w[q] = *reinterpret_cast<const Pack<T, 4> *>(vals + i0);
            }
#pragma unroll
            for (int q = 0; q < kRounds; ++q) {
                add(c[q].x, Vec<T>::to_f(w[q].v[0]));
                add(c[q].y, Vec<T>::to_f(w[q].v[1]));
                add(c[q].z, Vec<T>::to_f(w[q].v[2]));
                add(c[q].w, Vec<T>::to_f(w[q].v[3]));
            }
        }
        // the last partial pass
        for (; base < end; base += 128 * kRounds) {
            int4 c[kRounds];
            Pack<T, 4> w[kRounds];
#pragma unroll
            for (int q = 0; q < kRounds; ++q) {
                const int32_t i0 = base + 128 * q + 4 * lane;
                if (i0 + 3 < end) {
                    c[q] = *reinterpret_cast<const int4 *>(col_idx + i0);
                    w[q] = *reinterpret_cast<const Pack<T, 4> *>(vals + i0);
                } else {
                    c[q] = make_int4(i0 < end ? col_idx[i0] : 0, i0 + 1 < end ? col_idx[i0 + 1] : 0,
                                     i0 + 2 < end ? col_idx[i0 + 2] : 0, 0);
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        w[q].v[e] = i0 + e < end ? vals[i0 + e] : Vec<T>::from_f(0.f);
                }
            }
#pragma unroll
            for (int q = 0; q < kRounds; ++q) {
                const int32_t i0 = base + 128 * q + 4 * lane;
                const int32_t cq[4] = {c[q].x, c[q].y, c[q].z, c[q].w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (i0 + e < end) add(cq[e], Vec<T>::to_f(w[q].v[e]));
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], off);
        if (lane == 0) {
            if (slot >= 0) {
                float *dst = ws + ws_row0[slot] * (int64_t)V;   // n == V here
#pragma unroll
                for (int v = 0; v < V; ++v) dst[v] = acc[v];
            } else {
                Pack<T, V> out;
#pragma unroll
                for (int v = 0; v < V; ++v) out.v[v] = Vec<T>::from_f(acc[v]);
                *reinterpret_cast<Pack<T, V> *>(Y + (int64_t)row * ldy) = out;
            }
        }
    }
}

// X in shared memory: one 16-warp CTA per SM, streaming through the ring.
template <typename T, int V, typename I, int S = kG1Stages>
cudaError_t gather1_launch(const spmm_plan *p, int64_t n_items, const I *col, const void *X,
                           int64_t ldx, void *Y, int64_t ldy, cudaStream_t s) {
    const bool dyn = p->mode == SPMM_DYNAMIC;
    const size_t smem = g1_fixed_smem<T, I, S>() + (size_t)p->k * V * sizeof(T);
    static std::atomic<uint64_t> attrs{0};
    const cudaError_t e = set_smem_attrs_once(attrs, gather1_kernel<T, V, I, S>,
                                              g1_fixed_smem<T, I, S>() + g1_x_budget<T, I, S>(),
                                              false);
    if (e != cudaSuccess) return e;
    int64_t blocks = (n_items + kG1Warps - 1) / kG1Warps;
    const int64_t cap_blocks = (int64_t)std::max(p->sm_count, 1);
    if (blocks > cap_blocks) blocks = cap_blocks;
    if (blocks < 1) blocks = 1;
    // entries the index and value arrays hold (copies past them are not made)
    const int64_t cap = dyn ? p->nnzb_max : p->nnzb;
    pdl_launch(gather1_kernel<T, V, I, S>, dim3((unsigned)blocks), dim3(kG1Warps * 32), smem, s,
        p->d_items, n_items, col, (const T *)p->d_packed, cap, (const T *)X, ldx, p->k,
        (T *)Y, ldy, p->d_ws, p->d_ws_row0, dyn ? p->d_counts + kCntItems : nullptr, p->d_status);
    return cudaGetLastError();
}

// X in global memory: persistent 512-thread blocks, SPMM_G1_BLOCKS per SM.
template <typename T, int V>
cudaError_t gather1g_launch(const spmm_plan *p, int64_t n_items, const void *X, int64_t ldx,
                            void *Y, int64_t ldy, cudaStream_t s) {
    const bool dyn = p->mode == SPMM_DYNAMIC;
    int64_t blocks = (n_items * 32 + 511) / 512;
    const int64_t cap = (int64_t)std::max(p->sm_count, 1) * SPMM_G1_BLOCKS;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    pdl_launch(gather1g_kernel<T, V>, dim3((unsigned)blocks), dim3(512), 0, s, p->d_items,
        n_items, p->d_col_idx, (const T *)p->d_packed, (const T *)X, ldx, (T *)Y, ldy,
        p->d_ws, p->d_ws_row0, dyn ? p->d_counts + kCntItems : nullptr, p->d_status);
    return cudaGetLastError();
}

// Dense rows (ld = n) -> rows of stride ld (serving: X staged in one
// contiguous copy, re-strided for the kernels' aligned rows).
template <typename E>
__global__ void restride_kernel(const E *__restrict__ src, E *__restrict__ dst, int64_t rows,
                                int64_t n, int64_t ld) {
    pdl_enter();
    const int64_t total = rows * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / n, c = t - r * n;
        dst[r * ld + c] = src[t];
    }
}

// ------------------------------------------------- split-row reduction ---
// Rows split over several items: Y = sum of the chunks' FP32 partials in
// chunk order (deterministic), converted once.  bar_reset (dynamic plans
// with the fused re-partition): the re-partition's barrier words, zeroed
// here for the plan's next call; this launch follows the re-partition and
// the product in every call with a product, aborted or not.
template <typename T>
__global__ void reduce_kernel(const int32_t *__restrict__ red, const int32_t *__restrict__ grp_row0,
                              const int32_t *__restrict__ grp_rows, int rows_per_unit,
                              const float *__restrict__ ws, const int64_t *__restrict__ ws_row0,
                              T *__restrict__ Y, int64_t ldy, int64_t n, int64_t n_red,
                              const int32_t *__restrict__ n_red_dev,
                              const int32_t *__restrict__ status, int32_t *bar_reset) {
    pdl_enter();
  if (bar_reset && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) {
      bar_reset[0] = 0;
      bar_reset[1] = 0;
  }
  if (n_red_dev) {
      if (*status != 0) return;
      n_red = min(n_red, (int64_t)*n_red_dev);
  }
  for (int64_t q = blockIdx.z; q < n_red; q += gridDim.z) {
    const int32_t *rd = red + q * 3;
    const int32_t g = rd[0], slot0 = rd[1], nch = rd[2];
    const int64_t nrows = grp_rows ? (int64_t)grp_rows[g] * rows_per_unit : 1;
    const int64_t yrow0 = grp_row0 ? (int64_t)grp_row0[g] * rows_per_unit : g;
    for (int64_t r = blockIdx.y; r < nrows; r += gridDim.y) {
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
             j += (int64_t)gridDim.x * blockDim.x) {
            float acc = 0.f;
            for (int c = 0; c < nch; ++c) acc += ws[(ws_row0[slot0 + c] + r) * n + j];
            Y[(yrow0 + r) * ldy + j] = Vec<T>::from_f(acc);
        }
    }
  }
}

inline unsigned grid1d(int64_t total, int threads) {
    int64_t g = (total + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > (1 << 30)) g = 1 << 30;
    return (unsigned)g;
}

template <typename T, int V>
cudaError_t gather_launch(const spmm_plan *p, const void *X, int64_t n, int64_t ldx, void *Y,
                          int64_t ldy, cudaStream_t s) {
    const bool dyn = p->mode == SPMM_DYNAMIC;
    const int64_t n_items = dyn ? p->dyn.items_cap : p->n_items;
    const int64_t vecs = (n + V - 1) / V;
    int LN = 1;
    while (LN < 32 && LN < vecs) LN <<= 1;
    const int nchunk = (int)((n + (int64_t)LN * V - 1) / ((int64_t)LN * V));
    const int64_t warps = n_items * nchunk;
    if (warps == 0) return cudaSuccess;
    if (vecs == 1) {
        // n == V: one vector per X row; X in shared memory when it fits
        // (with the 16-bit column indices where the plan holds them)
        const int64_t xb = (int64_t)p->k * V * (int64_t)sizeof(T);
        if (p->d_col16 && xb <= g1_x_budget<T, uint16_t>())
            return gather1_launch<T, V, uint16_t>(p, n_items, p->d_col16, X, ldx, Y, ldy, s);
        if (p->d_col16 && xb <= g1_x_budget<T, uint16_t, kG1Stages - 1>())
            return gather1_launch<T, V, uint16_t, kG1Stages - 1>(p, n_items, p->d_col16, X, ldx,
                                                                 Y, ldy, s);
        if (xb <= g1_x_budget<T, int32_t>())
            return gather1_launch<T, V, int32_t>(p, n_items, p->d_col_idx, X, ldx, Y, ldy, s);
        return gather1g_launch<T, V>(p, n_items, X, ldx, Y, ldy, s);
    }
    pdl_launch(gather_kernel<T, V>, dim3(grid1d(warps * 32, 256)), dim3(256), 0, s, p->d_items,
        n_items, nchunk, LN, p->d_col_idx, (const T *)p->d_packed, (const T *)X, ldx, (T *)Y, ldy,
        n, p->d_ws, p->d_ws_row0, dyn ? p->d_counts + kCntItems : nullptr, p->d_status);
    return cudaGetLastError();
}

template <typename T>
cudaError_t gather_dispatch(const spmm_plan *p, const void *X, int64_t n, int64_t ldx, void *Y,
                            int64_t ldy, cudaStream_t s) {
    // widest vector that keeps every lane's load aligned and inside its row
    constexpr int Vmax = 16 / sizeof(T);
    auto ok = [&](int V) {
        const int64_t bytes = V * (int64_t)sizeof(T);
        return n % V == 0 && ldx % V == 0 && ldy % V == 0 &&
               ((uintptr_t)X % bytes) == 0 && ((uintptr_t)Y % bytes) == 0;
    };
    if (Vmax >= 8 && ok(8)) return gather_launch<T, (Vmax >= 8 ? 8 : 1)>(p, X, n, ldx, Y, ldy, s);
    if (ok(4)) return gather_launch<T, 4>(p, X, n, ldx, Y, ldy, s);
    if (ok(2)) return gather_launch<T, 2>(p, X, n, ldx, Y, ldy, s);
    return gather_launch<T, 1>(p, X, n, ldx, Y, ldy, s);
}

}  // namespace

cudaError_t launch_restride(const void *src, void *dst, int64_t rows, int64_t n, int64_t ld,
                            size_t elem, cudaStream_t s) {
    const int64_t total = rows * n;
    if (total == 0) return cudaSuccess;
    const unsigned g = grid1d(total, 256) > 2048u ? 2048u : grid1d(total, 256);
    if (elem == 2)
        pdl_launch(restride_kernel<uint16_t>, dim3(g), dim3(256), 0, s, (const uint16_t *)src,
            (uint16_t *)dst, rows, n, ld);
    else if (elem == 4)
        pdl_launch(restride_kernel<uint32_t>, dim3(g), dim3(256), 0, s, (const uint32_t *)src,
            (uint32_t *)dst, rows, n, ld);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// Row-slice plans: the kept blocks' values, gathered from the whole
// pattern's value array into the slice's order before packing.
template <typename U>
__global__ void gather_blocks_kernel(const U *__restrict__ src, const int32_t *__restrict__ idx,
                                     int64_t nblk, int64_t per, U *__restrict__ dst) {
    pdl_enter();
    const int64_t total = nblk * per;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = t / per, e = t - q * per;
        dst[t] = src[(int64_t)idx[q] * per + e];
    }
}

cudaError_t launch_gather_blocks(const void *src, const int32_t *idx, int64_t nblk,
                                 int64_t block_bytes, void *dst, cudaStream_t s) {
    if (nblk == 0 || block_bytes == 0) return cudaSuccess;
    const uintptr_t al = (uintptr_t)src | (uintptr_t)dst;
    int u = 1;
    for (int c : {16, 8, 4, 2})
        if (block_bytes % c == 0 && al % c == 0) {
            u = c;
            break;
        }
    const int64_t per = block_bytes / u;
    const unsigned g = grid1d(nblk * per, 256) > 8192u ? 8192u : grid1d(nblk * per, 256);
    switch (u) {
        case 16: pdl_launch(gather_blocks_kernel<uint4>, dim3(g), dim3(256), 0, s,
                     (const uint4 *)src, idx, nblk, per, (uint4 *)dst); break;
        case 8: pdl_launch(gather_blocks_kernel<uint2>, dim3(g), dim3(256), 0, s,
                    (const uint2 *)src, idx, nblk, per, (uint2 *)dst); break;
        case 4: pdl_launch(gather_blocks_kernel<uint32_t>, dim3(g), dim3(256), 0, s,
                    (const uint32_t *)src, idx, nblk, per, (uint32_t *)dst); break;
        case 2: pdl_launch(gather_blocks_kernel<uint16_t>, dim3(g), dim3(256), 0, s,
                    (const uint16_t *)src, idx, nblk, per, (uint16_t *)dst); break;
        default: pdl_launch(gather_blocks_kernel<uint8_t>, dim3(g), dim3(256), 0, s,
                     (const uint8_t *)src, idx, nblk, per, (uint8_t *)dst); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_pack_csr(const spmm_plan *p, const void *d_values, const int32_t *d_nnzb,
                            cudaStream_t s) {
    const int bb = p->b * p->b;
    const int64_t nmax = d_nnzb ? p->nnzb_max : p->nnzb;
    const int64_t total = nmax * bb;
    if (total == 0) return cudaSuccess;
    const unsigned g = grid1d(total, 256) > 4096u ? 4096u : grid1d(total, 256);
    const int32_t *st = d_nnzb ? p->d_status : nullptr;
    switch (dtype_size(p->wdt)) {
        case 4:
            pdl_launch(pack_csr_kernel<uint32_t>, dim3(g), dim3(256), 0, s,
                (const uint32_t *)d_values, p->d_perm, nmax, p->b, p->transposed ? 1 : 0, d_nnzb, st,
                (uint32_t *)p->d_packed);
            break;
        case 2:
            pdl_launch(pack_csr_kernel<uint16_t>, dim3(g), dim3(256), 0, s,
                (const uint16_t *)d_values, p->d_perm, nmax, p->b, p->transposed ? 1 : 0, d_nnzb, st,
                (uint16_t *)p->d_packed);
            break;
        case 1:   // E4M3 codes (BGATHER plans)
            pdl_launch(pack_csr_kernel<uint8_t>, dim3(g), dim3(256), 0, s,
                (const uint8_t *)d_values, p->d_perm, nmax, p->b, p->transposed ? 1 : 0, d_nnzb, st,
                (uint8_t *)p->d_packed);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_plain(const spmm_plan *p, const void *X, int64_t n, int64_t ldx, void *Y,
                         int64_t ldy, cudaStream_t s) {
    dim3 grid(grid1d(n, 128), (unsigned)(p->m < 65535 ? p->m : 65535));
    pdl_launch(plain_f32_kernel, dim3(grid), dim3(128), 0, s, p->d_row_ptr, p->d_col_idx,
        (const float *)p->d_packed, (const float *)X, ldx, (float *)Y, ldy, p->m, n, p->b);
    return cudaGetLastError();
}

cudaError_t launch_gather(const spmm_plan *p, const void *X, int64_t n, int64_t ldx, void *Y,
                          int64_t ldy, cudaStream_t s) {
    switch (p->xdt) {
        case SPMM_F32: return gather_dispatch<float>(p, X, n, ldx, Y, ldy, s);
        case SPMM_F16: return gather_dispatch<__half>(p, X, n, ldx, Y, ldy, s);
        case SPMM_BF16: return gather_dispatch<__nv_bfloat16>(p, X, n, ldx, Y, ldy, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_reduce(const spmm_plan *p, int64_t n, void *Y, int64_t ldy, cudaStream_t s) {
    const bool dyn = p->mode == SPMM_DYNAMIC;
    const int64_t n_red = dyn ? p->dyn.red_cap : p->n_red;
    const int32_t *n_red_dev = dyn ? p->d_counts + kCntRed : nullptr;
    if (n_red == 0 || n == 0) return cudaSuccess;
    const bool tc = p->kernel == SPMM_KERNEL_TC;
    const int rows_per_unit = tc ? kTile : 1;
    // about two waves of blocks whatever the capacity (every loop of the
    // kernel strides); a dynamic plan's capacity, launched in full with its
    // true count read on the device, is usually far above the reductions it
    // has (mostly none), so it gets about two blocks per SM and the empty
    // launch stays short
    const unsigned gx = grid1d(n, 128) > 64u ? 64u : grid1d(n, 128);
    const int64_t zcap = dyn ? 8 : 64;
    const unsigned gz = (unsigned)(n_red < zcap ? n_red : zcap);
    const int64_t want = (dyn ? 2 : 2 * 16) * (int64_t)std::max(p->sm_count, 1);
    int64_t gy = tc ? (int64_t)(kMaxGroupRows * kTile) : 1;
    gy = std::max<int64_t>(1, std::min<int64_t>(gy, want / ((int64_t)gx * gz)));
    dim3 grid(gx, (unsigned)gy, gz);
    const int32_t *r0 = tc ? p->d_grp_row0 : nullptr;
    const int32_t *rn = tc ? p->d_grp_rows : nullptr;
    int32_t *bar = dyn && p->dyn_fused ? p->dyn.bar : nullptr;
    switch (p->xdt) {
        case SPMM_F32:
            pdl_launch(reduce_kernel<float>, dim3(grid), dim3(128), 0, s, p->d_red, r0, rn,
                rows_per_unit, p->d_ws, p->d_ws_row0, (float *)Y, ldy, n, n_red, n_red_dev,
                p->d_status, bar);
            break;
        case SPMM_F16:
            pdl_launch(reduce_kernel<__half>, dim3(grid), dim3(128), 0, s, p->d_red, r0, rn,
                rows_per_unit, p->d_ws, p->d_ws_row0, (__half *)Y, ldy, n, n_red, n_red_dev,
                p->d_status, bar);
            break;
        case SPMM_BF16:
            pdl_launch(reduce_kernel<__nv_bfloat16>, dim3(grid), dim3(128), 0, s, p->d_red, r0, rn,
                rows_per_unit, p->d_ws, p->d_ws_row0, (__nv_bfloat16 *)Y, ldy, n, n_red, n_red_dev,
                p->d_status, bar);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace spmm
