// Allocation-free entry point for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc at all: code running while a CUDA
// graph is being captured by someone else, allocator-owning frameworks that
// forbid side allocations, or real-time loops that budget every byte up
// front.  spmm_gather_noalloc serves them: it runs the dynamic b = 1 product
// (device re-partition, value packing, gather kernel, split-row reduction)
// with every scratch buffer carved out of one file-scope device array,
// g_noalloc_scratch, instead of plan-owned allocations.
//
// Facts a caller needs:
//  * The array is about 14 MB and sits in every GPU that loads this library
//    until the process exits.
//  * Limits: m <= 8192, nnzb_max <= 262144, n <= 256; larger requests are
//    rejected with SPMM_ERR_SHAPE before anything is enqueued.
//  * Each device has its own copy of the array.  All calls on one device
//    share that copy, and it keeps the last call's contents: each call
//    clears what must start at zero (row counts, counters, the status
//    word).  Calls that overlap on one device (different streams, or host
//    threads without ordering) race on it: serialise them.
//  * A call looks up the array's device address (cudaGetSymbolAddress, with
//    the device current) whenever its stream is not being captured, so a
//    device reset or a re-created context is picked up.  A call inside a
//    stream capture uses the address of the device's last uncaptured call:
//    make one call on the device before any stream capture.
//  * No cudaMalloc, cudaFree or allocating library routine is called.
#include <cuda_runtime.h>

#include <mutex>

#include "spmm_internal.h"

namespace spmm {
namespace {

constexpr int64_t kNaMaxRows = 8192;
constexpr int64_t kNaMaxNnzb = 262144;
constexpr int64_t kNaMaxN = 256;
constexpr int64_t kNaItems = 2 * kNaMaxRows + 2;
constexpr int64_t kNaWsSlots = kNaMaxRows + 1;

constexpr int64_t al(int64_t x) { return (x + 255) / 256 * 256; }

// byte offsets of the carved regions
constexpr int64_t oRowCnt = 0;
constexpr int64_t oCursor = oRowCnt + al(4 * kNaMaxRows);
constexpr int64_t oRowIbeg = oCursor + al(4 * kNaMaxRows);
constexpr int64_t oRowWbeg = oRowIbeg + al(4 * kNaMaxRows);
constexpr int64_t oRowRbeg = oRowWbeg + al(4 * kNaMaxRows);
constexpr int64_t oRowPtr = oRowRbeg + al(4 * kNaMaxRows);
constexpr int64_t oTmpCol = oRowPtr + al(4 * (kNaMaxRows + 1));
constexpr int64_t oTmpPerm = oTmpCol + al(4 * kNaMaxNnzb);
constexpr int64_t oColIdx = oTmpPerm + al(4 * kNaMaxNnzb);
constexpr int64_t oPerm = oColIdx + al(4 * kNaMaxNnzb);
constexpr int64_t oCounts = oPerm + al(4 * kNaMaxNnzb);
constexpr int64_t oStatus = oCounts + al(4 * kCntCount);
constexpr int64_t oItems = oStatus + al(4);
constexpr int64_t oWsRow0 = oItems + al(4 * kItemFields * kNaItems);
constexpr int64_t oRed = oWsRow0 + al(8 * kNaWsSlots);
constexpr int64_t oPacked = oRed + al(4 * 3 * kNaMaxRows);
constexpr int64_t oWs = oPacked + al(4 * kNaMaxNnzb);
constexpr int64_t kNaBytes = oWs + al(4 * kNaWsSlots * kNaMaxN);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (the host-side
// symbol is not a device address).  Outside a stream capture it is looked up
// again on every call (no allocation; a reset device gets its new address);
// inside one, the address of the last uncaptured call on the device is used.
cudaError_t scratch_address(cudaStream_t s, void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    } else if (!g_addr[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace spmm

using namespace spmm;

extern "C" spmm_status spmm_gather_noalloc(int64_t m, int64_t k, spmm_dtype dtype,
                                           const int32_t *d_nnzb, const int32_t *d_brow,
                                           const int32_t *d_bcol, int64_t nnzb_max,
                                           const void *d_values, const void *d_X, int64_t n,
                                           int64_t ldx, void *d_Y, int64_t ldy,
                                           int32_t *d_status, void *stream) {
    if (dtype != SPMM_F32 && dtype != SPMM_F16 && dtype != SPMM_BF16) {
        set_error("spmm_gather_noalloc: dtype must be F32, F16 or BF16");
        return SPMM_ERR_ARG;
    }
    if (m <= 0 || k <= 0 || n < 0 || nnzb_max < 0 || m > kNaMaxRows || nnzb_max > kNaMaxNnzb ||
        n > kNaMaxN || k > (int64_t)1 << 30) {
        set_error("spmm_gather_noalloc: needs 0 < m <= %lld, 0 < k <= %lld, "
                  "0 <= nnzb_max <= %lld, 0 <= n <= %lld (got m=%lld, k=%lld, nnzb_max=%lld, "
                  "n=%lld)",
                  (long long)kNaMaxRows, (long long)1 << 30, (long long)kNaMaxNnzb,
                  (long long)kNaMaxN, (long long)m, (long long)k, (long long)nnzb_max,
                  (long long)n);
        return SPMM_ERR_SHAPE;
    }
    if (ldx < (n > 0 ? n : 1) || ldy < (n > 0 ? n : 1)) {
        set_error("spmm_gather_noalloc: ldx and ldy must be >= max(n, 1)");
        return SPMM_ERR_SHAPE;
    }
    if (!d_nnzb || !d_brow || !d_bcol || !d_values || (n > 0 && (!d_X || !d_Y))) {
        set_error("spmm_gather_noalloc: pattern, values, X and Y are required");
        return SPMM_ERR_ARG;
    }
    void *base = nullptr;
    cudaError_t e = scratch_address((cudaStream_t)stream, &base);
    if (e != cudaSuccess) {
        set_error("spmm_gather_noalloc: scratch address lookup failed: %s (inside a stream "
                  "capture, make one uncaptured call on the device first)",
                  cudaGetErrorString(e));
        return SPMM_ERR_CUDA;
    }
    char *sc = (char *)base;
    // a plan view over the scratch array (host object only, nothing allocated)
    spmm_plan p;
    p.m = m;
    p.k = k;
    p.b = 1;
    p.n_max = n;
    p.nnzb_max = nnzb_max;
    p.mode = SPMM_DYNAMIC;
    p.wdt = p.xdt = dtype;
    p.kernel = SPMM_KERNEL_GATHER;
    {
        // grid sizing of the persistent gather (an attribute query, no allocation)
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&p.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            p.sm_count = 1;
    }
    p.dyn.row_cnt = (int32_t *)(sc + oRowCnt);
    p.dyn.cursor = (int32_t *)(sc + oCursor);
    p.dyn.row_ibeg = (int32_t *)(sc + oRowIbeg);
    p.dyn.row_wbeg = (int32_t *)(sc + oRowWbeg);
    p.dyn.row_rbeg = (int32_t *)(sc + oRowRbeg);
    p.dyn.tmp_col = (int32_t *)(sc + oTmpCol);
    p.dyn.tmp_perm = (int32_t *)(sc + oTmpPerm);
    p.dyn.items_cap = 2 * m + 2;
    p.dyn.ws_slots_cap = m + 1;
    p.dyn.red_cap = m;
    p.d_row_ptr = (int32_t *)(sc + oRowPtr);
    p.d_col_idx = (int32_t *)(sc + oColIdx);
    p.d_perm = (int32_t *)(sc + oPerm);
    p.d_counts = (int32_t *)(sc + oCounts);
    p.d_status = d_status ? d_status : (int32_t *)(sc + oStatus);
    p.d_items = (int32_t *)(sc + oItems);
    p.d_ws_row0 = (int64_t *)(sc + oWsRow0);
    p.d_red = (int32_t *)(sc + oRed);
    p.d_packed = sc + oPacked;
    p.d_ws = (float *)(sc + oWs);
    p.n_items = p.dyn.items_cap;
    p.n_red = p.dyn.red_cap;
    cudaStream_t s = (cudaStream_t)stream;
    spmm_dpattern dp{d_nnzb, d_brow, d_bcol};
    e = launch_dynamic_partition(&p, &dp, s);
    if (e == cudaSuccess) e = launch_pack_csr(&p, d_values, d_nnzb, s);
    if (e == cudaSuccess && n > 0) e = launch_gather(&p, d_X, n, ldx, d_Y, ldy, s);
    if (e == cudaSuccess && n > 0) e = launch_reduce(&p, n, d_Y, ldy, s);
    if (e != cudaSuccess) {
        set_error("spmm_gather_noalloc: launch failed: %s", cudaGetErrorString(e));
        return SPMM_ERR_CUDA;
    }
    return SPMM_OK;
}
