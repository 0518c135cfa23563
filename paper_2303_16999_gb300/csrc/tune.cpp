// The autotuner: for a (b, density, n) bucket of static products, times
// each candidate launch configuration (kernel family, tensor-core stage
// geometry) on the device and keeps the fastest, which spmm_plan_create
// then applies to AUTO plans of the same bucket.  The paper tunes its
// partitions ahead of time for a fixed pattern (Section 3.2); this table
// is this library's analogue for the choice of GPU kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "spmm_internal.h"

namespace spmm {
namespace {

// (b, W type, X type, log2 m, log2 k, density bucket round(log2(1/d)),
// n bucket = ceil(log2 n))
using Key = std::tuple<int, int, int, int, int, int, int>;

struct Entry {
    spmm_tune_choice choice;
};

std::mutex g_mu;
std::map<Key, Entry> g_table;

int ilog2_ceil(int64_t v) {
    int r = 0;
    while (((int64_t)1 << r) < v) ++r;
    return r;
}

Key make_key(int64_t m, int64_t k, int b, int64_t nnzb, int64_t n, spmm_dtype w, spmm_dtype x) {
    const double cells = (double)(m / b) * (double)(k / b);
    const double d = cells > 0 && nnzb > 0 ? (double)nnzb / cells : 1.0;
    const int db = (int)std::lround(std::log2(1.0 / d));
    return Key(b, (int)w, (int)x, ilog2_ceil(m), ilog2_ceil(k), db, ilog2_ceil(std::max<int64_t>(n, 1)));
}

}  // namespace

bool tune_lookup(int64_t m, int64_t k, int b, int64_t nnzb, int64_t n, spmm_dtype w, spmm_dtype x,
                 spmm_tune_choice *out) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_table.find(make_key(m, k, b, nnzb, n, w, x));
    if (it == g_table.end()) return false;
    *out = it->second.choice;
    return true;
}

}  // namespace spmm

using namespace spmm;

extern "C" {

spmm_status spmm_tune(int64_t m, int64_t k, int64_t n, int32_t b, spmm_dtype w_dtype,
                      spmm_dtype x_dtype, const spmm_pattern *pattern, const void *d_values,
                      const float *d_scales, const void *d_X, int64_t ldx, int32_t reps,
                      void *stream, spmm_tune_result *out) {
    if (!pattern || !d_values || !d_X || !out || n <= 0 || reps <= 0 || reps > 64 ||
        (w_dtype == SPMM_E4M3 && !d_scales)) {
        set_error("tune: pattern, values (and E4M3 scales), X, out, n > 0 and 1 <= reps <= 64 "
                  "required");
        return SPMM_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::memset(out, 0, sizeof(*out));
    // the candidates: the tensor-core kernel with each stage geometry, with
    // the planner's groups and, where those shrink below 16 tile rows to
    // fill the CTA slots, with 16-row groups split along k instead; and the
    // CUDA-core block gather where it applies
    std::vector<spmm_tune_choice> cands = {{SPMM_KERNEL_TC, 1, 0, 0, 0}, {SPMM_KERNEL_TC, 2, 0, 0, 0}};
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            sms > 0 && m % kTile == 0) {
            const int64_t mt = m / kTile, g16 = (mt + kMaxGroupRows - 1) / kMaxGroupRows;
            const int64_t ntn = (n + kNTile - 1) / kNTile, slots = 2 * (int64_t)sms;
            if (g16 * ntn < slots) {
                const int32_t split =
                    (int32_t)std::min<int64_t>(1024, (slots + g16 * ntn - 1) / (g16 * ntn));
                cands.push_back({SPMM_KERNEL_TC, 1, kMaxGroupRows, split, 0});
                cands.push_back({SPMM_KERNEL_TC, 2, kMaxGroupRows, split, 0});
            }
        }
    }
    if (n > kNTile) {
        cands.push_back({SPMM_KERNEL_TC, 1, 0, 0, 2});
        cands.push_back({SPMM_KERNEL_TC, 2, 0, 0, 2});
    }
    const bool x16 = x_dtype == SPMM_F16 || x_dtype == SPMM_BF16;
    if (b >= 4 && n <= kBgMaxN && x16 && (w_dtype == x_dtype || w_dtype == SPMM_E4M3))
        cands.push_back({SPMM_KERNEL_BGATHER, 0, 0, 0, 0});
    void *d_Y = nullptr;
    cudaError_t e = cudaMalloc(&d_Y, (size_t)m * n * dtype_size(x_dtype));
    if (e != cudaSuccess) {
        set_error("tune: Y scratch: %s", cudaGetErrorString(e));
        return SPMM_ERR_OOM;
    }
    cudaEvent_t ev[2 * 64];
    int nev = 0;
    for (; nev < 2 * reps; ++nev)
        if (cudaEventCreate(&ev[nev]) != cudaSuccess) break;
    spmm_status st = SPMM_OK;
    float best = 0.f;
    int found = 0;
    for (size_t ci = 0; ci < cands.size() && ci < 8 && st == SPMM_OK && nev == 2 * reps; ++ci) {
        spmm_plan_opts o{};
        o.kernel = cands[ci].kernel;
        o.stage_geometry = cands[ci].stage_geometry;
        o.rows_per_group = cands[ci].rows_per_group;
        o.k_splits = cands[ci].k_splits;
        o.col_tiles = cands[ci].col_tiles;
        spmm_plan *p = nullptr;
        spmm_status cs = spmm_plan_create(m, k, n, b, SPMM_STATIC, w_dtype, x_dtype, pattern, 0,
                                          &o, &p);
        if (cs != SPMM_OK) continue;   // not applicable to this shape
        float t = -1.f;
        cs = spmm_pack_values(p, d_values, d_scales, stream);
        for (int w = 0; w < 2 && cs == SPMM_OK; ++w)
            cs = spmm_run(p, nullptr, nullptr, nullptr, d_X, n, ldx, d_Y, n, stream);
        std::vector<float> ts;
        for (int r = 0; r < reps && cs == SPMM_OK; ++r) {
            cudaEventRecord(ev[2 * r], s);
            cs = spmm_run(p, nullptr, nullptr, nullptr, d_X, n, ldx, d_Y, n, stream);
            cudaEventRecord(ev[2 * r + 1], s);
        }
        if (cs == SPMM_OK && cudaStreamSynchronize(s) == cudaSuccess) {
            for (int r = 0; r < reps; ++r) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[2 * r], ev[2 * r + 1]);
                ts.push_back(ms * 1e3f);
            }
            std::sort(ts.begin(), ts.end());
            t = ts[ts.size() / 2];
        }
        int32_t dev_status = 0;
        if (spmm_get_status(p, &dev_status) != SPMM_OK || dev_status != 0) t = -1.f;
        spmm_plan_info info{};
        spmm_plan_get_info(p, &info);
        spmm_plan_destroy(p);
        if (cs != SPMM_OK && cs != SPMM_ERR_UNSUPPORTED) st = cs;
        const int c = out->n_candidates++;
        out->cand[c] = cands[ci];
        if (cands[ci].kernel == SPMM_KERNEL_TC) out->cand[c].stage_geometry = info.stage_geometry + 1;
        out->cand_us[c] = t;
        if (t > 0.f && (!found || t < best)) {
            best = t;
            found = 1;
            out->choice = out->cand[c];
        }
    }
    for (int i = 0; i < nev; ++i) cudaEventDestroy(ev[i]);
    cudaFree(d_Y);
    if (st != SPMM_OK) return st;
    if (!found) {
        set_error("tune: no candidate ran");
        return SPMM_ERR_UNSUPPORTED;
    }
    out->best_us = best;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_table[make_key(m, k, b, pattern->nnzb, n, w_dtype, x_dtype)] = Entry{out->choice};
    }
    return SPMM_OK;
}

void spmm_tune_clear(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_table.clear();
}

int64_t spmm_tune_size(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    return (int64_t)g_table.size();
}

}  // extern "C"
