// C ABI of the block-sparse x dense product: plan lifetime, value packing,
// dispatch to the kernels, status and inspection.  No exception crosses the
// interface; every failure returns an spmm_status and leaves a thread-local
// message for spmm_last_error().
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "spmm_internal.h"

namespace spmm {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

size_t dtype_size(spmm_dtype t) {
    switch (t) {
        case SPMM_F32: return 4;
        case SPMM_F16:
        case SPMM_BF16: return 2;
        case SPMM_E4M3: return 1;
    }
    return 0;
}

bool build_csr_checked(int64_t mb, int64_t nnzb, const int32_t *brow, const int32_t *bcol,
                       HostPlan &hp);

static spmm_status cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SPMM_ERR_OOM : SPMM_ERR_CUDA;
}

template <typename T>
static cudaError_t dalloc(spmm_plan *p, T **ptr, int64_t count) {
    *ptr = nullptr;
    if (count <= 0) return cudaSuccess;
    void *v = nullptr;
    cudaError_t e = cudaMalloc(&v, (size_t)count * sizeof(T));
    if (e != cudaSuccess) return e;
    p->allocations.push_back(v);
    p->device_bytes += count * (int64_t)sizeof(T);
    *ptr = (T *)v;
    return cudaSuccess;
}

template <typename T>
static cudaError_t upload(spmm_plan *p, T **ptr, const std::vector<T> &v) {
    cudaError_t e = dalloc(p, ptr, (int64_t)v.size());
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpy(*ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

static void free_plan(spmm_plan *p) {
    if (!p) return;
    for (void *a : p->allocations) cudaFree(a);
    if (p->done) cudaEventDestroy(p->done);
    delete p;
}

static int pick_kernel(int req, int b, spmm_dtype w, spmm_dtype x, spmm_mode mode, int64_t n_max) {
    if (req != SPMM_KERNEL_AUTO) return req;
    if (b == 1) return SPMM_KERNEL_GATHER;
    if (w == SPMM_F32) return SPMM_KERNEL_PLAIN;
    // small n: every block read once on the CUDA cores beats 16 x 16 tiles
    // against 128-column MMA tiles
    // (measured on the batched FFN-like shapes: 16 x 16 blocks win on the
    // tensor cores from n = 11 on, smaller blocks keep the gather to n = 16)
    if (mode == SPMM_STATIC && n_max <= (b == 16 ? kBgAutoMaxN16 : kBgAutoMaxN) &&
        (x == SPMM_F16 || x == SPMM_BF16) && (w == x || w == SPMM_E4M3))
        return SPMM_KERNEL_BGATHER;
    return SPMM_KERNEL_TC;
}

static spmm_status check_types(int kernel, int b, spmm_dtype w, spmm_dtype x, int64_t m,
                               int64_t k) {
    const bool x16 = (x == SPMM_F16 || x == SPMM_BF16);
    switch (kernel) {
        case SPMM_KERNEL_PLAIN:
            if (w == SPMM_F32 && x == SPMM_F32) return SPMM_OK;
            set_error("PLAIN kernel is FP32 only (W and X F32)");
            return SPMM_ERR_UNSUPPORTED;
        case SPMM_KERNEL_GATHER:
            if (b != 1) {
                set_error("GATHER kernel needs b = 1");
                return SPMM_ERR_UNSUPPORTED;
            }
            if (w == x && w != SPMM_E4M3) return SPMM_OK;
            set_error("GATHER kernel needs W and X of one type in {F32, F16, BF16}");
            return SPMM_ERR_UNSUPPORTED;
        case SPMM_KERNEL_BGATHER:
            if (b < 4) {
                set_error("BGATHER kernel needs b in {4, 8, 16}");
                return SPMM_ERR_UNSUPPORTED;
            }
            if (x16 && (w == x || w == SPMM_E4M3)) return SPMM_OK;
            set_error("BGATHER kernel needs 16-bit X and W of the same type (or E4M3 W)");
            return SPMM_ERR_UNSUPPORTED;
        case SPMM_KERNEL_TC:
            if (m % kTile || k % kTile) {
                set_error("TC kernel needs m and k multiples of 16");
                return SPMM_ERR_UNSUPPORTED;
            }
            if (x16 && (w == x || w == SPMM_E4M3)) return SPMM_OK;
            set_error("TC kernel needs 16-bit X and W of the same type (or E4M3 W)");
            return SPMM_ERR_UNSUPPORTED;
        default:
            set_error("unknown kernel %d", kernel);
            return SPMM_ERR_ARG;
    }
}

// b = 1 and 16-bit X: the tensor-core kernel (element blocks packed into 16 x
// 16 tiles) wins once n fills its 128-column MMA tiles and the tiles are not
// nearly empty; otherwise the CUDA-core gather kernel.
static bool b1_prefers_tc(int64_t m, int64_t k, int64_t n_max, spmm_dtype w, spmm_dtype x,
                          const spmm_pattern *pat) {
    if (!pat || pat->nnzb <= 0 || !pat->brow || !pat->bcol || n_max < kNTile || m % kTile ||
        k % kTile)
        return false;
    if (!((x == SPMM_F16 || x == SPMM_BF16) && w == x)) return false;
    const int64_t kt = k / kTile;
    std::vector<int64_t> t(pat->nnzb);
    for (int64_t p = 0; p < pat->nnzb; ++p) {
        if (pat->brow[p] < 0 || pat->bcol[p] < 0) return false;  // validated later
        t[p] = (int64_t)(pat->brow[p] / kTile) * kt + pat->bcol[p] / kTile;
    }
    std::sort(t.begin(), t.end());
    const int64_t tiles = std::unique(t.begin(), t.end()) - t.begin();
    return pat->nnzb >= 4 * tiles;
}

// Tensor-core plans with work for at least a full wave at 16 rows per
// group: the number of near-equal tile-row groups that best fills the CTA
// slots (one per SM for two-column-tile launches, two otherwise; dynamic
// plans always launch one column tile per CTA, so they pass wide = false),
// measured by waves x rows per unit, ceil(q U / S) / q; 0 keeps the equal
// partition.  Groups keep at least 12 rows and a new count must be at least
// 3 % better.  At m = k = 4096, n = 2048 this gives 19 groups of 13-14 rows
// (19 x 8 units on 152 SMs), 2-8 % faster on every point of the sweep than
// 16 groups of 16.
static int64_t auto_groups(int64_t mt, int64_t n_max, int sms, bool wide) {
    if (sms <= 0 || mt <= 0) return 0;
    const int64_t ntn = std::max<int64_t>(1, (n_max + kNTile - 1) / kNTile);
    const int64_t U = wide ? (ntn + 1) / 2 : ntn, S = (int64_t)sms * (wide ? 1 : 2);
    const int64_t q16 = (mt + kMaxGroupRows - 1) / kMaxGroupRows;
    if (q16 * ntn < sms) return 0;   // small problems: the rows-per-group rule
    auto cost = [&](int64_t q) { return (double)((q * U + S - 1) / S) / (double)q; };
    int64_t best = q16;
    for (int64_t q = q16 + 1; q <= mt / 12; ++q)
        if (cost(q) < cost(best)) best = q;
    return cost(best) < 0.97 * cost(q16) ? best : 0;
}

static int default_R(int64_t mt, int64_t n_max, int sms) {
    const int64_t ntn = std::max<int64_t>(1, (n_max + kNTile - 1) / kNTile);
    int R = kMaxGroupRows;
    while (R > 1 && (int64_t)group_partition(mt, R).size() * ntn < sms) R /= 2;
    return R;
}

// Static GATHER plans whose block columns fit 16 bits keep a 16-bit copy of
// col_idx for the gather kernels.
static bool col16_plan(const spmm_plan *p) {
    return p->kernel == SPMM_KERNEL_GATHER && p->mode == SPMM_STATIC && p->k / p->b <= 65536;
}

static spmm_status upload_plan(spmm_plan *p) {
    HostPlan &hp = p->hp;
    cudaError_t e = cudaSuccess;
#define UP(field, vec) \
    if (e == cudaSuccess) e = upload(p, &p->field, hp.vec)
    UP(d_row_ptr, row_ptr);
    UP(d_col_idx, col_idx);
    UP(d_perm, perm);
    UP(d_items, items);
    UP(d_red, red);
    UP(d_ws_row0, ws_row0);
    if (col16_plan(p) && e == cudaSuccess) {
        // the b = 1 gather's column indices in half the bytes
        const std::vector<uint16_t> c16(hp.col_idx.begin(), hp.col_idx.end());
        e = upload(p, &p->d_col16, c16);
    }
    if (p->kernel == SPMM_KERNEL_TC) {
        UP(d_grp_row0, grp_row0);
        UP(d_grp_rows, grp_rows);
        UP(d_grp_ebeg, grp_ebeg);
        UP(d_ent_col, ent_col);
        UP(d_ent_tbeg, ent_tbeg);
        UP(d_ent_cover, ent_cover);
        UP(d_tile_row, tile_row);
        UP(d_blk_slot, blk_slot);
        UP(d_blk_off, blk_off);
        // one stage record per entry at most (every stage holds an entry)
        const int64_t E = std::max<int64_t>((int64_t)hp.ent_col.size(), 1);
        if (e == cudaSuccess) e = dalloc(p, &p->d_srec, E * stage_record_words());
        if (e == cudaSuccess) e = dalloc(p, &p->d_sprog, E * stage_prog_words());
    }
#undef UP
    if (e != cudaSuccess) return cuda_fail(e, "plan upload");
    return SPMM_OK;
}

// Device buffers of a dynamic plan, sized for nnzb_max blocks.  Work items
// and workspace are bounded independently of the pattern: the chunk size
// C >= 1.25 E / G keeps the split chunks below 1.6 G (TC); for b = 1,
// C1 >= 2 nnzb / mb keeps them below mb.
static spmm_status alloc_dynamic(spmm_plan *p) {
    DynBufs &d = p->dyn;
    const int64_t mb = p->m / p->b, cap = p->nnzb_max, G = p->n_groups;
    const bool tc = p->kernel == SPMM_KERNEL_TC;
    cudaError_t e = cudaSuccess;
#define AL(ptr, n) \
    if (e == cudaSuccess) e = dalloc(p, &(ptr), (int64_t)(n))
    AL(d.row_cnt, mb);
    AL(d.cursor, mb);
    AL(d.tmp_col, cap);
    AL(d.tmp_perm, cap);
    AL(p->d_row_ptr, mb + 1);
    AL(p->d_col_idx, cap);
    AL(p->d_perm, cap);
    AL(p->d_counts, kCntCount);
    if (tc) {
        d.items_cap = 2 * G + 2;
        d.ws_slots_cap = 2 * G + 2;
        d.red_cap = G;
        p->hp.ws_rows = d.ws_slots_cap * p->R * kTile;
        e = upload(p, &p->d_grp_row0, p->hp.grp_row0);
        if (e == cudaSuccess) e = upload(p, &p->d_grp_rows, p->hp.grp_rows);
        AL(d.grp_cnt, 2 * G);
        AL(d.grp_sbeg, G);
        AL(d.grp_ibeg, G);
        AL(d.grp_wbeg, G);
        AL(d.grp_rbeg, G);
        AL(d.grp_wrow, G);
        if (p->dyn_fused) {
            const int64_t kw = (p->k / p->b + 31) / 32;
            if (mb * kw > kFusedMaxBitmapWords) {
                p->dyn_fused = false;   // the launch chain needs no bitmap
            } else {
                AL(d.bits, mb * kw);
                AL(d.wpre, mb * kw);
                AL(d.gmask, G * (p->k / kTile));
                AL(d.bar, kFusedMaxCtas + 1);
            }
        }
        AL(p->d_grp_ebeg, G + 1);
        AL(p->d_ent_col, cap);
        AL(p->d_ent_tbeg, cap + 1);
        AL(p->d_ent_cover, cap);
        AL(p->d_tile_row, cap);
        AL(p->d_blk_slot, cap);
        AL(p->d_blk_off, cap);
        AL(p->d_srec, std::max<int64_t>(cap, 1) * stage_record_words());
        AL(p->d_sprog, std::max<int64_t>(cap, 1) * stage_prog_words());
    } else {
        d.items_cap = 2 * mb + 2;
        d.ws_slots_cap = mb + 1;
        d.red_cap = mb;
        p->hp.ws_rows = d.ws_slots_cap;
        AL(d.row_ibeg, mb);
        AL(d.row_wbeg, mb);
        AL(d.row_rbeg, mb);
    }
    AL(p->d_items, d.items_cap * kItemFields);
    AL(p->d_ws_row0, d.ws_slots_cap);
    AL(p->d_red, d.red_cap * 3);
#undef AL
    if (e != cudaSuccess) return cuda_fail(e, "dynamic plan allocation");
    p->n_items = d.items_cap;
    p->n_red = d.red_cap;
    return SPMM_OK;
}

template <typename T>
static cudaError_t download(std::vector<T> &dst, const T *src, int64_t n) {
    dst.resize(n < 0 ? 0 : n);
    if (n <= 0) return cudaSuccess;
    return cudaMemcpy(dst.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost);
}

// Dynamic plans: copies the arrays the last call built on the device into
// the host mirror, with their true lengths.
static spmm_status refresh_dynamic(spmm_plan *p) {
    if (p->mode != SPMM_DYNAMIC || p->host_only) return SPMM_OK;
    if (p->ran) {
        cudaError_t e = cudaEventSynchronize(p->done);
        if (e != cudaSuccess) return cuda_fail(e, "event synchronize");
    }
    int32_t c[kCntCount] = {0};
    cudaError_t e = cudaMemcpy(c, p->d_counts, sizeof(c), cudaMemcpyDeviceToHost);
    HostPlan &hp = p->hp;
    const int64_t mb = p->m / p->b, nnzb = c[kCntNnzb];
    p->nnzb = nnzb;
    p->C = c[kCntChunk];
    if (e == cudaSuccess) e = download(hp.row_ptr, p->d_row_ptr, mb + 1);
    if (e == cudaSuccess) e = download(hp.col_idx, p->d_col_idx, nnzb);
    if (e == cudaSuccess) e = download(hp.perm, p->d_perm, nnzb);
    if (e == cudaSuccess) e = download(hp.items, p->d_items, (int64_t)c[kCntItems] * kItemFields);
    if (e == cudaSuccess) e = download(hp.red, p->d_red, (int64_t)c[kCntRed] * 3);
    if (p->kernel == SPMM_KERNEL_TC) {
        const int64_t E = c[kCntEntries], S = c[kCntSlots];
        if (e == cudaSuccess) e = download(hp.ws_row0, p->d_ws_row0, (int64_t)c[kCntWsSlots]);
        if (e == cudaSuccess) e = download(hp.grp_ebeg, p->d_grp_ebeg, p->n_groups + 1);
        if (e == cudaSuccess) e = download(hp.ent_col, p->d_ent_col, E);
        if (e == cudaSuccess) e = download(hp.ent_tbeg, p->d_ent_tbeg, E + 1);
        if (e == cudaSuccess) e = download(hp.ent_cover, p->d_ent_cover, E);
        if (e == cudaSuccess) e = download(hp.tile_row, p->d_tile_row, S);
        if (e == cudaSuccess) e = download(hp.blk_slot, p->d_blk_slot, nnzb);
        if (e == cudaSuccess) e = download(hp.blk_off, p->d_blk_off, nnzb);
        p->n_entries = E;
        p->n_tiles = S;
    } else {
        if (e == cudaSuccess) e = download(hp.ws_row0, p->d_ws_row0, (int64_t)c[kCntWsRows]);
    }
    if (e != cudaSuccess) return cuda_fail(e, "dynamic plan download");
    p->dyn_ws_rows = c[kCntWsRows];
    p->dyn_items = c[kCntItems];
    p->dyn_red = c[kCntRed];
    return SPMM_OK;
}

}  // namespace spmm

using namespace spmm;

extern "C" {

const char *spmm_last_error(void) { return g_err; }

const char *spmm_version(void) { return "spmm-gb300 0.1 (sm_103a)"; }

spmm_status spmm_equal_partition(int64_t extent, int64_t q, int64_t *sizes) {
    if (extent < 0 || q <= 0 || !sizes) {
        set_error("equal_partition: extent >= 0, q > 0 and sizes required");
        return SPMM_ERR_ARG;
    }
    for (int64_t i = 0; i < q - 1; ++i) sizes[i] = extent / q;
    sizes[q - 1] = extent - (q - 1) * (extent / q);
    return SPMM_OK;
}

int64_t spmm_bucket_size(int64_t m, int64_t k, int64_t num, int64_t den, int64_t qm, int64_t qk) {
    if (m < 0 || k < 0 || num < 0 || den <= 0 || qm <= 0 || qk <= 0) return -1;
    // ceil(m * k * num / (den * qm * qk)) in 128-bit to avoid overflow
    const __int128 a = (__int128)m * k * num, d = (__int128)den * qm * qk;
    return (int64_t)((a + d - 1) / d);
}

static spmm_status plan_create(int64_t m, int64_t k, int64_t n_max, int32_t b, spmm_mode mode,
                               spmm_dtype w_dtype, spmm_dtype x_dtype, const spmm_pattern *pattern,
                               int64_t nnzb_max, const spmm_plan_opts *opts, spmm_plan **out);

// A transposed plan is the plan of W^T (k x m, block (c, r) holding W's
// block (r, c) transposed): the pattern is swapped here, the values are
// transposed block by block when packed, and a dynamic call's pattern is
// swapped before the re-partition.
spmm_status spmm_plan_create(int64_t m, int64_t k, int64_t n_max, int32_t b, spmm_mode mode,
                             spmm_dtype w_dtype, spmm_dtype x_dtype, const spmm_pattern *pattern,
                             int64_t nnzb_max, const spmm_plan_opts *opts, spmm_plan **out) {
    g_err[0] = 0;
    if (!opts || !opts->transposed)
        return plan_create(m, k, n_max, b, mode, w_dtype, x_dtype, pattern, nnzb_max, opts, out);
    spmm_pattern tp{};
    const spmm_pattern *pp = nullptr;
    if (pattern) {
        tp.nnzb = pattern->nnzb;
        tp.brow = pattern->bcol;
        tp.bcol = pattern->brow;
        pp = &tp;
    }
    spmm_status st = plan_create(k, m, n_max, b, mode, w_dtype, x_dtype, pp, nnzb_max, opts, out);
    if (st == SPMM_OK) (*out)->transposed = true;
    return st;
}

// A row-slice plan (opts row_begin / row_end): the plan of the slice's
// blocks (those of its block rows, in pattern order, rows counted from
// row_begin), plus each kept block's index in the whole pattern, through
// which the whole W's values are gathered before packing.
static spmm_status plan_create_slice(int64_t m, int64_t k, int64_t n_max, int32_t b,
                                     spmm_mode mode, spmm_dtype w_dtype, spmm_dtype x_dtype,
                                     const spmm_pattern *pattern, const spmm_plan_opts &o,
                                     spmm_plan **out) {
    *out = nullptr;
    if (mode != SPMM_STATIC) {
        set_error("row slices are for static plans");
        return SPMM_ERR_UNSUPPORTED;
    }
    if (!pattern) {
        set_error("static plans need a pattern");
        return SPMM_ERR_ARG;
    }
    spmm_status st = validate_pattern(m, k, b, pattern->nnzb, pattern->brow, pattern->bcol);
    if (st != SPMM_OK) return st;
    const int64_t rb = o.row_begin, re = o.row_end;
    if (rb < 0 || re <= rb || re > m || rb % b || re % b) {
        set_error("row slice [%lld, %lld): needs 0 <= row_begin < row_end <= m = %lld, both "
                  "multiples of b = %d", (long long)rb, (long long)re, (long long)m, b);
        return SPMM_ERR_SHAPE;
    }
    std::vector<int32_t> sb, sc, src;
    try {
        // the whole pattern is checked for repeated blocks, so every rank of
        // a row split accepts or rejects the same pattern
        const int64_t kb = k / b;
        std::vector<int64_t> key(pattern->nnzb);
        for (int64_t p = 0; p < pattern->nnzb; ++p)
            key[p] = (int64_t)pattern->brow[p] * kb + pattern->bcol[p];
        std::sort(key.begin(), key.end());
        if (std::adjacent_find(key.begin(), key.end()) != key.end()) {
            set_error("pattern: a block is given twice");
            return SPMM_ERR_PATTERN;
        }
        const int32_t r0 = (int32_t)(rb / b), r1 = (int32_t)(re / b);
        for (int64_t p = 0; p < pattern->nnzb; ++p) {
            const int32_t r = pattern->brow[p];
            if (r < r0 || r >= r1) continue;
            sb.push_back(r - r0);
            sc.push_back(pattern->bcol[p]);
            src.push_back((int32_t)p);
        }
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed while slicing the pattern");
        return SPMM_ERR_OOM;
    }
    spmm_plan_opts o2 = o;
    o2.row_begin = o2.row_end = 0;
    const spmm_pattern sub{(int64_t)sb.size(), sb.data(), sc.data()};
    st = plan_create(re - rb, k, n_max, b, mode, w_dtype, x_dtype, &sub, 0, &o2, out);
    if (st != SPMM_OK) return st;
    spmm_plan *p = *out;
    p->row_begin = rb;
    p->row_end = re;
    p->src_index = std::move(src);
    if (!p->host_only) {
        const int64_t nb = (int64_t)p->src_index.size();
        cudaError_t e = upload(p, &p->d_src_index, p->src_index);
        if (e == cudaSuccess)
            e = dalloc(p, (char **)&p->d_slice_vals, nb * b * b * (int64_t)dtype_size(w_dtype));
        if (e == cudaSuccess && w_dtype == SPMM_E4M3) e = dalloc(p, &p->d_slice_scales, nb);
        if (e != cudaSuccess) {
            free_plan(p);
            *out = nullptr;
            return cuda_fail(e, "row-slice allocation");
        }
    }
    return SPMM_OK;
}

static spmm_status plan_create(int64_t m, int64_t k, int64_t n_max, int32_t b, spmm_mode mode,
                               spmm_dtype w_dtype, spmm_dtype x_dtype, const spmm_pattern *pattern,
                               int64_t nnzb_max, const spmm_plan_opts *opts, spmm_plan **out) {
    if (!out) {
        set_error("out is NULL");
        return SPMM_ERR_ARG;
    }
    *out = nullptr;
    if (opts && (opts->row_begin || opts->row_end))
        return plan_create_slice(m, k, n_max, b, mode, w_dtype, x_dtype, pattern, *opts, out);
    if (n_max < 0 || (mode != SPMM_STATIC && mode != SPMM_DYNAMIC) || w_dtype < SPMM_F32 ||
        w_dtype > SPMM_E4M3 || x_dtype < SPMM_F32 || x_dtype > SPMM_BF16) {
        set_error("bad n_max, mode or dtype");
        return SPMM_ERR_ARG;
    }
    spmm_plan_opts o{};
    if (opts) o = *opts;
    spmm_status st = validate_pattern(m, k, b, 0, nullptr, nullptr);
    if (st != SPMM_OK) return st;
    int kernel = pick_kernel(o.kernel, b, w_dtype, x_dtype, mode, n_max);
    {
        // the autotuner's choice for this bucket, if it has one
        spmm_tune_choice tch{};
        if (o.kernel == SPMM_KERNEL_AUTO && o.stage_geometry == 0 && o.rows_per_group == 0 &&
            o.groups == 0 && o.k_splits == 0 && o.col_tiles == 0 && mode == SPMM_STATIC &&
            pattern && b >= 4 && tune_lookup(m, k, b, pattern->nnzb, n_max, w_dtype, x_dtype, &tch)) {
            kernel = tch.kernel;
            o.stage_geometry = tch.stage_geometry;
            o.rows_per_group = tch.rows_per_group;
            o.k_splits = tch.k_splits;
            o.col_tiles = tch.col_tiles;
        }
    }
    if (o.kernel == SPMM_KERNEL_AUTO && b == 1 && mode == SPMM_STATIC &&
        b1_prefers_tc(m, k, n_max, w_dtype, x_dtype, pattern))
        kernel = SPMM_KERNEL_TC;
    st = check_types(kernel, b, w_dtype, x_dtype, m, k);
    if (st != SPMM_OK) return st;
    if (kernel == SPMM_KERNEL_BGATHER && (mode != SPMM_STATIC || n_max > kBgMaxN)) {
        set_error("BGATHER plans are static with n_max <= %d", kBgMaxN);
        return SPMM_ERR_UNSUPPORTED;
    }
    if (o.rows_per_group < 0 || o.rows_per_group > kMaxGroupRows || o.max_per_item < 0 ||
        o.k_splits < 0 || o.k_splits > 1024 ||
        o.col_tiles < 0 || o.col_tiles > 2 || o.groups < 0 || o.stage_geometry < 0 ||
        o.stage_geometry > 2 || o.dyn_chain < 0 || o.dyn_chain > 1 ||
        (o.groups > 0 && (o.rows_per_group || o.groups > m / kTile ||
                          (m / kTile + o.groups - 1) / o.groups > kMaxGroupRows))) {
        set_error("rows_per_group must be in 0..%d, max_per_item >= 0, k_splits in 0..1024, "
                  "col_tiles and stage_geometry in 0..2, dyn_chain 0 or 1, groups in 0 or "
                  "ceil(m/16/%d)..m/16 without rows_per_group",
                  kMaxGroupRows, kMaxGroupRows);
        return SPMM_ERR_ARG;
    }
    if (mode == SPMM_DYNAMIC && (nnzb_max < 0 || nnzb_max > INT32_MAX || o.host_only)) {
        set_error("dynamic plans need 0 <= nnzb_max <= INT32_MAX and device memory");
        return SPMM_ERR_ARG;
    }
    if (mode == SPMM_STATIC && !pattern) {
        set_error("static plans need a pattern");
        return SPMM_ERR_ARG;
    }
    spmm_plan *p = new (std::nothrow) spmm_plan();
    if (!p) return SPMM_ERR_OOM;
    p->m = m;
    p->k = k;
    p->n_max = n_max;
    p->col_tiles = o.col_tiles;
    p->b = b;
    p->mode = mode;
    p->wdt = w_dtype;
    p->xdt = x_dtype;
    p->kernel = kernel;
    p->host_only = o.host_only != 0;
    p->sm_count = 152;
    if (!p->host_only) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            free_plan(p);
            return cuda_fail(e, "device query");
        }
    }
    const int64_t mb = m / b, mt = m / kTile;
    try {
        if (mode == SPMM_STATIC) {
            st = validate_pattern(m, k, b, pattern->nnzb, pattern->brow, pattern->bcol);
            if (st != SPMM_OK) {
                free_plan(p);
                return st;
            }
            p->nnzb = pattern->nnzb;
            if (!build_csr_checked(mb, p->nnzb, pattern->brow, pattern->bcol, p->hp)) {
                free_plan(p);
                return SPMM_ERR_PATTERN;
            }
            if (kernel == SPMM_KERNEL_BGATHER) {
                // the block CSR is the whole plan: a CTA per block row
            } else if (kernel == SPMM_KERNEL_GATHER) {
                const int64_t avg = mb ? (p->nnzb + mb - 1) / mb : 0;
                p->C = o.max_per_item ? o.max_per_item : (int)std::max<int64_t>(64, 2 * avg);
                build_row_plan(mb, p->C, true, p->hp);
            } else if (kernel == SPMM_KERNEL_TC) {
                p->groups = o.groups;
                if (!p->groups && !o.rows_per_group && p->sm_count > 0) {
                    // the launch shape the plan will take (two column tiles
                    // per CTA for dense-tile plans), from a 16-row probe
                    // when the two shapes would want different group counts
                    const bool can_wide = o.col_tiles == 2
                                              ? n_max > kNTile
                                              : (w_dtype != SPMM_E4M3 && o.col_tiles != 1 &&
                                                 n_max > kNTile && n_max % 64 == 0);
                    const int64_t qn = auto_groups(mt, n_max, p->sm_count, false);
                    const int64_t qw = can_wide ? auto_groups(mt, n_max, p->sm_count, true) : qn;
                    if (qn == qw) {
                        p->groups = qn;
                    } else {
                        HostPlan g16;
                        build_tc_plan(m, k, b, p->nnzb, pattern->brow, pattern->bcol, kMaxGroupRows,
                                      1 << 30, false, true, g16);
                        const double ent = (double)g16.ent_col.size();
                        const bool dense = ent > 0 && tc_geometry((double)g16.tile_row.size() / ent) == 0;
                        p->groups = (dense || o.col_tiles == 2) ? qw : qn;
                    }
                }
                if (p->groups > 0)
                    p->R = (int)((mt + p->groups - 1) / p->groups);
                else
                    p->R = o.rows_per_group ? o.rows_per_group : default_R(mt, n_max, p->sm_count);
                if (o.max_per_item && !o.k_splits) {
                    p->C = o.max_per_item;
                } else {
                    HostPlan probe;
                    build_tc_plan(m, k, b, p->nnzb, pattern->brow, pattern->bcol, p->R, 1 << 30,
                                  false, false, probe, p->groups);
                    const int64_t G = (int64_t)probe.grp_rows.size();
                    const int64_t E = (int64_t)probe.ent_col.size();
                    if (o.k_splits) {
                        // about k_splits items per group of mean length
                        const int64_t per = G ? (E + G * o.k_splits - 1) / (G * o.k_splits) : 1;
                        p->C = (int)std::max<int64_t>(1, per);
                    } else {
                        // entries per group if spread evenly, with headroom:
                        // only groups well above the mean are split
                        p->C = (int)std::max<int64_t>(16, G ? (5 * E + 4 * G - 1) / (4 * G) : 16);
                    }
                }
                build_tc_plan(m, k, b, p->nnzb, pattern->brow, pattern->bcol, p->R, p->C, true,
                              true, p->hp, p->groups);
            }
            p->n_items = (int64_t)p->hp.items.size() / kItemFields;
            p->n_red = (int64_t)p->hp.red.size() / 3;
            p->n_groups = (int64_t)p->hp.grp_rows.size();
            p->n_entries = (int64_t)p->hp.ent_col.size();
            p->n_tiles = (int64_t)p->hp.tile_row.size();
            if (kernel == SPMM_KERNEL_TC && p->n_entries > 0)
                p->tc_geo = tc_geometry((double)p->n_tiles / (double)p->n_entries);
            if (kernel == SPMM_KERNEL_TC && o.stage_geometry) p->tc_geo = o.stage_geometry - 1;
        } else {
            p->nnzb_max = nnzb_max;
            if (kernel == SPMM_KERNEL_TC) {
                if (k / kTile > kDynMaxTileCols) {
                    set_error("dynamic TC plans need k <= %d", kDynMaxTileCols * kTile);
                    free_plan(p);
                    return SPMM_ERR_UNSUPPORTED;
                }
                // near-equal groups as for static plans (dynamic launches
                // take one column tile per CTA), else the equal partition
                p->groups = o.groups;
                if (!p->groups && !o.rows_per_group)
                    p->groups = auto_groups(mt, n_max, p->sm_count, false);
                if (p->groups > 0)
                    p->R = (int)((mt + p->groups - 1) / p->groups);
                else
                    p->R = o.rows_per_group ? o.rows_per_group : default_R(mt, n_max, p->sm_count);
                const std::vector<int64_t> sz =
                    p->groups > 0 ? near_equal_partition(mt, p->groups) : group_partition(mt, p->R);
                int64_t acc = 0;
                for (int64_t v : sz) {
                    p->hp.grp_row0.push_back((int32_t)acc);
                    p->hp.grp_rows.push_back((int32_t)v);
                    acc += v;
                }
                p->n_groups = (int64_t)sz.size();
                // expected tiles per entry of a random pattern at nnzb_max:
                // a 16 x 16 tile is non-empty with probability q, an entry
                // (column of a group of R tile rows) holds R q / (1 - (1-q)^R)
                const double cells = (double)(m / b) * (double)(k / b);
                const double dm = cells > 0 ? std::min(1.0, (double)nnzb_max / cells) : 0.0;
                const double per = (double)(kTile / b) * (double)(kTile / b);
                const double q = 1.0 - std::pow(1.0 - dm, per);
                const double R = (double)p->R;
                const double hit = 1.0 - std::pow(1.0 - q, R);
                p->tc_geo = tc_geometry(hit > 0 ? R * q / hit : 0.0);
                if (o.stage_geometry) p->tc_geo = o.stage_geometry - 1;
                // one cooperative launch for the re-partition where the device
                // runs cooperative kernels (else the launch chain)
                if (!p->host_only) {
                    int dev = 0;
                    p->dyn_fused = cudaGetDevice(&dev) == cudaSuccess && dyn_fused_supported(dev) &&
                                   !o.dyn_chain;
                }
            } else if (kernel == SPMM_KERNEL_PLAIN) {
                set_error("dynamic plans use the GATHER (b = 1) or TC (b >= 4) kernels");
                free_plan(p);
                return SPMM_ERR_UNSUPPORTED;
            }
        }
    } catch (const std::bad_alloc &) {
        free_plan(p);
        set_error("host allocation failed while planning");
        return SPMM_ERR_OOM;
    }
    if (!p->host_only) {
        st = p->mode == SPMM_STATIC ? upload_plan(p) : alloc_dynamic(p);
        cudaError_t e = cudaSuccess;
        if (st == SPMM_OK) e = dalloc(p, &p->d_status, 1);
        if (st == SPMM_OK && e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int32_t));
        if (st == SPMM_OK && e == cudaSuccess && b == 16) {
            // the gathered SDDMM's work items: at most nnzb / 8 + one per block row
            const int64_t nb = p->mode == SPMM_STATIC ? p->nnzb : p->nnzb_max;
            p->sd_items_cap = nb / 8 + m / 16 + 1;
            e = dalloc(p, &p->d_sd_items, 1 + 3 * p->sd_items_cap);
        }
        if (st == SPMM_OK && e == cudaSuccess && p->hp.ws_rows > 0)
            e = dalloc(p, &p->d_ws, p->hp.ws_rows * std::max<int64_t>(n_max, 1));
        if (st == SPMM_OK && e == cudaSuccess) {
            // packed values: CSR order for PLAIN / GATHER, 16 x 16 tiles for TC
            const int64_t nb = p->mode == SPMM_STATIC ? p->nnzb : p->nnzb_max;
            const int64_t nt = p->mode == SPMM_STATIC ? p->n_tiles : p->nnzb_max;
            if (kernel == SPMM_KERNEL_TC)
                p->packed_bytes = nt * kTile * kTile * (int64_t)dtype_size(w_dtype);
            else
                p->packed_bytes = nb * b * b * (int64_t)dtype_size(w_dtype);
            e = dalloc(p, (char **)&p->d_packed, p->packed_bytes);
            // E4M3 scales: per 4 x 4 sub-square of each tile (TC), per
            // block in CSR order (BGATHER)
            if (e == cudaSuccess && w_dtype == SPMM_E4M3)
                e = dalloc(p, &p->d_tile_scale, kernel == SPMM_KERNEL_TC ? nt * 16 : nb);
        }
        if (st == SPMM_OK && e == cudaSuccess && kernel == SPMM_KERNEL_TC &&
            p->mode == SPMM_STATIC) {
            // the static plan's stage records, once (dynamic plans: every call)
            e = launch_stage_build(p, 0);
            if (e == cudaSuccess) e = cudaStreamSynchronize(0);
        }
        if (st == SPMM_OK && e != cudaSuccess) st = cuda_fail(e, "plan allocation");
        if (st != SPMM_OK) {
            free_plan(p);
            return st;
        }
    }
    *out = p;
    return SPMM_OK;
}

void spmm_plan_destroy(spmm_plan *plan) {
    if (plan && plan->ran && plan->done) cudaEventSynchronize(plan->done);
    free_plan(plan);
}

static bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

// A call inside a stream capture becomes part of a graph: it records no
// completion event and skips the cross-stream check (a graph's replays are
// ordered by the stream they are launched on).
static spmm_status busy_check(spmm_plan *p, cudaStream_t s) {
    if (capturing(s)) return SPMM_OK;
    if (p->ran && p->last_stream != s) {
        cudaError_t q = cudaEventQuery(p->done);
        if (q == cudaErrorNotReady) {
            set_error("plan is in flight on another stream");
            return SPMM_ERR_BUSY;
        }
        if (q != cudaSuccess) return cuda_fail(q, "event query");
    }
    return SPMM_OK;
}

static spmm_status finish_call(spmm_plan *p, cudaStream_t s) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    if (capturing(s)) return SPMM_OK;
    e = cudaEventRecord(p->done, s);
    if (e != cudaSuccess) return cuda_fail(e, "event record");
    p->last_stream = s;
    p->ran = true;
    return SPMM_OK;
}

static spmm_status do_pack(spmm_plan *p, const void *d_values, const float *d_scales,
                           cudaStream_t s) {
    if (p->nnzb > 0 && !d_values) {
        set_error("values required");
        return SPMM_ERR_ARG;
    }
    if (p->wdt == SPMM_E4M3 && p->nnzb > 0 && !d_scales) {
        set_error("E4M3 values need per-block scales");
        return SPMM_ERR_ARG;
    }
    cudaError_t e = cudaSuccess;
    if (p->d_src_index && p->nnzb > 0) {
        // row-slice plan: the kept blocks' values (and E4M3 scales) from the
        // whole W's arrays, in the slice's order
        const int64_t bb = (int64_t)p->b * p->b * (int64_t)dtype_size(p->wdt);
        e = launch_gather_blocks(d_values, p->d_src_index, p->nnzb, bb, p->d_slice_vals, s);
        if (e == cudaSuccess && p->wdt == SPMM_E4M3)
            e = launch_gather_blocks(d_scales, p->d_src_index, p->nnzb, 4, p->d_slice_scales, s);
        if (e != cudaSuccess) return cuda_fail(e, "row-slice gather");
        d_values = p->d_slice_vals;
        if (p->wdt == SPMM_E4M3) d_scales = p->d_slice_scales;
    }
    e = (p->kernel == SPMM_KERNEL_TC) ? launch_pack_tiles(p, d_values, d_scales, nullptr, s)
                                      : launch_pack_csr(p, d_values, nullptr, s);
    if (e == cudaSuccess && p->kernel == SPMM_KERNEL_BGATHER && p->wdt == SPMM_E4M3)
        e = launch_gather_blocks(d_scales, p->d_perm, p->nnzb, 4, p->d_tile_scale, s);
    if (e != cudaSuccess) return cuda_fail(e, "pack");
    p->packed = true;
    return SPMM_OK;
}

spmm_status spmm_pack_values(spmm_plan *plan, const void *d_values, const float *d_scales,
                             void *stream) {
    g_err[0] = 0;
    if (!plan || plan->host_only) {
        set_error("plan is NULL or host-only");
        return SPMM_ERR_ARG;
    }
    if (plan->mode != SPMM_STATIC) {
        set_error("spmm_pack_values is for static plans");
        return SPMM_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    spmm_status st = busy_check(plan, s);
    if (st != SPMM_OK) return st;
    st = do_pack(plan, d_values, d_scales, s);
    if (st != SPMM_OK) return st;
    return finish_call(plan, s);
}

static spmm_status launch_product(spmm_plan *p, const void *d_X, int64_t n, int64_t ldx,
                                  void *d_Y, int64_t ldy, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    switch (p->kernel) {
        case SPMM_KERNEL_PLAIN: e = launch_plain(p, d_X, n, ldx, d_Y, ldy, s); break;
        case SPMM_KERNEL_GATHER: e = launch_gather(p, d_X, n, ldx, d_Y, ldy, s); break;
        case SPMM_KERNEL_TC: e = launch_tc(p, d_X, n, ldx, d_Y, ldy, s); break;
        case SPMM_KERNEL_BGATHER: e = launch_bgather(p, d_X, n, ldx, d_Y, ldy, s); break;
        default: set_error("bad kernel"); return SPMM_ERR_ARG;
    }
    if (e == cudaSuccess && p->n_red > 0 && p->kernel != SPMM_KERNEL_PLAIN)
        e = launch_reduce(p, n, d_Y, ldy, s);
    if (e != cudaSuccess) return cuda_fail(e, "launch");
    return SPMM_OK;
}

// dev_x: X is the caller's device array that the kernels read in place
// (TMA alignment applies); false where the library stages X itself.
static spmm_status check_run_args(spmm_plan *p, const void *d_X, int64_t n, int64_t ldx,
                                  const void *d_Y, int64_t ldy, bool dev_x = true) {
    if (n < 0 || n > p->n_max) {
        set_error("n=%lld outside [0, n_max=%lld]", (long long)n, (long long)p->n_max);
        return SPMM_ERR_SHAPE;
    }
    if (ldx < std::max<int64_t>(n, 1) || ldy < std::max<int64_t>(n, 1)) {
        set_error("ldx/ldy must be >= max(n, 1)");
        return SPMM_ERR_SHAPE;
    }
    if (n > 0 && (!d_X || !d_Y)) {
        set_error("X and Y required");
        return SPMM_ERR_ARG;
    }
    if (dev_x && n > 0 && p->kernel == SPMM_KERNEL_TC && ((uintptr_t)d_X % 16 || ldx % 8)) {
        set_error("tensor-core plans read X by TMA: X must be 16-byte aligned with ldx a "
                  "multiple of 8 (ldx=%lld)", (long long)ldx);
        return SPMM_ERR_UNSUPPORTED;
    }
    return SPMM_OK;
}

spmm_status spmm_run(spmm_plan *plan, const void *d_values, const float *d_scales,
                     const spmm_dpattern *dpat, const void *d_X, int64_t n, int64_t ldx, void *d_Y,
                     int64_t ldy, void *stream) {
    g_err[0] = 0;
    if (!plan || plan->host_only) {
        set_error("plan is NULL or host-only");
        return SPMM_ERR_ARG;
    }
    spmm_status st = check_run_args(plan, d_X, n, ldx, d_Y, ldy);
    if (st != SPMM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = busy_check(plan, s);
    if (st != SPMM_OK) return st;
    if (plan->mode == SPMM_DYNAMIC) {
        if (!dpat || !dpat->d_nnzb || !dpat->d_brow || !dpat->d_bcol || !d_values) {
            set_error("dynamic runs need a device pattern and values");
            return SPMM_ERR_ARG;
        }
        if (plan->wdt == SPMM_E4M3 && !d_scales) {
            set_error("E4M3 values need per-block scales");
            return SPMM_ERR_ARG;
        }
        // a transposed plan reads W's pattern with rows and columns swapped
        const spmm_dpattern tdp{dpat->d_nnzb, dpat->d_bcol, dpat->d_brow};
        const spmm_dpattern *pp = plan->transposed ? &tdp : dpat;
        cudaError_t e = cudaSuccess;
        if (plan->dyn_fused) {
            // re-partition, packing and stage records in one cooperative launch
            e = launch_dynamic_tc_fused(plan, pp, d_values, d_scales, s);
        } else {
            e = launch_dynamic_partition(plan, pp, s);
            if (e == cudaSuccess)
                e = plan->kernel == SPMM_KERNEL_TC
                        ? launch_pack_tiles(plan, d_values, d_scales, dpat->d_nnzb, s)
                        : launch_pack_csr(plan, d_values, dpat->d_nnzb, s);
        }
        if (e != cudaSuccess) return cuda_fail(e, "dynamic re-partition");
        if (n > 0) {
            st = launch_product(plan, d_X, n, ldx, d_Y, ldy, s);
            if (st != SPMM_OK) return st;
            // the product's reduction launch cleared the fused launch's
            // barrier words for the next call
            if (plan->dyn_fused) plan->dyn.bar_clean = plan->n_red > 0;
        } else if (plan->dyn_fused) {
            e = cudaMemsetAsync(plan->dyn.bar, 0, sizeof(int32_t) * 2, s);
            if (e != cudaSuccess) return cuda_fail(e, "barrier reset");
            plan->dyn.bar_clean = true;
        }
        return finish_call(plan, s);
    }
    if (d_values) {
        st = do_pack(plan, d_values, d_scales, s);
        if (st != SPMM_OK) return st;
    }
    if (!plan->packed) {
        set_error("static plan has no values: call spmm_pack_values or pass d_values");
        return SPMM_ERR_NOT_PACKED;
    }
    if (n == 0) return finish_call(plan, s);
    st = launch_product(plan, d_X, n, ldx, d_Y, ldy, s);
    if (st != SPMM_OK) return st;
    return finish_call(plan, s);
}

spmm_status spmm_run_host(spmm_plan *plan, const void *h_X, int64_t n, int64_t ldx, void *h_Y,
                          int64_t ldy, void *stream) {
    g_err[0] = 0;
    if (!plan || plan->host_only || plan->mode != SPMM_STATIC) {
        set_error("spmm_run_host needs a device static plan");
        return SPMM_ERR_ARG;
    }
    spmm_status st = check_run_args(plan, h_X, n, ldx, h_Y, ldy, false);
    if (st != SPMM_OK) return st;
    if (!plan->packed) {
        set_error("static plan has no values");
        return SPMM_ERR_NOT_PACKED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    st = busy_check(plan, s);
    if (st != SPMM_OK) return st;
    const size_t es = dtype_size(plan->xdt);
    // the staged X's rows: 16-byte aligned for the tensor-core kernel's TMA
    const int64_t xld = plan->kernel == SPMM_KERNEL_TC ? (std::max<int64_t>(n, 1) + 7) / 8 * 8
                                                       : std::max<int64_t>(n, 1);
    const int64_t xb = plan->k * xld * (int64_t)es;
    const int64_t yb = plan->m * std::max<int64_t>(n, 1) * (int64_t)es;
    cudaError_t e = cudaSuccess;
    if (xb > plan->xbuf_bytes) {
        if (plan->d_xbuf) {
            cudaFree(plan->d_xbuf);
            plan->allocations.erase(std::find(plan->allocations.begin(), plan->allocations.end(), plan->d_xbuf));
            plan->device_bytes -= plan->xbuf_bytes;
        }
        e = dalloc(plan, (char **)&plan->d_xbuf, xb);
        plan->xbuf_bytes = e == cudaSuccess ? xb : 0;
    }
    if (e == cudaSuccess && yb > plan->ybuf_bytes) {
        if (plan->d_ybuf) {
            cudaFree(plan->d_ybuf);
            plan->allocations.erase(std::find(plan->allocations.begin(), plan->allocations.end(), plan->d_ybuf));
            plan->device_bytes -= plan->ybuf_bytes;
        }
        e = dalloc(plan, (char **)&plan->d_ybuf, yb);
        plan->ybuf_bytes = e == cudaSuccess ? yb : 0;
    }
    if (e != cudaSuccess) return cuda_fail(e, "staging allocation");
    if (n > 0) {
        // one contiguous copy when the host rows are dense (a pitched copy
        // moves k short rows one by one)
        e = (ldx == n && xld == n)
                ? cudaMemcpyAsync(plan->d_xbuf, h_X, plan->k * n * es, cudaMemcpyHostToDevice, s)
                : cudaMemcpy2DAsync(plan->d_xbuf, xld * es, h_X, ldx * es, n * es, plan->k,
                                    cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "X upload");
        st = launch_product(plan, plan->d_xbuf, n, xld, plan->d_ybuf, n, s);
        if (st != SPMM_OK) return st;
        e = ldy == n ? cudaMemcpyAsync(h_Y, plan->d_ybuf, plan->m * n * es, cudaMemcpyDeviceToHost, s)
                     : cudaMemcpy2DAsync(h_Y, ldy * es, plan->d_ybuf, n * es, n * es, plan->m,
                                         cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "Y download");
    }
    st = finish_call(plan, s);
    if (st != SPMM_OK) return st;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    return SPMM_OK;
}

spmm_status spmm_plan_set_wait(spmm_plan *plan, int64_t limit_ns, int32_t stall) {
    g_err[0] = 0;
    if (!plan || limit_ns < 0 || (stall != 0 && stall != 1)) {
        set_error("set_wait: plan required, limit_ns >= 0, stall 0 or 1");
        return SPMM_ERR_ARG;
    }
    plan->wait_ns = (uint64_t)limit_ns;
    plan->stall = stall;
    return SPMM_OK;
}

spmm_status spmm_get_status(spmm_plan *plan, int32_t *device_status) {
    g_err[0] = 0;
    if (!plan || !device_status || plan->host_only) {
        set_error("plan (device) and device_status required");
        return SPMM_ERR_ARG;
    }
    *device_status = 0;
    if (plan->ran) {
        cudaError_t e = cudaEventSynchronize(plan->done);
        if (e != cudaSuccess) return cuda_fail(e, "event synchronize");
    }
    cudaError_t e = cudaMemcpy(device_status, plan->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(plan->d_status, 0, sizeof(int32_t));
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    return SPMM_OK;
}

spmm_status spmm_plan_get_info(const spmm_plan *cp, spmm_plan_info *info) {
    if (!cp || !info) {
        set_error("plan and info required");
        return SPMM_ERR_ARG;
    }
    spmm_plan *p = const_cast<spmm_plan *>(cp);
    if (p->mode == SPMM_DYNAMIC && p->ran) {
        spmm_status rs = refresh_dynamic(p);
        if (rs != SPMM_OK) return rs;
    }
    spmm_plan_info i{};
    i.m = p->m;
    i.k = p->k;
    i.n_max = p->n_max;
    i.nnzb = p->nnzb;
    i.nnzb_max = p->nnzb_max;
    i.b = p->b;
    i.mode = p->mode;
    i.w_dtype = p->wdt;
    i.x_dtype = p->xdt;
    i.kernel = p->kernel;
    i.rows_per_group = p->groups > 0 ? 0 : p->R;
    i.max_per_item = p->C;
    const bool dynran = p->mode == SPMM_DYNAMIC && p->ran;
    i.n_items = dynran ? p->dyn_items : p->n_items;
    i.n_groups = p->n_groups;
    i.n_entries = p->n_entries;
    i.n_tiles = p->n_tiles;
    i.ws_rows = dynran ? p->dyn_ws_rows : p->hp.ws_rows;
    i.n_reductions = dynran ? p->dyn_red : p->n_red;
    i.device_bytes = p->device_bytes;
    i.stage_geometry = p->kernel == SPMM_KERNEL_TC ? p->tc_geo : 0;
    i.col_tiles = p->kernel == SPMM_KERNEL_TC ? p->col_tiles : 0;
    i.index_bytes = col16_plan(p) ? 2 : 4;
    i.sddmm_form = sddmm_gathers(p) ? 1 : 0;
    i.row_begin = p->row_end ? p->row_begin : 0;
    i.row_end = p->row_end ? p->row_end : p->m;
    *info = i;
    return SPMM_OK;
}

spmm_status spmm_plan_get_array(spmm_plan *p, spmm_array which, void *dst, int64_t capacity,
                                int64_t *count) {
    g_err[0] = 0;
    if (!p || !count) {
        set_error("plan and count required");
        return SPMM_ERR_ARG;
    }
    spmm_status rs = refresh_dynamic(p);
    if (rs != SPMM_OK) return rs;
    const HostPlan &hp = p->hp;
    const void *src = nullptr;
    int64_t n = 0;
    size_t es = 4;
    switch (which) {
        case SPMM_ARR_ROW_PTR: src = hp.row_ptr.data(); n = hp.row_ptr.size(); break;
        case SPMM_ARR_COL_IDX: src = hp.col_idx.data(); n = hp.col_idx.size(); break;
        case SPMM_ARR_PERM: src = hp.perm.data(); n = hp.perm.size(); break;
        case SPMM_ARR_ITEMS: src = hp.items.data(); n = hp.items.size(); break;
        case SPMM_ARR_GRP_ROW0: src = hp.grp_row0.data(); n = hp.grp_row0.size(); break;
        case SPMM_ARR_GRP_ROWS: src = hp.grp_rows.data(); n = hp.grp_rows.size(); break;
        case SPMM_ARR_GRP_EBEG: src = hp.grp_ebeg.data(); n = hp.grp_ebeg.size(); break;
        case SPMM_ARR_ENT_COL: src = hp.ent_col.data(); n = hp.ent_col.size(); break;
        case SPMM_ARR_ENT_TBEG: src = hp.ent_tbeg.data(); n = hp.ent_tbeg.size(); break;
        case SPMM_ARR_TILE_ROW: src = hp.tile_row.data(); n = hp.tile_row.size(); break;
        case SPMM_ARR_BLK_SLOT: src = hp.blk_slot.data(); n = hp.blk_slot.size(); break;
        case SPMM_ARR_BLK_OFF: src = hp.blk_off.data(); n = hp.blk_off.size(); break;
        case SPMM_ARR_WS_ROW0: src = hp.ws_row0.data(); n = hp.ws_row0.size(); es = 8; break;
        case SPMM_ARR_RED: src = hp.red.data(); n = hp.red.size(); break;
        case SPMM_ARR_ENT_COVER: src = hp.ent_cover.data(); n = hp.ent_cover.size(); break;
        case SPMM_ARR_SRC_INDEX: src = p->src_index.data(); n = p->src_index.size(); break;
        default: set_error("unknown array %d", (int)which); return SPMM_ERR_ARG;
    }
    *count = n;
    if (!dst) return SPMM_OK;
    if (capacity < n) {
        set_error("capacity %lld < %lld", (long long)capacity, (long long)n);
        return SPMM_ERR_ARG;
    }
    if (n) memcpy(dst, src, (size_t)n * es);
    return SPMM_OK;
}

spmm_status spmm_batch_run(int32_t count, spmm_plan *const *plans, const void *const *d_X,
                           const int64_t *n, const int64_t *ldx, void *const *d_Y,
                           const int64_t *ldy, void *stream) {
    g_err[0] = 0;
    if (count <= 0 || count > kMaxBatchProblems || !plans || !d_X || !n || !d_Y) {
        set_error("batch: 1 <= count <= %d and plans, X, n, Y required", kMaxBatchProblems);
        return SPMM_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < count; ++i) {
        spmm_plan *p = plans[i];
        if (!p || p->host_only || p->mode != SPMM_STATIC ||
            (p->kernel != SPMM_KERNEL_TC && p->kernel != SPMM_KERNEL_BGATHER)) {
            set_error("batch: problem %d is not a device static TC or BGATHER plan", i);
            return SPMM_ERR_UNSUPPORTED;
        }
        if (p->xdt != plans[0]->xdt || p->wdt != plans[0]->wdt) {
            set_error("batch: all problems must share W and X types");
            return SPMM_ERR_UNSUPPORTED;
        }
        if (!p->packed) {
            set_error("batch: problem %d has no packed values", i);
            return SPMM_ERR_NOT_PACKED;
        }
        const int64_t lx = ldx ? ldx[i] : n[i], ly = ldy ? ldy[i] : n[i];
        spmm_status st = check_run_args(p, d_X[i], n[i], lx, d_Y[i], ly);
        if (st != SPMM_OK) return st;
        st = busy_check(p, s);
        if (st != SPMM_OK) return st;
        for (int j = 0; j < i; ++j)
            if (plans[j] == p) {
                set_error("batch: a plan may appear once per launch");
                return SPMM_ERR_ARG;
            }
    }
    // the small-n problems (BGATHER) in one launch first, then the
    // tensor-core ones (one launch, or two when some plans take two column
    // tiles per CTA)
    spmm_plan *gp[kMaxBatchProblems], *tp[kMaxBatchProblems];
    const void *gx[kMaxBatchProblems], *tx[kMaxBatchProblems];
    void *gy[kMaxBatchProblems], *ty[kMaxBatchProblems];
    int64_t gn[kMaxBatchProblems], tn[kMaxBatchProblems], glx[kMaxBatchProblems],
        tlx[kMaxBatchProblems], gly[kMaxBatchProblems], tly[kMaxBatchProblems];
    int ng = 0, nt = 0;
    for (int i = 0; i < count; ++i) {
        const int64_t lx = ldx ? ldx[i] : n[i], ly = ldy ? ldy[i] : n[i];
        if (plans[i]->kernel == SPMM_KERNEL_BGATHER) {
            gp[ng] = plans[i], gx[ng] = d_X[i], gy[ng] = d_Y[i], gn[ng] = n[i];
            glx[ng] = lx, gly[ng] = ly;
            ++ng;
        } else {
            tp[nt] = plans[i], tx[nt] = d_X[i], ty[nt] = d_Y[i], tn[nt] = n[i];
            tlx[nt] = lx, tly[nt] = ly;
            ++nt;
        }
    }
    cudaError_t e = cudaSuccess;
    if (ng) e = launch_bgather_batch(ng, gp, gx, gn, glx, gy, gly, s);
    if (e == cudaSuccess && nt) e = launch_tc_batch(nt, tp, tx, tn, tlx, ty, tly, s, true);
    if (e != cudaSuccess) return cuda_fail(e, "batched launch");
    for (int i = 0; i < count; ++i) {
        spmm_plan *p = plans[i];
        if (p->kernel == SPMM_KERNEL_TC && p->n_red > 0 && n[i] > 0) {
            e = launch_reduce(p, n[i], d_Y[i], ldy ? ldy[i] : n[i], s);
            if (e != cudaSuccess) return cuda_fail(e, "batched reduction");
        }
        spmm_status st = finish_call(p, s);
        if (st != SPMM_OK) return st;
    }
    return SPMM_OK;
}

spmm_status spmm_quantize_e4m3(int64_t nnzb, int32_t b, spmm_dtype src_dtype, const void *d_src,
                               uint8_t *d_codes, float *d_scales, void *stream) {
    g_err[0] = 0;
    if (nnzb < 0 || !(b == 1 || b == 4 || b == 8 || b == 16) ||
        (nnzb > 0 && (!d_src || !d_codes || !d_scales)) ||
        !(src_dtype == SPMM_F32 || src_dtype == SPMM_F16 || src_dtype == SPMM_BF16)) {
        set_error("quantize: nnzb >= 0, b in {1,4,8,16}, F32/F16/BF16 source and buffers required");
        return SPMM_ERR_ARG;
    }
    cudaError_t e = launch_quantize_e4m3(nnzb, b, src_dtype, d_src, d_codes, d_scales,
                                         (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "quantize");
    return SPMM_OK;
}

spmm_status spmm_run_ell(spmm_plan *plan, const int32_t *d_ell_cols, int32_t ell_width,
                         const void *d_values, const void *d_X, int64_t n, int64_t ldx,
                         void *d_Y, int64_t ldy, void *stream) {
    g_err[0] = 0;
    if (!plan || plan->host_only || plan->mode != SPMM_DYNAMIC || plan->transposed ||
        plan->b != 16 || plan->kernel != SPMM_KERNEL_TC || plan->wdt != plan->xdt) {
        set_error("ell: needs a dynamic, untransposed b = 16 tensor-core plan with w = x dtype");
        return SPMM_ERR_UNSUPPORTED;
    }
    if (ell_width < 0 || ell_width > plan->k / 16) {
        set_error("ell: ell_width must be in [0, k/16]");
        return SPMM_ERR_SHAPE;
    }
    spmm_status st = check_run_args(plan, d_X, n, ldx, d_Y, ldy, false);
    if (st != SPMM_OK) return st;
    if (ell_width > 0 && (!d_ell_cols || !d_values || (uintptr_t)d_values % 16)) {
        set_error("ell: columns and 16-byte aligned values required");
        return SPMM_ERR_ARG;
    }
    if (n > 0 && ((uintptr_t)d_X % 16 || ldx % 8)) {
        set_error("ell: X must be 16-byte aligned with ldx a multiple of 8");
        return SPMM_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    st = busy_check(plan, s);
    if (st != SPMM_OK) return st;
    const cudaError_t e =
        launch_ell(plan, d_ell_cols, ell_width, d_values, d_X, n, ldx, d_Y, ldy, s);
    if (e != cudaSuccess) return cuda_fail(e, "ell");
    return finish_call(plan, s);
}

spmm_status spmm_sddmm(spmm_plan *plan, const spmm_dpattern *pattern, const void *d_dY,
                       int64_t lddy, const void *d_X, int64_t ldx, int64_t n, void *d_dW,
                       spmm_dtype dw_dtype, void *stream) {
    g_err[0] = 0;
    if (!plan || plan->host_only || plan->transposed) {
        set_error("sddmm: plan is NULL, host-only or transposed");
        return SPMM_ERR_ARG;
    }
    if (!(plan->xdt == SPMM_F16 || plan->xdt == SPMM_BF16)) {
        set_error("sddmm: the plan's x_dtype must be F16 or BF16");
        return SPMM_ERR_UNSUPPORTED;
    }
    if (!(dw_dtype == SPMM_F32 || dw_dtype == plan->xdt)) {
        set_error("sddmm: dw_dtype must be F32 or the plan's x_dtype");
        return SPMM_ERR_ARG;
    }
    if (n < 0 || lddy < std::max<int64_t>(n, 1) || ldx < std::max<int64_t>(n, 1) || lddy % 8 ||
        ldx % 8) {
        set_error("sddmm: n >= 0, lddy and ldx >= max(n, 1) and multiples of 8 elements");
        return SPMM_ERR_ARG;
    }
    if (!d_dW || (n > 0 && (!d_dY || !d_X)) ||
        ((uintptr_t)d_dY | (uintptr_t)d_X | (uintptr_t)d_dW) % 16) {
        set_error("sddmm: dW (and for n > 0 dY and X) required, 16-byte aligned");
        return SPMM_ERR_ARG;
    }
    const bool dyn = plan->mode == SPMM_DYNAMIC;
    if (dyn != (pattern != nullptr) ||
        (dyn && (!pattern->d_nnzb || !pattern->d_brow || !pattern->d_bcol))) {
        set_error("sddmm: dynamic plans need the step's device pattern, static plans none");
        return SPMM_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    spmm_status st = busy_check(plan, s);
    if (st != SPMM_OK) return st;
    if (!dyn && plan->nnzb == 0) return finish_call(plan, s);
    cudaError_t e = dyn ? launch_dynamic_csr(plan, pattern, s) : cudaSuccess;
    if (e == cudaSuccess) e = launch_sddmm(plan, d_dY, lddy, d_X, ldx, n, d_dW, dw_dtype, s);
    if (e != cudaSuccess) return cuda_fail(e, "sddmm");
    return finish_call(plan, s);
}

}  // extern "C"
