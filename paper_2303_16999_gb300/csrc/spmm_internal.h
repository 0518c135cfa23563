// Internal declarations shared by the host planner, the C ABI and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/spmm.h"

namespace spmm {

constexpr int kTile = 16;          // tensor-core tile edge (one MMA K step, one N step)
constexpr int kTileBytes16 = 512;  // 16 x 16 16-bit tile in the MMA operand layout
constexpr int kNTile = 128;        // n columns per tensor-core work unit (MMA M)
constexpr int kMaxGroupRows = 16;  // tile rows per group: 2 x 16 x 16 TMEM columns = 512
constexpr int kItemFields = 6;     // group/row, begin, end, chunk, n_chunks, ws_slot
constexpr int kDynMaxTileCols = 4096;  // dynamic TC plans: k <= 65536 (per-group smem bitmaps)

// dynamic plans: device-side counters written by the re-partition
enum CountIdx : int {
    kCntNnzb = 0,     // blocks of this call (clamped to capacity)
    kCntItems = 1,    // work items
    kCntEntries = 2,  // TC entries
    kCntSlots = 3,    // TC tile slots
    kCntWsSlots = 4,  // workspace slots (split items)
    kCntWsRows = 5,   // workspace rows
    kCntRed = 6,      // split groups / rows to reduce
    kCntChunk = 7,    // chunk size C chosen on the device
    kCntTicketRows = 8,    // blocks done with the row histogram (the last one scans)
    kCntTicketGroups = 9,  // blocks done with the group counts (the last one scans)
    kCntFlags = 10,        // errors found by the row histogram's blocks (bit 0 capacity, bit 1 pattern)
    kCntCount = 11
};

// device status word codes (mirrors spmm_status where applicable)
enum DeviceStatus : int32_t {
    kDevOk = 0,
    kDevPattern = SPMM_ERR_PATTERN,
    kDevCapacity = SPMM_ERR_CAPACITY,
    kDevTimeout = SPMM_ERR_TIMEOUT,
    kDevBadPlan = SPMM_ERR_CUDA,   // stage records inconsistent with the work items
};

void set_error(const char *fmt, ...);

// ---------------------------------------------------------------- host plan
struct HostPlan {
    // canonical block-CSR
    std::vector<int32_t> row_ptr, col_idx, perm;
    // work items (row items for GATHER, group items for TC), kItemFields each
    std::vector<int32_t> items;
    std::vector<int64_t> ws_row0;
    int64_t ws_rows = 0;
    std::vector<int32_t> red;  // 3 per split group/row
    // tensor-core tile structure
    std::vector<int32_t> grp_row0, grp_rows, grp_ebeg, ent_col, ent_tbeg, ent_cover, tile_row,
        blk_slot, blk_off;
};

// Validates shape and pattern; returns SPMM_OK, SPMM_ERR_SHAPE or SPMM_ERR_PATTERN.
spmm_status validate_pattern(int64_t m, int64_t k, int b, int64_t nnzb, const int32_t *brow,
                             const int32_t *bcol);
void build_csr(int64_t mb, int64_t nnzb, const int32_t *brow, const int32_t *bcol, HostPlan &hp);
std::vector<int64_t> group_partition(int64_t mt, int64_t R);
// mt tile rows in q groups whose sizes differ by at most one (larger first)
std::vector<int64_t> near_equal_partition(int64_t mt, int64_t q);
void build_row_plan(int64_t mb, int64_t C1, bool sort_items, HostPlan &hp);
// groups > 0: the tile rows in that many near-equal groups, else the
// equal partition with at most R rows per group
void build_tc_plan(int64_t m, int64_t k, int b, int64_t nnzb, const int32_t *brow,
                   const int32_t *bcol, int64_t R, int64_t C, bool sort_items, bool pad,
                   HostPlan &hp, int64_t groups = 0);

// ------------------------------------------------------------------- plan
// dynamic plans: scratch of the device re-partition
struct DynBufs {
    int32_t *row_cnt = nullptr, *cursor = nullptr, *tmp_col = nullptr, *tmp_perm = nullptr;
    int32_t *row_ibeg = nullptr, *row_wbeg = nullptr, *row_rbeg = nullptr;
    int32_t *grp_cnt = nullptr, *grp_sbeg = nullptr, *grp_ibeg = nullptr, *grp_wbeg = nullptr,
            *grp_rbeg = nullptr;
    int64_t *grp_wrow = nullptr;
    // fused re-partition (dynamic TC): block-column bitmap of every block
    // row (mb x ceil(kb/32) words), the groups' column masks (G x kt words)
    // and the grid barrier's arrival counter and generation word
    uint32_t *bits = nullptr, *gmask = nullptr;
    int32_t *wpre = nullptr;   // per bitmap word: blocks before it in row-major order
    int32_t *bar = nullptr;
    // host: the barrier words are zero in stream order (the last call's
    // reduction launch, or a memset after a call without a product, cleared
    // them); else the next fused launch clears them first
    bool bar_clean = false;
    // host: bar[2..3] (the Blocked-ELL validation's flag and ticket) were
    // zeroed once; the validation launch leaves them zero
    bool ell_clean = false;
    // host: the launch chain's row counts, tickets and error flags are zero
    // (the chain's own launches leave them so); else its first launch is
    // preceded by memsets
    bool chain_clean = false;
    int64_t items_cap = 0, ws_slots_cap = 0, red_cap = 0;
};
constexpr int kFusedMaxCtas = 128;           // CTAs of the fused re-partition (at most)
constexpr int64_t kFusedMaxBitmapWords = 1 << 22;  // 16 MB of block-column bitmap at most

}  // namespace spmm

struct spmm_plan {
    int64_t m = 0, k = 0, n_max = 0, nnzb = 0, nnzb_max = 0;
    int b = 0;
    spmm_mode mode = SPMM_STATIC;
    spmm_dtype wdt = SPMM_F32, xdt = SPMM_F32;
    int kernel = SPMM_KERNEL_AUTO;
    int R = 0, C = 0;
    bool host_only = false;
    spmm::HostPlan hp;

    // device copies (static) / device-built arrays (dynamic)
    int32_t *d_row_ptr = nullptr, *d_col_idx = nullptr, *d_perm = nullptr, *d_items = nullptr,
            *d_red = nullptr, *d_grp_row0 = nullptr, *d_grp_rows = nullptr, *d_ent_col = nullptr,
            *d_ent_tbeg = nullptr, *d_ent_cover = nullptr, *d_tile_row = nullptr, *d_blk_slot = nullptr,
            *d_blk_off = nullptr, *d_grp_ebeg = nullptr;
    uint32_t *d_srec = nullptr, *d_sprog = nullptr;  // TC: stage records and MMA programs
    uint16_t *d_col16 = nullptr;   // static GATHER plans, k <= 65536: col_idx in 16 bits
    // TC, batched with plans of the other stage geometry: this plan's stage
    // records cut for that geometry (built on first use), geometry alt_geo
    uint32_t *d_srec_alt = nullptr, *d_sprog_alt = nullptr;
    int alt_geo = -1;
    int tc_geo = 0;                // TC stage geometry: 0 dense tiles, 1 sparse tiles
    int col_tiles = 0;             // TC: column tiles per CTA, 0 automatic (launch-time choice)
    int64_t groups = 0;            // static TC: near-equal tile-row groups (0: equal partition by R)
    bool transposed = false;       // applies W^T: values arrive as W's blocks, packed transposed
    int32_t *d_sd_items = nullptr; // b = 16: SDDMM work items (count, then (row, e0, e1) triples)
    int64_t sd_items_cap = 0;
    int64_t *d_ws_row0 = nullptr;
    int64_t n_items = 0, n_groups = 0, n_entries = 0, n_tiles = 0, n_red = 0;
    void *d_packed = nullptr;      // packed values (kernel layout)
    float *d_tile_scale = nullptr; // E4M3: per-element-block scales in tile layout
    int64_t packed_bytes = 0;
    bool packed = false;
    float *d_ws = nullptr;         // split-row partials, ws_rows x n_max FP32
    int32_t *d_status = nullptr;   // device status word
    int32_t *d_counts = nullptr;   // dynamic: device counters (n_items, n_entries, ...)
    void *d_scratch = nullptr;     // dynamic: re-partition scratch
    int64_t scratch_bytes = 0;
    spmm::DynBufs dyn;
    int64_t dyn_ws_rows = 0, dyn_items = 0, dyn_red = 0;  // counts of the last dynamic call
    void *d_xbuf = nullptr, *d_ybuf = nullptr;  // spmm_run_host staging
    int64_t xbuf_bytes = 0, ybuf_bytes = 0;
    int64_t device_bytes = 0;
    int sm_count = 0;
    // row-slice plans: the slice of output rows and, for each kept block (the
    // slice's pattern order), its index in the whole pattern; values are
    // gathered into d_slice_vals (and E4M3 scales into d_slice_scales)
    // before packing
    int64_t row_begin = 0, row_end = 0;
    std::vector<int32_t> src_index;
    int32_t *d_src_index = nullptr;
    void *d_slice_vals = nullptr;
    float *d_slice_scales = nullptr;
    bool dyn_fused = false;        // dynamic TC: re-partition, packing and stage records in one
                                   // cooperative launch (else the launch chain)
    uint64_t wait_ns = 0;          // TC launches: limit of each device wait (0: 2 s)
    int32_t stall = 0;             // TC launches: failure-detection test hook (see spmm.h)
    cudaStream_t last_stream = nullptr;
    cudaEvent_t done = nullptr;
    bool ran = false;
    std::vector<void *> allocations;
};

namespace spmm {

// kernel launchers (return cudaSuccess or the launch error)
cudaError_t launch_pack_csr(const spmm_plan *p, const void *d_values, const int32_t *d_nnzb,
                            cudaStream_t s);
// dst block q = src block idx[q], nblk blocks of block_bytes bytes each
cudaError_t launch_gather_blocks(const void *src, const int32_t *idx, int64_t nblk,
                                 int64_t block_bytes, void *dst, cudaStream_t s);
cudaError_t launch_pack_tiles(const spmm_plan *p, const void *d_values, const float *d_scales,
                              const int32_t *d_nnzb, cudaStream_t s);
cudaError_t launch_plain(const spmm_plan *p, const void *d_X, int64_t n, int64_t ldx, void *d_Y,
                         int64_t ldy, cudaStream_t s);
cudaError_t launch_gather(const spmm_plan *p, const void *d_X, int64_t n, int64_t ldx, void *d_Y,
                          int64_t ldy, cudaStream_t s);
// dense rows (ld = n) of 2- or 4-byte values -> stride ld, on the device
cudaError_t launch_restride(const void *src, void *dst, int64_t rows, int64_t n, int64_t ld,
                            size_t elem, cudaStream_t s);
// TC stage records of every work item (plan arrays only; no values)
cudaError_t launch_stage_build(const spmm_plan *p, cudaStream_t s);
// entries (X slabs) and W tiles per stage of the plan's stage geometry
void stage_caps(const spmm_plan *p, int *ent_cap, int *tiles_cap);
// the device can run the fused dynamic re-partition (cooperative launches)
bool dyn_fused_supported(int dev);
int64_t stage_record_words();
// TC stage geometry for a plan whose entries hold this many tiles on average
int tc_geometry(double tiles_per_entry);
int64_t stage_prog_words();
cudaError_t launch_tc(const spmm_plan *p, const void *d_X, int64_t n, int64_t ldx, void *d_Y,
                      int64_t ldy, cudaStream_t s);
cudaError_t launch_reduce(const spmm_plan *p, int64_t n, void *d_Y, int64_t ldy, cudaStream_t s);
cudaError_t launch_tc_batch(int count, spmm_plan *const *plans, const void *const *X,
                            const int64_t *n, const int64_t *ldx, void *const *Y,
                            const int64_t *ldy, cudaStream_t s, bool schedule);
cudaError_t launch_quantize_e4m3(int64_t nnzb, int b, spmm_dtype src, const void *d_src,
                                 uint8_t *d_codes, float *d_scales, cudaStream_t s);
constexpr int kMaxBatchProblems = 64;
constexpr int kBgMaxBatch = 64;    // BGATHER problems per launch
constexpr int kBgMaxN = 16;        // BGATHER: largest n
constexpr int kBgAutoMaxN = 16;    // AUTO picks BGATHER (b = 4, 8, static) up to this n_max
constexpr int kBgAutoMaxN16 = 8;   // ... and for b = 16 up to this one
// the autotuner's choice for a static product's bucket (tune.cpp)
bool tune_lookup(int64_t m, int64_t k, int b, int64_t nnzb, int64_t n, spmm_dtype w, spmm_dtype x,
                 spmm_tune_choice *out);
// BGATHER (k_bgather.cu): CUDA-core block gather for small n
cudaError_t launch_bgather(const spmm_plan *p, const void *X, int64_t n, int64_t ldx, void *Y,
                           int64_t ldy, cudaStream_t s);
cudaError_t launch_bgather_batch(int count, spmm_plan *const *plans, const void *const *X,
                                 const int64_t *n, const int64_t *ldx, void *const *Y,
                                 const int64_t *ldy, cudaStream_t s);
cudaError_t launch_dynamic_partition(spmm_plan *p, const spmm_dpattern *dp, cudaStream_t s);
// dynamic TC plans: the whole re-partition, the value packing and the stage
// records in one cooperative launch (when p->dyn_fused)
cudaError_t launch_dynamic_tc_fused(spmm_plan *p, const spmm_dpattern *dp, const void *d_values,
                                    const float *d_scales, cudaStream_t s);
// the block CSR part of the re-partition only (row_ptr, col_idx, perm; validation)
cudaError_t launch_dynamic_csr(spmm_plan *p, const spmm_dpattern *dp, cudaStream_t s);
// Blocked-ELL product, b = 16 (k_ell.cu): validation + one product launch
cudaError_t launch_ell(spmm_plan *p, const int32_t *d_cols, int32_t E, const void *d_values,
                       const void *d_X, int64_t n, int64_t ldx, void *d_Y, int64_t ldy,
                       cudaStream_t s);
// sampled dense-dense product on the plan's block CSR (k_sddmm.cu); true when
// spmm_sddmm takes the gathered form on this plan
bool sddmm_gathers(const spmm_plan *p);
cudaError_t launch_sddmm(const spmm_plan *p, const void *d_dY, int64_t lddy, const void *d_X,
                         int64_t ldx, int64_t n, void *d_dW, spmm_dtype dw_dtype, cudaStream_t s);

size_t dtype_size(spmm_dtype t);

}  // namespace spmm
