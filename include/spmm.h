/*
 * spmm.h -- C ABI of the GB300 block-sparse x dense matrix product.
 *
 * Operation (Section 3, unnumbered equation):
 *     Y = (M (.) W) * X,      M_ij = Mhat_{floor(i/b), floor(j/b)}
 * W is m x k and holds its non-zeros in b x b blocks, b in {1, 4, 8, 16}
 * (Section 3.1); X is a dense k x n matrix and Y a dense m x n matrix.
 * Rows of Y whose block row holds no block are written as zeros.
 *
 * Two modes (Section 3.1, Table 1):
 *   SPMM_STATIC  -- the pattern is fixed when the plan is built (Section 3.2).
 *                   The host planner balances work, and the values are
 *                   re-ordered once into the kernel's layout
 *                   (spmm_pack_values), as the paper re-orders host-supplied
 *                   values to its fixed distribution.
 *   SPMM_DYNAMIC -- only the maximum block count is fixed (Section 3.3,
 *                   Appendix A.2).  Every spmm_run takes a device-resident
 *                   pattern and values and re-partitions them on the device.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Layouts.  X is k x n and Y is m x n, row-major, with leading dimensions
 *   ldx >= n and ldy >= n (in elements).  Values are nnzb blocks in the
 *   pattern's order, each b x b row-major (element (i, l) of block p at
 *   values[(p*b + i)*b + l]).  Pattern entry p is block (brow[p], bcol[p]) in
 *   the (m/b) x (k/b) block grid.
 * Types.  W in {F32, F16, BF16, E4M3}; X and Y share one type in {F32, F16,
 *   BF16}.  Products accumulate in FP32; 16-bit outputs are rounded to
 *   nearest-even from FP32.  E4M3 W carries one FP32 scale per block
 *   (value = decode(code) * scale[p]) and needs 16-bit X.
 * Pointers.  "d_" arguments are device pointers, "h_"/host arguments are
 *   host pointers.  `stream` is a cudaStream_t (NULL = legacy default
 *   stream).  Device work is enqueued asynchronously on `stream`.
 * Ownership.  A plan owns its device copies of indices, packed values,
 *   workspace and status word; the caller owns X, Y, values and patterns,
 *   which must stay valid until `stream` has reached the call.
 * Errors.  Argument, shape and host-detected pattern errors are returned
 *   synchronously and nothing is enqueued.  Errors found on the device
 *   (dynamic pattern invalid or over capacity, a bounded wait that timed
 *   out) are recorded in the plan's device status word, Y is left unwritten
 *   for a rejected dynamic pattern, and spmm_get_status reads the word.  No
 *   C++ exception crosses this interface.  spmm_last_error() returns a
 *   thread-local message for the last failing call on the calling thread.
 * Concurrency.  One plan runs on one stream at a time: a call on a second
 *   stream while the plan's previous call is still in flight on another
 *   stream returns SPMM_ERR_BUSY.  Different plans are independent.
 */
#ifndef SPMM_H
#define SPMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPMM_OK = 0,
    SPMM_ERR_ARG = 1,          /* null pointer, negative size, bad enum value */
    SPMM_ERR_SHAPE = 2,        /* b not in {1,4,8,16}; m or k not a multiple of b; n > n_max; ld < n */
    SPMM_ERR_PATTERN = 3,      /* block coordinate out of range, or a block given twice */
    SPMM_ERR_CAPACITY = 4,     /* dynamic: nnzb > nnzb_max (or < 0) */
    SPMM_ERR_UNSUPPORTED = 5,  /* dtype / kernel / alignment combination not provided */
    SPMM_ERR_CUDA = 6,         /* a CUDA runtime call failed; see spmm_last_error() */
    SPMM_ERR_OOM = 7,          /* device or host allocation failed */
    SPMM_ERR_TIMEOUT = 8,      /* a bounded device wait (or serve_wait) ran out */
    SPMM_ERR_BUSY = 9,         /* the plan is in flight on another stream */
    SPMM_ERR_NOT_PACKED = 10   /* static run without values and without spmm_pack_values */
} spmm_status;

typedef enum { SPMM_STATIC = 0, SPMM_DYNAMIC = 1 } spmm_mode;

typedef enum { SPMM_F32 = 0, SPMM_F16 = 1, SPMM_BF16 = 2, SPMM_E4M3 = 3 } spmm_dtype;

/* Kernel family.  AUTO picks, for b = 1: TC for a static plan with 16-bit
 * W = X type, n_max >= 128, m and k multiples of 16 and on average at least
 * 4 non-zeros per non-empty 16 x 16 tile (the tensor cores then beat the
 * gather), else GATHER; for b >= 4: BGATHER for a static plan with 16-bit X,
 * 16-bit or E4M3 W and n_max <= 16 (n_max <= 8 for b = 16; small n: the
 * tensor-core tiles would cost more than the product), else TC for 16-bit
 * or E4M3 W, and PLAIN for FP32 W.  A choice tuned by spmm_tune for the
 * plan's (b, density, n) bucket overrides these rules. */
typedef enum {
    SPMM_KERNEL_AUTO = 0,
    SPMM_KERNEL_PLAIN = 1,   /* plain FP32 CUDA-core kernel: one thread per (row, column), F32 only */
    SPMM_KERNEL_GATHER = 2,  /* b = 1 gather kernel: 128-bit X row loads, warp-shuffle reductions */
    SPMM_KERNEL_TC = 3,      /* b >= 4 tensor-core kernel (tcgen05 + TMEM + TMA), 16-bit X */
    SPMM_KERNEL_BGATHER = 4  /* b in {4, 8, 16} CUDA-core block gather for n <= 16: static plans,
                                16-bit X, W of the same type or E4M3; each block read once in CSR
                                order, FP32 accumulation */
} spmm_kernel;

/* Host pattern (static mode): nnzb entries, block (brow[p], bcol[p]). */
typedef struct {
    int64_t nnzb;
    const int32_t *brow;
    const int32_t *bcol;
} spmm_pattern;

/* Device pattern (dynamic mode): the block count lives on the device
 * (*d_nnzb, read by the kernels, so no host synchronisation is needed);
 * d_brow / d_bcol hold nnzb_max entries of which the first *d_nnzb count. */
typedef struct {
    const int32_t *d_nnzb;
    const int32_t *d_brow;
    const int32_t *d_bcol;
} spmm_dpattern;

/* Planner options; pass NULL for defaults (all fields 0). */
typedef struct {
    int32_t kernel;               /* spmm_kernel */
    int32_t rows_per_group;       /* TC: tile rows (16 rows each) per group, 1..16; 0 = planner's choice */
    int32_t max_per_item;         /* TC: entries per work item; GATHER: blocks per row item; 0 = planner's choice */
    int32_t host_only;            /* 1 = build the static plan on the host only (no device memory, no
                                     CUDA calls): for inspection with spmm_plan_get_array */
    int32_t transposed;           /* 1 = the plan applies W^T: spmm_run computes Z = W^T.Y (Z k x n,
                                     Y m x n) for the W that the pattern and values describe in W's own
                                     coordinates (m x k, blocks row-major); internally the plan is the
                                     block-transposed operand, so plan info and arrays report k x m */
    int32_t col_tiles;            /* TC, static plans: 128-column tiles of n per CTA.  1 = one;
                                     2 = two whenever n > 128 (16-bit or E4M3 weights): the two
                                     tiles share every W stage (and its E4M3 expansion), one CTA
                                     per SM; 0 = automatic (two for 16-bit dense-tile plans with n
                                     a multiple of 64 and enough work units).  Results are
                                     identical either way.  Other values SPMM_ERR_ARG. */
    int64_t groups;               /* TC plans: split the m/16 tile rows into exactly this many
                                     groups of near-equal size (sizes differ by at most one, larger
                                     first; at most 16 rows each), instead of the equal partition with
                                     rows_per_group rows.  0 = planner's choice.  Plan info then
                                     reports rows_per_group = 0 and n_groups = groups.  Not combined
                                     with rows_per_group; SPMM_ERR_ARG if out of range. */
    int32_t stage_geometry;       /* TC plans: the pipeline's stage shape.  0 = by the plan's tiles
                                     per entry (at least 8: dense), 1 = dense-tile stages (few X
                                     slabs, many W tiles), 2 = sparse-tile stages (many slabs, fewer
                                     tiles).  Results are identical either way; other values
                                     SPMM_ERR_ARG. */
    int32_t dyn_chain;            /* dynamic TC plans: 1 = run each call's re-partition, packing and
                                     stage records as a chain of launches instead of one cooperative
                                     launch (identical results; the chain is also what runs where the
                                     device has no cooperative launch).  0 or 1, else SPMM_ERR_ARG. */
    int64_t row_begin, row_end;   /* static plans: a slice of the output rows, rows [row_begin,
                                     row_end) of Y = W.X (of Z = W^T.Y for transposed plans), for
                                     running one product row-split over several GPUs (Section 3.2's
                                     distribution of the non-zeros over workers, X replicated).
                                     Both multiples of b (of 16 for the TC kernel), 0 <= row_begin
                                     < row_end <= m, else SPMM_ERR_SHAPE; 0, 0 = all rows.  The
                                     pattern and values passed are the WHOLE W's: the plan keeps
                                     the blocks of its block rows (in pattern order, rows counted
                                     from row_begin), and spmm_pack_values / spmm_run read each
                                     kept block's values from the whole W's value array.  spmm_run
                                     writes the slice only: Y is (row_end - row_begin) x n.  The
                                     whole pattern is validated (a repeated or out-of-range block
                                     anywhere is SPMM_ERR_PATTERN).  Plan info and arrays describe
                                     the slice (m = row_end - row_begin); spmm_sddmm on a
                                     slice writes the kept blocks in the slice's order.
                                     Dynamic plans: SPMM_ERR_UNSUPPORTED. */
    int32_t k_splits;             /* static TC plans: split every tile-row group's entries (its
                                     tile columns, i.e. its share of k) into about this many work
                                     items of near-equal length, whose FP32 partials the split-row
                                     reduction sums in a fixed order; 0 = only groups well above the
                                     mean length are split.  Overrides max_per_item.  0 .. 1024,
                                     else SPMM_ERR_ARG. */
} spmm_plan_opts;

typedef struct spmm_plan spmm_plan;

/*
 * spmm_plan_create -- builds a plan (Section 3.2 static partitioner /
 * Section 3.3 and Appendix A.2 dynamic planner).
 *   m, k      : W is m x k; both multiples of b, m/b and k/b at most INT32_MAX
 *               (block indices are int32; else SPMM_ERR_SHAPE).
 *   n_max     : largest n any spmm_run of this plan will pass (sizes workspace).
 *   b         : block size, 1, 4, 8 or 16.
 *   mode      : SPMM_STATIC (pattern != NULL, host arrays, nnzb_max ignored)
 *               or SPMM_DYNAMIC (pattern ignored, 0 <= nnzb_max <= INT32_MAX fixes
 *               capacity, else SPMM_ERR_ARG).  A static pattern->nnzb above
 *               INT32_MAX is SPMM_ERR_SHAPE.
 *   w_dtype, x_dtype : see "Types" above.
 *   opts      : NULL or options.
 *   out       : receives the plan (NULL on error).
 * Static patterns are validated here: SPMM_ERR_PATTERN for an out-of-range or
 * repeated block.  The host arrays are read during the call only.
 */
spmm_status spmm_plan_create(int64_t m, int64_t k, int64_t n_max, int32_t b, spmm_mode mode,
                             spmm_dtype w_dtype, spmm_dtype x_dtype,
                             const spmm_pattern *pattern, int64_t nnzb_max,
                             const spmm_plan_opts *opts, spmm_plan **out);

/*
 * spmm_pack_values -- static mode: re-orders the nnzb user-order blocks at
 * d_values (device, w_dtype) into the kernel's layout held by the plan
 * (Section 3.2: host-supplied values re-ordered to the fixed distribution).
 * d_scales: device float[nnzb], one scale per block, E4M3 only (else NULL).
 * Later spmm_run calls may pass d_values = NULL to use the packed copy.
 */
spmm_status spmm_pack_values(spmm_plan *plan, const void *d_values, const float *d_scales,
                             void *stream);

/*
 * spmm_run -- Y = W.X on `stream`.
 *   d_values : static: NULL to use packed values, else user-order values that
 *              are packed first on the same stream.  dynamic: required,
 *              user-order values matching the device pattern.
 *   d_scales : E4M3 per-block scales for d_values (NULL otherwise / if packed).
 *   dpat     : dynamic mode only: the device pattern of this call.
 *   d_X, n, ldx : X (k x n), 0 <= n <= n_max.  Tensor-core plans read X
 *                 by TMA: d_X 16-byte aligned and ldx a multiple of 8, else
 *                 SPMM_ERR_UNSUPPORTED (pad X's rows).
 *   d_Y, ldy    : Y (m x n).
 * In dynamic mode the device validates the pattern; on an invalid pattern or
 * nnzb outside [0, nnzb_max] the status word is set (see spmm_get_status)
 * and Y is not written.
 */
spmm_status spmm_run(spmm_plan *plan, const void *d_values, const float *d_scales,
                     const spmm_dpattern *dpat, const void *d_X, int64_t n, int64_t ldx,
                     void *d_Y, int64_t ldy, void *stream);

/*
 * spmm_run_host -- the same product with X and Y in HOST memory: copies X to
 * a device buffer owned by the plan, runs, copies Y back, and synchronises
 * `stream` before returning.  Static plans with packed values only.
 * h_X is k x n (ldx), h_Y is m x n (ldy), both in x_dtype.
 */
spmm_status spmm_run_host(spmm_plan *plan, const void *h_X, int64_t n, int64_t ldx, void *h_Y,
                          int64_t ldy, void *stream);

/*
 * spmm_get_status -- synchronises the plan's last stream and returns the
 * device status word in *device_status (0 = ok, else an spmm_status value
 * recorded on the device), then clears it.
 */
spmm_status spmm_get_status(spmm_plan *plan, int32_t *device_status);

/*
 * spmm_plan_set_wait -- failure detection of the tensor-core launches (the
 * product and spmm_batch_run, which takes the first plan's setting).  Every
 * wait of such a launch on its copy / MMA pipeline is bounded: once a wait
 * has lasted `limit_ns` (0 = the default, 2 s) the CTA records
 * SPMM_ERR_TIMEOUT in the plan's status word, stops, lets its copies and
 * MMAs in flight complete, frees its tensor memory and exits; Y is then not
 * to be trusted, and spmm_get_status reports the timeout.  The context
 * stays usable and the next call runs normally.  Dynamic tensor-core plans
 * bound the grid barriers of their re-partition launch the same way (the
 * launch ends, the product launch skips).  stall = 1 is a test hook: after
 * their first stage the MMA warps wait on a barrier that nothing arrives
 * on, and in a dynamic plan's re-partition one CTA skips its arrival at the
 * first grid barrier, so that every CTA takes the timeout path after
 * limit_ns (use a short limit).  This library's own extension, not in the
 * paper.
 * Returns SPMM_ERR_ARG for a NULL plan, limit_ns < 0 or stall not 0/1.
 */
spmm_status spmm_plan_set_wait(spmm_plan *plan, int64_t limit_ns, int32_t stall);

/* Plan facts for reporting and tests. */
typedef struct {
    int64_t m, k, n_max, nnzb, nnzb_max;
    int32_t b, mode, w_dtype, x_dtype, kernel;
    int32_t rows_per_group, max_per_item;   /* rows_per_group 0: near-equal groups (opts.groups) */
    int64_t n_items, n_groups, n_entries, n_tiles, ws_rows, n_reductions;
    int64_t device_bytes;         /* device memory the plan holds */
    int32_t stage_geometry;       /* TC: 0 dense-tile stages, 1 sparse-tile stages (other kernels: 0) */
    int32_t sddmm_form;           /* spmm_sddmm on this plan: 0 dense tiles, 1 gathered blocks */
    int64_t row_begin, row_end;   /* the plan's slice of output rows (0, m for a whole plan) */
    int32_t col_tiles;            /* TC: the col_tiles option the plan runs with (0, 1 or 2) */
    int32_t index_bytes;          /* bytes per column index the product reads: 2 for static
                                     GATHER plans with k <= 65536 (a 16-bit copy of col_idx,
                                     read by the n <= 8 kernel that keeps X in shared memory),
                                     else 4 */
} spmm_plan_info;

spmm_status spmm_plan_get_info(const spmm_plan *plan, spmm_plan_info *info);

/* Integer plan arrays, in the exact definitions the oracle states.  After a
 * dynamic spmm_run the device-built arrays are returned (the call
 * synchronises the plan's last stream). */
typedef enum {
    SPMM_ARR_ROW_PTR = 0,   /* int32[m/b + 1] block-CSR row pointers */
    SPMM_ARR_COL_IDX = 1,   /* int32[nnzb] block column of each CSR slot */
    SPMM_ARR_PERM = 2,      /* int32[nnzb] user index of each CSR slot */
    SPMM_ARR_ITEMS = 3,     /* int32[n_items * 6]: group/row, begin, end, chunk, n_chunks, ws_slot */
    SPMM_ARR_GRP_ROW0 = 4,  /* TC: int32[n_groups] first tile row of each group */
    SPMM_ARR_GRP_ROWS = 5,  /* TC: int32[n_groups] tile rows in each group */
    SPMM_ARR_GRP_EBEG = 6,  /* TC: int32[n_groups + 1] first entry of each group */
    SPMM_ARR_ENT_COL = 7,   /* TC: int32[n_entries] tile column of each entry */
    SPMM_ARR_ENT_TBEG = 8,  /* TC: int32[n_entries + 1] first tile slot of each entry */
    SPMM_ARR_TILE_ROW = 9,  /* TC: int32[n_tiles] group row of each tile slot (slots of an entry
                               cover its MMA intervals; rows without a block are zero tiles) */
    SPMM_ARR_BLK_SLOT = 10, /* TC: int32[nnzb] tile slot of each user block */
    SPMM_ARR_BLK_OFF = 11,  /* TC: int32[nnzb] offset (row*16 + col) of the block in its tile */
    SPMM_ARR_WS_ROW0 = 12,  /* int64[n_ws_slots] first workspace row of each split item */
    SPMM_ARR_RED = 13,      /* int32[n_reductions * 3]: group/row, first ws slot, n_chunks */
    SPMM_ARR_ENT_COVER = 14,/* TC: int32[n_entries]: bits 0-15 rows covered by the entry's MMA
                               intervals, bits 16-31 the rows where an interval starts */
    SPMM_ARR_SRC_INDEX = 15 /* row-slice plans: int32[nnzb] index in the whole pattern of each
                               block the slice keeps (the slice's pattern order); whole plans:
                               empty */
} spmm_array;

/* Copies array `which` into host memory `dst` (capacity in elements) and
 * stores the element count in *count.  dst may be NULL to query the count. */
spmm_status spmm_plan_get_array(spmm_plan *plan, spmm_array which, void *dst, int64_t capacity,
                                int64_t *count);

void spmm_plan_destroy(spmm_plan *plan);

/* Appendix A.2 planner formulas, exposed for reporting:
 * equal partition of `extent` into q parts -> sizes[q] (q - 1 parts of
 * floor(extent/q), the last extent - (q-1)*floor(extent/q));
 * bucket size N_nz = ceil(m * k * d_max / (q_m * q_k)), d_max = num/den. */
spmm_status spmm_equal_partition(int64_t extent, int64_t q, int64_t *sizes);
int64_t spmm_bucket_size(int64_t m, int64_t k, int64_t d_max_num, int64_t d_max_den, int64_t q_m,
                         int64_t q_k);

/*
 * spmm_batch_run -- `count` (<= 64) static TC or BGATHER plans with packed
 * values, run as persistent launches: the BGATHER problems (small n, CUDA
 * cores) in one launch, then the tensor-core problems in one launch (two
 * when some plans take two column tiles per CTA: col_tiles = 2 with
 * n > 128; those run in a launch of their own).  Tensor-core plans of both stage geometries run
 * in the geometry that holds most of the batch's work; the others use
 * stage records cut for it (built once per plan on first use; results are
 * identical).  The tensor-core launch's CTAs walk one schedule of
 * (problem, work item, n tile) units, precomputed on the host when the
 * plan set is first run (costliest units first) and cached; each CTA takes
 * every gridDim-th unit of it (no atomic work queue).  Each problem with
 * rows split over several work items adds one reduction launch.  d_X[i],
 * n[i], ldx[i], d_Y[i], ldy[i] as in spmm_run (ldx/ldy may be NULL for
 * dense n).  All plans must share w_dtype and x_dtype; uneven m, k, n, b and
 * density are allowed.  The first call with a plan set allocates (its
 * schedule, other-geometry stage records): make it outside any stream
 * capture; later calls are CUDA-graph capturable.
 */
spmm_status spmm_batch_run(int32_t count, spmm_plan *const *plans, const void *const *d_X,
                           const int64_t *n, const int64_t *ldx, void *const *d_Y,
                           const int64_t *ldy, void *stream);

/*
 * spmm_gather_noalloc -- the dynamic b = 1 product (device re-partition,
 * gather kernel, split-row reduction) for callers that cannot allocate
 * device memory: it calls no cudaMalloc / cudaFree / allocating library
 * routine and needs no plan.  The paper has no counterpart; this is a
 * deployment convenience of this library.
 *   m, k          : W is m x k (b = 1), m <= 8192.
 *   dtype         : F32, F16 or BF16 for values, X and Y alike.
 *   d_nnzb, d_brow, d_bcol : device pattern as in spmm_dpattern, nnzb_max <= 262144.
 *   d_values      : device values in pattern order (nnzb_max entries).
 *   d_X, n, ldx / d_Y, ldy : X (k x n) and Y (m x n), n <= 256.
 *   d_status      : optional device int32 that receives the pattern status
 *                   (0 or an spmm_status code); NULL keeps it internal.
 * All scratch lives in one file-scope device array of about 14 MB that every
 * GPU loading the library holds until exit; sizes beyond the limits above
 * (or k > 2^30) return SPMM_ERR_SHAPE before anything is enqueued.  Each
 * device has its own copy of the array, and all calls on one device share
 * it (each clears what must start at zero): calls that overlap on one
 * device race, so serialise them.  Outside a stream capture a call looks up
 * the array's device address afresh (so a reset device is picked up);
 * inside a capture it uses the address of the last uncaptured call on the
 * device, so make one uncaptured call on the device before capturing.
 */
spmm_status spmm_gather_noalloc(int64_t m, int64_t k, spmm_dtype dtype, const int32_t *d_nnzb,
                                const int32_t *d_brow, const int32_t *d_bcol, int64_t nnzb_max,
                                const void *d_values, const void *d_X, int64_t n, int64_t ldx,
                                void *d_Y, int64_t ldy, int32_t *d_status, void *stream);

/*
 * spmm_quantize_e4m3 -- per-block FP8 quantiser for E4M3 plans (the
 * precision form of the value packing step, Section 3.2's host-supplied
 * values): for each of the nnzb b x b blocks at d_src (src_dtype F32, F16 or
 * BF16, pattern order), scale = max|w| / 448 (1 for an all-zero block) and
 * code = the E4M3 value nearest w / scale (round to nearest even,
 * saturating).  Writes d_codes[nnzb * b * b] and d_scales[nnzb] (device).
 */
spmm_status spmm_quantize_e4m3(int64_t nnzb, int32_t b, spmm_dtype src_dtype, const void *d_src,
                               uint8_t *d_codes, float *d_scales, void *stream);

/*
 * spmm_run_ell -- Y = W.X with W in Blocked-ELL form (padded block lists per
 * block row, the FP16 block-sparse layout Section 5 discusses for GPUs),
 * for dynamic sparsity without a device re-partition: a call validates the
 * layout and runs one product launch.  b = 16 only.
 *   plan        : a DYNAMIC device plan with b = 16 and w_dtype = x_dtype in
 *                 {F16, BF16} (m, k multiples of 16); its re-partition
 *                 buffers are not used.
 *   d_ell_cols  : int32[(m/16) * ell_width] device: row r lists its block
 *                 columns in slots r*ell_width ... in strictly increasing
 *                 order, then -1 in every unused slot.
 *   ell_width   : 0 <= ell_width <= k/16.
 *   d_values    : (m/16) * ell_width blocks of 16 x 16 (x_dtype, row-major),
 *                 block (r, slot e) at index r*ell_width + e, 16-byte
 *                 aligned; values of padding slots are ignored.
 *   d_X, n, ldx : X (k x n), 16-byte aligned, ldx a multiple of 8, n <= n_max.
 *   d_Y, ldy    : Y (m x n).
 * A layout that breaks these rules sets the status word to SPMM_ERR_PATTERN
 * on the device and Y is not written.
 */
spmm_status spmm_run_ell(spmm_plan *plan, const int32_t *d_ell_cols, int32_t ell_width,
                         const void *d_values, const void *d_X, int64_t n, int64_t ldx,
                         void *d_Y, int64_t ldy, void *stream);

/*
 * spmm_sddmm -- the sampled dense-dense product on the plan's block mask,
 * i.e. the gradient of Section 3's product with respect to the stored blocks
 * (the weight-gradient step of sparse training, Section 1):
 *   dW[p][ii][l] = sum_{j < n} dY[brow_p*b + ii, j] * X[bcol_p*b + l, j]
 * for every block p of the pattern, FP32 accumulation.
 *   plan          : a device plan for W (not transposed, not host-only) whose
 *                   x_dtype is F16 or BF16; its w_dtype plays no part.
 *   pattern       : dynamic plans: the device pattern of this step (rebuilt
 *                   into the plan's block CSR and validated on the device, as
 *                   in spmm_run; a rejected pattern sets the status word and
 *                   dW is not written).  Static plans: NULL (the plan's own).
 *   d_dY, lddy    : dY (m x n, x_dtype), row-major, lddy >= n.
 *   d_X, ldx      : X (k x n, x_dtype), row-major, ldx >= n.
 *                   Both base addresses 16-byte aligned and lddy, ldx
 *                   multiples of 8 elements (rows are read by TMA), else
 *                   SPMM_ERR_ARG.
 *   n             : >= 0 (no n_max limit); n = 0 writes zero blocks (dY and
 *                   X may then be NULL).
 *   d_dW          : device output, the pattern's blocks in the pattern's
 *                   order, each b x b row-major (the layout spmm_pack_values
 *                   reads), 16-byte aligned; static: nnzb blocks, dynamic:
 *                   room for nnzb_max blocks, of which *d_nnzb are written.
 *   dw_dtype      : F32, or the plan's x_dtype (rounded to nearest even).
 * Asynchronous on `stream`, CUDA-graph capturable for static plans.
 */
spmm_status spmm_sddmm(spmm_plan *plan, const spmm_dpattern *pattern, const void *d_dY,
                       int64_t lddy, const void *d_X, int64_t ldx, int64_t n, void *d_dW,
                       spmm_dtype dw_dtype, void *stream);

/*
 * spmm_tune -- the autotuner of this library (the paper fixes its
 * partitions ahead of time for a known pattern, Section 3.2; here the
 * tuned quantity is the GPU launch configuration).  For the static product
 * described by (m, k, n, b, types, pattern, d_values, d_scales, d_X, ldx)
 * it builds one plan per candidate -- the tensor-core kernel with dense-tile
 * and with sparse-tile stages, each with the planner's default groups and,
 * where those shrink below 16 tile rows to fill the GPU, with 16-row groups
 * split along k into enough work items to fill it (k_splits); for n > 128
 * both geometries with two column tiles per CTA (col_tiles = 2); and the
 * CUDA-core block gather (BGATHER) where n <= 16 and b >= 4 -- times `reps`
 * runs of each on `stream` after
 * two warm-up runs (CUDA events, median), and records the fastest for the
 * product's bucket: (b, W and X types, ceil(log2 m), ceil(log2 k),
 * round(log2(1/d)) with d the block density, ceil(log2 n)).  From then on
 * spmm_plan_create, for a static plan with kernel AUTO, no forced
 * stage_geometry, rows_per_group, groups, k_splits or col_tiles, takes the tuned
 * choice for its bucket (n = its n_max).
 *   reps          : 1 .. 64.
 *   out           : the choice and each candidate's median time (us, -1 if
 *                   it failed).
 * Allocates a Y scratch of m x n, synchronises `stream`; not for use inside
 * a stream capture.  SPMM_ERR_UNSUPPORTED if no candidate could run.
 */
typedef struct {
    int32_t kernel;          /* spmm_kernel */
    int32_t stage_geometry;  /* TC: 1 dense-tile, 2 sparse-tile stages; 0 otherwise */
    int32_t rows_per_group;  /* TC: 16 = 16-row groups split along k (see k_splits); 0 = default */
    int32_t k_splits;        /* TC: work items per group when rows_per_group = 16 */
    int32_t col_tiles;       /* TC: 2 = two column tiles per CTA (spmm_plan_opts.col_tiles); 0 */
} spmm_tune_choice;

typedef struct {
    spmm_tune_choice choice;
    float best_us;
    int32_t n_candidates;
    spmm_tune_choice cand[8];
    float cand_us[8];
} spmm_tune_result;

spmm_status spmm_tune(int64_t m, int64_t k, int64_t n, int32_t b, spmm_dtype w_dtype,
                      spmm_dtype x_dtype, const spmm_pattern *pattern, const void *d_values,
                      const float *d_scales, const void *d_X, int64_t ldx, int32_t reps,
                      void *stream, spmm_tune_result *out);

/* Forgets every tuned choice; the number of buckets tuned so far. */
void spmm_tune_clear(void);
int64_t spmm_tune_size(void);

/* Thread-local message describing the last error on this thread ("" if none). */
const char *spmm_last_error(void);

/* Library version string. */
const char *spmm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPMM_H */
