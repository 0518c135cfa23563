/*
 * spmm_serve.h -- serving loop over block-sparse weights kept resident on
 * the device (the weight-sparse inference setting of Section 1 and the
 * "batch size n is a free parameter" reading of Section 5: requests are
 * column blocks X_r (k x n_r) aimed at one registered weight W).
 *
 * Model: requests queue in arrival order.  A request is admitted when its
 * device staging (X_r and Y_r, 16-bit) fits the HBM budget; admitted
 * requests of any mix of weights are launched together in one persistent
 * tensor-core launch on one of up to max_inflight streams ("slots"), so
 * requests that arrive while others run are admitted as slots and budget
 * free up and their work overlaps on the device (continuous batching).
 * Y_r is copied back to the caller's host buffer when its launch finishes.
 * Column j of Y depends only on column j of X, and the work order of a
 * column does not depend on its neighbours, so a result is the same alone
 * and in a mix.
 *
 * Threads: serve_* may be called from any thread.  Host buffers passed to
 * serve_submit must stay valid until serve_wait returns for that ticket
 * (pinned memory gives asynchronous copies; pageable memory works, slower).
 */
#ifndef SPMM_SERVE_H
#define SPMM_SERVE_H

#include <stdint.h>

#include "spmm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct serve_server serve_server;

typedef struct {
    int64_t hbm_budget_bytes;  /* device bytes for request staging (X_r + Y_r); > 0 */
    int32_t max_inflight;      /* concurrent launches (streams), 1..8 */
    int32_t max_batch;         /* requests per launch, 1..64 */
    int64_t max_batch_n;       /* total columns per launch, >= 1 */
    int32_t inject_delay_us;   /* fault injection (tests): batcher sleeps this long before each launch */
    int32_t inject_alloc_fail; /* fault injection (tests): 1 = every staging allocation fails */
} serve_config;

typedef struct {
    int64_t submitted, admitted, completed, rejected, failed, queued, in_flight;
    int64_t launches;
    double mean_requests_per_launch, mean_cols_per_launch;
    double p50_us, p99_us, mean_us, max_us;  /* arrival -> completion observed, completed requests */
    double span_s;                           /* first arrival -> last completion */
    double throughput_rps;                   /* completed / span_s */
    double tflops_nz;                        /* non-zero FLOPs of completed requests / span_s */
} serve_stats_t;

/* Creates a server on the current device; allocates the staging pool of
 * hbm_budget_bytes.  SPMM_ERR_ARG for bad limits, SPMM_ERR_OOM / _CUDA. */
spmm_status serve_create(const serve_config *cfg, serve_server **out);

/* Registers a static plan with packed values as a resident weight (the
 * plan stays owned by the caller and must outlive the server).  Plans of
 * the tensor-core kernel with 16-bit X are batched; others (e.g. the plain
 * FP32 kernel) run one request per launch. */
spmm_status serve_register_weight(serve_server *srv, spmm_plan *packed_plan, int32_t *weight_id);

/* Queues one request: h_X is k x n (row-major, ldx = n) and h_Y receives the
 * m x n result (row-major), both in the weight's X type, in host memory.
 * SPMM_ERR_CAPACITY if the request's staging can never fit the budget;
 * SPMM_ERR_SHAPE if n < 1 or n > the plan's n_max or max_batch_n. */
spmm_status serve_submit(serve_server *srv, int32_t weight_id, const void *h_X, int64_t n,
                         void *h_Y, uint64_t *ticket);

/* Waits up to timeout_ms (< 0: forever) for a request; on SPMM_OK its Y is
 * in the caller's buffer and the ticket is retired.  SPMM_ERR_TIMEOUT if it
 * is not done yet (the ticket stays valid); SPMM_ERR_ARG for an unknown
 * ticket; the request's own error code if its launch failed. */
spmm_status serve_wait(serve_server *srv, uint64_t ticket, int64_t timeout_ms);

/* Statistics since creation (or the last serve_reset_stats). */
spmm_status serve_stats(serve_server *srv, serve_stats_t *out);
spmm_status serve_reset_stats(serve_server *srv);

/* Trace replay, for load tests without a client in the loop: resets the
 * statistics, submits request i at t_arrive_s[i] seconds after the call
 * starts (busy-waiting on the calling thread; times ascending), aimed at
 * weight[i] with n[i] columns and host buffers h_X[i] / h_Y[i], waits for
 * all of them and writes the statistics to *out.  Returns the first error. */
spmm_status serve_replay(serve_server *srv, int64_t count, const double *t_arrive_s,
                         const int32_t *weight, const int64_t *n, const void *const *h_X,
                         void *const *h_Y, serve_stats_t *out);

/* Drains in-flight work, stops the threads and frees the staging pool. */
void serve_destroy(serve_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* SPMM_SERVE_H */
