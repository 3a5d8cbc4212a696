/*
 * libme serving layer -- continuous batching of |M|^2 requests on one GPU.
 *
 * The paper runs many MadEvent jobs per GPU through its Python driver's
 * worker/job queue (arXiv:2507.21039 Sec. 3.3) and notes that host-device
 * latency dominates small GPU jobs (Sec. 5); this layer serves requests for
 * different processes and batch sizes as they arrive, on top of the C ABI of
 * me.h:
 *   - per-(process, precision) handles stay resident on the device (colour
 *     matrices, helicity masks, couplings), created and filtered on first use;
 *   - a scheduler thread groups queued requests of the same (process,
 *     precision) into one batch, up to max_batch events;
 *   - batches run on `lanes` CUDA streams at once; a batch is admitted only
 *     while the device bytes of all batches in flight (momenta + |M|^2, plus
 *     the global scratch of launches that use one: the FP64 colour-flow
 *     vectors of gg_ttxggg) stay within hbm_budget_bytes, so requests that
 *     arrive while others run start as soon as a lane and memory are free; a
 *     later, smaller batch that fits may start before an older one that does
 *     not (the older one waits for room after being passed over 8 times);
 *   - each lane replays its batch as a CUDA graph (H2D momenta, |M|^2 kernel,
 *     D2H results), captured per batch and updated in place;
 *   - results do not depend on the batch a request lands in (every event is
 *     computed independently of its neighbours).
 * Latency of a request = time from srv_submit to its results being in the
 * caller's host buffer.  All calls return ME_* status codes (me.h).
 */
#ifndef LIBME_ME_SERVE_H
#define LIBME_ME_SERVE_H

#include <stdint.h>

#include "me.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct srv_server srv_server;

typedef struct srv_config {
    int lanes;                 /* concurrent batches (CUDA streams), 1..16 */
    int64_t max_batch;         /* events per batch (and per request), >= 1 */
    uint64_t hbm_budget_bytes; /* device bytes of the batches in flight */
    int use_graphs;            /* 1: replay each batch as a CUDA graph */
} srv_config;

/* srv_create -- start a server on the current CUDA device.  Allocates each
 * lane's device and pinned host buffers for max_batch events of the largest
 * process (7 particles).  Errors: ME_EINVAL, ME_ENOMEM, ME_ECUDA. */
int srv_create(srv_server** s, const srv_config* cfg);

/* srv_submit -- queue |M|^2 for nevt events of `process` at `precision`
 * (ME_PREC_*): momenta [nevt][npar][4] and me2_out [nevt] are host buffers
 * (pinned buffers are copied without an extra staging step) that must stay
 * valid until the request completes or is cancelled.  *ticket identifies it.
 * Errors: ME_EINVAL (unknown process, nevt <= 0 or > max_batch, null
 * pointers), ME_ENOMEM. */
int srv_submit(srv_server* s, const char* process, int precision, const double* momenta, int64_t nevt,
               double* me2_out, uint64_t* ticket);

/* srv_wait -- wait up to timeout_ms (< 0: no limit) for a request.  Returns
 * ME_OK when its results are in me2_out (and stores the request's latency in
 * microseconds in *latency_us, nullable), ME_ETIMEOUT if the time ran out,
 * the request's own error status if it failed, ME_EINVAL for an unknown or
 * already collected ticket.  A completed ticket is released by this call. */
int srv_wait(srv_server* s, uint64_t ticket, int timeout_ms, double* latency_us);

/* srv_cancel -- drop a request that has not started (ME_OK), or mark one in
 * flight so that its results are discarded (ME_OK; me2_out is then not
 * written after this call returns).  The ticket is released. */
int srv_cancel(srv_server* s, uint64_t ticket);

/* srv_stats -- JSON object with counters written into buf (cap bytes):
 * requests, batches, events, queue depth, bytes in flight, graph updates, and
 *   max_lanes_busy          most lanes holding a launched, unfinished batch at once;
 *   max_device_concurrency  most batches seen running on the device at the same
 *                           time (from timing events around each batch: the
 *                           batches of different lanes overlap on the GPU);
 *   head_bypasses           batches started ahead of an older request that did
 *                           not fit the budget yet (at most 8 in a row for one);
 *   lane_buffer_bytes       the lanes' fixed device buffers (outside the budget). */
int srv_stats(srv_server* s, char* buf, int cap);

/* srv_destroy -- stop the scheduler after finishing the batches in flight;
 * queued requests are dropped.  NULL is a no-op. */
void srv_destroy(srv_server* s);

#ifdef __cplusplus
}
#endif
#endif /* LIBME_ME_SERVE_H */
