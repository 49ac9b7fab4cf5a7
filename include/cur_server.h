/*
 * cur_server.h -- serving form of IterativeCUR: a request loop with continuous
 * batching on one GPU.
 *
 * The paper treats one matrix at a time and has no serving counterpart.  Every
 * request is decomposed by exactly the method of cur_run (cur.h; Algorithm 1 of
 * arXiv 2509.21963 with the Lemma 1 residual recurrence, Sec. 4.2, and
 * U = A(I,J)^+ by pivoted QR at exit, Sec. 3.3).
 *
 * How requests flow:
 *   submit      a request joins a FIFO of pending requests (host only).
 *   admission   a scheduler thread admits pending requests in arrival order
 *               (with limited backfill: up to 16 later requests that fit may
 *               pass a head request that does not) whenever their HBM
 *               footprint fits in the server's budget: the request's scratch
 *               (sketch S and G, the Lemma 1 factors L and Rt, the pivot
 *               masks, the core QR; sized by min(m, n) or max_rank) and its
 *               outputs (I, J, U, rho history), plus a copy of A when A
 *               arrives in host memory.  Memory comes from one arena of
 *               `hbm_budget` bytes (first-fit, coalescing).
 *   waves       admitted requests are launched together as a wave: one kernel
 *               in which each request owns one thread-block cluster of `team`
 *               CTAs and keeps its sketch and pivot state resident in its own
 *               workspace until it finishes.  Waves go round-robin to several
 *               CUDA streams, so requests admitted while earlier ones are still
 *               on the GPU start as soon as SMs free up (the hardware block
 *               scheduler interleaves clusters of all waves in flight).
 *   completion  when a wave's event fires, each request's scratch returns to
 *               the arena at once; its outputs stay on the device until
 *               cur_server_release.
 * A request's result does not depend on what else is in flight: its cluster
 * runs the same instructions on the same data whatever the mix.
 *
 * Conventions are those of cur.h.  A server belongs to the context it was
 * created on; its calls may come from any one host thread at a time (the
 * scheduler runs on its own thread).
 */
#ifndef CUR_SERVER_H
#define CUR_SERVER_H

#include <stddef.h>
#include <stdint.h>

#include "cur.h"
#include "cur_batch.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cur_server cur_server;

/* Counters since creation.  waves: wave kernels launched plus large requests
 * run; launches: kernels launched (one per wave, all of each large request's);
 * bytes_*: arena bytes held now, at most, and the budget; pending: requests
 * not yet admitted; in_flight: admitted and not yet completed. */
typedef struct cur_server_stats {
  int64_t submitted, admitted, completed, waves;
  size_t bytes_in_use, bytes_peak, budget;
  int64_t pending, in_flight, launches;
} cur_server_stats;

/* Create a server.
 *   hbm_budget    bytes of device memory the server may hold for requests
 *                 (one arena, allocated here; CUR_ENOMEM if it cannot be).
 *   dtype         CUR_F32 or CUR_F64: the element type of every request's A.
 *   team          CTAs (thread-block cluster size, 1..8) per request.
 *   streams       CUDA streams waves are spread over (1..16).
 *   big_elements  requests with m * n >= big_elements (0: none) are large:
 *                 each runs on the whole GPU through the single-matrix path
 *                 (the kernels of cur_run, workspace outside the arena) once
 *                 the waves in flight have drained; smaller requests keep
 *                 flowing in waves before and after them.
 *   big_lanes     large requests that may run at once (1..4), each on its own
 *                 private context, stream and host thread: their launch and
 *                 host-synchronisation gaps overlap.  (Each cooperative
 *                 kernel waits only on its own CTAs, so a kernel of one lane
 *                 at most queues behind another lane's for one kernel; every
 *                 kernel's shared-memory ceiling is set to one fixed value, so
 *                 launches from several lanes never race on it.)
 * The scheduler thread starts here and stops in cur_server_free. */
int cur_server_create(cur_ctx *ctx, size_t hbm_budget, int dtype, int team, int streams,
                      int64_t big_elements, int big_lanes, cur_server **out);

/* Stop the scheduler (after the requests in flight finish) and release
 * everything.  NULL is a no-op. */
void cur_server_free(cur_server *srv);

/* Queue a request.  job: as for cur_batch_create (block_size <= 64,
 * sketch_size <= 128; large requests follow cur_run's rules).  a_on_host = 0: job->A is device memory, borrowed
 * until the request completes; a_on_host = 1: job->A is host memory, copied
 * to the device when the request is admitted (it must stay valid until then).
 * *ticket identifies the request.  CUR_EINVAL for a malformed job,
 * CUR_EBUDGET if its footprint exceeds the whole budget. */
int cur_server_submit(cur_server *srv, const cur_batch_job *job, int a_on_host, uint64_t *ticket);

/* Block until the request completes or timeout_s passes (CUR_ETIMEOUT; the
 * request keeps running).  timeout_s < 0 waits without limit. */
int cur_server_wait(cur_server *srv, uint64_t ticket, double timeout_s);

/* Non-blocking: *done = 1 once the request has completed. */
int cur_server_poll(cur_server *srv, uint64_t ticket, int *done);

/* Block until every submitted request has completed. */
int cur_server_drain(cur_server *srv);

/* Result of a completed request: rank, iterations, final rho, status (as in
 * cur_batch_job_result), and times in ms measured on the host clock:
 * latency = submit -> completion observed, queue = submit -> admission.
 * When a large request failed (status CUR_ECUDA, CUR_ETIMEOUT, ...), the
 * reason becomes the context's cur_last_error text. */
int cur_server_result(cur_server *srv, uint64_t ticket, int64_t *rank, int64_t *iters,
                      double *rho, int *status, double *latency_ms, double *queue_ms);

/* Copy a completed request's I, J (rank entries), U (rank^2, row-major,
 * |J| x |I|) and rho history (iterations entries) to host buffers (any may
 * be NULL). */
int cur_server_copy(cur_server *srv, uint64_t ticket, int64_t *I, int64_t *J, double *U,
                    double *rho_history);

/* Release a completed request's outputs (device memory returns to the arena)
 * and forget the ticket. */
int cur_server_release(cur_server *srv, uint64_t ticket);

int cur_server_get_stats(cur_server *srv, cur_server_stats *out);

#ifdef __cplusplus
}
#endif

#endif /* CUR_SERVER_H */
