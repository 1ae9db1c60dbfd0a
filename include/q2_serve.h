/*
 * q2_serve.h -- admission core of the request loop (host only, no device work).
 *
 * The paper's workflow submits one circuit evaluation after another
 * (Fig. 1b); serving many (Hamiltonian, ansatz, theta, want_grad) requests
 * concurrently is this library's addition, so these calls have no paper
 * counterpart.  The core keeps the ledger that lets a request loop admit
 * requests by device-memory footprint.  The bytes in use are the workspaces
 * of the running requests plus the resident tables (Hamiltonian and ansatz
 * handles) of every problem the loop keeps on the device; a problem's tables
 * are charged once, however many requests share them.
 *
 *   - submit   queues a request with its workspace bytes and its problem's
 *              key and table bytes (FIFO);
 *   - admit    moves queued requests to running, in FIFO order, while their
 *              workspace (and their problem's tables, if not resident) fit
 *              the budget and a slot is free (later requests that fit may
 *              pass a larger head request).  To make room it releases the
 *              tables of problems with no queued or running request, least
 *              recently used first;
 *   - take_evicted  hands the caller the keys of the problems released that
 *              way, whose device tables the caller then frees;
 *   - expire   removes requests that waited in the queue longer than the
 *              queue timeout (they are reported as timed out, Q2_ERR_TIMEOUT
 *              to the caller of the loop);
 *   - complete releases a running request's workspace bytes and slot and
 *              records its latency (completion time - submission time).
 *
 * Times are caller-supplied seconds on any monotonic clock.  All calls are
 * thread-safe.  Errors: Q2_ERR_INVALID for NULL handles, unknown or repeated
 * ids, negative times; Q2_ERR_OOM from submit when a request's workspace and
 * its problem's tables together exceed the whole budget.
 */
#ifndef Q2_SERVE_H
#define Q2_SERVE_H

#include "q2.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct q2_server q2_server;

q2_status q2_server_create(size_t budget_bytes, int max_slots, double queue_timeout_s, q2_server **out);
q2_status q2_server_destroy(q2_server *server);

q2_status q2_server_submit(q2_server *server, int64_t id, size_t bytes, int64_t problem,
                           size_t table_bytes, double now_s);

/* Admit queued requests; writes up to `cap` admitted ids; returns their number (or -1 on error). */
int q2_server_admit(q2_server *server, double now_s, int64_t *ids_out, int cap);

/* Remove queued requests older than the queue timeout; returns their number (or -1). */
int q2_server_expire(q2_server *server, double now_s, int64_t *ids_out, int cap);

q2_status q2_server_complete(q2_server *server, int64_t id, double now_s);

/* Keys of problems whose tables admit released since the last call; returns their number (or -1). */
int q2_server_take_evicted(q2_server *server, int64_t *problems_out, int cap);

/*
 * out[0..13]: submitted, admitted, completed, expired, queued, running,
 * bytes in use (workspaces + resident tables), high-water bytes, latency p50 (s),
 * latency p99 (s), mean latency (s), resident table bytes, resident problems,
 * evictions so far.
 */
q2_status q2_server_stats(const q2_server *server, double *out14);

#ifdef __cplusplus
}
#endif

#endif /* Q2_SERVE_H */
