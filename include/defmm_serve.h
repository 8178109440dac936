/* Serving layer of the defmm application phase: caller-owned workspaces,
 * fixed batches of applies replayed as one CUDA graph, and a request server
 * with continuous batching.
 *
 * What it serves: the operator of defmm_apply (include/defmm.h), applied over
 * and over to fixed point clouds, as boundary-integral solvers do (Sec. 1:
 * the N-body problem comes from BIEs; Sec. 5.3: particle positions do not
 * change from one application to the next; Sec. 7: integration in an
 * iterative solver).  The paper describes no batching or serving machinery;
 * nothing here computes anything beyond defmm_apply, and every result equals
 * the one defmm_apply gives for the same plan and right-hand sides (up to the
 * summation-order differences stated at defmm_server_submit).
 *
 * Conventions are those of defmm.h: status codes, never exceptions; the
 * thread-local message of defmm_last_error(); complex values interleaved
 * (re, im); right-hand-side blocks column-major (points fastest).
 */
#ifndef DEFMM_SERVE_H
#define DEFMM_SERVE_H

#include <stddef.h>
#include <stdint.h>

#include "defmm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- workspaces
 * The device scratch of one apply (Morton-ordered charges and potentials,
 * multipole, Fourier-domain and local expansions, near-field partial sums).
 * defmm_apply uses one workspace owned by the plan, so two applies on one
 * plan cannot overlap (DEFMM_ERR_BUSY).  With caller-owned workspaces they
 * can: the plan is only read by defmm_apply_ws.                             */
typedef struct defmm_workspace_s* defmm_workspace;

/* Bytes of scratch an apply of nrhs right-hand sides of dtype needs on this
 * plan (*bytes, host).  Errors: DEFMM_ERR_ARG.                               */
defmm_status defmm_workspace_bytes(defmm_plan plan, int nrhs, defmm_dtype dtype, size_t* bytes);

/* Allocates (cudaMalloc, current device) a workspace for applies of up to
 * nrhs right-hand sides of dtype on plan.  The workspace belongs to the
 * caller and to this plan; destroy it before the plan.
 * Errors: DEFMM_ERR_ARG, DEFMM_ERR_UNSUPPORTED (host-only plan or dtype),
 * DEFMM_ERR_OOM.                                                              */
defmm_status defmm_workspace_create(defmm_plan plan, int nrhs, defmm_dtype dtype, defmm_workspace* out);

/* The same over caller memory: mem is a device pointer, 256-byte aligned,
 * with at least defmm_workspace_bytes(plan, nrhs, dtype) bytes, borrowed for
 * the workspace's lifetime (defmm_workspace_destroy does not free it).
 * Errors: DEFMM_ERR_ARG (NULL, misaligned or too small).                     */
defmm_status defmm_workspace_wrap(defmm_plan plan, int nrhs, defmm_dtype dtype, void* mem, size_t bytes,
                                  defmm_workspace* out);

defmm_status defmm_workspace_destroy(defmm_workspace ws);

/* defmm_apply with scratch from ws: q (device, ny x nrhs) -> p (device,
 * nx x nrhs, overwritten), stream-ordered on stream.  nrhs may be at most
 * the workspace's capacity and dtype must be its dtype.  Applies on one plan
 * with distinct workspaces may run at the same time on different streams or
 * threads; a workspace must not be used by two applies at once (not
 * checked).  No phase events are recorded (defmm_profile_* see only
 * defmm_apply).  It always computes the whole operator, whatever the plan's
 * shard setting (defmm_plan_set_shard); results equal those of defmm_apply
 * on a plan that is not sharded, bit for bit.
 * Errors: DEFMM_ERR_ARG (NULL, foreign workspace, nrhs out of range, dtype
 * mismatch), DEFMM_ERR_CUDA (launch failure).                                */
defmm_status defmm_apply_ws(defmm_plan plan, defmm_workspace ws, const void* q, void* p, int nrhs,
                            defmm_dtype dtype, void* stream);

/* ---------------------------------------------------------------- graph batches
 * A fixed list of applies (plan i with nrhs[i] right-hand sides, all of one
 * dtype) recorded once into a CUDA graph and replayed with one
 * cudaGraphLaunch.  Entry i is an independent branch of the graph (its own
 * workspace, owned by the batch); the branches are spread over `branches`
 * streams while the graph is captured, so the GPU runs the kernels of
 * different geometries concurrently.  The kernels themselves are those of
 * defmm_apply; results equal defmm_apply's bit for bit.                      */
typedef struct defmm_batch_s* defmm_batch;

/* plans[n], nrhs[n] (host arrays, copied); branches in [1, 64] (0: min(n, 8)).
 * The plans are borrowed: they must outlive the batch.
 * Errors: DEFMM_ERR_ARG, DEFMM_ERR_UNSUPPORTED (host-only plan),
 * DEFMM_ERR_OOM, DEFMM_ERR_CUDA.                                             */
defmm_status defmm_batch_create(const defmm_plan* plans, const int* nrhs, int n, defmm_dtype dtype, int branches,
                                defmm_batch* out);

/* q[i] (device, ny_i x nrhs[i]) -> p[i] (device, nx_i x nrhs[i]) for every
 * entry, ordered after earlier work on stream and before later work on it.
 * The first call captures the graph (the calling thread must not be
 * capturing another stream); a call whose pointers differ from the previous
 * call's captures again and updates the executable graph in place.  A batch
 * must not be applied from two threads at once (DEFMM_ERR_BUSY).
 * Errors: DEFMM_ERR_ARG, DEFMM_ERR_BUSY, DEFMM_ERR_CUDA.                      */
defmm_status defmm_batch_apply(defmm_batch b, const void* const* q, void* const* p, void* stream);

/* Kernel launches and graph nodes of the captured graph (0 before the first
 * apply).                                                                     */
defmm_status defmm_batch_info(defmm_batch b, int64_t* kernel_launches, int64_t* graph_nodes);

defmm_status defmm_batch_destroy(defmm_batch b);

/* ---------------------------------------------------------------- request server
 * A worker thread owning `streams` CUDA streams and one device arena of
 * hbm_budget bytes.  Requests (geometry g, nrhs right-hand sides in host
 * memory) queue in arrival order.  Whenever a stream is free the worker
 * admits the oldest waiting request together with the later waiting requests
 * on the same geometry, up to max_batch_rhs right-hand sides in all, as one
 * batch: if its scratch (defmm_workspace_bytes for the summed nrhs, plus the
 * device copies of q and p) fits in the arena it is launched at once (copies
 * in, one apply, copies out on that stream), otherwise it waits for running
 * batches to free memory.  Batches on different streams overlap on the
 * device, and requests that arrive while others run join the next batch:
 * continuous batching by memory and stream availability.                     */
typedef struct defmm_server_s* defmm_server;

typedef struct {
    int streams;           /* batches in flight at once (default 4, at most 32) */
    int max_batch_rhs;     /* right-hand sides merged into one apply (default 16; a
                              larger single request still runs, alone) */
    size_t hbm_budget;     /* bytes of the device arena for in-flight batches
                              (default 4 GiB) */
} defmm_server_options;

void defmm_server_default_options(defmm_server_options* opt);

/* plans[nplans] (host array, copied; plans borrowed, must outlive the server),
 * all served in dtype; opt NULL for defaults.  Allocates the arena.
 * Errors: DEFMM_ERR_ARG, DEFMM_ERR_UNSUPPORTED (host-only plan),
 * DEFMM_ERR_OOM, DEFMM_ERR_CUDA.                                              */
defmm_status defmm_server_create(const defmm_plan* plans, int nplans, defmm_dtype dtype,
                                 const defmm_server_options* opt, defmm_server* out);

/* Queues a request: apply plans[geometry] to q_host (host, ny x nrhs) and
 * write p_host (host, nx x nrhs).  Both are borrowed until the request
 * completes; page-locked memory lets the copies overlap other batches.
 * Returns at once with *ticket.  Within a batch a request's columns are
 * applied together with other requests' columns: each column's result
 * equals a lone apply of that column up to the summation order of the
 * kernels' right-hand-side blocking (a few ulps; see the tests).
 * Errors: DEFMM_ERR_ARG, DEFMM_ERR_UNSUPPORTED (the request alone can never
 * fit in the arena), DEFMM_ERR_CUDA (the worker stopped on a CUDA error).    */
defmm_status defmm_server_submit(defmm_server s, int geometry, const void* q_host, void* p_host, int nrhs,
                                 uint64_t* ticket);

/* Waits for a ticket, at most timeout_ms milliseconds (< 0: no limit).  On
 * DEFMM_OK, *latency_ms (may be NULL) is the time from submit to the result
 * being in host memory.  A ticket can be waited for once.
 * Errors: DEFMM_ERR_ARG (unknown ticket), DEFMM_ERR_TIMEOUT (not done yet;
 * wait again), DEFMM_ERR_CUDA (the request's batch failed).                   */
defmm_status defmm_server_wait(defmm_server s, uint64_t ticket, double timeout_ms, double* latency_ms);

typedef struct {
    int64_t submitted, completed;
    int64_t batches;              /* applies launched */
    int64_t rhs_applied;          /* right-hand sides over all batches */
    int64_t max_batch_requests;   /* most requests merged into one batch */
    int64_t max_inflight;         /* most batches in flight at once */
    size_t arena_bytes, peak_arena_bytes;
    int64_t kernel_launches;      /* kernels launched by all batches */
} defmm_server_stats;

defmm_status defmm_server_get_stats(defmm_server s, defmm_server_stats* out);

/* Waits for every queued request, stops the worker and frees the arena. */
defmm_status defmm_server_destroy(defmm_server s);

#ifdef __cplusplus
}
#endif
#endif /* DEFMM_SERVE_H */
