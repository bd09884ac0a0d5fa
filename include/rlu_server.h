/* Serving form of the randomized LU (Algorithm 1 of "Randomized LU Decomposition",
 * arXiv 1310.7202): a device-resident request loop. The paper has no counterpart; it
 * describes one factorization at a time. The loop admits requests of mixed sizes and
 * precisions as in-flight slots and workspace memory free up, runs each one as an
 * rlu_factor call on its own CUDA stream (so the work of different requests overlaps on the
 * GPU), and records per-request times on the host.
 *
 * Ownership. A, P, Q, L, U and info of a request are device buffers owned by the caller;
 * they must stay valid until the request is done. The server owns one workspace arena of
 * the byte budget given at creation (allocated once, in rlu_server_create) and the slot
 * streams. Requests never allocate.
 *
 * Admission. A request is admitted when a slot is free and its workspace
 * (rlu_workspace_size) fits in the arena. Requests are considered in arrival order; a
 * request that does not fit may be passed by later ones that do (continuous batching), but
 * at most 64 times, after which nothing else is admitted until it fits.
 *
 * Times are host steady-clock nanoseconds: submit = when rlu_server_submit ran; start =
 * when its work was enqueued; done = when the stream reached the end of its work (a host
 * function enqueued after it).
 *
 * Thread safety: every function may be called from any host thread. */
#ifndef RLU_SERVER_H
#define RLU_SERVER_H

#include <stddef.h>
#include <stdint.h>

#include "rlu.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rlu_server rlu_server;

/* One factorization request; the fields are the arguments of rlu_factor. */
typedef struct {
  const void* A;
  int32_t dtype;
  int64_t m, n, lda;
  int32_t k, l;
  uint64_t seed;
  int32_t prec;
  int32_t* P;
  int32_t* Q;
  void* L;
  int64_t ldl;
  void* U;
  int64_t ldu;
  rlu_info* info;
} rlu_request;

enum { RLU_REQ_QUEUED = 0, RLU_REQ_RUNNING = 1, RLU_REQ_DONE = 2, RLU_REQ_FAILED = 3 };

/* Creates a server on the current device with a workspace arena of budget_bytes and up to
 * max_inflight concurrently running requests (1..64). RLU_ENOMEM if the arena cannot be
 * allocated, RLU_EINVAL for a bad argument. */
int32_t rlu_server_create(size_t budget_bytes, int32_t max_inflight, rlu_server** out);

/* Queues a request; writes its id (0, 1, 2, ... in submission order). Checks the
 * arguments as rlu_factor does and returns its error synchronously; RLU_ENOMEM if the
 * request's workspace exceeds the whole budget. */
int32_t rlu_server_submit(rlu_server* s, const rlu_request* req, int64_t* id);

/* State of request id (RLU_REQ_*), the rlu_status of its launch (RLU_OK unless FAILED) and
 * its submit/start/done times (ns; 0 when not reached). Any output pointer may be NULL. */
int32_t rlu_server_poll(rlu_server* s, int64_t id, int32_t* state, int32_t* status,
                        int64_t* t_submit_ns, int64_t* t_start_ns, int64_t* t_done_ns);

/* Blocks until every submitted request is done or failed. */
int32_t rlu_server_wait_all(rlu_server* s);

/* Counters: [0] submitted, [1] done, [2] failed, [3] peak arena bytes in use, [4] peak
 * requests running at once, [5] requests admitted past an earlier waiting one. */
int32_t rlu_server_stats(rlu_server* s, int64_t* out6);

/* Waits for all requests, then frees the arena and the streams. */
int32_t rlu_server_destroy(rlu_server* s);

#ifdef __cplusplus
}
#endif

#endif /* RLU_SERVER_H */
