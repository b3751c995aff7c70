/*
 * gbserve.h — serving engine of the GB300 GEMV / DOT / GER library.
 *
 * Not an operation of the paper (Singh & Bassoy, arXiv 2108.02025, whose
 * GEMV, DOT and GER run one call at a time, Sec. 4): a host runtime that
 * takes a stream of requests of different sizes and serves them with
 * continuous batching on one GPU.
 *
 *   request   GB_REQ_GEMV  c <- c + alpha A x     (Def. GEMV, Sec. 3.1),
 *                          A m x n row-major, stored FP32 or BF16
 *             GB_REQ_DOT   alpha <- alpha + x.y   (Def. DOT)
 *             GB_REQ_GER   C <- C + alpha x y^T   (Def. GEM), C m x n
 *
 * Life of a request.  gb_engine_submit queues it with its arrival time.
 * The engine's worker thread admits queued requests in arrival order once
 * they have arrived, while the HBM budget (an arena of budget_bytes of
 * device memory, allocated at creation) has room for the request's operands
 * and fewer than max_inflight requests are admitted; a request larger than
 * the whole budget is refused at submission.  Admitted requests are
 * launched as a step on one of `streams` CUDA streams as soon as one is
 * free: one copy of the step's descriptors, one operand kernel (it draws
 * the operands of requests without GB_REQ_POOL, copies the initial outputs
 * of pool requests and computes their GERs), one persistent launch (the
 * batched kernel of gb_sgemv_batch) for all the step's GEMVs (FP32 or BF16
 * A), DOTs (GB_BATCH_DOT_F32 tiles) and the GERs of drawn requests, then
 * the copies of the results to the requests' host buffers and an event.
 * GEMV sums are FP32 fma chains of at most 64 products in a compensated
 * FP32 sum; a DOT takes compensated FP32 products and sums per thread
 * (Dot2) and sums the threads' parts and the initial alpha in FP64, rounded
 * once to FP32, as gb_sdot; GER is one fma per element.  Requests that arrive while steps are
 * on the GPU are admitted and launched in the next step on another stream,
 * so steps overlap on the device.  When a step's event completes, its
 * requests complete (a request in chunks once all its chunks are done),
 * their memory returns to the arena and more requests are admitted.
 *
 * Operands.  A request's inputs are drawn on the device from the counter-
 * based SplitMix64 generator (Steele, Lea and Flood, OOPSLA 2014) with the
 * request's seed: key(seed, s) = mix(mix(seed + G) ^ (s * 0xD1B54A32D192ED03)),
 * one word u_k = mix(key + (k + 1) G) per pair of elements: element 2k takes
 * b = bits 63..40 of u_k, element 2k+1 bits 39..16, value b * 2^-23 - 1
 * (FP32 uniform in [-1, 1)), rounded to nearest even for BF16 storage
 * (synth.uniform_pairs on the host).  Streams s: GEMV A=1,
 * x=2, c=3; DOT x=1, y=2, alpha=3; GER C=1, x=2, y=3.  Matrices are stored
 * row-major with the leading dimension rounded up to 4 elements (FP32) or 8
 * (BF16); element (i, j) takes index k = i * ld + j of its stream.
 *
 * Resident operands (GB_REQ_POOL).  An engine created with pool_elems = P
 * > 0 places two operand pools on the device at creation, outside the
 * budget: P FP32 values (the generator above with pool_seed, stream 1) and
 * P BF16 values (stream 2, rounded to nearest even).  A request flagged
 * GB_REQ_POOL reads its inputs from the pools instead of having them drawn:
 * operand s (same stream numbers as above) of extent L_s elements (a
 * matrix m * ld, a vector its length) starts at element
 *     o_s = 8 * (mix(key(seed, s)) mod (floor((P - L_s) / 8) + 1))
 * of the FP32 pool (the BF16 pool for the A of a BF16 GEMV), so
 * element (i, j) of a matrix is pool[o_s + i * ld + j].  Only the output is
 * allocated in the arena (GEMV: c, DOT: alpha, GER: C, m x ld): its initial
 * value (c0, alpha0, C0) is the pool operand of stream 3, 3 and 1, copied
 * by the step (GER computes C0 + alpha x y^T straight into the output), so
 * the pools are never written.  A request whose operand is longer than P is
 * refused (-2).
 *
 * Chunks (chunk_bytes > 0).  A step takes the admitted requests that are
 * launched whole first, in admission order, then rows of the chunked
 * requests (GB_REQ_POOL GEMVs and GERs that move more than chunk_bytes in
 * all, counting per row the A row and the c element, or the C0 and C rows)
 * in admission order, at least one row and about chunk_bytes of them per
 * step.
 * A large request then holds the GPU a chunk at a time, so smaller requests
 * that arrive meanwhile run between its chunks.  Rows are independent
 * (each row's sum, or each element, is computed as it would be whole), so
 * the results do not change; the request completes when its last chunk and
 * every earlier one are done.
 *
 * Results.  `out`, when not NULL, must be page-locked host memory (for
 * example from cudaHostAlloc or a pinned tensor): GEMV writes m floats (c),
 * DOT one float (alpha), GER m * n floats (C, row-major, packed).  The copy
 * is done when the request's completion is returned by gb_engine_poll.
 *
 * Determinism.  Every kernel of a request depends only on its own shape
 * (and the engine's tuning table), so a request gives bit-identical results
 * alone and in any mix.
 *
 * Threads.  submit, poll, drain and stats may be called from any thread;
 * destroy from one thread once no other call is running.
 *
 * Host-only mode (GB_ENGINE_HOST_ONLY): no device is touched; the arena is
 * bookkeeping only and a step completes after (its operand bytes) /
 * sim_bytes_per_ns nanoseconds.  It exercises admission, batching, overlap
 * and failure handling without a GPU.
 *
 * Fault injection (host side): GB_FAULT_INJECT=step:<k> makes the k-th step
 * (1-based) complete without being launched: its requests (a request in
 * chunks once its other chunks are done) complete with status
 * GB_ERR_INJECTED and the engine goes on.
 */
#ifndef GBSERVE_H
#define GBSERVE_H

#include <stddef.h>
#include <stdint.h>

#include "gbblas.h"

#ifdef __cplusplus
extern "C" {
#endif

#define GB_ERR_BUDGET (-104)  /* the request alone exceeds the budget */
#define GB_ERR_TIMEOUT (-105) /* gb_engine_drain ran out of time */

typedef enum { GB_REQ_GEMV = 0, GB_REQ_DOT = 1, GB_REQ_GER = 2 } gb_req_op;
typedef enum { GB_FORM_F32 = 0, GB_FORM_BF16 = 1 } gb_req_form;
typedef enum { GB_ENGINE_HOST_ONLY = 1 } gb_engine_flags;
typedef enum { GB_REQ_POOL = 1 } gb_req_flags;

typedef struct {
  size_t budget_bytes;          /* HBM admission budget, >= 1 MiB */
  int32_t streams;              /* steps in flight at once, 1..16 */
  int32_t max_inflight;         /* admitted, unfinished requests at most, >= 1 */
  int32_t max_step_requests;    /* requests per step at most, >= 1 */
  int32_t flags;                /* gb_engine_flags */
  double sim_bytes_per_ns;      /* host-only mode: simulated bandwidth, > 0 */
  const gb_batch_tuning *table; /* GB_BATCH_BUCKETS entries (copied), or NULL */
  int64_t pool_elems;           /* resident operand pool: elements (0 = none, else a
                                   multiple of 8, at most 2^40) */
  uint64_t pool_seed;           /* generator seed of the pool */
  size_t chunk_bytes;           /* 0, or: pool GEMVs and GERs moving more than this
                                   are launched in row chunks of about this many
                                   bytes (see Chunks) */
} gb_engine_config;

typedef struct {
  int64_t id;         /* caller's tag, returned in the completion */
  int32_t op;         /* gb_req_op */
  int32_t form;       /* gb_req_form (GEMV only; others GB_FORM_F32) */
  int64_t m, n;       /* GEMV, GER: m x n (1 <= m, n <= 2^31 - 1); DOT: n (m ignored) */
  float alpha;        /* GEMV, GER: scale (DOT: ignored) */
  int32_t flags;      /* gb_req_flags */
  uint64_t seed;      /* operands from the generator with this seed */
  void *out;          /* page-locked host buffer for the result, or NULL */
  int64_t arrival_ns; /* arrival, gb_engine_now_ns clock; 0 = at submission */
} gb_request;

typedef struct {
  int64_t id;
  int32_t status; /* GB_OK, GB_ERR_CUDA or GB_ERR_INJECTED */
  int32_t op;
  int64_t arrival_ns, admitted_ns, launched_ns, done_ns;
  int64_t step;     /* index of the step it ran in (0-based) */
  int64_t bytes;    /* device bytes it held */
} gb_completion;

typedef struct {
  int64_t submitted, admitted, completed, failed, steps;
  int64_t inflight_peak;    /* admitted, unfinished requests, at most at once */
  int64_t steps_inflight_peak;
  size_t bytes_in_use, bytes_peak, budget_bytes;
  size_t pool_bytes;        /* device bytes of the operand pools (outside the budget) */
} gb_engine_stats;

typedef struct gb_engine gb_engine;

/* Monotonic clock of the engine, in nanoseconds. */
int64_t gb_engine_now_ns(void);

/* Create an engine (and start its worker thread).  Returns GB_OK and the
   handle in *out; -1 for an invalid config (NULL, a field out of range, an
   invalid table entry), -2 for out NULL, GB_ERR_CUDA if device memory, a
   stream or the thread cannot be had (nothing is left allocated).  With a
   pool, creation returns once the pools are filled. */
int gb_engine_create(const gb_engine_config *cfg, gb_engine **out);

/* Queue one request.  Returns GB_OK; -1 engine NULL; -2 request NULL or a
   field out of range (op, form, m, n, flags, out not page-locked;
   GB_REQ_POOL without a pool or with an operand longer than the pool);
   GB_ERR_BUDGET when its arena bytes alone exceed the budget. */
int gb_engine_submit(gb_engine *e, const gb_request *r);

/* Copy up to `max` completions (oldest first) into out; returns how many,
   or -1 for an invalid argument. */
int gb_engine_poll(gb_engine *e, gb_completion *out, int max);

/* Wait until every submitted request has completed, at most timeout_ms
   milliseconds.  GB_OK, GB_ERR_TIMEOUT or -1. */
int gb_engine_drain(gb_engine *e, int64_t timeout_ms);

/* Counters; -1 for an invalid argument. */
int gb_engine_stats_get(gb_engine *e, gb_engine_stats *out);

/* Arena bytes a request would hold (its operands, or its output alone
   with GB_REQ_POOL; 256-byte aligned pieces); 0 for an invalid request. */
size_t gb_engine_request_bytes(const gb_request *r);

/* Finish outstanding work (up to 60 s), stop the worker and free
   everything.  NULL is ignored. */
void gb_engine_destroy(gb_engine *e);

#ifdef __cplusplus
}
#endif

#endif /* GBSERVE_H */
