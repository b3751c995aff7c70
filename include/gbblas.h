/*
 * gbblas.h — C ABI of the GB300 (sm_103a) GEMV / DOT / GER library.
 *
 * The three operations are the problem definitions of Singh & Bassoy, "High
 * Performance Level-1 and Level-2 BLAS" (arXiv 2108.02025), Sec. 3.1, with a
 * scale alpha on GEMV and GER:
 *
 *   GEMV (Def. GEMV; Alg. 1 column-major, Alg. 2 row-major):
 *       c_i <- c_i + alpha * sum_j A_ij x_j,   i < m, j < n
 *   DOT  (Def. DOT; Algs. 3 and 4):
 *       *alpha <- *alpha + sum_p x_p y_p,      p < n   (alpha is the in/out
 *       accumulator of the definition, not a scale)
 *   GER  (Def. GEM; Alg. 2):
 *       C_ij <- fma(x_i, fl(alpha * y_j), C_ij) i < m, j < n
 *
 * Matrix element (i, j) is M[i*ld + j] for GB_ROW_MAJOR (ld >= max(1, n)) and
 * M[i + j*ld] for GB_COL_MAJOR (ld >= max(1, m)).  Vectors are contiguous
 * (unit stride).
 *
 * Memory and ownership.  Every pointer argument except the stream is a
 * DEVICE pointer owned by the caller (for example memory from PyTorch).  The
 * library never allocates, frees or synchronises: each call validates its
 * arguments on the host, enqueues its kernel(s) on `stream` and returns.
 * Results are ready when the stream reaches that point.  A NULL stream is
 * the legacy default stream.
 *
 * Workspace.  GEMV and DOT may split a sum across thread blocks; the partial
 * sums and the arrival counters that pick the block which finishes the sum
 * live in a caller-owned workspace of gb_workspace_bytes() bytes (0 means
 * none is needed and ws may be NULL).  The workspace must be 16-byte aligned
 * and zero-filled before its first use (gb_workspace_init, or memory that is
 * already zero); every call leaves its counters at zero again, so one
 * workspace serves any number of calls in stream order.  Two calls that run
 * at the same time (different streams) must not share a workspace.
 *
 * Determinism.  The split of every sum depends only on (op, dtype, layout,
 * m, n) and partial sums are combined in a fixed order with no floating
 * point atomics, so repeated calls give bit-identical results.
 *
 * Errors.  Every function returns GB_OK (0) or a negative status:
 *   -k (1 <= k < 100)  argument number k (1-based) is invalid; nothing was
 *                      enqueued.  This covers m or n < 0, a leading
 *                      dimension that is too small, a NULL pointer for a
 *                      non-empty operand, an unknown layout, an output that
 *                      overlaps an input, and a misaligned workspace;
 *   GB_ERR_WORKSPACE   ws_bytes < gb_workspace_bytes(...);
 *   GB_ERR_CUDA        the kernel launch failed (cudaPeekAtLastError);
 *   GB_ERR_INJECTED    a fault requested through the GB_FAULT_INJECT
 *                      environment variable (see below); nothing enqueued.
 * Quick returns (GB_OK, nothing read or written): m == 0 or n == 0 for GEMV
 * and GER; alpha == 0 for GEMV and GER; n == 0 for DOT (alpha unchanged).
 * Pointers of any alignment are accepted; misaligned operands take a scalar
 * GPU path.  There is no CPU fallback.
 *
 * Rounding.  IEEE round-to-nearest everywhere, no flush to zero.  GER is one
 * fma per element and therefore exact to the last bit.  GEMV and DOT
 * reassociate the sum (any order is a valid reading of the definitions):
 * FP32 GEMV sums at most 64 products in one FP32 chain and adds the chains
 * with a compensated FP32 sum (TwoSum), split partials in FP64; FP32 DOT
 * uses a compensated FP32 dot product per thread and FP64 above that; FP64
 * GEMV and DOT form part of their products in FP64 and part exactly with
 * FP32 instructions (each operand cut into two FP32 parts, TwoProduct,
 * TwoSum into an FP32 pair folded into the FP64 sum every 16 products or
 * fewer; each such product within 2.5 * 2^-45 of exact, each pair within
 * 7.8e-13 of the sum of |a x| of its products), operands outside
 * 2^-30 <= |v| < 2^34 always in FP64; the last reduction of DOT is FP64.
 *
 * Fault injection (host side, for failure tests): GB_FAULT_INJECT=<op>:<k>
 * with <op> one of gemv, dot, ger makes the k-th call (1-based, counted per
 * op within the process, after argument validation) return GB_ERR_INJECTED
 * without enqueuing anything.
 */
#ifndef GBBLAS_H
#define GBBLAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { GB_ROW_MAJOR = 0, GB_COL_MAJOR = 1 } gb_layout;
typedef enum {
  GB_OP_GEMV = 0,
  GB_OP_DOT = 1,
  GB_OP_GER = 2,
  GB_OP_GEMV_BF16 = 3, /* gb_gemv_bf16 (dtype ignored, row-major only) */
  GB_OP_GEMV_E4M3 = 4  /* gb_gemv_e4m3 (dtype ignored, row-major only) */
} gb_op;
typedef enum { GB_F32 = 0, GB_F64 = 1 } gb_dtype;

enum {
  GB_OK = 0,
  GB_ERR_WORKSPACE = -100,
  GB_ERR_UNSUPPORTED = -101,
  GB_ERR_CUDA = -102,
  GB_ERR_INJECTED = -103
};

/* A cudaStream_t passed as an opaque handle (NULL = legacy default stream). */
typedef void *gb_stream;

/* Library version, major*10000 + minor*100 + patch. */
int gb_version(void);

/* Text of a status code (static storage; never NULL). */
const char *gb_status_string(int status);

/* Bytes of workspace a call with these arguments needs (0 = none).  op is a
   gb_op, dtype a gb_dtype, layout a gb_layout (ignored for DOT; m ignored
   for DOT, where n is the vector length).  A pure function of its
   arguments: it touches no device.  Invalid arguments give 0. */
size_t gb_workspace_bytes(int op, int dtype, int layout, int64_t m, int64_t n);

/* Zero ws_bytes bytes at ws on `stream` (cudaMemsetAsync).  Call once on a
   fresh workspace.  Returns GB_OK, -1 if ws is NULL with ws_bytes > 0, or
   GB_ERR_CUDA. */
int gb_workspace_init(void *ws, size_t ws_bytes, gb_stream stream);

/* Copy `bytes` bytes from device memory `src` to page-locked host memory
   `dst` (cudaHostAlloc, cudaHostRegister or a pinned tensor) with a kernel
   on `stream` that stores through the host buffer's device mapping, so the
   copy uses no copy engine and overlaps copy-engine transfers in the other
   direction.  Any alignment (16-byte aligned pointers take the wide path).
   Returns GB_OK (also for bytes == 0), -1 if dst is NULL or not page-locked
   host memory, -2 if src is NULL or overlaps dst, GB_ERR_CUDA if the launch
   failed.  Not an operation of the paper: IO for callers whose results go
   back to host memory. */
int gb_copy_to_host(void *dst, const void *src, size_t bytes, gb_stream stream);

/* GEMV, Def. GEMV (Sec. 3.1), Alg. 1 (column-major) and Alg. 2 (row-major):
   c_i <- c_i + alpha * sum_j A_ij x_j for i < m.
     layout  GB_ROW_MAJOR or GB_COL_MAJOR                         (arg 1)
     m, n    rows and columns of A, >= 0                          (args 2, 3)
     alpha   scale of the product                                 (arg 4)
     A       device matrix, element (i, j) as described above     (arg 5)
     lda     leading dimension (row-major >= max(1,n), col-major
             >= max(1,m))                                         (arg 6)
     x       device vector of n elements, read only               (arg 7)
     c       device vector of m elements, read and written; must
             not overlap A or x                                   (arg 8)
     ws      device workspace (see above), 16-byte aligned        (arg 9)
     ws_bytes its size in bytes                                   (arg 10)
     stream  CUDA stream the kernels are enqueued on              (arg 11) */
int gb_dgemv(int layout, int64_t m, int64_t n, double alpha, const double *A, int64_t lda,
             const double *x, double *c, void *ws, size_t ws_bytes, gb_stream stream);
int gb_sgemv(int layout, int64_t m, int64_t n, float alpha, const float *A, int64_t lda,
             const float *x, float *c, void *ws, size_t ws_bytes, gb_stream stream);

/* DOT, Def. DOT (Sec. 3.1), Alg. 3 (one block for small n) and Alg. 4
   (blocks of the index range, then one combined sum for large n):
   *alpha <- *alpha + sum_p x_p y_p.
     n       vector length, >= 0                                  (arg 1)
     x, y    device vectors of n elements, read only              (args 2, 3)
     alpha   device pointer to ONE element, read and written;
             must not overlap x or y                              (arg 4)
     ws, ws_bytes, stream as for GEMV                             (args 5-7)
   The sum of products is formed in FP64 (FP32 inputs: compensated FP32
   per thread, FP64 above), added to *alpha in FP64 and rounded once to the
   element type. */
int gb_ddot(int64_t n, const double *x, const double *y, double *alpha, void *ws,
            size_t ws_bytes, gb_stream stream);
int gb_sdot(int64_t n, const float *x, const float *y, float *alpha, void *ws, size_t ws_bytes,
            gb_stream stream);

/* GER, Def. GEM (Sec. 3.1), Alg. 2: C_ij <- fma(x_i, t_j, C_ij) with
   t_j = fl(alpha * y_j), one rounding per element (bit-exact).  Every
   element of C has exactly one writer.
     layout  GB_ROW_MAJOR or GB_COL_MAJOR                         (arg 1)
     m, n    rows and columns of C, >= 0                          (args 2, 3)
     alpha   scale                                                (arg 4)
     x       device vector of m elements                          (arg 5)
     y       device vector of n elements                          (arg 6)
     C       device matrix, read and written; must not overlap
             x or y                                               (arg 7)
     ldc     leading dimension of C                               (arg 8)
     stream  CUDA stream                                          (arg 9)
   Needs no workspace. */
int gb_dger(int layout, int64_t m, int64_t n, double alpha, const double *x, const double *y,
            double *C, int64_t ldc, gb_stream stream);
int gb_sger(int layout, int64_t m, int64_t n, float alpha, const float *x, const float *y,
            float *C, int64_t ldc, gb_stream stream);

/* Reduced-precision storage of A (not in the paper, whose GEMV is FP64 /
   FP32): fewer bytes of A per product for the HBM-bound GEMV.  Row-major
   only; x and c stay FP32.

   gb_quantize_bf16: Q_ij = BF16(A_ij), the top 16 bits of the binary32
   rounded to nearest, ties to even.
     m, n (args 1, 2); A device FP32, row-major, lda >= max(1,n) (args 3, 4);
     Q device uint16 output, ldq >= max(1,n), not overlapping A (args 5, 6);
     stream (arg 7).
   gb_quantize_e4m3: per row i, s_i = fl32(amax_j |A_ij| / 448) and
   Q_ij = E4M3(fl32(A_ij / s_i)), OCP FP8 E4M3 (bias 7, 3 mantissa bits),
   round to nearest even, saturating at +-448; an all-zero row gets s_i = 0
   and codes 0.  A must be finite.
     m, n (1, 2); A, lda (3, 4); Q device uint8 output, ldq (5, 6);
     scales device FP32 output of m values (7); stream (8). */
int gb_quantize_bf16(int64_t m, int64_t n, const float *A, int64_t lda, uint16_t *Q, int64_t ldq,
                     gb_stream stream);
int gb_quantize_e4m3(int64_t m, int64_t n, const float *A, int64_t lda, uint8_t *Q, int64_t ldq,
                     float *scales, gb_stream stream);

/* GEMV with A stored in reduced precision:
     c_i <- c_i + alpha * s_i * sum_j Q_ij x_j   (s_i = 1 for BF16)
   The products are FP32 fmas of the exactly decoded codes with x, in chains
   of at most 32 folded into a compensated FP32 sum, then a fixed-order FP32
   block sum (split partials in FP64).  Row-major Q with 16-byte aligned
   rows (Q 16-byte aligned, ldq * element bytes a multiple of 16) and x
   16-byte aligned; otherwise the argument is reported invalid.  E4M3 codes
   0x7F and 0xFF (NaN) are not supported in Q (the quantiser never writes
   them).
   gb_gemv_bf16: m, n (1, 2); alpha (3); Q uint16, ldq (4, 5); x (6);
     c (7); ws, ws_bytes (8, 9) sized by gb_workspace_bytes(GB_OP_GEMV_BF16,
     0, GB_ROW_MAJOR, m, n); stream (10).
   gb_gemv_e4m3: m, n (1, 2); alpha (3); Q uint8, ldq (4, 5); scales (6);
     x (7); c (8); ws, ws_bytes (9, 10) sized by
     gb_workspace_bytes(GB_OP_GEMV_E4M3, ...); stream (11). */
int gb_gemv_bf16(int64_t m, int64_t n, float alpha, const uint16_t *Q, int64_t ldq,
                 const float *x, float *c, void *ws, size_t ws_bytes, gb_stream stream);
int gb_gemv_e4m3(int64_t m, int64_t n, float alpha, const uint8_t *Q, int64_t ldq,
                 const float *scales, const float *x, float *c, void *ws, size_t ws_bytes,
                 gb_stream stream);

/* Batched FP32 GEMV: `count` independent row-major problems
       c_p <- c_p + alpha_p * A_p x_p     (Def. GEMV, Sec. 3.1; m_p x n_p, lda_p)
   in ONE persistent kernel launch.  Not an operation of the paper: it is the
   GPU answer to the thread overhead that the paper finds dominating small
   problems (Sec. 4.1, speedup bound; Sec. 4.2, Analysis), here a launch per
   small GEMV.

   Plan, then launch.  gb_sgemv_batch_plan (host only, no CUDA call) writes
   the problems and their tiles into a caller-owned HOST buffer of
   gb_sgemv_batch_plan_bytes() bytes, 16-byte aligned.  The caller copies
   those bytes unchanged into DEVICE memory (16-byte aligned) and passes both
   copies to gb_sgemv_batch, which enqueues one kernel that reads only the
   device copy: the launch can be captured in a CUDA graph and replayed for
   as long as the operands stay where the plan says.  Problems with m, n or
   alpha zero are skipped (c untouched).  No c may overlap another problem's
   c, or any A or x of the batch.

   Tiling and tuning.  A problem's rows are cut into tiles of whole rows of
   about `tile_bytes` bytes of A (a multiple of the block's 256 / lanes_per_row
   row groups); each block of the launch processes the tiles whose cost
   falls in its equal share of the batch's total.  In a tile, groups of
   `lanes_per_row` lanes sum one row each, `packs_per_iter` 16-byte packs of
   A per lane in flight; every lane forms FP32 fma chains of at most 64
   products folded into a compensated FP32 sum (TwoSum), and the group adds
   its lanes by a fixed butterfly.  The parameters come from a table of
   GB_BATCH_BUCKETS entries indexed by the bucket ceil(log2(n_p)) (n_p = 1:
   bucket 0; a BF16 item of gb_batch_plan takes the bucket of ceil(n_p / 2),
   the same row length in 4-byte words); NULL selects the built-in table.  A row's result depends only
   on n_p and its bucket's entry: under the same table a problem gives
   bit-identical results alone or in any batch.  Problems whose A or x is not
   16-byte aligned, or whose lda is not a multiple of 4, take a scalar path
   in the same launch. */
#define GB_BATCH_BUCKETS 32
typedef struct {
  int32_t lanes_per_row;  /* 1, 2, 4, 8, 16 or 32 */
  int32_t packs_per_iter; /* 1, 2 or 4 */
  int32_t tile_bytes;     /* target bytes of A per tile, >= 4096 */
  int32_t reserved;       /* 0 */
} gb_batch_tuning;

/* The built-in table (GB_BATCH_BUCKETS entries written to `table`). */
void gb_sgemv_batch_default_tuning(gb_batch_tuning *table);

/* Bytes of the plan of a batch (a pure function of count, m, n, alpha and
   the table); 0 when count < 0, m or n is NULL with count > 0, some m_p or
   n_p is negative or above INT32_MAX, or the table has an invalid entry. */
size_t gb_sgemv_batch_plan_bytes(int64_t count, const int64_t *m, const int64_t *n,
                                 const float *alpha, const gb_batch_tuning *table);

/* Build the plan.  Host arrays of `count` entries: m (2), n (3), lda (4,
   >= max(1, n_p)), alpha (5), and DEVICE pointers A (6), x (7), c (8);
   table (9, NULL = built-in); plan (10), plan_bytes (11).  Returns GB_OK or
   -k for the first invalid argument k (including overlaps, reported on c,
   and m_p, n_p above INT32_MAX). */
int gb_sgemv_batch_plan(int64_t count, const int64_t *m, const int64_t *n, const int64_t *lda,
                        const float *alpha, const float *const *A, const float *const *x,
                        float *const *c, const gb_batch_tuning *table, void *plan,
                        size_t plan_bytes);

/* Enqueue the batch on `stream`: one launch.  plan_host (1) is the host
   plan (from gb_sgemv_batch_plan or gb_batch_plan; read for the launch
   size), plan_dev (2) its device copy.  Returns
   GB_OK, -1 (not a plan), -2 (plan_dev NULL or misaligned) or GB_ERR_CUDA. */
int gb_sgemv_batch(const void *plan_host, const void *plan_dev, gb_stream stream);

/* Number of tiles in a host plan (-1 if it is not a plan). */
int64_t gb_sgemv_batch_tiles(const void *plan_host);

/* Mixed batches: GEMVs with FP32 or BF16-stored A and GERs in one plan, run
   by the same launch (gb_sgemv_batch).  Problem p is described by an item:
     GB_BATCH_GEMV_F32   c <- c + alpha A x, A FP32 m x n (lda elements)
     GB_BATCH_GEMV_BF16  the same with A stored as BF16 codes (uint16, the
                         top half of the binary32, decoded exactly)
     GB_BATCH_GER_F32    C <- C + alpha x y^T as fma(x_i, fl(alpha y_j), C_ij)
                         (bit-exact, as gb_sger), C FP32 m x n (lda)
     GB_BATCH_DOT_F32    c[0] <- c[0] + A.x (Def. DOT, Sec. 3.1; Algs. 3-4
                         of Sec. 4.3), A and x FP32 n-vectors, m = 1,
                         alpha = 1: per-thread compensated products and
                         sums in FP32 (Dot2), the partials and the initial
                         c[0] summed in FP64, rounded once to FP32 (as
                         gb_sdot)
   Item fields: A = the matrix (GEMV: read; GER: C, read and written; DOT:
   the first vector); x = the n-vector (GEMV: x; GER: y; DOT: the second
   vector); c = the m-vector (GEMV: c, read and written; GER: x, read; DOT:
   the accumulator).  Items with m, n or alpha zero are skipped.  The
   16-byte path needs A and x 16-byte aligned and lda * element bytes a
   multiple of 16; otherwise a scalar path runs in the same launch.  No
   output (GEMV c, GER C) may overlap another output or any input.
   gb_batch_plan returns GB_OK, -1 (count < 0), -2 (an invalid item: kind,
   shape, lda, a NULL pointer of an active item, an overlap), -3 (table),
   -4 (plan NULL or misaligned), -5 (plan_bytes too small).
   gb_batch_plan_bytes returns 0 for an invalid count, kind, shape or table. */
typedef enum {
  GB_BATCH_GEMV_F32 = 0,
  GB_BATCH_GEMV_BF16 = 1,
  GB_BATCH_GER_F32 = 2,
  GB_BATCH_DOT_F32 = 3
} gb_batch_kind;
typedef struct {
  int32_t kind;     /* gb_batch_kind */
  int32_t reserved; /* 0 */
  int64_t m, n, lda;
  float alpha;
  int32_t reserved2; /* 0 */
  void *A;
  const float *x;
  float *c;
} gb_batch_item;
size_t gb_batch_plan_bytes(int64_t count, const gb_batch_item *items, const gb_batch_tuning *table);
int gb_batch_plan(int64_t count, const gb_batch_item *items, const gb_batch_tuning *table, void *plan,
                  size_t plan_bytes);

/* GEMV without allocation.  The paper has no counterpart: this entry point
   exists for callers that cannot allocate device memory (a runtime that owns
   the whole device heap, or code that must not allocate once it is set up)
   and so cannot pass the workspace of gb_dgemv.
   It computes exactly what gb_dgemv computes, with the same kernels, but its
   split sums use a scratch array of GB_NOALLOC_SCRATCH_BYTES compiled into
   the library, which every GPU that loads the library holds until the
   process exits.  It calls no cudaMalloc, cudaFree or other allocating
   routine.  Like every call here it uses the CUDA runtime, so it must not be
   called from a host callback or stream callback (cudaLaunchHostFunc),
   where CUDA calls are not allowed.
     Arguments 1-8 as for gb_dgemv; stream is argument 9.
     Returns what gb_dgemv returns, and GB_ERR_WORKSPACE (nothing enqueued)
     when the call would need more than GB_NOALLOC_SCRATCH_BYTES of scratch,
     that is when gb_workspace_bytes(GB_OP_GEMV, GB_F64, layout, m, n)
     exceeds it.  A call refused for any reason (invalid argument, too large,
     GB_FAULT_INJECT) enqueues nothing.
   The first call on a device looks up the array's device address with that
   device current (cudaGetSymbolAddress), and looks it up again when the
   device's context has changed (after cudaDeviceReset); make that first call
   before any stream capture.  A call that uses the array first zeroes its
   counters on `stream` (cudaMemsetAsync): the kernels return them to zero
   as they finish, but a call that did not run to the end, or that
   overlapped another, can leave them set, and the array otherwise keeps the
   previous call's contents.  All calls share the one array: calls that
   overlap on the GPU (different streams, different threads) race and give
   wrong results; serialise them. */
#define GB_NOALLOC_SCRATCH_BYTES ((size_t)256 << 10)  /* 256 KiB */
int gb_dgemv_noalloc(int layout, int64_t m, int64_t n, double alpha, const double *A,
                     int64_t lda, const double *x, double *c, gb_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* GBBLAS_H */
