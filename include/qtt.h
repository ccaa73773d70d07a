/*
 * qtt.h -- C-ABI of libqtt: QTT matrix x dense-vector products on one GB300
 * GPU (sm_103a), and the solves built on them.
 *
 * The operation is the "matrix-vector product for an uncompressed vector" of
 * Corona, Rahimian and Zorin, "A Tensor-Train accelerated solver for integral
 * equations in complex geometries" (Sec. 4.2, Algorithm 2): a matrix A of
 * size 2^d x 2^d held in quantized tensor-train (QTT) format is applied to
 * dense vectors of length N = 2^d by contracting one core at a time.
 *
 * Conventions used by every entry point:
 *   - Cores.  A QTT matrix has d cores; core k (k = 0..d-1) is
 *     G_k(alpha_k, i_k, j_k, alpha_{k+1}) with ranks ranks[k], ranks[k+1]
 *     and ranks[0] = ranks[d] = 1 (Sec. 2.2, eq. (TTdeccores) and the dummy
 *     ranks; matrix cores on the product tree with b_k = (i_k, j_k),
 *     Sec. 3.1).  They are passed as ONE host array of doubles holding the
 *     cores one after another, each in C order
 *     [ranks[k]][2 (row bit i_k)][2 (column bit j_k)][ranks[k+1]].
 *   - Index.  Element t of a vector is indexed least-significant bit first:
 *     t = sum_k t_k 2^k, bit k belonging to core k (the paper's Matlab
 *     reshape order, Sec. 2.1, with the finest tree level first, Sec. 2.4).
 *     A(i, j) = G_0[i_0, j_0] G_1[i_1, j_1] ... G_{d-1}[i_{d-1}, j_{d-1}].
 *   - Vectors.  nrhs vectors of length N stored one after another with
 *     leading dimension ld >= N elements (column-major N x nrhs), in DEVICE
 *     memory owned by the caller unless an entry point says otherwise.
 *   - Streams.  `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream).  Calls are asynchronous on that stream unless stated.
 *   - Errors.  No exception crosses the ABI.  Every size and pointer is
 *     validated before any launch; invalid input returns QTT_ERR_INVALID_ARG
 *     and launches nothing.  Device memory is checked against free memory
 *     before allocation and a shortfall returns QTT_ERR_OOM.  A CUDA error
 *     returns QTT_ERR_CUDA (the message is kept for qtt_last_error()).
 *   - Threads.  Distinct operators may be used from distinct threads.  One
 *     operator may be applied concurrently on several streams: it is
 *     read-only after qtt_create.
 *   - Devices.  An operator lives on the device that was current at
 *     qtt_create; every call that uses it needs that device current and
 *     returns QTT_ERR_INVALID_ARG otherwise.
 */
#ifndef QTT_H_
#define QTT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qtt_op qtt_op; /* opaque; cores resident in device memory */

typedef enum {
  QTT_OK = 0,
  QTT_ERR_INVALID_ARG = 1,
  QTT_ERR_OOM = 2,
  QTT_ERR_CUDA = 3,
  QTT_ERR_NOT_CONVERGED = 4,
  QTT_ERR_TIMEOUT = 5,
  QTT_ERR_UNSUPPORTED = 6,
  QTT_ERR_CHECK = 7  /* checked build only: a kernel met an out-of-range index */
} qtt_status;

/* Element / arithmetic types.  QTT_TF32 names FP32 storage with operands
 * rounded to TF32 (round to nearest) before each multiply. */
typedef enum { QTT_F64 = 0, QTT_F32 = 1, QTT_TF32 = 2, QTT_BF16 = 3 } qtt_dtype;

/* Bits of `precision_mask` in qtt_create: which packed copies of the cores
 * to build besides FP64 (always built). */
#define QTT_PACK_F32 (1u << 1)
#define QTT_PACK_TF32 (1u << 2)
#define QTT_PACK_BF16 (1u << 3)

/* qtt_create -- copy a QTT matrix to the device (Algorithm 2, step 5: each
 * core is permuted once into the (2 r_{k+1}) x (2 r_k) matrix M_k that the
 * contraction multiplies; here that packing happens once, at creation).
 *   out    : receives the operator handle (set to NULL on failure).
 *   d      : number of cores, 1 <= d <= 30.
 *   ranks  : host array of d+1 ints, ranks[0] = ranks[d] = 1, 1 <= ranks[k]
 *            <= 4096.
 *   cores  : host array of d pointers; cores[k] holds the 4 ranks[k]
 *            ranks[k+1] doubles of core k (layout above).  Copied; the
 *            caller keeps ownership.
 *   precision_mask : QTT_PACK_* bits for the reduced-precision copies.
 *   stream : stream for the uploads; the call returns after they finish.
 * Errors: QTT_ERR_INVALID_ARG (bad d, ranks, NULL pointers),
 *         QTT_ERR_OOM, QTT_ERR_CUDA. */
qtt_status qtt_create(qtt_op **out, int d, const int *ranks,
                      const double *const *cores, unsigned precision_mask,
                      void *stream);
/* qtt_create_flat -- the same, with the cores concatenated in one host array
 * (core k at offset sum_{l<k} 4 ranks[l] ranks[l+1]). */
qtt_status qtt_create_flat(qtt_op **out, int d, const int *ranks,
                           const double *cores, unsigned precision_mask,
                           void *stream);

/* The .qtt operator file (no counterpart in the paper): a 24-byte header --
 * magic "QTT1", format version 1, d, element type 0 (FP64), core layout 0
 * (the layout above), a reserved word; every field a little-endian uint32
 * -- then the d + 1 ranks (uint32) and the cores as little-endian FP64, in
 * qtt_create's order.  Host-only.
 * qtt_write_file: d, ranks, cores as for qtt_create; QTT_ERR_INVALID_ARG for
 *   bad arguments or an I/O failure.
 * qtt_read_file: sets *d and *cores_len (sum_k 4 r_k r_{k+1}); fills ranks
 *   (ranks_cap >= d + 1) and cores (cores_cap >= *cores_len) when they are
 *   not NULL, so a first call with NULL arrays sizes the buffers.
 *   QTT_ERR_INVALID_ARG for a missing or malformed file (magic, d, ranks,
 *   length) or too small a buffer, QTT_ERR_UNSUPPORTED for another version,
 *   element type or layout. */
qtt_status qtt_write_file(const char *path, int d, const int *ranks, const double *cores);
qtt_status qtt_read_file(const char *path, int *d, int *ranks, int ranks_cap, double *cores,
                         int64_t cores_cap, int64_t *cores_len);

/* qtt_destroy -- release the operator.  Returns at once: its device memory
 * goes back to the library's pool once the work already queued that reads
 * it has finished (every apply, solve, plan replay and batch run records
 * its use on its stream), without synchronising the device or holding up
 * other streams.  NULL is a no-op.  The handle is invalid afterwards. */
qtt_status qtt_destroy(qtt_op *A);

/* Queries (host-side, no device work). */
int qtt_op_d(const qtt_op *A);
int qtt_op_rank(const qtt_op *A, int k); /* ranks[k], 0 <= k <= d, else -1 */
/* 4 N sum_k r_k r_{k+1}: floating-point operations of one apply per right-
 * hand side (Sec. 4.2: 2 m_k r_{k+1} r_k N per core, m_k = n_k = 2). */
double qtt_op_flops(const qtt_op *A);

/* qtt_apply -- y = A x for nrhs right-hand sides (Algorithm 2, the
 * uncompressed-vector product).  The sweep runs over k = 0..d-1; step k
 * contracts column bit j_k and rank alpha_k of the intermediate with core k
 * and produces row bit i_k and rank alpha_{k+1} (the column merge, the
 * product phi_k = M_k b_k and the row split of Algorithm 2 fused: the
 * merge and split are addressing only).
 *   x, y     : device pointers, N x nrhs, leading dimension ld (elements),
 *              element type io_dtype.  x and y must not overlap.
 *   nrhs     : >= 0 (0 is a no-op).
 *   ld       : >= N.
 *   io_dtype : element type of x and y.
 *   compute  : arithmetic of the contraction: QTT_F64 (FP64 multiply-adds),
 *              QTT_F32 (FP32), QTT_TF32 (TF32 operands, FP32 accumulate) or
 *              QTT_BF16 (BF16 cores and intermediates, FP32 accumulate).
 *              The operator must have been created with the matching
 *              QTT_PACK_* bit for the reduced precisions.
 *   stream   : cudaStream_t.
 * Scratch for the intermediate (max_k r_k x N x nrhs elements, two
 * buffers) is taken stream-ordered from a pool owned by the library.
 * Errors: QTT_ERR_INVALID_ARG, QTT_ERR_UNSUPPORTED (combination not built),
 *         QTT_ERR_OOM, QTT_ERR_CUDA. */
qtt_status qtt_apply(const qtt_op *A, const void *x, void *y, int64_t nrhs,
                     int64_t ld, qtt_dtype io_dtype, qtt_dtype compute,
                     void *stream);

/* qtt_apply_host -- qtt_apply with x and y in HOST memory: x goes to the
 * device, the apply runs, y comes back, all ordered on `stream`.  With more
 * than one chunk the right-hand sides pass through two device staging slots
 * so that the copy of chunk i+1 in, the apply of chunk i and the copy of
 * chunk i-1 out overlap (the copies on two streams the library keeps per
 * device, ordered by events; the applies on `stream`).
 *   x_host, y_host : host pointers, N x nrhs, leading dimension ld, element
 *                    type io_dtype (QTT_F64, QTT_F32 or QTT_BF16); they must
 *                    not overlap.  Page-locked memory (cudaHostAlloc,
 *                    cudaHostRegister) lets the copies run asynchronously;
 *                    pageable memory works, but then the copies block the
 *                    calling thread and nothing overlaps.
 *   nrhs, ld, io_dtype, compute : as for qtt_apply.
 *   chunk  : right-hand sides per chunk; 0 lets the library choose (a
 *            quarter of nrhs, at most 1 GiB of staging for x and y).
 *   stream : cudaStream_t; the call returns once the work is queued, and
 *            y_host holds the result when the stream has drained.
 * Staging (2 slots x chunk x N x element size, for x and y) comes from the
 * library's stream-ordered pool.  Every right-hand side's result is bitwise
 * what qtt_apply gives it.  Rows ld > N of y_host keep their padding.
 * Errors: as qtt_apply; QTT_ERR_UNSUPPORTED for a device index above 63. */
qtt_status qtt_apply_host(const qtt_op *A, const void *x_host, void *y_host,
                          int64_t nrhs, int64_t ld, qtt_dtype io_dtype,
                          qtt_dtype compute, int64_t chunk, void *stream);

/* ------------------------------------------------------------ fusion plan */
/* How an apply in each arithmetic runs -- which steps are merged into one
 * launch and on which kernels -- is a per-operator plan; the paper has no
 * counterpart (its Algorithm 2 runs one step at a time).  Plan codes:
 * fusion + 2 pairs + 8 groups2 + 16 staged, where
 *   fusion  (1): merge steps -- the first and last 2-3 low-rank steps in one
 *                launch each, middle steps in fused pairs (merge depth 2);
 *                0: one launch per step;
 *   pairs   (0-2): fused-pair family for BF16: 2 tcgen05 (TMA + TMEM),
 *                1 mma.sync, 0 no pairs;
 *   groups2 (1): tcgen05 pairs with two epilogue groups (else as many as
 *                fit beside three input stages);
 *   staged  (1): FP32/TF32 single steps on the shared-memory staged kernel.
 * The untuned plan is 1 + 4 + 16 = 21.
 * qtt_apply_autotune: times every candidate plan for `compute` on this
 *   operator with nrhs right-hand sides (one warm-up, then `reps` applies
 *   each, on `stream`; the arithmetic does not depend on the values, so the
 *   vectors are zeros from the library's scratch) and keeps the fastest for
 *   later qtt_apply calls in that arithmetic; *plan and *seconds (per apply)
 *   receive the choice.  Synchronises `stream`.
 * qtt_apply_set_plan / qtt_apply_get_plan: set or read the plan of one
 *   arithmetic (e.g. a choice cached from an earlier process).
 * Every plan computes the same product; plans differ in rounding only where
 * the arithmetic itself differs (the fused BF16 pairs keep the unfused
 * rounding points).  Errors: QTT_ERR_INVALID_ARG, QTT_ERR_OOM, QTT_ERR_CUDA. */
qtt_status qtt_apply_autotune(qtt_op *A, int64_t nrhs, qtt_dtype compute, int reps, void *stream,
                              int *plan, double *seconds);
qtt_status qtt_apply_set_plan(qtt_op *A, qtt_dtype compute, int plan);
qtt_status qtt_apply_get_plan(const qtt_op *A, qtt_dtype compute, int *plan);

/* qtt_apply_noalloc -- y = A x in FP64 without allocating any memory.  The
 * paper has no counterpart: this exists for callers that cannot allocate
 * device memory at the time they apply an operator -- for instance a process
 * whose device memory is already reserved by another allocator (a framework
 * arena or a budget fixed at start-up), or a latency-bound loop where an
 * allocation call could synchronise the device or fail under fragmentation.
 * Same product, layout and arguments as qtt_apply with io_dtype = compute =
 * QTT_F64; the two intermediate buffers of the sweep live in one static
 * device array of 64 MiB (8,388,608 doubles) that every GPU loading the
 * library holds until the process exits.
 *   Limit : d > 1 needs 2 x max_{0<k<d} ranks[k] x N x nrhs <= 8,388,608
 *           doubles; larger calls return QTT_ERR_INVALID_ARG (use qtt_apply).
 *   Set-up: the array is committed on a device when the module holding it
 *           is first loaded there.  qtt_create does that (it allocates the
 *           operator anyway), so create the operator on each device BEFORE
 *           handing the rest of the device's memory to another allocator;
 *           qtt_apply_noalloc then allocates nothing.  Each call looks up
 *           the array's device address with the current device (which must
 *           be the operator's).  After a device reset the module and the
 *           64 MiB are loaded again by the next lookup.
 *   Races : every call on a device shares the one array, which keeps the
 *           last call's contents (nothing in it needs to start at zero).
 *           Calls whose work overlaps on the GPU -- on different streams, or
 *           from different threads -- race on it; order them.
 * Calls no cudaMalloc, cudaFree or other allocating routine.
 * Errors: QTT_ERR_INVALID_ARG, QTT_ERR_CUDA. */
qtt_status qtt_apply_noalloc(const qtt_op *A, const double *x, double *y,
                             int64_t nrhs, int64_t ld, void *stream);

/* ------------------------------------------------------ recorded applies */
/* qtt_plan_* -- one qtt_apply recorded once as a CUDA graph and replayed.
 * The paper has no counterpart: a small operator (the 8^3 volume problem has
 * d = 9) spends more time launching its d kernels than running them, and a
 * replay issues the whole sweep (its scratch allocation and every step) as
 * one graph launch.
 *   qtt_plan_create : records y = A x exactly as qtt_apply(A, x, y, nrhs, ld,
 *                     io_dtype, compute) would run it (same checks, same
 *                     kernels) on a private stream; nothing is executed.
 *                     The addresses x, y (device, caller-owned) are fixed in
 *                     the plan: their CONTENTS are read and written at each
 *                     replay.  A must outlive the plan.  Returns the same
 *                     errors as qtt_apply, or QTT_ERR_CUDA if the runtime
 *                     refuses to record it.
 *   qtt_plan_run    : one replay, asynchronous on `stream` (ordered after
 *                     prior work on it); the result is bitwise that of
 *                     qtt_apply with the same arguments.
 *   qtt_plan_destroy: frees the graph (NULL is a no-op).
 * A plan may be run on several streams, but replays of one plan must not
 * overlap (they share x, y and the graph's scratch). */
typedef struct qtt_plan qtt_plan;
qtt_status qtt_plan_create(qtt_plan **out, const qtt_op *A, const void *x, void *y,
                           int64_t nrhs, int64_t ld, qtt_dtype io_dtype, qtt_dtype compute);
qtt_status qtt_plan_run(qtt_plan *P, void *stream);
qtt_status qtt_plan_destroy(qtt_plan *P);

/* ---------------------------------------------------- compressed vectors */
/* qtt_apply_tt -- the compressed matrix-vector product c = A b of Sec. 4.2,
 * for a right-hand side b given in QTT form: core k of c merges A's and b's
 * rank pairs (alpha, beta) into alpha s_k + beta and sums over the column
 * bit j_k:
 *   C_k[alpha s + beta][i][alpha' s' + beta']
 *       = sum_j G_k[alpha][i][j][alpha'] b_k[beta][j][beta'],
 * so c's ranks are r_k s_k (no rounding).  Each entry is computed in FP64
 * as fma(a_1, b_1, fl(a_0 b_0)) (one product, one fused multiply-add).
 *   b_ranks : host array of d + 1 ranks s_0 .. s_d (s_0 = s_d = 1, each in
 *             [1, 4096], every r_k s_k <= 32767), d = A's d.
 *   b_cores : device FP64, b's cores back to back, core k [s_k][2][s_{k+1}]
 *             C order (bit j_k of the vector index, least significant
 *             first, as for x in qtt_apply).
 *   c_cores : device FP64, caller-owned, qtt_apply_tt_size() elements; c's
 *             cores back to back, core k [r_k s_k][2][r_{k+1} s_{k+1}].
 * Asynchronous on `stream`; d launches.  Errors: QTT_ERR_INVALID_ARG (NULL
 * pointer, bad ranks, sizes past the limits), QTT_ERR_CUDA. */
qtt_status qtt_apply_tt_size(const qtt_op *A, const int *b_ranks, int64_t *n_elems);
qtt_status qtt_apply_tt(const qtt_op *A, const int *b_ranks, const double *b_cores,
                        double *c_cores, void *stream);

/* ------------------------------------------------ general mode sizes */
/* A QTT matrix whose core k has m_k row modes and n_k column modes (the
 * tensorisation of Sec. 3.1 with m_k x n_k modes; Sec. 4.2 counts 2 m_k n_k
 * r_k r_{k+1} flops per column of a core step), so that the matrix is
 * (prod m_k) x (prod n_k) -- rectangular when the products differ.
 *   qtt_gcreate : d in [1, 60]; ranks[0..d] with ranks[0] = ranks[d] = 1,
 *                 each in [1, 4096]; m[k], n[k] in [1, 16]; cores: host FP64,
 *                 core k as [ranks[k]][m[k]][n[k]][ranks[k+1]] in C order,
 *                 back to back (copied; the caller keeps ownership).  The
 *                 row index is i = sum_k i_k prod_{l<k} m_l and the column
 *                 index j = sum_k j_k prod_{l<k} n_l (first mode fastest, as
 *                 for the binary operators).  Returns after the uploads on
 *                 `stream`.  Errors: QTT_ERR_INVALID_ARG, QTT_ERR_OOM,
 *                 QTT_ERR_CUDA.
 *   qtt_gapply  : y = A x (transpose = 0: x has prod n_k entries per
 *                 right-hand side, y prod m_k) or y = A^T x (transpose = 1:
 *                 the lengths exchanged), FP64, by the sweep of Algorithm 2
 *                 with mixed-radix positions.  x, y: device FP64, nrhs
 *                 columns with leading dimensions ldx, ldy >= their
 *                 lengths; no overlap.  Scratch (two buffers of the largest
 *                 intermediate) from the library's pool; right-hand sides in
 *                 chunks when it is short.  Asynchronous on `stream`.
 *                 Errors: QTT_ERR_INVALID_ARG, QTT_ERR_OOM, QTT_ERR_CUDA.
 *   qtt_gdestroy: releases A after the work queued on it (no device-wide
 *                 synchronisation); NULL is a no-op.
 *   qtt_gop_rows/cols: prod m_k / prod n_k (-1 for NULL);
 *   qtt_gop_flops: flops of one apply per right-hand side (transposed or
 *                 not). */
typedef struct qtt_gop qtt_gop;
qtt_status qtt_gcreate(qtt_gop **out, int d, const int *ranks, const int *m, const int *n,
                       const double *cores, void *stream);
qtt_status qtt_gapply(const qtt_gop *A, const double *x, double *y, int64_t nrhs,
                      int64_t ldx, int64_t ldy, int transpose, void *stream);
qtt_status qtt_gdestroy(qtt_gop *A);
int64_t qtt_gop_rows(const qtt_gop *A);
int64_t qtt_gop_cols(const qtt_gop *A);
double qtt_gop_flops(const qtt_gop *A, int transpose);

/* ----------------------------------------- whole-core QTT operations */
/* qtt_tt_round -- TT rounding of a QTT vector or matrix held on the device
 * (the recompression that keeps the ranks of the compressed product of
 * Sec. 4.2 bounded; Tables 1-2, "QTT Solve"): left-to-right Householder QR
 * orthogonalisation, then right-to-left truncated SVDs of the unfoldings,
 * each keeping the smallest rank whose discarded singular values have 2-norm
 * <= eps ||t||_F / sqrt(d - 1) -- the threshold of Algorithm 1 -- so that
 * ||t - round(t)||_F <= eps ||t||_F.  FP64 throughout.
 *   d, ranks : d cores, ranks[0..d] with ranks[0] = ranks[d] = 1, each in
 *              [1, 32768]; n: entries per mode, 1..256 (2 for a QTT vector,
 *              4 for a binary QTT matrix, whose core [r][2][2][r'] is
 *              [r][4][r'] here).
 *   cores_in : device FP64, core k as [ranks[k]][n][ranks[k+1]] in C order,
 *              back to back (not modified).
 *   eps      : >= 0 (0 drops only exactly-zero singular values).
 *   ranks_out: host, d + 1 ints, the rounded ranks (never above the input
 *              ranks).
 *   cores_out: device FP64 with room for the INPUT cores (the rounded cores,
 *              same layout, back to back, fit in it); may equal cores_in.
 * Synchronous: it reads each unfolding's singular values back to choose the
 * rank, and returns when cores_out is written.  Scratch (a few copies of the
 * largest core) from the library's pool.  Errors: QTT_ERR_INVALID_ARG,
 * QTT_ERR_OOM, QTT_ERR_CUDA. */
qtt_status qtt_tt_round(int d, const int *ranks, int n, const double *cores_in, double eps,
                        int *ranks_out, double *cores_out, void *stream);

/* qtt_tt_svd -- Algorithm 1 (TT-SVD) on the device: the QTT decomposition
 * of a dense 2^d x 2^d matrix A (device FP64, row-major, A(i, j) at i 2^d +
 * j, 1 <= d <= 13).  The tensor's modes are the bit pairs (i_k, j_k),
 * k = 0 .. d-1, least significant first; each unfolding is split by a
 * truncated SVD that keeps the smallest rank whose discarded singular values
 * have 2-norm <= eps ||A||_F / sqrt(d - 1), so ||A - A_tt||_F <= eps
 * ||A||_F.  The cores come out in qtt_create's layout ([r_k][2 i][2 j]
 * [r_{k+1}], back to back) in cores_out (device FP64, `capacity` doubles);
 * ranks_out (host, d + 1) and *n_out (doubles needed) are always set.  If
 * capacity < *n_out nothing is written and QTT_ERR_INVALID_ARG is returned
 * (call again with room).  Synchronous, like qtt_tt_round.  Errors:
 * QTT_ERR_INVALID_ARG, QTT_ERR_OOM, QTT_ERR_CUDA. */
qtt_status qtt_tt_svd(int d, const double *A, double eps, int *ranks_out, double *cores_out,
                      int64_t capacity, int64_t *n_out, void *stream);

/* qtt_op_product -- C = A B for two QTT matrices of the same d, core by core
 * (Sec. 4.2: the compressed product, with a QTT matrix in place of the
 * vector; e.g. K^2 for a Neumann preconditioner or M Y for a product
 * preconditioner): C_k[a s + b][i][p][a' s' + b'] = sum_j A_k[a][i][j][a']
 * B_k[b][j][p][b'] (s, s' = B's ranks), each entry fl(fl(A_0 B_0) +
 * fl(A_1 B_1)).  c_ranks (host, d + 1) receives r_k s_k (each must be <=
 * 32768); c_cores (device FP64, `capacity` doubles, at least
 * 4 sum_k r_k s_k r_{k+1} s_{k+1}) receives C's cores in qtt_create's layout.
 * Asynchronous on `stream`.  Errors: QTT_ERR_INVALID_ARG, QTT_ERR_CUDA. */
qtt_status qtt_op_product(const qtt_op *A, const qtt_op *B, double *c_cores, int64_t capacity,
                          int *c_ranks, void *stream);

/* qtt_tt_sum -- sum_t coefs[t] T_t of nterms QTT tensors with d cores and n
 * entries per mode (2: vectors, 4: binary matrices), by concatenating the
 * ranks (Sec. 3.3: the ranks of a sum add up): first cores side by side,
 * middle cores block-diagonal, last cores stacked and scaled by coefs[t].
 *   ranks[t]  : host, d + 1 ints of term t (ranks[t][0] = ranks[t][d] = 1);
 *   cores[t]  : device FP64, term t's cores back to back ([r][n][r']);
 *   ranks_out : host, d + 1 ints, the summed ranks;
 *   cores_out : device FP64, `capacity` doubles (at least sum_k n R_k
 *               R_{k+1} for the summed ranks R), must not overlap the terms.
 * Asynchronous on `stream`.  Errors: QTT_ERR_INVALID_ARG, QTT_ERR_CUDA. */
qtt_status qtt_tt_sum(int d, int n, int nterms, const int *const *ranks,
                      const double *const *cores, const double *coefs, int *ranks_out,
                      double *cores_out, int64_t capacity, void *stream);

/* qtt_local_apply -- the left-hand side of the inversion's local linear
 * system (appendix on local linear systems; Sec. 4.1): with X in QTT form and
 * every core but W_k fixed, the reduced operator applied to W_k is the
 * three-core product
 *   y[b][i][p][B] = sum_{a, g, j, A, C} Psi[a][b][g] G[a][i][j][A] Phi[A][B][C]
 *                                        W[g][j][p][C]
 * (a, A: ranks of the operator's core G = G_k; b, g and B, C: ranks of X
 * before and after core k; i, j, p: mode bits), evaluated as three FP64 GEMMs
 * with two reorderings.
 *   ra, ra2 : operator ranks r_k, r_{k+1}; rx, rx2: X's ranks.
 *   psi     : device, [ra][rx][rx]; G: [ra][2][2][ra2]; phi: [ra2][rx2][rx2].
 *   W, y    : device, nvec blocks of [rx][2][2][rx2] back to back (y must not
 *             overlap the inputs).
 * Asynchronous on `stream`; scratch from the library's pool.  Errors:
 * QTT_ERR_INVALID_ARG, QTT_ERR_OOM, QTT_ERR_CUDA. */
qtt_status qtt_local_apply(int ra, int ra2, int rx, int rx2, const double *psi, const double *G,
                           const double *phi, const double *W, double *y, int64_t nvec,
                           void *stream);

/* qtt_residual -- r = f - (a x + K x), all FP64, the forward residual of the
 * second-kind system (a I + K) x = f (Sec. 3, eq. (nystrom): A = a I +
 * B K W C), with the subtraction fused into the last core step of the K
 * apply.  f, x, r: device FP64, N x nrhs, leading dimension ld; r must not
 * overlap f or x.  Errors as qtt_apply. */
qtt_status qtt_residual(const qtt_op *K, double a, const double *f,
                        const double *x, double *r, int64_t nrhs, int64_t ld,
                        void *stream);

/* ---------------------------------------------------------------- solves */
typedef enum {
  QTT_SOLVE_DIRECT = 0, /* x = P f: a QTT inverse used as a direct solver
                           (Tables 1-2, "Solve" column).  K unused. */
  QTT_SOLVE_GMRES = 1,  /* right-preconditioned GMRES(restart) with P
                           (Sec. 5.3: QTT preconditioner inside GMRES). */
  QTT_SOLVE_REFINE = 2  /* iterative refinement x <- x + M (f - (a I + K) x)
                           with the residual in FP64 (mixed-precision
                           refinement): M = P, or inner_iters steps of
                           a low-precision Richardson iteration on
                           (a I + K) z = r preconditioned by P. */
} qtt_solve_kind;

typedef struct {
  qtt_solve_kind kind;
  double a;              /* A = a I + K */
  double tol;            /* stop when ||f - A x||_2 <= tol ||f||_2 */
  int restart;           /* GMRES cycle length m (>= 1) */
  int max_iter;          /* cap on outer corrections (REFINE) or Arnoldi steps */
  qtt_dtype precond_compute; /* arithmetic of the P applies (and of the inner
                                K applies of REFINE) */
  int inner_iters;       /* REFINE and GMRES: the correction / flexible
                            preconditioner is M r = P r when 0; when s > 0,
                            s inner steps z <- z + P (r - (a z + K z)) from
                            z = P r (P = identity if NULL) with K and P
                            applied in precond_compute and vectors in FP64.
                            K then needs the matching QTT_PACK_* copy. */
} qtt_solve_params;

typedef struct {
  int iters;           /* P applications (REFINE), Arnoldi steps (GMRES) */
  double rel_residual; /* final ||f - A x|| / ||f||, FP64 */
  qtt_status status;   /* QTT_OK or QTT_ERR_NOT_CONVERGED */
} qtt_solve_info;

/* qtt_solve -- solve (a I + K) x = f for nrhs right-hand sides.
 *   K     : forward operator (may be NULL for DIRECT).
 *   P     : preconditioner / approximate inverse (NULL = identity; required
 *           for DIRECT).
 *   f, x  : device FP64, N x nrhs, leading dimension ld.  x is output only
 *           (the initial guess is 0 for GMRES, P f for REFINE).
 *   info  : host array of nrhs entries, filled on return.
 * The call synchronises `stream` (convergence tests read one norm per RHS
 * and iteration back to the host).  Returns QTT_ERR_NOT_CONVERGED if any
 * right-hand side missed tol within max_iter (x holds the last iterate).
 * Scratch (Krylov basis (restart+1) x N x nrhs FP64 for GMRES) comes from
 * the library's pool; QTT_ERR_OOM if it does not fit. */
qtt_status qtt_solve(const qtt_op *K, const qtt_op *P, const double *f,
                     double *x, int64_t nrhs, int64_t ld,
                     const qtt_solve_params *prm, qtt_solve_info *info,
                     void *stream);

/* ------------------------------------------------------- batched applies */
/* A batch applies many independent, uneven QTT operators (different d,
 * ranks and numbers of right-hand sides) to their own vectors: y_i = A_i x_i.
 * Each wave of operators whose scratch fits the memory budget is ONE
 * persistent kernel launch that walks a step-major work list of (operator,
 * core step, right-hand side, chunk of position pairs) items, each item one
 * Algorithm 2 contraction; an item waits (bounded) until its operator's
 * previous step is complete.  All waves are captured in one CUDA graph at
 * creation; qtt_batch_run replays it.  Some operators are not put in a wave
 * but applied with the single-operator apply after the graph, on the same
 * stream: with QTT_TF32 every operator whose TF32 apply runs step pairs on
 * the tcgen05 tensor cores (ranks 8..40 in its middle steps), with QTT_F32
 * every operator with d >= 16 (one such operator fills the GPU).  The paper
 * has no batched form; it is the same Algorithm 2 per operator.
 *   ops[i], nrhs[i] (>= 1), x[i], y[i] (device FP32, N_i x nrhs[i], leading
 *   dimension ld[i] >= N_i), bound at creation and read at every run.
 *   compute     : QTT_F32 or QTT_TF32 (operands rounded to TF32, FP32
 *                 accumulate); each operator needs the matching QTT_PACK_*.
 *   mem_budget  : bytes of intermediate per wave (0 = min(free/3, 64 GiB)).
 * Ranks above 48 return QTT_ERR_UNSUPPORTED. */
typedef struct qtt_batch qtt_batch;
qtt_status qtt_batch_create(qtt_batch **out, int nops, const qtt_op *const *ops,
                            const int64_t *nrhs, const void *const *x,
                            void *const *y, const int64_t *ld,
                            qtt_dtype compute, size_t mem_budget,
                            void *stream);
/* Launch the captured graph on `stream` (asynchronous). */
qtt_status qtt_batch_run(qtt_batch *B, void *stream);
/* qtt_batch_run_host -- the same run with every operator's x and y in HOST
 * memory: x_host[i] and y_host[i] are N_i x nrhs_i FP32 arrays, compact
 * (leading dimension N_i = 2^d_i), best page-locked.  The batch's device
 * vectors (given at creation) serve as the staging: the wave operators'
 * inputs are copied in, the waves run, their outputs are copied out while
 * the directly applied operators run, each of those with its input copied
 * in ahead and its output copied out behind it (two copy streams the
 * library keeps per device, ordered by events; the applies on `stream`).
 * Returns once queued; y_host is complete when `stream` has drained.  The
 * results are bitwise qtt_batch_run's.
 * Errors: QTT_ERR_INVALID_ARG (NULL arrays or vectors), QTT_ERR_CUDA. */
qtt_status qtt_batch_run_host(qtt_batch *B, const float *const *x_host,
                              float *const *y_host, void *stream);
/* Synchronise `stream`; QTT_ERR_TIMEOUT if a dependency wait in the last
 * runs gave up (the status word is then cleared). */
qtt_status qtt_batch_status(qtt_batch *B, void *stream);
/* qtt_batch_selftest_timeout -- exercises the batch kernel's bounded
 * dependency wait without a fault (no counterpart in the paper): launches the
 * batch's first wave alone, with its work list started past every item that
 * has no dependency, so that the items it runs wait on work that is never
 * done; each wait gives up after `seconds` (0 < seconds <= 10), the kernel
 * records QTT_ERR_TIMEOUT and every CTA returns.  The next qtt_batch_status
 * then returns QTT_ERR_TIMEOUT; the batch stays usable (each run resets its
 * counters).  QTT_ERR_UNSUPPORTED if no operator of the first wave has d > 1. */
qtt_status qtt_batch_selftest_timeout(qtt_batch *B, double seconds, void *stream);
/* Tile variant = pairs per lane (2 or 4: chunks of 64 or 128 position pairs,
 * wider for small ranks) + 100 x chunks per work item (1..64, default 8)
 * + 10000 x depth of the cp.async ring (2 or 3, default 3); re-plans and
 * re-captures. */
qtt_status qtt_batch_set_variant(qtt_batch *B, int variant, void *stream);
/* Time every variant (`reps` runs each, after one warm-up) and keep the
 * fastest; reports it and its seconds per run. */
qtt_status qtt_batch_autotune(qtt_batch *B, int reps, void *stream,
                              int *chosen, double *seconds_per_run);
qtt_status qtt_batch_info(const qtt_batch *B, int *waves, int *variant,
                          int *grid, double *flops, size_t *scratch_bytes);
/* Number of the batch's operators applied with the single-operator apply
 * instead of in a wave. */
qtt_status qtt_batch_direct_ops(const qtt_batch *B, int *count);
qtt_status qtt_batch_destroy(qtt_batch *B);

/* ---------------------------------------------------------- solve server */
/* A server serves qtt_solve and qtt_apply requests of any d and nrhs by
 * continuous batching (the paper has no serving layer; each request is one of
 * the solves or applies above).  Requests wait in a FIFO queue; the head is
 * admitted while fewer than `slots` requests are active and its device-memory
 * estimate fits in what is left of `mem_budget` (0 = 80 % of free memory).
 * One scheduler thread advances every active request by one step per tick:
 * its preconditioner work on its own stream, then ONE grouped launch per core
 * step for the forward applies of all active requests (launch L runs core
 * step L of every request with d > L), then its Gram-Schmidt and norms; one
 * synchronisation per tick, after which requests that finished leave and
 * queued ones join.  A request's arithmetic is that of qtt_solve /
 * qtt_apply on its own buffers, so its result is bitwise the same alone, in
 * any mix, and through those calls.
 *   prm       : solve parameters shared by all solve requests (kind, a, tol,
 *               restart, max_iter, precond_compute, inner_iters).
 * qtt_server_submit: a solve of (a I + K) x = f.  f_host / x_host are HOST
 *   arrays of nrhs x N doubles (contiguous), owned by the caller and
 *   untouched until the request is retired by qtt_server_poll; QTT_ERR_OOM if
 *   the request alone exceeds the budget.  *request_id receives its id.
 * qtt_server_submit_apply: y = A x for nrhs host vectors (x_host, y_host as
 *   above) with arithmetic `compute` (QTT_F64: grouped with the other
 *   requests' forward applies; reduced precisions need A's QTT_PACK_* copy
 *   and run on the request's stream); info reports iters = 1.
 * qtt_server_poll: done = 1 once finished (wait = 1 blocks until then); on
 *   completion fills info (nrhs entries) and the host timestamps (seconds,
 *   one steady clock) of submission, admission and completion, returns the
 *   request's status and retires the id.
 * qtt_server_ticks: ticks run and grouped launches issued so far.
 * qtt_server_destroy: finishes all submitted requests, then stops. */
typedef struct qtt_server qtt_server;
qtt_status qtt_server_create(qtt_server **out, int slots, size_t mem_budget,
                             const qtt_solve_params *prm);
qtt_status qtt_server_submit(qtt_server *S, const qtt_op *K, const qtt_op *P,
                             const double *f_host, double *x_host,
                             int64_t nrhs, int64_t *request_id);
qtt_status qtt_server_submit_apply(qtt_server *S, const qtt_op *A, const double *x_host,
                                   double *y_host, int64_t nrhs, qtt_dtype compute,
                                   int64_t *request_id);
qtt_status qtt_server_poll(qtt_server *S, int64_t request_id, int wait,
                           int *done, qtt_solve_info *info, double *t_submit,
                           double *t_admit, double *t_finish);
qtt_status qtt_server_stats(qtt_server *S, int *pending, int *running,
                            size_t *in_use, size_t *peak_in_use,
                            int *peak_running);
qtt_status qtt_server_ticks(qtt_server *S, uint64_t *ticks, uint64_t *grouped_launches);
qtt_status qtt_server_destroy(qtt_server *S);

/* ------------------------------------------------------------ diagnostics */
const char *qtt_status_string(qtt_status s);
/* Kernels launched by the library since it was loaded (all threads); for
 * counting the launches inside a timed region. */
uint64_t qtt_kernel_launches(void);
/* Message of the last failing call on this thread ("" if none). */
const char *qtt_last_error(void);
/* 1 in the checked build (libqtt_checked.so, compiled with -DQTT_CHECKED:
 * the kernels check their derived indices, clamp an out-of-range one to a
 * valid index and record where; qtt_sync_status then returns QTT_ERR_CHECK
 * once), 0 otherwise. */
int qtt_checked_build(void);
/* Checked build: launches a kernel that derives one index out of its range
 * on purpose (clamped, so nothing is accessed out of bounds); the next
 * qtt_sync_status returns QTT_ERR_CHECK.  QTT_ERR_UNSUPPORTED in the normal
 * build. */
qtt_status qtt_check_selftest(void *stream);
/* Synchronise `stream` and report device-side errors (QTT_ERR_CUDA for a
 * sticky CUDA error, QTT_ERR_TIMEOUT if a bounded wait in a library kernel
 * gave up).  The status word is cleared once reported. */
qtt_status qtt_sync_status(void *stream);

/* qtt_set_scratch_limit -- cap the scratch (the sweep's intermediates,
 * Krylov bases) that all applies and solves of the process hold at once, in
 * bytes; 0 removes the cap.  The paper has no counterpart: it bounds the
 * library's own memory beside a caller's other allocations.  Under the cap,
 * qtt_apply and the solves process right-hand sides in chunks (results are
 * bitwise the same) and return QTT_ERR_OOM when one right-hand side does not
 * fit. */
qtt_status qtt_set_scratch_limit(size_t bytes);
/* qtt_scratch_stats -- bytes of scratch handed out and not yet returned (all
 * devices), and the current device's pool: bytes reserved from the device
 * and bytes in use (scratch plus operator cores and batch tables).  Any
 * pointer may be NULL. */
qtt_status qtt_scratch_stats(size_t *in_use, size_t *pool_reserved, size_t *pool_used);

/* qtt_selftest_wait -- exercises the failure path of the library's device
 * waits without a fault (no counterpart in the paper): launches one kernel
 * whose bounded wait, on a barrier phase that nothing completes, runs out
 * after `seconds` (0 < seconds <= 10); the kernel records QTT_ERR_TIMEOUT in
 * the device status word and returns, so the next qtt_sync_status(stream)
 * returns QTT_ERR_TIMEOUT and the context stays usable. */
qtt_status qtt_selftest_wait(double seconds, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* QTT_H_ */
