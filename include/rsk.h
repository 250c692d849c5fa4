/*
 * rsk.h -- C ABI of the GB300 structured-sketch library (librsk.so).
 *
 * Method: "Faster Linear Algebra Algorithms with Structured Random Matrices" (arxiv 2508.21189).
 * Every entry point is extern "C", takes plain pointers and sizes, and returns rsk_status.
 *
 * Conventions shared by all calls
 *   - Matrices are row-major with an explicit leading dimension (elements between rows).
 *   - Pointers documented as "device" are device memory owned by the caller; the library never
 *     frees or retains them beyond the call.  "host" pointers are ordinary host memory.
 *   - Calls are asynchronous on the given stream unless documented as synchronous; results are
 *     valid once the stream has been synchronised.  Scratch memory comes from the handle, which
 *     owns a workspace that grows on demand (stream-ordered allocation on the call's stream).
 *     A handle must not be used from two host threads at once.
 *   - Invalid arguments are rejected with RSK_ERR_INVALID_ARG before anything is launched.
 *     CUDA errors map to RSK_ERR_CUDA.  rsk_last_error() returns a message for the last failure.
 *   - Kernels that detect a problem on the device (a bounded wait that ran out, an index out of
 *     range) record it in a device status word; rsk_sync_status() synchronises the stream and
 *     returns it (RSK_ERR_TIMEOUT / RSK_ERR_INTERNAL).
 *   - Determinism: identical inputs, seed, options and GPU model give bit-identical outputs.
 *
 * Randomness.  The paper asks for iid Rademacher signs and positions sampled uniformly without
 * replacement but fixes no generator.  All random draws come from the counter-based generator
 * Philox4x32-10 (Salmon et al., SC'11):
 *     word(seed, stream, entity, t) = Philox4x32-10(key = (seed_lo, seed_hi),
 *                                                   ctr = (entity_lo, entity_hi, stream, t >> 2))[t & 3]
 * Streams: 0 = sparse sign left sketch, 1 = SRTT diagonal D, 2 = SRTT subsample P,
 *          3 = RSVD test matrix Omega, 4 = SparseStack, 5 = SparseRTT's SparseCol positions.
 */
#ifndef RSK_H
#define RSK_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RSK_OK = 0,
    RSK_ERR_INVALID_ARG = 1,
    RSK_ERR_NOMEM = 2,
    RSK_ERR_CUDA = 3,
    RSK_ERR_NOT_CONVERGED = 4,
    RSK_ERR_TIMEOUT = 5,
    RSK_ERR_UNSUPPORTED = 6,
    RSK_ERR_INTERNAL = 7
} rsk_status;

/* RSK_F32X2 is the interleaved double-float form: each element is two FP32 values (hi, lo), 8
 * bytes, value hi + lo (about 48 significant bits).  Accepted as A by rsk_sparse_sign_apply
 * (double-float accumulation, FP64 or FP32 result) and as sketch or inner precision of the
 * single-problem least-squares solver; rsk_split_pairs produces it from FP64. */
typedef enum { RSK_F64 = 0, RSK_F32 = 1, RSK_BF16 = 2, RSK_F32X2 = 3 } rsk_dtype;

typedef struct rsk_handle rsk_handle;

/* Create a handle bound to the CUDA device current on the calling thread.  *out receives the
 * handle (host pointer owned by the library until rsk_destroy). */
rsk_status rsk_create(rsk_handle** out);
/* Release the handle and its workspace.  Synchronises the device first. */
rsk_status rsk_destroy(rsk_handle* h);
/* Message describing the last failure on this handle ("" if none).  Owned by the handle. */
const char* rsk_last_error(const rsk_handle* h);
/* Synchronise `stream` and return the device status word recorded by kernels of this handle
 * since the previous call (then clear it). */
rsk_status rsk_sync_status(rsk_handle* h, cudaStream_t stream);
/* Iteration limit of the bounded polls on global-memory flags that this handle's kernels make
 * (the persistent QR's grid barrier and reflector-ready flags): a poll that reaches it gives up,
 * records RSK_ERR_TIMEOUT in the device status word and the kernel returns, so a wait that can
 * never end (a CTA that is not resident, a flag nothing sets) cannot hang the GPU.  spins = 0
 * restores the default (about 4 million polls, seconds).  The mbarrier waits on TMA and bulk
 * copies keep the default.  Not a step of the paper: failure detection of the library. */
rsk_status rsk_set_wait_limit(rsk_handle* h, uint32_t spins);
/* Library version as major*10000 + minor*100 + patch. */
int32_t rsk_version(void);

/* Per-kernel timing.  While enabled, the handle records a CUDA event pair on the launch stream
 * around every kernel launch it makes, tagged with one of these ids. */
typedef enum {
    RSK_KERNEL_SKETCH_INDEX = 0,   /* k_index: draw S + chunked inverted index      */
    RSK_KERNEL_SKETCH_APPLY = 1,   /* k_apply: gather S*A into per-range partials   */
    RSK_KERNEL_SKETCH_REDUCE = 2,  /* k_reduce: ordered sum of partials, scale      */
    RSK_KERNEL_SKETCH_GENERATE = 3,/* k_generate: rows/signs of S                   */
    RSK_KERNEL_SRTT_APPLY = 4,
    RSK_KERNEL_SRTT_REDUCE = 5,
    RSK_KERNEL_DENSE = 6,          /* LSQ / RSVD dense helpers (QR, solves, matvecs) */
    RSK_KERNEL_GEMM = 7,           /* BF16 tensor-core GEMMs of the RSVD             */
    RSK_KERNEL_FACTOR = 8,         /* small Cholesky factorisations and R^{-1}       */
    RSK_KERNEL_SMALL_SVD = 9,      /* one-sided Jacobi SVD of a small matrix         */
    RSK_KERNEL_CONVERT = 10,       /* BF16 conversions and three-term splits         */
    RSK_KERNEL_GEMM_SPLIT = 11,    /* FP32-accurate products from split operands     */
    RSK_KERNEL_BATCH_SKETCH = 12,  /* batched solver phase: all problems' sketches   */
    RSK_KERNEL_BATCH_QR = 13,      /* batched solver phase: QR, R^{-1}, warm start   */
    RSK_KERNEL_BATCH_RESID = 14,   /* batched solver phase: residual passes + eta    */
    RSK_KERNEL_BATCH_CG = 15,      /* batched solver phase: CG graph replays         */
    RSK_KERNEL_COUNT = 16
} rsk_kernel_id;
/* Turn recording on (on != 0) or off.  Turning it on clears earlier records. */
rsk_status rsk_profile_enable(rsk_handle* h, int32_t on);
/* Synchronise on the recorded events and return, for kernel id `kernel`, the summed device time
 * in milliseconds and the number of launches recorded (host outputs). */
rsk_status rsk_profile_read(rsk_handle* h, int32_t kernel, double* total_ms, int64_t* launches);

/* ---------------------------------------------------------------------------------------------
 * Sparse sign embedding S (d x n), the left form of SparseUniform.
 * Paper: Def. "SparseUniform" (Sec. 3.2.1): exactly zeta entries zeta^{-1/2}*rho per row of the
 * right test matrix Omega (= per column of S = Omega^T), positions uniform without replacement,
 * rho Rademacher.  Sampling rule (both the library and its test oracle): Floyd's algorithm over
 * column j with draws w_q = word(seed, 0, j, q):  m = d - zeta + q, t = floor(w_q (m+1) / 2^32),
 * row_q = (t already chosen) ? m : t;  sign of row_q is -1 iff bit q of w_zeta is set.
 * Limits: 1 <= zeta <= min(d, 32), 1 <= d <= 8192, 1 <= n < 2^31.
 * ------------------------------------------------------------------------------------------- */

/* a1: draw S.  rows: device int32[n*zeta], rows[j*zeta + q] = q-th row chosen for column j (in
 * Floyd insertion order).  sign_bits: device uint32[n], bit q set <=> entry (rows[j*zeta+q], j)
 * is -zeta^{-1/2}.  Either output may be NULL to skip it. */
rsk_status rsk_sparse_sign_generate(rsk_handle* h, int64_t n, int64_t d, int32_t zeta, uint64_t seed,
                                    int32_t* rows, uint32_t* sign_bits, cudaStream_t stream);

/* Shape of the inverted index built by rsk_sparse_sign_index for (n, d, zeta): S's columns are
 * grouped in chunks of *chunk_rows consecutive columns (768 for zeta <= 8; the last chunk may be
 * shorter), *n_chunks chunks, and each chunk's offsets row has *offsets_pitch >= d + 1 entries.
 * Host outputs. */
rsk_status rsk_sparse_sign_index_dims(int64_t n, int64_t d, int32_t zeta, int64_t* chunk_rows,
                                      int64_t* n_chunks, int64_t* offsets_pitch);

/* a2: the inverted index of S, chunked.  For chunk c (columns j in [c*C, min((c+1)*C, n)),
 * C = chunk_rows, P = offsets_pitch) the entries of sketch row i are
 *     entries[c*C*zeta + offsets[c*P + i] ... c*C*zeta + offsets[c*P + i + 1] - 1],
 * each a uint16 (j - c*C) | (negative << 15), in ascending j; offsets[c*P + d .. c*P + P - 1]
 * hold the chunk's entry count.  Concatenating chunks in order gives the CSR of S with columns
 * ascending in every row.  offsets: device uint16[n_chunks*P]; entries: device uint16[n*zeta],
 * 16-byte aligned. */
rsk_status rsk_sparse_sign_index(rsk_handle* h, int64_t n, int64_t d, int32_t zeta, uint64_t seed,
                                 uint16_t* offsets, uint16_t* entries, cudaStream_t stream);

/* a3: SA = S * A.
 * A: device, n x k row-major, leading dimension lda >= k, element type a_dtype (F64, F32, BF16).
 * SA: device, d x k row-major, leading dimension ldsa >= k, element type sa_dtype (F64 or F32).
 * Accumulation is FP64 for F64 input and FP32 otherwise; the +-1 pattern is summed in a fixed
 * order (ascending j within a chunk, chunks in order, row blocks reduced in index order) and
 * scaled by zeta^{-1/2} once.  S is drawn from `seed` exactly as rsk_sparse_sign_generate. */
rsk_status rsk_sparse_sign_apply(rsk_handle* h, const void* A, rsk_dtype a_dtype, int64_t n, int64_t k,
                                 int64_t lda, int64_t d, int32_t zeta, uint64_t seed, void* SA,
                                 rsk_dtype sa_dtype, int64_t ldsa, cudaStream_t stream);

/* a3 on a block of rows of A, for a row-sharded A (one process per GPU): with S the d x N sparse
 * sign of `seed` (N the rows of the whole A), SA = S[:, row0 : row0 + n] * A_block, where A is the
 * n x k block holding rows row0 .. row0 + n - 1 of the whole A (device, row-major, lda >= k).  The
 * columns of S depend only on their global index, so the blocks of any row partition give partial
 * sketches whose sum is S * A_whole; SA is such a partial (scaled by zeta^{-1/2}).  Paper: the sketch
 * application cost O(zeta nnz(A)) (Sec. 3.2) is additive over row blocks.  rsk_sparse_sign_apply is
 * this call with row0 = 0.  Requires 0 <= row0 and row0 + n < 2^31; otherwise as rsk_sparse_sign_apply. */
rsk_status rsk_sparse_sign_apply_rows(rsk_handle* h, const void* A, rsk_dtype a_dtype, int64_t n, int64_t k,
                                      int64_t lda, int64_t row0, int64_t d, int32_t zeta, uint64_t seed, void* SA,
                                      rsk_dtype sa_dtype, int64_t ldsa, cudaStream_t stream);

/* out = parts[0] + parts[1] + ... + parts[count-1], summed in that order for every element (so the
 * result does not depend on how the partials were produced or gathered).  parts: device, count
 * packed d x k blocks (row-major, leading dimension k) of dtype F32 or F64, block g starting at
 * element g * part_stride (part_stride >= d*k).  out: device d x k, leading dimension ldo >= k, same
 * dtype.  The reduction step of a row-sharded sketch: each rank's partial from
 * rsk_sparse_sign_apply_rows or rsk_srtt_apply_rows, gathered in rank order, summed in rank order. */
rsk_status rsk_sketch_sum_partials(rsk_handle* h, const void* parts, rsk_dtype dtype, int32_t count,
                                   int64_t part_stride, int64_t d, int64_t k, void* out, int64_t ldo,
                                   cudaStream_t stream);

/* a3 with A in HOST memory (pinned for the copies to overlap; pageable works, serialised): the
 * same SA = S * A as rsk_sparse_sign_apply, computed while A streams to the device.  A is cut into
 * row blocks of whole index chunks (about 256 MB each); block b is copied on an internal stream into
 * one of two device staging buffers while block b-1 is sketched on `stream`; SA is the sum of the
 * block sketches in block order (deterministic; it can differ from rsk_sparse_sign_apply in the
 * last bits because the partial sums are grouped by block).  SA is a device array.  Asynchronous
 * with respect to the host: A_host must stay valid until `stream` has passed this call.  Not a step
 * of the paper: the end-to-end form of a3 when A lives on the host. */
rsk_status rsk_sparse_sign_apply_host(rsk_handle* h, const void* A_host, rsk_dtype a_dtype, int64_t n, int64_t k,
                                      int64_t lda, int64_t d, int32_t zeta, uint64_t seed, void* SA,
                                      rsk_dtype sa_dtype, int64_t ldsa, cudaStream_t stream);

/* The same SA = S * A for callers that cannot allocate device memory (code where cudaMalloc is
 * unavailable or forbidden, e.g. inside a host application that owns every device buffer, or a
 * path that must not allocate after start-up).  The paper has no counterpart: this is a deployment
 * variant of rsk_sparse_sign_apply with the same arguments minus the handle, and bit-identical
 * results.  Scratch comes from one fixed 64 MiB array in device memory that every GPU loading the
 * library holds until exit; no call allocates or frees anything.  Invalid arguments return
 * RSK_ERR_INVALID_ARG before anything else; valid sizes whose scratch (inverted index plus partial
 * sums) exceeds 64 MiB return RSK_ERR_UNSUPPORTED before any launch.  The first call on each device
 * looks up the array's device address (make it before any stream capture).  All calls share the
 * array: calls that overlap on the GPU race, and the set-up is not thread safe.  The return code
 * carries the errors found on the host (no handle, no message); a failure found on the device
 * while the call runs (a bounded wait that ran out, a failed bounds check) cannot be returned by
 * an asynchronous call, so the call's last kernel then fills SA with NaN. */
rsk_status rsk_sparse_sign_apply_noalloc(const void* A, rsk_dtype a_dtype, int64_t n, int64_t k, int64_t lda,
                                         int64_t d, int32_t zeta, uint64_t seed, void* SA, rsk_dtype sa_dtype,
                                         int64_t ldsa, cudaStream_t stream);

/* ---------------------------------------------------------------------------------------------
 * SparseStack (Def. SparseStack, Sec. 1.5): zeta stacked CountSketches.  With b = d / zeta, every
 * column j of S (d x n) has exactly one entry +-zeta^{-1/2} in each block of b consecutive rows:
 * row q*b + floor(w_q * b / 2^32) of block q, w_q = word(seed, 4, j, q) (Philox stream 4); its sign
 * is -1 iff bit q of w_zeta is set.  Limits as SparseUniform plus d % zeta == 0
 * (RSK_ERR_INVALID_ARG otherwise).  The inverted index and gather are those of
 * rsk_sparse_sign_apply: only the column draw differs.
 * ------------------------------------------------------------------------------------------- */
/* Draw S: rows device int32[n*zeta] (entry q of column j in block q), sign_bits device uint32[n]. */
rsk_status rsk_sparse_stack_generate(rsk_handle* h, int64_t n, int64_t d, int32_t zeta, uint64_t seed,
                                     int32_t* rows, uint32_t* sign_bits, cudaStream_t stream);
/* SA = S * A with the conventions, accumulation and summation order of rsk_sparse_sign_apply. */
rsk_status rsk_sparse_stack_apply(rsk_handle* h, const void* A, rsk_dtype a_dtype, int64_t n, int64_t k,
                                  int64_t lda, int64_t d, int32_t zeta, uint64_t seed, void* SA,
                                  rsk_dtype sa_dtype, int64_t ldsa, cudaStream_t stream);

/* Right sketch Y = A Omega with Omega = S^T (Sec. 2: the test matrices of Algs. 1, 2, 4, 5 multiply A
 * from the right), S the k x dc sparse sign of the given kind (0 SparseUniform, 1 SparseStack with
 * k % zeta == 0) drawn from `seed` on Philox stream `philox_stream` (-1: the kind's own stream, 0 or 4;
 * the RSVD test matrix is stream 3).  A device FP32 n x dc row-major (lda >= dc); Y device FP32 n x k
 * column-major (ldy >= n): Y[i, c] = zeta^{-1/2} sum over the entries (j, sign) of row c of S of
 * sign * A[i, j], summed in increasing j (deterministic).  Limits: k <= 512, 1 <= zeta <= min(k, 32).
 * The inverted index of S comes from the handle's workspace.  Asynchronous. */
rsk_status rsk_sparse_sign_apply_right(rsk_handle* h, int32_t kind, const float* A, int64_t n, int64_t dc,
                                       int64_t lda, int64_t k, int32_t zeta, uint64_t seed, int32_t philox_stream,
                                       float* Y, int64_t ldy, cudaStream_t stream);

/* Plans keep the inverted index of one S for repeated application (e.g. to A and then to b).
 * The plan owns device memory allocated on `stream`; destroy it with rsk_sparse_sign_plan_destroy. */
typedef struct rsk_sketch_plan rsk_sketch_plan;
rsk_status rsk_sparse_sign_plan_create(rsk_handle* h, int64_t n, int64_t d, int32_t zeta, uint64_t seed,
                                       rsk_sketch_plan** plan, cudaStream_t stream);
rsk_status rsk_sparse_sign_plan_apply(rsk_handle* h, const rsk_sketch_plan* plan, const void* A,
                                      rsk_dtype a_dtype, int64_t k, int64_t lda, void* SA,
                                      rsk_dtype sa_dtype, int64_t ldsa, cudaStream_t stream);
rsk_status rsk_sparse_sign_plan_destroy(rsk_handle* h, rsk_sketch_plan* plan, cudaStream_t stream);

/* ---------------------------------------------------------------------------------------------
 * Subsampled randomized trigonometric transform with the Walsh-Hadamard transform (SRTT).
 * Paper: Omega = D F S (Sec. 1.6, Eq. "intro-srtt"): D iid Rademacher diagonal, F the unitary
 * WHT, S a restriction to d coordinates drawn uniformly without replacement, rescaled so Omega is
 * isotropic; cost steps 1-3 and their subsampled variant (Sec. 4.x "Arithmetic costs").  As a left
 * sketch of a tall A:  Y = sqrt(n/d) P (H_n / sqrt(n)) D A = d^{-1/2} P H_n D A, with
 * H_n[i, l] = (-1)^{popcount(i & l)} (Sylvester order).
 * D_i = -1 iff bit (i & 31) of word(seed, 1, i >> 7, (i >> 5) & 3) is set.  P = Floyd's algorithm
 * over [0, n) with draws word(seed, 2, 0, q); output row q is the q-th inserted coordinate.
 * Limits: n = 2^m < 2^31, k >= 1; 1 <= d <= min(n, 8192) for rsk_srtt_draw and
 * 1 <= d <= min(n, 2048) for rsk_srtt_apply (RSK_ERR_UNSUPPORTED beyond).
 * ------------------------------------------------------------------------------------------- */

/* Random ingredients of the SRTT.  rows: device int64[d] (P in draw order), dbits: device
 * uint32[ceil(n/32)] (bit j of word w set <=> D_{32w+j} = -1).  Either may be NULL. */
rsk_status rsk_srtt_draw(rsk_handle* h, int64_t n, int64_t d, uint64_t seed, int64_t* rows, uint32_t* dbits,
                         cudaStream_t stream);

/* a4: Y = d^{-1/2} P H_n D A.  A: device n x k row-major (lda >= k), F32 or BF16 (TMA staging when
 * the base address and row pitch are 16-byte aligned, plain loads otherwise).  Y: device d x k
 * row-major (ldy >= k), F32 or F64.  FP32 arithmetic; partial sums over 2048-row blocks are
 * reduced in a fixed order (deterministic). */
rsk_status rsk_srtt_apply(rsk_handle* h, const void* A, rsk_dtype a_dtype, int64_t n, int64_t k, int64_t lda,
                          int64_t d, uint64_t seed, void* Y, rsk_dtype y_dtype, int64_t ldy, cudaStream_t stream);

/* a4 on a block of rows of A (row-sharded A): Y = d^{-1/2} P H_N[:, row0 : row0 + n_rows] D_block A_block
 * for the SRTT of an N-row A (N = 2^m; P and D drawn for N exactly as rsk_srtt_apply), with A_block
 * the n_rows x k block holding rows row0 .. row0 + n_rows - 1.  Because H_N = H_{N/2048} (x) H_2048,
 * a block that starts on a 2048-row boundary contributes sum_b (-1)^{popcount(p_hi & b)} (H_2048 x_b)
 * over its own 2048-row blocks b only, so the partials of any such partition sum to the whole Y.
 * Requires row0 % 2048 == 0 and row0 + n_rows <= N; otherwise as rsk_srtt_apply, which is this call
 * with row0 = 0 and n_rows = N. */
rsk_status rsk_srtt_apply_rows(rsk_handle* h, const void* A, rsk_dtype a_dtype, int64_t n_rows, int64_t k,
                               int64_t lda, int64_t row0, int64_t n, int64_t d, uint64_t seed, void* Y,
                               rsk_dtype y_dtype, int64_t ldy, cudaStream_t stream);

/* ---------------------------------------------------------------------------------------------
 * SparseRTT (Def. SparseRTT with Def. SparseCol, Sec. 4): Omega = D F S with D the Rademacher
 * diagonal of the SRTT, F the unitary WHT (Sylvester order), S a SparseCol matrix whose columns
 * are iid copies of sqrt(n/xi) sum_{t<xi} rho_t e_{s_t} scaled by d^{-1/2}, the xi positions s_t of
 * a column distinct and uniform on [0, n).  As a left sketch of a tall A:
 *     Y[q, :] = (d xi)^{-1/2} sum_{t < xi} rho_{qt} (H_n D A)[s_{qt}, :].
 * Draw rule: column q's positions are Floyd's algorithm over [0, n) with draws
 * w_t = word(seed, 5, q, t), t < xi (Philox stream 5); rho_{qt} = -1 iff bit t of w_xi is set.
 * D_i is the SRTT's (stream 1).  xi = 0 selects the recommended ceil(1.5 ln d) (Sec. 4,
 * "Implementation guidance").  Limits: n = 2^m < 2^31, 1 <= d <= 2048, 1 <= xi <= min(n, 32).
 * ------------------------------------------------------------------------------------------- */
/* The recommended column sparsity ceil(1.5 ln d), clamped to [1, 32]. */
int32_t rsk_sparse_rtt_default_xi(int64_t d);
/* The SparseCol positions: positions device int32[d*xi] (positions[q*xi + t] = s_qt, Floyd
 * insertion order), sign_bits device uint32[d] (bit t set <=> rho_qt = -1).  Either may be NULL. */
rsk_status rsk_sparse_rtt_draw(rsk_handle* h, int64_t n, int64_t d, int32_t xi, uint64_t seed, int32_t* positions,
                               uint32_t* sign_bits, cudaStream_t stream);
/* Y = Omega^T A for A device n x k (F32 or BF16, lda >= k); Y device d x k (F32 or F64, ldy >= k).
 * One pass over A: each 2048-row block is transformed on chip as in rsk_srtt_apply and every output
 * row adds its xi signed transformed rows; FP32 arithmetic, partials summed in a fixed order. */
rsk_status rsk_sparse_rtt_apply(rsk_handle* h, const void* A, rsk_dtype a_dtype, int64_t n, int64_t k, int64_t lda,
                                int64_t d, int32_t xi, uint64_t seed, void* Y, rsk_dtype y_dtype, int64_t ldy,
                                cudaStream_t stream);

/* Split an FP64 matrix (n x k, row-major, lda >= k) into the interleaved F32X2 form P (n x k pairs,
 * packed: 2 k floats per row): hi = FP32 round-to-nearest-even of a, lo = FP32 round-to-nearest-
 * even of a - hi, computed with integer operations.  Values outside the FP32 normal range are
 * flushed (|a| < 2^-126 -> (+-0, 0); |a| > FLT_MAX -> +-inf; lo < 2^-126 -> 0).  Not a step of the
 * paper: the storage form of the double-float solvers.  Device pointers; asynchronous. */
rsk_status rsk_split_pairs(rsk_handle* h, const double* A, int64_t n, int64_t k, int64_t lda, float* P,
                           cudaStream_t stream);

/* ---------------------------------------------------------------------------------------------
 * Sketch-and-precondition least squares, min_x ||A x - b||_2 (rows a5-a7).
 * Paper: sketch-and-solve (Alg. 3, Sec. 2.3) for the warm start; sketch-and-precondition is named
 * as the standard high-accuracy method (remark closing Sec. 2.3) but not spelled out.  Steps:
 *   [Ahat | bhat] = S [A | b] (sparse sign, d rows, zeta per column, seed);
 *   Householder QR of Ahat in FP64 -> R and Q^T bhat;  x0 = R^{-1} Q^T bhat;
 *   refinement: g = A^T (b - A x) in FP64; eta = min(||g|| / (||A||_F ||r||),
 *   ||r|| / (||A||_F ||x|| + ||b||)) (LSQR's stopping quantities for least-squares and consistent
 *   problems); stop at eta <= tol_backward; else CG on (M^T M) z = R^{-T} g with M = A R^{-1} in
 *   inner_dtype, then x += R^{-1} z.
 * Precision notes: inner_dtype F32 converges when u_32 * kappa(A) is well below 1 or when A's
 * ill-conditioning is a column scaling; for kappa(A) ~ 1e8 with mixed columns use F64 or F32X2.
 * F32X2 (sketch or inner): A is split once per solve into interleaved (hi, lo) pairs; the sketch
 * then accumulates in double-float arithmetic and the CG operator runs in double-float arithmetic,
 * both on FP32 units.  The residual passes read an F64 A as stored (48 bits of hi + lo would move
 * the fixed point) and an F32 A (exact as (a, 0)) through the double-float pass.
 * ------------------------------------------------------------------------------------------- */
typedef struct {
    int64_t d;               /* sketch rows (k <= d <= 8192) */
    int32_t zeta;            /* nonzeros per column of S */
    uint64_t seed;           /* Philox seed of S */
    rsk_dtype sketch_dtype;  /* precision A is sketched in: F64, F32 or BF16 (FP32 accumulation),
                                F32X2 (double-float accumulation of the split pairs) */
    rsk_dtype inner_dtype;   /* precision of the CG operator: F64, F32, or F32X2 (double-float pair) */
    double tol_backward;     /* target eta (default 1e-10 when <= 0) */
    int32_t max_refine;      /* refinement steps; 0 returns the warm start x0; < 0 selects 20 */
    int32_t max_inner_iters; /* CG iterations per step (default 50 when <= 0) */
    double inner_tol;        /* relative CG residual reduction per step (default 1e-6 when <= 0) */
    rsk_dtype qr_dtype;      /* precision of the batched solver's Householder QR of the sketch: F64 (the
                                default, 0) or F32; the single solve always factors in FP64 */
} rsk_lsq_opts;

typedef struct {
    double backward_err;     /* eta(x) at exit */
    double residual_norm;    /* ||b - A x||_2 */
    double frobenius_norm;   /* ||A||_F */
    int32_t refine_steps;    /* refinement steps taken */
    int32_t inner_iters;     /* total CG iterations */
    rsk_status status;       /* RSK_OK or RSK_ERR_NOT_CONVERGED */
} rsk_lsq_info;

/* A: device n x k row-major (lda >= k), F64 or F32; 1 <= k <= 1024, n >= k.  b: device FP64[n].
 * x: device FP64[k] (output).  info: host (may be NULL).  Synchronous: returns after the solve
 * (the refinement loop reads eta on the host).  Returns RSK_ERR_NOT_CONVERGED, with x the last
 * iterate and info filled, if eta stays above tol_backward after max_refine steps. */
rsk_status rsk_lstsq_sketch_precond(rsk_handle* h, const void* A, rsk_dtype a_dtype, int64_t n, int64_t k,
                                    int64_t lda, const double* b, double* x, const rsk_lsq_opts* opts,
                                    rsk_lsq_info* info, cudaStream_t stream);

/* One problem of a batch (row a8): A device n x k row-major (lda >= k), F64 or F32, k <= 256;
 * b device FP64[n]; x device FP64[k] (output); d sketch rows (0 selects 4k). */
typedef struct {
    const void* A;
    rsk_dtype a_dtype;
    int64_t n, k, lda, d;
    const double* b;
    double* x;
} rsk_lsq_problem;

/* a8: solve `count` independent problems together.  Problem i is sketched with seed opts->seed + i
 * (opts->d is ignored; each problem carries its own d) and refined exactly as in
 * rsk_lstsq_sketch_precond; opts->sketch_dtype must be F64 or F32.  The fused passes of all
 * problems run in one persistent launch over (problem, 2048-row block) tiles taken from a work
 * queue; per-problem results are reduced in tile order (deterministic).  One CG iteration is a
 * captured CUDA graph.  The Householder QR of [S A_i | S b_i] runs in FP64, or in FP32 when
 * opts->qr_dtype is F32 (R_i and Q_i^T S b_i are then used in FP64).  With inner_dtype F32 and FP32
 * storage, the FP64-accuracy residual passes use double-float (FP32 pair) arithmetic.
 * probs and infos are host arrays of `count` entries;
 * synchronous; RSK_ERR_NOT_CONVERGED if any problem stays above tol_backward (infos[i].status says
 * which). */
rsk_status rsk_lstsq_sketch_precond_batched(rsk_handle* h, int32_t count, const rsk_lsq_problem* probs,
                                            const rsk_lsq_opts* opts, rsk_lsq_info* infos, cudaStream_t stream);

/* ---------------------------------------------------------------------------------------------
 * Autotuning of launch parameters (not a step of the paper).  Knobs (kernel ids): 0 = the number of
 * row ranges of the sparse gather apply (sparse sign, SparseStack, the solvers' sketches), 1 = the
 * number of row bands of the SRTT / SparseRTT, 2 = the rows per work tile of the batched
 * least-squares passes.  Tuned values live in a process-wide table keyed by (kernel, dtype, n, k, d,
 * SM count) -- for kernel 2: (inner dtype, total rows, problem count, 0, SM count) -- and are used
 * by every later call with that key; a tuned value regroups partial sums, so results are
 * deterministic for a fixed table but may differ in the last bits from untuned ones.  If the
 * environment variable RSK_TUNE_CACHE names a file, the table is read from it at the first lookup
 * and written back after every autotune call.  File format: text lines
 *     rsk-tune v1 kernel=<int> dtype=<int> n=<int> k=<int> d=<int> sms=<int> value=<int>
 * ('#' starts a comment line; later lines override earlier ones).  The table calls are host-only
 * and thread safe. */
rsk_status rsk_tune_cache_load(const char* path);      /* merge a cache file into the table */
rsk_status rsk_tune_cache_save(const char* path);      /* write the whole table */
rsk_status rsk_tune_cache_clear(void);                 /* empty the table (and skip RSK_TUNE_CACHE) */
rsk_status rsk_tune_cache_set(int32_t kernel, int32_t dtype, int64_t n, int64_t k, int64_t d, int32_t sms,
                              int32_t value);
/* *value = the tuned value for the key, 0 when none. */
rsk_status rsk_tune_cache_get(int32_t kernel, int32_t dtype, int64_t n, int64_t k, int64_t d, int32_t sms,
                              int32_t* value);
/* Time the default rule and candidate values around it for kernel 0 (rsk_sparse_sign_apply) or 1
 * (rsk_srtt_apply) on an n x k matrix of a_dtype with d sketch rows (zeta for kernel 0), keep the
 * fastest in the table (0 = the default rule won; the key is then left untuned).  Allocates its
 * buffers on `stream`; synchronous.  *chosen and *best_ms (may be NULL) are host outputs. */
rsk_status rsk_autotune_sketch(rsk_handle* h, int32_t kernel, rsk_dtype a_dtype, int64_t n, int64_t k, int64_t d,
                               int32_t zeta, int32_t* chosen, double* best_ms, cudaStream_t stream);
/* Time the batched least-squares solver on the caller's problems with 1024, 2048, 4096 and 8192 rows
 * per work tile (and the default), keep the fastest for this batch's key.  Synchronous; the
 * problems' x are overwritten by the solves. */
rsk_status rsk_autotune_batched(rsk_handle* h, int32_t count, const rsk_lsq_problem* probs, const rsk_lsq_opts* opts,
                                int32_t* chosen, double* best_ms, cudaStream_t stream);

/* ---------------------------------------------------------------------------------------------
 * Dense steps of the low-rank algorithms (Algs. 1, 2, 4, 5 name them svd_econ, qr_econ / orth,
 * chol): FP32, column-major (column c of X at X + c * ldx), device pointers, asynchronous.
 * ------------------------------------------------------------------------------------------- */
/* Thin SVD A = U diag(s) V^T of A (m x q, m >= q) by one-sided block Jacobi (Hestenes): plane
 * rotations of column pairs until no pair has |a_i . a_j| > 2 sqrt(m) u_32 ||a_i|| ||a_j|| (at most 40
 * sweeps).  U m x q (ldu >= m), s[q] descending, V q x q (ldv >= q; may be NULL).  A is not
 * modified.  Limits: q <= 1024, m <= 4096 (RSK_ERR_UNSUPPORTED beyond). */
rsk_status rsk_svd_econ(rsk_handle* h, const float* A, int64_t m, int64_t q, int64_t lda, float* U, int64_t ldu,
                        float* s, float* V, int64_t ldv, cudaStream_t stream);
/* Thin QR X = Q R of X (m x q, m >= q) by shifted Cholesky QR3 (one round of Cholesky QR on X^T X +
 * s I with s = 11 (m q + q (q + 1)) u_32 ||X||_F^2, then two plain rounds): Q m x q (ldq >= m) with
 * orthonormal columns, R q x q upper triangular (leading dimension q; may be NULL).  Limits: q <= 330.
 * A Cholesky pivot that is not positive is recorded in the device status word (rsk_sync_status). */
rsk_status rsk_qr_econ(rsk_handle* h, const float* X, int64_t m, int64_t q, int64_t ldx, float* Q, int64_t ldq,
                       float* R, cudaStream_t stream);
/* Upper Cholesky factor (Alg. 2's chol): R^T R = sym(G) + s I with s = shift_coeff * trace(G), G
 * read from its upper triangle, R q x q upper triangular with zeros below the diagonal.  Blocked
 * right-looking factorisation in one CTA (q <= 330, RSK_ERR_UNSUPPORTED beyond).  A pivot that is not
 * positive is recorded in the device status word (rsk_sync_status) and R is then undefined. */
rsk_status rsk_cholesky(rsk_handle* h, const float* G, int64_t q, int64_t ldg, float shift_coeff, float* R,
                        int64_t ldr, cudaStream_t stream);
/* Ri = R^{-1} for an upper triangular R (q x q, ldr; Ri has leading dimension ldr, zeros below the
 * diagonal; Ri must not overlap R): blocked over 32 x 32 blocks, the diagonal blocks inverted by back
 * substitution, then each block column by block back substitution.  q <= 880 (RSK_ERR_UNSUPPORTED
 * beyond). */
rsk_status rsk_trinv(rsk_handle* h, const float* R, int64_t q, int64_t ldr, float* Ri, cudaStream_t stream);

/* ---------------------------------------------------------------------------------------------
 * Randomized Nystrom approximation of a psd matrix (Alg. 2, Sec. 2.2) with a structured test matrix:
 * Y = A Omega; nu = sqrt(n) eps ||Y||; Y_nu = Y + nu Omega; C = chol(Omega^T Y_nu);
 * B = Y_nu C^{-1}; [U, Sigma, ~] = svd(B); Lambda = max(0, Sigma^2 - nu I), truncated to `rank`.
 * Omega = S^T with S the k x n SparseStack (kind = 1, needs k % zeta == 0) or SparseUniform
 * (kind = 0) sketch of this library (zeta nonzeros per row of Omega, drawn from `seed` exactly as
 * rsk_sparse_stack_generate / rsk_sparse_sign_generate).  Readings: eps = 2^-24 (FP32 arithmetic)
 * and ||Y|| the Frobenius norm (never smaller than the spectral norm).
 * A: device FP32 n x n, symmetric positive semidefinite, row-major (lda >= n); only S A is formed,
 * which the symmetry makes equal to Y^T (one pass over A).  U: device FP32 n x rank column-major
 * (ldu >= n), orthonormal columns.  lambda: device FP32[rank], descending.  A ~ U diag(lambda) U^T.
 * Limits: 1 <= rank <= k <= min(n, 330).  A failed Cholesky (A not psd) is recorded in the device
 * status word (rsk_sync_status returns RSK_ERR_INTERNAL).  Asynchronous; allocates its buffers
 * stream-ordered on `stream`. */
rsk_status rsk_nystrom_psd(rsk_handle* h, const float* A, int64_t n, int64_t lda, int32_t k, int32_t rank, int32_t zeta,
                           uint64_t seed, int32_t kind, float* U, int64_t ldu, float* lambda, cudaStream_t stream);

/* ---------------------------------------------------------------------------------------------
 * Generalized Nystrom approximation of a general A (Algs. 4 and 5, Sec. 2.4) with structured test
 * matrices Omega (d x k) and Psi (n x p), k <= p (the paper recommends p = ceil(1.5 k)):
 * Y = A Omega and X = A^T Psi, one pass over A each (the right and the left sparse sketch).
 *   form 0 (Alg. 4, outer-product form): [U, Sigma, V] = svd(X^T Omega); r = #{sigma_i > 5 eps sigma_1};
 *          F = Y V_r Sigma_r^{-1} (out1, n x k), G = X U_r (out2, d x k); A ~ F G^T (columns >= r zero).
 *   form 1 (Alg. 5, SVD form): Q = qr(Y), [P, T] = qr(X), [U1, S1, V1] = svd(Psi^T Q),
 *          C = V1_r S1_r^{-1} U1_r^T T^T, [Uh, Sigma, Vh] = svd(C); U = Q Uh (out1, n x k),
 *          sigma (k, descending), V = P Vh (out2, d x k); A ~ U diag(sigma) V^T.
 * Omega = S^T for the k x d sketch S of `seed`, Psi = S'^T for the p x n sketch S' of seed + 1, both of
 * the given kind (0 SparseUniform, 1 SparseStack: k and p multiples of zeta).  eps = 2^-24.
 * A: device FP32 n x d row-major (lda >= d).  out1, out2: device FP32 column-major (ld1 >= n,
 * ld2 >= d).  rank: device int32, the numerical rank r.  The thin QRs are Cholesky QR2 with the Gram
 * accumulated in FP64 (Y and X must have full numerical rank, kappa up to ~1e7).  Limits:
 * 1 <= k <= p <= min(n, d), k <= 512, p <= 1024.  Asynchronous; allocates stream-ordered. */
rsk_status rsk_gen_nystrom(rsk_handle* h, const float* A, int64_t n, int64_t d, int64_t lda, int32_t k, int32_t p,
                           int32_t zeta, uint64_t seed, int32_t kind, int32_t form, float* out1, int64_t ld1,
                           float* sigma, float* out2, int64_t ld2, int32_t* rank, cudaStream_t stream);

/* ---------------------------------------------------------------------------------------------
 * Injectivity and dilation on the adversarial subspace (Fig. 2, Sec. 1.5; discussed in Sec. 3):
 * for Q = [e_1 ... e_r] and embedding dimension k, alpha = sigma_min^2(Omega^T Q) and
 * beta = sigma_max^2(Omega^T Q), Omega^T Q being the first r columns S_r of the k x d sketch of the
 * given kind (0 SparseUniform, 1 SparseStack with k % zeta == 0) drawn from `seed`.  Estimated by
 * `iters` Lanczos steps on S_r^T S_r from v_1 = (1, ..., 1) / sqrt(r) (FP64 vectors, products with a
 * deterministic CSR of S_r and with its columns as drawn), then bisection on the Lanczos tridiagonal:
 * *alpha is the smallest Ritz value (>= the true alpha), *beta the largest (<= the true beta); with
 * iters >= r they are the eigenvalues to rounding.  Host outputs; synchronous.  Limits: r, k < 2^31,
 * r * zeta < 2^31, 1 <= zeta <= min(k, 32), 1 <= iters <= 100000.  Device memory: about
 * r (8 zeta + 28) + 28 k bytes from the handle's workspace. */
rsk_status rsk_osi_estimate(rsk_handle* h, int64_t r, int64_t k, int32_t zeta, uint64_t seed, int32_t kind,
                            int32_t iters, double* alpha, double* beta, cudaStream_t stream);

/* D = A B^T on the BF16 tensor cores (tcgen05, FP32 accumulation in tensor memory): A device BF16
 * M x K row-major (lda >= K), B device BF16 N x K row-major (ldb >= K) -- both K-major --, D device
 * FP32 M x N column-major (ldd >= M).  The dense product step of Alg. 1 (Z = A^T Q, Y = A Z) with the
 * rank as N.  1 <= N <= 512 (N rounded up to an even multiple of 16 internally: 2 x 16 .. 2 x 256);
 * A, B 16-byte aligned with 16-byte row pitches.  nsplit > 1 splits K that many ways for every
 * 128-row tile (the partials come from the handle's workspace and are summed in split order); nsplit
 * 0 chooses: K splits that keep the SMs busiest, and without a split a last round of row tiles that
 * would leave more than half the SMs idle is split over K instead (those rows summed from partials).
 * The kernel is persistent: one CTA per SM, the row tiles dealt round-robin.  Asynchronous. */
rsk_status rsk_gemm_bf16(rsk_handle* h, const void* A, int64_t M, int64_t K, int64_t lda, const void* B, int64_t N,
                         int64_t ldb, float* D, int64_t ldd, int32_t nsplit, cudaStream_t stream);
/* The same product with the operand and output layouts of the RSVD's steps: a_mn != 0 takes A
 * MN-major, i.e. element (m, k) at A[k * lda + m] (lda >= M: A^T of a row-major K x M matrix, so that
 * Z = A^T Q reads A in place); d_row_major != 0 stores D row-major (element (m, n) at D[m * ldd + n],
 * ldd >= N) instead of column-major.  cluster = 1, 2 or 4 row tiles per thread-block cluster share the
 * B tile (each CTA loads its part and multicasts it: B's traffic from L2 falls by that factor; 4 only
 * when N rounds to 256, 320 or 512 columns), 0 takes 2 with at least 8 row tiles, else 1.  Alignment,
 * limits and nsplit as rsk_gemm_bf16. */
rsk_status rsk_gemm_bf16_ex(rsk_handle* h, int32_t a_mn, const void* A, int64_t M, int64_t K, int64_t lda,
                            const void* B, int64_t N, int64_t ldb, float* D, int64_t ldd, int32_t d_row_major,
                            int32_t nsplit, int32_t cluster, cudaStream_t stream);
/* D = A B^T for FP32 device A, B at FP32 accuracy on the BF16 tensor cores: each operand is split into
 * three BF16 terms (x = x1 + x2 + x3 + O(2^-24 |x|)) and the six products x_i y_j with i + j <= 4
 * accumulate in FP32 in tensor memory, the corrections first and x1 y1 last.  The tensor cores' FP32
 * accumulation rounds toward zero, so a same-sign sum carries a relative bias of up to about 2^-24
 * per 16-wide K step accumulated per split (ceil(K / nsplit / 16) steps); split K to bound it.  The
 * products of the RSVD's orthonormalisation (Gram matrices X^T X, X R^{-1}) and of U = Q Uhat.  Layouts as rsk_gemm_bf16_ex (FP32 elements); any lda, ldb
 * covering the operand.  The splits and the split-K partials come from the handle's workspace.
 * Asynchronous. */
rsk_status rsk_gemm_f32(rsk_handle* h, int32_t a_mn, const float* A, int64_t M, int64_t K, int64_t lda, const float* B,
                        int64_t N, int64_t ldb, float* D, int64_t ldd, int32_t d_row_major, int32_t nsplit,
                        cudaStream_t stream);

/* ---------------------------------------------------------------------------------------------
 * a9: randomized SVD with a sparse sign test matrix (Alg. 1, Sec. 2.1) and power_iters subspace
 * iterations (re-orthonormalising after every product; Alg. 1 itself has none).
 * A: device FP32 m x n row-major (lda >= n).  Omega (n x r) has zeta nonzeros +-zeta^{-1/2} per row,
 * drawn as the left sparse sign of Philox stream 3 (rsk_sparse_sign_generate's rule with stream 3).
 * Outputs (device): U FP32 m x r row-major, s FP64[r] descending, Vt FP32 r x n row-major, with
 * A ~ U diag(s) Vt.  Products run on BF16 copies of A with FP32 accumulation; orthonormalisation is
 * shifted CholeskyQR3 in FP32 (the factor's inverse applied as a product); the r x r eigenproblem of
 * B B^T is solved in FP32 (B B^T is formed in FP32).  The first call for a shape times cuBLASLt's
 * candidate algorithms once.
 * Limits: 1 <= r <= min(m, n, 320), 1 <= zeta <= min(r, 32), m, n < 2^31.  Needs cuBLAS, cuBLASLt
 * and cuSOLVER at run time (RSK_ERR_UNSUPPORTED when they cannot be loaded). */
rsk_status rsk_rsvd(rsk_handle* h, const float* A, int64_t m, int64_t n, int64_t lda, int32_t r, int32_t power_iters,
                    int32_t zeta, uint64_t seed, float* U, double* s, float* Vt, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* RSK_H */
