// Small dense linear algebra on the GPU for the low-rank consumers of the sketches (the Nystrom
// approximations and the randomized SVD): FP64-accumulated Gram matrices, tall-by-small products,
// Cholesky, triangular inverses, a one-sided Jacobi SVD and FP64-Gram Cholesky QR.  FP32 storage and
// arithmetic, column-major matrices (column c of X at X + c * ldx).  Every routine is asynchronous
// on `stream`, carves its scratch from the caller's buffer and reports device-side failures (a
// Cholesky pivot that is not positive, a bounded wait that ran out) in the handle's status word.
#pragma once

#include "common.cuh"

namespace rsk {
namespace dense {

// Scratch bytes gram64() needs (per precision word) for an m x p by m x q product.
size_t gram_scratch_bytes(int64_t m, int p, int q);

// C (m x q, ldc) = X (m x p, ldx) * M (p x q, ldm).  C must not alias X or M.
rsk_status matmul_ts(rsk_handle* h, const float* X, int64_t m, int p, int64_t ldx, const float* M, int q,
                     int64_t ldm, float* C, int64_t ldc, cudaStream_t stream);

// Upper Cholesky factor R (q x q, ldr, zeros below the diagonal) of sym(G) + s I, s = shift_coeff *
// trace(G), G read from its upper triangle (q <= 330).  A pivot that is not positive (or not finite)
// sets RSK_DEV_BOUNDS and R is then undefined.
rsk_status cholesky(rsk_handle* h, const float* G, int q, int64_t ldg, float shift_coeff, float* R, int64_t ldr,
                    cudaStream_t stream);

// Ri = R^{-1} for an upper triangular q x q R (both ldr; Ri upper, zeros below).
rsk_status trinv(rsk_handle* h, const float* R, int q, int64_t ldr, float* Ri, cudaStream_t stream);

// One-sided Jacobi SVD of X (m x q, ldx, m >= q): X V = U diag(s), columns of U orthonormal, s
// descending.  X is overwritten by U; V (q x q, ldv) may be null.  s has q entries.  Limits:
// q <= 1024, m <= 4096.  scratch: svd_scratch_bytes(m, q).
size_t svd_scratch_bytes(int64_t m, int q);
rsk_status svd(rsk_handle* h, float* X, int64_t m, int q, int64_t ldx, float* s, float* V, int64_t ldv,
               void* scratch, cudaStream_t stream);

// Q = orth(X) for X m x q (ldx, m >= q), in place; R (q x q, upper) receives the accumulated factor
// with X_in = Q R when R is not null.  scratch: orth_scratch_bytes(m, q).
size_t orth_scratch_bytes(int64_t m, int q);
// By Cholesky QR2 with the Gram accumulated in FP64 from the FP32 entries and the Cholesky factor and
// its inverse in FP64: orthonormal to O(u_32) for kappa(X) up to ~1e7.  q <= 1024.  (The tensor-core
// Cholesky QR of gemm_tc.cuh is the fast form for q <= 330.)
rsk_status orth_accurate(rsk_handle* h, float* X, int64_t m, int q, int64_t ldx, float* R, void* scratch,
                         cudaStream_t stream);
// G (FP64) = X^T Y with FP64 accumulation of the FP32 products; scratch: 2 * gram_scratch_bytes.
rsk_status gram64(rsk_handle* h, const float* X, int64_t m, int p, int64_t ldx, const float* Y, int q, int64_t ldy,
                  double* G, int64_t ldg, void* scratch, cudaStream_t stream);

}  // namespace dense
}  // namespace rsk
