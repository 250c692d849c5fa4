// Dense products on the fifth-generation tensor cores (tcgen05) for the low-rank algorithms.
//
//     D (M x N, FP32) = sum over passes p of  A_{pa[p]} (M x K) * B_{pb[p]} (N x K)^T
//
// A operands are BF16 and either K-major (element (m, k) at A[m * lda + k]) or MN-major (element
// (m, k) at A[k * lda + m], i.e. the transpose of a row-major K x M matrix); B operands are BF16
// K-major (element (n, j) at B[n * ldb + j]).  Several passes over the same K range accumulate into
// one tensor-memory accumulator: with the three-term BF16 splits of two FP32 matrices this gives
// products of FP32 accuracy (the six pairs whose split orders sum to at most four).  D is column-major
// (element (m, n) at D[n * ldd + m]) or row-major (D[m * ldd + n]).  1 <= N <= 512.  Every pointer is
// 16-byte aligned and every leading dimension a multiple of 8 elements (TMA row pitch).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace rsk {
namespace tc {

constexpr int kMaxOperands = 3;
constexpr int kMaxPasses = 6;

struct Product {
    bool a_mn = false;  // A MN-major
    const __nv_bfloat16* a[kMaxOperands] = {};
    int na = 0;
    int64_t lda = 0;
    const __nv_bfloat16* b[kMaxOperands] = {};
    int nb = 0;
    int64_t ldb = 0;
    int npass = 0;
    uint8_t pa[kMaxPasses] = {}, pb[kMaxPasses] = {};
    int64_t M = 0, K = 0;
    int N = 0;
    float* D = nullptr;
    int64_t ldd = 0;
    bool d_row_major = false;
};

// Scratch for split-K partials (nsplit > 1).
size_t gemm_scratch_bytes(int64_t M, int N, int nsplit);
// K splits (at most max_split) that keep the SMs busiest for an M x K product with the automatic
// cluster: the fraction of SM time in full waves, discounted by each CTA's fixed cost (setup,
// pipeline fill, epilogue) relative to its K loop.  A 262144-row product gets 1, an 8192-row product
// with K = 262144 gets 7 (448 CTAs: 98% of three waves on 152 SMs, against 84% of one with 2).
int wave_splits(int64_t M, int64_t K, int num_sms, int max_split = 16);
// Runs the product with K split nsplit ways for every row tile (partials summed in split order).
// cluster: row tiles per thread-block cluster that share (multicast) the B tile, 1, 2 or 4 (4 for N
// halves 128, 160, 256 only); 0 picks 2 with at least 8 row tiles, else 1.  The kernel is persistent
// (one cluster per group of SMs, tiles dealt round-robin).  split_last (nsplit = 1, scratch of
// scratch_bytes): a last round of tiles that would leave more than half the clusters idle is split
// over K instead, its rows summed from partials.
rsk_status gemm(rsk_handle* h, const Product& p, int nsplit, float* scratch, cudaStream_t stream, int cluster = 0,
                size_t scratch_bytes = 0, bool split_last = false);

// The six split pairs (3,1), (1,3), (2,2), (2,1), (1,2), (1,1) of two three-term splits, in that
// order.  The accumulation truncates: a same-sign sum's relative bias grows by up to about 2^-24 per
// 16-wide K step a split accumulates (nsplit bounds it).
void set_split_passes(Product& p);

// X (rows x cols FP32, column c at X + c * ldx) -> three BF16 terms X = X1 + X2 + X3 + O(2^-24 |X|),
// each rows x cols with column c at Xt + c * ldt (ldt >= rows, a multiple of 8), written to out[0..2].
rsk_status split3(rsk_handle* h, const float* X, int64_t rows, int64_t cols, int64_t ldx, __nv_bfloat16* const* out,
                  int64_t ldt, cudaStream_t stream);
// X (FP32, same layout) -> bf16(X) with leading dimension ldt.
rsk_status to_bf16(rsk_handle* h, const float* X, int64_t rows, int64_t cols, int64_t ldx, __nv_bfloat16* out,
                   int64_t ldt, cudaStream_t stream);

// Product of FP32 matrices at FP32 accuracy: A (M x K; MN-major when a_mn, i.e. element (m, k) at
// A[k * lda + m], else A[m * lda + k]), B (N x K, element (n, j) at B[n * ldb + j]); the splits and the
// partials come from `scratch` (f32_product_scratch_bytes).
size_t f32_product_scratch_bytes(bool a_mn, int64_t M, int64_t K, int N, int nsplit);
rsk_status f32_product(rsk_handle* h, bool a_mn, const float* A, int64_t lda, const float* B, int64_t ldb, int64_t M,
                       int64_t K, int N, float* D, int64_t ldd, bool d_row_major, int nsplit, void* scratch,
                       cudaStream_t stream);

inline int64_t pad8(int64_t x) { return (x + 7) & ~int64_t(7); }

// Orthonormal basis of range(X) for a tall FP32 X (rows x r, column-major, ldx a multiple of 8 >= rows,
// r <= 330) by `rounds` Cholesky QR rounds: per round the three-term BF16 split of X, G = X^T X as
// split products (K split into accumulators of at most 16 K blocks), the Cholesky factor R of
// G + s I (s = 3e-5 trace(G) in the first `shifted` rounds, 0 after), R^{-1}, and X <- X R^{-1} as
// split products.  The result is in *X on return (the routine swaps *X and *Xalt, an rows x r
// buffer of the same leading dimension, as it goes).  Racc (r x r, column-major), when not null,
// receives the accumulated upper factor with X_in = Q Racc.  The shift suits a Gram accurate to a few
// 1e-6: each shifted round divides kappa by ~1 / sqrt(3e-5) ~ 180, and the plain rounds that follow
// need kappa below ~1e3.  A Cholesky pivot that is not positive sets RSK_DEV_BOUNDS.
size_t orth_scratch_bytes(int64_t rows, int r);
rsk_status orth(rsk_handle* h, float** X, float** Xalt, int64_t rows, int r, int64_t ldx, int rounds, int shifted,
                float* Racc, void* scratch, cudaStream_t stream);

}  // namespace tc
}  // namespace rsk
