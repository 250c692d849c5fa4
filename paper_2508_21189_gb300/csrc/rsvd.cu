// Randomized SVD with a sparse sign test matrix (row a9), on this library's kernels only.
// Paper: Alg. 1 (Sec. 2.1): Y = A Omega, Q = orth(Y), B = Q^T A, [Uhat, Sigma, V] = svd(B),
// U = Q Uhat.  Omega (n x r) is SparseUniform with zeta nonzeros per row (Def. SparseUniform),
// drawn from Philox stream 3 as the left sparse sign S = Omega^T (r rows, n columns).  Alg. 1 has no
// power iterations; q subspace iterations Q = orth(A^T Q), Q = orth(A Q) are applied after the
// sketch (re-orthonormalising after every product).
//
// Every tall matrix (Y, Q, Z) is FP32 column-major, leading dimension a multiple of 8.
//   A          converted once to BF16 (row-major); Y = A Omega and Y = A Z read it K-major, Z = A^T Q
//              reads the same copy MN-major (tcgen05 GEMMs, FP32 accumulation, no transposed copy)
//   orth(X)    Cholesky QR rounds: the three-term BF16 split of X, G = X^T X on the tensor cores (six
//              split products, K split so that each accumulator takes few steps: the tensor cores'
//              FP32 accumulation truncates), the Cholesky factor R of G (+ shift on the first round)
//              (blocked, one CTA) and R^{-1} (a warp per column), X <- X R^{-1} (split products again)
//   svd(B)     B = Z^T with Z = A^T Q: Z = Q_z R_z (orth with R accumulated), then a one-sided Jacobi
//              SVD of R_z^T = U_j Sigma V_j^T, so Uhat = U_j and V = Q_z V_j; no squared condition
//              number (B B^T is never formed)
//   U, V^T     U = Q Uhat (row-major output) and V = Q_z V_j (column-major n x r = row-major V^T)
//              as split products
#include <math.h>
#include <string.h>

#include <algorithm>
#include <utility>

#include "common.cuh"
#include "dense.cuh"
#include "gemm_tc.cuh"

namespace {

constexpr int kMaxRank = 320;  // the Cholesky kernel's limit (330) rounded down to the tested range

// Omega^T (r x n, ldo) = the +-1 pattern of the sparse sign S drawn from stream 3 (the 1/sqrt(zeta)
// scale is left out: the orthonormalisation that follows does not see it).
__global__ void k_omega_t(const int32_t* __restrict__ rows, const uint32_t* __restrict__ signs, int64_t n, int zeta,
                          __nv_bfloat16* __restrict__ Ot, int64_t ldo) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t sb = signs[j];
    for (int q = 0; q < zeta; ++q) {
        const int i = rows[j * zeta + q];
        Ot[int64_t(i) * ldo + j] = __float2bfloat16_rn(((sb >> q) & 1u) ? -1.f : 1.f);
    }
}

// T = X^T for a small column-major q x q X (both leading dimension q).
__global__ void k_transpose_sq(const float* __restrict__ X, int q, float* __restrict__ T) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= int64_t(q) * q) return;
    const int c = int(idx / q), i = int(idx - int64_t(c) * q);
    T[int64_t(i) * q + c] = X[idx];
}

__global__ void k_to_f64(const float* __restrict__ x, int n, double* __restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = double(x[i]);
}

struct Ws {
    __nv_bfloat16* Abf;      // m x n row-major, row pitch lda_bf
    int64_t lda_bf;
    __nv_bfloat16* Ot;       // r x n, pitch lda_bf
    float *Y, *Y2;           // m x r, ld ldm
    float *Z, *Z2;           // n x r, ld ldn
    int64_t ldm, ldn;
    __nv_bfloat16* Qbf;      // bf16 of the current basis, max(m, n) x r
    float *Racc, *Xs, *Vj, *sv;  // r x r (ld r), sv r
    float* part;             // split-K partials of the big products
    size_t part_bytes;
    void* oscratch;          // the orthonormalisations' scratch, then the final split products'
    void* svd_scratch;
    int32_t* orow;
    uint32_t* osgn;
};

}  // namespace

namespace rsk {

// D (M x r, column-major ld ldd) = A (BF16) * Bt^T for Bt = bf16 of a column-major K x r basis (its
// column c is row c of the K-major operand).
static rsk_status big_product(rsk_handle* h, bool a_mn, const __nv_bfloat16* A, int64_t lda, int64_t M, int64_t K,
                              const __nv_bfloat16* Bt, int64_t ldb, int r, float* D, int64_t ldd, Ws& w,
                              cudaStream_t s) {
    tc::Product p;
    p.a_mn = a_mn;
    p.a[0] = A;
    p.na = 1;
    p.lda = lda;
    p.b[0] = Bt;
    p.nb = 1;
    p.ldb = ldb;
    p.npass = 1;
    p.M = M;
    p.K = K;
    p.N = r;
    p.D = D;
    p.ldd = ldd;
    // split K when the row tiles alone leave SMs idle
    int nsplit = tc::wave_splits(M, K, h->num_sms);
    while (nsplit > 1 && tc::gemm_scratch_bytes(M, r, nsplit) > w.part_bytes) --nsplit;
    return tc::gemm(h, p, nsplit, w.part, s, 0, w.part_bytes, true);
}

}  // namespace rsk

extern "C" rsk_status rsk_rsvd(rsk_handle* h, const float* A, int64_t m, int64_t n, int64_t lda, int32_t r,
                               int32_t power_iters, int32_t zeta, uint64_t seed, float* U, double* s, float* Vt,
                               cudaStream_t stream) {
    using namespace rsk;
    if (!h) return RSK_ERR_INVALID_ARG;
    if (!A || !U || !s || !Vt) return fail(h, RSK_ERR_INVALID_ARG, "null pointer");
    if (m < 1 || n < 1 || lda < n || r < 1 || r > kMaxRank || r > std::min(m, n) || power_iters < 0)
        return fail(h, RSK_ERR_INVALID_ARG, "need 1 <= r <= min(m, n, %d), lda >= n, power_iters >= 0", kMaxRank);
    if (zeta < 1 || zeta > r || zeta > 32) return fail(h, RSK_ERR_INVALID_ARG, "need 1 <= zeta <= min(r, 32)");
    if (m >= (int64_t(1) << 31) || n >= (int64_t(1) << 31)) return fail(h, RSK_ERR_INVALID_ARG, "m, n < 2^31");

    Ws w;
    w.lda_bf = tc::pad8(n);
    w.ldm = tc::pad8(m);
    w.ldn = tc::pad8(n);
    const int64_t mx = std::max(w.ldm, w.ldn);
    // split-K partials of the K-split big products (Z = A^T Q; Y = A Z when m is small)
    const size_t part_bytes = std::max(tc::gemm_scratch_bytes(n, r, tc::wave_splits(n, m, h->num_sms)),
                                       tc::gemm_scratch_bytes(m, r, tc::wave_splits(m, n, h->num_sms)));
    const size_t fbytes = std::max(tc::f32_product_scratch_bytes(true, std::max(m, n), r, r, 1),
                                   tc::orth_scratch_bytes(mx, r));
    size_t bytes = 0;
    auto add = [&](size_t b_) { bytes += Carver::round(b_); };
    add(size_t(m) * w.lda_bf * 2);                  // A bf16
    add(size_t(r) * w.lda_bf * 2);                  // Omega^T
    add(size_t(w.ldm) * r * 4 * 2);                 // Y, Y2
    add(size_t(w.ldn) * r * 4 * 2);                 // Z, Z2
    add(size_t(mx) * r * 2);                        // Qbf
    add(fbytes);                                    // orthonormalisation / final products' scratch
    add(size_t(r) * r * 4 * 3 + size_t(r) * 4);     // small matrices
    add(part_bytes);
    add(dense::svd_scratch_bytes(r, r));
    add(size_t(n) * zeta * 4 + size_t(n) * 4);
    rsk_status st = ensure_workspace(h, bytes + 32 * 256, stream);
    if (st != RSK_OK) return st;
    Carver cv(h->ws);
    w.Abf = cv.take<__nv_bfloat16>(size_t(m) * w.lda_bf);
    w.Ot = cv.take<__nv_bfloat16>(size_t(r) * w.lda_bf);
    w.Y = cv.take<float>(size_t(w.ldm) * r);
    w.Y2 = cv.take<float>(size_t(w.ldm) * r);
    w.Z = cv.take<float>(size_t(w.ldn) * r);
    w.Z2 = cv.take<float>(size_t(w.ldn) * r);
    w.Qbf = cv.take<__nv_bfloat16>(size_t(mx) * r);
    w.oscratch = cv.take<char>(fbytes);
    w.Racc = cv.take<float>(size_t(r) * r);
    w.Xs = cv.take<float>(size_t(r) * r);
    w.Vj = cv.take<float>(size_t(r) * r);
    w.sv = cv.take<float>(size_t(r));
    w.part = cv.take<float>(part_bytes / 4 + 1);
    w.part_bytes = part_bytes;
    w.svd_scratch = cv.take<char>(dense::svd_scratch_bytes(r, r));
    w.orow = cv.take<int32_t>(size_t(n) * zeta);
    w.osgn = cv.take<uint32_t>(size_t(n));

    // ---- A in BF16 (row-major, pitch lda_bf); Omega^T dense +-1 from stream 3
    st = tc::to_bf16(h, A, n, m, lda, w.Abf, w.lda_bf, stream);
    if (st != RSK_OK) return st;
    RSK_CUDA_TRY(h, cudaMemsetAsync(w.Ot, 0, size_t(r) * w.lda_bf * 2, stream));
    st = sketch_generate(h, n, r, zeta, seed, 3u, w.orow, w.osgn, stream);
    if (st != RSK_OK) return st;
    k_omega_t<<<unsigned((n + 255) / 256), 256, 0, stream>>>(w.orow, w.osgn, n, zeta, w.Ot, w.lda_bf);
    RSK_LAUNCH_CHECK(h);

    // ---- range finder
    float* Y = w.Y;
    float* Y2 = w.Y2;
    float* Z = w.Z;
    float* Z2 = w.Z2;
    st = big_product(h, false, w.Abf, w.lda_bf, m, n, w.Ot, w.lda_bf, r, Y, w.ldm, w, stream);  // Y = A Omega
    if (st == RSK_OK) st = tc::orth(h, &Y, &Y2, m, r, w.ldm, power_iters > 0 ? 2 : 3, 1, nullptr, w.oscratch, stream);
    for (int it = 0; st == RSK_OK && it < power_iters; ++it) {
        st = tc::to_bf16(h, Y, m, r, w.ldm, w.Qbf, w.ldm, stream);
        if (st == RSK_OK)                                                                       // Z = A^T Q
            st = big_product(h, true, w.Abf, w.lda_bf, n, m, w.Qbf, w.ldm, r, Z, w.ldn, w, stream);
        if (st == RSK_OK) st = tc::orth(h, &Z, &Z2, n, r, w.ldn, 2, 1, nullptr, w.oscratch, stream);
        if (st == RSK_OK) st = tc::to_bf16(h, Z, n, r, w.ldn, w.Qbf, w.ldn, stream);
        if (st == RSK_OK)                                                                       // Y = A Z
            st = big_product(h, false, w.Abf, w.lda_bf, m, n, w.Qbf, w.ldn, r, Y, w.ldm, w, stream);
        if (st == RSK_OK) st = tc::orth(h, &Y, &Y2, m, r, w.ldm, it + 1 < power_iters ? 2 : 3, 1, nullptr, w.oscratch, stream);
    }
    if (st != RSK_OK) return st;
    // ---- B = Q^T A = Z^T with Z = A^T Q; Z = Q_z R_z
    st = tc::to_bf16(h, Y, m, r, w.ldm, w.Qbf, w.ldm, stream);
    if (st == RSK_OK) st = big_product(h, true, w.Abf, w.lda_bf, n, m, w.Qbf, w.ldm, r, Z, w.ldn, w, stream);
    if (st == RSK_OK) st = tc::orth(h, &Z, &Z2, n, r, w.ldn, 3, 1, w.Racc, w.oscratch, stream);
    if (st != RSK_OK) return st;
    // ---- B = Z^T = R_z^T Q_z^T;  svd(R_z^T) = U_j Sigma V_j^T (one-sided Jacobi, U_j overwrites Xs):
    // Uhat = U_j
    k_transpose_sq<<<unsigned((int64_t(r) * r + 255) / 256), 256, 0, stream>>>(w.Racc, r, w.Xs);
    RSK_LAUNCH_CHECK(h);
    {
        const int pr = prof_begin(h, stream, RSK_KERNEL_SMALL_SVD);
        st = dense::svd(h, w.Xs, r, r, r, w.sv, w.Vj, r, w.svd_scratch, stream);
        prof_end(h, stream, pr);
        if (st != RSK_OK) return st;
    }
    k_to_f64<<<unsigned((r + 255) / 256), 256, 0, stream>>>(w.sv, r, s);
    RSK_LAUNCH_CHECK(h);
    // ---- U = Q Uhat (row-major m x r); V = Q_z V_j, column-major n x r = row-major V^T (r x n)
    // (B_op[c][k] = Uhat[k][c]: column c of the column-major Uhat, and likewise for V_j)
    st = tc::f32_product(h, true, Y, w.ldm, w.Xs, r, m, r, r, U, r, true, 1, w.oscratch, stream);
    if (st == RSK_OK) st = tc::f32_product(h, true, Z, w.ldn, w.Vj, r, n, r, r, Vt, n, false, 1, w.oscratch, stream);
    return st;
}
