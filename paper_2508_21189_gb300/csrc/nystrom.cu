// Randomized Nystrom approximation of a psd matrix with a structured (sparse) test matrix.
// Paper: Alg. 2 (Sec. 2.2): Y = A Omega; nu = sqrt(n) eps ||Y||; Y_nu = Y + nu Omega;
// C = chol(Omega^T Y_nu); B = Y_nu C^{-1}; [U, Sigma, ~] = svd(B); Lambda = max(0, Sigma^2 - nu I).
//
// Omega = S^T with S the k x n SparseStack (Def. SparseStack; the paper's suggestion for Alg. 2) or
// SparseUniform sketch of this library, zeta nonzeros per row of Omega.  Because A is symmetric,
// Y^T = Omega^T A = S A is the left sketch of A: one pass over A by the sparse sign gather, whose
// k x n output is Y in column-major order.  nu uses eps = 2^-24 (the FP32 working precision) and the
// Frobenius norm of Y (never smaller than the spectral norm).  The second sketch Omega^T Y_nu = S Y_nu
// is the same gather on the n x k matrix Y_nu.  The dense steps (Cholesky, triangular inverse, the
// thin QR and SVD of B = Q_B R_B, R_B = U_R Sigma V_R^T, U = Q_B U_R) are the dense module's kernels.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "dense.cuh"
#include "gemm_tc.cuh"

namespace {

constexpr float kU32 = 5.9604645e-8f;

// Device buffer allocated stream-ordered for one call (the sketches use the handle's workspace).
struct DevBuf {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    ~DevBuf() {
        if (p) cudaFreeAsync(p, s);
    }
    rsk_status alloc(rsk_handle* h, size_t bytes, cudaStream_t stream) {
        s = stream;
        const char* inj = getenv("RSK_FAULT_NOMEM");
        if (inj && inj[0] == '1') return rsk::fail(h, RSK_ERR_NOMEM, "allocation of %zu bytes refused (RSK_FAULT_NOMEM=1)", bytes);
        cudaError_t e = cudaMallocAsync(&p, bytes, stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return rsk::fail(h, RSK_ERR_NOMEM, "allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        }
        return RSK_OK;
    }
};

// Sum of squares of x[0 .. count), per CTA, then summed in CTA order (deterministic).
__global__ void k_sumsq_part(const float* __restrict__ x, int64_t count, double* __restrict__ part) {
    __shared__ double red[32];
    double t = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
        t += double(x[i]) * double(x[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

// nu = sqrt(n) * u32 * sqrt(sum of the parts)
__global__ void k_shift(const double* __restrict__ part, int nparts, int64_t n, float* __restrict__ nu) {
    double s = 0.0;
    for (int i = 0; i < nparts; ++i) s += part[i];
    *nu = float(sqrt(double(n)) * double(kU32) * sqrt(s));
}

// Y_nu^T = Y^T + nu Omega^T: column j of S has entries (rows[j*zeta + q], j), sign bit q of signs[j],
// value +-zeta^{-1/2}; Y^T is k x n row-major (leading dimension n).  The rows of one column are
// distinct, so no two threads touch the same element.
__global__ void k_add_shift(float* __restrict__ Yt, int64_t n, const int32_t* __restrict__ rows,
                            const uint32_t* __restrict__ signs, int zeta, const float* __restrict__ nu) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float v = *nu * rsqrtf(float(zeta));
    const uint32_t sb = signs[j];
    for (int q = 0; q < zeta; ++q) {
        const int r = rows[j * zeta + q];
        Yt[int64_t(r) * n + j] += ((sb >> q) & 1u) ? -v : v;
    }
}

// out (cols x rows, row-major) = in (rows x cols, row-major)^T, through a padded shared tile.
__global__ void k_transpose(const float* __restrict__ in, int64_t rows, int64_t cols, float* __restrict__ out) {
    __shared__ float t[32][33];
    const int64_t r0 = int64_t(blockIdx.y) * 32, c0 = int64_t(blockIdx.x) * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[i][threadIdx.x] = in[r * cols + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[c * rows + r] = t[threadIdx.x][i];
    }
}

// Msym = (M + M^T) / 2 for a k x k row-major M (the result is symmetric, so its storage order is moot).
__global__ void k_symmetrize(const float* __restrict__ M, int k, float* __restrict__ S) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= int64_t(k) * k) return;
    const int i = int(idx / k), j = int(idx - int64_t(i) * k);
    S[idx] = 0.5f * (M[int64_t(i) * k + j] + M[int64_t(j) * k + i]);
}

__global__ void k_lambda(const float* __restrict__ s, const float* __restrict__ nu, int rank, float* __restrict__ lam) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < rank) lam[i] = fmaxf(0.f, s[i] * s[i] - *nu);
}

}  // namespace

extern "C" rsk_status rsk_nystrom_psd(rsk_handle* h, const float* A, int64_t n, int64_t lda, int32_t k, int32_t rank,
                                      int32_t zeta, uint64_t seed, int32_t kind, float* U, int64_t ldu, float* lambda,
                                      cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    if (!A || !U || !lambda) return rsk::fail(h, RSK_ERR_INVALID_ARG, "null pointer");
    if (kind != 0 && kind != 1) return rsk::fail(h, RSK_ERR_INVALID_ARG, "kind must be 0 (SparseUniform) or 1 (SparseStack)");
    if (n < 1 || n >= (int64_t(1) << 31) || lda < n || k < 1 || k > n || rank < 1 || rank > k || ldu < n)
        return rsk::fail(h, RSK_ERR_INVALID_ARG, "need 1 <= rank <= k <= n < 2^31, lda >= n, ldu >= n");
    if (zeta < 1 || zeta > 32 || zeta > k || (kind == 1 && k % zeta != 0))
        return rsk::fail(h, RSK_ERR_INVALID_ARG, "need 1 <= zeta <= min(k, 32) (and k a multiple of zeta for SparseStack)");
    if (k > 330) return rsk::fail(h, RSK_ERR_UNSUPPORTED, "k <= 330 (the dense steps' limit)");
    using rsk::Carver;
    const size_t nk = size_t(n) * k;
    const int nparts = 256;
    // the tensor-core path (split products, Cholesky QR on the tensor cores) needs k within the
    // Cholesky kernel's 330; B is kept with a leading dimension that is a multiple of 8
    const bool tcp = k <= 330;
    const int64_t ldb = rsk::tc::pad8(n);
    const size_t bk = size_t(ldb) * k;
    const size_t scr = std::max({rsk::dense::orth_scratch_bytes(n, k), rsk::dense::svd_scratch_bytes(k, k),
                                 tcp ? rsk::tc::orth_scratch_bytes(n, k) : 0,
                                 tcp ? rsk::tc::f32_product_scratch_bytes(true, n, k, k, 1) : 0});
    const size_t bytes = 2 * Carver::round(nk * 4) + 2 * Carver::round(bk * 4) + 5 * Carver::round(size_t(k) * k * 4) +
                         Carver::round(size_t(n) * zeta * 4) + Carver::round(size_t(n) * 4) + Carver::round(nparts * 8) +
                         Carver::round(size_t(k) * 4) + 256 + scr + 256;
    DevBuf buf;
    rsk_status st = buf.alloc(h, bytes, stream);
    if (st != RSK_OK) return st;
    Carver cv(buf.p);
    float* Yt = cv.take<float>(nk);     // Y^T (k x n row-major) = Y column-major, then Y_nu, then Q_B
    float* Yrm = cv.take<float>(nk);    // Y_nu row-major (n x k)
    float* B = cv.take<float>(bk);      // B = Y_nu C^{-1} (n x k column-major, leading dimension ldb)
    float* B2 = cv.take<float>(bk);     // the orthonormalisation's second buffer
    float* M = cv.take<float>(size_t(k) * k);
    float* Ms = cv.take<float>(size_t(k) * k);
    float* C = cv.take<float>(size_t(k) * k);
    float* Ci = cv.take<float>(size_t(k) * k);
    float* RB = cv.take<float>(size_t(k) * k);
    int32_t* rows = cv.take<int32_t>(size_t(n) * zeta);
    uint32_t* signs = cv.take<uint32_t>(size_t(n));
    double* part = cv.take<double>(nparts);
    float* sv = cv.take<float>(size_t(k));
    float* nu = cv.take<float>(1);
    void* scratch = cv.take<char>(scr);

    // Y^T = S A (one pass over A)
    st = rsk::sketch_apply_kind(h, kind, A, RSK_F32, n, n, lda, k, zeta, seed, Yt, RSK_F32, n, stream);
    if (st != RSK_OK) return st;
    // nu = sqrt(n) u ||Y||_F, then Y_nu = Y + nu Omega
    k_sumsq_part<<<nparts, 256, 0, stream>>>(Yt, int64_t(nk), part);
    k_shift<<<1, 1, 0, stream>>>(part, nparts, n, nu);
    RSK_LAUNCH_CHECK(h);
    st = rsk::sketch_generate_kind(h, n, k, zeta, seed, kind, rows, signs, stream);
    if (st != RSK_OK) return st;
    k_add_shift<<<unsigned((n + 255) / 256), 256, 0, stream>>>(Yt, n, rows, signs, zeta, nu);
    // Omega^T Y_nu = S Y_nu (Y_nu row-major), symmetrised
    k_transpose<<<dim3(unsigned((n + 31) / 32), unsigned((k + 31) / 32)), dim3(32, 8), 0, stream>>>(Yt, k, n, Yrm);
    RSK_LAUNCH_CHECK(h);
    st = rsk::sketch_apply_kind(h, kind, Yrm, RSK_F32, n, k, k, k, zeta, seed, M, RSK_F32, k, stream);
    if (st != RSK_OK) return st;
    k_symmetrize<<<unsigned((int64_t(k) * k + 255) / 256), 256, 0, stream>>>(M, k, Ms);
    RSK_LAUNCH_CHECK(h);
    // C = chol(Omega^T Y_nu) (upper), B = Y_nu C^{-1}
    st = rsk::dense::cholesky(h, Ms, k, k, 0.f, C, k, stream);
    if (st == RSK_OK) st = rsk::dense::trinv(h, C, k, k, Ci, stream);
    if (st != RSK_OK) return st;
    if (tcp) {
        // B = Y_nu C^{-1} as a split product (Y_nu column-major is the MN-major operand; column c of the
        // column-major C^{-1} is row c of the K-major one); svd(B): B = Q_B R_B by Cholesky QR on the
        // tensor cores (kappa(B) = kappa(A_hat)^{1/2}: one shifted round, two plain), R_B = U_R Sigma
        // V_R^T, U = Q_B U_R as a split product
        st = rsk::tc::f32_product(h, true, Yt, n, Ci, k, n, k, k, B, ldb, false, 1, scratch, stream);
        float* Bq = B;
        float* Balt = B2;
        if (st == RSK_OK) st = rsk::tc::orth(h, &Bq, &Balt, n, k, ldb, 3, 1, RB, scratch, stream);
        if (st == RSK_OK) st = rsk::dense::svd(h, RB, k, k, k, sv, nullptr, 0, scratch, stream);
        if (st == RSK_OK) st = rsk::tc::f32_product(h, true, Bq, ldb, RB, k, n, k, rank, U, ldu, false, 1, scratch, stream);
    } else {
        st = rsk::dense::matmul_ts(h, Yt, n, k, n, Ci, k, k, B, ldb, stream);
        // svd(B): B = Q_B R_B (FP64 Gram), R_B = U_R Sigma V_R^T, U = Q_B U_R
        if (st == RSK_OK) st = rsk::dense::orth_accurate(h, B, n, k, ldb, RB, scratch, stream);
        if (st == RSK_OK) st = rsk::dense::svd(h, RB, k, k, k, sv, nullptr, 0, scratch, stream);
        if (st == RSK_OK) st = rsk::dense::matmul_ts(h, B, n, k, ldb, RB, rank, k, U, ldu, stream);
    }
    if (st != RSK_OK) return st;
    k_lambda<<<unsigned((rank + 255) / 256), 256, 0, stream>>>(sv, nu, rank, lambda);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

// ------------------------------------------------------------------------------------------
// Generalized Nystrom (Algs. 4 and 5, Sec. 2.4): Y = A Omega (n x k) and X = A^T Psi (d x p) from one
// pass each over A (the right and left sparse sketches), then small dense steps.
// ------------------------------------------------------------------------------------------
namespace {

// r = #{i : s[i] > 5 u32 s[0]} (s descending)
__global__ void k_numrank(const float* __restrict__ s, int q, int* __restrict__ r) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const float cut = 5.f * kU32 * s[0];
    int c = 0;
    for (int i = threadIdx.x; i < q; i += blockDim.x) c += (s[i] > cut) ? 1 : 0;
    atomicAdd(&cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) *r = s[0] > 0.f ? cnt : 0;
}

// X (rows x q, column-major, ldx): column i scaled by 1 / s[i] (scale_inv) or kept, and zeroed for i >= *r.
__global__ void k_scale_trunc(float* __restrict__ X, int rows, int q, int64_t ldx, const float* __restrict__ s,
                              const int* __restrict__ r, bool scale_inv) {
    const int c = blockIdx.y;
    const float f = c < *r ? (scale_inv ? 1.f / s[c] : 1.f) : 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) X[int64_t(c) * ldx + i] *= f;
}

}  // namespace

extern "C" rsk_status rsk_gen_nystrom(rsk_handle* h, const float* A, int64_t n, int64_t d, int64_t lda, int32_t k,
                                      int32_t p, int32_t zeta, uint64_t seed, int32_t kind, int32_t form, float* out1,
                                      int64_t ld1, float* sigma, float* out2, int64_t ld2, int32_t* rank,
                                      cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    if (!A || !out1 || !out2 || !rank || (form == 1 && !sigma)) return rsk::fail(h, RSK_ERR_INVALID_ARG, "null pointer");
    if (kind != 0 && kind != 1) return rsk::fail(h, RSK_ERR_INVALID_ARG, "kind must be 0 (SparseUniform) or 1 (SparseStack)");
    if (form != 0 && form != 1) return rsk::fail(h, RSK_ERR_INVALID_ARG, "form must be 0 (Alg. 4) or 1 (Alg. 5)");
    if (n < 1 || d < 1 || n >= (int64_t(1) << 31) || d >= (int64_t(1) << 31) || lda < d || k < 1 || p < k ||
        p > std::min(n, d) || ld1 < n || ld2 < d)
        return rsk::fail(h, RSK_ERR_INVALID_ARG, "need 1 <= k <= p <= min(n, d), lda >= d, ld1 >= n, ld2 >= d");
    if (zeta < 1 || zeta > 32 || zeta > k || (kind == 1 && (k % zeta != 0 || p % zeta != 0)))
        return rsk::fail(h, RSK_ERR_INVALID_ARG, "need 1 <= zeta <= min(k, 32) (and k, p multiples of zeta for SparseStack)");
    if (k > 512 || p > 1024) return rsk::fail(h, RSK_ERR_UNSUPPORTED, "k <= 512 and p <= 1024");
    using rsk::Carver;
    const size_t nk = size_t(n) * k, pd = size_t(p) * d;
    // tensor-core QRs (Alg. 5) where the Cholesky kernel's limit and the leading dimensions allow
    const bool tcq = form == 1 && k <= 330 && p <= 330 && n % 8 == 0 && d % 8 == 0;
    const size_t scr = std::max({rsk::dense::orth_scratch_bytes(n, k), rsk::dense::orth_scratch_bytes(d, p),
                                 rsk::dense::svd_scratch_bytes(p, k), rsk::tc::f32_product_scratch_bytes(true, n, k, k, 1),
                                 rsk::tc::f32_product_scratch_bytes(true, d, p, k, 1),
                                 tcq ? rsk::tc::orth_scratch_bytes(std::max(n, d), std::max(k, p)) : 0});
    const size_t bytes = 2 * Carver::round(nk * 4) + Carver::round(pd * 4) + 3 * Carver::round(size_t(p) * k * 4) +
                         3 * Carver::round(size_t(k) * k * 4) + Carver::round(size_t(p) * p * 4) +
                         2 * Carver::round(size_t(k) * 4) + Carver::round(scr) + (tcq ? Carver::round(pd * 4) : 0) + 1024;
    DevBuf buf;
    rsk_status st = buf.alloc(h, bytes, stream);
    if (st != RSK_OK) return st;
    Carver cv(buf.p);
    float* Y = cv.take<float>(nk);               // A Omega, n x k column-major; Q in Alg. 5
    float* Qrm = cv.take<float>(nk);             // Q row-major (Alg. 5)
    float* Xt = cv.take<float>(pd);              // Psi^T A, p x d row-major = X column-major (d x p); P
    float* W = cv.take<float>(size_t(p) * k);    // p x k column-major work
    float* Z = cv.take<float>(size_t(p) * k);
    float* E = cv.take<float>(size_t(p) * k);
    float* V1 = cv.take<float>(size_t(k) * k);
    float* Vt = cv.take<float>(size_t(k) * k);
    float* V2 = cv.take<float>(size_t(k) * k);
    float* T = cv.take<float>(size_t(p) * p);
    float* s1 = cv.take<float>(size_t(k));
    float* s2 = cv.take<float>(size_t(k));
    void* scratch = cv.take<char>(scr);
    float* Xalt = tcq ? cv.take<float>(pd) : nullptr;   // second buffer of X's orthonormalisation

    // sketches: Y = A Omega (Omega = S^T, S k x d from seed), X^T = Psi^T A (Psi = S'^T, S' p x n from seed + 1)
    st = rsk::sketch_apply_right(h, kind, A, n, d, lda, k, zeta, seed, Y, n, stream);
    if (st == RSK_OK) st = rsk::sketch_apply_kind(h, kind, A, RSK_F32, n, d, lda, p, zeta, seed + 1, Xt, RSK_F32, d, stream);
    if (st != RSK_OK) return st;
    const dim3 tb(32, 8);
    if (form == 0) {
        // Alg. 4: [U, Sigma, V] = svd(X^T Omega); F = Y V_r Sigma_r^{-1}; G = X U_r
        st = rsk::sketch_apply_right(h, kind, Xt, p, d, d, k, zeta, seed, W, p, stream);
        if (st == RSK_OK) st = rsk::dense::svd(h, W, p, k, p, s1, V1, k, scratch, stream);
        if (st != RSK_OK) return st;
        k_numrank<<<1, 256, 0, stream>>>(s1, k, rank);
        k_scale_trunc<<<dim3(1, unsigned(k)), 256, 0, stream>>>(V1, k, k, k, s1, rank, true);
        k_scale_trunc<<<dim3(4, unsigned(k)), 256, 0, stream>>>(W, p, k, p, s1, rank, false);
        RSK_LAUNCH_CHECK(h);
        // F = Y (V Sigma^{-1})_r, G = X U_r as split products (column c of the column-major right factor
        // is row c of the K-major operand)
        st = rsk::tc::f32_product(h, true, Y, n, V1, k, n, k, k, out1, ld1, false, 1, scratch, stream);
        if (st == RSK_OK) st = rsk::tc::f32_product(h, true, Xt, d, W, p, d, p, k, out2, ld2, false, 1, scratch, stream);
        return st;
    }
    // Alg. 5: Q = qr(Y); [P, T] = qr(X); [U1, S1, V1] = svd(Psi^T Q); C = V1_r S1_r^{-1} U1_r^T T^T;
    // [Uh, Sigma, Vh] = svd(C); U = Q Uh; V = P Vh.  C is k x p, so svd(C^T) = (Vh, Sigma, Uh) is taken.
    if (tcq) {
        // Cholesky QR on the tensor cores: two shifted rounds and two plain ones (kappa(A Omega) can be
        // large: each shifted round divides it by ~180); the results are copied back when they end in
        // the second buffer (Q row-major's storage serves Y, which is written only later)
        float* Yq = Y;
        float* Yalt = Qrm;
        st = rsk::tc::orth(h, &Yq, &Yalt, n, k, n, 4, 2, nullptr, scratch, stream);
        if (st == RSK_OK && Yq != Y)
            RSK_CUDA_TRY(h, cudaMemcpyAsync(Y, Yq, nk * 4, cudaMemcpyDeviceToDevice, stream));
        float* Xq = Xt;
        float* Xa = Xalt;
        if (st == RSK_OK) st = rsk::tc::orth(h, &Xq, &Xa, d, p, d, 4, 2, T, scratch, stream);
        if (st == RSK_OK && Xq != Xt)
            RSK_CUDA_TRY(h, cudaMemcpyAsync(Xt, Xq, pd * 4, cudaMemcpyDeviceToDevice, stream));
    } else {
        st = rsk::dense::orth_accurate(h, Y, n, k, n, nullptr, scratch, stream);
        if (st == RSK_OK) st = rsk::dense::orth_accurate(h, Xt, d, p, d, T, scratch, stream);
    }
    if (st != RSK_OK) return st;
    k_transpose<<<dim3(unsigned((n + 31) / 32), unsigned((k + 31) / 32)), tb, 0, stream>>>(Y, k, n, Qrm);
    RSK_LAUNCH_CHECK(h);
    st = rsk::sketch_apply_kind(h, kind, Qrm, RSK_F32, n, k, k, p, zeta, seed + 1, Z, RSK_F32, k, stream);
    if (st != RSK_OK) return st;
    k_transpose<<<dim3(unsigned((k + 31) / 32), unsigned((p + 31) / 32)), tb, 0, stream>>>(Z, p, k, W);
    RSK_LAUNCH_CHECK(h);
    st = rsk::dense::svd(h, W, p, k, p, s1, V1, k, scratch, stream);
    if (st != RSK_OK) return st;
    k_numrank<<<1, 256, 0, stream>>>(s1, k, rank);
    RSK_LAUNCH_CHECK(h);
    // C^T = (T U1 S1^{-1})_r V1^T  (p x k)
    st = rsk::dense::matmul_ts(h, T, p, p, p, W, k, p, E, p, stream);
    if (st != RSK_OK) return st;
    k_scale_trunc<<<dim3(4, unsigned(k)), 256, 0, stream>>>(E, p, k, p, s1, rank, true);
    k_transpose<<<dim3(unsigned((k + 31) / 32), unsigned((k + 31) / 32)), tb, 0, stream>>>(V1, k, k, Vt);
    RSK_LAUNCH_CHECK(h);
    st = rsk::dense::matmul_ts(h, E, p, k, p, Vt, k, k, Z, p, stream);
    // svd(C^T) = Vh Sigma Uh^T: Z -> Vh (p x k), V2 = Uh (k x k)
    if (st == RSK_OK) st = rsk::dense::svd(h, Z, p, k, p, s2, V2, k, scratch, stream);
    if (st == RSK_OK) st = rsk::tc::f32_product(h, true, Y, n, V2, k, n, k, k, out1, ld1, false, 1, scratch, stream);
    if (st == RSK_OK) st = rsk::tc::f32_product(h, true, Xt, d, Z, p, d, p, k, out2, ld2, false, 1, scratch, stream);
    if (st != RSK_OK) return st;
    RSK_CUDA_TRY(h, cudaMemcpyAsync(sigma, s2, size_t(k) * 4, cudaMemcpyDeviceToDevice, stream));
    return RSK_OK;
}
