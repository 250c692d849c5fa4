// Randomized SVD with a sparse sign test matrix (row a9).
// Paper: Alg. 1 (Sec. 2.1): Y = A Omega, Q = orth(Y), B = Q^T A, [Uhat, Sigma, V] = svd(B),
// U = Q Uhat.  Omega (n x r) is SparseUniform with zeta nonzeros per row (Def. SparseUniform),
// drawn from Philox stream 3 as the left sparse sign S = Omega^T (r rows, n columns).  Alg. 1 has no
// power iterations; q subspace iterations Q = orth(A^T Q), Q = orth(A Q) are applied after the
// sketch (re-orthonormalising after every product).
//
// Precision plan.  A (FP32) is converted once to BF16 in both orientations (A and A^T) so that
// every product is a GEMM with both operands K-major:
//     Y = A Omega      : [m x n] * [r x n]^T      Z = A^T Q : [n x m] * [r x m]^T
// with FP32 accumulation on the tensor cores.  orth() is shifted CholeskyQR3 in FP32 (one shifted
// round, two plain ones): the Gram G = X^T X, a Cholesky of G (+ shift) in shared memory, and
// X <- X R^{-1}; the shift keeps the first Cholesky defined up to kappa(X) ~ u^{-1}, the plain rounds
// restore orthogonality to O(u_32), below the BF16 error of the products.  The small SVD of
// B = Z^T comes from the symmetric eigenproblem of Z^T Z (r x r, FP64).
//
// The plain products (GEMM, SYRK, TRSM) go through cuBLAS and the r x r eigenproblem through
// cuSOLVER, both loaded at first use with dlopen; everything else is this file's kernels.
#include <cuda_bf16.h>
#include <dlfcn.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace {

// ------------------------------------------------------------------------------------------
// Minimal cuBLAS / cuSOLVER surface (types and constants from their public headers' values).
// ------------------------------------------------------------------------------------------
typedef void* cublasH;
typedef void* cusolverH;
enum { kOpN = 0, kOpT = 1 };
enum { kFillLower = 0, kFillUpper = 1 };
enum { kSideLeft = 0, kSideRight = 1 };
enum { kDiagNonUnit = 0 };
enum { kR32F = 0, kR64F = 1, kR16BF = 14 };
enum { kCompute32F = 68 };
enum { kGemmDefault = -1 };
enum { kEigModeVector = 1 };

struct Libs {
    bool tried = false, ok = false;
    void *blas = nullptr, *solver = nullptr;
    int (*blasCreate)(cublasH*);
    int (*blasSetStream)(cublasH, cudaStream_t);
    int (*gemmEx)(cublasH, int, int, int, int, int, const void*, const void*, int, int, const void*, int, int,
                  const void*, void*, int, int, int, int);
    int (*ssyrk)(cublasH, int, int, int, int, const float*, const float*, int, const float*, float*, int);
    int (*strsm)(cublasH, int, int, int, int, int, int, const float*, const float*, int, float*, int);
    int (*sgemm)(cublasH, int, int, int, int, int, const float*, const float*, int, const float*, int, const float*,
                 float*, int);
    int (*solverCreate)(cusolverH*);
    int (*solverSetStream)(cusolverH, cudaStream_t);
    int (*dsyevdBuf)(cusolverH, int, int, int, const double*, int, const double*, int*);
    int (*dsyevd)(cusolverH, int, int, int, double*, int, double*, double*, int, int*);
    cublasH bh = nullptr;
    cusolverH sh = nullptr;
};
Libs g_libs;

template <typename F>
bool sym(void* lib, const char* name, F& fn) {
    fn = reinterpret_cast<F>(dlsym(lib, name));
    return fn != nullptr;
}

rsk_status load_libs(rsk_handle* h) {
    Libs& L = g_libs;
    if (L.tried) return L.ok ? RSK_OK : rsk::fail(h, RSK_ERR_UNSUPPORTED, "cuBLAS/cuSOLVER could not be loaded");
    L.tried = true;
    L.blas = dlopen("libcublas.so.13", RTLD_NOW | RTLD_LOCAL);
    if (!L.blas) L.blas = dlopen("libcublas.so", RTLD_NOW | RTLD_LOCAL);
    L.solver = dlopen("libcusolver.so.12", RTLD_NOW | RTLD_LOCAL);
    if (!L.solver) L.solver = dlopen("libcusolver.so", RTLD_NOW | RTLD_LOCAL);
    if (!L.blas || !L.solver) return rsk::fail(h, RSK_ERR_UNSUPPORTED, "cuBLAS/cuSOLVER not found");
    bool ok = sym(L.blas, "cublasCreate_v2", L.blasCreate) && sym(L.blas, "cublasSetStream_v2", L.blasSetStream) &&
              sym(L.blas, "cublasGemmEx", L.gemmEx) && sym(L.blas, "cublasSsyrk_v2", L.ssyrk) &&
              sym(L.blas, "cublasStrsm_v2", L.strsm) && sym(L.blas, "cublasSgemm_v2", L.sgemm) &&
              sym(L.solver, "cusolverDnCreate", L.solverCreate) &&
              sym(L.solver, "cusolverDnSetStream", L.solverSetStream) &&
              sym(L.solver, "cusolverDnDsyevd_bufferSize", L.dsyevdBuf) && sym(L.solver, "cusolverDnDsyevd", L.dsyevd);
    if (!ok) return rsk::fail(h, RSK_ERR_UNSUPPORTED, "cuBLAS/cuSOLVER symbols missing");
    if (L.blasCreate(&L.bh) != 0 || L.solverCreate(&L.sh) != 0)
        return rsk::fail(h, RSK_ERR_CUDA, "cuBLAS/cuSOLVER handle creation failed");
    L.ok = true;
    return RSK_OK;
}

// ------------------------------------------------------------------------------------------
// Kernels.
// ------------------------------------------------------------------------------------------
__global__ void k_to_bf16(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda, __nv_bfloat16* __restrict__ B) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= m * n) return;
    const int64_t i = idx / n, j = idx - i * n;
    B[idx] = __float2bfloat16_rn(A[i * lda + j]);
}

// B = bf16(A^T): A m x n (lda), B n x m row-major; 32 x 32 tiles through shared memory.
__global__ void k_transpose_bf16(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                                 __nv_bfloat16* __restrict__ B) {
    __shared__ float tile[32][33];
    const int64_t i0 = int64_t(blockIdx.y) * 32, j0 = int64_t(blockIdx.x) * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = i0 + r, j = j0 + threadIdx.x;
        tile[r][threadIdx.x] = (i < m && j < n) ? A[i * lda + j] : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t j = j0 + r, i = i0 + threadIdx.x;
        if (j < n && i < m) B[j * m + i] = __float2bfloat16_rn(tile[threadIdx.x][r]);
    }
}

// X (rows x r, FP32, row-major) -> bf16(X^T) (r x rows)
__global__ void k_transpose_f32_bf16(const float* __restrict__ X, int64_t rows, int r, __nv_bfloat16* __restrict__ T) {
    __shared__ float tile[32][33];
    const int64_t i0 = int64_t(blockIdx.y) * 32;
    const int j0 = blockIdx.x * 32;
    for (int rr = threadIdx.y; rr < 32; rr += blockDim.y) {
        const int64_t i = i0 + rr;
        const int j = j0 + threadIdx.x;
        tile[rr][threadIdx.x] = (i < rows && j < r) ? X[i * r + j] : 0.f;
    }
    __syncthreads();
    for (int rr = threadIdx.y; rr < 32; rr += blockDim.y) {
        const int j = j0 + rr;
        const int64_t i = i0 + threadIdx.x;
        if (j < r && i < rows) T[int64_t(j) * rows + i] = __float2bfloat16_rn(tile[threadIdx.x][rr]);
    }
}

// Omega^T (r x n, bf16) = +-1 pattern of the sparse sign S drawn from stream 3 (scale applied later).
__global__ void k_omega_t(const int32_t* __restrict__ rows, const uint32_t* __restrict__ signs, int64_t n, int zeta,
                          __nv_bfloat16* __restrict__ Ot) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t sb = signs[j];
    for (int q = 0; q < zeta; ++q) {
        const int i = rows[j * zeta + q];
        Ot[int64_t(i) * n + j] = __float2bfloat16_rn(((sb >> q) & 1u) ? -1.f : 1.f);
    }
}

__global__ void k_scale(float* __restrict__ X, int64_t count, float s) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx < count) X[idx] *= s;
}

// Cholesky of G (+ shift) in shared memory, packed lower triangle, FP32.  G: r x r symmetric with
// the lower triangle valid in column-major storage (G[k*r + i], i >= k).  Writes R = L^T into Rout
// (column-major upper triangle: Rout[i*r + k] = L[i][k] for k <= i, zero elsewhere).  shift_mode 1
// adds 11 (rows*r + r(r+1)) u_32 trace(G) to the diagonal (the shift of shifted CholeskyQR).
__global__ void __launch_bounds__(1024) k_cholesky(const float* __restrict__ G, int r, float* __restrict__ Rout,
                                                   int shift_mode, double rows, unsigned int* status) {
    extern __shared__ float L[];  // r(r+1)/2
    __shared__ float piv;
    __shared__ double tr;
    auto at = [](int i, int k) { return i * (i + 1) / 2 + k; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < r; ++i) t += double(G[size_t(i) * r + i]);
        tr = t;
    }
    __syncthreads();
    const float shift = shift_mode ? float(11.0 * (rows * r + double(r) * (r + 1)) * 5.960464477539063e-08 * tr) : 0.f;
    for (int i = warp; i < r; i += nw)
        for (int k = lane; k <= i; k += 32) L[at(i, k)] = G[size_t(k) * r + i] + (i == k ? shift : 0.f);
    __syncthreads();
    for (int j = 0; j < r; ++j) {
        if (threadIdx.x == 0) {
            const float djj = L[at(j, j)];
            if (!(djj > 0.f)) atomicOr(status, RSK_DEV_BOUNDS);
            piv = sqrtf(fmaxf(djj, 1e-30f));
            L[at(j, j)] = piv;
        }
        __syncthreads();
        const float p = piv;
        for (int i = j + 1 + threadIdx.x; i < r; i += blockDim.x) L[at(i, j)] /= p;
        __syncthreads();
        for (int i = j + 1 + warp; i < r; i += nw) {
            const float lij = L[at(i, j)];
            for (int k = j + 1 + lane; k <= i; k += 32) L[at(i, k)] -= lij * L[at(k, j)];
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
        const int i = idx / r, k = idx - i * r;
        Rout[size_t(i) * r + k] = (k <= i) ? L[at(i, k)] : 0.f;
    }
}

// T (cols x rows, row-major) = X^T for X (rows x cols, row-major), FP32.
__global__ void k_transpose_f32(const float* __restrict__ X, int64_t rows, int cols, float* __restrict__ T) {
    __shared__ float tile[32][33];
    const int64_t i0 = int64_t(blockIdx.y) * 32;
    const int j0 = blockIdx.x * 32;
    for (int rr = threadIdx.y; rr < 32; rr += blockDim.y) {
        const int64_t i = i0 + rr;
        const int j = j0 + threadIdx.x;
        tile[rr][threadIdx.x] = (i < rows && j < cols) ? X[i * cols + j] : 0.f;
    }
    __syncthreads();
    for (int rr = threadIdx.y; rr < 32; rr += blockDim.y) {
        const int j = j0 + rr;
        const int64_t i = i0 + threadIdx.x;
        if (j < cols && i < rows) T[int64_t(j) * rows + i] = tile[threadIdx.x][rr];
    }
}

__global__ void k_f32_to_f64(const float* __restrict__ a, double* __restrict__ b, int64_t count) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx < count) b[idx] = double(a[idx]);
}

// eigenvalues ascending (w) and vectors (columns of V, column-major) -> descending s = sqrt(max(w,0)),
// Uhat (r x r, FP32 column-major of reversed columns), sinv
__global__ void k_eig_post(const double* __restrict__ w, const double* __restrict__ V, int r, double* __restrict__ s,
                           float* __restrict__ Uh, float* __restrict__ sinv) {
    for (int idx = threadIdx.x + blockIdx.x * blockDim.x; idx < r * r; idx += blockDim.x * gridDim.x) {
        const int c = idx / r, i = idx - c * r;       // column c of Uhat = column r-1-c of V
        Uh[size_t(c) * r + i] = float(V[size_t(r - 1 - c) * r + i]);
    }
    for (int c = threadIdx.x + blockIdx.x * blockDim.x; c < r; c += blockDim.x * gridDim.x) {
        const double lam = w[r - 1 - c];
        const double sv = lam > 0.0 ? sqrt(lam) : 0.0;
        s[c] = sv;
        sinv[c] = sv > 0.0 ? float(1.0 / sv) : 0.f;
    }
}

// scale columns: X (rows x r row-major) X[:, c] *= f[c]
__global__ void k_scale_cols(float* __restrict__ X, int64_t rows, int r, const float* __restrict__ f) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= rows * r) return;
    X[idx] *= f[idx % r];
}

struct Ws {
    __nv_bfloat16 *Abf, *Atbf, *Ot, *Xt;
    float *Y, *Z, *G, *R, *Uh, *sinv;
    double *Gd, *w, *work;
    int* info;
    int32_t* orow;
    uint32_t* osgn;
    int lwork;
};

}  // namespace

namespace rsk {

// C (M x N, row-major, ldc = N) = A (M x K, K-major bf16) * B (N x K, K-major bf16)^T, FP32 accumulation.
static rsk_status gemm_nt(rsk_handle* h, const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int64_t M,
                          int64_t N, int64_t K, float alpha, cudaStream_t s) {
    Libs& L = g_libs;
    L.blasSetStream(L.bh, s);
    const float beta = 0.f;
    const int pr = prof_begin(h, s, RSK_KERNEL_GEMM);
    int st = L.gemmEx(L.bh, kOpT, kOpN, int(N), int(M), int(K), &alpha, B, kR16BF, int(K), A, kR16BF, int(K), &beta, C,
                      kR32F, int(N), kCompute32F, kGemmDefault);
    prof_end(h, s, pr);
    if (st != 0) return fail(h, RSK_ERR_CUDA, "cublasGemmEx failed (%d)", st);
    return RSK_OK;
}

// X (rows x r, row-major FP32) <- orthonormal basis of range(X): shifted CholeskyQR3.
static rsk_status orth(rsk_handle* h, float* X, int64_t rows, int r, Ws& w, cudaStream_t s) {
    Libs& L = g_libs;
    L.blasSetStream(L.bh, s);
    const float one = 1.f, zero = 0.f;
    const size_t smem = size_t(r) * (r + 1) / 2 * 4;
    if (smem > 227 * 1024) return fail(h, RSK_ERR_UNSUPPORTED, "r = %d too large for the shared-memory Cholesky", r);
    RSK_CUDA_TRY(h, cudaFuncSetAttribute(k_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    for (int round = 0; round < 3; ++round) {
        // G = X^T X: X row-major = column-major X^T (r x rows)
        int st = L.ssyrk(L.bh, kFillLower, kOpN, r, int(rows), &one, X, r, &zero, w.G, r);
        if (st != 0) return fail(h, RSK_ERR_CUDA, "cublasSsyrk failed (%d)", st);
        const int pr = prof_begin(h, s, RSK_KERNEL_DENSE);
        k_cholesky<<<1, 1024, smem, s>>>(w.G, r, w.R, round == 0 ? 1 : 0, double(rows), h->dev_status);
        prof_end(h, s, pr);
        RSK_LAUNCH_CHECK(h);
        // X <- X R^{-1}:  (X R^{-1})^T = R^{-T} X^T, i.e. solve R^T Y = X^T with R upper (column-major)
        st = L.strsm(L.bh, kSideLeft, kFillUpper, kOpT, kDiagNonUnit, r, int(rows), &one, w.R, r, X, r);
        if (st != 0) return fail(h, RSK_ERR_CUDA, "cublasStrsm failed (%d)", st);
    }
    return RSK_OK;
}

}  // namespace rsk

extern "C" rsk_status rsk_rsvd(rsk_handle* h, const float* A, int64_t m, int64_t n, int64_t lda, int32_t r,
                               int32_t power_iters, int32_t zeta, uint64_t seed, float* U, double* s, float* Vt,
                               cudaStream_t stream) {
    using namespace rsk;
    if (!h) return RSK_ERR_INVALID_ARG;
    if (!A || !U || !s || !Vt) return fail(h, RSK_ERR_INVALID_ARG, "null pointer");
    if (m < 1 || n < 1 || lda < n || r < 1 || r > 380 || r > std::min(m, n) || power_iters < 0)
        return fail(h, RSK_ERR_INVALID_ARG, "need 1 <= r <= min(m, n, 380), lda >= n, power_iters >= 0");
    if (zeta < 1 || zeta > r || zeta > 32) return fail(h, RSK_ERR_INVALID_ARG, "need 1 <= zeta <= min(r, 32)");
    if (m >= (int64_t(1) << 31) || n >= (int64_t(1) << 31)) return fail(h, RSK_ERR_INVALID_ARG, "m, n < 2^31");
    rsk_status st = load_libs(h);
    if (st != RSK_OK) return st;
    Libs& L = g_libs;
    L.solverSetStream(L.sh, stream);
    int lwork = 0;
    if (L.dsyevdBuf(L.sh, kEigModeVector, kFillLower, r, nullptr, r, nullptr, &lwork) != 0)
        return fail(h, RSK_ERR_CUDA, "cusolverDnDsyevd_bufferSize failed");

    size_t bytes = 0;
    auto add = [&](size_t b_) { bytes += Carver::round(b_); };
    add(size_t(m) * n * 2);      // A bf16
    add(size_t(m) * n * 2);      // A^T bf16
    add(size_t(r) * n * 2);      // Omega^T
    add(size_t(r) * std::max(m, n) * 2);  // X^T bf16
    add(size_t(std::max(m, n)) * r * 4);      // Y (also the n x r scratch of the final step)
    add(size_t(n) * r * 4);      // Z
    add(size_t(r) * r * 4 * 3);  // G, R, Uh
    add(size_t(r) * 4);          // sinv
    add(size_t(r) * r * 8 + size_t(r) * 8 + size_t(lwork) * 8 + 64);
    add(size_t(n) * zeta * 4 + size_t(n) * 4);
    st = ensure_workspace(h, bytes + 4096, stream);
    if (st != RSK_OK) return st;
    Carver cv(h->ws);
    Ws w;
    w.Abf = cv.take<__nv_bfloat16>(size_t(m) * n);
    w.Atbf = cv.take<__nv_bfloat16>(size_t(m) * n);
    w.Ot = cv.take<__nv_bfloat16>(size_t(r) * n);
    w.Xt = cv.take<__nv_bfloat16>(size_t(r) * std::max(m, n));
    w.Y = cv.take<float>(size_t(std::max(m, n)) * r);
    w.Z = cv.take<float>(size_t(n) * r);
    w.G = cv.take<float>(size_t(r) * r);
    w.R = cv.take<float>(size_t(r) * r);
    w.Uh = cv.take<float>(size_t(r) * r);
    w.sinv = cv.take<float>(size_t(r));
    w.Gd = cv.take<double>(size_t(r) * r);
    w.w = cv.take<double>(size_t(r));
    w.work = cv.take<double>(size_t(lwork));
    w.info = cv.take<int>(16);
    w.orow = cv.take<int32_t>(size_t(n) * zeta);
    w.osgn = cv.take<uint32_t>(size_t(n));

    // ---- A in BF16, both orientations; Omega^T dense +-1
    const unsigned g1 = unsigned((m * n + 255) / 256);
    k_to_bf16<<<g1, 256, 0, stream>>>(A, m, n, lda, w.Abf);
    k_transpose_bf16<<<dim3(unsigned((n + 31) / 32), unsigned((m + 31) / 32)), dim3(32, 8), 0, stream>>>(A, m, n, lda, w.Atbf);
    RSK_CUDA_TRY(h, cudaMemsetAsync(w.Ot, 0, size_t(r) * n * 2, stream));
    st = sketch_generate(h, n, r, zeta, seed, 3u, w.orow, w.osgn, stream);
    if (st != RSK_OK) return st;
    k_omega_t<<<unsigned((n + 255) / 256), 256, 0, stream>>>(w.orow, w.osgn, n, zeta, w.Ot);
    RSK_LAUNCH_CHECK(h);

    // ---- range finder
    const float zs = float(1.0 / sqrt(double(zeta)));
    st = gemm_nt(h, w.Abf, w.Ot, w.Y, m, r, n, zs, stream);                 // Y = A Omega
    if (st == RSK_OK) st = orth(h, w.Y, m, r, w, stream);
    for (int it = 0; st == RSK_OK && it < power_iters; ++it) {
        k_transpose_f32_bf16<<<dim3(unsigned((r + 31) / 32), unsigned((m + 31) / 32)), dim3(32, 8), 0, stream>>>(w.Y, m, r, w.Xt);
        st = gemm_nt(h, w.Atbf, w.Xt, w.Z, n, r, m, 1.f, stream);          // Z = A^T Q
        if (st == RSK_OK) st = orth(h, w.Z, n, r, w, stream);
        if (st != RSK_OK) break;
        k_transpose_f32_bf16<<<dim3(unsigned((r + 31) / 32), unsigned((n + 31) / 32)), dim3(32, 8), 0, stream>>>(w.Z, n, r, w.Xt);
        st = gemm_nt(h, w.Abf, w.Xt, w.Y, m, r, n, 1.f, stream);          // Y = A Z
        if (st == RSK_OK) st = orth(h, w.Y, m, r, w, stream);
    }
    if (st != RSK_OK) return st;
    // ---- B = Q^T A = Z^T with Z = A^T Q
    k_transpose_f32_bf16<<<dim3(unsigned((r + 31) / 32), unsigned((m + 31) / 32)), dim3(32, 8), 0, stream>>>(w.Y, m, r, w.Xt);
    st = gemm_nt(h, w.Atbf, w.Xt, w.Z, n, r, m, 1.f, stream);
    if (st != RSK_OK) return st;
    // ---- small SVD: Z^T Z = Uhat Sigma^2 Uhat^T
    L.blasSetStream(L.bh, stream);
    const float one = 1.f, zero = 0.f;
    if (L.ssyrk(L.bh, kFillLower, kOpN, r, int(n), &one, w.Z, r, &zero, w.G, r) != 0)
        return fail(h, RSK_ERR_CUDA, "cublasSsyrk failed");
    k_f32_to_f64<<<unsigned((size_t(r) * r + 255) / 256), 256, 0, stream>>>(w.G, w.Gd, int64_t(r) * r);
    RSK_LAUNCH_CHECK(h);
    if (L.dsyevd(L.sh, kEigModeVector, kFillLower, r, w.Gd, r, w.w, w.work, lwork, w.info) != 0)
        return fail(h, RSK_ERR_CUDA, "cusolverDnDsyevd failed");
    k_eig_post<<<8, 256, 0, stream>>>(w.w, w.Gd, r, s, w.Uh, w.sinv);
    RSK_LAUNCH_CHECK(h);
    // U = Q Uhat  (row-major m x r = (Uhat^T Q^T)^T): column-major U^T (r x m) = Uhat^T (r x r) * Q^T (r x m)
    if (L.sgemm(L.bh, kOpT, kOpN, r, int(m), r, &one, w.Uh, r, w.Y, r, &zero, U, r) != 0)
        return fail(h, RSK_ERR_CUDA, "cublasSgemm (U) failed");
    // Vt = Sigma^{-1} Uhat^T Z^T: row-major Vt (r x n) is column-major Vt^T (n x r) = Z Uhat Sigma^{-1};
    // first W = Z Uhat (row-major n x r) = column-major (Uhat^T Z^T) r x n
    if (L.sgemm(L.bh, kOpT, kOpN, r, int(n), r, &one, w.Uh, r, w.Z, r, &zero, w.Y, r) != 0)
        return fail(h, RSK_ERR_CUDA, "cublasSgemm (V) failed");
    k_scale_cols<<<unsigned((int64_t(n) * r + 255) / 256), 256, 0, stream>>>(w.Y, n, r, w.sinv);
    // Vt (r x n row-major) = W^T
    k_transpose_f32<<<dim3(unsigned((r + 31) / 32), unsigned((n + 31) / 32)), dim3(32, 8), 0, stream>>>(w.Y, n, r, Vt);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}
