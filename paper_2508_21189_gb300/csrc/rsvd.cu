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
// The plain products (the BF16 GEMMs, the FP32 Gram matrices and the FP32 products X R^{-1}) go
// through cuBLASLt matmuls, each shape autotuned once (the heuristic's candidates timed on the
// operands, the fastest kept; the FP32 ones use cuBLAS's FP32 emulation on the BF16 tensor cores
// when it is offered); R^{-1} comes from this file's Cholesky kernel, so no triangular solve
// runs on the tall basis.  The r x r eigenproblem goes through cuSOLVER.  Both libraries are loaded at
// first use with dlopen; everything else is this file's kernels.
#include <cublasLt.h>
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

// cuBLASLt: function pointers (types from cublasLt.h), one handle, autotuned plans per shape.
struct LtLib {
    void* so = nullptr;
    decltype(&cublasLtCreate) create = nullptr;
    decltype(&cublasLtMatmulDescCreate) descCreate = nullptr;
    decltype(&cublasLtMatmulDescSetAttribute) descSet = nullptr;
    decltype(&cublasLtMatrixLayoutCreate) layoutCreate = nullptr;
    decltype(&cublasLtMatmulPreferenceCreate) prefCreate = nullptr;
    decltype(&cublasLtMatmulPreferenceSetAttribute) prefSet = nullptr;
    decltype(&cublasLtMatmulPreferenceDestroy) prefDestroy = nullptr;
    decltype(&cublasLtMatmulAlgoGetHeuristic) heuristic = nullptr;
    decltype(&cublasLtMatmul) matmul = nullptr;
    decltype(&cublasLtMatmulDescDestroy) descDestroy = nullptr;
    decltype(&cublasLtMatrixLayoutDestroy) layoutDestroy = nullptr;
    cublasLtHandle_t lh = nullptr;
};
LtLib g_lt;

struct LtPlan {
    int device, ta, tb, atype, ctype, compute;
    int64_t m, n, k, lda, ldb, ldc;
    cublasLtMatmulDesc_t desc;
    cublasLtMatrixLayout_t la, lb, lc;
    cublasLtMatmulAlgo_t algo;
    size_t ws;
};
std::vector<LtPlan> g_plans;
constexpr size_t kLtWorkspace = size_t(64) << 20;

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
    LtLib& T = g_lt;
    T.so = dlopen("libcublasLt.so.13", RTLD_NOW | RTLD_LOCAL);
    if (!T.so) T.so = dlopen("libcublasLt.so", RTLD_NOW | RTLD_LOCAL);
    if (!T.so) return rsk::fail(h, RSK_ERR_UNSUPPORTED, "cuBLASLt not found");
    ok = sym(T.so, "cublasLtCreate", T.create) && sym(T.so, "cublasLtMatmulDescCreate", T.descCreate) &&
         sym(T.so, "cublasLtMatmulDescSetAttribute", T.descSet) &&
         sym(T.so, "cublasLtMatrixLayoutCreate", T.layoutCreate) &&
         sym(T.so, "cublasLtMatmulPreferenceCreate", T.prefCreate) &&
         sym(T.so, "cublasLtMatmulPreferenceSetAttribute", T.prefSet) &&
         sym(T.so, "cublasLtMatmulPreferenceDestroy", T.prefDestroy) &&
         sym(T.so, "cublasLtMatmulAlgoGetHeuristic", T.heuristic) && sym(T.so, "cublasLtMatmul", T.matmul) &&
         sym(T.so, "cublasLtMatmulDescDestroy", T.descDestroy) &&
         sym(T.so, "cublasLtMatrixLayoutDestroy", T.layoutDestroy);
    if (!ok || T.create(&T.lh) != CUBLAS_STATUS_SUCCESS)
        return rsk::fail(h, RSK_ERR_UNSUPPORTED, "cuBLASLt symbols missing or handle creation failed");
    L.ok = true;
    return RSK_OK;
}

// D (m x n, column-major, ldc) = alpha op(A) op(B), op given by ta / tb (0 = N, 1 = T), through the
// fastest of cuBLASLt's heuristic candidates for this shape (timed on first use with these operands).
rsk_status lt_matmul(rsk_handle* h, int ta, int tb, int64_t m, int64_t n, int64_t k, const void* A, cudaDataType_t at,
                     int64_t lda, const void* B, int64_t ldb, void* C, cudaDataType_t ct, int64_t ldc, float alpha,
                     cublasComputeType_t compute, void* ws, cudaStream_t stream) {
    LtLib& T = g_lt;
    const float beta = 0.f;
    LtPlan* plan = nullptr;
    for (auto& p : g_plans)
        if (p.device == h->device && p.ta == ta && p.tb == tb && p.atype == int(at) && p.ctype == int(ct) &&
            p.compute == int(compute) && p.m == m && p.n == n && p.k == k && p.lda == lda && p.ldb == ldb &&
            p.ldc == ldc)
            plan = &p;
    if (!plan) {
        LtPlan p{};
        p.device = h->device;
        p.ta = ta;
        p.tb = tb;
        p.atype = int(at);
        p.ctype = int(ct);
        p.compute = int(compute);
        p.m = m;
        p.n = n;
        p.k = k;
        p.lda = lda;
        p.ldb = ldb;
        p.ldc = ldc;
        if (T.descCreate(&p.desc, compute, CUDA_R_32F) != CUBLAS_STATUS_SUCCESS)
            return rsk::fail(h, RSK_ERR_CUDA, "cublasLtMatmulDescCreate failed");
        const cublasOperation_t opa = ta ? CUBLAS_OP_T : CUBLAS_OP_N, opb = tb ? CUBLAS_OP_T : CUBLAS_OP_N;
        T.descSet(p.desc, CUBLASLT_MATMUL_DESC_TRANSA, &opa, sizeof(opa));
        T.descSet(p.desc, CUBLASLT_MATMUL_DESC_TRANSB, &opb, sizeof(opb));
        if (T.layoutCreate(&p.la, at, ta ? k : m, ta ? m : k, lda) != CUBLAS_STATUS_SUCCESS ||
            T.layoutCreate(&p.lb, at, tb ? n : k, tb ? k : n, ldb) != CUBLAS_STATUS_SUCCESS ||
            T.layoutCreate(&p.lc, ct, m, n, ldc) != CUBLAS_STATUS_SUCCESS)
            return rsk::fail(h, RSK_ERR_CUDA, "cublasLtMatrixLayoutCreate failed");
        cublasLtMatmulPreference_t pref;
        T.prefCreate(&pref);
        const uint64_t wsb = kLtWorkspace;
        T.prefSet(pref, CUBLASLT_MATMUL_PREF_MAX_WORKSPACE_BYTES, &wsb, sizeof(wsb));
        cublasLtMatmulHeuristicResult_t cand[16];
        int found = 0;
        const cublasStatus_t hs = T.heuristic(T.lh, p.desc, p.la, p.lb, p.lc, p.lc, pref, 16, cand, &found);
        T.prefDestroy(pref);
        if (hs != CUBLAS_STATUS_SUCCESS || found < 1) return rsk::fail(h, RSK_ERR_UNSUPPORTED, "no cuBLASLt algorithm");
        cudaEvent_t e0, e1;
        RSK_CUDA_TRY(h, cudaEventCreate(&e0));
        RSK_CUDA_TRY(h, cudaEventCreate(&e1));
        float best = 1e30f;
        int bi = -1;
        for (int i = 0; i < found; ++i) {
            if (cand[i].state != CUBLAS_STATUS_SUCCESS || cand[i].workspaceSize > kLtWorkspace) continue;
            if (T.matmul(T.lh, p.desc, &alpha, A, p.la, B, p.lb, &beta, C, p.lc, C, p.lc, &cand[i].algo, ws,
                         kLtWorkspace, stream) != CUBLAS_STATUS_SUCCESS)
                continue;
            cudaEventRecord(e0, stream);
            for (int rep = 0; rep < 2; ++rep)
                T.matmul(T.lh, p.desc, &alpha, A, p.la, B, p.lb, &beta, C, p.lc, C, p.lc, &cand[i].algo, ws,
                         kLtWorkspace, stream);
            cudaEventRecord(e1, stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bi = i;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaGetLastError();
        if (bi < 0) return rsk::fail(h, RSK_ERR_UNSUPPORTED, "no cuBLASLt algorithm ran");
        p.algo = cand[bi].algo;
        p.ws = cand[bi].workspaceSize;
        g_plans.push_back(p);
        plan = &g_plans.back();
    }
    if (T.matmul(T.lh, plan->desc, &alpha, A, plan->la, B, plan->lb, &beta, C, plan->lc, C, plan->lc, &plan->algo, ws,
                 kLtWorkspace, stream) != CUBLAS_STATUS_SUCCESS)
        return rsk::fail(h, RSK_ERR_CUDA, "cublasLtMatmul failed");
    return RSK_OK;
}

// ------------------------------------------------------------------------------------------
// Kernels.
// ------------------------------------------------------------------------------------------
// B (m x n, packed) = bf16(A) (lda); grid (ceil(n / 1024), <= 65535) striding over rows, 4
// consecutive elements per thread.
__global__ void k_to_bf16(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda, __nv_bfloat16* __restrict__ B) {
    const int64_t j = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) * 4;
    if (j >= n) return;
    for (int64_t i = blockIdx.y; i < m; i += gridDim.y) {
        const float* a = A + i * lda + j;
        __nv_bfloat16* b = B + i * n + j;
        if (j + 4 <= n && (reinterpret_cast<uintptr_t>(a) & 15) == 0 && (reinterpret_cast<uintptr_t>(b) & 7) == 0) {
            const float4 v = *reinterpret_cast<const float4*>(a);
            __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
            uint2 o;
            o.x = *reinterpret_cast<uint32_t*>(&lo);
            o.y = *reinterpret_cast<uint32_t*>(&hi);
            *reinterpret_cast<uint2*>(b) = o;
        } else {
            for (int e = 0; e < 4 && j + e < n; ++e) b[e] = __float2bfloat16_rn(a[e]);
        }
    }
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

// X (rows x r, FP32, row-major, row stride ldx) -> bf16(X^T) (rp x rows; rows r..rp-1 zero)
__global__ void k_transpose_f32_bf16(const float* __restrict__ X, int64_t rows, int r, int ldx, int rp,
                                     __nv_bfloat16* __restrict__ T) {
    __shared__ float tile[32][33];
    const int64_t i0 = int64_t(blockIdx.y) * 32;
    const int j0 = blockIdx.x * 32;
    for (int rr = threadIdx.y; rr < 32; rr += blockDim.y) {
        const int64_t i = i0 + rr;
        const int j = j0 + threadIdx.x;
        tile[rr][threadIdx.x] = (i < rows && j < r) ? X[i * ldx + j] : 0.f;
    }
    __syncthreads();
    for (int rr = threadIdx.y; rr < 32; rr += blockDim.y) {
        const int j = j0 + rr;
        const int64_t i = i0 + threadIdx.x;
        if (j < rp && i < rows) T[int64_t(j) * rows + i] = __float2bfloat16_rn(tile[threadIdx.x][rr]);
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

constexpr int kMaxRank = 320;  // the tiled factor (55 tiles of 4 KB) within 227 KB of shared memory

// Cholesky of G (+ shift) in shared memory, FP32, blocked by 32.  G: r x r symmetric, read from its
// lower triangle (column-major, G[k*ld + i], i >= k).  The lower triangle is held as nt(nt+1)/2
// tiles of 32 x 32 (nt = ceil(r/32)), element (i, j) of a tile at i*32 + (j ^ i) so that reading a
// tile row or a tile column is free of bank conflicts; rows and columns beyond r are padded with the
// identity.  Per block column kb: one warp factors the diagonal tile, one thread per panel row solves
// the panel against it, one warp per trailing tile subtracts P_i P_j^T.  Writes L (lower,
// column-major, ld x ld, zeros above and in the padding) with G + shift = L L^T, and the identity
// into Linv for the triangular solve that turns it into L^{-1}; the orthonormalised basis is
// X R^{-1} with R = L^T, i.e. (X R^{-1})^T = L^{-1} X^T.  shift_mode 1 adds
// 11 (rows*r + r(r+1)) u_32 trace(G) to the diagonal (the shift of shifted CholeskyQR).
constexpr int kCholThreads = 512;
__device__ __forceinline__ int chol_tile(int bi, int bj) { return (bi * (bi + 1) / 2 + bj) * 1024; }
__device__ __forceinline__ int chol_el(int i, int j) { return i * 32 + (j ^ i); }

__global__ void __launch_bounds__(kCholThreads) k_cholesky(const float* __restrict__ G, int r, int ld,
                                                           float* __restrict__ Lout, float* __restrict__ Linv,
                                                           int shift_mode, double rows, unsigned int* status) {
    extern __shared__ float T[];
    __shared__ double tr;
    const int nt = (r + 31) >> 5;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = kCholThreads / 32;
    if (tid == 0) {
        double t = 0.0;
        for (int i = 0; i < r; ++i) t += double(G[size_t(i) * ld + i]);
        tr = t;
    }
    __syncthreads();
    const float shift = shift_mode ? float(11.0 * (rows * r + double(r) * (r + 1)) * 5.960464477539063e-08 * tr) : 0.f;
    const int ntiles = nt * (nt + 1) / 2;
    for (int e = tid; e < ntiles * 1024; e += kCholThreads) {
        // tile index -> (bi, bj)
        const int t = e >> 10, within = e & 1023;
        int bi = 0;
        while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
        const int bj = t - bi * (bi + 1) / 2;
        const int i = within & 31, j = within >> 5;  // consecutive threads read consecutive rows of G
        const int R = bi * 32 + i, Cc = bj * 32 + j;
        float v;
        if (R >= r || Cc >= r) v = (R == Cc) ? 1.f : 0.f;
        else if (R >= Cc) v = G[size_t(Cc) * ld + R] + (R == Cc ? shift : 0.f);
        else v = 0.f;  // above the diagonal inside a diagonal tile: unused
        T[chol_tile(bi, bj) + chol_el(i, j)] = v;
    }
    __syncthreads();
    for (int kb = 0; kb < nt; ++kb) {
        float* D = T + chol_tile(kb, kb);
        // (a) diagonal tile, one warp (lane = row)
        if (warp == 0) {
            for (int j = 0; j < 32; ++j) {
                if (lane == j) {
                    const float djj = D[chol_el(j, j)];
                    if (!(djj > 0.f) && kb * 32 + j < r) atomicOr(status, RSK_DEV_BOUNDS);
                    D[chol_el(j, j)] = sqrtf(fmaxf(djj, 1e-30f));
                }
                __syncwarp();
                const float piv = D[chol_el(j, j)];
                if (lane > j) D[chol_el(lane, j)] /= piv;
                __syncwarp();
                if (lane > j) {
                    const float lij = D[chol_el(lane, j)];
                    for (int k = j + 1; k <= lane; ++k) D[chol_el(lane, k)] -= lij * D[chol_el(k, j)];
                }
                __syncwarp();
            }
        }
        __syncthreads();
        // (b) panel: every row of tiles (bi, kb), bi > kb, solves x D^T = a by forward substitution
        const int prow = (nt - kb - 1) * 32;
        for (int pr = tid; pr < prow; pr += kCholThreads) {
            const int bi = kb + 1 + (pr >> 5), i = pr & 31;
            float* P = T + chol_tile(bi, kb);
            float x[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                float a = P[chol_el(i, j)];
#pragma unroll
                for (int t = 0; t < j; ++t) a -= x[t] * D[chol_el(j, t)];
                x[j] = a / D[chol_el(j, j)];
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) P[chol_el(i, j)] = x[j];
        }
        __syncthreads();
        // (c) trailing tiles (bi, bj), kb < bj <= bi: T -= P_bi P_bj^T, one warp per tile, lane = row
        const int m = nt - kb - 1;
        const int ntr = m * (m + 1) / 2;
        for (int tt = warp; tt < ntr; tt += nw) {
            int a = 0;
            while ((a + 1) * (a + 2) / 2 <= tt) ++a;
            const int bi = kb + 1 + a, bj = kb + 1 + (tt - a * (a + 1) / 2);
            const float* Pi = T + chol_tile(bi, kb);
            const float* Pj = T + chol_tile(bj, kb);
            float acc[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] = 0.f;
            for (int t = 0; t < 32; ++t) {
                const float p = Pi[chol_el(lane, t)];
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[j] = fmaf(p, Pj[chol_el(j, t)], acc[j]);
            }
            float* Tij = T + chol_tile(bi, bj);
#pragma unroll
            for (int j = 0; j < 32; ++j) Tij[chol_el(lane, j)] -= acc[j];
        }
        __syncthreads();
    }
    // ld x ld outputs; rows and columns beyond r are zero (padding of the GEMM dimensions)
    for (int idx = tid; idx < ld * ld; idx += kCholThreads) {
        const int c = idx / ld, i = idx - c * ld;
        float v = 0.f;
        if (i >= c && i < r && c < r) v = T[chol_tile(i >> 5, c >> 5) + chol_el(i & 31, c & 31)];
        Lout[idx] = v;
        Linv[idx] = (i == c && i < r) ? 1.f : 0.f;
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
    float *Y, *Z, *X2, *G, *R, *Lf, *Uh, *sinv;
    void* ltws;
    double *Gd, *w, *work;
    int* info;
    int32_t* orow;
    uint32_t* osgn;
    int lwork;
};

}  // namespace

namespace rsk {

// FP32 products of the orthonormalisation: cuBLAS's FP32 emulation on the BF16 tensor cores (each
// FP32 operand split into three BF16 parts, FP32 accumulation) where the library offers it, else
// plain FP32.  Decided once per process by a probe matmul.
static cublasComputeType_t fp32_compute(rsk_handle* h) {
    static int mode = -1;  // 1 emulated, 0 plain
    if (mode < 0) {
        LtLib& T = g_lt;
        cublasLtMatmulDesc_t d;
        mode = 0;
        if (T.descCreate(&d, CUBLAS_COMPUTE_32F_EMULATED_16BFX9, CUDA_R_32F) == CUBLAS_STATUS_SUCCESS) {
            cublasLtMatrixLayout_t l;
            if (T.layoutCreate(&l, CUDA_R_32F, 256, 256, 256) == CUBLAS_STATUS_SUCCESS) {
                cublasLtMatmulPreference_t pref;
                T.prefCreate(&pref);
                const uint64_t wsb = kLtWorkspace;
                T.prefSet(pref, CUBLASLT_MATMUL_PREF_MAX_WORKSPACE_BYTES, &wsb, sizeof(wsb));
                cublasLtMatmulHeuristicResult_t c[1];
                int found = 0;
                if (T.heuristic(T.lh, d, l, l, l, l, pref, 1, c, &found) == CUBLAS_STATUS_SUCCESS && found > 0) mode = 1;
                T.prefDestroy(pref);
                T.layoutDestroy(l);
            }
            T.descDestroy(d);
        }
        (void)h;
    }
    return mode == 1 ? CUBLAS_COMPUTE_32F_EMULATED_16BFX9 : CUBLAS_COMPUTE_32F;
}

// C (M x N, row-major, ldc = N) = alpha A (M x K, K-major bf16) * B (N x K, K-major bf16)^T, FP32
// accumulation on the tensor cores.  In column-major terms C^T (N x M) = B^T A.
static rsk_status gemm_nt(rsk_handle* h, const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int64_t M,
                          int64_t N, int64_t K, float alpha, Ws& w, cudaStream_t s) {
    const int pr = prof_begin(h, s, RSK_KERNEL_GEMM);
    const rsk_status st = lt_matmul(h, 1, 0, N, M, K, B, CUDA_R_16BF, K, A, K, C, CUDA_R_32F, N, alpha,
                                    CUBLAS_COMPUTE_32F, w.ltws, s);
    prof_end(h, s, pr);
    return st;
}

// X (rows x r, row-major FP32, row stride rp, columns r..rp-1 zero) <- orthonormal basis of
// range(X): shifted CholeskyQR3.  Each round: G = X^T X (FP32 matmul, rp x rp), G + shift = L L^T on
// the leading r x r block and L^{-1} by a triangular solve (both padded with zeros to rp x rp),
// X <- X L^{-T} computed as (X L^{-T})^T = L^{-1} X^T (FP32 matmul into a second buffer, copied
// back; the zero padding keeps columns r..rp-1 of X zero).  The dimensions are padded to rp, a
// multiple of 8, because the GEMM library only takes its fast paths for such shapes.
static rsk_status orth(rsk_handle* h, float* X, int64_t rows, int r, int rp, Ws& w, cudaStream_t s) {
    Libs& L = g_libs;
    const int nt = (r + 31) / 32;
    const size_t smem = size_t(nt) * (nt + 1) / 2 * 1024 * 4;
    if (smem > 227 * 1024) return fail(h, RSK_ERR_UNSUPPORTED, "r = %d too large for the shared-memory Cholesky", r);
    RSK_CUDA_TRY(h, cudaFuncSetAttribute(k_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    for (int round = 0; round < 3; ++round) {
        // X row-major is X^T column-major (rp x rows, ld rp):  G = X^T (X^T)^T
        int pr = prof_begin(h, s, RSK_KERNEL_DENSE);
        rsk_status st = lt_matmul(h, 0, 1, rp, rp, rows, X, CUDA_R_32F, rp, X, rp, w.G, CUDA_R_32F, rp, 1.f,
                                  fp32_compute(h), w.ltws, s);
        prof_end(h, s, pr);
        if (st != RSK_OK) return st;
        pr = prof_begin(h, s, RSK_KERNEL_DENSE);
        k_cholesky<<<1, kCholThreads, smem, s>>>(w.G, r, rp, w.Lf, w.R, round == 0 ? 1 : 0, double(rows),
                                                  h->dev_status);
        prof_end(h, s, pr);
        RSK_LAUNCH_CHECK(h);
        // w.R <- L^{-1} on the leading r x r block: solve L X = I (lower, column-major, ld rp)
        const float one = 1.f;
        L.blasSetStream(L.bh, s);
        if (L.strsm(L.bh, kSideLeft, kFillLower, kOpN, kDiagNonUnit, r, r, &one, w.Lf, rp, w.R, rp) != 0)
            return fail(h, RSK_ERR_CUDA, "cublasStrsm failed");
        pr = prof_begin(h, s, RSK_KERNEL_DENSE);
        st = lt_matmul(h, 0, 0, rp, rows, rp, w.R, CUDA_R_32F, rp, X, rp, w.X2, CUDA_R_32F, rp, 1.f, fp32_compute(h),
                       w.ltws, s);
        prof_end(h, s, pr);
        if (st != RSK_OK) return st;
        RSK_CUDA_TRY(h, cudaMemcpyAsync(X, w.X2, size_t(rows) * rp * 4, cudaMemcpyDeviceToDevice, s));
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
    if (m < 1 || n < 1 || lda < n || r < 1 || r > kMaxRank || r > std::min(m, n) || power_iters < 0)
        return fail(h, RSK_ERR_INVALID_ARG, "need 1 <= r <= min(m, n, %d), lda >= n, power_iters >= 0", kMaxRank);
    if (zeta < 1 || zeta > r || zeta > 32) return fail(h, RSK_ERR_INVALID_ARG, "need 1 <= zeta <= min(r, 32)");
    if (m >= (int64_t(1) << 31) || n >= (int64_t(1) << 31)) return fail(h, RSK_ERR_INVALID_ARG, "m, n < 2^31");
    rsk_status st = load_libs(h);
    if (st != RSK_OK) return st;
    Libs& L = g_libs;
    L.solverSetStream(L.sh, stream);
    int lwork = 0;
    if (L.dsyevdBuf(L.sh, kEigModeVector, kFillLower, r, nullptr, r, nullptr, &lwork) != 0)
        return fail(h, RSK_ERR_CUDA, "cusolverDnDsyevd_bufferSize failed");

    const int rp = (r + 7) & ~7;  // GEMM dimension padded to a multiple of 8 (zero columns)
    size_t bytes = 0;
    auto add = [&](size_t b_) { bytes += Carver::round(b_); };
    add(size_t(m) * n * 2);      // A bf16
    add(size_t(m) * n * 2);      // A^T bf16
    add(size_t(rp) * n * 2);     // Omega^T
    add(size_t(rp) * std::max(m, n) * 2);  // X^T bf16
    add(size_t(std::max(m, n)) * rp * 4);  // Y (also the n x r scratch of the final step)
    add(size_t(n) * rp * 4);     // Z
    add(size_t(std::max(m, n)) * rp * 4);  // X2 (second buffer of orth)
    add(kLtWorkspace);           // cuBLASLt workspace
    add(size_t(rp) * rp * 4 * 4);  // G, R (L^{-1}), L, Uh
    add(size_t(r) * 4);          // sinv
    add(size_t(r) * r * 8 + size_t(r) * 8 + size_t(lwork) * 8 + 64);
    add(size_t(n) * zeta * 4 + size_t(n) * 4);
    st = ensure_workspace(h, bytes + 4096, stream);
    if (st != RSK_OK) return st;
    Carver cv(h->ws);
    Ws w;
    w.Abf = cv.take<__nv_bfloat16>(size_t(m) * n);
    w.Atbf = cv.take<__nv_bfloat16>(size_t(m) * n);
    w.Ot = cv.take<__nv_bfloat16>(size_t(rp) * n);
    w.Xt = cv.take<__nv_bfloat16>(size_t(rp) * std::max(m, n));
    w.Y = cv.take<float>(size_t(std::max(m, n)) * rp);
    w.Z = cv.take<float>(size_t(n) * rp);
    w.X2 = cv.take<float>(size_t(std::max(m, n)) * rp);
    w.ltws = cv.take<char>(kLtWorkspace);
    w.G = cv.take<float>(size_t(rp) * rp);
    w.R = cv.take<float>(size_t(rp) * rp);
    w.Lf = cv.take<float>(size_t(rp) * rp);
    w.Uh = cv.take<float>(size_t(rp) * rp);
    w.sinv = cv.take<float>(size_t(r));
    w.Gd = cv.take<double>(size_t(r) * r);
    w.w = cv.take<double>(size_t(r));
    w.work = cv.take<double>(size_t(lwork));
    w.info = cv.take<int>(16);
    w.orow = cv.take<int32_t>(size_t(n) * zeta);
    w.osgn = cv.take<uint32_t>(size_t(n));

    // ---- A in BF16, both orientations; Omega^T dense +-1 (rows r..rp-1 zero)
    k_to_bf16<<<dim3(unsigned((n + 1023) / 1024), unsigned(std::min<int64_t>(m, 65535))), 256, 0, stream>>>(
        A, m, n, lda, w.Abf);
    k_transpose_bf16<<<dim3(unsigned((n + 31) / 32), unsigned((m + 31) / 32)), dim3(32, 8), 0, stream>>>(A, m, n, lda, w.Atbf);
    RSK_CUDA_TRY(h, cudaMemsetAsync(w.Ot, 0, size_t(rp) * n * 2, stream));
    st = sketch_generate(h, n, r, zeta, seed, 3u, w.orow, w.osgn, stream);
    if (st != RSK_OK) return st;
    k_omega_t<<<unsigned((n + 255) / 256), 256, 0, stream>>>(w.orow, w.osgn, n, zeta, w.Ot);
    RSK_LAUNCH_CHECK(h);

    // ---- range finder (every product has rp columns; columns r..rp-1 stay zero)
    const float zs = float(1.0 / sqrt(double(zeta)));
    const unsigned tx = unsigned((rp + 31) / 32);
    st = gemm_nt(h, w.Abf, w.Ot, w.Y, m, rp, n, zs, w, stream);                // Y = A Omega
    if (st == RSK_OK) st = orth(h, w.Y, m, r, rp, w, stream);
    for (int it = 0; st == RSK_OK && it < power_iters; ++it) {
        k_transpose_f32_bf16<<<dim3(tx, unsigned((m + 31) / 32)), dim3(32, 8), 0, stream>>>(w.Y, m, r, rp, rp, w.Xt);
        st = gemm_nt(h, w.Atbf, w.Xt, w.Z, n, rp, m, 1.f, w, stream);         // Z = A^T Q
        if (st == RSK_OK) st = orth(h, w.Z, n, r, rp, w, stream);
        if (st != RSK_OK) break;
        k_transpose_f32_bf16<<<dim3(tx, unsigned((n + 31) / 32)), dim3(32, 8), 0, stream>>>(w.Z, n, r, rp, rp, w.Xt);
        st = gemm_nt(h, w.Abf, w.Xt, w.Y, m, rp, n, 1.f, w, stream);         // Y = A Z
        if (st == RSK_OK) st = orth(h, w.Y, m, r, rp, w, stream);
    }
    if (st != RSK_OK) return st;
    // ---- B = Q^T A = Z^T with Z = A^T Q
    k_transpose_f32_bf16<<<dim3(tx, unsigned((m + 31) / 32)), dim3(32, 8), 0, stream>>>(w.Y, m, r, rp, rp, w.Xt);
    st = gemm_nt(h, w.Atbf, w.Xt, w.Z, n, rp, m, 1.f, w, stream);
    if (st != RSK_OK) return st;
    // ---- small SVD: Z^T Z = Uhat Sigma^2 Uhat^T
    L.blasSetStream(L.bh, stream);
    const float one = 1.f, zero = 0.f;
    if (L.ssyrk(L.bh, kFillLower, kOpN, r, int(n), &one, w.Z, rp, &zero, w.G, r) != 0)
        return fail(h, RSK_ERR_CUDA, "cublasSsyrk failed");
    k_f32_to_f64<<<unsigned((size_t(r) * r + 255) / 256), 256, 0, stream>>>(w.G, w.Gd, int64_t(r) * r);
    RSK_LAUNCH_CHECK(h);
    if (L.dsyevd(L.sh, kEigModeVector, kFillLower, r, w.Gd, r, w.w, w.work, lwork, w.info) != 0)
        return fail(h, RSK_ERR_CUDA, "cusolverDnDsyevd failed");
    k_eig_post<<<8, 256, 0, stream>>>(w.w, w.Gd, r, s, w.Uh, w.sinv);
    RSK_LAUNCH_CHECK(h);
    // U = Q Uhat  (row-major m x r = (Uhat^T Q^T)^T): column-major U^T (r x m) = Uhat^T (r x r) * Q^T (r x m)
    if (L.sgemm(L.bh, kOpT, kOpN, r, int(m), r, &one, w.Uh, r, w.Y, rp, &zero, U, r) != 0)
        return fail(h, RSK_ERR_CUDA, "cublasSgemm (U) failed");
    // Vt = Sigma^{-1} Uhat^T Z^T: row-major Vt (r x n) is column-major Vt^T (n x r) = Z Uhat Sigma^{-1};
    // first W = Z Uhat (row-major n x r) = column-major (Uhat^T Z^T) r x n
    if (L.sgemm(L.bh, kOpT, kOpN, r, int(n), r, &one, w.Uh, r, w.Z, rp, &zero, w.Y, r) != 0)
        return fail(h, RSK_ERR_CUDA, "cublasSgemm (V) failed");
    k_scale_cols<<<unsigned((int64_t(n) * r + 255) / 256), 256, 0, stream>>>(w.Y, n, r, w.sinv);
    // Vt (r x n row-major) = W^T
    k_transpose_f32<<<dim3(unsigned((r + 31) / 32), unsigned((n + 31) / 32)), dim3(32, 8), 0, stream>>>(w.Y, n, r, Vt);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}
