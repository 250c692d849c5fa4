// Randomized SVD with a sparse sign test matrix (row a9).
// Paper: Alg. 1 (Sec. 2.1): Y = A Omega, Q = orth(Y), B = Q^T A, [Uhat, Sigma, V] = svd(B),
// U = Q Uhat.  Omega (n x r) is SparseUniform with zeta nonzeros per row (Def. SparseUniform),
// drawn from Philox stream 3 as the left sparse sign S = Omega^T (r rows, n columns).  Alg. 1 has no
// power iterations; q subspace iterations Q = orth(A^T Q), Q = orth(A Q) are applied after the
// sketch (re-orthonormalising after every product).
//
// Precision plan.  A (FP32) is converted once to BF16 in both orientations (A and A^T, one pass
// over A) so that every product is a GEMM with both operands K-major:
//     Y = A Omega      : [m x n] * [r x n]^T      Z = A^T Q : [n x m] * [r x m]^T
// with FP32 accumulation on the tensor cores.  orth() is shifted CholeskyQR3 in FP32 (one shifted
// round, two plain ones): the Gram G = X^T X, a Cholesky of G (+ shift) by cuSOLVER, and
// X <- X R^{-1}; the shift keeps the first Cholesky defined up to kappa(X) ~ u^{-1}, the plain rounds
// restore orthogonality to O(u_32), below the BF16 error of the products.  The small SVD of
// B = Z^T comes from the symmetric eigenproblem of Z^T Z (r x r, FP32: Z^T Z is formed in FP32, so
// an FP64 eigensolver would add no accuracy).
//
// The plain products (the BF16 GEMMs, the FP32 Gram matrices and the FP32 products X R^{-1}) go
// through cuBLASLt matmuls, each shape autotuned once (the heuristic's candidates timed on the
// operands, the fastest kept; the FP32 ones use cuBLAS's FP32 emulation on the BF16 tensor cores
// when it is offered); R^{-1} comes from a triangular solve on the r x r factor, so no triangular
// solve runs on the tall basis.  The r x r Cholesky and eigenproblem go through cuSOLVER.  Both
// libraries are loaded at first use with dlopen; everything else is this file's kernels.
#include <cublasLt.h>
#include <cuda_bf16.h>
#include <dlfcn.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <utility>
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
    int (*ssyevdBuf)(cusolverH, int, int, int, const float*, int, const float*, int*);
    int (*ssyevd)(cusolverH, int, int, int, float*, int, float*, float*, int, int*);
    int (*spotrfBuf)(cusolverH, int, int, float*, int, int*);
    int (*spotrf)(cusolverH, int, int, float*, int, float*, int, int*);
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
    decltype(&cublasLtEmulationDescCreate) emuCreate = nullptr;       // optional
    decltype(&cublasLtEmulationDescSetAttribute) emuSet = nullptr;    // optional
    cublasLtEmulationDesc_t emu = nullptr;  // emulation without special-value handling
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
              sym(L.solver, "cusolverDnSsyevd_bufferSize", L.ssyevdBuf) && sym(L.solver, "cusolverDnSsyevd", L.ssyevd) &&
              sym(L.solver, "cusolverDnSpotrf_bufferSize", L.spotrfBuf) && sym(L.solver, "cusolverDnSpotrf", L.spotrf);
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
    // The FP32 products only ever see finite operands (orthonormalisation intermediates; a failed
    // factorization is reported through the status word), so the emulated matmuls are told not to
    // scan for and patch infinities and NaNs.
    if (ok && sym(T.so, "cublasLtEmulationDescCreate", T.emuCreate) && sym(T.so, "cublasLtEmulationDescSetAttribute", T.emuSet) &&
        T.emuCreate(&T.emu) == CUBLAS_STATUS_SUCCESS) {
        const int32_t none = int32_t(CUDA_EMULATION_SPECIAL_VALUES_SUPPORT_NONE);
        if (T.emuSet(T.emu, CUBLASLT_EMULATION_DESC_SPECIAL_VALUES_SUPPORT, &none, sizeof(none)) != CUBLAS_STATUS_SUCCESS)
            T.emu = nullptr;
    }
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
        if (compute == CUBLAS_COMPUTE_32F_EMULATED_16BFX9 && T.emu)
            T.descSet(p.desc, CUBLASLT_MATMUL_DESC_EMULATION_DESCRIPTOR, &T.emu, sizeof(T.emu));
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
// B = bf16(A) (m x n, packed) and Bt = bf16(A^T) (n x m, packed) in one pass over A: one CTA per
// 64 x 64 tile; the tile is written row-major straight from the loads and column-major through a
// padded shared-memory transpose.  vec: A rows 16-byte aligned (float4 loads) and n % 4 == 0;
// m % 2 == 0 for the paired transposed stores.
constexpr int kCvt = 64;
__global__ void __launch_bounds__(256) k_to_bf16_both(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                                                      int vec, __nv_bfloat16* __restrict__ B,
                                                      __nv_bfloat16* __restrict__ Bt) {
    __shared__ float tT[kCvt][kCvt + 1];  // tT[j][i]
    const int64_t ntj = (n + kCvt - 1) / kCvt;
    const int64_t ti = int64_t(blockIdx.x) / ntj, tj = int64_t(blockIdx.x) - ti * ntj;
    const int64_t i0 = ti * kCvt, j0 = tj * kCvt;
    for (int e = threadIdx.x; e < kCvt * kCvt / 4; e += blockDim.x) {
        const int il = e >> 4, jl = (e & 15) * 4;
        const int64_t i = i0 + il, j = j0 + jl;
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        if (i < m) {
            const float* a = A + i * lda + j;
            if (vec && j + 4 <= n) {
                const float4 f = *reinterpret_cast<const float4*>(a);
                v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
                const __nv_bfloat162 lo = __floats2bfloat162_rn(f.x, f.y), hi = __floats2bfloat162_rn(f.z, f.w);
                uint2 o;
                o.x = *reinterpret_cast<const uint32_t*>(&lo);
                o.y = *reinterpret_cast<const uint32_t*>(&hi);
                *reinterpret_cast<uint2*>(B + i * n + j) = o;
            } else {
                for (int c = 0; c < 4; ++c)
                    if (j + c < n) {
                        v[c] = a[c];
                        B[i * n + j + c] = __float2bfloat16_rn(v[c]);
                    }
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) tT[jl + c][il] = v[c];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kCvt * kCvt / 2; e += blockDim.x) {
        const int jl = e >> 5, il = (e & 31) * 2;
        const int64_t j = j0 + jl, i = i0 + il;
        if (j >= n || i >= m) continue;
        __nv_bfloat16* d = Bt + j * m + i;
        if (vec && i + 2 <= m) {
            const __nv_bfloat162 p = __floats2bfloat162_rn(tT[jl][il], tT[jl][il + 1]);
            *reinterpret_cast<__nv_bfloat162*>(d) = p;
        } else {
            d[0] = __float2bfloat16_rn(tT[jl][il]);
            if (i + 1 < m) d[1] = __float2bfloat16_rn(tT[jl][il + 1]);
        }
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

constexpr int kMaxRank = 320;  // largest rank the workspace plan and the tests cover

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

// eigenvalues ascending (w) and vectors (columns of V, column-major) -> descending s = sqrt(max(w,0)),
// Uhat (r x r, FP32 column-major of reversed columns), sinv
__global__ void k_eig_post(const float* __restrict__ w, const float* __restrict__ V, int r, double* __restrict__ s,
                             float* __restrict__ Uh, float* __restrict__ sinv) {
    for (int idx = threadIdx.x + blockIdx.x * blockDim.x; idx < r * r; idx += blockDim.x * gridDim.x) {
        const int c = idx / r, i = idx - c * r;       // column c of Uhat = column r-1-c of V
        Uh[size_t(c) * r + i] = V[size_t(r - 1 - c) * r + i];
    }
    for (int c = threadIdx.x + blockIdx.x * blockDim.x; c < r; c += blockDim.x * gridDim.x) {
        const double lam = double(w[r - 1 - c]);
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
    float *w, *work;
    int* info;
    float* cwork;
    int clwork;
    int* cinfo;
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

// Lout (ld x ld, column-major) = lower triangle of G + shift I on the leading r x r block, zero
// elsewhere; Linv = I on the leading r x r block, zero elsewhere.  With shift_mode the shift is
// 11 (rows r + r (r + 1)) u trace(G), u = 2^-24 (the shifted CholeskyQR rule).
__global__ void __launch_bounds__(256) k_chol_prep(const float* __restrict__ G, int r, int ld, float* __restrict__ Lout,
                                                   float* __restrict__ Linv, int shift_mode, double rows) {
    // one CTA per column c of the ld x ld outputs; every CTA forms the (same) trace
    __shared__ double part[8];
    const int tid = threadIdx.x, c = blockIdx.x;
    double t = 0.0;
    if (shift_mode)
        for (int i = tid; i < r; i += blockDim.x) t += double(G[size_t(i) * ld + i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((tid & 31) == 0) part[tid >> 5] = t;
    __syncthreads();
    double tr = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) tr += part[w];
    const float shift = shift_mode ? float(11.0 * (rows * r + double(r) * (r + 1)) * 5.960464477539063e-08 * tr) : 0.f;
    for (int i = tid; i < ld; i += blockDim.x) {
        const size_t idx = size_t(c) * ld + i;
        const bool in = i < r && c < r;
        Lout[idx] = (in && i >= c) ? G[idx] + (i == c ? shift : 0.f) : 0.f;
        Linv[idx] = (in && i == c) ? 1.f : 0.f;
    }
}

// A failed factorization (a non-positive pivot) is recorded in the handle's status word.
__global__ void k_chol_check(const int* __restrict__ info, unsigned int* status) {
    if (threadIdx.x == 0 && *info != 0) atomicOr(status, RSK_DEV_BOUNDS);
}

// X (rows x r, row-major FP32, row stride rp, columns r..rp-1 zero) <- orthonormal basis of
// range(X): shifted CholeskyQR3.  Each round: G = X^T X (FP32 matmul, rp x rp), G + shift = L L^T on
// the leading r x r block and L^{-1} by a triangular solve (both padded with zeros to rp x rp),
// X <- X L^{-T} computed as (X L^{-T})^T = L^{-1} X^T (FP32 matmul into a second buffer, copied
// back; the zero padding keeps columns r..rp-1 of X zero).  The dimensions are padded to rp, a
// multiple of 8, because the GEMM library only takes its fast paths for such shapes.
static rsk_status orth(rsk_handle* h, float* X, int64_t rows, int r, int rp, Ws& w, cudaStream_t s) {
    Libs& L = g_libs;
    float* src = X;
    float* dst = w.X2;
    for (int round = 0; round < 3; ++round) {
        // X row-major is X^T column-major (rp x rows, ld rp):  G = X^T (X^T)^T
        int pr = prof_begin(h, s, RSK_KERNEL_DENSE);
        rsk_status st = lt_matmul(h, 0, 1, rp, rp, rows, src, CUDA_R_32F, rp, src, rp, w.G, CUDA_R_32F, rp, 1.f,
                                  fp32_compute(h), w.ltws, s);
        prof_end(h, s, pr);
        if (st != RSK_OK) return st;
        pr = prof_begin(h, s, RSK_KERNEL_DENSE);
        k_chol_prep<<<unsigned(rp), 256, 0, s>>>(w.G, r, rp, w.Lf, w.R, round == 0 ? 1 : 0, double(rows));
        RSK_LAUNCH_CHECK(h);
        if (L.spotrf(L.sh, kFillLower, r, w.Lf, rp, w.cwork, w.clwork, w.cinfo) != 0)
            return fail(h, RSK_ERR_CUDA, "cusolverDnSpotrf failed");
        k_chol_check<<<1, 32, 0, s>>>(w.cinfo, h->dev_status);
        prof_end(h, s, pr);
        RSK_LAUNCH_CHECK(h);
        // w.R <- L^{-1} on the leading r x r block: solve L X = I (lower, column-major, ld rp)
        const float one = 1.f;
        L.blasSetStream(L.bh, s);
        if (L.strsm(L.bh, kSideLeft, kFillLower, kOpN, kDiagNonUnit, r, r, &one, w.Lf, rp, w.R, rp) != 0)
            return fail(h, RSK_ERR_CUDA, "cublasStrsm failed");
        pr = prof_begin(h, s, RSK_KERNEL_DENSE);
        st = lt_matmul(h, 0, 0, rp, rows, rp, w.R, CUDA_R_32F, rp, src, rp, dst, CUDA_R_32F, rp, 1.f, fp32_compute(h),
                       w.ltws, s);
        prof_end(h, s, pr);
        if (st != RSK_OK) return st;
        std::swap(src, dst);
    }
    if (src != X) RSK_CUDA_TRY(h, cudaMemcpyAsync(X, src, size_t(rows) * rp * 4, cudaMemcpyDeviceToDevice, s));
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
    if (L.ssyevdBuf(L.sh, kEigModeVector, kFillLower, r, nullptr, r, nullptr, &lwork) != 0)
        return fail(h, RSK_ERR_CUDA, "cusolverDnSsyevd_bufferSize failed");

    const int rp = (r + 7) & ~7;  // GEMM dimension padded to a multiple of 8 (zero columns)
    int clwork = 0;
    if (L.spotrfBuf(L.sh, kFillLower, r, nullptr, rp, &clwork) != 0)
        return fail(h, RSK_ERR_CUDA, "cusolverDnSpotrf_bufferSize failed");
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
    add(size_t(r) * 4 + size_t(lwork) * 4 + 64);   // eigenvalues, eigensolver work, info
    add(size_t(n) * zeta * 4 + size_t(n) * 4);
    add(size_t(clwork) * 4 + 64);
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
    w.w = cv.take<float>(size_t(r));
    w.work = cv.take<float>(size_t(lwork));
    w.info = cv.take<int>(16);
    w.orow = cv.take<int32_t>(size_t(n) * zeta);
    w.osgn = cv.take<uint32_t>(size_t(n));
    w.cwork = cv.take<float>(size_t(clwork) + 1);
    w.clwork = clwork;
    w.cinfo = cv.take<int>(16);

    // ---- A in BF16, both orientations; Omega^T dense +-1 (rows r..rp-1 zero)
    {
        const int vec = (reinterpret_cast<uintptr_t>(A) % 16 == 0 && lda % 4 == 0 && n % 4 == 0 && m % 2 == 0) ? 1 : 0;
        const int64_t tiles = ((m + kCvt - 1) / kCvt) * ((n + kCvt - 1) / kCvt);
        k_to_bf16_both<<<unsigned(tiles), 256, 0, stream>>>(A, m, n, lda, vec, w.Abf, w.Atbf);
        RSK_LAUNCH_CHECK(h);
    }
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
    if (L.ssyevd(L.sh, kEigModeVector, kFillLower, r, w.G, r, w.w, w.work, lwork, w.info) != 0)
        return fail(h, RSK_ERR_CUDA, "cusolverDnSsyevd failed");
    k_eig_post<<<8, 256, 0, stream>>>(w.w, w.G, r, s, w.Uh, w.sinv);
    RSK_LAUNCH_CHECK(h);
    // U = Q Uhat  (row-major m x r = (Uhat^T Q^T)^T): column-major U^T (r x m) = Uhat^T (r x r) * Q^T (r x m)
    st = lt_matmul(h, 1, 0, r, m, r, w.Uh, CUDA_R_32F, r, w.Y, rp, U, CUDA_R_32F, r, 1.f, fp32_compute(h), w.ltws,
                   stream);
    if (st != RSK_OK) return st;
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
