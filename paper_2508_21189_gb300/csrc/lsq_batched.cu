// Batched sketch-and-precondition least squares (row a8): many problems of uneven n_i and k_i
// solved together.  Per problem the steps are those of rsk_lstsq_sketch_precond (sketch,
// Householder QR, warm start, refinement on the FP64 normal-equation residual with CG on
// M_i = A_i R_i^{-1}); the QR runs in FP64, or in FP32 on request (R_i and Q_i^T S b_i then go to
// FP64 for the triangular steps).  Across problems the work is batched:
//   * sketches: the inverted index is built once per problem and applied to A_i and b_i, spread
//     over a small pool of streams;
//   * k_qr_b / k_rinv_b / k_trmv_b / k_cg_*_b: one CTA per problem;
//   * k_pass_b: a persistent grid pulls (problem, row-block) tiles from an atomic work queue and
//     writes one partial per tile; k_reduce_b sums a problem's tiles in tile order, so results do
//     not depend on which CTA ran which tile;
//   * one CG iteration (6 kernels and a queue reset) is captured in a CUDA graph and replayed.
// The FP64-accuracy residual pass on FP32-stored A runs in double-float arithmetic (pairs of FP32
// values, Dekker's exact product and Knuth's exact sum), which keeps it at the HBM roofline on a
// part whose FP64 rate is far below its FP32 rate.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace {

constexpr int kBThreads = 256;
constexpr int kBMaxK = 256;
constexpr int kTileRows = 2048;
constexpr int kStreams = 8;

struct BProb {
    const void* A;      // truth storage
    const void* Ain;    // storage the CG pass reads (A, or an FP32 copy)
    const double* b;
    double* xout;
    int64_t n, lda, lda_in;
    int k, d, a_f32, in_f32;
    double* W;          // d x (k+1) column-major
    float* W32;         // the same in FP32 when the QR runs in FP32, else null
    double* tau;        // k
    double* Rinv;       // k x k column-major
    double* v;          // x g c z res p s t | stats[3] (8k + 8)
    float* yf;          // k
    double* cg;         // 8
    void* part;         // ntiles x k (double)
    double* part_s;     // ntiles x 3
    const float2* bsplit;  // b as FP32 pairs (hi, lo) for the double-float residual pass, else null
    int tile0, ntiles;
};

struct Tile {
    int p, r0, r1, pad;
};

template <typename T>
__device__ __forceinline__ T block_sum_b(T v, T* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    T s = T(0);
    for (int i = 0; i < int(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

// ---- Householder QR of W = [S A | S b], one CTA per problem, in FP64 (T = double, on W) or FP32
// (T = float, on W32) --------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T* qr_buf(const BProb& q);
template <>
__device__ __forceinline__ double* qr_buf<double>(const BProb& q) { return q.W; }
template <>
__device__ __forceinline__ float* qr_buf<float>(const BProb& q) { return q.W32; }

template <typename T>
__device__ void qr_one(const BProb& q, T* red);

// Persistent: one CTA per SM pulls problems from a queue ordered by decreasing work (d k^2), so
// the largest factorizations start first and the small ones fill in behind them (LPT order).
template <typename T>
__global__ void __launch_bounds__(1024) k_qr_b(BProb* P, const int* __restrict__ order, int count,
                                              unsigned int* queue) {
    __shared__ T red[32];
    __shared__ int next_s;
    for (;;) {
        if (threadIdx.x == 0) next_s = int(atomicAdd(queue, 1u));
        __syncthreads();
        const int slot = next_s;
        __syncthreads();
        if (slot >= count) break;
        qr_one<T>(P[order[slot]], red);
    }
}

// Reflector j: v = (1, W[j+1:, j] / (alpha - beta)), tau = (beta - alpha) / beta, R_jj = beta; the
// reflector is applied to the columns right of j (the last one is S b, so Q^T S b builds up there).
template <typename T>
__device__ void qr_one(const BProb& q, T* red) {
    const int d = q.d, k = q.k, cols = k + 1;
    T* W = qr_buf<T>(q);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = 0; j < k; ++j) {
        T* colj = W + size_t(j) * d;
        T s = T(0);
        for (int i = j + 1 + threadIdx.x; i < d; i += blockDim.x) s += colj[i] * colj[i];
        const T sigma = block_sum_b<T>(s, red);
        const T alpha = colj[j];
        T tau = T(0), beta = alpha, scale = T(1);
        if (sigma > T(0)) {
            const T nrm = sqrt(alpha * alpha + sigma);
            beta = alpha > T(0) ? -nrm : nrm;
            tau = (beta - alpha) / beta;
            scale = T(1) / (alpha - beta);
            for (int i = j + 1 + threadIdx.x; i < d; i += blockDim.x) colj[i] *= scale;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            colj[j] = beta;
            q.tau[j] = double(tau);
        }
        __syncthreads();
        for (int c = j + 1 + warp; c < cols; c += nw) {
            T* col = W + size_t(c) * d;
            T t = T(0);
            for (int i = j + 1 + lane; i < d; i += 32) t += colj[i] * col[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            const T w = tau * (col[j] + t);
            if (lane == 0) col[j] -= w;
            for (int i = j + 1 + lane; i < d; i += 32) col[i] -= w * colj[i];
        }
        __syncthreads();
    }
}

// After the FP32 QR: rows 0..k-1 of every column of W32 (R and the leading k entries of Q^T S b) to
// the FP64 W that k_rinv_b and k_trmv_b read.
__global__ void k_qr32_to_w_b(BProb* P) {
    const BProb& q = P[blockIdx.x];
    if (!q.W32) return;
    const int k = q.k, d = q.d;
    for (int idx = threadIdx.x; idx < k * (k + 1); idx += blockDim.x) {
        const int c = idx / k, i = idx - c * k;
        q.W[size_t(c) * d + i] = double(q.W32[size_t(c) * d + i]);
    }
}

__global__ void __launch_bounds__(512) k_rinv_b(BProb* P) {
    const BProb& q = P[blockIdx.x];
    const int k = q.k, d = q.d;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int c = warp; c < k; c += nw) {
        double* x = q.Rinv + size_t(c) * k;
        for (int i = lane; i < k; i += 32) x[i] = (i == c) ? 1.0 : 0.0;
        __syncwarp();
        for (int l = c; l >= 0; --l) {
            const double* Rl = q.W + size_t(l) * d;
            const double xl = x[l] / Rl[l];
            __syncwarp();
            if (lane == 0) x[l] = xl;
            for (int i = lane; i < l; i += 32) x[i] -= Rl[i] * xl;
            __syncwarp();
        }
    }
}

// dst = op(R^{-1}) src; src/dst are vector slots of q.v (slot -1 = the Q^T S b column of W).
__global__ void k_trmv_b(BProb* P, int trans, int src_slot, int dst_slot, int only_active_cg) {
    const BProb& q = P[blockIdx.x];
    if (only_active_cg && q.cg[2] != 0.0) return;
    const int k = q.k;
    const double* src = src_slot < 0 ? q.W + size_t(k) * q.d : q.v + size_t(src_slot) * k;
    double* dst = q.v + size_t(dst_slot) * k;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = warp; i < k; i += nw) {
        double s = 0.0;
        if (!trans)
            for (int l = i + lane; l < k; l += 32) s += q.Rinv[size_t(l) * k + i] * src[l];
        else
            for (int l = lane; l <= i; l += 32) s += q.Rinv[size_t(i) * k + l] * src[l];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) dst[i] = s;
    }
}

__global__ void k_cast_b(BProb* P, int src_slot) {
    const BProb& q = P[blockIdx.x];
    if (q.cg[2] != 0.0) return;
    for (int j = threadIdx.x; j < q.k; j += blockDim.x) q.yf[j] = float(q.v[size_t(src_slot) * q.k + j]);
}

// ---- double-float helpers (Dekker's exact product, Knuth's exact sum) -------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void df_acc(float& hi, float& lo, float a, float xh, float xl) {
    const float p = a * xh;
    const float pe = fmaf(a, xh, -p);        // exact: a*xh = p + pe
    float s, e;
    two_sum(hi, p, s, e);
    e += lo + fmaf(a, xl, pe);
    hi = s + e;
    lo = e - (hi - s);
}
__device__ __forceinline__ void df_merge(float& hi, float& lo, float oh, float ol) {
    float s, e;
    two_sum(hi, oh, s, e);
    e += lo + ol;
    hi = s + e;
    lo = e - (hi - s);
}

// ---- fused passes over tiles of all problems ---------------------------------------------
// MODE 0: CG pass, FP32 storage and arithmetic: q = A^T A y (y = yf).
// MODE 1: CG pass in FP64 arithmetic (F64 or F32 storage): q = A^T A t (t = slot 7).
// MODE 2: residual pass in FP64: r = b - A x, g = A^T r, rr, ff.
// MODE 3: residual pass in double-float FP32 arithmetic (F32 storage only), b pre-split into
//         FP32 pairs so that no FP64 instruction runs per row.
// A warp takes R rows at a time: lanes hold columns lane + 32 m of each row, the R partial dot
// products are reduce-scattered across the warp (lane L ends with row 2*bit4(L) + bit3(L) for
// R = 4, bit4(L) for R = 2), and each row's result is read back from its owner lane.
constexpr unsigned kFull = 0xffffffffu;

template <int R>
__device__ __forceinline__ int row_owner(int r) {
    return R == 4 ? (((r >> 1) & 1) << 4) | ((r & 1) << 3) : (r << 4);
}

template <int R, typename T>
__device__ __forceinline__ T reduce_scatter(const T (&p)[R], int lane) {
    T k;
    if constexpr (R == 4) {
        const bool b4 = lane & 16;
        T k0 = b4 ? p[2] : p[0], k1 = b4 ? p[3] : p[1];
        const T s0 = b4 ? p[0] : p[2], s1 = b4 ? p[1] : p[3];
        k0 += __shfl_xor_sync(kFull, s0, 16);
        k1 += __shfl_xor_sync(kFull, s1, 16);
        const bool b3 = lane & 8;
        k = b3 ? k1 : k0;
        k += __shfl_xor_sync(kFull, b3 ? k0 : k1, 8);
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) k += __shfl_xor_sync(kFull, k, o);
    } else {
        const bool b4 = lane & 16;
        k = b4 ? p[1] : p[0];
        k += __shfl_xor_sync(kFull, b4 ? p[0] : p[1], 16);
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) k += __shfl_xor_sync(kFull, k, o);
    }
    return k;
}

// the same on double-float pairs
__device__ __forceinline__ void df_xor_merge(float& h, float& l, float sh, float sl, int o) {
    const float oh = __shfl_xor_sync(kFull, sh, o), ol = __shfl_xor_sync(kFull, sl, o);
    df_merge(h, l, oh, ol);
}
__device__ __forceinline__ void reduce_scatter_df4(const float (&ph)[4], const float (&pl)[4], int lane, float& h,
                                                   float& l) {
    const bool b4 = lane & 16;
    float k0h = b4 ? ph[2] : ph[0], k0l = b4 ? pl[2] : pl[0];
    float k1h = b4 ? ph[3] : ph[1], k1l = b4 ? pl[3] : pl[1];
    df_xor_merge(k0h, k0l, b4 ? ph[0] : ph[2], b4 ? pl[0] : pl[2], 16);
    df_xor_merge(k1h, k1l, b4 ? ph[1] : ph[3], b4 ? pl[1] : pl[3], 16);
    const bool b3 = lane & 8;
    h = b3 ? k1h : k0h;
    l = b3 ? k1l : k0l;
    df_xor_merge(h, l, b3 ? k0h : k1h, b3 ? k0l : k1l, 8);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) df_xor_merge(h, l, h, l, o);
}

// The row loop of one tile, specialised on the number of 32-column blocks the problem uses (MK), so
// that no predicated-off work is issued for the blocks beyond the problem's k.
template <int MODE, int M, int MK>
__device__ __forceinline__ void pass_rows(const BProb& q, const Tile& T, int k, int lane, int warp, int nw,
                                          const double* ys, const float* yh, const float* yl, const float* Af,
                                          int64_t ldf, int want_frob, double (&g)[M], float (&gh)[M], float (&gl)[M],
                                          double& rr, double& ff, double& bb, float& rrf, float& fff, float& bbf) {
    constexpr bool F64 = MODE == 1 || MODE == 2;
    constexpr int R = F64 ? 2 : 4;
        for (int i0 = T.r0 + warp * R; i0 < T.r1; i0 += nw * R) {
        if constexpr (!F64) {
            float a[R][M];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const bool valid = i0 + r < T.r1;
                const float* row = Af + int64_t(i0 + r) * ldf;
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    const int j = lane + 32 * m;
                    a[r][m] = (m < MK && valid && j < k) ? row[j] : 0.f;
                }
            }
            if constexpr (MODE == 0) {
                float p[R];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    p[r] = 0.f;
#pragma unroll
                    for (int m = 0; m < M; ++m)
                        if (m < MK) p[r] = fmaf(a[r][m], yh[lane + 32 * m], p[r]);
                }
                const float w = reduce_scatter<R, float>(p, lane);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float wr = __shfl_sync(kFull, w, row_owner<R>(r));
#pragma unroll
                    for (int m = 0; m < M; ++m)
                        if (m < MK) gh[m] = fmaf(wr, a[r][m], gh[m]);
                }
            } else {  // MODE 3
                float ph[R], pl[R];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    ph[r] = 0.f;
                    pl[r] = 0.f;
#pragma unroll
                    for (int m = 0; m < M; ++m)
                        if (m < MK) {
                            const int j = lane + 32 * m;
                            df_acc(ph[r], pl[r], a[r][m], yh[j], yl[j]);
                            fff = fmaf(a[r][m], a[r][m], fff);
                        }
                }
                float dh, dl;
                reduce_scatter_df4(ph, pl, lane, dh, dl);
                // this lane's row: r = b - a.x in double-float
                const int rho = ((lane >> 4) & 1) * 2 + ((lane >> 3) & 1);
                const int irow = i0 + rho;
                float rh = 0.f, rl = 0.f;
                if (irow < T.r1) {
                    const float2 bs = q.bsplit[irow];
                    float s, e;
                    two_sum(bs.x, -dh, s, e);
                    e += bs.y - dl;
                    rh = s + e;
                    rl = e - (rh - s);
                    if ((lane & 7) == 0) {
                        rrf = fmaf(rh, rh, rrf);
                        bbf = fmaf(bs.x, bs.x, bbf);
                    }
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float wh = __shfl_sync(kFull, rh, row_owner<R>(r));
                    const float wl = __shfl_sync(kFull, rl, row_owner<R>(r));
#pragma unroll
                    for (int m = 0; m < M; ++m)
                        if (m < MK) df_acc(gh[m], gl[m], a[r][m], wh, wl);
                }
            }
        } else {
            double a[R][M];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const bool valid = i0 + r < T.r1;
                if (q.a_f32) {
                    const float* row = static_cast<const float*>(q.A) + int64_t(i0 + r) * q.lda;
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        const int j = lane + 32 * m;
                        a[r][m] = (m < MK && valid && j < k) ? double(row[j]) : 0.0;
                    }
                } else {
                    const double* row = static_cast<const double*>(q.A) + int64_t(i0 + r) * q.lda;
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        const int j = lane + 32 * m;
                        a[r][m] = (m < MK && valid && j < k) ? row[j] : 0.0;
                    }
                }
            }
            double p[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                p[r] = 0.0;
#pragma unroll
                for (int m = 0; m < M; ++m)
                    if (m < MK) p[r] = fma(a[r][m], ys[lane + 32 * m], p[r]);
            }
            double w = reduce_scatter<R, double>(p, lane);
            if constexpr (MODE == 2) {
                const int irow = i0 + ((lane >> 4) & 1);
                if (irow < T.r1) {
                    const double bi = q.b[irow];
                    w = bi - w;
                    if ((lane & 15) == 0) {
                        rr += w * w;
                        bb += bi * bi;
                    }
                } else {
                    w = 0.0;
                }
                if (want_frob) {
#pragma unroll
                    for (int r = 0; r < R; ++r)
#pragma unroll
                        for (int m = 0; m < M; ++m)
                            if (m < MK) ff = fma(a[r][m], a[r][m], ff);
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const double wr = __shfl_sync(kFull, w, row_owner<R>(r));
#pragma unroll
                for (int m = 0; m < M; ++m)
                    if (m < MK) g[m] = fma(wr, a[r][m], g[m]);
            }
        }
    }
}

template <int MODE, int M>
__global__ void __launch_bounds__(kBThreads) k_pass_b(BProb* P, const Tile* __restrict__ tiles, int ntiles,
                                                       unsigned int* queue, const int* __restrict__ active,
                                                       int want_frob) {
    constexpr bool F64 = MODE == 1 || MODE == 2;
    constexpr int R = F64 ? 2 : 4;
    __shared__ double ys[kBMaxK];
    __shared__ float yh[kBMaxK], yl[kBMaxK];
    __shared__ double gs[kBThreads / 32][kBMaxK];
    __shared__ double ss[kBThreads / 32][3];
    __shared__ int tile_s;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = kBThreads / 32;
    for (;;) {
        if (threadIdx.x == 0) tile_s = int(atomicAdd(queue, 1u));
        __syncthreads();
        const int tid = tile_s;
        if (tid >= ntiles) break;
        const Tile T = tiles[tid];
        const BProb& q = P[T.p];
        const bool skip = !active[T.p] || ((MODE == 0 || MODE == 1) && q.cg[2] != 0.0);
        if (skip) {
            __syncthreads();
            continue;
        }
        const int k = q.k;
        const int mk = (k + 31) >> 5;  // column blocks this problem uses (warp-uniform)
        for (int j = threadIdx.x; j < 32 * M; j += kBThreads) {
            double y = 0.0;
            if (j < k) {
                if (MODE == 0) y = double(q.yf[j]);
                else if (MODE == 1) y = q.v[size_t(7) * k + j];
                else y = q.v[j];  // x
            }
            ys[j] = y;
            const float h = float(y);
            yh[j] = h;
            yl[j] = float(y - double(h));
        }
        __syncthreads();
        double g[M];
        float gh[M], gl[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            g[m] = 0.0;
            gh[m] = 0.f;
            gl[m] = 0.f;
        }
        double rr = 0.0, ff = 0.0, bb = 0.0;
        float rrf = 0.f, fff = 0.f, bbf = 0.f;
        const float* Af = static_cast<const float*>(MODE == 0 ? q.Ain : q.A);
        const int64_t ldf = MODE == 0 ? q.lda_in : q.lda;
        const int mk_ = (k + 31) >> 5;
#define RSK_PASS_ROWS(MKV)                                                                                   \
    pass_rows<MODE, M, MKV>(q, T, k, lane, warp, nw, ys, yh, yl, Af, ldf, want_frob, g, gh, gl, rr, ff, bb, rrf, \
                            fff, bbf)
        switch (mk_) {
            case 1: RSK_PASS_ROWS(1); break;
            case 2: RSK_PASS_ROWS(2); break;
            case 3: RSK_PASS_ROWS(3); break;
            case 4: RSK_PASS_ROWS(4); break;
            case 5: if constexpr (M >= 5) RSK_PASS_ROWS(5); break;
            case 6: if constexpr (M >= 6) RSK_PASS_ROWS(6); break;
            case 7: if constexpr (M >= 7) RSK_PASS_ROWS(7); break;
            default: if constexpr (M >= 8) RSK_PASS_ROWS(8); break;
        }
#undef RSK_PASS_ROWS
        if constexpr (MODE == 3) {
            rr = double(rrf);
            ff = double(fff);
            bb = double(bbf);
        }
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int j = lane + 32 * m;
            if (j < k) {
                if (MODE == 0) gs[warp][j] = double(gh[m]);
                else if (MODE == 3) gs[warp][j] = double(gh[m]) + double(gl[m]);
                else gs[warp][j] = g[m];
            }
        }
        if (MODE >= 2) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                rr += __shfl_xor_sync(kFull, rr, o);
                ff += __shfl_xor_sync(kFull, ff, o);
                bb += __shfl_xor_sync(kFull, bb, o);
            }
            if (lane == 0) {
                ss[warp][0] = rr;
                ss[warp][1] = ff;
                ss[warp][2] = bb;
            }
        }
        __syncthreads();
        double* part = static_cast<double*>(q.part) + size_t(tid - q.tile0) * k;
        for (int j = threadIdx.x; j < k; j += kBThreads) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += gs[w][j];
            part[j] = s;
        }
        if (MODE >= 2 && threadIdx.x == 0) {
            double a0 = 0.0, a1 = 0.0, a2 = 0.0;
            for (int w = 0; w < nw; ++w) {
                a0 += ss[w][0];
                a1 += ss[w][1];
                a2 += ss[w][2];
            }
            q.part_s[3 * (tid - q.tile0)] = a0;
            q.part_s[3 * (tid - q.tile0) + 1] = a1;
            q.part_s[3 * (tid - q.tile0) + 2] = a2;
        }
        __syncthreads();
    }
}

// Sum a problem's tile partials in tile order into slot dst_slot; MODE >= 2 also rr, ff -> stats.
__global__ void k_reduce_b(BProb* P, const int* __restrict__ active, int dst_slot, int with_stats, int cg_gate,
                           int first) {
    const BProb& q = P[blockIdx.x];
    if (!active[blockIdx.x] || (cg_gate && q.cg[2] != 0.0)) return;
    const int k = q.k;
    const double* part = static_cast<const double*>(q.part);
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        double s = 0.0;
        for (int t = 0; t < q.ntiles; ++t) s += part[size_t(t) * k + j];
        q.v[size_t(dst_slot) * k + j] = s;
    }
    if (with_stats && threadIdx.x < 3) {
        double s = 0.0;
        for (int t = 0; t < q.ntiles; ++t) s += q.part_s[3 * t + threadIdx.x];
        double* stats = q.v + size_t(8) * k;
        if (threadIdx.x == 0) stats[0] = s;                 // ||r||^2
        else if (first) stats[threadIdx.x] = s;              // ||A||_F^2, ||b||^2 (first pass only)
    }
}

// eta_i = min(||g|| / (||A||_F ||r||), ||r|| / (||A||_F ||x|| + ||b||)) into eta[3i]
__global__ void k_eta_b(BProb* P, const int* __restrict__ active, double* __restrict__ eta) {
    __shared__ double red[32];
    const BProb& q = P[blockIdx.x];
    if (!active[blockIdx.x]) return;
    double s = 0.0, xs = 0.0;
    for (int j = threadIdx.x; j < q.k; j += blockDim.x) {
        s += q.v[size_t(1) * q.k + j] * q.v[size_t(1) * q.k + j];
        xs += q.v[j] * q.v[j];
    }
    const double gn = sqrt(block_sum_b(s, red));
    const double xn = sqrt(block_sum_b(xs, red));
    if (threadIdx.x == 0) {
        const double* stats = q.v + size_t(8) * q.k;
        const double rn = sqrt(stats[0]), fn = sqrt(stats[1]), bn = sqrt(stats[2]);
        double e = 0.0;
        if (rn > 0.0) {
            const double ls = fn > 0.0 ? gn / (fn * rn) : 0.0;
            const double den = fn * xn + bn;
            e = fmin(ls, den > 0.0 ? rn / den : ls);
        }
        eta[3 * blockIdx.x] = e;
        eta[3 * blockIdx.x + 1] = rn;
        eta[3 * blockIdx.x + 2] = fn;
    }
}

__global__ void k_cg_init_b(BProb* P, const int* __restrict__ active) {
    __shared__ double red[32];
    const BProb& q = P[blockIdx.x];
    if (!active[blockIdx.x]) {
        if (threadIdx.x == 0) q.cg[2] = 1.0;
        return;
    }
    const int k = q.k;
    const double* c = q.v + size_t(2) * k;
    double *z = q.v + size_t(3) * k, *res = q.v + size_t(4) * k, *p = q.v + size_t(5) * k;
    double s = 0.0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        z[j] = 0.0;
        res[j] = c[j];
        p[j] = c[j];
        s += c[j] * c[j];
    }
    const double rho = block_sum_b(s, red);
    if (threadIdx.x == 0) {
        q.cg[0] = rho;
        q.cg[1] = rho;
        q.cg[2] = rho > 0.0 ? 0.0 : 1.0;
        q.cg[3] = 0.0;
    }
}

__global__ void k_cg_step_b(BProb* P, double tol, unsigned int* running) {
    __shared__ double red[32];
    const BProb& q = P[blockIdx.x];
    if (q.cg[2] != 0.0) return;
    const int k = q.k;
    const double* s = q.v + size_t(6) * k;
    double *z = q.v + size_t(3) * k, *res = q.v + size_t(4) * k, *p = q.v + size_t(5) * k;
    double ps = 0.0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) ps += p[j] * s[j];
    const double pAp = block_sum_b(ps, red);
    const double rho = q.cg[0];
    const double alpha = pAp > 0.0 ? rho / pAp : 0.0;
    double rn = 0.0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        z[j] += alpha * p[j];
        res[j] -= alpha * s[j];
        rn += res[j] * res[j];
    }
    const double rho_new = block_sum_b(rn, red);
    const double beta = rho > 0.0 ? rho_new / rho : 0.0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) p[j] = res[j] + beta * p[j];
    __syncthreads();
    if (threadIdx.x == 0) {
        q.cg[0] = rho_new;
        q.cg[3] += 1.0;
        if (!(pAp > 0.0) || rho_new <= tol * tol * q.cg[1]) q.cg[2] = 1.0;
        else atomicAdd(running, 1u);
    }
}

// x += t (slot 7) for active problems; count CG iterations
__global__ void k_update_b(BProb* P, const int* __restrict__ active, double* __restrict__ iters) {
    const BProb& q = P[blockIdx.x];
    if (!active[blockIdx.x]) return;
    for (int j = threadIdx.x; j < q.k; j += blockDim.x) q.v[j] += q.v[size_t(7) * q.k + j];
    if (threadIdx.x == 0) iters[blockIdx.x] += q.cg[3];
}

__global__ void k_finish_b(BProb* P) {
    const BProb& q = P[blockIdx.x];
    for (int j = threadIdx.x; j < q.k; j += blockDim.x) q.xout[j] = q.v[j];
}

template <typename S, typename T>
__global__ void k_to_colmajor_b(const S* __restrict__ SA, const double* __restrict__ Sb, int d, int k,
                                T* __restrict__ W) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= int64_t(d) * (k + 1)) return;
    const int c = int(idx / d), i = int(idx - int64_t(c) * d);
    W[idx] = c < k ? T(SA[int64_t(i) * k + c]) : T(Sb[i]);
}

// b as double-float pairs (hi = float(b), lo = float(b - hi)) for every problem in one launch
// (blockIdx.y = problem).
__global__ void k_split_vec_b(const BProb* __restrict__ P) {
    const BProb& q = P[blockIdx.y];
    float2* out = const_cast<float2*>(q.bsplit);
    if (!out) return;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < q.n; i += int64_t(gridDim.x) * blockDim.x) {
        const double v = q.b[i];
        const float h = float(v);
        out[i] = make_float2(h, float(v - double(h)));
    }
}

__global__ void k_f32_to_f64(const float* __restrict__ A, int64_t n, int k, int64_t lda, double* __restrict__ B) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= n * k) return;
    const int64_t i = idx / k, j = idx - i * k;
    B[idx] = double(A[i * lda + j]);
}
__global__ void k_f64_to_f32(const double* __restrict__ A, int64_t n, int k, int64_t lda, float* __restrict__ B) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= n * k) return;
    const int64_t i = idx / k, j = idx - i * k;
    B[idx] = float(A[i * lda + j]);
}

template <int MODE>
void launch_pass_b(BProb* P, const Tile* tiles, int ntiles, unsigned int* queue, const int* active, int frob,
                   int grid, int maxk, cudaStream_t s) {
    if (maxk <= 128) k_pass_b<MODE, 4><<<grid, kBThreads, 0, s>>>(P, tiles, ntiles, queue, active, frob);
    else k_pass_b<MODE, 8><<<grid, kBThreads, 0, s>>>(P, tiles, ntiles, queue, active, frob);
}

}  // namespace

extern "C" rsk_status rsk_lstsq_sketch_precond_batched(rsk_handle* h, int32_t count, const rsk_lsq_problem* probs,
                                                       const rsk_lsq_opts* opts, rsk_lsq_info* infos,
                                                       cudaStream_t stream) {
    using namespace rsk;
    if (!h) return RSK_ERR_INVALID_ARG;
    if (count < 1 || !probs || !opts) return fail(h, RSK_ERR_INVALID_ARG, "need count >= 1, problems and options");
    if (opts->inner_dtype != RSK_F64 && opts->inner_dtype != RSK_F32)
        return fail(h, RSK_ERR_INVALID_ARG, "inner dtype must be F64 or F32");
    if (opts->sketch_dtype != RSK_F64 && opts->sketch_dtype != RSK_F32)
        return fail(h, RSK_ERR_INVALID_ARG, "batched sketch dtype must be F64 or F32");
    if (opts->qr_dtype != RSK_F64 && opts->qr_dtype != RSK_F32)
        return fail(h, RSK_ERR_INVALID_ARG, "QR dtype must be F64 or F32");
    const bool qr32 = opts->qr_dtype == RSK_F32;
    const int zeta = opts->zeta;
    std::vector<BProb> hp(count);
    std::vector<Tile> tiles;
    int maxk = 0;
    size_t bytes = 0;
    auto add = [&](size_t b_) { bytes += Carver::round(b_); };
    size_t max_sketch_scratch = 0;
    // rows per work tile: tuned for this batch (keyed by its total rows and problem count) or 2048
    int64_t total_rows = 0;
    for (int i = 0; i < count; ++i) total_rows += probs[i].n;
    const int tuned_tile = rsk::tuned_value(h, rsk::kTuneBatchTile, int(opts->inner_dtype), total_rows, count, 0);
    const int tile_rows = tuned_tile > 0 ? tuned_tile : kTileRows;
    for (int i = 0; i < count; ++i) {
        const rsk_lsq_problem& pr = probs[i];
        if (!pr.A || !pr.b || !pr.x) return fail(h, RSK_ERR_INVALID_ARG, "problem %d: null pointer", i);
        if (pr.a_dtype != RSK_F64 && pr.a_dtype != RSK_F32)
            return fail(h, RSK_ERR_INVALID_ARG, "problem %d: A must be F64 or F32", i);
        if (pr.k < 1 || pr.k > kBMaxK || pr.n < pr.k || pr.n >= (int64_t(1) << 31) || pr.lda < pr.k)
            return fail(h, RSK_ERR_INVALID_ARG, "problem %d: need 1 <= k <= %d, k <= n < 2^31, lda >= k", i, kBMaxK);
        const int64_t d = pr.d > 0 ? pr.d : 4 * pr.k;
        if (d < pr.k || d > 8192 || zeta > d)
            return fail(h, RSK_ERR_INVALID_ARG, "problem %d: need k <= d <= 8192 and zeta <= d", i);
        BProb& q = hp[i];
        q.A = pr.A;
        q.b = pr.b;
        q.xout = pr.x;
        q.n = pr.n;
        q.lda = pr.lda;
        q.k = int(pr.k);
        q.d = int(d);
        q.a_f32 = pr.a_dtype == RSK_F32;
        q.in_f32 = opts->inner_dtype == RSK_F32;
        q.tile0 = int(tiles.size());
        q.ntiles = int((pr.n + tile_rows - 1) / tile_rows);
        for (int t = 0; t < q.ntiles; ++t) {
            Tile T;
            T.p = i;
            T.r0 = t * tile_rows;
            T.r1 = int(std::min<int64_t>(pr.n, int64_t(t + 1) * tile_rows));
            T.pad = 0;
            tiles.push_back(T);
        }
        maxk = std::max(maxk, q.k);
        add(size_t(d) * (q.k + 1) * 8);
        if (qr32) add(size_t(d) * (q.k + 1) * 4);
        add(size_t(q.k) * 8);
        add(size_t(q.k) * q.k * 8);
        add((size_t(8) * q.k + 8) * 8);
        add(size_t(q.k) * 4);
        add(64);
        add(size_t(q.ntiles) * q.k * 8);
        add(size_t(q.ntiles) * 3 * 8);
        const bool sk_copy = (opts->sketch_dtype == RSK_F64) != (pr.a_dtype == RSK_F64);
        const bool in_copy = q.in_f32 && !q.a_f32;
        add(size_t(pr.n) * 8);  // b split into FP32 pairs (double-float residual pass)
        if (sk_copy) add(size_t(pr.n) * pr.k * (opts->sketch_dtype == RSK_F64 ? 8 : 4));
        if (in_copy && !(sk_copy && opts->sketch_dtype == RSK_F32)) add(size_t(pr.n) * pr.k * 4);
        const size_t sk = sketch_index_bytes(pr.n, d, zeta) +
                          Carver::round(std::max(sketch_partial_bytes(h, pr.n, pr.k, d, zeta, opts->sketch_dtype),
                                                 sketch_vec_scratch_bytes(pr.n, d, zeta))) +
                          Carver::round(size_t(d) * pr.k * 8) + Carver::round(size_t(d) * 8) + 1024;
        max_sketch_scratch = std::max(max_sketch_scratch, sk);
    }
    const int ntiles = int(tiles.size());
    add(size_t(count) * sizeof(BProb));
    add(size_t(ntiles) * sizeof(Tile));
    add(size_t(count) * 4);          // active flags
    add(size_t(count) * 3 * 8);      // eta, rnorm, fnorm
    add(size_t(count) * 8);          // CG iteration counts
    add(256);                        // queue counters
    add(size_t(count) * 4);          // QR order (decreasing d k^2)
    add(size_t(kStreams) * max_sketch_scratch);
    rsk_status st = ensure_workspace(h, bytes + 8192, stream);
    if (st != RSK_OK) return st;
    if (infos) memset(infos, 0, sizeof(rsk_lsq_info) * size_t(count));

    Carver cv(h->ws);
    std::vector<void*> sk_copy_ptr(count, nullptr);
    for (int i = 0; i < count; ++i) {
        BProb& q = hp[i];
        const rsk_lsq_problem& pr = probs[i];
        q.W = cv.take<double>(size_t(q.d) * (q.k + 1));
        q.W32 = qr32 ? cv.take<float>(size_t(q.d) * (q.k + 1)) : nullptr;
        q.tau = cv.take<double>(size_t(q.k));
        q.Rinv = cv.take<double>(size_t(q.k) * q.k);
        q.v = cv.take<double>(size_t(8) * q.k + 8);
        q.yf = cv.take<float>(size_t(q.k));
        q.cg = cv.take<double>(8);
        q.part = cv.take<double>(size_t(q.ntiles) * q.k);
        q.part_s = cv.take<double>(size_t(q.ntiles) * 3);
        q.bsplit = cv.take<float2>(size_t(pr.n));
        const bool sk_copy = (opts->sketch_dtype == RSK_F64) != (pr.a_dtype == RSK_F64);
        const bool in_copy = q.in_f32 && !q.a_f32;
        if (sk_copy) sk_copy_ptr[i] = cv.take<char>(size_t(pr.n) * pr.k * (opts->sketch_dtype == RSK_F64 ? 8 : 4));
        q.Ain = q.A;
        q.lda_in = q.lda;
        if (in_copy) {
            q.Ain = (sk_copy && opts->sketch_dtype == RSK_F32) ? sk_copy_ptr[i] : cv.take<char>(size_t(pr.n) * pr.k * 4);
            q.lda_in = q.k;
        }
    }
    BProb* dP = cv.take<BProb>(size_t(count));
    Tile* dT = cv.take<Tile>(size_t(ntiles));
    int* dactive = cv.take<int>(size_t(count));
    double* deta = cv.take<double>(size_t(count) * 3);
    double* diters = cv.take<double>(size_t(count));
    unsigned int* dqueue = cv.take<unsigned int>(64);   // [0] tile queue, [16] QR queue, [32] CG running
    int* dorder = cv.take<int>(size_t(count));
    char* sk_scratch = cv.take<char>(size_t(kStreams) * max_sketch_scratch);

    // all work runs on the handle's internal streams, ordered after the caller's stream
    st = ensure_streams(h, kStreams + 1);
    if (st != RSK_OK) return st;
    cudaStream_t main_s = h->streams[0];
    cudaEvent_t ev_start, ev_done;
    RSK_CUDA_TRY(h, cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming));
    RSK_CUDA_TRY(h, cudaEventCreateWithFlags(&ev_done, cudaEventDisableTiming));
    RSK_CUDA_TRY(h, cudaEventRecord(ev_start, stream));
    RSK_CUDA_TRY(h, cudaStreamWaitEvent(main_s, ev_start, 0));
    RSK_CUDA_TRY(h, cudaMemcpyAsync(dP, hp.data(), sizeof(BProb) * size_t(count), cudaMemcpyHostToDevice, main_s));
    RSK_CUDA_TRY(h, cudaMemcpyAsync(dT, tiles.data(), sizeof(Tile) * size_t(ntiles), cudaMemcpyHostToDevice, main_s));
    std::vector<int> act(count, 1);
    RSK_CUDA_TRY(h, cudaMemcpyAsync(dactive, act.data(), 4 * size_t(count), cudaMemcpyHostToDevice, main_s));
    RSK_CUDA_TRY(h, cudaMemsetAsync(diters, 0, 8 * size_t(count), main_s));
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b_) {
        return double(hp[a].d) * hp[a].k * hp[a].k > double(hp[b_].d) * hp[b_].k * hp[b_].k;
    });
    RSK_CUDA_TRY(h, cudaMemcpyAsync(dorder, order.data(), 4 * size_t(count), cudaMemcpyHostToDevice, main_s));
    // the sketch phase as a whole (forked from and joined back to main_s), for phase timing
    const int prs = prof_begin(h, main_s, RSK_KERNEL_BATCH_SKETCH);
    RSK_CUDA_TRY(h, cudaEventRecord(ev_done, main_s));

    // ---- sketches, spread over the stream pool
    const rsk_dtype sa_dt = opts->sketch_dtype;
    for (int i = 0; i < count; ++i) {
        const int si = 1 + i % kStreams;
        cudaStream_t s = h->streams[si];
        if (i < kStreams) RSK_CUDA_TRY(h, cudaStreamWaitEvent(s, ev_done, 0));
        BProb& q = hp[i];
        const rsk_lsq_problem& pr = probs[i];
        char* scr = sk_scratch + size_t(si - 1) * max_sketch_scratch;
        Carver sc(scr);
        void* index = sc.take<char>(sketch_index_bytes(pr.n, q.d, zeta));
        double* SA = sc.take<double>(size_t(q.d) * q.k);
        double* Sb = sc.take<double>(size_t(q.d));
        void* parts = sc.take<char>(std::max(sketch_partial_bytes(h, pr.n, pr.k, q.d, zeta, sa_dt),
                                             sketch_vec_scratch_bytes(pr.n, q.d, zeta)));
        const unsigned cgrid = unsigned((pr.n * pr.k + 255) / 256);
        const void* A_sk = pr.A;
        int64_t lda_sk = pr.lda;
        if (sk_copy_ptr[i]) {
            if (sa_dt == RSK_F64) k_f32_to_f64<<<cgrid, 256, 0, s>>>((const float*)pr.A, pr.n, q.k, pr.lda, (double*)sk_copy_ptr[i]);
            else k_f64_to_f32<<<cgrid, 256, 0, s>>>((const double*)pr.A, pr.n, q.k, pr.lda, (float*)sk_copy_ptr[i]);
            RSK_LAUNCH_CHECK(h);
            A_sk = sk_copy_ptr[i];
            lda_sk = pr.k;
        }
        if (q.Ain != q.A && q.Ain != sk_copy_ptr[i]) {
            k_f64_to_f32<<<cgrid, 256, 0, s>>>((const double*)pr.A, pr.n, q.k, pr.lda, (float*)const_cast<void*>(q.Ain));
            RSK_LAUNCH_CHECK(h);
        }
        st = sketch_build_index(h, pr.n, q.d, zeta, opts->seed + uint64_t(i), index, s);
        if (st == RSK_OK)
            st = sketch_apply_built(h, index, pr.n, q.d, zeta, A_sk, sa_dt, pr.k, lda_sk, SA,
                                    sa_dt == RSK_F64 ? RSK_F64 : RSK_F32, pr.k, parts, s);
        // S b after S A (the partials buffer is reused; same stream, so in order)
        if (st == RSK_OK) st = sketch_apply_vec_built(h, index, pr.n, q.d, zeta, pr.b, Sb, static_cast<double*>(parts), s);
        if (st != RSK_OK) return st;
        const unsigned gw = unsigned((int64_t(q.d) * (q.k + 1) + 255) / 256);
        const float* SA32 = reinterpret_cast<const float*>(SA);
        if (q.W32) {
            if (sa_dt == RSK_F64) k_to_colmajor_b<double, float><<<gw, 256, 0, s>>>(SA, Sb, q.d, q.k, q.W32);
            else k_to_colmajor_b<float, float><<<gw, 256, 0, s>>>(SA32, Sb, q.d, q.k, q.W32);
        } else {
            if (sa_dt == RSK_F64) k_to_colmajor_b<double, double><<<gw, 256, 0, s>>>(SA, Sb, q.d, q.k, q.W);
            else k_to_colmajor_b<float, double><<<gw, 256, 0, s>>>(SA32, Sb, q.d, q.k, q.W);
        }
        RSK_LAUNCH_CHECK(h);
    }
    // the double-float split of every b (for the residual passes), one launch for the whole batch
    k_split_vec_b<<<dim3(64, unsigned(count)), 256, 0, main_s>>>(dP);
    RSK_LAUNCH_CHECK(h);
    for (int si = 1; si <= kStreams; ++si) {
        RSK_CUDA_TRY(h, cudaEventRecord(ev_done, h->streams[si]));
        RSK_CUDA_TRY(h, cudaStreamWaitEvent(main_s, ev_done, 0));
    }
    prof_end(h, main_s, prs);

    // ---- QR, R^{-1}, warm start
    const int pr0 = prof_begin(h, main_s, RSK_KERNEL_BATCH_QR);
    RSK_CUDA_TRY(h, cudaMemsetAsync(dqueue + 16, 0, 4, main_s));
    if (qr32) {
        k_qr_b<float><<<std::min(count, h->num_sms), 1024, 0, main_s>>>(dP, dorder, count, dqueue + 16);
        k_qr32_to_w_b<<<count, 256, 0, main_s>>>(dP);
    } else {
        k_qr_b<double><<<std::min(count, h->num_sms), 1024, 0, main_s>>>(dP, dorder, count, dqueue + 16);
    }
    k_rinv_b<<<count, 512, 0, main_s>>>(dP);
    k_trmv_b<<<count, 256, 0, main_s>>>(dP, 0, -1, 0, 0);
    prof_end(h, main_s, pr0);
    RSK_LAUNCH_CHECK(h);

    // ---- refinement
    const double tol = opts->tol_backward > 0 ? opts->tol_backward : 1e-10;
    const int max_refine = opts->max_refine >= 0 ? opts->max_refine : 20;
    const int max_inner = opts->max_inner_iters > 0 ? opts->max_inner_iters : 50;
    const double inner_tol = opts->inner_tol > 0 ? opts->inner_tol : 1e-6;
    const int grid = 2 * h->num_sms;
    const bool df_resid = opts->inner_dtype == RSK_F32;  // double-float residual on FP32 storage
    std::vector<double> heta(size_t(count) * 3);
    std::vector<int> steps(count, 0);
    cudaGraphExec_t cg_exec = nullptr;
    volatile unsigned int* running_host = reinterpret_cast<volatile unsigned int*>(h->host_flags + 4);
    *running_host = 1u;
    int step = 0;
    for (step = 0;; ++step) {
        RSK_CUDA_TRY(h, cudaMemsetAsync(dqueue, 0, 4, main_s));
        // residual pass: problems with FP32 storage use double-float arithmetic when the inner
        // precision is FP32 (mixed form); the all-FP64 form uses FP64 arithmetic throughout
        bool all_f32 = true;
        for (int i = 0; i < count; ++i) all_f32 = all_f32 && hp[i].a_f32;
        const int pr1 = prof_begin(h, main_s, RSK_KERNEL_BATCH_RESID);
        if (df_resid && all_f32) launch_pass_b<3>(dP, dT, ntiles, dqueue, dactive, step == 0, grid, maxk, main_s);
        else launch_pass_b<2>(dP, dT, ntiles, dqueue, dactive, step == 0, grid, maxk, main_s);
        k_reduce_b<<<count, 256, 0, main_s>>>(dP, dactive, 1, 1, 0, step == 0);
        k_eta_b<<<count, 256, 0, main_s>>>(dP, dactive, deta);
        prof_end(h, main_s, pr1);
        RSK_LAUNCH_CHECK(h);
        RSK_CUDA_TRY(h, cudaMemcpyAsync(heta.data(), deta, 24 * size_t(count), cudaMemcpyDeviceToHost, main_s));
        RSK_CUDA_TRY(h, cudaStreamSynchronize(main_s));
        int nact = 0;
        for (int i = 0; i < count; ++i) {
            if (act[i] && (heta[3 * i] <= tol || step >= max_refine)) act[i] = 0;
            if (act[i]) {
                ++nact;
                steps[i] = step + 1;
            }
            if (infos) {
                infos[i].backward_err = heta[3 * i];
                infos[i].residual_norm = heta[3 * i + 1];
                if (step == 0) infos[i].frobenius_norm = heta[3 * i + 2];
            }
        }
        if (nact == 0) break;
        RSK_CUDA_TRY(h, cudaMemcpyAsync(dactive, act.data(), 4 * size_t(count), cudaMemcpyHostToDevice, main_s));
        // c = R^{-T} g; CG iterations replayed from a captured graph
        k_trmv_b<<<count, 256, 0, main_s>>>(dP, 1, 1, 2, 0);
        k_cg_init_b<<<count, 256, 0, main_s>>>(dP, dactive);
        RSK_LAUNCH_CHECK(h);
        if (!cg_exec) {
            cudaGraph_t graph;
            RSK_CUDA_TRY(h, cudaStreamBeginCapture(main_s, cudaStreamCaptureModeThreadLocal));
            cudaMemsetAsync(dqueue, 0, 4, main_s);
            cudaMemsetAsync(dqueue + 32, 0, 4, main_s);
            k_trmv_b<<<count, 256, 0, main_s>>>(dP, 0, 5, 7, 1);  // t = R^{-1} p
            if (opts->inner_dtype == RSK_F32) {
                k_cast_b<<<count, 256, 0, main_s>>>(dP, 7);
                launch_pass_b<0>(dP, dT, ntiles, dqueue, dactive, 0, grid, maxk, main_s);
            } else {
                launch_pass_b<1>(dP, dT, ntiles, dqueue, dactive, 0, grid, maxk, main_s);
            }
            k_reduce_b<<<count, 256, 0, main_s>>>(dP, dactive, 1, 0, 1, 0);   // g = A^T A t
            k_trmv_b<<<count, 256, 0, main_s>>>(dP, 1, 1, 6, 1);             // s = R^{-T} g
            k_cg_step_b<<<count, 256, 0, main_s>>>(dP, inner_tol, dqueue + 32);
            cudaMemcpyAsync(const_cast<unsigned int*>(running_host), dqueue + 32, 4, cudaMemcpyDeviceToHost, main_s);
            const cudaError_t ce = cudaStreamEndCapture(main_s, &graph);
            if (ce != cudaSuccess) return fail(h, RSK_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
            RSK_CUDA_TRY(h, cudaGraphInstantiate(&cg_exec, graph, 0));
            cudaGraphDestroy(graph);
        }
        const int pr2 = prof_begin(h, main_s, RSK_KERNEL_BATCH_CG);
        // replay until no problem's CG is running; the count is copied to pinned memory at the end
        // of each replay, and the host reads it two replays behind so the GPU never waits for it
        for (int it = 0; it < max_inner; ++it) {
            if (it >= 2) {
                RSK_CUDA_TRY(h, cudaEventSynchronize(h->flag_ev[it & 1]));
                if (*running_host == 0u) break;
            }
            RSK_CUDA_TRY(h, cudaGraphLaunch(cg_exec, main_s));
            RSK_CUDA_TRY(h, cudaEventRecord(h->flag_ev[it & 1], main_s));
        }
        prof_end(h, main_s, pr2);
        k_trmv_b<<<count, 256, 0, main_s>>>(dP, 0, 3, 7, 0);  // t = R^{-1} z
        k_update_b<<<count, 256, 0, main_s>>>(dP, dactive, diters);
        RSK_LAUNCH_CHECK(h);
    }
    if (cg_exec) cudaGraphExecDestroy(cg_exec);
    k_finish_b<<<count, 256, 0, main_s>>>(dP);
    RSK_LAUNCH_CHECK(h);
    std::vector<double> hit(count);
    RSK_CUDA_TRY(h, cudaMemcpyAsync(hit.data(), diters, 8 * size_t(count), cudaMemcpyDeviceToHost, main_s));
    RSK_CUDA_TRY(h, cudaEventRecord(ev_done, main_s));
    RSK_CUDA_TRY(h, cudaStreamWaitEvent(stream, ev_done, 0));
    RSK_CUDA_TRY(h, cudaStreamSynchronize(main_s));
    cudaEventDestroy(ev_start);
    cudaEventDestroy(ev_done);
    int bad = 0;
    for (int i = 0; i < count; ++i) {
        const bool ok = heta[3 * i] <= tol;
        bad += !ok;
        if (infos) {
            infos[i].refine_steps = steps[i];
            infos[i].inner_iters = int(hit[i]);
            infos[i].status = ok ? RSK_OK : RSK_ERR_NOT_CONVERGED;
        }
    }
    rsk_status dev = rsk_sync_status(h, main_s);
    if (dev != RSK_OK) return dev;
    if (bad) return fail(h, RSK_ERR_NOT_CONVERGED, "%d of %d problems above the backward-error tolerance", bad, count);
    return RSK_OK;
}
