// Small dense linear algebra for the low-rank consumers of the sketches: FP32, column-major.
//
// Kernels
//   k_gram          X^T Y over a chunk of rows: 64 x 64 output tile per CTA, 4 x 4 per thread, the rows
//                   staged 32 at a time, FP64 accumulation; per-chunk partials summed in chunk order by
//                   k_gram_reduce.
//   k_matmul_ts     C = X M for tall X: 128 x 64 output tile per CTA, K in steps of 16.
//   k_cholesky      one CTA: blocked right-looking Cholesky on the packed upper triangle in shared
//                   memory (16-row panels, the diagonal block inverted for the panel solve,
//                   register-tiled trailing update).
//   k_trinv_diag,   R^{-1} blocked over 32 x 32 blocks: the diagonal blocks inverted one warp each, then
//   k_trinv_blk     each block column by block back substitution (small products in shared memory).
//   k_jacobi        one-sided block Jacobi (Hestenes) on a cooperative grid: the q columns are dealt
//                   into nb = 2G blocks; in each of the nb - 1 rounds of a sweep CTA g takes one pair
//                   of blocks (round-robin), copies their columns (and V's) into shared memory,
//                   orthogonalises every pair of them with plane rotations (one warp per pair, the
//                   pairs of a local round disjoint), and writes them back; a bounded grid barrier
//                   separates the rounds.  Sweeps stop when one makes no rotation.
//   k_jacobi_cluster the same sweeps on one thread-block cluster when the columns fit in its shared
//                   memory: blocks stay on chip and move between rounds through distributed shared
//                   memory, cluster barriers instead of the grid barrier.
//   k_svd_post      singular values = column norms, sorted descending; U = X / s, V permuted alike.
#include <math.h>
#include <string.h>

#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"
#include "dense.cuh"

namespace {

constexpr float kU32 = 5.9604645e-8f;  // 2^-24

// ------------------------------------------------------------------------------------------
// Gram matrix.
// ------------------------------------------------------------------------------------------
constexpr int kGT = 64;      // output tile
constexpr int kGRows = 32;   // rows staged per step
constexpr int kGChunk = 2048;
constexpr int kGPitch = kGT + 4;

template <typename Acc>
__global__ void __launch_bounds__(256) k_gram(const float* __restrict__ X, int64_t m, int p, int64_t ldx,
                                             const float* __restrict__ Y, int q, int64_t ldy, bool sym, int ntq,
                                             Acc* __restrict__ part, int64_t pstride, int pp) {
    __shared__ __align__(16) float Xs[kGRows][kGPitch];
    __shared__ __align__(16) float Ys[kGRows][kGPitch];
    const int tile = blockIdx.x;
    const int tp = tile / ntq, tq = tile - (tile / ntq) * ntq;
    if (sym && tp > tq) return;
    const int64_t r0 = int64_t(blockIdx.y) * kGChunk;
    const int64_t r1 = min(m, r0 + kGChunk);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int p0 = tp * kGT, q0 = tq * kGT;
    Acc acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = Acc(0);
    for (int64_t rb = r0; rb < r1; rb += kGRows) {
        // coalesced loads along rows: element e of the thread is (row = tid % 32, col = tid / 32 + 8 e)
        const int rr = tid & 31;
        const int64_t row = rb + rr;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int c = (tid >> 5) + 8 * e;
            Xs[rr][c] = (row < r1 && p0 + c < p) ? X[int64_t(p0 + c) * ldx + row] : 0.f;
            Ys[rr][c] = (row < r1 && q0 + c < q) ? Y[int64_t(q0 + c) * ldy + row] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int r = 0; r < kGRows; ++r) {
            const float4 a = *reinterpret_cast<const float4*>(&Xs[r][ty * 4]);
            const float4 b = *reinterpret_cast<const float4*>(&Ys[r][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(Acc(av[i]), Acc(bv[j]), acc[i][j]);
        }
        __syncthreads();
    }
    Acc* out = part + int64_t(blockIdx.y) * pstride;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gi = p0 + ty * 4 + i, gj = q0 + tx * 4 + j;
            out[int64_t(gj) * pp + gi] = acc[i][j];
        }
}

// G[i, j] = sum over chunks (in order) of part[chunk][j * pp + i]; the symmetric case mirrors the
// computed triangle (tiles with tp <= tq).
template <typename Acc>
__global__ void k_gram_reduce(const Acc* __restrict__ part, int64_t pstride, int nchunks, int p, int q, int pp,
                              bool sym, Acc* __restrict__ G, int64_t ldg) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= int64_t(p) * q) return;
    const int j = int(idx / p), i = int(idx - int64_t(j) * p);
    int si = i, sj = j;
    if (sym && (i / kGT) > (j / kGT)) {
        si = j;
        sj = i;
    }
    Acc s = Acc(0);
    for (int c = 0; c < nchunks; ++c) s += part[int64_t(c) * pstride + int64_t(sj) * pp + si];
    G[int64_t(j) * ldg + i] = s;
}

// ------------------------------------------------------------------------------------------
// Tall-by-small product.
// ------------------------------------------------------------------------------------------
constexpr int kMR = 128, kMC = 64, kMK = 16;

__global__ void __launch_bounds__(256) k_matmul_ts(const float* __restrict__ X, int64_t m, int p, int64_t ldx,
                                                  const float* __restrict__ M, int q, int64_t ldm,
                                                  float* __restrict__ C, int64_t ldc) {
    __shared__ __align__(16) float Xs[kMK][kMR];
    __shared__ __align__(16) float Ms[kMK][kMC];
    const int64_t r0 = int64_t(blockIdx.x) * kMR;
    const int c0 = blockIdx.y * kMC;
    const int tid = threadIdx.x, tr = tid & 15, tc = tid >> 4;
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < p; k0 += kMK) {
        // X tile: 16 columns x 128 rows, rows contiguous in memory
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int lin = tid + 256 * e;
            const int rr = lin & (kMR - 1), kk = lin >> 7;
            const int64_t row = r0 + rr;
            Xs[kk][rr] = (row < m && k0 + kk < p) ? X[int64_t(k0 + kk) * ldx + row] : 0.f;
        }
        // M tile: 16 rows x 64 columns, rows of a column contiguous
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int lin = tid + 256 * e;
            const int kk = lin & (kMK - 1), cc = lin >> 4;
            Ms[kk][cc] = (k0 + kk < p && c0 + cc < q) ? M[int64_t(c0 + cc) * ldm + k0 + kk] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kMK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&Xs[kk][tr * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&Xs[kk][tr * 8 + 4]);
            const float4 b = *reinterpret_cast<const float4*>(&Ms[kk][tc * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int col = c0 + tc * 4 + j;
        if (col >= q) continue;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t row = r0 + tr * 8 + i;
            if (row < m) C[int64_t(col) * ldc + row] = acc[i][j];
        }
    }
}

// ------------------------------------------------------------------------------------------
// Cholesky (packed upper triangle in shared memory) and triangular inverse.
// ------------------------------------------------------------------------------------------
constexpr int kCholMax = 330;  // packed triangle + panel buffer within 227 KB of shared memory
__device__ __forceinline__ int pk(int i, int j, int q) { return i * q - (i * (i - 1)) / 2 + (j - i); }

// Blocked right-looking Cholesky sym(G) + s I = R^T R (s = shift_coeff * trace(G)) in one CTA, the
// upper triangle packed in shared memory.  Per panel of kCP rows (16; 8 when q > 320, so that the
// triangle and the panel buffer fit in shared memory) (c0 .. c1-1):
//   A  warp 0 factors the diagonal block in registers (a lane per column, shuffles for the rows; the
//      pivots' reciprocal square roots scale the rows), then inverts it (W = R_pp^{-1}, lane c taking
//      column c by back substitution against the block's rows in shared memory);
//   B  one thread per trailing column t >= c1 forms R(c0:c1, t) = W^T U(c0:c1, t), into the panel
//      buffer P and the triangle (a product: no dependent chain);
//   C  the trailing upper triangle takes the rank-kCP update U(a, b) -= sum_k P(k, a) P(k, b), in
//      4 x 4 register tiles (two 16-byte loads per k).  Look-ahead: warp 0 updates only the next
//      panel's diagonal block and then runs A for it, while the other warps update the rest (tile
//      rows dealt round-robin, lanes across a row), so the next panel's serial factorisation overlaps
//      this panel's update.
// Two barriers per panel; R is written from the packed factor at the end.  A pivot that is not
// positive (or not finite) stops the factorisation and sets RSK_DEV_BOUNDS.
constexpr int kCholThreads = 512;  // 128 registers a thread: the 4 x 4 tiles and the solve stay in registers
template <int kCP>
__global__ void __launch_bounds__(kCholThreads) k_cholesky(const float* __restrict__ G, int q, int64_t ldg, float shift_coeff,
                                                  float* __restrict__ R, int64_t ldr, unsigned int* status) {
    extern __shared__ __align__(16) float U[];
    const int qp = (q + 3) & ~3;                                 // panel buffer pitch (16-byte rows)
    float* P = U + (q * (q + 1) / 2 + 3) / 4 * 4;                // kCP x qp
    __shared__ float part[32];
    __shared__ float Rpp[kCP * kCP];   // the panel's diagonal block R(c0 + i, c0 + j), i <= j
    __shared__ float Wpp[kCP * kCP];   // its inverse W(i, j), zero for i > j
    __shared__ int fail_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    float t = 0.f;
    for (int i = tid; i < q; i += blockDim.x) t += G[int64_t(i) * ldg + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) part[warp] = t;
    if (tid == 0) fail_s = 0;
    __syncthreads();
    float trace = 0.f;
    for (int w = 0; w < nw; ++w) trace += part[w];
    const float shift = shift_coeff * trace;
    // the upper triangle column by column (coalesced: column j's rows 0 .. j are contiguous)
    for (int j = warp; j < q; j += nw)
#pragma unroll 4
        for (int i = lane; i <= j; i += 32) U[pk(i, j, q)] = G[int64_t(j) * ldg + i] + (i == j ? shift : 0.f);
    for (int e = tid; e < kCP * (qp - q); e += blockDim.x) P[(e / (qp - q)) * qp + q + e % (qp - q)] = 0.f;
    __syncthreads();
    // A for the panel at c0 (warp 0): the diagonal block, in registers: lane j < nb holds column j
    // (a[i] = U(c0+i, c0+j), i <= j); at step k lane k's diagonal d is broadcast, row k is scaled by
    // d^{-1/2} (lane k keeps d^{1/2} and d^{-1/2}), and lane j >= i takes a[i] -= R(k, i) R(k, j) with
    // R(k, i) broadcast from lane i.  Then W = R_pp^{-1}, lane c taking column c.
    auto factor_diag = [&](int c0) {
        const int nb = min(kCP, q - c0);
        float a[kCP];
#pragma unroll
        for (int i = 0; i < kCP; ++i) a[i] = (lane < nb && i <= lane) ? U[pk(c0 + i, c0 + lane, q)] : 0.f;
        bool bad = false;
        float inv_own = 1.f;
#pragma unroll
        for (int k = 0; k < kCP; ++k) {
            if (k < nb) {
                const float dk = __shfl_sync(0xffffffffu, a[k], k);
                const bool ok = dk > 0.f && isfinite(dk);
                bad = bad || !ok;
                const float inv = ok ? rsqrtf(dk) : 1.f;
                if (lane == k) {
                    a[k] = dk * inv;
                    inv_own = inv;
                } else if (lane > k) {
                    a[k] *= inv;
                }
#pragma unroll
                for (int i = k + 1; i < kCP; ++i) {
                    const float rki = __shfl_sync(0xffffffffu, a[k], i);
                    if (lane >= i) a[i] -= rki * a[k];
                }
            }
        }
        if (lane < nb) {
#pragma unroll
            for (int i = 0; i < kCP; ++i)
                if (i <= lane) {
                    U[pk(c0 + i, c0 + lane, q)] = a[i];
                    Rpp[i * kCP + lane] = a[i];
                }
        }
        __syncwarp();
        // W(i, c) = (delta_ic - sum_{l > i} R(i, l) W(l, c)) / R(i, i), W(l, c) = 0 for l > c
        float w[kCP];
#pragma unroll
        for (int i = kCP - 1; i >= 0; --i) {
            float s = (i == lane) ? 1.f : 0.f;
#pragma unroll
            for (int l = i + 1; l < kCP; ++l)
                if (l < nb) s -= Rpp[i * kCP + l] * w[l];
            const float ri = __shfl_sync(0xffffffffu, inv_own, i);
            w[i] = (i <= lane && lane < nb) ? s * ri : 0.f;
        }
        if (lane < nb) {
#pragma unroll
            for (int i = 0; i < kCP; ++i) Wpp[i * kCP + lane] = w[i];
        }
        if (lane == 0 && bad) fail_s = 1;
    };
    // one 4 x 4 tile (a0 <= b0) of the rank-kCP trailing update from the panel buffer
    auto update_tile = [&](int a0, int b0) {
        float acc[4][4] = {};
#pragma unroll
        for (int k = 0; k < kCP; ++k) {
            const float4 pa = *reinterpret_cast<const float4*>(P + k * qp + a0);
            const float4 pb = *reinterpret_cast<const float4*>(P + k * qp + b0);
            const float va[4] = {pa.x, pa.y, pa.z, pa.w}, vb[4] = {pb.x, pb.y, pb.z, pb.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j2 = 0; j2 < 4; ++j2) acc[i][j2] = fmaf(va[i], vb[j2], acc[i][j2]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int a = a0 + i;
            if (a >= q) break;
            const int base = pk(a, a, q) - a;
#pragma unroll
            for (int j2 = 0; j2 < 4; ++j2) {
                const int b = b0 + j2;
                if (b >= a && b < q) U[base + b] -= acc[i][j2];
            }
        }
    };
    if (warp == 0) factor_diag(0);
    __syncthreads();
    for (int c0 = 0; c0 < q; c0 += kCP) {
        const int c1 = min(q, c0 + kCP), nb = c1 - c0;
        if (fail_s) break;
        // B: the panel's rows right of the block, one thread per column: x = W^T U(c0:c1, t)
        for (int tt = c1 + tid; tt < q; tt += blockDim.x) {
            float u[kCP];
#pragma unroll
            for (int k = 0; k < kCP; ++k) u[k] = k < nb ? U[pk(c0 + k, tt, q)] : 0.f;
#pragma unroll
            for (int k = 0; k < kCP; ++k) {
                if (k < nb) {
                    float x = 0.f;
#pragma unroll
                    for (int i = 0; i <= k; ++i) x = fmaf(Wpp[i * kCP + k], u[i], x);
                    P[k * qp + tt] = x;
                    U[pk(c0 + k, tt, q)] = x;
                }
            }
        }
        for (int k = nb + warp; k < kCP; k += nw)   // rows of a short last panel: zero
            for (int tt = lane; tt < qp; tt += 32) P[k * qp + tt] = 0.f;
        __syncthreads();
        // C: trailing update in 4 x 4 tiles (a0 <= b0, both multiples of 4 from c1), tile indices
        // below nt.  Look-ahead: warp 0 updates the next panel's diagonal block (tile indices below
        // kb4) and factors it while warps 1 .. nw-1 update every other tile, rows ia = warp - 1,
        // warp - 1 + (nw - 1), ..., lanes across the row's tiles.
        const int nt = (q - c1 + 3) / 4;
        const int kb4 = min(kCP / 4, nt);
        if (warp == 0) {
            if (nt > 0) {
                if (lane < kb4 * kb4) {
                    const int ia = lane / kb4, ib = lane - ia * kb4;
                    if (ib >= ia) update_tile(c1 + 4 * ia, c1 + 4 * ib);
                }
                __syncwarp();
                factor_diag(c1);
            }
        } else {
            for (int ia = warp - 1; ia < nt; ia += nw - 1) {
                const int ib0 = ia < kb4 ? kb4 : ia;
                for (int ib = ib0 + lane; ib < nt; ib += 32) update_tile(c1 + 4 * ia, c1 + 4 * ib);
            }
        }
        __syncthreads();
    }
    if (fail_s) {
        if (tid == 0) atomicOr(status, RSK_DEV_BOUNDS);
        return;
    }
    // R from the packed factor, column by column (coalesced), zeros below the diagonal
    for (int c = warp; c < q; c += nw)
#pragma unroll 4
        for (int i = lane; i < q; i += 32) R[int64_t(c) * ldr + i] = i <= c ? U[pk(i, c, q)] : 0.f;
}

// Ri = R^{-1} for an upper triangular R (column-major, ldr), blocked over 32 x 32 blocks: k_trinv_diag
// inverts the diagonal blocks (W_II), then k_trinv_blk forms each block column J above its diagonal
// block by block back substitution, X_IJ = -W_II sum_{K=I+1..J} R_IK X_KJ for I = J-1 .. 0 (X_JJ =
// W_JJ): small products without a dependent chain longer than one block.
constexpr int kTB = 32;
constexpr int kXS = kTB * (kTB + 1);   // one 32 x 32 block, column pitch 33
constexpr int kTrinvMax = 880;         // (q / 32) blocks of 4.2 KB of shared memory per CTA

// One warp per diagonal block I (the last one may be partial: padded with the identity): lane c takes
// column c of W_II by back substitution against the block's rows in shared memory (broadcast reads);
// the block goes to Ri's diagonal block, zeros below its diagonal.
__global__ void __launch_bounds__(32) k_trinv_diag(const float* __restrict__ R, int q, int64_t ldr, float* __restrict__ Ri) {
    __shared__ float Rs[kTB][kTB + 1];   // Rs[i][l] = R(i0 + i, i0 + l); then Rs[c][i] = W(i, c)
    const int i0 = blockIdx.x * kTB, lane = threadIdx.x, nb = min(kTB, q - i0);
    for (int l = 0; l < kTB; ++l)
        Rs[lane][l] = (lane < nb && l < nb) ? (lane <= l ? R[int64_t(i0 + l) * ldr + i0 + lane] : 0.f)
                                            : (lane == l ? 1.f : 0.f);
    __syncwarp();
    const float rinv_own = 1.f / Rs[lane][lane];
    float w[kTB];
#pragma unroll
    for (int i = kTB - 1; i >= 0; --i) {
        float s = (i == lane) ? 1.f : 0.f;
#pragma unroll
        for (int l = i + 1; l < kTB; ++l) s -= Rs[i][l] * w[l];
        const float ri = __shfl_sync(0xffffffffu, rinv_own, i);
        w[i] = (i <= lane) ? s * ri : 0.f;
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < kTB; ++i) Rs[lane][i] = w[i];   // Rs[c][i] = W(i, c)
    __syncwarp();
    for (int c = 0; c < nb; ++c)
        if (lane < nb) Ri[int64_t(i0 + c) * ldr + i0 + lane] = Rs[c][lane];
}

// CTA J: block column J of Ri outside its diagonal block.  256 threads; thread t computes rows
// 4 (t % 8) .. + 3 of column t / 8 of a 32 x 32 block.  X blocks live in shared memory (column pitch
// 33), the R blocks and W_II are staged transposed (At[m][r] = A(r, m)), double-buffered, the next one
// loaded while the current one is used.
__global__ void __launch_bounds__(256) k_trinv_blk(const float* __restrict__ R, int q, int64_t ldr, float* __restrict__ Ri) {
    extern __shared__ __align__(16) float xs[];               // (J + 1) blocks: xs[K kXS + c 33 + m] = X_KJ(m, c)
    __shared__ __align__(16) float At[2][kTB * kTB];
    __shared__ float Ss[kXS];                                  // Ss[c 33 + m] = S(m, c)
    const int J = blockIdx.x, tid = threadIdx.x, c = tid >> 3, r0 = (tid & 7) * 4;
    const int j0 = J * kTB;
    // stage element e = tid + 256 k (k < 4) of a block: row r = e & 31 of A, column m = e >> 5
    auto load_r = [&](int I, int K, float (&v)[4]) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = tid + 256 * k, r = e & 31, m = e >> 5;
            const int row = I * kTB + r, col = K * kTB + m;
            v[k] = (row < q && col < q && row <= col) ? R[int64_t(col) * ldr + row] : 0.f;
        }
    };
    auto load_w = [&](int I, float (&v)[4]) {   // W_II from Ri's diagonal block, identity padding
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = tid + 256 * k, r = e & 31, m = e >> 5;
            const int row = I * kTB + r, col = I * kTB + m;
            v[k] = (row < q && col < q) ? (r <= m ? Ri[int64_t(col) * ldr + row] : 0.f) : (r == m ? 1.f : 0.f);
        }
    };
    auto store_a = [&](int b, const float (&v)[4]) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = tid + 256 * k;
            At[b][(e >> 5) * kTB + (e & 31)] = v[k];
        }
    };
    // X_JJ = W_JJ
    {
        float v[4];
        load_w(J, v);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = tid + 256 * k, r = e & 31, m = e >> 5;
            xs[J * kXS + m * (kTB + 1) + r] = v[k];   // X(r, m): column m, row r
        }
    }
    float nxt[4];
    int buf = 0;
    if (J > 0) load_r(J - 1, J, nxt);
    __syncthreads();
    for (int I = J - 1; I >= 0; --I) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int K = I + 1; K <= J + 1; ++K) {
            // K <= J: the product R_IK X_KJ; K = J + 1: W_II, applied to S below
            store_a(buf, nxt);
            __syncthreads();
            if (K < J) load_r(I, K + 1, nxt);
            else if (K == J) load_w(I, nxt);
            else if (I > 0) load_r(I - 1, I, nxt);
            if (K <= J) {
                const float* X = xs + K * kXS + c * (kTB + 1);
#pragma unroll 8
                for (int m = 0; m < kTB; ++m) {
                    const float4 a = *reinterpret_cast<const float4*>(&At[buf][m * kTB + r0]);
                    const float x = X[m];
                    acc[0] = fmaf(a.x, x, acc[0]);
                    acc[1] = fmaf(a.y, x, acc[1]);
                    acc[2] = fmaf(a.z, x, acc[2]);
                    acc[3] = fmaf(a.w, x, acc[3]);
                }
                if (K == J) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) Ss[c * (kTB + 1) + r0 + k] = acc[k];
                }
            } else {
                // At[buf] = W_II (transposed); S complete in Ss (written before this iteration's barrier)
                float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
                for (int m = 0; m < kTB; ++m) {
                    const float4 a = *reinterpret_cast<const float4*>(&At[buf][m * kTB + r0]);
                    const float s = Ss[c * (kTB + 1) + m];
                    o[0] = fmaf(a.x, s, o[0]);
                    o[1] = fmaf(a.y, s, o[1]);
                    o[2] = fmaf(a.z, s, o[2]);
                    o[3] = fmaf(a.w, s, o[3]);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) xs[I * kXS + c * (kTB + 1) + r0 + k] = -o[k];
            }
            buf ^= 1;
        }
    }
    __syncthreads();
    // block column J: rows above the diagonal block from X, rows below it zero
    for (int cc = tid >> 5; cc < kTB; cc += 8) {
        const int col = j0 + cc;
        if (col >= q) break;
        for (int row = tid & 31; row < q; row += 32) {
            if (row < j0) Ri[int64_t(col) * ldr + row] = xs[(row >> 5) * kXS + cc * (kTB + 1) + (row & 31)];
            else if (row >= j0 + kTB) Ri[int64_t(col) * ldr + row] = 0.f;
        }
    }
}

// FP64 variant for the accurate orthonormalisation: R (q x q column-major, ldr) holds G on entry
// (upper triangle read) and its upper Cholesky factor on exit (zeros below); the shift is
// shift_coeff * trace(G).  One CTA; the matrix stays in L2 (read through ld.cg).
__global__ void __launch_bounds__(1024) k_cholesky64(double* __restrict__ R, int q, int64_t ldr, double shift_coeff,
                                                    unsigned int* status) {
    __shared__ double piv_s, shift_s;
    __shared__ int fail_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) {
        double t = 0.0;
        for (int i = 0; i < q; ++i) t += R[int64_t(i) * ldr + i];
        shift_s = shift_coeff * t;
        fail_s = 0;
    }
    __syncthreads();
    for (int i = tid; i < q; i += blockDim.x) R[int64_t(i) * ldr + i] += shift_s;
    __syncthreads();
    for (int j = 0; j < q; ++j) {
        if (tid == 0) {
            const double d = __ldcg(R + int64_t(j) * ldr + j);
            if (!(d > 0.0) || !isfinite(d)) fail_s = 1;
            piv_s = fail_s ? 1.0 : sqrt(d);
            __stcg(R + int64_t(j) * ldr + j, piv_s);
        }
        __syncthreads();
        if (fail_s) break;
        const double rinv = 1.0 / piv_s;
        for (int k = j + 1 + tid; k < q; k += blockDim.x) __stcg(R + int64_t(k) * ldr + j, __ldcg(R + int64_t(k) * ldr + j) * rinv);
        __threadfence_block();
        __syncthreads();
        // trailing update of the upper triangle: R(i, k) -= R(j, i) R(j, k) for j < i <= k; warps take
        // columns k, lanes rows i (contiguous in memory)
        for (int k = j + 1 + warp; k < q; k += nw) {
            const double rjk = __ldcg(R + int64_t(k) * ldr + j);
            for (int i = j + 1 + lane; i <= k; i += 32)
                __stcg(R + int64_t(k) * ldr + i, __ldcg(R + int64_t(k) * ldr + i) - __ldcg(R + int64_t(i) * ldr + j) * rjk);
        }
        __threadfence_block();
        __syncthreads();
    }
    if (fail_s) {
        if (tid == 0) atomicOr(status, RSK_DEV_BOUNDS);
        return;
    }
    for (int k = warp; k < q; k += nw)
        for (int i = k + 1 + lane; i < q; i += 32) R[int64_t(k) * ldr + i] = 0.0;
}

// Ri (float, q x q, ldr) = R^{-1} for the FP64 upper triangular R: back substitution in FP64, one CTA
// per column, the result rounded to FP32 for the FP32 product X R^{-1}.
__global__ void __launch_bounds__(256) k_trinv64(const double* __restrict__ R, int q, int64_t ldr, float* __restrict__ Ri,
                                                double* __restrict__ Ri64) {
    extern __shared__ double x64[];
    const int j = blockIdx.x, tid = threadIdx.x;
    for (int i = tid; i < q; i += blockDim.x) x64[i] = (i == j) ? 1.0 : 0.0;
    __syncthreads();
    for (int i = j; i >= 0; --i) {
        const double xi = x64[i] / R[int64_t(i) * ldr + i];
        __syncthreads();
        if (tid == 0) x64[i] = xi;
        for (int k = tid; k < i; k += blockDim.x) x64[k] -= R[int64_t(i) * ldr + k] * xi;
        __syncthreads();
    }
    for (int i = tid; i < q; i += blockDim.x) {
        Ri[int64_t(j) * ldr + i] = float(x64[i]);
        if (Ri64) Ri64[int64_t(j) * ldr + i] = x64[i];
    }
}

// C (FP64, q x q) = A (FP64 upper, q x q) * B (FP64 upper, q x q): product of two triangular factors.
__global__ void k_trmm64(const double* __restrict__ A, const double* __restrict__ B, int q, double* __restrict__ C) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= int64_t(q) * q) return;
    const int j = int(idx / q), i = int(idx - int64_t(j) * q);
    double t = 0.0;
    for (int l = i; l <= j; ++l) t += A[int64_t(l) * q + i] * B[int64_t(j) * q + l];
    C[idx] = i <= j ? t : 0.0;
}

__global__ void k_to_f32(const double* __restrict__ X, int64_t count, float* __restrict__ Y) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < count) Y[i] = float(X[i]);
}

// ------------------------------------------------------------------------------------------
// One-sided block Jacobi SVD.
// ------------------------------------------------------------------------------------------
struct JacobiArgs {
    float* X;
    int64_t ldx;
    int m, q, nb, w;   // w = columns per block (the last ones may hold fewer)
    float* V;
    int64_t ldv;
    float tol;
    int max_sweeps;
    unsigned int* flags;   // one word per sweep: set when the sweep rotated
    unsigned int* bar;     // grid barrier (2 words)
    unsigned int* status;
    uint32_t limit;
};

// Block held by position p of the round-robin table in round r (position 0 fixed).
__device__ __forceinline__ int rr_block(int pos, int r, int n) { return pos == 0 ? 0 : 1 + (pos - 1 + r) % (n - 1); }

__global__ void __launch_bounds__(1024) k_jacobi(const JacobiArgs a) {
    extern __shared__ __align__(16) float sm[];
    const int g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int mv = a.V ? a.q : 0;          // rows of V's columns
    // a local column: the X part padded to a multiple of 4 floats, then the V part likewise (zeros in
    // the padding stay zero under rotations), so both parts are 16-byte aligned float4 runs
    const int mp = (a.m + 3) & ~3, vp = (mv + 3) & ~3, cl = mp + vp;
    __shared__ int cols_s[256];            // global column of each local column
    __shared__ int nloc_s;
    __shared__ int rot_s;
    for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
        for (int r = 0; r < a.nb - 1; ++r) {
            const int b0 = rr_block(g, r, a.nb), b1 = rr_block(a.nb - 1 - g, r, a.nb);
            if (tid == 0) {
                int n = 0;
                for (int bb = 0; bb < 2; ++bb) {
                    const int b = bb ? b1 : b0;
                    const int c0 = b * a.w, c1 = min(a.q, c0 + a.w);
                    for (int c = c0; c < c1; ++c) cols_s[n++] = c;
                }
                nloc_s = n;
                rot_s = 0;
            }
            __syncthreads();
            const int L = nloc_s;
            // columns another CTA rotated in the previous round: read through L2 (ld.cg), never from
            // a line this SM's L1 may still hold from an earlier round
            // (all threads over the L x cl floats, so that many loads are in flight at once)
#pragma unroll 4
            for (int e = tid; e < L * cl; e += blockDim.x) {
                const int l = e / cl, i = e - l * cl, c = cols_s[l];
                float v = 0.f;
                if (i < a.m) v = __ldcg(a.X + int64_t(c) * a.ldx + i);
                else if (i >= mp && i - mp < mv) v = __ldcg(a.V + int64_t(c) * a.ldv + (i - mp));
                sm[e] = v;
            }
            __syncthreads();
            // one local sweep over every pair of the L columns (round-robin on Le = L rounded up)
            const int Le = L + (L & 1);
            for (int lr = 0; lr < Le - 1; ++lr) {
                for (int pi = warp; pi < Le / 2; pi += nw) {
                    const int pa = rr_block(pi, lr, Le), pb = rr_block(Le - 1 - pi, lr, Le);
                    if (pa >= L || pb >= L) continue;
                    float4* ca = reinterpret_cast<float4*>(sm + pa * cl);
                    float4* cb = reinterpret_cast<float4*>(sm + pb * cl);
                    float al = 0.f, be = 0.f, ga = 0.f;
                    for (int i = lane; i < mp / 4; i += 32) {
                        const float4 x = ca[i], y = cb[i];
                        al = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, al))));
                        be = fmaf(y.x, y.x, fmaf(y.y, y.y, fmaf(y.z, y.z, fmaf(y.w, y.w, be))));
                        ga = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, ga))));
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        al += __shfl_xor_sync(0xffffffffu, al, o);
                        be += __shfl_xor_sync(0xffffffffu, be, o);
                        ga += __shfl_xor_sync(0xffffffffu, ga, o);
                    }
                    if (ga == 0.f || !(fabsf(ga) > a.tol * sqrtf(al) * sqrtf(be))) continue;
                    const float zeta = (be - al) / (2.f * ga);
                    const float t = fabsf(zeta) > 1e15f ? 0.5f / zeta
                                                        : copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
                    const float c = rsqrtf(1.f + t * t), s = c * t;
                    for (int i = lane; i < cl / 4; i += 32) {
                        const float4 x = ca[i], y = cb[i];
                        ca[i] = make_float4(c * x.x - s * y.x, c * x.y - s * y.y, c * x.z - s * y.z, c * x.w - s * y.w);
                        cb[i] = make_float4(s * x.x + c * y.x, s * x.y + c * y.y, s * x.z + c * y.z, s * x.w + c * y.w);
                    }
                    if (lane == 0) rot_s = 1;
                }
                __syncthreads();
            }
            for (int e = tid; e < L * cl; e += blockDim.x) {
                const int l = e / cl, i = e - l * cl, c = cols_s[l];
                if (i < a.m) __stcg(a.X + int64_t(c) * a.ldx + i, sm[e]);
                else if (i >= mp && i - mp < mv) __stcg(a.V + int64_t(c) * a.ldv + (i - mp), sm[e]);
            }
            if (tid == 0 && rot_s) atomicOr(a.flags + sweep, 1u);
            if (!rskd::grid_barrier(a.bar, a.bar + 1, gridDim.x, a.status, a.limit)) return;
        }
        if (*static_cast<volatile unsigned int*>(a.flags + sweep) == 0u) return;  // converged
    }
}

// The same one-sided block Jacobi on one thread-block cluster whose CTAs keep their column blocks in
// shared memory: CTA g holds the blocks at positions g and nb - 1 - g of the round-robin table (nb = 2G
// blocks of w columns, zero columns past q), orthogonalises every pair of its 2w columns, and between
// rounds every block moves to its next position (position 0 fixed, 1..nb-1 rotating: every pair of
// blocks meets once per sweep) through distributed shared memory into the next holder's second buffer,
// between two cluster barriers.  A sweep's "anything rotated" flag is OR-ed into CTA 0's shared memory
// and read by every CTA between two barriers.  No waits other than the cluster barriers.
struct JacobiCArgs {
    float* X;
    int64_t ldx;
    int m, q, w;
    float* V;
    int64_t ldv;
    float tol;
    int max_sweeps;
};

constexpr int kJacobiSweepsMax = 40;

__global__ void __launch_bounds__(1024) k_jacobi_cluster(const JacobiCArgs a) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) float smc[];
    __shared__ int rot_flags[kJacobiSweepsMax];  // CTA 0's copy is the cluster's
    __shared__ int ids[2][2];                    // block id per [buffer][slot]
    __shared__ int rot_s;
    const int G = int(cluster.num_blocks()), g = int(cluster.block_rank()), nb = 2 * G;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int mv = a.V ? a.q : 0;
    const int mp = (a.m + 3) & ~3, vp = (mv + 3) & ~3, cl = mp + vp;
    const int W = a.w;
    const int slot = W * cl;                     // floats per block
    float* buf[2] = {smc, smc + 2 * slot};      // per buffer: slot 0 (position g), slot 1 (position nb - 1 - g)
    for (int i = tid; i < kJacobiSweepsMax; i += blockDim.x) rot_flags[i] = 0;
    if (tid < 2) ids[0][tid] = tid == 0 ? g : nb - 1 - g;
    for (int e = tid; e < 2 * slot; e += blockDim.x) {
        const int sl = e / slot, rem = e - sl * slot, l = rem / cl, i = rem - l * cl;
        const int c = (sl == 0 ? g : nb - 1 - g) * W + l;
        float v = 0.f;
        if (c < a.q) {
            if (i < a.m) v = a.X[int64_t(c) * a.ldx + i];
            else if (i >= mp && i - mp < mv) v = a.V[int64_t(c) * a.ldv + (i - mp)];
        }
        buf[0][e] = v;
    }
    cluster.sync();
    int cur = 0;
    const int Le = 2 * W;
    for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
        if (tid == 0) rot_s = 0;
        __syncthreads();
        for (int r = 0; r < nb - 1; ++r) {
            float* smx = buf[cur];
            for (int lr = 0; lr < Le - 1; ++lr) {
                for (int pi = warp; pi < Le / 2; pi += nw) {
                    const int pa = rr_block(pi, lr, Le), pb = rr_block(Le - 1 - pi, lr, Le);
                    float4* ca = reinterpret_cast<float4*>(smx + pa * cl);
                    float4* cb = reinterpret_cast<float4*>(smx + pb * cl);
                    float al = 0.f, be = 0.f, ga = 0.f;
                    for (int i = lane; i < mp / 4; i += 32) {
                        const float4 x = ca[i], y = cb[i];
                        al = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, al))));
                        be = fmaf(y.x, y.x, fmaf(y.y, y.y, fmaf(y.z, y.z, fmaf(y.w, y.w, be))));
                        ga = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, ga))));
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        al += __shfl_xor_sync(0xffffffffu, al, o);
                        be += __shfl_xor_sync(0xffffffffu, be, o);
                        ga += __shfl_xor_sync(0xffffffffu, ga, o);
                    }
                    if (ga == 0.f || !(fabsf(ga) > a.tol * sqrtf(al) * sqrtf(be))) continue;
                    const float zeta = (be - al) / (2.f * ga);
                    const float t = fabsf(zeta) > 1e15f ? 0.5f / zeta
                                                        : copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
                    const float c = rsqrtf(1.f + t * t), sn = c * t;
                    for (int i = lane; i < cl / 4; i += 32) {
                        const float4 x = ca[i], y = cb[i];
                        ca[i] = make_float4(c * x.x - sn * y.x, c * x.y - sn * y.y, c * x.z - sn * y.z, c * x.w - sn * y.w);
                        cb[i] = make_float4(sn * x.x + c * y.x, sn * x.y + c * y.y, sn * x.z + c * y.z, sn * x.w + c * y.w);
                    }
                    if (lane == 0) rot_s = 1;
                }
                __syncthreads();
            }
            // both blocks to their next positions, into the next holder's other buffer
            for (int sl = 0; sl < 2; ++sl) {
                const int p = sl == 0 ? g : nb - 1 - g;
                const int pn = p == 0 ? 0 : (p == nb - 1 ? 1 : p + 1);
                const int dcta = pn < G ? pn : nb - 1 - pn, dslot = pn < G ? 0 : 1;
                float4* dst = reinterpret_cast<float4*>(cluster.map_shared_rank(buf[cur ^ 1], dcta) + dslot * slot);
                const float4* src = reinterpret_cast<const float4*>(smx + sl * slot);
                for (int e = tid; e < slot / 4; e += blockDim.x) dst[e] = src[e];
                if (tid == 0) cluster.map_shared_rank(&ids[cur ^ 1][0], dcta)[dslot] = ids[cur][sl];
            }
            cluster.sync();
            cur ^= 1;
        }
        if (tid == 0 && rot_s) atomicOr(cluster.map_shared_rank(&rot_flags[sweep], 0), 1);
        cluster.sync();
        const int any = *cluster.map_shared_rank(&rot_flags[sweep], 0);
        cluster.sync();   // every CTA has read the flag before any leaves
        if (!any) break;
    }
    for (int e = tid; e < 2 * slot; e += blockDim.x) {
        const int sl = e / slot, rem = e - sl * slot, l = rem / cl, i = rem - l * cl;
        const int c = ids[cur][sl] * W + l;
        if (c >= a.q) continue;
        if (i < a.m) a.X[int64_t(c) * a.ldx + i] = buf[cur][e];
        else if (i >= mp && i - mp < mv) a.V[int64_t(c) * a.ldv + (i - mp)] = buf[cur][e];
    }
}

__global__ void k_identity(float* __restrict__ V, int q, int64_t ldv) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= int64_t(q) * q) return;
    const int j = int(idx / q), i = int(idx - int64_t(j) * q);
    V[int64_t(j) * ldv + i] = i == j ? 1.f : 0.f;
}

// Column norms of X (one warp per column).
__global__ void k_colnorms(const float* __restrict__ X, int m, int q, int64_t ldx, float* __restrict__ s) {
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (c >= q) return;
    float t = 0.f;
    for (int i = lane; i < m; i += 32) t = fmaf(X[int64_t(c) * ldx + i], X[int64_t(c) * ldx + i], t);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) s[c] = sqrtf(t);
}

// Rank of each column by descending norm (ties by index), one thread per column.
__global__ void k_rank(const float* __restrict__ s, int q, int* __restrict__ rank) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= q) return;
    const float v = s[c];
    int r = 0;
    for (int o = 0; o < q; ++o) r += (s[o] > v) || (s[o] == v && o < c);
    rank[c] = r;
}

// out[:, rank[c]] = X[:, c] * (scale ? 1 / s[c] : 1) (0 where s[c] == 0); s_out[rank[c]] = s[c].
__global__ void k_permute_cols(const float* __restrict__ X, int m, int q, int64_t ldx, const int* __restrict__ rank,
                               const float* __restrict__ s, bool scale, float* __restrict__ out, int64_t ldo,
                               float* __restrict__ s_out) {
    const int c = blockIdx.y;
    const int rc = rank[c];
    const float f = scale ? (s[c] > 0.f ? 1.f / s[c] : 0.f) : 1.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        out[int64_t(rc) * ldo + i] = X[int64_t(c) * ldx + i] * f;
    if (s_out && blockIdx.x == 0 && threadIdx.x == 0) s_out[rc] = s[c];
}

__global__ void k_copy_cols(const float* __restrict__ src, int64_t lds, int m, int q, float* __restrict__ dst,
                            int64_t ldd) {
    const int c = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        dst[int64_t(c) * ldd + i] = src[int64_t(c) * lds + i];
}

struct JacobiPlan {
    int G, nb, w;
    size_t smem;
};
// Columns per block about 10: a local sweep then has ~10 independent pairs per step for a CTA's
// warps, and the sweep's 2G - 1 rounds (each ending in a grid barrier) stay few enough; more blocks
// only while a CTA's 2w columns do not fit in shared memory.
JacobiPlan jacobi_plan(int64_t m, int q, bool with_v, int num_sms) {
    JacobiPlan p;
    const size_t cl = size_t((m + 3) & ~int64_t(3)) + size_t(with_v ? (q + 3) & ~3 : 0);
    p.G = std::max(8, (q + 19) / 20);
    for (;;) {
        p.nb = 2 * p.G;
        p.w = (q + p.nb - 1) / p.nb;
        p.smem = size_t(2 * p.w) * cl * 4;
        if ((p.smem <= 200 * 1024 && 2 * p.w <= 256) || p.G >= 128) break;
        p.G *= 2;
    }
    // blocks of at least one column, and no more CTAs than can be resident
    while (p.G > 1 && (p.nb > q || p.G > num_sms)) {
        p.G /= 2;
        p.nb = 2 * p.G;
        p.w = (q + p.nb - 1) / p.nb;
        p.smem = size_t(2 * p.w) * cl * 4;
    }
    return p;
}

constexpr int kMaxSweeps = 40;

}  // namespace

namespace rsk {
namespace dense {

size_t gram_scratch_bytes(int64_t m, int p, int q) {
    const int64_t nch = (m + kGChunk - 1) / kGChunk;
    const int64_t pp = (p + kGT - 1) / kGT * kGT, qq = (q + kGT - 1) / kGT * kGT;
    return size_t(nch) * size_t(pp * qq) * 4 + 256;
}

template <typename Acc>
rsk_status gram_t(rsk_handle* h, const float* X, int64_t m, int p, int64_t ldx, const float* Y, int q, int64_t ldy,
                  Acc* G, int64_t ldg, void* scratch, cudaStream_t stream) {
    if (m < 1 || p < 1 || q < 1) return fail(h, RSK_ERR_INVALID_ARG, "gram: empty operand");
    const int nch = int((m + kGChunk - 1) / kGChunk);
    const int ntp = (p + kGT - 1) / kGT, ntq = (q + kGT - 1) / kGT;
    const int pp = ntp * kGT;
    const int64_t pstride = int64_t(pp) * (int64_t(ntq) * kGT);
    const bool sym = (X == Y) && (p == q) && (ldx == ldy);
    Acc* part = static_cast<Acc*>(scratch);
    k_gram<Acc><<<dim3(unsigned(ntp * ntq), unsigned(nch)), 256, 0, stream>>>(X, m, p, ldx, Y, q, ldy, sym, ntq, part,
                                                                              pstride, pp);
    RSK_LAUNCH_CHECK(h);
    const int64_t tot = int64_t(p) * q;
    k_gram_reduce<Acc><<<unsigned((tot + 255) / 256), 256, 0, stream>>>(part, pstride, nch, p, q, pp, sym, G, ldg);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

rsk_status gram64(rsk_handle* h, const float* X, int64_t m, int p, int64_t ldx, const float* Y, int q, int64_t ldy,
                  double* G, int64_t ldg, void* scratch, cudaStream_t stream) {
    return gram_t<double>(h, X, m, p, ldx, Y, q, ldy, G, ldg, scratch, stream);
}

rsk_status matmul_ts(rsk_handle* h, const float* X, int64_t m, int p, int64_t ldx, const float* M, int q,
                     int64_t ldm, float* C, int64_t ldc, cudaStream_t stream) {
    if (m < 1 || p < 1 || q < 1) return fail(h, RSK_ERR_INVALID_ARG, "matmul: empty operand");
    const dim3 grid(unsigned((m + kMR - 1) / kMR), unsigned((q + kMC - 1) / kMC));
    k_matmul_ts<<<grid, 256, 0, stream>>>(X, m, p, ldx, M, q, ldm, C, ldc);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

rsk_status cholesky(rsk_handle* h, const float* G, int q, int64_t ldg, float shift_coeff, float* R, int64_t ldr,
                    cudaStream_t stream) {
    if (q < 1 || q > kCholMax) return fail(h, RSK_ERR_UNSUPPORTED, "cholesky supports 1 <= q <= %d (got %d)", kCholMax, q);
    const int panel = q <= 320 ? 16 : 8;
    const int smem = int(((size_t(q) * (q + 1) / 2 + 3) / 4 * 4 + size_t(panel) * ((q + 3) & ~3)) * 4);
    auto go = [&](auto kern) -> rsk_status {
        RSK_CUDA_TRY(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        kern<<<1, kCholThreads, smem, stream>>>(G, q, ldg, shift_coeff, R, ldr, h->dev_status);
        RSK_LAUNCH_CHECK(h);
        return RSK_OK;
    };
    return panel == 16 ? go(k_cholesky<16>) : go(k_cholesky<8>);
}

rsk_status trinv(rsk_handle* h, const float* R, int q, int64_t ldr, float* Ri, cudaStream_t stream) {
    if (q < 1 || q > kTrinvMax) return fail(h, RSK_ERR_UNSUPPORTED, "trinv supports 1 <= q <= %d (got %d)", kTrinvMax, q);
    const int nblk = (q + kTB - 1) / kTB;
    const int smem = nblk * kXS * 4;
    k_trinv_diag<<<unsigned(nblk), kTB, 0, stream>>>(R, q, ldr, Ri);
    RSK_LAUNCH_CHECK(h);
    RSK_CUDA_TRY(h, cudaFuncSetAttribute(k_trinv_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_trinv_blk<<<unsigned(nblk), 256, smem, stream>>>(R, q, ldr, Ri);
    RSK_LAUNCH_CHECK(h);
    return RSK_OK;
}

size_t svd_scratch_bytes(int64_t m, int q) {
    return Carver::round(size_t(m) * q * 4) + Carver::round(size_t(q) * q * 4) + 2 * Carver::round(size_t(q) * 8) +
           Carver::round(size_t(kMaxSweeps + 2) * 4) + 1024;
}

rsk_status svd(rsk_handle* h, float* X, int64_t m, int q, int64_t ldx, float* s, float* V, int64_t ldv, void* scratch,
               cudaStream_t stream) {
    if (q < 1 || q > 1024 || m < q || m > 4096)
        return fail(h, RSK_ERR_UNSUPPORTED, "svd supports 1 <= q <= 1024, q <= m <= 4096 (got m=%lld, q=%d)",
                    (long long)m, q);
    Carver cv(scratch);
    float* Ut = cv.take<float>(size_t(m) * q);
    float* Vt = cv.take<float>(size_t(q) * q);
    float* sn = cv.take<float>(size_t(q));
    float* vn = cv.take<float>(size_t(q));
    int* rank = cv.take<int>(size_t(q));
    unsigned int* words = cv.take<unsigned int>(size_t(kMaxSweeps + 2));
    // V starts as the identity (held in Vt), then rotates with X
    const bool with_v = V != nullptr;
    if (with_v) {
        k_identity<<<unsigned((int64_t(q) * q + 255) / 256), 256, 0, stream>>>(Vt, q, q);
        RSK_LAUNCH_CHECK(h);
    }
    RSK_CUDA_TRY(h, cudaMemsetAsync(words, 0, size_t(kMaxSweeps + 2) * 4, stream));
    bool done = false;
    if (q > 1) {
        // one cluster of G <= 16 CTAs (about 10 columns per block) when the columns fit in their shared
        // memory (two buffers of two blocks per CTA)
        const int64_t clw = ((m + 3) & ~int64_t(3)) + (with_v ? ((q + 3) & ~3) : 0);
        for (int G : {std::min(16, std::max(2, (q + 19) / 20)), 8}) {
            if (done || 2 * G > q) continue;
            const int w = (q + 2 * G - 1) / (2 * G);
            const size_t smem = size_t(4) * w * size_t(clw) * 4;
            if (smem > 200 * 1024) continue;
            RSK_CUDA_TRY(h, cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
            if (G > 8) RSK_CUDA_TRY(h, cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(unsigned(G));
            cfg.blockDim = dim3(1024);
            cfg.dynamicSmemBytes = smem;
            cfg.stream = stream;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = unsigned(G);
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int clusters = 0;
            if (cudaOccupancyMaxActiveClusters(&clusters, k_jacobi_cluster, &cfg) != cudaSuccess || clusters < 1) {
                cudaGetLastError();
                continue;
            }
            JacobiCArgs ca;
            ca.X = X;
            ca.ldx = ldx;
            ca.m = int(m);
            ca.q = q;
            ca.w = w;
            ca.V = with_v ? Vt : nullptr;
            ca.ldv = q;
            ca.tol = 2.f * sqrtf(float(m)) * kU32;
            ca.max_sweeps = std::min(kMaxSweeps, kJacobiSweepsMax);
            RSK_CUDA_TRY(h, cudaLaunchKernelEx(&cfg, k_jacobi_cluster, ca));
            done = true;
        }
    }
    if (q > 1 && !done) {
        const JacobiPlan jp = jacobi_plan(m, q, with_v, h->num_sms);
        if (jp.smem > 227 * 1024 || 2 * jp.w > 256)
            return fail(h, RSK_ERR_UNSUPPORTED, "svd: %lld x %d needs too much shared memory", (long long)m, q);
        JacobiArgs ja;
        ja.X = X;
        ja.ldx = ldx;
        ja.m = int(m);
        ja.q = q;
        ja.nb = jp.nb;
        ja.w = jp.w;
        ja.V = with_v ? Vt : nullptr;
        ja.ldv = q;
        ja.tol = 2.f * sqrtf(float(m)) * kU32;
        ja.max_sweeps = kMaxSweeps;
        ja.flags = words;
        ja.bar = words + kMaxSweeps;
        ja.status = h->dev_status;
        ja.limit = h->wait_limit;
        RSK_CUDA_TRY(h, cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, int(jp.smem)));
        int per_sm = 0;
        RSK_CUDA_TRY(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi, 1024, jp.smem));
        if (per_sm * h->num_sms < jp.G) return fail(h, RSK_ERR_UNSUPPORTED, "svd: %d CTAs cannot be resident", jp.G);
        void* args[] = {&ja};
        RSK_CUDA_TRY(h, cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k_jacobi), dim3(jp.G), dim3(1024), args,
                                                    jp.smem, stream));
    }
    k_colnorms<<<unsigned((q + 7) / 8), 256, 0, stream>>>(X, int(m), q, ldx, sn);
    k_rank<<<unsigned((q + 255) / 256), 256, 0, stream>>>(sn, q, rank);
    RSK_LAUNCH_CHECK(h);
    const unsigned gx = unsigned(std::min<int64_t>(8, (m + 255) / 256));
    k_permute_cols<<<dim3(gx, unsigned(q)), 256, 0, stream>>>(X, int(m), q, ldx, rank, sn, true, Ut, m, s);
    k_copy_cols<<<dim3(gx, unsigned(q)), 256, 0, stream>>>(Ut, m, int(m), q, X, ldx);
    RSK_LAUNCH_CHECK(h);
    if (with_v) {
        // V's columns drift from unit length by the rounding of many FP32 rotations (their mutual
        // orthogonality holds to a few u); renormalise them while permuting
        k_colnorms<<<unsigned((q + 7) / 8), 256, 0, stream>>>(Vt, q, q, q, vn);
        const unsigned gv = unsigned(std::min(8, (q + 255) / 256));
        k_permute_cols<<<dim3(gv, unsigned(q)), 256, 0, stream>>>(Vt, q, q, q, rank, vn, true, V, ldv, nullptr);
        RSK_LAUNCH_CHECK(h);
    }
    return RSK_OK;
}

size_t orth_scratch_bytes(int64_t m, int q) {
    return 2 * Carver::round(gram_scratch_bytes(m, q, q)) + 4 * Carver::round(size_t(q) * q * 4) +
           4 * Carver::round(size_t(q) * q * 8) + Carver::round(size_t(m) * q * 4) + 1024;
}

rsk_status orth_accurate(rsk_handle* h, float* X, int64_t m, int q, int64_t ldx, float* R, void* scratch,
                         cudaStream_t stream) {
    if (q < 1 || q > 1024 || m < q)
        return fail(h, RSK_ERR_UNSUPPORTED, "orth supports 1 <= q <= 1024, m >= q (got m=%lld, q=%d)", (long long)m, q);
    Carver cv(scratch);
    void* gs = cv.take<char>(2 * gram_scratch_bytes(m, q, q));
    double* G = cv.take<double>(size_t(q) * q);
    double* R64 = cv.take<double>(size_t(q) * q);
    double* Racc = cv.take<double>(size_t(q) * q);
    double* Rtmp = cv.take<double>(size_t(q) * q);
    float* Ri = cv.take<float>(size_t(q) * q);
    float* T = cv.take<float>(size_t(m) * q);
    // Cholesky QR2 with the Gram in FP64 (exact products of the FP32 entries, FP64 sums): a relative
    // shift of 8 q u_64 keeps the first factorisation defined for kappa(X) up to ~1e7; the second
    // round restores orthogonality to O(u_32)
    const double coeff[2] = {8.0 * q * 1.1102230246251565e-16, 0.0};
    for (int round = 0; round < 2; ++round) {
        rsk_status st = gram64(h, X, m, q, ldx, X, q, ldx, G, q, gs, stream);
        if (st != RSK_OK) return st;
        RSK_CUDA_TRY(h, cudaMemcpyAsync(R64, G, size_t(q) * q * 8, cudaMemcpyDeviceToDevice, stream));
        k_cholesky64<<<1, 1024, 0, stream>>>(R64, q, q, coeff[round], h->dev_status);
        k_trinv64<<<unsigned(q), 256, size_t(q) * 8, stream>>>(R64, q, q, Ri, nullptr);
        RSK_LAUNCH_CHECK(h);
        st = matmul_ts(h, X, m, q, ldx, Ri, q, q, T, m, stream);
        if (st != RSK_OK) return st;
        const unsigned gx = unsigned(std::min<int64_t>(64, (m + 255) / 256));
        k_copy_cols<<<dim3(gx, unsigned(q)), 256, 0, stream>>>(T, m, int(m), q, X, ldx);
        RSK_LAUNCH_CHECK(h);
        if (R) {
            if (round == 0) {
                RSK_CUDA_TRY(h, cudaMemcpyAsync(Racc, R64, size_t(q) * q * 8, cudaMemcpyDeviceToDevice, stream));
            } else {
                k_trmm64<<<unsigned((int64_t(q) * q + 255) / 256), 256, 0, stream>>>(R64, Racc, q, Rtmp);
                RSK_LAUNCH_CHECK(h);
                RSK_CUDA_TRY(h, cudaMemcpyAsync(Racc, Rtmp, size_t(q) * q * 8, cudaMemcpyDeviceToDevice, stream));
            }
        }
    }
    if (R) {
        k_to_f32<<<unsigned((int64_t(q) * q + 255) / 256), 256, 0, stream>>>(Racc, int64_t(q) * q, R);
        RSK_LAUNCH_CHECK(h);
    }
    return RSK_OK;
}

}  // namespace dense
}  // namespace rsk

extern "C" {

rsk_status rsk_svd_econ(rsk_handle* h, const float* A, int64_t m, int64_t q, int64_t lda, float* U, int64_t ldu,
                        float* s, float* V, int64_t ldv, cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    if (!A || !U || !s) return rsk::fail(h, RSK_ERR_INVALID_ARG, "null pointer");
    if (q < 1 || m < q || lda < m || ldu < m || (V && ldv < q))
        return rsk::fail(h, RSK_ERR_INVALID_ARG, "need 1 <= q <= m, lda >= m, ldu >= m, ldv >= q");
    if (q > 1024 || m > 4096) return rsk::fail(h, RSK_ERR_UNSUPPORTED, "svd_econ supports q <= 1024, m <= 4096");
    const size_t need = rsk::dense::svd_scratch_bytes(m, int(q)) + 256;
    rsk_status st = rsk::ensure_workspace(h, need, stream);
    if (st != RSK_OK) return st;
    RSK_CUDA_TRY(h, cudaMemcpy2DAsync(U, size_t(ldu) * 4, A, size_t(lda) * 4, size_t(m) * 4, size_t(q),
                                      cudaMemcpyDeviceToDevice, stream));
    return rsk::dense::svd(h, U, m, int(q), ldu, s, V, ldv, h->ws, stream);
}

rsk_status rsk_qr_econ(rsk_handle* h, const float* X, int64_t m, int64_t q, int64_t ldx, float* Q, int64_t ldq,
                       float* R, cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    if (!X || !Q) return rsk::fail(h, RSK_ERR_INVALID_ARG, "null pointer");
    if (q < 1 || m < q || ldx < m || ldq < m) return rsk::fail(h, RSK_ERR_INVALID_ARG, "need 1 <= q <= m, ldx, ldq >= m");
    if (q > 1024) return rsk::fail(h, RSK_ERR_UNSUPPORTED, "qr_econ supports q <= 1024");
    rsk_status st = rsk::ensure_workspace(h, rsk::dense::orth_scratch_bytes(m, int(q)) + 256, stream);
    if (st != RSK_OK) return st;
    RSK_CUDA_TRY(h, cudaMemcpy2DAsync(Q, size_t(ldq) * 4, X, size_t(ldx) * 4, size_t(m) * 4, size_t(q),
                                      cudaMemcpyDeviceToDevice, stream));
    return rsk::dense::orth_accurate(h, Q, m, int(q), ldq, R, h->ws, stream);
}

rsk_status rsk_cholesky(rsk_handle* h, const float* G, int64_t q, int64_t ldg, float shift_coeff, float* R,
                        int64_t ldr, cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    if (!G || !R) return rsk::fail(h, RSK_ERR_INVALID_ARG, "null pointer");
    if (q < 1 || ldg < q || ldr < q) return rsk::fail(h, RSK_ERR_INVALID_ARG, "need q >= 1, ldg, ldr >= q");
    const int pr = rsk::prof_begin(h, stream, RSK_KERNEL_FACTOR);
    const rsk_status st = rsk::dense::cholesky(h, G, int(q), ldg, shift_coeff, R, ldr, stream);
    rsk::prof_end(h, stream, pr);
    return st;
}

rsk_status rsk_trinv(rsk_handle* h, const float* R, int64_t q, int64_t ldr, float* Ri, cudaStream_t stream) {
    if (!h) return RSK_ERR_INVALID_ARG;
    if (!R || !Ri) return rsk::fail(h, RSK_ERR_INVALID_ARG, "null pointer");
    if (q < 1 || ldr < q) return rsk::fail(h, RSK_ERR_INVALID_ARG, "need q >= 1, ldr >= q");
    const int pr = rsk::prof_begin(h, stream, RSK_KERNEL_DENSE);
    const rsk_status st = rsk::dense::trinv(h, R, int(q), ldr, Ri, stream);
    rsk::prof_end(h, stream, pr);
    return st;
}

}  // extern "C"
