// Per-atom Born-charge network: features, BF16-weight forward and backward, AdamW training.
//
// The paper's dipole derivatives come from finite differences ("the computational bottleneck",
// Results) or from Mulliken charges (cheap, non-conservative, heating). This network stands in for
// them. Per atom j of a cell:
//   x_j (32): 11 Gaussian radial terms per neighbour element (centres 0.8 + 0.7 a bohr, width
//             exp(-2 (r - mu)^2)), 8 angular terms 2^(1-z) sum_{k<l} (1 + lam cos theta)^z
//             exp(-0.05 (r_k^2 + r_l^2)) fc fc for z in {1,2,4,8}, lam = +-1, element one-hot;
//             cosine cutoff fc at 8 bohr, neighbours = the other atoms of the cell;
//   R_j      : rows e1 (to the nearest neighbour), e2 (second-nearest, orthogonalised), e3 = e1 x e2;
//   y_j      : W3 silu(W2 silu(W1 x + b1) + b2) + b3, 32 -> 128 -> 128 -> 9, BF16 weights, FP32 math;
//   Z_j      = Q_j I + R_j^T T_j R_j - mean over the cell (T_j = y_j as 3 x 3), so the sum rule
//              sum_j Z_j = Q_cell I holds and a zero network is the Mulliken model;
//   b_j      = pol^T Z_j.
// Training minimises sum |Z - Z_ref|^2 / (9 n_atoms) with AdamW on FP32 master weights; the
// gradient reduction over atom tiles is a fixed-order sum (bitwise reproducible).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <random>
#include <string>
#include <vector>

#include "cavmd_internal.cuh"
#include "tc_common.cuh"

namespace {

constexpr int NF = CAVMD_MLP_NFEAT;
constexpr int NH = CAVMD_MLP_HIDDEN;
constexpr int NO = 9;
constexpr int OFF_W1 = 0, OFF_B1 = NH * NF, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NO * NH, NPAR = OFF_B3 + NO;
static_assert(NPAR == CAVMD_MLP_NPARAMS, "parameter count");
constexpr int TILE = 16;          // atoms per block in the forward and backward kernels
constexpr float RC = 8.0f;

__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}
__device__ __forceinline__ float fcut(float r) { return r < RC ? 0.5f * (cospif(r / RC) + 1.0f) : 0.0f; }
__device__ __forceinline__ float wv(const __nv_bfloat16 *w, int i) { return __bfloat162float(w[i]); }

// features (n_atoms x 32) and frames (n_atoms x 9, rows e1 e2 e3) of every atom; thread per atom
__global__ void k_features(int n_cells, const int *__restrict__ off, const int *__restrict__ species,
                           const double *__restrict__ r, float *__restrict__ X, float *__restrict__ R,
                           unsigned *__restrict__ status) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const int a0 = off[c], a1 = off[c + 1];
    for (int j = a0; j < a1; ++j) {
        float x[NF];
        for (int i = 0; i < NF; ++i) x[i] = 0.0f;
        int k1 = -1, k2 = -1;
        float r1 = 1e30f, r2 = 1e30f;
        for (int k = a0; k < a1; ++k) {
            if (k == j) continue;
            const float dx = (float)(r[3 * k] - r[3 * j]), dy = (float)(r[3 * k + 1] - r[3 * j + 1]),
                        dz = (float)(r[3 * k + 2] - r[3 * j + 2]);
            const float rk = sqrtf(dx * dx + dy * dy + dz * dz);
            if (!(rk < RC)) continue;
            const float fc = fcut(rk);
            const int e = species[k];   // radial channels: O (0) and H (1); every index below is constant
            const float w0 = e == 0 ? fc : 0.0f, w1 = e == 1 ? fc : 0.0f;
#pragma unroll
            for (int a = 0; a < 11; ++a) {
                const float t = rk - (0.8f + 0.7f * a);
                const float g = __expf(-2.0f * t * t);
                x[a] = fmaf(g, w0, x[a]);
                x[11 + a] = fmaf(g, w1, x[11 + a]);
            }
            if (rk < r1 || (rk == r1 && k < k1)) { r2 = r1; k2 = k1; r1 = rk; k1 = k; }
            else if (rk < r2 || (rk == r2 && k < k2)) { r2 = rk; k2 = k; }
            for (int l = k + 1; l < a1; ++l) {
                if (l == j) continue;
                const float ex = (float)(r[3 * l] - r[3 * j]), ey = (float)(r[3 * l + 1] - r[3 * j + 1]),
                            ez = (float)(r[3 * l + 2] - r[3 * j + 2]);
                const float rl = sqrtf(ex * ex + ey * ey + ez * ez);
                if (!(rl < RC)) continue;
                const float cs = (dx * ex + dy * ey + dz * ez) / (rk * rl);
                const float rad = __expf(-0.05f * (rk * rk + rl * rl)) * fc * fcut(rl);
                // 2^(1-z) (1 +- cos)^z for z = 1, 2, 4, 8: powers by repeated squaring
                const float pre[4] = {1.0f, 0.5f, 0.125f, 0.0078125f};   // 2^(1-z)
                float pp = 1.0f + cs, pm = fmaxf(1.0f - cs, 0.0f);
#pragma unroll
                for (int zi = 0; zi < 4; ++zi) {
                    if (zi > 0) {
                        pp *= pp;
                        pm *= pm;
                    }
                    x[22 + 2 * zi] = fmaf(pre[zi] * pp, rad, x[22 + 2 * zi]);
                    x[22 + 2 * zi + 1] = fmaf(pre[zi] * pm, rad, x[22 + 2 * zi + 1]);
                }
            }
        }
        x[30] = species[j] == 0 ? 1.0f : 0.0f;
        x[31] = species[j] == 1 ? 1.0f : 0.0f;
        float4 *Xj = reinterpret_cast<float4 *>(X + (size_t)j * NF);
#pragma unroll
        for (int i = 0; i < NF / 4; ++i) Xj[i] = make_float4(x[4 * i], x[4 * i + 1], x[4 * i + 2], x[4 * i + 3]);
        float fr[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        if (k2 >= 0) {
            float e1[3], v[3];
            for (int q = 0; q < 3; ++q) {
                e1[q] = (float)(r[3 * k1 + q] - r[3 * j + q]) / r1;
                v[q] = (float)(r[3 * k2 + q] - r[3 * j + q]);
            }
            const float ve = v[0] * e1[0] + v[1] * e1[1] + v[2] * e1[2];
            for (int q = 0; q < 3; ++q) v[q] -= ve * e1[q];
            const float vn = rsqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            const float e2[3] = {v[0] * vn, v[1] * vn, v[2] * vn};
            const float e3[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                                 e1[0] * e2[1] - e1[1] * e2[0]};
            for (int q = 0; q < 3; ++q) {
                fr[q] = e1[q];
                fr[3 + q] = e2[q];
                fr[6 + q] = e3[q];
            }
        } else {
            atomicOr(status, (unsigned)ERRBIT_NONFINITE);   // a frame needs two neighbours
        }
        for (int q = 0; q < 9; ++q) R[(size_t)j * 9 + q] = fr[q];
    }
}

// forward over a tile of TILE atoms: Zl = R^T T R; with `store`, keeps z1, z2, h1, h2 for backward
__global__ void __launch_bounds__(NH) k_forward(int n, const float *__restrict__ X, const float *__restrict__ R,
                                                const __nv_bfloat16 *__restrict__ w, float *__restrict__ Zl,
                                                float *__restrict__ z1g, float *__restrict__ z2g,
                                                float *__restrict__ h1g, float *__restrict__ h2g) {
    __shared__ float xs[TILE][NF + 1];
    __shared__ float h1[TILE][NH + 1];
    __shared__ float h2[TILE][NH + 1];
    __shared__ float ys[TILE][NO];
    const int t0 = blockIdx.x * TILE;
    const int u = threadIdx.x;
    for (int e = u; e < TILE * NF; e += NH) {
        const int a = e / NF, i = e - a * NF;
        xs[a][i] = (t0 + a < n) ? X[(size_t)(t0 + a) * NF + i] : 0.0f;
    }
    __syncthreads();
    {
        float wr[NF];
        for (int i = 0; i < NF; ++i) wr[i] = wv(w, OFF_W1 + u * NF + i);
        const float b = wv(w, OFF_B1 + u);
        for (int a = 0; a < TILE; ++a) {
            float z = b;
#pragma unroll
            for (int i = 0; i < NF; ++i) z = fmaf(wr[i], xs[a][i], z);
            h1[a][u] = silu(z);
            if (z1g && t0 + a < n) z1g[(size_t)(t0 + a) * NH + u] = z;
        }
    }
    __syncthreads();
    {
        float acc[TILE];
        const float b = wv(w, OFF_B2 + u);
        for (int a = 0; a < TILE; ++a) acc[a] = b;
        for (int v0 = 0; v0 < NH; v0 += 16) {
            float wr[16];
#pragma unroll
            for (int t = 0; t < 16; ++t) wr[t] = wv(w, OFF_W2 + u * NH + v0 + t);
#pragma unroll
            for (int a = 0; a < TILE; ++a)
#pragma unroll
                for (int t = 0; t < 16; ++t) acc[a] = fmaf(wr[t], h1[a][v0 + t], acc[a]);
        }
        for (int a = 0; a < TILE; ++a) {
            h2[a][u] = silu(acc[a]);
            if (z2g && t0 + a < n) {
                z2g[(size_t)(t0 + a) * NH + u] = acc[a];
                h1g[(size_t)(t0 + a) * NH + u] = h1[a][u];
            }
        }
    }
    __syncthreads();
    if (h2g)
        for (int a = 0; a < TILE; ++a)
            if (t0 + a < n) h2g[(size_t)(t0 + a) * NH + u] = h2[a][u];
    for (int e = u; e < TILE * NO; e += NH) {
        const int a = e / NO, o = e - a * NO;
        float y = wv(w, OFF_B3 + o);
        for (int v = 0; v < NH; ++v) y = fmaf(wv(w, OFF_W3 + o * NH + v), h2[a][v], y);
        ys[a][o] = y;
    }
    __syncthreads();
    if (u < TILE && t0 + u < n) {
        const float *Rj = R + (size_t)(t0 + u) * 9;
        // Zl[i][k] = sum_{a,b} R[a][i] T[a][b] R[b][k]
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) {
                float s = 0.0f;
                for (int aa = 0; aa < 3; ++aa)
                    for (int bb = 0; bb < 3; ++bb) s = fmaf(Rj[3 * aa + i] * ys[u][3 * aa + bb], Rj[3 * bb + k], s);
                Zl[(size_t)(t0 + u) * 9 + 3 * i + k] = s;
            }
    }
}

// Inference forward for the time step on the fifth-generation tensor cores (tcgen05). A tile of
// 128 atoms sits on the 128 TMEM lanes and each layer is one BF16 MMA chain D = A B^T with FP32
// accumulation in TMEM:
//   A = the layer input, 128 atoms x K, split into three BF16 parts: hi + mid + lo carries a
//       float's 24-bit significand, so A B^T equals the FP32 products to accumulation rounding;
//   B = the layer's BF16 weights (exact), N outputs x K, K-major core matrices.
// L1: K = 32, N = 128 into TMEM columns 0..127; L2: K = 128, N = 128 into columns 128..255;
// L3: K = 128, N = 16 (the 9 outputs, zero-padded) into columns 0..15, free again once L1's
// epilogue has read them. The epilogues read TMEM (warp w of 16: lanes 32 (w mod 4) .. + 31,
// columns 32 (w div 4) .. + 31), add the bias, apply silu and write the next layer's split operand to
// shared memory; the last forms Zl = R^T T R for its atom. One persistent CTA per SM loads the
// weights once; every mbarrier wait is bounded (timeout: status bit, TMEM still released).
constexpr int MT = 128;                              // atoms per tile = TMEM lanes
constexpr int FWD_THREADS = 512;                     // 16 warps: four per TMEM lane quadrant
constexpr uint32_t LBO_A = (MT / 8) * 128;           // A operand: K-group stride (128 rows)
constexpr uint32_t LBO_W = (NH / 8) * 128;           // W1, W2: 128 rows
constexpr uint32_t LBO_W3 = (16 / 8) * 128;          // W3 padded to 16 rows
constexpr uint32_t A_SPLIT = MT * NH * 2;            // one BF16 part of A, K up to 128
constexpr uint32_t SW1 = NH * NF * 2, SW2 = NH * NH * 2, SW3 = 16 * NH * 2;
constexpr size_t FWD_SMEM = SW1 + SW2 + SW3 + 3 * (size_t)A_SPLIT + (2 * NH + 16) * 4 + 64;
static_assert(NF % 16 == 0 && NH % 16 == 0, "MMA K steps of 16");

// Two floats -> two BF16 (round to nearest even, one packed conversion) and their exact remainders.
__device__ __forceinline__ uint32_t bf16x2_split(float &a, float &b) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
    const uint32_t u = *reinterpret_cast<const uint32_t *>(&p);
    a -= __uint_as_float(u << 16);              // low half holds a
    b -= __uint_as_float(u & 0xffff0000u);
    return u;
}

// 8 consecutive K of one row of A, split into hi / mid / lo BF16 parts (16 bytes each).
__device__ __forceinline__ void split_store8(uint8_t *sa, uint32_t off, const float (&x)[8]) {
    float r[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) r[q] = x[q];
    uint4 part[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        part[s].x = bf16x2_split(r[0], r[1]);
        part[s].y = bf16x2_split(r[2], r[3]);
        part[s].z = bf16x2_split(r[4], r[5]);
        part[s].w = bf16x2_split(r[6], r[7]);
    }
    *reinterpret_cast<uint4 *>(sa + off) = part[0];
    *reinterpret_cast<uint4 *>(sa + A_SPLIT + off) = part[1];
    *reinterpret_cast<uint4 *>(sa + 2 * A_SPLIT + off) = part[2];
}

// silu with the reciprocal of the special-function unit (the training kernels divide exactly; the
// two differ by a few ulp)
__device__ __forceinline__ float silu_fast(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

// BF16 weights [rows][K] (row-major in the parameter vector) into the K-major core-matrix layout;
// rows >= nrows are zero.
__device__ __forceinline__ void load_weights(uint8_t *dst, const uint16_t *src, int rows, int nrows, int K,
                                             uint32_t lbo) {
    for (int c = threadIdx.x; c < rows * (K / 8); c += blockDim.x) {
        const int g = c / rows, row = c - g * rows;
        __align__(16) uint16_t v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = row < nrows ? src[row * K + 8 * g + q] : (uint16_t)0;
        *reinterpret_cast<uint4 *>(dst + tc::core_offset(row, 8 * g, lbo)) = *reinterpret_cast<const uint4 *>(v);
    }
}

// One layer's MMA chain (thread 0): D (+)= sum over K steps and the three parts of A.
__device__ __forceinline__ void layer_mma(uint32_t tmem_d, uint32_t sa, uint32_t sw, uint32_t lbo_w, int K,
                                          uint32_t idesc) {
    for (int k = 0; k < K / 16; ++k) {
        const uint64_t bd = tc::make_desc(sw + (uint32_t)k * 2 * lbo_w, lbo_w, 128);
#pragma unroll
        for (int s = 0; s < 3; ++s)
            tc::mma_bf16(tmem_d, tc::make_desc(sa + s * A_SPLIT + (uint32_t)k * 2 * LBO_A, LBO_A, 128), bd, idesc,
                         (k > 0 || s > 0) ? 1u : 0u);
    }
}

// Hidden-layer epilogue: 32 TMEM columns of this thread's atom -> silu(d + b) -> split A operand.
__device__ __forceinline__ void hidden_epilogue(uint32_t taddr, int col0, const float *b, uint8_t *sa, int row) {
    float v[32];
    tc::tmem_ld32(taddr, v);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        float x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) x[q] = silu_fast(v[8 * g + q] + b[col0 + 8 * g + q]);
        split_store8(sa, tc::core_offset(row, col0 + 8 * g, LBO_A), x);
    }
}

__global__ void __launch_bounds__(FWD_THREADS, 1) k_forward_tc(int n, const float *__restrict__ X,
                                                             const float *__restrict__ R,
                                                             const __nv_bfloat16 *__restrict__ w,
                                                             float *__restrict__ Zl, unsigned *__restrict__ status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sw1 = smem, *sw2 = sw1 + SW1, *sw3 = sw2 + SW2, *sa = sw3 + SW3;   // sa: [hi][mid][lo]
    float *bias = reinterpret_cast<float *>(sa + 3 * A_SPLIT);                  // b1 [128] b2 [128] b3 [16]
    uint64_t *done = reinterpret_cast<uint64_t *>(bias + 2 * NH + 16);
    uint32_t *slot = reinterpret_cast<uint32_t *>(done + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(slot, 256);
    if (tid == 0) tc::mbar_init(done, 1);
    const uint16_t *wr = reinterpret_cast<const uint16_t *>(w);
    load_weights(sw1, wr + OFF_W1, NH, NH, NF, LBO_W);
    load_weights(sw2, wr + OFF_W2, NH, NH, NH, LBO_W);
    load_weights(sw3, wr + OFF_W3, 16, NO, NH, LBO_W3);
    for (int e = tid; e < 2 * NH + 16; e += FWD_THREADS)
        bias[e] = e < 2 * NH ? wv(w, (e < NH ? OFF_B1 : OFF_B2 - NH) + e) : (e - 2 * NH < NO ? wv(w, OFF_B3 + e - 2 * NH) : 0.0f);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t sa_u = tc::smem_u32(sa), sw1_u = tc::smem_u32(sw1), sw2_u = tc::smem_u32(sw2),
                   sw3_u = tc::smem_u32(sw3);
    const uint32_t quad = warp & 3, slice = warp >> 2;   // lane quadrant; 32-column slice
    const uint32_t lanes = tmem + ((32u * quad) << 16);   // this warp's TMEM lanes
    const int row = 32 * quad + lane;                      // this thread's atom in the tile
    const float *b1 = bias, *b2 = bias + NH, *b3 = bias + 2 * NH;
    constexpr uint32_t ID128 = tc::idesc_bf16(MT, NH), ID16 = tc::idesc_bf16(MT, 16);
    const int n_tiles = (n + MT - 1) / MT;
    uint32_t pd = 0u;
    bool ok = true;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int t0 = t * MT;
        // input features -> A (K = 32)
        for (int c = tid; c < MT * (NF / 8); c += FWD_THREADS) {
            const int g = c / MT, r = c - g * MT;
            float x[8];
            if (t0 + r < n) {
                const float4 u0 = *reinterpret_cast<const float4 *>(X + (size_t)(t0 + r) * NF + 8 * g);
                const float4 u1 = *reinterpret_cast<const float4 *>(X + (size_t)(t0 + r) * NF + 8 * g + 4);
                x[0] = u0.x; x[1] = u0.y; x[2] = u0.z; x[3] = u0.w;
                x[4] = u1.x; x[5] = u1.y; x[6] = u1.z; x[7] = u1.w;
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) x[q] = 0.0f;
            }
            split_store8(sa, tc::core_offset(r, 8 * g, LBO_A), x);
        }
        for (int layer = 0; layer < 3; ++layer) {
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();   // the operand is in shared memory; the previous TMEM reads are done
            if (tid == 0) {
                tc::fence_after_sync();
                if (layer == 0) layer_mma(tmem, sa_u, sw1_u, LBO_W, NF, ID128);
                else if (layer == 1) layer_mma(tmem + NH, sa_u, sw2_u, LBO_W, NH, ID128);
                else layer_mma(tmem, sa_u, sw3_u, LBO_W3, NH, ID16);
                tc::mma_commit(done);
            }
            const bool mg = tc::mbar_wait(done, pd);
            pd ^= 1u;
            if (!__syncthreads_and(mg)) { ok = false; break; }
            tc::fence_after_sync();
            if (layer == 0) hidden_epilogue(lanes + 32 * slice, 32 * slice, b1, sa, row);
            else if (layer == 1) hidden_epilogue(lanes + NH + 32 * slice, 32 * slice, b2, sa, row);
            else if (slice == 0) {   // outputs: Zl[i][k] = sum_{a,b} R[a][i] T[a][b] R[b][k]
                float v[32];
                tc::tmem_ld32(lanes, v);
                if (t0 + row < n) {
                    float y[NO];
#pragma unroll
                    for (int o = 0; o < NO; ++o) y[o] = v[o] + b3[o];
                    const float *Rj = R + (size_t)(t0 + row) * 9;
                    for (int i = 0; i < 3; ++i)
                        for (int k = 0; k < 3; ++k) {
                            float s = 0.0f;
                            for (int aa = 0; aa < 3; ++aa)
                                for (int bb = 0; bb < 3; ++bb) s = fmaf(Rj[3 * aa + i] * y[3 * aa + bb], Rj[3 * bb + k], s);
                            Zl[(size_t)(t0 + row) * 9 + 3 * i + k] = s;
                        }
                }
            }
        }
        if (!ok) break;
    }
    if (!ok && tid == 0) atomicOr(status, (unsigned)ERRBIT_TIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// per cell: Z = Q I + Zl - mean; with Zref: squared-error partial and gy = R (gZ - mean gZ) R^T
__global__ void k_cell_tensors(int n_cells, const int *__restrict__ off, const float *__restrict__ Zl,
                               const float *__restrict__ R, const double *__restrict__ Q,
                               const double *__restrict__ Zref, double inv_count, double *__restrict__ Zout,
                               float *__restrict__ gy, double *__restrict__ loss_part, double pol0,
                               double pol1, double pol2, double *__restrict__ b) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const int a0 = off[c], a1 = off[c + 1];
    if (b && !Zref && !Zout) {
        // the time step's b only: the network part in FP32 (the precision of Zl), then the FP64
        // charge term, b_j = sum_a pol_a (Zl_j - mean)[a][.] + pol Q_j
        float mf[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int j = a0; j < a1; ++j)
#pragma unroll
            for (int q = 0; q < 9; ++q) mf[q] += Zl[(size_t)j * 9 + q];
        const float ic = 1.0f / (float)(a1 - a0);
#pragma unroll
        for (int q = 0; q < 9; ++q) mf[q] *= ic;
        const float pf[3] = {(float)pol0, (float)pol1, (float)pol2};
        const double pol[3] = {pol0, pol1, pol2};
        for (int j = a0; j < a1; ++j) {
            const float *z = Zl + (size_t)j * 9;
            const double Qj = Q[j];
#pragma unroll
            for (int be = 0; be < 3; ++be) {
                float sv = 0.0f;
#pragma unroll
                for (int aa = 0; aa < 3; ++aa) sv = fmaf(pf[aa], z[3 * aa + be] - mf[3 * aa + be], sv);
                b[3 * j + be] = fma(pol[be], Qj, (double)sv);
            }
        }
        return;
    }
    const double cnt = (double)(a1 - a0);
    double mean[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int j = a0; j < a1; ++j)
        for (int q = 0; q < 9; ++q) mean[q] += Zl[(size_t)j * 9 + q];
    for (int q = 0; q < 9; ++q) mean[q] /= cnt;
    double lsum = 0.0, gmean[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int j = a0; j < a1; ++j) {
        double Z[9];
        for (int q = 0; q < 9; ++q) Z[q] = (double)Zl[(size_t)j * 9 + q] - mean[q] + ((q % 4 == 0) ? Q[j] : 0.0);
        if (Zout)
            for (int q = 0; q < 9; ++q) Zout[(size_t)j * 9 + q] = Z[q];
        if (b) {
            const double pol[3] = {pol0, pol1, pol2};
            for (int be = 0; be < 3; ++be)
                b[3 * j + be] = pol[0] * Z[be] + pol[1] * Z[3 + be] + pol[2] * Z[6 + be];
        }
        if (Zref) {
            for (int q = 0; q < 9; ++q) {
                const double d = Z[q] - Zref[(size_t)j * 9 + q];
                lsum += d * d;
                gmean[q] += 2.0 * d * inv_count;
            }
        }
    }
    if (!Zref) return;
    loss_part[c] = lsum;
    for (int q = 0; q < 9; ++q) gmean[q] /= cnt;
    for (int j = a0; j < a1; ++j) {
        float gz[9];
        for (int q = 0; q < 9; ++q) {
            const double d = (double)Zl[(size_t)j * 9 + q] - mean[q] + ((q % 4 == 0) ? Q[j] : 0.0) -
                             Zref[(size_t)j * 9 + q];
            gz[q] = (float)(2.0 * d * inv_count - gmean[q]);
        }
        const float *Rj = R + (size_t)j * 9;
        // gT[a][b] = sum_{i,k} R[a][i] gZl[i][k] R[b][k]
        for (int aa = 0; aa < 3; ++aa)
            for (int bb = 0; bb < 3; ++bb) {
                float s = 0.0f;
                for (int i = 0; i < 3; ++i)
                    for (int k = 0; k < 3; ++k) s = fmaf(Rj[3 * aa + i] * gz[3 * i + k], Rj[3 * bb + k], s);
                gy[(size_t)j * 9 + 3 * aa + bb] = s;
            }
    }
}

// backward over a tile: per-tile partial gradient of every parameter (fixed-order sums)
__global__ void __launch_bounds__(NH) k_backward(int n, const float *__restrict__ X, const float *__restrict__ gy,
                                                 const float *__restrict__ z1g, const float *__restrict__ z2g,
                                                 const float *__restrict__ h1g, const float *__restrict__ h2g,
                                                 const __nv_bfloat16 *__restrict__ w, float *__restrict__ part) {
    __shared__ float xs[TILE][NF + 1];
    __shared__ float bufA[TILE][NH + 1];   // h2, then gz1
    __shared__ float gz2[TILE][NH + 1];
    __shared__ float h1[TILE][NH + 1];
    __shared__ float gys[TILE][NO];
    const int t0 = blockIdx.x * TILE;
    const int u = threadIdx.x;
    float *P = part + (size_t)blockIdx.x * NPAR;
    for (int e = u; e < TILE * NF; e += NH) {
        const int a = e / NF, i = e - a * NF;
        xs[a][i] = (t0 + a < n) ? X[(size_t)(t0 + a) * NF + i] : 0.0f;
    }
    for (int e = u; e < TILE * NO; e += NH) {
        const int a = e / NO, o = e - a * NO;
        gys[a][o] = (t0 + a < n) ? gy[(size_t)(t0 + a) * NO + o] : 0.0f;
    }
    for (int a = 0; a < TILE; ++a) {
        const bool ok = t0 + a < n;
        bufA[a][u] = ok ? h2g[(size_t)(t0 + a) * NH + u] : 0.0f;
        h1[a][u] = ok ? h1g[(size_t)(t0 + a) * NH + u] : 0.0f;
    }
    __syncthreads();
    // layer 3: dW3[o][u] = sum_a gy[a][o] h2[a][u], db3; gz2[a][u] = silu'(z2) sum_o gy[a][o] W3[o][u]
    {
        float w3[NO];
        for (int o = 0; o < NO; ++o) w3[o] = wv(w, OFF_W3 + o * NH + u);
        for (int o = 0; o < NO; ++o) {
            float s = 0.0f;
            for (int a = 0; a < TILE; ++a) s = fmaf(gys[a][o], bufA[a][u], s);
            P[OFF_W3 + o * NH + u] = s;
        }
        if (u < NO) {
            float s = 0.0f;
            for (int a = 0; a < TILE; ++a) s += gys[a][u];
            P[OFF_B3 + u] = s;
        }
        for (int a = 0; a < TILE; ++a) {
            float s = 0.0f;
            for (int o = 0; o < NO; ++o) s = fmaf(gys[a][o], w3[o], s);
            gz2[a][u] = (t0 + a < n) ? s * dsilu(z2g[(size_t)(t0 + a) * NH + u]) : 0.0f;
        }
    }
    __syncthreads();
    // layer 2: dW2[u][v] = sum_a gz2[a][u] h1[a][v]; db2; gh1[a][v] = sum_u gz2[a][u] W2[u][v]
    {
        float b = 0.0f;
        for (int a = 0; a < TILE; ++a) b += gz2[a][u];
        P[OFF_B2 + u] = b;
        for (int v = 0; v < NH; ++v) {
            float s = 0.0f;
#pragma unroll
            for (int a = 0; a < TILE; ++a) s = fmaf(gz2[a][u], h1[a][v], s);
            P[OFF_W2 + u * NH + v] = s;
        }
        // thread u now plays the role of input unit v = u
        float acc[TILE];
        for (int a = 0; a < TILE; ++a) acc[a] = 0.0f;
        for (int uu = 0; uu < NH; ++uu) {
            const float wuv = wv(w, OFF_W2 + uu * NH + u);
#pragma unroll
            for (int a = 0; a < TILE; ++a) acc[a] = fmaf(gz2[a][uu], wuv, acc[a]);
        }
        __syncthreads();   // bufA (h2) is no longer read
        for (int a = 0; a < TILE; ++a)
            bufA[a][u] = (t0 + a < n) ? acc[a] * dsilu(z1g[(size_t)(t0 + a) * NH + u]) : 0.0f;
    }
    __syncthreads();
    // layer 1: dW1[u][i] = sum_a gz1[a][u] x[a][i]; db1
    {
        float b = 0.0f;
        for (int a = 0; a < TILE; ++a) b += bufA[a][u];
        P[OFF_B1 + u] = b;
        for (int i = 0; i < NF; ++i) {
            float s = 0.0f;
#pragma unroll
            for (int a = 0; a < TILE; ++a) s = fmaf(bufA[a][u], xs[a][i], s);
            P[OFF_W1 + u * NF + i] = s;
        }
    }
}

__global__ void k_reduce_grad(int n_tiles, const float *__restrict__ part, float *__restrict__ g) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPAR) return;
    double s = 0.0;
    for (int t = 0; t < n_tiles; ++t) s += part[(size_t)t * NPAR + p];
    g[p] = (float)s;
}

__global__ void k_reduce_loss(int n, const double *__restrict__ part, double scale, double *__restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < 256; ++i) t += red[i];
        *out = t * scale;
    }
}

__global__ void k_adamw(const float *__restrict__ g, float *__restrict__ master, float *__restrict__ m1,
                        float *__restrict__ m2, __nv_bfloat16 *__restrict__ w, float lr, float wd, float c1,
                        float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPAR) return;
    const float b1 = 0.9f, b2 = 0.999f;
    const float gp = g[p];
    const float m = b1 * m1[p] + (1.0f - b1) * gp;
    const float v = b2 * m2[p] + (1.0f - b2) * gp * gp;
    m1[p] = m;
    m2[p] = v;
    const float mh = m / c1, vh = v / c2;
    const float x = master[p] - lr * (mh / (sqrtf(vh) + 1e-8f) + wd * master[p]);
    master[p] = x;
    w[p] = __float2bfloat16_rn(x);
}

__global__ void k_to_bf16(const float *__restrict__ src, __nv_bfloat16 *__restrict__ dst, int n) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) dst[p] = __float2bfloat16_rn(src[p]);
}

__global__ void k_permute_cells(int n_cells, const int *__restrict__ perm, const float *__restrict__ X,
                                const float *__restrict__ R, const double *__restrict__ Q,
                                const double *__restrict__ Zr, float *__restrict__ Xo, float *__restrict__ Ro,
                                double *__restrict__ Qo, double *__restrict__ Zo) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const int s = perm[c];
    for (int j = 0; j < 3; ++j) {
        const int dj = 3 * c + j, sj = 3 * s + j;
        for (int i = 0; i < NF; ++i) Xo[(size_t)dj * NF + i] = X[(size_t)sj * NF + i];
        for (int q = 0; q < 9; ++q) {
            Ro[(size_t)dj * 9 + q] = R[(size_t)sj * 9 + q];
            Zo[(size_t)dj * 9 + q] = Zr[(size_t)sj * 9 + q];
        }
        Qo[dj] = Q[sj];
    }
}

}  // namespace

// --------------------------------------------------------------------------------------------- host

cudaError_t launch_mlp_features(int n_cells, const int *off, const int *species, const double *r, float *X,
                                float *R, unsigned *status, cudaStream_t st) {
    k_features<<<(n_cells + 127) / 128, 128, 0, st>>>(n_cells, off, species, r, X, R, status);
    return cudaGetLastError();
}

cudaError_t prepare_mlp_forward() {
    return cudaFuncSetAttribute(k_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FWD_SMEM);
}

cudaError_t launch_mlp_forward(int n_atoms, const float *X, const float *R, const void *w_bf16, float *Zl,
                               unsigned *status, cudaStream_t st) {
    if (n_atoms <= 0) return cudaSuccess;
    int dev = 0, n_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int tiles = (n_atoms + MT - 1) / MT;
    const int grid = std::min(tiles, n_sm);
    k_forward_tc<<<grid, FWD_THREADS, FWD_SMEM, st>>>(n_atoms, X, R, (const __nv_bfloat16 *)w_bf16, Zl, status);
    return cudaGetLastError();
}

cudaError_t launch_mlp_born(int n_cells, const int *off, const float *Zl, const float *R, const double *Q,
                            double pol0, double pol1, double pol2, double *b, cudaStream_t st) {
    k_cell_tensors<<<(n_cells + 127) / 128, 128, 0, st>>>(n_cells, off, Zl, R, Q, nullptr, 0.0, nullptr, nullptr,
                                                          nullptr, pol0, pol1, pol2, b);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float *src, void *dst, int n, cudaStream_t st) {
    k_to_bf16<<<(n + 255) / 256, 256, 0, st>>>(src, (__nv_bfloat16 *)dst, n);
    return cudaGetLastError();
}

struct cavmd_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    int n_cells = 0, n_atoms = 0;
    float *master = nullptr, *m1 = nullptr, *m2 = nullptr, *g = nullptr, *part = nullptr;
    __nv_bfloat16 *w = nullptr;
    int *off = nullptr, *species = nullptr, *perm = nullptr;
    double *r = nullptr, *Q = nullptr, *Zref = nullptr, *Zout = nullptr, *lpart = nullptr, *loss = nullptr;
    float *X = nullptr, *R = nullptr, *Xp = nullptr, *Rp = nullptr, *Zl = nullptr, *gy = nullptr;
    float *z1 = nullptr, *z2 = nullptr, *h1 = nullptr, *h2 = nullptr;
    double *Qp = nullptr, *Zp = nullptr;
    unsigned *status = nullptr;
    int64_t adam_t = 0;
    std::vector<void *> allocs;
    std::string err;
};

namespace {

int mlp_fail(cavmd_mlp *m, int code, const std::string &msg) {
    if (m) m->err = msg;
    cavmd_set_global_error(msg);
    return code;
}

#define MCK(call)                                                                            \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return mlp_fail(m, CAVMD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
int mlp_alloc(cavmd_mlp *m, T **p, size_t n) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) return mlp_fail(m, CAVMD_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    m->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return CAVMD_OK;
}

#define MAL(ptr, n)                               \
    do {                                          \
        int rc_ = mlp_alloc(m, &(ptr), (size_t)(n)); \
        if (rc_) return rc_;                      \
    } while (0)

void mlp_free_data(cavmd_mlp *m, size_t keep) {
    for (size_t i = keep; i < m->allocs.size(); ++i) cudaFree(m->allocs[i]);
    m->allocs.resize(keep);
}

// forward + loss + gradient over atoms [0, n) of the (permuted) arrays
int mlp_loss_grad_range(cavmd_mlp *m, int cell0, int ncells, const float *X, const float *R, const double *Q,
                        const double *Zr, double inv_count) {
    const int a0 = 3 * cell0, na = 3 * ncells;
    const int tiles = (na + TILE - 1) / TILE;
    k_forward<<<tiles, NH, 0, m->stream>>>(na, X + (size_t)a0 * NF, R + (size_t)a0 * 9, m->w, m->Zl, m->z1, m->z2,
                                           m->h1, m->h2);
    k_cell_tensors<<<(ncells + 127) / 128, 128, 0, m->stream>>>(ncells, m->off, m->Zl, R + (size_t)a0 * 9, Q + a0,
                                                                Zr + (size_t)a0 * 9, inv_count, nullptr, m->gy,
                                                                m->lpart, 0, 0, 0, nullptr);
    k_backward<<<tiles, NH, 0, m->stream>>>(na, X + (size_t)a0 * NF, m->gy, m->z1, m->z2, m->h1, m->h2, m->w,
                                            m->part);
    k_reduce_grad<<<(NPAR + 255) / 256, 256, 0, m->stream>>>(tiles, m->part, m->g);
    k_reduce_loss<<<1, 256, 0, m->stream>>>(ncells, m->lpart, inv_count, m->loss);
    MCK(cudaGetLastError());
    return CAVMD_OK;
}

}  // namespace

extern "C" {

int cavmd_mlp_create(cavmd_mlp **out, const float *params, int32_t n_params, int32_t device) {
    if (!out || !params || n_params != CAVMD_MLP_NPARAMS) {
        cavmd_set_global_error("cavmd_mlp_create: need params[CAVMD_MLP_NPARAMS]");
        return CAVMD_ERR_INVALID_ARG;
    }
    *out = nullptr;
    cavmd_mlp *m = new cavmd_mlp();
    m->device = device;
    int rc = CAVMD_OK;
    auto done = [&](int code) {
        if (code) {
            mlp_free_data(m, 0);
            if (m->stream) cudaStreamDestroy(m->stream);
            delete m;
        }
        return code;
    };
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return done(mlp_fail(nullptr, CAVMD_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e)));
    e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return done(mlp_fail(nullptr, CAVMD_ERR_CUDA, "cudaStreamCreate"));
    e = prepare_mlp_forward();
    if (e != cudaSuccess) return done(mlp_fail(nullptr, CAVMD_ERR_CUDA, "cudaFuncSetAttribute (network forward)"));
    if ((rc = mlp_alloc(m, &m->master, NPAR)) || (rc = mlp_alloc(m, &m->m1, NPAR)) ||
        (rc = mlp_alloc(m, &m->m2, NPAR)) || (rc = mlp_alloc(m, &m->g, NPAR)) || (rc = mlp_alloc(m, &m->w, NPAR)) ||
        (rc = mlp_alloc(m, &m->loss, 1)) || (rc = mlp_alloc(m, &m->status, 1)))
        return done(rc);
    e = cudaMemcpy(m->master, params, sizeof(float) * NPAR, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->m1, 0, sizeof(float) * NPAR);
    if (e == cudaSuccess) e = cudaMemset(m->m2, 0, sizeof(float) * NPAR);
    if (e == cudaSuccess) e = cudaMemset(m->status, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = launch_to_bf16(m->master, m->w, NPAR, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return done(mlp_fail(nullptr, CAVMD_ERR_CUDA, cudaGetErrorString(e)));
    *out = m;
    return CAVMD_OK;
}

int cavmd_mlp_set_data(cavmd_mlp *m, int32_t n_cells, const int32_t *species, const double *r, const double *Q,
                       const double *Z_ref) {
    if (!m || n_cells < 1 || !species || !r || !Q) return mlp_fail(m, CAVMD_ERR_INVALID_ARG, "bad data arguments");
    for (int i = 0; i < 3 * n_cells; ++i)
        if (species[i] < 0 || species[i] > 1) return mlp_fail(m, CAVMD_ERR_INVALID_ARG, "species must be 0 or 1");
    MCK(cudaSetDevice(m->device));
    mlp_free_data(m, 7);   // keep the parameter and optimiser buffers
    m->n_cells = n_cells;
    m->n_atoms = 3 * n_cells;
    const int na = m->n_atoms;
    std::vector<int> off(n_cells + 1);
    for (int c = 0; c <= n_cells; ++c) off[c] = 3 * c;
    MAL(m->off, n_cells + 1); MAL(m->species, na); MAL(m->perm, n_cells);
    MAL(m->r, 3 * na); MAL(m->Q, na); MAL(m->Zref, 9 * na); MAL(m->Zout, 9 * na); MAL(m->lpart, n_cells);
    MAL(m->X, (size_t)na * NF); MAL(m->R, 9 * na); MAL(m->Xp, (size_t)na * NF); MAL(m->Rp, 9 * na);
    MAL(m->Qp, na); MAL(m->Zp, 9 * na); MAL(m->Zl, 9 * na); MAL(m->gy, 9 * na);
    MAL(m->z1, (size_t)na * NH); MAL(m->z2, (size_t)na * NH); MAL(m->h1, (size_t)na * NH); MAL(m->h2, (size_t)na * NH);
    MAL(m->part, (size_t)((na + TILE - 1) / TILE) * NPAR);
    MCK(cudaMemcpy(m->off, off.data(), sizeof(int) * (n_cells + 1), cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(m->species, species, sizeof(int) * na, cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(m->r, r, sizeof(double) * 3 * na, cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(m->Q, Q, sizeof(double) * na, cudaMemcpyHostToDevice));
    if (Z_ref) MCK(cudaMemcpy(m->Zref, Z_ref, sizeof(double) * 9 * na, cudaMemcpyHostToDevice));
    else MCK(cudaMemset(m->Zref, 0, sizeof(double) * 9 * na));
    MCK(launch_mlp_features(n_cells, m->off, m->species, m->r, m->X, m->R, m->status, m->stream));
    MCK(cudaStreamSynchronize(m->stream));
    return CAVMD_OK;
}

int cavmd_mlp_loss_grad(cavmd_mlp *m, double *loss, float *grad) {
    if (!m || !m->n_cells || !loss) return mlp_fail(m, CAVMD_ERR_INVALID_ARG, "no data or NULL output");
    MCK(cudaSetDevice(m->device));
    int rc = mlp_loss_grad_range(m, 0, m->n_cells, m->X, m->R, m->Q, m->Zref, 1.0 / (9.0 * m->n_atoms));
    if (rc) return rc;
    MCK(cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    if (grad) MCK(cudaMemcpyAsync(grad, m->g, sizeof(float) * NPAR, cudaMemcpyDeviceToHost, m->stream));
    MCK(cudaStreamSynchronize(m->stream));
    return CAVMD_OK;
}

int cavmd_mlp_train(cavmd_mlp *m, int32_t epochs, int32_t batch_cells, float lr, float weight_decay,
                    uint64_t seed, double *epoch_loss) {
    if (!m || !m->n_cells || epochs < 1 || batch_cells < 1 || !(lr > 0.0f))
        return mlp_fail(m, CAVMD_ERR_INVALID_ARG, "bad training arguments");
    MCK(cudaSetDevice(m->device));
    std::vector<int> perm(m->n_cells);
    std::mt19937_64 rng(seed);
    for (int ep = 0; ep < epochs; ++ep) {
        std::iota(perm.begin(), perm.end(), 0);
        std::shuffle(perm.begin(), perm.end(), rng);
        MCK(cudaMemcpyAsync(m->perm, perm.data(), sizeof(int) * m->n_cells, cudaMemcpyHostToDevice, m->stream));
        k_permute_cells<<<(m->n_cells + 127) / 128, 128, 0, m->stream>>>(m->n_cells, m->perm, m->X, m->R, m->Q,
                                                                         m->Zref, m->Xp, m->Rp, m->Qp, m->Zp);
        double ep_loss = 0.0;
        for (int c0 = 0; c0 < m->n_cells; c0 += batch_cells) {
            const int nb = std::min(batch_cells, m->n_cells - c0);
            int rc = mlp_loss_grad_range(m, c0, nb, m->Xp, m->Rp, m->Qp, m->Zp, 1.0 / (9.0 * 3 * nb));
            if (rc) return rc;
            ++m->adam_t;
            const float c1 = 1.0f - powf(0.9f, (float)m->adam_t), c2 = 1.0f - powf(0.999f, (float)m->adam_t);
            k_adamw<<<(NPAR + 255) / 256, 256, 0, m->stream>>>(m->g, m->master, m->m1, m->m2, m->w, lr,
                                                               weight_decay, c1, c2);
            MCK(cudaGetLastError());
            if (epoch_loss) {
                double l = 0.0;
                MCK(cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
                MCK(cudaStreamSynchronize(m->stream));
                ep_loss += l * nb;
            }
        }
        if (epoch_loss) epoch_loss[ep] = ep_loss / m->n_cells;
    }
    MCK(cudaStreamSynchronize(m->stream));
    return CAVMD_OK;
}

int cavmd_mlp_predict(cavmd_mlp *m, double *Z_out) {
    if (!m || !m->n_cells || !Z_out) return mlp_fail(m, CAVMD_ERR_INVALID_ARG, "no data or NULL output");
    MCK(cudaSetDevice(m->device));
    MCK(launch_mlp_forward(m->n_atoms, m->X, m->R, m->w, m->Zl, m->status, m->stream));
    k_cell_tensors<<<(m->n_cells + 127) / 128, 128, 0, m->stream>>>(m->n_cells, m->off, m->Zl, m->R, m->Q, nullptr,
                                                                    0.0, m->Zout, nullptr, nullptr, 0, 0, 0, nullptr);
    MCK(cudaGetLastError());
    MCK(cudaMemcpyAsync(Z_out, m->Zout, sizeof(double) * 9 * m->n_atoms, cudaMemcpyDeviceToHost, m->stream));
    MCK(cudaStreamSynchronize(m->stream));
    return CAVMD_OK;
}

int cavmd_mlp_get_params(cavmd_mlp *m, float *params) {
    if (!m || !params) return mlp_fail(m, CAVMD_ERR_INVALID_ARG, "NULL argument");
    MCK(cudaSetDevice(m->device));
    std::vector<__nv_bfloat16> w(NPAR);
    MCK(cudaMemcpy(w.data(), m->w, sizeof(__nv_bfloat16) * NPAR, cudaMemcpyDeviceToHost));
    for (int p = 0; p < NPAR; ++p) params[p] = __bfloat162float(w[p]);
    return CAVMD_OK;
}

void cavmd_mlp_destroy(cavmd_mlp *m) {
    if (!m) return;
    cudaSetDevice(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    mlp_free_data(m, 0);
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

}  // extern "C"
