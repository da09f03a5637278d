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
//   y_j      : W3 silu(W2 silu(W1 x + b1) + b2) + b3, 32 -> 128 -> 128 -> 9, BF16 weights, FP32 math
//              (tcgen05 MMAs with the activations split into BF16 parts, FP32 accumulation);
//   Z_j      = Q_j I + R_j^T T_j R_j - mean over the cell (T_j = y_j as 3 x 3), so the sum rule
//              sum_j Z_j = Q_cell I holds and a zero network is the Mulliken model;
//   b_j      = pol^T Z_j.
// Training minimises sum |Z - Z_ref|^2 / (9 n_atoms) with AdamW on FP32 master weights. Forward,
// backward and weight gradients run on the tensor cores; the gradient reduction over CTAs is a
// fixed-order sum (bitwise reproducible).
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
constexpr float RC = 8.0f;

__device__ __forceinline__ float dsilu(float z) {
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}
__device__ __forceinline__ float fcut(float r) { return r < RC ? 0.5f * (cospif(r / RC) + 1.0f) : 0.0f; }
__device__ __forceinline__ float wv(const __nv_bfloat16 *w, int i) { return __bfloat162float(w[i]); }

// features x (32) and frame fr (9, rows e1 e2 e3) of atom j of the cell of atoms [a0, a1)
__device__ __forceinline__ void atom_features(int a0, int a1, int j, const int *__restrict__ species,
                                              const double *__restrict__ r, float (&x)[NF], float (&fr)[9],
                                              unsigned *__restrict__ status) {
#pragma unroll
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
#pragma unroll
    for (int q = 0; q < 9; ++q) fr[q] = (q % 4 == 0) ? 1.0f : 0.0f;
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
}

// features (n_atoms x 32) and frames (n_atoms x 9) of every atom; thread per cell, cells of any size
__global__ void k_features(int n_cells, const int *__restrict__ off, const int *__restrict__ species,
                           const double *__restrict__ r, float *__restrict__ X, float *__restrict__ R,
                           unsigned *__restrict__ status) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const int a0 = off[c], a1 = off[c + 1];
    for (int j = a0; j < a1; ++j) {
        float x[NF], fr[9];
        atom_features(a0, a1, j, species, r, x, fr, status);
        float4 *Xj = reinterpret_cast<float4 *>(X + (size_t)j * NF);
#pragma unroll
        for (int i = 0; i < NF / 4; ++i) Xj[i] = make_float4(x[4 * i], x[4 * i + 1], x[4 * i + 2], x[4 * i + 3]);
        for (int q = 0; q < 9; ++q) R[(size_t)j * 9 + q] = fr[q];
    }
}

// The same for cells of 3 atoms each (water systems, atoms 3 c .. 3 c + 2), in three rounds: round
// a forms atom a of every cell of the block, stages the rows in shared memory and writes them out
// row by row (a warp writes one 128-byte feature row per store; a thread's own rows would be
// 384 bytes apart from its neighbours').
constexpr int FEAT_CELLS = 128;                 // cells (threads) per block
constexpr int FEAT_LD = NF + 4;                 // staged row stride in floats (16-byte rows, no bank conflicts)
__global__ void __launch_bounds__(FEAT_CELLS) k_features_w3(int n_cells, const int *__restrict__ species,
                                                            const double *__restrict__ r, float *__restrict__ X,
                                                            float *__restrict__ R, unsigned *__restrict__ status) {
    __shared__ __align__(16) float sx[FEAT_CELLS * FEAT_LD];
    __shared__ float sr[FEAT_CELLS * 9];
    const int c0 = blockIdx.x * FEAT_CELLS, c = c0 + threadIdx.x;
    const int nc = min(FEAT_CELLS, n_cells - c0);   // cells of this block
    for (int at = 0; at < 3; ++at) {
        if (c < n_cells) {
            float x[NF], fr[9];
            atom_features(3 * c, 3 * c + 3, 3 * c + at, species, r, x, fr, status);
            float4 *sxj = reinterpret_cast<float4 *>(sx + threadIdx.x * FEAT_LD);
#pragma unroll
            for (int i = 0; i < NF / 4; ++i) sxj[i] = make_float4(x[4 * i], x[4 * i + 1], x[4 * i + 2], x[4 * i + 3]);
#pragma unroll
            for (int q = 0; q < 9; ++q) sr[threadIdx.x * 9 + q] = fr[q];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nc * NF; i += FEAT_CELLS) {   // row i / NF: atom 3 (c0 + row) + at
            const int row = i / NF, col = i - row * NF;
            X[((size_t)3 * (c0 + row) + at) * NF + col] = sx[row * FEAT_LD + col];
        }
        for (int i = threadIdx.x; i < nc * 9; i += FEAT_CELLS) {
            const int row = i / 9, q = i - row * 9;
            R[((size_t)3 * (c0 + row) + at) * 9 + q] = sr[i];
        }
        __syncthreads();
    }
}

// Network forward on the fifth-generation tensor cores (tcgen05), for the time step and for
// training (the same kernel, so inference and training see the same numbers). A tile of
// 128 atoms sits on the 128 TMEM lanes and each layer is one BF16 MMA chain D = A B^T with FP32
// accumulation in TMEM:
//   A = the layer input, 128 atoms x K, split into three BF16 parts: hi + mid + lo carries a
//       float's 24-bit significand, so A B^T equals the FP32 products to accumulation rounding;
//   B = the layer's BF16 weights (exact), N outputs x K, K-major core matrices.
// L1: K = 32, N = 128 into TMEM columns 0..127; L2: K = 128, N = 128 into columns 128..255;
// L3: K = 128, N = 16 (the 9 outputs, zero-padded) into columns 128..143, which the second
// epilogue has read in its first round. Sixteen epilogue warps read TMEM (warp w: lanes
// 32 (w mod 4) .. + 31), add the bias, apply silu and write the next layer's split operand to
// shared memory in four rounds of 32 columns (K chunks; warp w takes columns 8 (w div 4) + 32 c of
// round c), and a seventeenth warp issues the MMAs: each K chunk of L2 and L3 as soon as all
// sixteen warps have written it, so the next layer's MMAs run under the rest of the epilogue. The
// MMA order is that of one chain per layer (K steps ascending, parts hi, mid, lo), so the sums do
// not depend on the overlap. The next tile's inputs are loaded during the second epilogue and the
// last layer's outputs (Zl = R^T T R per atom) are formed while the next tile's first layer runs.
// One persistent CTA per SM loads the weights once; every mbarrier wait is bounded (timeout:
// status bit, the MMAs in flight drained, TMEM still released).
// Training keeps what the backward pass reads (FwdStore): the pre-activations z1, z2 atom-major,
// and the layer inputs x, h1, h2 feature-major per tile ([tile][feature][atom of the tile]), the
// layout in which the weight-gradient kernel stages them as K-major operands over atoms.
constexpr int MT = 128;                              // atoms per tile = TMEM lanes
constexpr int FWD_THREADS = 512;                     // 16 warps: four per TMEM lane quadrant
constexpr int FWD_TC_THREADS = FWD_THREADS + 32;     // the forward: 16 epilogue warps and one MMA warp
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

// silu with the reciprocal of the special-function unit
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

struct FwdStore {       // training outputs of the forward (all NULL in the time step)
    float *z1, *z2;     // [atoms][128] pre-activations
    float *h1t, *h2t;   // [tile][128][128] silu(z1), silu(z2), feature-major per tile
    float *xt;          // [tile][32][128] network inputs, feature-major per tile
};

// Hidden-layer epilogue, one 8-column chunk of this thread's atom (the accumulator values v):
// z = d + b -> silu -> split A operand; zg (this atom's row of z) and ht (this atom's column of the
// tile's activations) may be NULL.
__device__ __forceinline__ void hidden_chunk(const uint32_t (&v)[8], int col, const float *b, uint8_t *sa, int row,
                                             float *zg, float *ht) {
    float x[8], z[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        z[q] = __uint_as_float(v[q]) + b[col + q];
        x[q] = silu_fast(z[q]);
    }
    if (zg) {
        *reinterpret_cast<float4 *>(zg + col) = make_float4(z[0], z[1], z[2], z[3]);
        *reinterpret_cast<float4 *>(zg + col + 4) = make_float4(z[4], z[5], z[6], z[7]);
    }
    if (ht)
#pragma unroll
        for (int q = 0; q < 8; ++q) ht[(size_t)(col + q) * MT] = x[q];
    split_store8(sa, tc::core_offset(row, col, LBO_A), x);
}

// Eight input features of one atom (chunk c of the tile: features 8 (c / MT) .., atom c mod MT), or
// zeros past the last atom.
__device__ __forceinline__ void load_x8(const float *X, int n, int t0, int c, float (&x)[8]) {
    const int g = c / MT, r = c - g * MT;
    if (t0 + r < n) {
        const float4 u0 = *reinterpret_cast<const float4 *>(X + (size_t)(t0 + r) * NF + 8 * g);
        const float4 u1 = *reinterpret_cast<const float4 *>(X + (size_t)(t0 + r) * NF + 8 * g + 4);
        x[0] = u0.x; x[1] = u0.y; x[2] = u0.z; x[3] = u0.w;
        x[4] = u1.x; x[5] = u1.y; x[6] = u1.z; x[7] = u1.w;
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) x[q] = 0.0f;
    }
}

// ... into the K = 32 operand of L1 (and, in training, the tile's feature-major copy).
__device__ __forceinline__ void store_x8(uint8_t *sa, int t, int c, const float (&x)[8], float *xt) {
    const int g = c / MT, r = c - g * MT;
    if (xt)
#pragma unroll
        for (int q = 0; q < 8; ++q) xt[((size_t)t * NF + 8 * g + q) * MT + r] = x[q];
    split_store8(sa, tc::core_offset(r, 8 * g, LBO_A), x);
}

// K steps k0, k0 + 1 of one layer (issued by one thread), in the order of the whole chain: for each
// K step the parts hi, mid, lo; the first product of the chain overwrites the accumulator.
__device__ __forceinline__ void chunk_mma(uint32_t tmem_d, uint32_t sa, uint32_t sw, uint32_t lbo_w, int k0,
                                          uint32_t idesc) {
#pragma unroll
    for (int k = k0; k < k0 + 2; ++k) {
        const uint64_t bd = tc::make_desc(sw + (uint32_t)k * 2 * lbo_w, lbo_w, 128);
#pragma unroll
        for (int s = 0; s < 3; ++s)
            tc::mma_bf16(tmem_d, tc::make_desc(sa + s * A_SPLIT + (uint32_t)k * 2 * LBO_A, LBO_A, 128), bd, idesc,
                         (k > 0 || s > 0) ? 1u : 0u);
    }
}

// Outputs of one atom: y = the L3 accumulator + b3, Zl[i][k] = sum_{a,b} R[a][i] T[a][b] R[b][k].
__device__ __forceinline__ void output_atom(const float (&v)[32], const float *b3, const float (&Rj)[9], float *zl) {
    float y[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) y[o] = v[o] + b3[o];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
            float s = 0.0f;
            for (int aa = 0; aa < 3; ++aa)
                for (int bb = 0; bb < 3; ++bb) s = fmaf(Rj[3 * aa + i] * y[3 * aa + bb], Rj[3 * bb + k], s);
            zl[3 * i + k] = s;
        }
}

__global__ void __launch_bounds__(FWD_TC_THREADS, 1) k_forward_tc(int n, const float *__restrict__ X,
                                                                const float *__restrict__ R,
                                                                const __nv_bfloat16 *__restrict__ w,
                                                                float *__restrict__ Zl, unsigned *__restrict__ status,
                                                                const FwdStore st) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sw1 = smem, *sw2 = sw1 + SW1, *sw3 = sw2 + SW2, *sa = sw3 + SW3;   // sa: [hi][mid][lo]
    float *bias = reinterpret_cast<float *>(sa + 3 * A_SPLIT);                  // b1 [128] b2 [128] b3 [16]
    uint64_t *done = reinterpret_cast<uint64_t *>(bias + 2 * NH + 16);        // a layer's MMAs finished
    uint64_t *chunk = done + 1;                                                // [4] K chunk c written
    uint64_t *drain = chunk + 4;                                               // error path: MMAs in flight
    uint32_t *slot = reinterpret_cast<uint32_t *>(drain + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool mma_warp = warp == FWD_THREADS / 32;
    if (warp == 0) tc::tmem_alloc(slot, 256);
    if (tid == 0) {
        tc::mbar_init(done, 1);
        for (int c = 0; c < 4; ++c) tc::mbar_init(&chunk[c], FWD_THREADS / 32);
        tc::mbar_init(drain, 1);
    }
    const uint16_t *wr = reinterpret_cast<const uint16_t *>(w);
    load_weights(sw1, wr + OFF_W1, NH, NH, NF, LBO_W);
    load_weights(sw2, wr + OFF_W2, NH, NH, NH, LBO_W);
    load_weights(sw3, wr + OFF_W3, 16, NO, NH, LBO_W3);
    for (int e = tid; e < 2 * NH + 16; e += blockDim.x)
        bias[e] = e < 2 * NH ? wv(w, (e < NH ? OFF_B1 : OFF_B2 - NH) + e) : (e - 2 * NH < NO ? wv(w, OFF_B3 + e - 2 * NH) : 0.0f);
    const int n_tiles = (n + MT - 1) / MT;
    if (!mma_warp && (int)blockIdx.x < n_tiles) {   // the first tile's inputs
        float x[8];
        load_x8(X, n, blockIdx.x * MT, tid, x);
        store_x8(sa, blockIdx.x, tid, x, st.xt);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t sa_u = tc::smem_u32(sa), sw1_u = tc::smem_u32(sw1), sw2_u = tc::smem_u32(sw2),
                   sw3_u = tc::smem_u32(sw3);
    const uint32_t quad = warp & 3, part = (warp >> 2) & 3;   // lane quadrant; column part of each chunk
    const uint32_t lanes = tmem + ((32u * quad) << 16);       // this warp's TMEM lanes
    const int row = 32 * quad + lane;                          // this thread's atom in the tile
    const float *b1 = bias, *b2 = bias + NH, *b3 = bias + 2 * NH;
    constexpr uint32_t ID128 = tc::idesc_bf16(MT, NH), ID16 = tc::idesc_bf16(MT, 16);
    uint32_t pd = 0u, pc = 0u;   // phase parities: done (epilogue warps), chunk[c] in bit c (MMA warp)
    bool ok = true;
    float Rp[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, Rc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    int t_prev = -1;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int t0 = t * MT, tn = t + gridDim.x;
        if (mma_warp) {
            if (lane == 0) {
                layer_mma(tmem, sa_u, sw1_u, LBO_W, NF, ID128);   // L1, the whole chain
                tc::mma_commit(done);
                for (int layer = 0; layer < 2; ++layer)
                    for (int c = 0; c < 4; ++c) {   // L2 (L3) K chunk c once the first (second) epilogue wrote it
                        const bool g = ok && tc::mbar_wait(&chunk[c], (pc >> c) & 1u);
                        pc ^= 1u << c;
                        ok = g;
                        if (!ok) continue;
                        tc::fence_after_sync();
                        if (layer == 0) chunk_mma(tmem + NH, sa_u, sw2_u, LBO_W, 2 * c, ID128);
                        else chunk_mma(tmem + NH, sa_u, sw3_u, LBO_W3, 2 * c, ID16);
                        if (c == 3) tc::mma_commit(done);
                    }
            }
            __syncwarp();
        } else {
            if (t_prev >= 0 && part == 0) {   // outputs of the previous tile (its L3 is complete)
                float v[32];
                tc::tmem_ld32(lanes + NH, v);
                if (t_prev * MT + row < n) output_atom(v, b3, Rp, Zl + (size_t)(t_prev * MT + row) * 9);
            }
            if (part == 0) {
                if (t0 + row < n) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) Rc[q] = R[(size_t)(t0 + row) * 9 + q];
                } else {
#pragma unroll
                    for (int q = 0; q < 9; ++q) Rc[q] = 0.0f;
                }
            }
            float xn[8];
            for (int layer = 0; layer < 2; ++layer) {
                ok = tc::mbar_wait(done, pd) && ok;   // L1 (L2) finished
                pd ^= 1u;
                tc::fence_after_sync();
                uint32_t v[4][8];
                const uint32_t acc = lanes + (layer == 0 ? 0u : (uint32_t)NH) + 8 * part;
#pragma unroll
                for (int c = 0; c < 4; ++c) tc::tmem_ld8_nowait(acc + 32 * c, v[c]);
                tc::tmem_wait_ld();
                if (layer == 1 && tn < n_tiles) load_x8(X, n, tn * MT, tid, xn);   // the next tile's inputs
                float *zb = layer == 0 ? st.z1 : st.z2;
                float *hb = layer == 0 ? st.h1t : st.h2t;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int col = 32 * c + 8 * part;
                    hidden_chunk(v[c], col, layer == 0 ? b1 : b2, sa, row, zb ? zb + (size_t)(t0 + row) * NH : nullptr,
                                 hb ? hb + (size_t)t * NH * MT + row : nullptr);
                    tc::fence_proxy_async();   // the operand chunk is visible to the MMAs
                    tc::fence_before_sync();   // and this round's TMEM reads are ordered before them
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&chunk[c]);
                }
            }
            ok = tc::mbar_wait(done, pd) && ok;   // L3 finished: the operand buffer is free
            pd ^= 1u;
            tc::fence_after_sync();
            if (tn < n_tiles) store_x8(sa, tn, tid, xn, st.xt);
#pragma unroll
            for (int q = 0; q < 9; ++q) Rp[q] = Rc[q];
            t_prev = t;
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        if (!__syncthreads_and(ok)) { ok = false; break; }
        tc::fence_after_sync();
    }
    if (ok && t_prev >= 0 && !mma_warp && part == 0) {   // the last tile's outputs
        float v[32];
        tc::tmem_ld32(lanes + NH, v);
        if (t_prev * MT + row < n) output_atom(v, b3, Rp, Zl + (size_t)(t_prev * MT + row) * 9);
    }
    if (!ok) {
        if (tid == 0) atomicOr(status, (unsigned)ERRBIT_TIMEOUT);
        if (mma_warp && lane == 0) {   // every MMA issued so far completes before TMEM is released
            tc::mma_commit(drain);
            tc::mbar_wait(drain, 0);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// BF16 weights W[K][rows] (row-major) into the K-major core-matrix layout of B[row][k] = W[k][row].
__device__ __forceinline__ void load_weights_t(uint8_t *dst, const uint16_t *src, int rows, int K, uint32_t lbo) {
    for (int c = threadIdx.x; c < rows * (K / 8); c += blockDim.x) {
        const int g = c / rows, row = c - g * rows;
        __align__(16) uint16_t v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = src[(8 * g + q) * rows + row];
        *reinterpret_cast<uint4 *>(dst + tc::core_offset(row, 8 * g, lbo)) = *reinterpret_cast<const uint4 *>(v);
    }
}

// Backward through the activations, per 128-atom tile on the tensor cores. With gy = dL/dy (the
// 9 outputs, from the cell tensors):
//   gz2[a][u] = silu'(z2[a][u]) sum_o gy[a][o] W3[o][u]      (CUDA cores, 9 terms)
//   gh1[a][v] = sum_u gz2[a][u] W2[u][v]                      (MMA: A = gz2 in three BF16 parts, so the
//                                                              products are the FP32 ones; B = W2^T, BF16)
//   gz1[a][v] = silu'(z1[a][v]) gh1[a][v]                     (TMEM epilogue)
// gz2, gz1 and gy leave feature-major per tile ([tile][feature][atom]) for the weight gradients;
// atoms beyond n get zeros, so they add nothing there.
constexpr size_t BWA_SMEM = SW2 + 3 * (size_t)A_SPLIT + ((size_t)NO * NH + MT * 16) * 4 + 64;

__global__ void __launch_bounds__(FWD_THREADS, 1) k_backward_act_tc(int n, const float *__restrict__ gy,
                                                                  const float *__restrict__ z1,
                                                                  const float *__restrict__ z2,
                                                                  const __nv_bfloat16 *__restrict__ w,
                                                                  float *__restrict__ gz2t, float *__restrict__ gz1t,
                                                                  float *__restrict__ gyt, unsigned *__restrict__ status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sw2t = smem, *sa = sw2t + SW2;                       // W2^T (rows v, K = u); gz2 [hi][mid][lo]
    float *w3 = reinterpret_cast<float *>(sa + 3 * A_SPLIT);     // [9][128]
    float *gys = w3 + NO * NH;                                   // [128 atoms][16]
    uint64_t *done = reinterpret_cast<uint64_t *>(gys + MT * 16);
    uint32_t *slot = reinterpret_cast<uint32_t *>(done + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(slot, NH);
    if (tid == 0) tc::mbar_init(done, 1);
    load_weights_t(sw2t, reinterpret_cast<const uint16_t *>(w) + OFF_W2, NH, NH, LBO_W);
    for (int e = tid; e < NO * NH; e += FWD_THREADS) w3[e] = wv(w, OFF_W3 + e);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t sa_u = tc::smem_u32(sa), sw_u = tc::smem_u32(sw2t);
    const uint32_t quad = warp & 3, slice = warp >> 2;
    const uint32_t lanes = tmem + ((32u * quad) << 16);
    const int row = 32 * quad + lane;
    constexpr uint32_t ID128 = tc::idesc_bf16(MT, NH);
    const int n_tiles = (n + MT - 1) / MT;
    uint32_t pd = 0u;
    bool ok = true;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int t0 = t * MT;
        const bool real = t0 + row < n;
        for (int e = tid; e < MT * 16; e += FWD_THREADS) {
            const int at = e >> 4, o = e & 15;
            const float v = (o < NO && t0 + at < n) ? gy[(size_t)(t0 + at) * NO + o] : 0.0f;
            gys[e] = v;
            gyt[((size_t)t * 16 + o) * MT + at] = v;
        }
        __syncthreads();
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            float x[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int u = 32 * slice + 8 * g + q;
                float acc = 0.0f;
#pragma unroll
                for (int o = 0; o < NO; ++o) acc = fmaf(gys[row * 16 + o], w3[o * NH + u], acc);
                const float gz = real ? acc * dsilu(z2[(size_t)(t0 + row) * NH + u]) : 0.0f;
                x[q] = gz;
                gz2t[((size_t)t * NH + u) * MT + row] = gz;
            }
            split_store8(sa, tc::core_offset(row, 32 * slice + 8 * g, LBO_A), x);
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            layer_mma(tmem, sa_u, sw_u, LBO_W, NH, ID128);
            tc::mma_commit(done);
        }
        const bool mg = tc::mbar_wait(done, pd);
        pd ^= 1u;
        if (!__syncthreads_and(mg)) { ok = false; break; }
        tc::fence_after_sync();
        float v[32];
        tc::tmem_ld32(lanes + 32 * slice, v);
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const int u = 32 * slice + q;
            gz1t[((size_t)t * NH + u) * MT + row] = real ? v[q] * dsilu(z1[(size_t)(t0 + row) * NH + u]) : 0.0f;
        }
        tc::fence_before_sync();
        __syncthreads();   // TMEM read and gy tile consumed before the next tile
    }
    if (!ok && tid == 0) atomicOr(status, (unsigned)ERRBIT_TIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, NH);
}

// Weight gradients on the tensor cores: contractions over atoms, split over CTAs (each CTA sums its
// tiles in TMEM and writes one partial gradient; the partials are added in a fixed order). Per chunk
// of 32 atoms, with the feature-major tiles of the forward and backward kernels as K-major operands
// (K = atoms), each split into BF16 hi and lo and multiplied as hi hi + hi lo + lo hi:
//   D1[u][v] = sum_a gz2[a][u] [h1 | 1][a][v]   -> dW2[u][v] (v < 128) and db2[u] (column 128)
//   D2[u][i] = sum_a gz1[a][u] [x | 1][a][i]    -> dW1[u][i] (i < 32) and db1[u] (column 32)
//   D3[u][o] = sum_a h2[a][u] gy[a][o]           -> dW3[o][u]
// and db3[o] = sum_a gy[a][o] on the CUDA cores. TMEM columns: D1 0..143, D2 160..207, D3 224..239.
constexpr int WG_THREADS = 256;
constexpr int WG_K = 32;                                      // atoms per chunk
constexpr int WN1 = NH + 16, WN2 = NF + 16, WN3 = 16;         // B rows (the ones row, then zero rows)
constexpr uint32_t WGA = NH * WG_K * 2;                       // one BF16 part of a 128-row A operand
constexpr uint32_t WGB1 = WN1 * WG_K * 2, WGB2 = WN2 * WG_K * 2, WGB3 = WN3 * WG_K * 2;
constexpr uint32_t WG_OP = 2 * (3 * WGA + WGB1 + WGB2 + WGB3);
constexpr size_t WG_SMEM = WG_OP + 64;
constexpr uint32_t D2COL = 160, D3COL = 224;

// Rows [0, R_src) of a feature-major tile (rows of MT atoms) for atoms chunk*32 .. +31, the ones row
// (if any) and zero rows up to R, split into BF16 hi / lo in the K-major core layout (K = atoms).
__device__ __forceinline__ void wg_operand(uint8_t *hi, uint8_t *lo, const float *src, int R_src, int ones, int R,
                                           int chunk) {
    const uint32_t lbo = (uint32_t)(R / 8) * 128;
    for (int c = threadIdx.x; c < R * (WG_K / 8); c += WG_THREADS) {
        const int g = c / R, r = c - g * R;
        float x[8];
        if (r < R_src) {
            const float *p = src + (size_t)r * MT + chunk * WG_K + 8 * g;
            const float4 u0 = *reinterpret_cast<const float4 *>(p), u1 = *reinterpret_cast<const float4 *>(p + 4);
            x[0] = u0.x; x[1] = u0.y; x[2] = u0.z; x[3] = u0.w;
            x[4] = u1.x; x[5] = u1.y; x[6] = u1.z; x[7] = u1.w;
        } else {
            const float f = r == ones ? 1.0f : 0.0f;
#pragma unroll
            for (int q = 0; q < 8; ++q) x[q] = f;
        }
        uint4 ph, pl;
        ph.x = bf16x2_split(x[0], x[1]); ph.y = bf16x2_split(x[2], x[3]);
        ph.z = bf16x2_split(x[4], x[5]); ph.w = bf16x2_split(x[6], x[7]);
        pl.x = bf16x2_split(x[0], x[1]); pl.y = bf16x2_split(x[2], x[3]);
        pl.z = bf16x2_split(x[4], x[5]); pl.w = bf16x2_split(x[6], x[7]);
        const uint32_t off = tc::core_offset(r, 8 * g, lbo);
        *reinterpret_cast<uint4 *>(hi + off) = ph;
        *reinterpret_cast<uint4 *>(lo + off) = pl;
    }
}

__global__ void __launch_bounds__(WG_THREADS, 1) k_weight_grad_tc(int n, const float *__restrict__ gz2t,
                                                                const float *__restrict__ gz1t,
                                                                const float *__restrict__ h1t,
                                                                const float *__restrict__ h2t,
                                                                const float *__restrict__ xt,
                                                                const float *__restrict__ gyt,
                                                                float *__restrict__ part, unsigned *__restrict__ status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *a1h = smem, *a1l = a1h + WGA, *a2h = a1l + WGA, *a2l = a2h + WGA, *a3h = a2l + WGA, *a3l = a3h + WGA;
    uint8_t *b1h = a3l + WGA, *b1l = b1h + WGB1, *b2h = b1l + WGB1, *b2l = b2h + WGB2, *b3h = b2l + WGB2,
            *b3l = b3h + WGB3;
    uint64_t *done = reinterpret_cast<uint64_t *>(smem + WG_OP);
    uint32_t *slot = reinterpret_cast<uint32_t *>(done + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(slot, 256);
    if (tid == 0) tc::mbar_init(done, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    constexpr uint32_t LA = (NH / 8) * 128, L1 = (WN1 / 8) * 128, L2 = (WN2 / 8) * 128, L3 = (WN3 / 8) * 128;
    constexpr uint32_t I1 = tc::idesc_bf16(NH, WN1), I2 = tc::idesc_bf16(NH, WN2), I3 = tc::idesc_bf16(NH, WN3);
    const int n_tiles = (n + MT - 1) / MT;
    float db3 = 0.0f;   // thread o < 9: sum over this CTA's atoms of gy[.][o]
    uint32_t pd = 0u;
    bool ok = true, first = true, pending = false;
    for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        if (tid < NO)
            for (int at = 0; at < MT; ++at) db3 += gyt[((size_t)t * 16 + tid) * MT + at];
        for (int ch = 0; ch < MT / WG_K; ++ch) {
            if (pending) {   // the previous chunk's MMAs read the operands: wait before overwriting
                const bool mg = tc::mbar_wait(done, pd);
                pd ^= 1u;
                pending = false;
                if (!__syncthreads_and(mg)) { ok = false; break; }
            }
            wg_operand(a1h, a1l, gz2t + (size_t)t * NH * MT, NH, -1, NH, ch);
            wg_operand(a2h, a2l, gz1t + (size_t)t * NH * MT, NH, -1, NH, ch);
            wg_operand(a3h, a3l, h2t + (size_t)t * NH * MT, NH, -1, NH, ch);
            wg_operand(b1h, b1l, h1t + (size_t)t * NH * MT, NH, NH, WN1, ch);
            wg_operand(b2h, b2l, xt + (size_t)t * NF * MT, NF, NF, WN2, ch);
            wg_operand(b3h, b3l, gyt + (size_t)t * 16 * MT, NO, -1, WN3, ch);
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
                const uint32_t s0 = tc::smem_u32(smem);
                const uint32_t A1h = s0, A1l = A1h + WGA, A2h = A1l + WGA, A2l = A2h + WGA, A3h = A2l + WGA,
                               A3l = A3h + WGA, B1h = A3l + WGA, B1l = B1h + WGB1, B2h = B1l + WGB1,
                               B2l = B2h + WGB2, B3h = B2l + WGB2, B3l = B3h + WGB3;
                for (int k = 0; k < WG_K / 16; ++k) {
                    const uint32_t acc = (first && k == 0) ? 0u : 1u;
                    const uint32_t oa = k * 2 * LA;
                    const uint64_t a1hd = tc::make_desc(A1h + oa, LA, 128), a1ld = tc::make_desc(A1l + oa, LA, 128);
                    const uint64_t a2hd = tc::make_desc(A2h + oa, LA, 128), a2ld = tc::make_desc(A2l + oa, LA, 128);
                    const uint64_t a3hd = tc::make_desc(A3h + oa, LA, 128), a3ld = tc::make_desc(A3l + oa, LA, 128);
                    const uint64_t b1hd = tc::make_desc(B1h + k * 2 * L1, L1, 128), b1ld = tc::make_desc(B1l + k * 2 * L1, L1, 128);
                    const uint64_t b2hd = tc::make_desc(B2h + k * 2 * L2, L2, 128), b2ld = tc::make_desc(B2l + k * 2 * L2, L2, 128);
                    const uint64_t b3hd = tc::make_desc(B3h + k * 2 * L3, L3, 128), b3ld = tc::make_desc(B3l + k * 2 * L3, L3, 128);
                    tc::mma_bf16(tmem, a1hd, b1hd, I1, acc);
                    tc::mma_bf16(tmem, a1hd, b1ld, I1, 1u);
                    tc::mma_bf16(tmem, a1ld, b1hd, I1, 1u);
                    tc::mma_bf16(tmem + D2COL, a2hd, b2hd, I2, acc);
                    tc::mma_bf16(tmem + D2COL, a2hd, b2ld, I2, 1u);
                    tc::mma_bf16(tmem + D2COL, a2ld, b2hd, I2, 1u);
                    tc::mma_bf16(tmem + D3COL, a3hd, b3hd, I3, acc);
                    tc::mma_bf16(tmem + D3COL, a3hd, b3ld, I3, 1u);
                    tc::mma_bf16(tmem + D3COL, a3ld, b3hd, I3, 1u);
                }
                tc::mma_commit(done);
            }
            pending = true;
            first = false;
        }
    }
    if (pending) {
        const bool mg = tc::mbar_wait(done, pd);
        if (!__syncthreads_and(mg)) ok = false;
    }
    ok = __syncthreads_and(ok) != 0;
    if (!ok && tid == 0) atomicOr(status, (unsigned)ERRBIT_TIMEOUT);
    tc::fence_after_sync();
    float *P = part + (size_t)blockIdx.x * NPAR;
    if (warp < 4) {   // one weight row u per thread (TMEM lane u)
        const int u = 32 * warp + lane;
        const uint32_t lanes = tmem + ((32u * warp) << 16);
        const bool have = ok && !first;
        float v[32];
        for (int c0 = 0; c0 < WN1; c0 += 32) {
            tc::tmem_ld32(lanes + c0, v);
            for (int q = 0; q < 32 && c0 + q <= NH; ++q) {
                const float x = have ? v[q] : 0.0f;
                if (c0 + q < NH) P[OFF_W2 + u * NH + c0 + q] = x;
                else P[OFF_B2 + u] = x;
            }
        }
        for (int c0 = 0; c0 < WN2; c0 += 32) {
            tc::tmem_ld32(lanes + D2COL + c0, v);
            for (int q = 0; q < 32 && c0 + q <= NF; ++q) {
                const float x = have ? v[q] : 0.0f;
                if (c0 + q < NF) P[OFF_W1 + u * NF + c0 + q] = x;
                else P[OFF_B1 + u] = x;
            }
        }
        tc::tmem_ld32(lanes + D3COL, v);
        for (int o = 0; o < NO; ++o) P[OFF_W3 + o * NH + u] = have ? v[o] : 0.0f;
    }
    if (tid < NO) P[OFF_B3 + tid] = ok ? db3 : 0.0f;
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
                                float *R, unsigned *status, cudaStream_t st, int atoms_per_cell) {
    if (atoms_per_cell == 3)
        k_features_w3<<<(n_cells + FEAT_CELLS - 1) / FEAT_CELLS, FEAT_CELLS, 0, st>>>(n_cells, species, r, X, R,
                                                                                     status);
    else
        k_features<<<(n_cells + 127) / 128, 128, 0, st>>>(n_cells, off, species, r, X, R, status);
    return cudaGetLastError();
}

cudaError_t prepare_mlp_forward() {
    return cudaFuncSetAttribute(k_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FWD_SMEM);
}

static cudaError_t prepare_mlp_training() {
    cudaError_t e = prepare_mlp_forward();
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_backward_act_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BWA_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_weight_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WG_SMEM);
    return e;
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
    k_forward_tc<<<grid, FWD_TC_THREADS, FWD_SMEM, st>>>(n_atoms, X, R, (const __nv_bfloat16 *)w_bf16, Zl, status,
                                                    FwdStore{nullptr, nullptr, nullptr, nullptr, nullptr});
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
    // training activations: z1, z2 atom-major; h1t, h2t, gz2t, gz1t, xt, gyt feature-major per tile
    float *z1 = nullptr, *z2 = nullptr, *h1t = nullptr, *h2t = nullptr, *gz2t = nullptr, *gz1t = nullptr;
    float *xt = nullptr, *gyt = nullptr;
    int n_sm = 0;
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

// forward + loss + gradient over the cells [cell0, cell0 + ncells) of the (permuted) arrays, every
// product on the tensor cores: forward (the time step's kernel, keeping its activations), cell
// tensors and dL/dy, backward through the activations, weight gradients split over CTAs, and a
// fixed-order FP64 sum of the CTA partials
int mlp_loss_grad_range(cavmd_mlp *m, int cell0, int ncells, const float *X, const float *R, const double *Q,
                        const double *Zr, double inv_count) {
    const int a0 = 3 * cell0, na = 3 * ncells;
    const int tiles = (na + MT - 1) / MT;
    const int grid = std::min(tiles, m->n_sm);
    k_forward_tc<<<grid, FWD_TC_THREADS, FWD_SMEM, m->stream>>>(na, X + (size_t)a0 * NF, R + (size_t)a0 * 9, m->w,
                                                             m->Zl, m->status,
                                                             FwdStore{m->z1, m->z2, m->h1t, m->h2t, m->xt});
    k_cell_tensors<<<(ncells + 127) / 128, 128, 0, m->stream>>>(ncells, m->off, m->Zl, R + (size_t)a0 * 9, Q + a0,
                                                                Zr + (size_t)a0 * 9, inv_count, nullptr, m->gy,
                                                                m->lpart, 0, 0, 0, nullptr);
    k_backward_act_tc<<<grid, FWD_THREADS, BWA_SMEM, m->stream>>>(na, m->gy, m->z1, m->z2, m->w, m->gz2t, m->gz1t,
                                                                  m->gyt, m->status);
    k_weight_grad_tc<<<grid, WG_THREADS, WG_SMEM, m->stream>>>(na, m->gz2t, m->gz1t, m->h1t, m->h2t, m->xt, m->gyt,
                                                               m->part, m->status);
    k_reduce_grad<<<(NPAR + 255) / 256, 256, 0, m->stream>>>(grid, m->part, m->g);
    k_reduce_loss<<<1, 256, 0, m->stream>>>(ncells, m->lpart, inv_count, m->loss);
    MCK(cudaGetLastError());
    return CAVMD_OK;
}

// Reads and clears the device status word of the network's kernels.
int mlp_status(cavmd_mlp *m) {
    unsigned st = 0;
    MCK(cudaStreamSynchronize(m->stream));
    MCK(cudaMemcpy(&st, m->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (!st) return CAVMD_OK;
    MCK(cudaMemset(m->status, 0, sizeof(unsigned)));
    if (st & ERRBIT_TIMEOUT)
        return mlp_fail(m, CAVMD_ERR_DEVICE_TIMEOUT, "a tensor-core wait of the network kernels ran out");
    return mlp_fail(m, CAVMD_ERR_NONFINITE, "an atom has fewer than two neighbours within the cutoff (no local frame)");
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
    e = prepare_mlp_training();
    if (e != cudaSuccess) return done(mlp_fail(nullptr, CAVMD_ERR_CUDA, "cudaFuncSetAttribute (network kernels)"));
    e = cudaDeviceGetAttribute(&m->n_sm, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return done(mlp_fail(nullptr, CAVMD_ERR_CUDA, "cudaDeviceGetAttribute"));
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
    const size_t tiles = (size_t)(na + MT - 1) / MT, npad = tiles * MT;
    MAL(m->z1, npad * NH); MAL(m->z2, npad * NH);
    MAL(m->h1t, npad * NH); MAL(m->h2t, npad * NH); MAL(m->gz2t, npad * NH); MAL(m->gz1t, npad * NH);
    MAL(m->xt, npad * NF); MAL(m->gyt, npad * 16);
    MAL(m->part, (size_t)m->n_sm * NPAR);
    MCK(cudaMemcpy(m->off, off.data(), sizeof(int) * (n_cells + 1), cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(m->species, species, sizeof(int) * na, cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(m->r, r, sizeof(double) * 3 * na, cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(m->Q, Q, sizeof(double) * na, cudaMemcpyHostToDevice));
    if (Z_ref) MCK(cudaMemcpy(m->Zref, Z_ref, sizeof(double) * 9 * na, cudaMemcpyHostToDevice));
    else MCK(cudaMemset(m->Zref, 0, sizeof(double) * 9 * na));
    MCK(launch_mlp_features(n_cells, m->off, m->species, m->r, m->X, m->R, m->status, m->stream));
    return mlp_status(m);
}

int cavmd_mlp_loss_grad(cavmd_mlp *m, double *loss, float *grad) {
    if (!m || !m->n_cells || !loss) return mlp_fail(m, CAVMD_ERR_INVALID_ARG, "no data or NULL output");
    MCK(cudaSetDevice(m->device));
    int rc = mlp_loss_grad_range(m, 0, m->n_cells, m->X, m->R, m->Q, m->Zref, 1.0 / (9.0 * m->n_atoms));
    if (rc) return rc;
    MCK(cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    if (grad) MCK(cudaMemcpyAsync(grad, m->g, sizeof(float) * NPAR, cudaMemcpyDeviceToHost, m->stream));
    return mlp_status(m);
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
    return mlp_status(m);
}

int cavmd_mlp_predict(cavmd_mlp *m, double *Z_out) {
    if (!m || !m->n_cells || !Z_out) return mlp_fail(m, CAVMD_ERR_INVALID_ARG, "no data or NULL output");
    MCK(cudaSetDevice(m->device));
    MCK(launch_mlp_forward(m->n_atoms, m->X, m->R, m->w, m->Zl, m->status, m->stream));
    k_cell_tensors<<<(m->n_cells + 127) / 128, 128, 0, m->stream>>>(m->n_cells, m->off, m->Zl, m->R, m->Q, nullptr,
                                                                    0.0, m->Zout, nullptr, nullptr, 0, 0, 0, nullptr);
    MCK(cudaGetLastError());
    MCK(cudaMemcpyAsync(Z_out, m->Zout, sizeof(double) * 9 * m->n_atoms, cudaMemcpyDeviceToHost, m->stream));
    return mlp_status(m);
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
