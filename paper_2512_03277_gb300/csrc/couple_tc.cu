// Mixed-precision coupling contraction on the fifth-generation tensor cores (modes on a uniform
// in-plane grid).
//
// Modes a = (jx, jy, s), k_a = (jx dkx, jy dky, 0), u_a(R) = cos(k_a.R) (s = 0) or sin(k_a.R)
// (s = 1), index a = s + 2 (jy + Ky2 jx). With thx_n = dkx X_n, thy_n = dky Y_n the phases
// factorise (cos(a + b) = cos a cos b - sin a sin b, sin(a + b) = sin a cos b + cos a sin b), so
//   forward:  G = A B^T,  A[i][n] = cos(jx thx_n) (i = jx) | sin(jx thx_n) (i = Kx + jx),
//             B[j][n] = M_n cos(jy thy_n) (j = jy) | M_n sin(jy thy_n) (j = Ky2 + jy),
//             D_cos = lambda (G[jx][jy] - G[Kx+jx][Ky2+jy]),  D_sin = lambda (G[Kx+jx][jy] + G[jx][Ky2+jy]);
//   back:     E_n = sum_i A[i][n] T[i][n],  T = Wt Y^T,  Y[n][j] = cos|sin(jy thy_n),
//             Wt[jx][jy] = Wc, Wt[jx][Ky2+jy] = Ws, Wt[Kx+jx][jy] = Ws, Wt[Kx+jx][Ky2+jy] = -Wc,
// the exact contraction of the k-space form of the coupling (no N x M phase matrix is stored).
// Operands are split x = hi + lo into bfloat16 pairs and multiplied as hi hi + hi lo + lo hi
// with FP32 accumulation in TMEM (BF16x3). The forward product is split over cells across CTAs;
// every TMEM accumulator covers one 32-cell stage and is folded into compensated FP32 sums, and the
// partial Gram matrices of the CTAs are summed in a fixed order in FP64.
#include <cuda_bf16.h>

#include <algorithm>

#include "tc_common.cuh"

namespace {

constexpr int KXP = 128;          // MMA M: 2 Kx rows padded to 128
constexpr int FWD_CELLS = 64;     // cells (K) per tile of the forward panels in HBM
constexpr int FWD_SC = 32;        // cells (K) per forward stage: half a panel tile
constexpr int FWD_NST = 4;        // forward stages in flight
constexpr int FWD_THREADS = 512;  // sixteen warps: four per TMEM lane quadrant in the forward fold
constexpr int BACK_CELLS = 128;   // cells (N) per back tile

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Stores of one phase value into the panels, in tile-major core-matrix order.
struct Panels {
    int Npad, KY;
    __nv_bfloat16 *Ahi, *Alo, *Yhi, *Ylo;
    float *Af, *Bsrc;
    // x phase row i of cell n: forward A (hi, lo; tile t = n / 64, K = n % 64, LBO = 16 row groups x
    // 128 B) and the FP32 back-epilogue panel Af[i][n]
    __device__ __forceinline__ void put_x(int n, int i, float v) const {
        const int t = n / FWD_CELLS, kk = n - t * FWD_CELLS;
        __nv_bfloat16 hi, lo;
        split_bf16(v, hi, lo);
        const size_t e = (size_t)t * KXP * FWD_CELLS + tc::core_offset(i, kk, (KXP / 8) * 128) / 2;
        Ahi[e] = hi;
        Alo[e] = lo;
        Af[(size_t)i * Npad + n] = v;
    }
    // y phase column j of cell n: forward B source (FP32, same tiles as A) and back Y (hi, lo; tile
    // tb = n / 128, row n % 128, K = j)
    __device__ __forceinline__ void put_y(int n, int j, float v) const {
        const int t = n / FWD_CELLS, kk = n - t * FWD_CELLS;
        Bsrc[(size_t)t * KY * FWD_CELLS + tc::core_offset(j, kk, (KY / 8) * 128) / 2] = v;
        const int tb = n / BACK_CELLS, rb = n - tb * BACK_CELLS;
        const size_t eb = (size_t)tb * BACK_CELLS * KY + tc::core_offset(rb, j, (BACK_CELLS / 8) * 128) / 2;
        __nv_bfloat16 hi, lo;
        split_bf16(v, hi, lo);
        Yhi[eb] = hi;
        Ylo[eb] = lo;
    }
};

// Init: phase panels from the x and y phases in FP64 (cos / sin rounded once to FP32). Padding
// rows, columns and cells are written as zeros.
__global__ void k_tc_panels(int N, int Kx, int Ky2, double dkx, double dky, const double *__restrict__ R,
                            const Panels P) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= P.Npad) return;
    const bool real = n < N;
    const double tx = real ? dkx * R[3 * n] : 0.0, ty = real ? dky * R[3 * n + 1] : 0.0;
    for (int i = 0; i < KXP; ++i) {
        double v = 0.0;
        if (real && i < 2 * Kx) v = (i < Kx) ? cos(i * tx) : sin((i - Kx) * tx);
        P.put_x(n, i, (float)v);
    }
    for (int j = 0; j < P.KY; ++j) {
        double v = 0.0;
        if (real && j < 2 * Ky2) v = (j < Ky2) ? cos(j * ty) : sin((j - Ky2) * ty);
        P.put_y(n, j, (float)v);
    }
}

// A phase angle held as a fraction of a turn in 64-bit fixed point (units of 2^-64 turn, modulo
// one turn), from t turns in FP64: t - rint(t) is exact and so is its scaling by 2^63.
__device__ __forceinline__ uint64_t turns_fixed(double t) {
    const double g = t - rint(t);
    return (uint64_t)__double2ll_rn(g * 0x1p63) << 1;
}

// cos and sin of the angle j T (T in fixed-point turns). The product j T is exact modulo one turn;
// its nearest quarter turn q comes from the top two bits (after adding 1/8 turn) and the remainder r,
// |r| <= 1/8 turn, is converted to FP32 with integer operations only (normalised by its leading
// zeros, significand truncated: relative error below 2^-23, also near the zeros of cos and sin);
// sincospif evaluates the remainder (CUDA states at most 1 ulp) and the quarter turn permutes and
// negates the pair exactly: (cos, sin)(q/4 turn + r) = (c, s), (-s, c), (-c, -s), (s, -c).
__device__ __forceinline__ void turn_sincos(uint64_t T, unsigned j, float &c, float &s) {
    const uint64_t u = T * (uint64_t)j + (1ull << 61);
    const unsigned q = (unsigned)(u >> 62);
    const long long rem = (long long)(u & ((1ull << 62) - 1ull)) - (1ll << 61);   // r in units of 2^-64 turn
    const unsigned long long a = rem < 0 ? (unsigned long long)(-rem) : (unsigned long long)rem;
    float x = 0.0f;   // 2 r: the remainder in half turns
    if (a != 0ull) {
        const int lz = __clzll((long long)a);   // >= 3, as a < 2^61
        const unsigned long long m = a << lz;
        const uint32_t bits = ((uint32_t)(127 - lz) << 23) | ((uint32_t)(m >> 40) & 0x7fffffu);
        x = __uint_as_float(bits | (rem < 0 ? 0x80000000u : 0u));
    }
    float sr, cr;
    sincospif(x, &sr, &cr);
    switch (q) {
        case 0: c = cr; s = sr; break;
        case 1: c = -sr; s = cr; break;
        case 2: c = -cr; s = -sr; break;
        default: c = sr; s = -cr; break;
    }
}

// Every step with moving mode positions: the phase panels at the cells' centres of mass
// R_n = sum_j m_j r_j / m_n (summed over the cell's atoms in order), with the phases cos | sin(jx dkx X_n)
// and cos | sin(jy dky Y_n) from turn_sincos (the FP32 values carry a relative error of at most
// about 3 * 2^-24). One block per 64-cell forward tile, four threads per cell (each a quarter of
// the wave numbers). The tile's forward panels and its half of a back tile are built in shared
// memory (zeros first, so padding rows, columns and cells stay zero) and leave as 16-byte stores
// of whole contiguous runs; the FP32 x panel goes out directly (coalesced over the cells).
constexpr int PCOM_THREADS = 256;
__host__ __device__ constexpr size_t pcom_smem(int KY) {
    return 2 * (size_t)KXP * FWD_CELLS * 2 + (size_t)KY * FWD_CELLS * 4 + 2 * (size_t)KY * FWD_CELLS * 2;
}
__global__ void __launch_bounds__(PCOM_THREADS) k_tc_panels_com(int N, int Kx, int Ky2, double x_turns,
                                                                  double y_turns, const double *__restrict__ r,
                                                                  const double *__restrict__ mass,
                                                                  const int *__restrict__ off, const Panels P) {
    extern __shared__ __align__(16) uint8_t psm[];
    const int KY = P.KY;
    const uint32_t A_B = KXP * FWD_CELLS * 2, B_B = KY * FWD_CELLS * 4, Y_B = KY * FWD_CELLS * 2;
    __nv_bfloat16 *sAhi = reinterpret_cast<__nv_bfloat16 *>(psm), *sAlo = sAhi + KXP * FWD_CELLS;
    float *sB = reinterpret_cast<float *>(psm + 2 * A_B);
    __nv_bfloat16 *sYhi = reinterpret_cast<__nv_bfloat16 *>(psm + 2 * A_B + B_B), *sYlo = sYhi + KY * FWD_CELLS;
    const uint32_t total = 2 * A_B + B_B + 2 * Y_B;
    for (uint32_t e = threadIdx.x; e < total / 16; e += PCOM_THREADS)
        reinterpret_cast<uint4 *>(psm)[e] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    const int t = blockIdx.x, c = threadIdx.x & (FWD_CELLS - 1), qq = threadIdx.x / FWD_CELLS;
    const int n = t * FWD_CELLS + c;
    const int h = t & 1;   // which half of its 128-cell back tile this forward tile is
    if (n < N) {
        double mt = 0.0, x0 = 0.0, x1 = 0.0;
        for (int j = off[n]; j < off[n + 1]; ++j) {
            const double m = mass[j];
            mt += m;
            x0 = fma(m, r[3 * j], x0);
            x1 = fma(m, r[3 * j + 1], x1);
        }
        const uint64_t Tx = turns_fixed(x0 / mt * x_turns), Ty = turns_fixed(x1 / mt * y_turns);
        auto put_x = [&](int i, float v) {
            __nv_bfloat16 hi, lo;
            split_bf16(v, hi, lo);
            const uint32_t e = tc::core_offset(i, c, (KXP / 8) * 128) / 2;
            sAhi[e] = hi;
            sAlo[e] = lo;
            P.Af[(size_t)i * P.Npad + n] = v;
        };
        auto put_y = [&](int j, float v) {
            sB[tc::core_offset(j, c, (KY / 8) * 128) / 2] = v;
            // back Y: row c of this half tile, K = j: (j / 8) runs of 1 KB in the staging buffer
            const uint32_t e = ((uint32_t)(j >> 3) * 1024u + (uint32_t)(c >> 3) * 128u + (uint32_t)(c & 7) * 16u +
                                (uint32_t)(j & 7) * 2u) / 2;
            __nv_bfloat16 hi, lo;
            split_bf16(v, hi, lo);
            sYhi[e] = hi;
            sYlo[e] = lo;
        };
        for (int jx = qq; jx < Kx; jx += PCOM_THREADS / FWD_CELLS) {
            float cs, sn;
            turn_sincos(Tx, (unsigned)jx, cs, sn);
            put_x(jx, cs);
            put_x(Kx + jx, sn);
        }
        for (int jy = qq; jy < Ky2; jy += PCOM_THREADS / FWD_CELLS) {
            float cs, sn;
            turn_sincos(Ty, (unsigned)jy, cs, sn);
            put_y(jy, cs);
            put_y(Ky2 + jy, sn);
        }
    }
    __syncthreads();
    // whole runs out: the forward tile's A hi, A lo and B (contiguous), the half back tile's Y in
    // KY / 8 runs of 1 KB (its 64 rows of every K group)
    uint4 *gAhi = reinterpret_cast<uint4 *>(P.Ahi + (size_t)t * KXP * FWD_CELLS);
    uint4 *gAlo = reinterpret_cast<uint4 *>(P.Alo + (size_t)t * KXP * FWD_CELLS);
    uint4 *gB = reinterpret_cast<uint4 *>(P.Bsrc + (size_t)t * KY * FWD_CELLS);
    const uint4 *s4 = reinterpret_cast<const uint4 *>(psm);
    for (uint32_t e = threadIdx.x; e < A_B / 16; e += PCOM_THREADS) {
        gAhi[e] = s4[e];
        gAlo[e] = s4[A_B / 16 + e];
    }
    for (uint32_t e = threadIdx.x; e < B_B / 16; e += PCOM_THREADS) gB[e] = s4[2 * A_B / 16 + e];
    const size_t ybase = (size_t)(t >> 1) * BACK_CELLS * KY;   // elements
    for (uint32_t e = threadIdx.x; e < Y_B / 16; e += PCOM_THREADS) {
        const uint32_t kc = e / 64, w = e - kc * 64;   // 64 uint4 per 1 KB run
        const size_t g = ybase + ((size_t)kc * 2048 + (size_t)h * 1024) / 2;   // elements
        reinterpret_cast<uint4 *>(P.Yhi + g)[w] = s4[(2 * A_B + B_B) / 16 + e];
        reinterpret_cast<uint4 *>(P.Ylo + g)[w] = s4[(2 * A_B + B_B + Y_B) / 16 + e];
    }
}

// Forward Gram product, split over cells: partial[cta][i][j] = sum over the CTA's cells of A B^T.
// Each 32-cell stage arrives by bulk copies (the BF16 hi / lo panels of A and the FP32 y-phase panel
// of B, all pre-arranged in core-matrix order); up to FWD_NST stages are in flight. The sixteen warps
// scale the y phases by M_n (converted and staged in shared memory one stage ahead) and split them
// into the BF16 hi / lo panels of B in shared memory, and one thread issues the stage's MMAs into a
// fresh TMEM accumulator (two, alternating) and the bulk copies. The FP32 run of an accumulator is
// therefore one stage: 32 cells, 6 MMAs. While the next stage's MMAs run, the warps fold the
// finished accumulator into per-thread compensated FP32 sums (two-sum: the rounding error of every
// addition is carried in a second register), so the accumulated error does not grow with the
// number of cells a CTA owns. The partials leave as FP64 (sum + carried error).
template <int KY>
__global__ void __launch_bounds__(FWD_THREADS, 1) k_tc_forward(int n_stage_total, int st_per_cta,
                                                                const __nv_bfloat16 *__restrict__ Ahi,
                                                                const __nv_bfloat16 *__restrict__ Alo,
                                                                const float *__restrict__ Bsrc,
                                                                const double *__restrict__ Mc, int N,
                                                                double *__restrict__ partial,
                                                                unsigned *__restrict__ status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr uint32_t A_BYTES = KXP * FWD_SC * 2, B_BYTES = KY * FWD_SC * 2, S_BYTES = KY * FWD_SC * 4;
    constexpr uint32_t STAGE = 2 * A_BYTES + 2 * B_BYTES + S_BYTES;   // [A hi][A lo][B hi][B lo][B source]
    constexpr uint32_t LBO_A = (KXP / 8) * 128, LBO_B = (KY / 8) * 128;
    constexpr uint32_t TC = KY <= 32 ? 32 : (KY <= 64 ? 64 : 128);    // columns of one accumulator
    constexpr int NGRP = KY / 8;                                       // 8-column groups of an accumulator
    constexpr int GPT = (NGRP + 3) / 4;                                // groups folded per thread (at most)
    constexpr int NCHUNK = KY * FWD_SC / 8;                            // split chunks: 8 cells of one row
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + FWD_NST * STAGE);   // [NST] stage data arrived
    uint64_t *done = full + FWD_NST;                                         // [NST] stage MMAs finished
    uint32_t *slot = reinterpret_cast<uint32_t *>(done + FWD_NST);
    float *ms = reinterpret_cast<float *>(slot + 4);                         // [2][32] M_n of two stages
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q0 = blockIdx.x * st_per_cta;
    const int nq = max(0, min(n_stage_total, q0 + st_per_cta) - q0);
    if (warp == 0) tc::tmem_alloc(slot, 2 * TC);
    if (tid == 0) {
        for (int s = 0; s < FWD_NST; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&done[s], 1);
        }
    }
    // the dipoles of local stage i in FP32 (converted once: a conversion from FP64 runs on the FP64
    // pipe), loaded by warp 1 a stage ahead and stored into ms[i & 1] after its fold
    auto load_m = [&](int i) -> float {
        const int n = (q0 + i) * FWD_SC + lane;
        return (warp == 1 && i < nq && n < N) ? (float)__ldg(Mc + n) : 0.0f;
    };
    if (warp == 1) ms[lane] = load_m(0);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t idesc = tc::idesc_bf16(KXP, KY);
    // warps w, w + 4, w + 8, w + 12 read the same TMEM lane quadrant (w & 3); warp part p = w / 4
    // folds the 8-column groups p, p + 4, ...
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const int part = warp >> 2;
    auto issue = [&](int i) {   // thread 0: the copies of local stage i into slot i % NST
        const int s = i % FWD_NST;
        const size_t q = (size_t)(q0 + i);
        uint8_t *st = smem + s * STAGE;
        tc::mbar_arrive_expect_tx(&full[s], 2 * A_BYTES + S_BYTES);
        tc::bulk_g2s(st, Ahi + q * KXP * FWD_SC, A_BYTES, &full[s]);
        tc::bulk_g2s(st + A_BYTES, Alo + q * KXP * FWD_SC, A_BYTES, &full[s]);
        tc::bulk_g2s(st + 2 * A_BYTES + 2 * B_BYTES, Bsrc + q * KY * FWD_SC, S_BYTES, &full[s]);
    };
    float acc_s[GPT * 8], acc_c[GPT * 8];
#pragma unroll
    for (int j = 0; j < GPT * 8; ++j) {
        acc_s[j] = 0.0f;
        acc_c[j] = 0.0f;
    }
    // all threads: the accumulator of local stage i (TMEM buffer i & 1) into the compensated sums
    auto fold = [&](int i) {
        const uint32_t base = tmem + lane_base + (uint32_t)((i & 1) * TC);
        uint32_t r[GPT][8];
#pragma unroll
        for (int g = 0; g < GPT; ++g)
            if (part + 4 * g < NGRP) tc::tmem_ld8_nowait(base + (uint32_t)(8 * (part + 4 * g)), r[g]);
        tc::tmem_wait_ld();
#pragma unroll
        for (int g = 0; g < GPT; ++g) {
            if (part + 4 * g >= NGRP) continue;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int j = 8 * g + k;
                const float x = __uint_as_float(r[g][k]);
                const float s = acc_s[j];
                const float t = __fadd_rn(s, x);
                const float z = __fsub_rn(t, s);
                const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(x, z));   // s + x - t exactly
                acc_s[j] = t;
                acc_c[j] = __fadd_rn(acc_c[j], e);
            }
        }
    };
    int n_issued = 0;   // thread 0's count of stages whose copies were issued
    if (tid == 0)
        for (; n_issued < min(nq, FWD_NST - 1); ++n_issued) issue(n_issued);
    bool ok = true, wd = true;   // wd: the last wait for a stage's MMAs (checked at the next barrier)
    int i = 0;
    for (; i < nq; ++i) {
        const int s = i % FWD_NST;
        const bool w = tc::mbar_wait(&full[s], (i / FWD_NST) & 1);   // stage i's data arrived
        if (!__syncthreads_and(w && wd)) { ok = false; break; }
        uint8_t *st = smem + s * STAGE;
        const float *bs = reinterpret_cast<const float *>(st + 2 * A_BYTES + 2 * B_BYTES);
        const float *mi = ms + (i & 1) * FWD_SC;
        for (int c = tid; c < NCHUNK; c += FWD_THREADS) {   // 8 consecutive cells of one row per chunk
            const int kgrp = c / KY, row = c - kgrp * KY;
            const uint32_t off = tc::core_offset(row, 8 * kgrp, LBO_B);
            const float4 v0 = *reinterpret_cast<const float4 *>(bs + off / 2);
            const float4 v1 = *reinterpret_cast<const float4 *>(bs + off / 2 + 4);
            const float vv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
            __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) split_bf16(vv[q] * mi[8 * kgrp + q], hi[q], lo[q]);
            *reinterpret_cast<uint4 *>(st + 2 * A_BYTES + off) = *reinterpret_cast<const uint4 *>(hi);
            *reinterpret_cast<uint4 *>(st + 2 * A_BYTES + B_BYTES + off) = *reinterpret_cast<const uint4 *>(lo);
        }
        tc::fence_before_sync();   // the previous fold's TMEM reads are complete before MMAs reuse its buffer
        tc::fence_proxy_async();
        __syncthreads();
        const float m_next = load_m(i + 1);   // in flight during the fold
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t sa = tc::smem_u32(st), sb = sa + 2 * A_BYTES;
            const uint32_t d = tmem + (uint32_t)((i & 1) * TC);
#pragma unroll
            for (int k = 0; k < FWD_SC / 16; ++k) {
                const uint32_t oa = k * 2 * LBO_A, ob = k * 2 * LBO_B;
                const uint64_t ahd = tc::make_desc(sa + oa, LBO_A, 128), ald = tc::make_desc(sa + A_BYTES + oa, LBO_A, 128);
                const uint64_t bhd = tc::make_desc(sb + ob, LBO_B, 128), bld = tc::make_desc(sb + B_BYTES + ob, LBO_B, 128);
                tc::mma_bf16(d, ahd, bhd, idesc, k > 0 ? 1u : 0u);   // a fresh accumulator every stage
                tc::mma_bf16(d, ahd, bld, idesc, 1u);
                tc::mma_bf16(d, ald, bhd, idesc, 1u);
            }
            tc::mma_commit(&done[s]);
        }
        __syncwarp();
        // while stage i's MMAs run: stage i - 1's are done, so its slot is refilled (with stage
        // i + NST - 1; at i = 0 the one slot the prologue left empty) and its accumulator folded
        if (i > 0) wd = tc::mbar_wait(&done[(i - 1) % FWD_NST], ((i - 1) / FWD_NST) & 1);
        if (tid == 0 && wd && n_issued < nq && n_issued == i + FWD_NST - 1) issue(n_issued++);
        if (i > 0) {
            tc::fence_after_sync();
            fold(i - 1);
        }
        if (warp == 1) ms[((i + 1) & 1) * FWD_SC + lane] = m_next;   // read at stage i + 1, after a barrier
    }
    if (ok && nq > 0) {   // the last stage
        const bool w = tc::mbar_wait(&done[(nq - 1) % FWD_NST], ((nq - 1) / FWD_NST) & 1);
        if (__syncthreads_and(w && wd)) {
            tc::fence_after_sync();
            fold(nq - 1);
        } else {
            ok = false;
        }
    } else if (!ok && tid == 0) {   // a wait gave up at stage i: let what is in flight land first
        if (i > 0) tc::mbar_wait(&done[(i - 1) % FWD_NST], ((i - 1) / FWD_NST) & 1);
        for (int j = i; j < n_issued; ++j) tc::mbar_wait(&full[j % FWD_NST], (j / FWD_NST) & 1);
    }
    ok = __syncthreads_and(ok) != 0;
    if (!ok && tid == 0) atomicOr(status, (unsigned)ERRBIT_TIMEOUT);
    double *P = partial + (size_t)blockIdx.x * KXP * KY + (size_t)(32 * (warp & 3) + lane) * KY;
#pragma unroll
    for (int g = 0; g < GPT; ++g) {
        if (part + 4 * g >= NGRP) continue;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            P[8 * (part + 4 * g) + k] = ok ? (double)acc_s[8 * g + k] + (double)acc_c[8 * g + k] : 0.0;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 2 * TC);
}

__global__ void k_tc_reduce(int n_part, int size, const double *__restrict__ partial, double *__restrict__ G) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= size) return;
    double s = 0.0;
    for (int p = 0; p < n_part; ++p) s += partial[(size_t)p * size + e];
    G[e] = s;
}

// Back product, persistent over tiles of 128 cells: D[n][i] = sum_j Y[n][j] Wt[i][j] (cells on the
// TMEM lanes) for one or two weight matrices (Wt2 -> E2, Wt1 -> E1), then E_n = sum_i A[i][n] D[n][i]
// with one thread per cell reading A coalesced (FP32 within each 32-row chunk, FP64 across chunks).
// The weights are split into BF16 hi / lo once per CTA; each tile's Y panels arrive by bulk copy,
// issued as soon as the previous tile's MMAs have finished, so the copy overlaps the epilogue.
//
// GRAD (moving mode positions; one weight matrix Wt2): also the gradient of E_n with respect to the
// cell's centre, G_n = sum_a W_a grad u_a(R_n) (k_a in plane, so G_z = 0). With the factorised
// phases, d/dX acts on the x rows: d cos(jx thx)/dX = -jx dkx sin(jx thx), d sin(jx thx)/dX =
// jx dkx cos(jx thx), so G_x = sum_i A'[i][n] D[n][i] with A'[jx] = -jx dkx A[Kx + jx] and
// A'[Kx + jx] = jx dkx A[jx], in the same epilogue. d/dY acts on the y columns; moved onto the
// weights, D'[n][i] = sum_j Y[n][j] V[i][j] with V[i][jy] = jy dky Wt[i][Ky2 + jy] and
// V[i][Ky2 + jy] = -jy dky Wt[i][jy], a second accumulator, and G_y = sum_i A[i][n] D'[n][i].
template <int KY, bool GRAD>
__global__ void __launch_bounds__(128) k_tc_back(int N, int Npad, int n_tiles, const float *__restrict__ Wt2,
                                                 const float *__restrict__ Wt1, const __nv_bfloat16 *__restrict__ Yhi,
                                                 const __nv_bfloat16 *__restrict__ Ylo, const float *__restrict__ Af,
                                                 double *__restrict__ E2, double *__restrict__ E1,
                                                 double *__restrict__ G, int Kx, int Ky2, float dkx, float dky,
                                                 unsigned *__restrict__ status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr uint32_t W_BYTES = KXP * KY * 2, Y_BYTES = BACK_CELLS * KY * 2;
    constexpr uint32_t LBO_W = (KXP / 8) * 128, LBO_Y = (BACK_CELLS / 8) * 128;
    uint8_t *sw = smem;                       // [Wt2 hi][Wt2 lo][Wt1 hi][Wt1 lo] (GRAD: [.. V hi][V lo])
    uint8_t *sy = smem + 4 * W_BYTES;         // [Y hi][Y lo]
    uint64_t *full = reinterpret_cast<uint64_t *>(sy + 2 * Y_BYTES);
    uint64_t *done = full + 1;
    uint32_t *slot = reinterpret_cast<uint32_t *>(done + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nacc = (GRAD || Wt1) ? 2 : 1;
    if (warp == 0) tc::tmem_alloc(slot, 256);
    if (tid == 0) {
        tc::mbar_init(full, 1);
        tc::mbar_init(done, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    auto issue = [&](int t) {   // thread 0: the Y panels of tile t
        tc::mbar_arrive_expect_tx(full, 2 * Y_BYTES);
        tc::bulk_g2s(sy, Yhi + (size_t)t * BACK_CELLS * KY, Y_BYTES, full);
        tc::bulk_g2s(sy + Y_BYTES, Ylo + (size_t)t * BACK_CELLS * KY, Y_BYTES, full);
    };
    if (tid == 0 && (int)blockIdx.x < n_tiles) issue(blockIdx.x);
    bool pending = (int)blockIdx.x < n_tiles;
    // weights: 8 consecutive K (j) of one row i per chunk, split into hi / lo (once per CTA)
    for (int w = 0; w < nacc; ++w) {
        for (int c = tid; c < KXP * KY / 8; c += 128) {
            const int kgrp = c / KXP, row = c - kgrp * KXP;
            const uint32_t off = tc::core_offset(row, 8 * kgrp, LBO_W);
            __align__(16) __nv_bfloat16 hi[8], lo[8];
            for (int q = 0; q < 8; ++q) {
                const int j = 8 * kgrp + q;
                float v;
                if (!GRAD || w == 0) {
                    v = (w == 0 ? Wt2 : Wt1)[row * KY + j];
                } else if (j < Ky2) {
                    v = ((float)j * dky) * Wt2[row * KY + Ky2 + j];
                } else if (j < 2 * Ky2) {
                    v = -((float)(j - Ky2) * dky) * Wt2[row * KY + j - Ky2];
                } else {
                    v = 0.0f;
                }
                split_bf16(v, hi[q], lo[q]);
            }
            *reinterpret_cast<uint4 *>(sw + (2 * w) * W_BYTES + off) = *reinterpret_cast<const uint4 *>(hi);
            *reinterpret_cast<uint4 *>(sw + (2 * w + 1) * W_BYTES + off) = *reinterpret_cast<const uint4 *>(lo);
        }
    }
    tc::fence_proxy_async();
    __syncthreads();
    const uint32_t tmem = *slot;
    const uint32_t idesc = tc::idesc_bf16(BACK_CELLS, KXP);
    uint32_t pf = 0u, pd = 0u;
    bool ok = true;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const bool got = tc::mbar_wait(full, pf);
        if (got) {
            pf ^= 1u;
            pending = false;
        }
        if (!__syncthreads_and(got)) { ok = false; break; }
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t sws = tc::smem_u32(sw), sys = tc::smem_u32(sy);
            for (int w = 0; w < nacc; ++w) {
                const uint32_t d = tmem + (uint32_t)(w * KXP);
                for (int k = 0; k < KY / 16; ++k) {
                    const uint32_t ow = k * 2 * LBO_W, oy = k * 2 * LBO_Y;
                    const uint64_t whd = tc::make_desc(sws + (2 * w) * W_BYTES + ow, LBO_W, 128);
                    const uint64_t wld = tc::make_desc(sws + (2 * w + 1) * W_BYTES + ow, LBO_W, 128);
                    const uint64_t yhd = tc::make_desc(sys + oy, LBO_Y, 128), yld = tc::make_desc(sys + Y_BYTES + oy, LBO_Y, 128);
                    tc::mma_bf16(d, yhd, whd, idesc, k > 0 ? 1u : 0u);
                    tc::mma_bf16(d, yld, whd, idesc, 1u);
                    tc::mma_bf16(d, yhd, wld, idesc, 1u);
                }
            }
            tc::mma_commit(done);
        }
        const bool mg = tc::mbar_wait(done, pd);
        pd ^= 1u;
        if (!__syncthreads_and(mg)) { ok = false; break; }
        tc::fence_after_sync();
        if (t + (int)gridDim.x < n_tiles) {   // the Y stage is free again: fetch the next tile now
            if (tid == 0) issue(t + gridDim.x);
            pending = true;
        }
        const int n = t * BACK_CELLS + tid;   // this thread's cell (TMEM lane)
        const uint32_t lanes = (uint32_t)(32 * warp) << 16;
        if (GRAD) {
            double e = 0.0, gx = 0.0, gy = 0.0;
            for (int c0 = 0; c0 < KXP; c0 += 32) {
                float v[32], vd[32];
                tc::tmem_ld32(tmem + lanes + (uint32_t)c0, v);
                tc::tmem_ld32(tmem + lanes + (uint32_t)(KXP + c0), vd);
                // A'[i][n] = g_i A[swap(i)][n]: swap(i) = Kx + i, g_i = -i dkx (i < Kx); swap(i) = i - Kx,
                // g_i = (i - Kx) dkx (i < 2 Kx); padding rows g_i = 0. Loads without branches, so that
                // the 64 loads of a chunk are all in flight before the sums.
                float a[32], as[32];
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const int i = c0 + q;
                    const int sw = i < Kx ? Kx + i : (i < 2 * Kx ? i - Kx : i);
                    a[q] = Af[(size_t)i * Npad + n];
                    as[q] = Af[(size_t)sw * Npad + n];
                }
                float s = 0.0f, sx = 0.0f, sy2 = 0.0f;
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const int i = c0 + q;
                    const float g = i < Kx ? -((float)i * dkx) : (i < 2 * Kx ? (float)(i - Kx) * dkx : 0.0f);
                    s = fmaf(a[q], v[q], s);
                    sy2 = fmaf(a[q], vd[q], sy2);
                    sx = fmaf(g * as[q], v[q], sx);
                }
                e += (double)s;
                gx += (double)sx;
                gy += (double)sy2;
            }
            if (n < N) {
                E2[n] = e;
                G[3 * n] = gx;
                G[3 * n + 1] = gy;
                G[3 * n + 2] = 0.0;
            }
        } else {
            for (int w = 0; w < nacc; ++w) {
                double e = 0.0;
                for (int c0 = 0; c0 < KXP; c0 += 32) {
                    float v[32];
                    tc::tmem_ld32(tmem + lanes + (uint32_t)(w * KXP + c0), v);
                    float s = 0.0f;
#pragma unroll
                    for (int q = 0; q < 32; ++q) s = fmaf(Af[(size_t)(c0 + q) * Npad + n], v[q], s);
                    e += (double)s;
                }
                if (n < N) (w == 0 ? E2 : E1)[n] = e;
            }
        }
        tc::fence_before_sync();
        __syncthreads();   // TMEM reads done before the next tile's MMAs
    }
    if (tid == 0 && pending) tc::mbar_wait(full, pf);   // a copy still in flight lands before exit
    if (!ok && tid == 0) atomicOr(status, (unsigned)ERRBIT_TIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

template <typename F>
cudaError_t set_smem(F f, size_t bytes) {
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

// ---------------------------------------------------------------------------------------- host

size_t tc_fwd_smem(int KY) {
    return FWD_NST * (2 * (size_t)KXP * FWD_SC * 2 + 2 * (size_t)KY * FWD_SC * 2 + (size_t)KY * FWD_SC * 4) + 512;
}
int tc_fwd_stage_cells() { return FWD_SC; }
size_t tc_back_smem(int KY) { return 4 * (size_t)KXP * KY * 2 + 2 * (size_t)BACK_CELLS * KY * 2 + 64; }

cudaError_t tc_prepare(int KY) {
    const size_t f = tc_fwd_smem(KY), b = tc_back_smem(KY);
    cudaError_t e = cudaErrorInvalidValue;
#define PREP_CASE(KYV)                                                        \
    case KYV:                                                                 \
        e = set_smem(k_tc_forward<KYV>, f);                                   \
        if (e == cudaSuccess) e = set_smem(k_tc_back<KYV, false>, b);         \
        if (e == cudaSuccess) e = set_smem(k_tc_back<KYV, true>, b);          \
        break;
    switch (KY) { PREP_CASE(16) PREP_CASE(32) PREP_CASE(48) PREP_CASE(64) PREP_CASE(96) PREP_CASE(128) }
#undef PREP_CASE
    if (e == cudaSuccess) e = set_smem(k_tc_panels_com, pcom_smem(KY));
    return e;
}

static Panels panels_of(const TcPlan &p) {
    Panels P;
    P.Npad = p.Npad;
    P.KY = p.KY;
    P.Ahi = p.Ahi; P.Alo = p.Alo; P.Yhi = p.Yhi; P.Ylo = p.Ylo; P.Af = p.Af; P.Bsrc = p.Bsrc;
    return P;
}

cudaError_t launch_tc_panels(const TcPlan &p, const double *R, cudaStream_t st) {
    k_tc_panels<<<(p.Npad + 127) / 128, 128, 0, st>>>(p.N, p.Kx, p.Ky2, p.dkx, p.dky, R, panels_of(p));
    return cudaGetLastError();
}

cudaError_t launch_tc_panels_com(const TcPlan &p, const double *r, const double *mass, const int *cell_offset,
                                 cudaStream_t st) {
    const double two_pi = 6.283185307179586;
    const int tiles = (p.N + FWD_CELLS - 1) / FWD_CELLS;
    k_tc_panels_com<<<tiles, PCOM_THREADS, pcom_smem(p.KY), st>>>(p.N, p.Kx, p.Ky2, p.dkx / two_pi, p.dky / two_pi, r,
                                                                   mass, cell_offset, panels_of(p));
    return cudaGetLastError();
}

cudaError_t launch_tc_forward(const TcPlan &p, const double *Mc, double *G, unsigned *status, cudaStream_t st) {
    const int nq = p.Npad / FWD_SC;
    const int per = (nq + p.n_fwd_cta - 1) / p.n_fwd_cta;
    const size_t sm = tc_fwd_smem(p.KY);
    cudaError_t e = cudaSuccess;
#define FWD_CASE(KYV)                                                                                     \
    case KYV:                                                                                             \
            k_tc_forward<KYV><<<p.n_fwd_cta, FWD_THREADS, sm, st>>>(nq, per, p.Ahi, p.Alo, p.Bsrc, Mc, p.N, \
                                                            p.partial, status);                           \
        break;
    switch (p.KY) {
        FWD_CASE(16) FWD_CASE(32) FWD_CASE(48) FWD_CASE(64) FWD_CASE(96) FWD_CASE(128)
        default: return cudaErrorInvalidValue;
    }
#undef FWD_CASE
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int size = KXP * p.KY;
    k_tc_reduce<<<(size + 255) / 256, 256, 0, st>>>(p.n_fwd_cta, size, p.partial, G);
    return cudaGetLastError();
}

cudaError_t launch_tc_back(const TcPlan &p, const float *Wt2, const float *Wt1, double *E2, double *E1,
                           unsigned *status, cudaStream_t st, double *G) {
    const size_t sm = tc_back_smem(p.KY);
    const int n_tiles = p.Npad / BACK_CELLS;
    const int grid = std::min(n_tiles, p.n_sm);
    const float fx = (float)p.dkx, fy = (float)p.dky;
#define BACK_CASE(KYV)                                                                                        \
    case KYV:                                                                                                 \
        if (G)                                                                                                \
            k_tc_back<KYV, true><<<grid, 128, sm, st>>>(p.N, p.Npad, n_tiles, Wt2, nullptr, p.Yhi, p.Ylo, p.Af, \
                                                        E2, nullptr, G, p.Kx, p.Ky2, fx, fy, status);        \
        else                                                                                                  \
            k_tc_back<KYV, false><<<grid, 128, sm, st>>>(p.N, p.Npad, n_tiles, Wt2, Wt1, p.Yhi, p.Ylo, p.Af,  \
                                                         E2, E1, nullptr, p.Kx, p.Ky2, fx, fy, status);      \
        break;
    switch (p.KY) {
        BACK_CASE(16) BACK_CASE(32) BACK_CASE(48) BACK_CASE(64) BACK_CASE(96) BACK_CASE(128)
        default: return cudaErrorInvalidValue;
    }
#undef BACK_CASE
    return cudaGetLastError();
}
