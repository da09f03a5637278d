// On-device autocorrelation functions for the linear spectra.
//
// The paper's molecular spectrum is the w^2-weighted cosine transform of <mu_x(t) mu_x(0)> and its
// angle-resolved photonic spectrum that of <q_k(t) q_k(0)> (Results). Long runs of many modes
// would have to copy M coordinates to the host every step; instead every synchronised state is
// folded into running lag products on the device:
//   channel c < M: the photon coordinate q_c; channel M: the total projected dipole sum_n M_n;
//   a ring of the last L + B samples, the first L samples and the running sum S_c; every B steps
//   the B newest samples are folded into the lag products, acc[c][l] += sum over those samples t
//   of x_c(t) x_c(t - l) (t in increasing order), so the L lag products are read and written once
//   per B steps instead of every step (at 8193 channels x 1024 lags that table is 67 MB). The
//   samples not yet folded are added at read-out from the ring.
// From these the finalisation forms the mean-removed unbiased estimator exactly:
//   C(l) = [P(l) - xbar (A(l) + B(l)) + (n - l) xbar^2] / (n - l),  xbar = S / n,
//   P(l) = sum_{t=l}^{n-1} x_t x_{t-l},  A(l) = S - (last l samples),  B(l) = S - (first l samples).
// One warp per photon channel; the total dipole is summed over slices of the cells by all blocks and
// finished by the last one. Every sum runs in a fixed order, so the result is deterministic.
#include "cavmd_internal.cuh"

namespace {

constexpr int ACF_THREADS = 256;

constexpr int ACF_WARPS = ACF_THREADS / 32;   // channels per block: one warp each

// Block reduction in a fixed order (threads strided, then a shuffle tree, then the warps in order).
__device__ double block_sum(double s, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(CAVMD_FULL_MASK, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double v = 0.0;
    for (int w = 0; w < ACF_WARPS; ++w) v += red[w];
    __syncthreads();
    return v;
}

// One sample of channel c, by one warp: store it in the ring (and the head while t < L), add it to
// the running sum, and fold the B newest samples into the lag products when the block of B is
// complete (lanes over the lags).
__device__ void acf_push(const AcfArgs &a, int c, long long t, double xs) {
    const int L = a.L, R = a.L + a.B, lane = threadIdx.x & 31;
    double *ring = a.ring + (size_t)c * R;
    if (lane == 0) {
        ring[t % R] = xs;
        if (t < L) a.head[(size_t)c * L + t] = xs;
        a.sum[c] += xs;
    }
    __syncwarp();
    if ((t + 1) % a.B == 0) {   // fold samples t - B + 1 .. t
        double *acc = a.acc + (size_t)c * L;
        for (int l = lane; l < L; l += 32) {
            double v = acc[l];
            for (long long u = t - a.B + 1; u <= t; ++u)
                if (u >= l) v = fma(ring[u % R], ring[(u - l) % R], v);
            acc[l] = v;
        }
    }
}

// Grid: G blocks, G >= M / ACF_WARPS. Warp w of block b pushes the photon coordinate of channel
// b ACF_WARPS + w (< M); every block also sums its slice of the per-cell dipoles into part[b]; the
// last block to finish (ticket) sums the G partial sums in block order into the total dipole,
// pushes it as channel M with its first warp and advances the sample counter.
__global__ void __launch_bounds__(ACF_THREADS) k_acf(const AcfArgs a, const double *__restrict__ q_sync,
                                                     const double *__restrict__ M_cell, int N) {
    __shared__ double red[ACF_WARPS];
    __shared__ bool last;
    const int b = blockIdx.x;
    const long long t = *a.n;   // every block reads it before the last block advances it
    const int slice = (N + a.G - 1) / a.G;
    const int n0 = min(N, b * slice), n1 = min(N, n0 + slice);
    double s = 0.0;
    for (int n = n0 + threadIdx.x; n < n1; n += ACF_THREADS) s += M_cell[n];
    s = block_sum(s, red);
    if (threadIdx.x == 0) a.part[b] = s;
    const int c = b * ACF_WARPS + (threadIdx.x >> 5);
    if (c < a.M) acf_push(a, c, t, q_sync[c]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned tk = atomicAdd(a.ticket, 1u);
        last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = 0.0;
    for (int i = threadIdx.x; i < a.G; i += ACF_THREADS) v += __ldcg(a.part + i);
    v = block_sum(v, red);
    if (threadIdx.x < 32) acf_push(a, a.M, t, v);
    if (threadIdx.x == 0) {
        *a.n = t + 1;
        *a.ticket = 0u;
    }
}

__global__ void k_acf_finalize(const AcfArgs a, double *__restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.C) return;
    const long long n = *a.n;
    const int L = a.L, R = a.L + a.B;
    const double S = a.sum[c];
    const double xb = n > 0 ? S / (double)n : 0.0;
    const double *ring = a.ring + (size_t)c * R, *head = a.head + (size_t)c * L, *acc = a.acc + (size_t)c * L;
    const long long folded = n - n % a.B;   // samples already in the lag products
    double first = 0.0, lastsum = 0.0;   // sums of the first l and of the last l samples
    for (int l = 0; l < L; ++l) {
        if (l >= n) {
            out[(size_t)c * L + l] = 0.0;
            continue;
        }
        double P = acc[l];
        for (long long u = folded; u < n; ++u)
            if (u >= l) P = fma(ring[u % R], ring[(u - l) % R], P);
        const double A = S - lastsum, B = S - first, m = (double)(n - l);
        out[(size_t)c * L + l] = (P - xb * (A + B) + m * xb * xb) / m;
        first += head[l];
        lastsum += ring[(n - 1 - l) % R];
    }
}

}  // namespace

cudaError_t launch_acf(const AcfArgs &a, const double *q_sync, const double *M_cell, int N, cudaStream_t st) {
    k_acf<<<a.G, ACF_THREADS, 0, st>>>(a, q_sync, M_cell, N);
    return cudaGetLastError();
}

cudaError_t launch_acf_finalize(const AcfArgs &a, double *out, cudaStream_t st) {
    k_acf_finalize<<<(a.C + 127) / 128, 128, 0, st>>>(a, out);
    return cudaGetLastError();
}
