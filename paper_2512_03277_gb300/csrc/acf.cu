// On-device autocorrelation functions for the linear spectra.
//
// The paper's molecular spectrum is the w^2-weighted cosine transform of <mu_x(t) mu_x(0)> and its
// angle-resolved photonic spectrum that of <q_k(t) q_k(0)> (Results). Long runs of many modes
// would have to copy M coordinates to the host every step; instead every synchronised state is
// folded into running lag products on the device:
//   channel c < M: the photon coordinate q_c; channel M: the total projected dipole sum_n M_n;
//   acc[c][l] += x_c(t) x_c(t - l) for l = 0 .. min(t, L - 1), a ring of the last L samples,
//   the first L samples and the running sum S_c.
// From these the finalisation forms the mean-removed unbiased estimator exactly:
//   C(l) = [P(l) - xbar (A(l) + B(l)) + (n - l) xbar^2] / (n - l),  xbar = S / n,
//   P(l) = sum_{t=l}^{n-1} x_t x_{t-l},  A(l) = S - (last l samples),  B(l) = S - (first l samples).
// One block per channel; every sum runs in a fixed order, so the result is deterministic.
#include "cavmd_internal.cuh"

namespace {

constexpr int ACF_THREADS = 256;

__global__ void __launch_bounds__(ACF_THREADS) k_acf(const AcfArgs a, const double *__restrict__ q_sync,
                                                     const double *__restrict__ M_cell, int N) {
    __shared__ double red[ACF_THREADS / 32];
    __shared__ double xs;
    __shared__ bool last;
    const int c = blockIdx.x;
    const long long t = *a.n;   // every block reads it before the last block advances it
    if (c < a.M) {
        if (threadIdx.x == 0) xs = q_sync[c];
    } else {   // total dipole: fixed-order block reduction over the cells
        double s = 0.0;
        for (int n = threadIdx.x; n < N; n += ACF_THREADS) s += M_cell[n];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(CAVMD_FULL_MASK, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double v = 0.0;
            for (int w = 0; w < ACF_THREADS / 32; ++w) v += red[w];
            xs = v;
        }
    }
    const int L = a.L;
    const int s = (int)(t % L);
    double *ring = a.ring + (size_t)c * L;
    if (threadIdx.x == 0) {
        ring[s] = xs;
        if (t < L) a.head[(size_t)c * L + t] = xs;
        a.sum[c] += xs;
    }
    __syncthreads();
    const double x = xs;
    double *acc = a.acc + (size_t)c * L;
    const int lmax = (int)(t < L - 1 ? t : L - 1);
    for (int l = threadIdx.x; l <= lmax; l += ACF_THREADS) {
        const int i = s - l < 0 ? s - l + L : s - l;
        acc[l] = fma(x, ring[i], acc[l]);
    }
    if (threadIdx.x == 0) {
        const unsigned tk = atomicAdd(a.ticket, 1u);
        last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        *a.n = t + 1;
        *a.ticket = 0u;
    }
}

__global__ void k_acf_finalize(const AcfArgs a, double *__restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.C) return;
    const long long n = *a.n;
    const int L = a.L;
    const double S = a.sum[c];
    const double xb = n > 0 ? S / (double)n : 0.0;
    const double *ring = a.ring + (size_t)c * L, *head = a.head + (size_t)c * L, *acc = a.acc + (size_t)c * L;
    double first = 0.0, lastsum = 0.0;   // sums of the first l and of the last l samples
    for (int l = 0; l < L; ++l) {
        if (l >= n) {
            out[(size_t)c * L + l] = 0.0;
            continue;
        }
        const double A = S - lastsum, B = S - first, m = (double)(n - l);
        out[(size_t)c * L + l] = (acc[l] - xb * (A + B) + m * xb * xb) / m;
        first += head[l];
        long long i = (n - 1 - l) % L;
        lastsum += ring[i];
    }
}

}  // namespace

cudaError_t launch_acf(const AcfArgs &a, const double *q_sync, const double *M_cell, int N, cudaStream_t st) {
    k_acf<<<a.C, ACF_THREADS, 0, st>>>(a, q_sync, M_cell, N);
    return cudaGetLastError();
}

cudaError_t launch_acf_finalize(const AcfArgs &a, double *out, cudaStream_t st) {
    k_acf_finalize<<<(a.C + 127) / 128, 128, 0, st>>>(a, out);
    return cudaGetLastError();
}
