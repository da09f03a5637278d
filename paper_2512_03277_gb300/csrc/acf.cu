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
    const int L = a.L, R = a.L + a.B;
    double *ring = a.ring + (size_t)c * R;
    if (threadIdx.x == 0) {
        ring[t % R] = xs;
        if (t < L) a.head[(size_t)c * L + t] = xs;
        a.sum[c] += xs;
    }
    __syncthreads();
    if ((t + 1) % a.B == 0) {   // fold samples t - B + 1 .. t
        double *acc = a.acc + (size_t)c * L;
        for (int l = threadIdx.x; l < L; l += ACF_THREADS) {
            double v = acc[l];
            for (long long u = t - a.B + 1; u <= t; ++u)
                if (u >= l) v = fma(ring[u % R], ring[(u - l) % R], v);
            acc[l] = v;
        }
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
    k_acf<<<a.C, ACF_THREADS, 0, st>>>(a, q_sync, M_cell, N);
    return cudaGetLastError();
}

cudaError_t launch_acf_finalize(const AcfArgs &a, double *out, cudaStream_t st) {
    k_acf_finalize<<<(a.C + 127) / 128, 128, 0, st>>>(a, out);
    return cudaGetLastError();
}
