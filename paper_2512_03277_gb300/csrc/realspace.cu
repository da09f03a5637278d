// The paper's real-space / reciprocal-space propagation (CAVMD_SPLIT_REAL_SPACE): Eq. hlm3 with the
// velocity-Verlet Step 1 (Eq. pj1) and the transforms and rotation of Steps 2-4 (Eqs. qkink_ak, qknk,
// qkink_an).
//
// Every cell n carries one real-space photon coordinate q_n and momentum p_n. With sqrt(omega_k)
// taken as sqrt(omega_0) in the coupling, the light-matter terms are local,
//     eta q_n M_n + eta^2 / (2 omega_0^2) M_n^2,   eta = sqrt(2N) g0 omega_0,
// so Step 1 kicks p_n by -eta M_n and the nuclei by -(eta q_n + eta^2 M_n / omega_0^2) dM_n/dr_j with
// q_n held fixed. Steps 2-4 map the omega_0-normalised amplitudes alpha_n = x_n + i y_n,
// x_n = sqrt(omega_0 / 2) q_n, y_n = p_n / sqrt(2 omega_0), to the modes (a unitary transform when the
// cells sit on a lattice and the modes on its grid), turn every mode amplitude by exp(-i omega_k dt)
// with its own omega_k, and map back. In the library's real modes u_a (cos and sin members of each
// +-k pair, amplitude lambda_a) the transform pair is
//     X_a + i Y_a = sum_n u_a(R_n) alpha_n,   alpha_n <- sum_a w_a u_a(R_n) (X'_a + i Y'_a),
//     w_a = lambda_a^2 / (2 N g0^2)   (1/N for a single real mode, 2/N for each member of a pair),
// since sum_a w_a u_a(R_n) u_a(R_m) = (1/N) sum_k exp(ik(R_n - R_m)). The free photon energy is
// sum_a w_a omega_a (X_a^2 + Y_a^2), which for a flat dispersion is the local
// sum_n (p_n^2 + omega_0^2 q_n^2) / 2.
//
// Launches of one step: k_rs_second (the photon half-kick and the nuclear field of the second
// half-kick, per cell), k_rs_forward (Step 2 and the rotation of Step 3, one block per mode, fixed-order
// sums), k_rs_back (Step 4, the energies of the synchronised state and the field and photon kick of
// the next first half-kick, per cell); the nuclear kicks and the drift run in the kick kernel with
// these fields (FLD_E_GIVEN). Energies of a cell and of the mode with the same index share one
// row of e_mode, which needs as many modes as cells.
#include "cavmd_internal.cuh"

namespace {

constexpr int RS_THREADS = 256;

__device__ __forceinline__ double rs_field(const RsArgs &r, double q, double M) {
    return -fma(r.eta, q, r.eta2_w0sq * M);   // -(eta q_n + eta^2 M_n / omega_0^2)
}

// Synchronised photon state (init or set_state): q_n, p_n, then the amplitudes x_n, y_n.
__global__ void k_rs_init(RsArgs r, StepArgs a, int mode) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= a.N) return;
    double q, p;
    if (mode == 1) {          // Step 0 at frozen nuclei ends at the photon minimum
        q = -r.eta * a.M_cell[n] * r.inv_w0sq;
        p = 0.0;
    } else if (mode == 2) {   // photons at zero
        q = 0.0;
        p = 0.0;
    } else {                  // keep the synchronised state
        q = a.q_sync[n];
        p = a.pq_sync[n];
    }
    a.q_sync[n] = q;
    a.pq_sync[n] = p;
    r.x[n] = r.sq * q;
    r.y[n] = r.isq * p;
}

// Opening first half-kick of a call, from the synchronised state.
__global__ void k_rs_open(RsArgs r, StepArgs a) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= a.N) return;
    const double q = a.q_sync[n], M = a.M_cell[n];
    a.q[n] = q;
    a.pq[n] = fma(a.tau * r.eta, -M, a.pq_sync[n]);
    r.E1[n] = a.tau * rs_field(r, q, M);
}

// Second half-kick of Step 1 at the new positions, with q_n held: p_n += h (-eta M_n) and the
// nuclear field h (-(eta q_n + eta^2 M_n / omega_0^2)); then the amplitudes of Step 2.
__global__ void k_rs_second(RsArgs r, StepArgs a) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= a.N) return;
    const double q = a.q[n], M = a.M_cell[n];
    const double p = fma(a.tau * r.eta, -M, a.pq[n]);
    r.E2[n] = a.tau * rs_field(r, q, M);
    r.x[n] = r.sq * q;
    r.y[n] = r.isq * p;
}

// Step 2 and the rotation of Step 3 for mode a: X + iY = sum_n u_a(R_n) (x_n + i y_n), turned by
// exp(-i omega_a dt) when `rotate`; the free energy of the mode and the weighted amplitudes of Step 4.
__global__ void __launch_bounds__(RS_THREADS) k_rs_forward(RsArgs r, StepArgs a, int rotate) {
    __shared__ double red[2][RS_THREADS / 32];
    const int al = blockIdx.x;
    const double *u = a.U + (size_t)al * a.N;
    double X = 0.0, Y = 0.0;
    for (int n = threadIdx.x; n < a.N; n += RS_THREADS) {
        const double un = u[n];
        X = fma(un, r.x[n], X);
        Y = fma(un, r.y[n], Y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {   // fixed-order tree, then the warp sums in order
        X += __shfl_xor_sync(CAVMD_FULL_MASK, X, o);
        Y += __shfl_xor_sync(CAVMD_FULL_MASK, Y, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = X;
        red[1][threadIdx.x >> 5] = Y;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    X = 0.0;
    Y = 0.0;
    for (int w = 0; w < RS_THREADS / 32; ++w) {
        X += red[0][w];
        Y += red[1][w];
    }
    if (rotate) {
        const double c = r.cdt[al], s = r.sdt[al];
        const double Xn = fma(c, X, s * Y);
        Y = fma(c, Y, -s * X);
        X = Xn;
    }
    const double wa = r.w[al];
    r.Xw[al] = wa * X;
    r.Yw[al] = wa * Y;
    a.e_mode[4 * al + 3] = wa * a.omega[al] * fma(X, X, Y * Y);
}

// Step 4 for cell n (when `back`: alpha_n = sum_a w_a u_a(R_n) (X'_a + i Y'_a) becomes the
// synchronised state), the local energies of the synchronised state, and the next first half-kick
// (the photon kick when `first`, and its nuclear field, kept for the next call as well).
__global__ void k_rs_back(RsArgs r, StepArgs a, int back, int first) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= a.N) return;
    double q, p;
    if (back) {
        double x = 0.0, y = 0.0;
        for (int al = 0; al < a.M; ++al) {
            const double un = a.U[(size_t)al * a.N + n];
            x = fma(un, r.Xw[al], x);
            y = fma(un, r.Yw[al], y);
        }
        q = x * r.inv_sq;
        p = y * r.inv_isq;
        a.q_sync[n] = q;
        a.pq_sync[n] = p;
    } else {
        q = a.q_sync[n];
        p = a.pq_sync[n];
    }
    const double M = a.M_cell[n];
    double *e = a.e_mode + 4 * n;
    e[1] = r.eta * q * M;
    e[2] = 0.5 * r.eta2_w0sq * M * M;
    e[0] = e[1] + e[2] + e[3];
    r.E1[n] = a.tau * rs_field(r, q, M);
    a.q[n] = q;
    a.pq[n] = first ? fma(a.tau * r.eta, -M, p) : p;
}

}  // namespace

cudaError_t launch_rs(const RsArgs &r, const StepArgs &a, int what, int flags, cudaStream_t st) {
    const int gb = (a.N + 127) / 128;
    switch (what) {
        case RS_INIT: k_rs_init<<<gb, 128, 0, st>>>(r, a, flags); break;
        case RS_OPEN: k_rs_open<<<gb, 128, 0, st>>>(r, a); break;
        case RS_SECOND: k_rs_second<<<gb, 128, 0, st>>>(r, a); break;
        case RS_FORWARD: k_rs_forward<<<a.M, RS_THREADS, 0, st>>>(r, a, flags); break;
        case RS_BACK: k_rs_back<<<gb, 128, 0, st>>>(r, a, flags & 1, (flags >> 1) & 1); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
