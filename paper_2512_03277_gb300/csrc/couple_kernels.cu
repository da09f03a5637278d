// Light-matter coupling and time-step kernels (FP64).
//
// With real modes u_a(R) = cos(k_a . R + phi_a) the k-space form of the paper's Hamiltonian
// (Eq. hlm2) has photon energy sum_a 1/2 p_a^2 + 1/2 (omega_a q_a - D_a)^2 with
// D_a = lambda_a sum_n u_a(R_n) M_n, the gather of the paper's Step 2 done as a reduction over
// cells. The step is H_2(dt/2) - drift(dt) - H_2(dt/2), where H_2 = V + H_ph is solved exactly at
// frozen nuclei: each mode turns about its displaced centre D_a / omega_a by omega_a tau (the
// rotation of Eq. qknk) and every nucleus j of cell n receives the time-integrated force
//     dp_j = tau F_j + E_n b_j,  E_n = sum_a u_a(R_n) W_a,
//     W_a = lambda_a [y_a sin(omega_a tau) + p_a (1 - cos(omega_a tau)) / omega_a],  y_a = q_a - D_a/omega_a,
// the k-space form of the nuclear coupling force of Eq. dpj integrated over the half step (the
// scatter of the paper's Step 4).
//
// k_photon: one block per mode; the deterministic block reduction forms D_a from the cell
//           dipoles, then one thread applies the half-flows of that mode and records its energy.
// k_field:  each block owns 16 cells and splits their mode sums over 16 slices; a fixed-order
//           reduction combines the slices, then the cells' atoms are kicked (and drifted) by the
//           slices in parallel. The last
//           block to finish sums the per-block energy partials in block order (deterministic)
//           and appends the energies of the synchronised state to the history ring.
// k_kick:   the same kicks, drift and energy record when the tensor-core back product has
//           already formed the fields: one thread per Cartesian component of an atom (one thread
//           per cell with moving mode positions).
#include <algorithm>

#include "cavmd_internal.cuh"

namespace {

constexpr int PH_THREADS = 256;
constexpr int PHM_THREADS = 128;   // modes per block of the one-thread-per-mode photon kernel
constexpr int FLD_CELLS = 16;    // cells per block (N / 16 blocks fill every SM for N >= 2432)
constexpr int FLD_SLICES = 16;   // mode slices: thread (cell, slice) sums every 16th mode of its cell
constexpr int KICK_THREADS = 64;    // cells per block of the kick-only kernel (moving mode positions)
constexpr int KA_THREADS = 256;     // atom components per block of the component-parallel kick
constexpr int KA_MAX_BLOCKS = 1024; // its grid-stride launch: about one resident wave on 152 SMs

__global__ void k_mode_functions(const double *__restrict__ k, const double *__restrict__ phi,
                                 const double *__restrict__ R, int M, int N, double *__restrict__ U) {
    const long long total = (long long)M * N;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(t / N), n = (int)(t - (long long)a * N);
        const double arg = k[3 * a] * R[3 * n] + k[3 * a + 1] * R[3 * n + 1] + k[3 * a + 2] * R[3 * n + 2] + phi[a];
        U[t] = cos(arg);
    }
}

__device__ __forceinline__ double block_sum_ordered(double v, double *red) {
    // fixed-order tree: warp shuffles (xor pattern is the same on every launch), then warp sums
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(CAVMD_FULL_MASK, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;   // valid in thread 0
}

// Weight W of mode (jx, jy, s) into the back-product matrix Wt (rows cos|sin of jx, columns
// cos|sin of jy): cos modes at (jx, jy) and -(Kx + jx, Ky2 + jy), sin modes at (jx, Ky2 + jy) and
// (Kx + jx, jy).
__device__ __forceinline__ void put_weight(const StepArgs &a, float *Wt, int al, double W) {
    const int jx = al / (2 * a.Ky2), rem = al - jx * 2 * a.Ky2, jy = rem >> 1, sm = rem & 1;
    if (sm == 0) {
        Wt[jx * a.KY + jy] = (float)W;
        Wt[(a.Kx + jx) * a.KY + a.Ky2 + jy] = (float)(-W);
    } else {
        Wt[jx * a.KY + a.Ky2 + jy] = (float)W;
        Wt[(a.Kx + jx) * a.KY + jy] = (float)W;
    }
}

// Exact half-flow of one mode at frozen nuclei: rotation about the centre cen = D / omega by
// omega tau (c = cos, s = sin), and the field weight lam [y sin + p (1 - cos) / omega] of the
// same half-flow. Every rounding is explicit (no multiply-add contraction left to the compiler),
// so the rotation applied at the end of a step and the one applied at the opening of the next
// call give the same bits.
__device__ __forceinline__ void mode_half_flow(double q, double p, double cen, double c, double s, double w,
                                               double iw, double &qo, double &po) {
    const double y = __dsub_rn(q, cen);
    qo = __dadd_rn(cen, fma(y, c, __dmul_rn(__dmul_rn(p, s), iw)));
    po = fma(p, c, __dmul_rn(__dmul_rn(-w, y), s));
}
__device__ __forceinline__ double mode_weight(double q, double p, double cen, double s, double omc, double lam) {
    return __dmul_rn(lam, fma(__dsub_rn(q, cen), s, __dmul_rn(p, omc)));
}

// The paper's step order (CAVMD_SPLIT_PAPER; Eq. pj1, then the rotation of Eq. qknk, Step 3): the
// nuclei and photon momenta take half-kicks with the instantaneous force, p_a += h omega_a D_a and
// field weights W_a = h lambda_a (omega_a q_a - D_a), h = dt/2; after the second half-kick each
// mode turns freely by omega_a dt. The synchronised state is the rotated one. The same weights
// feed the field, tensor-core and position-term kernels as the exact half-flows' do.
// CAVMD_SPLIT_STRANG (a.strang) takes the same kicks but turns the modes between them, together
// with the nuclear drift: kick(h), free flow of the nuclei and the modes over dt, kick(h), so the
// second kick sees the turned coordinates and the synchronised state is the kicked one.
__device__ __forceinline__ double paper_weight(double q, double D, double w, double lam, double h) {
    return __dmul_rn(h * lam, fma(w, q, -D));
}
__device__ __forceinline__ void put_weights(const StepArgs &a, int al, double W, double *Wv, float *Wt, double *Wk) {
    Wv[al] = W;
    if (Wt) put_weight(a, Wt, al, W);
    if (Wk)
        for (int k = 0; k < 3; ++k) Wk[3 * al + k] = -W * a.kvec[3 * al + k];
}
__device__ __forceinline__ void photon_paper_order(const StepArgs &a, int flags, int al, double D, double D_sync,
                                                   double w, double iw, double lam, double c, double s, double cen) {
    const double h = a.tau, hw = h * w;
    const double cdt = fma(c, c, -s * s), sdt = 2.0 * s * c;   // cos, sin of omega dt
    auto turn = [&](double &q, double &p) {                    // free rotation by omega dt
        const double qn = fma(q, cdt, p * sdt * iw);
        p = fma(p, cdt, -w * q * sdt);
        q = qn;
    };
    double qs, ps;
    if (flags & PH_INIT_RELAXED) {
        qs = cen;
        ps = 0.0;
    } else if (flags & PH_INIT_ZERO) {
        qs = 0.0;
        ps = 0.0;
    } else if (flags & PH_SECOND) {
        double q, p;
        if (flags & PH_OPEN) {   // the opening first half-kick, from the synchronised state
            q = a.q_sync[al];
            p = fma(hw, D_sync, a.pq_sync[al]);
            if (a.strang) turn(q, p);
        } else {
            q = a.q[al];
            p = a.pq[al];
        }
        put_weights(a, al, paper_weight(q, D, w, lam, h), a.W2, a.Wt2, a.Wk2);
        p = fma(hw, D, p);
        if (!a.strang) turn(q, p);
        qs = q;
        ps = p;
    } else {
        qs = a.q_sync[al];
        ps = a.pq_sync[al];
    }
    a.q_sync[al] = qs;
    a.pq_sync[al] = ps;
    if (flags & PH_ENERGY) {
        const double x = fma(w, qs, -D);
        double *e = a.e_mode + 4 * al;
        e[0] = 0.5 * fma(ps, ps, x * x);
        e[1] = -w * qs * D;
        e[2] = 0.5 * D * D;
        e[3] = 0.5 * fma(ps, ps, (w * qs) * (w * qs));
    }
    if (flags & (PH_FIRST | PH_W1)) put_weights(a, al, paper_weight(qs, D, w, lam, h), a.W1, a.Wt1, a.Wk1);
    double q1 = qs, p1 = ps;
    if (flags & PH_FIRST) {
        p1 = fma(hw, D, ps);
        if (a.strang) turn(q1, p1);
    }
    a.q[al] = q1;
    a.pq[al] = p1;
}

// Everything of k_photon after the mode's field D is known, for mode al (one thread).
__device__ __forceinline__ void photon_mode(const StepArgs &a, const int flags, const int al, const double D,
                                            const double D_sync) {
    const double w = a.omega[al], iw = a.inv_omega[al], lam = a.lam[al];
    const double c = a.cos_h[al], s = a.sin_h[al], omc = a.omc_h[al];
    const double cen = __dmul_rn(D, iw);
    if (a.paper) {
        photon_paper_order(a, flags, al, D, D_sync, w, iw, lam, c, s, cen);
        return;
    }
    double qs, ps;
    if (flags & PH_INIT_RELAXED) {
        qs = cen;
        ps = 0.0;
    } else if (flags & PH_INIT_ZERO) {
        qs = 0.0;
        ps = 0.0;
    } else if (flags & PH_SECOND) {
        double q, p;
        if (flags & PH_OPEN)   // the opening first half-flow (as a PH_FIRST launch of its own)
            mode_half_flow(a.q_sync[al], a.pq_sync[al], __dmul_rn(D_sync, iw), c, s, w, iw, q, p);
        else {
            q = a.q[al];
            p = a.pq[al];
        }
        a.W2[al] = mode_weight(q, p, cen, s, omc, lam);
        if (a.Wt2) put_weight(a, a.Wt2, al, a.W2[al]);
        if (a.Wk2)
            for (int k = 0; k < 3; ++k) a.Wk2[3 * al + k] = -a.W2[al] * a.kvec[3 * al + k];
        mode_half_flow(q, p, cen, c, s, w, iw, qs, ps);
    } else {
        qs = a.q_sync[al];
        ps = a.pq_sync[al];
    }
    a.q_sync[al] = qs;
    a.pq_sync[al] = ps;
    if (flags & PH_ENERGY) {
        const double x = fma(w, qs, -D);
        double *e = a.e_mode + 4 * al;
        e[0] = 0.5 * fma(ps, ps, x * x);
        e[1] = -w * qs * D;
        e[2] = 0.5 * D * D;
        e[3] = 0.5 * fma(ps, ps, (w * qs) * (w * qs));
    }
    if (flags & (PH_FIRST | PH_W1)) {
        a.W1[al] = mode_weight(qs, ps, cen, s, omc, lam);
        if (a.Wt1) put_weight(a, a.Wt1, al, a.W1[al]);
        if (a.Wk1)
            for (int k = 0; k < 3; ++k) a.Wk1[3 * al + k] = -a.W1[al] * a.kvec[3 * al + k];
    }
    if (flags & PH_FIRST) {
        double q1, p1;
        mode_half_flow(qs, ps, cen, c, s, w, iw, q1, p1);
        a.q[al] = q1;
        a.pq[al] = p1;
    } else {
        a.q[al] = qs;
        a.pq[al] = ps;
    }
}


__global__ void __launch_bounds__(PH_THREADS) k_photon(const StepArgs a, const int flags) {
    __shared__ double red[PH_THREADS / 32];
    const int al = blockIdx.x;
    double D = 0.0;
    // PH_OPEN: the field of the synchronised state, read before the forward replaces it
    const double D_sync = ((flags & PH_OPEN) && threadIdx.x == 0) ? a.D[al] : 0.0;
    const double *u = a.U + (size_t)al * a.N;
    double s = 0.0;
#pragma unroll 4
    for (int n = threadIdx.x; n < a.N; n += PH_THREADS) s = fma(u[n], a.M_cell[n], s);
    s = block_sum_ordered(s, red);
    if (threadIdx.x != 0) return;
    D = a.lam[al] * s;
    a.D[al] = D;
    photon_mode(a, flags, al, D, D_sync);
}

// k_photon without the FP64 forward contraction (D from the factorised Gram matrix, or the stored
// D): one thread per mode.
__global__ void __launch_bounds__(PHM_THREADS) k_photon_modes(const StepArgs a, const int flags) {
    const int al = blockIdx.x * PHM_THREADS + threadIdx.x;
    if (al >= a.M) return;
    const double D_sync = (flags & PH_OPEN) ? a.D[al] : 0.0;   // read before the field is replaced
    double D;
    if (flags & PH_FORWARD_G) {   // mode (jx, jy, s) from the factorised Gram matrix
        const int jx = al / (2 * a.Ky2), rem = al - jx * 2 * a.Ky2, jy = rem >> 1, sm = rem & 1;
        const double *g = a.G;
        const double v = sm == 0 ? g[jx * a.KY + jy] - g[(a.Kx + jx) * a.KY + a.Ky2 + jy]
                                 : g[(a.Kx + jx) * a.KY + jy] + g[jx * a.KY + a.Ky2 + jy];
        D = a.lam[al] * v;
        a.D[al] = D;
    } else {
        D = a.D[al];
    }
    photon_mode(a, flags, al, D, D_sync);
}

// Partial field sums over the modes a = sl, sl + FLD_SLICES, ... for cell n; the loads of u are
// independent of the accumulation, so the unrolled loop keeps several of them in flight.
template <bool TWO, bool ONE>
__device__ __forceinline__ void field_partial(const StepArgs &a, int n, int sl, double &e2, double &e1) {
    const double *u = a.U + n;
#pragma unroll 8
    for (int al = sl; al < a.M; al += FLD_SLICES) {
        const double v = u[(size_t)al * a.N];
        if (TWO) e2 = fma(v, __ldg(a.W2 + al), e2);
        if (ONE) e1 = fma(v, __ldg(a.W1 + al), e1);
    }
}

// Second half-flow kick (field e2), kinetic energy of the synchronised state, then the next first
// half-flow kick (field e1) and the drift, for the atoms of cell n.
// Atom j of a cell with fields e2, e1: kinetic energy returned. Every load of the atom is issued
// before its stores (the arrays do not alias), so an atom costs one memory round trip.
__device__ __forceinline__ double kick_atom(const StepArgs &a, int flags, int j, double e2, double e1) {
    const double *__restrict__ F = a.F;
    const double *__restrict__ b = a.b;
    double *__restrict__ p = a.p;
    double *__restrict__ r = a.r;
    const double im = a.inv_mass[j];
    double pj[3], f[3], bb[3], rj[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        pj[k] = p[3 * j + k];
        f[k] = F[3 * j + k];
        bb[k] = b[3 * j + k];
        rj[k] = (flags & FLD_FIRST) ? r[3 * j + k] : 0.0;
    }
    double kin = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (flags & FLD_SECOND) pj[k] = fma(a.tau, f[k], fma(e2, bb[k], pj[k]));
        kin = fma(0.5 * im * pj[k], pj[k], kin);
        if (flags & FLD_FIRST) {
            pj[k] = fma(a.tau, f[k], fma(e1, bb[k], pj[k]));
            r[3 * j + k] = fma(a.dt * im, pj[k], rj[k]);
        }
        p[3 * j + k] = pj[k];
    }
    return kin;
}

// kick_atom with the position term of moving mode positions: wm = (m_j / m_n) M_n times G_n of
// each half-flow (g2, g1: 3 components; g2 unused without FLD_SECOND, g1 without FLD_FIRST).
__device__ __forceinline__ double kick_atom_moving(const StepArgs &a, int flags, int j, double e2, double e1,
                                                   const double *g2, const double *g1, double wm) {
    const double *__restrict__ F = a.F;
    const double *__restrict__ b = a.b;
    double *__restrict__ p = a.p;
    double *__restrict__ r = a.r;
    const double im = a.inv_mass[j];
    double pj[3], f[3], bb[3], rj[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        pj[k] = p[3 * j + k];
        f[k] = F[3 * j + k];
        bb[k] = b[3 * j + k];
        rj[k] = (flags & FLD_FIRST) ? r[3 * j + k] : 0.0;
    }
    double kin = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (flags & FLD_SECOND) pj[k] = fma(wm, g2[k], fma(a.tau, f[k], fma(e2, bb[k], pj[k])));
        kin = fma(0.5 * im * pj[k], pj[k], kin);
        if (flags & FLD_FIRST) {
            pj[k] = fma(wm, g1[k], fma(a.tau, f[k], fma(e1, bb[k], pj[k])));
            r[3 * j + k] = fma(a.dt * im, pj[k], rj[k]);
        }
        p[3 * j + k] = pj[k];
    }
    return kin;
}

// All atoms of cell n (one thread).
__device__ __forceinline__ void kick_cell(const StepArgs &a, int flags, int n, double e2, double e1, double &kin) {
    const int j0 = a.cell_offset[n], j1 = a.cell_offset[n + 1];
    for (int j = j0; j < j1; ++j) kin += kick_atom(a, flags, j, e2, e1);
}

// Run by the last block of a launch that left per-block kinetic and DFTB energy partials: totals in
// a fixed order (block partials, then the per-mode photon energies) and the energy record of the
// synchronised state. NT threads; scr holds 6 x NT/32 doubles.
template <int NT>
__device__ void record_energies(const StepArgs &a, int flags, int nblocks, double *scr) {
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nblocks; i += NT) {
        v[0] += __ldcg(a.e_kin_part + i);
        v[1] += __ldcg(a.e_dftb_part + i);
    }
    for (int al = threadIdx.x; al < a.M; al += NT) {
        const double *e = a.e_mode + 4 * al;
        v[2] += e[0];
        v[3] += e[1];
        v[4] += e[2];
        v[5] += e[3];
    }
    const int w = threadIdx.x >> 5;
    __syncthreads();   // scr may alias buffers the block read before
#pragma unroll
    for (int k = 0; k < 6; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(CAVMD_FULL_MASK, v[k], o);
        if ((threadIdx.x & 31) == 0) scr[k * (NT / 32) + w] = v[k];
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double t[6];
    for (int k = 0; k < 6; ++k) {
        t[k] = 0.0;
        for (int i = 0; i < NT / 32; ++i) t[k] += scr[k * (NT / 32) + i];
    }
    long long step = *a.step_counter;
    if (flags & FLD_SECOND) {
        step += 1;
        *a.step_counter = step;
    }
    double *h = a.hist + 8 * (size_t)(step % a.hist_cap);
    h[0] = t[0];
    h[1] = t[1];
    h[2] = t[2];
    h[3] = t[3];
    h[4] = t[4];
    h[5] = t[5];
    h[6] = t[0] + t[1] + t[2];
    h[7] = (double)step;
    if (!(isfinite(t[0]) && isfinite(t[1]) && isfinite(t[2]))) atomicOr(a.status, (unsigned)ERRBIT_NONFINITE);
    *a.done_counter = 0u;
}

__global__ void __launch_bounds__(FLD_CELLS *FLD_SLICES) k_field(const StepArgs a, const int flags) {
    __shared__ double red2[FLD_SLICES][FLD_CELLS];
    __shared__ double red1[FLD_SLICES][FLD_CELLS];
    __shared__ double es2[FLD_CELLS], es1[FLD_CELLS];
    __shared__ bool last;
    const int cl = threadIdx.x & (FLD_CELLS - 1);
    const int sl = threadIdx.x / FLD_CELLS;
    const int n = blockIdx.x * FLD_CELLS + cl;
    double e2 = 0.0, e1 = 0.0;
    if (n < a.N) {
        const bool two = flags & FLD_SECOND, one = flags & (FLD_FIRST | FLD_E1_STORE);
        if (two && one) field_partial<true, true>(a, n, sl, e2, e1);
        else if (two) field_partial<true, false>(a, n, sl, e2, e1);
        else if (one) field_partial<false, true>(a, n, sl, e2, e1);
    }
    red2[sl][cl] = e2;
    red1[sl][cl] = e1;
    __syncthreads();
    if (sl == 0) {   // fixed-order slice sums of cell cl
        for (int s = 1; s < FLD_SLICES; ++s) {
            e2 += red2[s][cl];
            e1 += red1[s][cl];
        }
        es2[cl] = e2;
        es1[cl] = e1;
        if ((flags & FLD_E1_STORE) && n < a.N) a.E1store[n] = e1;
    }
    __syncthreads();
    // the atoms of cell cl are spread over the 32 slices
    double kin = 0.0, edf = 0.0;
    if (n < a.N) {
        const int j1 = a.cell_offset[n + 1];
        for (int j = a.cell_offset[n] + sl; j < j1; j += FLD_SLICES) kin += kick_atom(a, flags, j, es2[cl], es1[cl]);
        if (sl == 0) edf = a.E_cell[n];
    }
    if (!(flags & FLD_ENERGY)) return;
    // per-block partials: fixed shuffle tree in every warp, then the 32 warp sums in order; the
    // last block to arrive forms the totals with the whole block in a fixed order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kin += __shfl_xor_sync(CAVMD_FULL_MASK, kin, o);
        edf += __shfl_xor_sync(CAVMD_FULL_MASK, edf, o);
    }
    constexpr int NW = FLD_CELLS * FLD_SLICES / 32;
    if ((threadIdx.x & 31) == 0) {
        red2[0][threadIdx.x >> 5] = kin;   // red2 / red1 are free after the slice sums
        red1[0][threadIdx.x >> 5] = edf;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double k = 0.0, d = 0.0;
        for (int w = 0; w < NW; ++w) {
            k += red2[0][w];
            d += red1[0][w];
        }
        a.e_kin_part[blockIdx.x] = k;
        a.e_dftb_part[blockIdx.x] = d;
        __threadfence();
        const unsigned ticket = atomicAdd(a.done_counter, 1u);
        last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    record_energies<FLD_CELLS * FLD_SLICES>(a, flags, gridDim.x, &red2[0][0]);
}

// Kicks and drift with the field on every cell given (the tensor-core back product wrote E2 / E1):
// one thread per cell, per-block energy partials, the last block records the energies.
__global__ void __launch_bounds__(KICK_THREADS) k_kick(const StepArgs a, const int flags) {
    __shared__ double scr[6 * (KICK_THREADS / 32)];
    __shared__ bool last;
    const int n = blockIdx.x * KICK_THREADS + threadIdx.x;
    double kin = 0.0, edf = 0.0;
    if (n < a.N) {
        const double e2 = (flags & FLD_SECOND) ? a.E2in[n] : 0.0;
        const double e1 = (flags & FLD_FIRST) ? a.E1in[n] : 0.0;
        if (a.G1in) {   // moving mode positions (G2 given by the tensor-core back product only)
            double g2[3] = {0.0, 0.0, 0.0}, g1[3] = {0.0, 0.0, 0.0};
            for (int k = 0; k < 3; ++k) {
                if ((flags & FLD_SECOND) && a.G2in) g2[k] = a.G2in[3 * n + k];
                if (flags & FLD_FIRST) g1[k] = a.G1in[3 * n + k];
            }
            const double Mn = a.M_cell[n];
            for (int j = a.cell_offset[n]; j < a.cell_offset[n + 1]; ++j)
                kin += kick_atom_moving(a, flags, j, e2, e1, g2, g1, a.w_atom[j] * Mn);
        } else {
            kick_cell(a, flags, n, e2, e1, kin);
        }
        edf = a.E_cell[n];
    }
    if (!(flags & FLD_ENERGY)) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kin += __shfl_xor_sync(CAVMD_FULL_MASK, kin, o);
        edf += __shfl_xor_sync(CAVMD_FULL_MASK, edf, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        scr[w] = kin;
        scr[KICK_THREADS / 32 + w] = edf;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double k = 0.0, d = 0.0;
        for (int i = 0; i < KICK_THREADS / 32; ++i) {
            k += scr[i];
            d += scr[KICK_THREADS / 32 + i];
        }
        a.e_kin_part[blockIdx.x] = k;
        a.e_dftb_part[blockIdx.x] = d;
        __threadfence();
        const unsigned ticket = atomicAdd(a.done_counter, 1u);
        last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    record_energies<KICK_THREADS>(a, flags, gridDim.x, scr);
}

// The kicks and the drift of k_kick with fixed mode positions, one thread per Cartesian component
// of an atom (grid-stride over the 3 n_atoms components, so the loads and stores of p, F, b and r
// are coalesced); the field of the atom's cell comes through the atom-to-cell index. Each thread
// also adds the DFTB energies of the cells i, i + stride, ...; the block partials and their totals
// are summed in a fixed order, so the energy record is deterministic. p and r are those of
// kick_atom bit for bit.
__global__ void __launch_bounds__(KA_THREADS) k_kick_atoms(const StepArgs a, const int flags) {
    __shared__ double scr[6 * (KA_THREADS / 32)];
    __shared__ bool last;
    const int stride = gridDim.x * KA_THREADS;
    const int n3 = 3 * a.n_atoms;
    // distinct arrays: the loads of later iterations may be issued ahead of this one's stores
    const double *__restrict__ F = a.F;
    const double *__restrict__ b = a.b;
    const double *__restrict__ im_ = a.inv_mass;
    const double *__restrict__ E2 = a.E2in;
    const double *__restrict__ E1 = a.E1in;
    const int *__restrict__ acell = a.atom_cell;
    double *__restrict__ p = a.p;
    double *__restrict__ r = a.r;
    double kin = 0.0, edf = 0.0;
#pragma unroll 4
    for (int i = blockIdx.x * KA_THREADS + threadIdx.x; i < n3; i += stride) {
        const int j = i / 3;
        const int n = acell[j];
        const double im = im_[j];
        const double f = F[i], bb = b[i];
        double pj = p[i];
        if (flags & FLD_SECOND) pj = fma(a.tau, f, fma(E2[n], bb, pj));
        kin = fma(0.5 * im * pj, pj, kin);
        if (flags & FLD_FIRST) {
            pj = fma(a.tau, f, fma(E1[n], bb, pj));
            r[i] = fma(a.dt * im, pj, r[i]);
        }
        p[i] = pj;
    }
    if (!(flags & FLD_ENERGY)) return;
    for (int n = blockIdx.x * KA_THREADS + threadIdx.x; n < a.N; n += stride) edf += a.E_cell[n];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kin += __shfl_xor_sync(CAVMD_FULL_MASK, kin, o);
        edf += __shfl_xor_sync(CAVMD_FULL_MASK, edf, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        scr[w] = kin;
        scr[KA_THREADS / 32 + w] = edf;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double k = 0.0, d = 0.0;
        for (int i = 0; i < KA_THREADS / 32; ++i) {
            k += scr[i];
            d += scr[KA_THREADS / 32 + i];
        }
        a.e_kin_part[blockIdx.x] = k;
        a.e_dftb_part[blockIdx.x] = d;
        __threadfence();
        const unsigned ticket = atomicAdd(a.done_counter, 1u);
        last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    record_energies<KA_THREADS>(a, flags, gridDim.x, scr);
}

// k_field for moving mode positions: besides E_n of both half-flows, the position-term vectors
// G_n = sum_a Us[a][n] Wk_a (Wk_a = -W_a k_a, written by k_photon), summed over the same 16 mode
// slices and combined in the same fixed order; the kicks add (m_j / m_n) M_n G_n.
__global__ void __launch_bounds__(FLD_CELLS *FLD_SLICES) k_field_moving(const StepArgs a, const int flags) {
    __shared__ double red[8][FLD_SLICES][FLD_CELLS];   // e2, e1, G2 (3), G1 (3)
    __shared__ double es[8][FLD_CELLS];
    __shared__ bool last;
    const int cl = threadIdx.x & (FLD_CELLS - 1);
    const int sl = threadIdx.x / FLD_CELLS;
    const int n = blockIdx.x * FLD_CELLS + cl;
    const bool two = flags & FLD_SECOND, one = flags & (FLD_FIRST | FLD_E1_STORE);
    double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (n < a.N) {
        const double *u = a.U + n, *us = a.Us + n;
#pragma unroll 4
        for (int al = sl; al < a.M; al += FLD_SLICES) {
            const double c = u[(size_t)al * a.N], sn = us[(size_t)al * a.N];
            if (two) {
                v[0] = fma(c, __ldg(a.W2 + al), v[0]);
#pragma unroll
                for (int k = 0; k < 3; ++k) v[2 + k] = fma(sn, __ldg(a.Wk2 + 3 * al + k), v[2 + k]);
            }
            if (one) {
                v[1] = fma(c, __ldg(a.W1 + al), v[1]);
#pragma unroll
                for (int k = 0; k < 3; ++k) v[5 + k] = fma(sn, __ldg(a.Wk1 + 3 * al + k), v[5 + k]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) red[i][sl][cl] = v[i];
    __syncthreads();
    if (sl == 0) {   // fixed-order slice sums of cell cl
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            for (int q = 1; q < FLD_SLICES; ++q) v[i] += red[i][q][cl];
            es[i][cl] = v[i];
        }
        if ((flags & FLD_E1_STORE) && n < a.N) {
            a.E1store[n] = v[1];
            for (int k = 0; k < 3; ++k) a.G1store[3 * n + k] = v[5 + k];
        }
    }
    __syncthreads();
    double kin = 0.0, edf = 0.0;
    if (n < a.N) {
        const int j1 = a.cell_offset[n + 1];
        const double Mn = a.M_cell[n];
        for (int j = a.cell_offset[n] + sl; j < j1; j += FLD_SLICES) {
            const double g2[3] = {es[2][cl], es[3][cl], es[4][cl]};
            const double g1[3] = {es[5][cl], es[6][cl], es[7][cl]};
            kin += kick_atom_moving(a, flags, j, es[0][cl], es[1][cl], g2, g1, a.w_atom[j] * Mn);
        }
        if (sl == 0) edf = a.E_cell[n];
    }
    if (!(flags & FLD_ENERGY)) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kin += __shfl_xor_sync(CAVMD_FULL_MASK, kin, o);
        edf += __shfl_xor_sync(CAVMD_FULL_MASK, edf, o);
    }
    constexpr int NW = FLD_CELLS * FLD_SLICES / 32;
    double *scr = &red[0][0][0];   // free after the slice sums
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        scr[threadIdx.x >> 5] = kin;
        scr[NW + (threadIdx.x >> 5)] = edf;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double k = 0.0, d = 0.0;
        for (int w = 0; w < NW; ++w) {
            k += scr[w];
            d += scr[NW + w];
        }
        a.e_kin_part[blockIdx.x] = k;
        a.e_dftb_part[blockIdx.x] = d;
        __threadfence();
        const unsigned ticket = atomicAdd(a.done_counter, 1u);
        last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    record_energies<FLD_CELLS * FLD_SLICES>(a, flags, gridDim.x, scr);
}

// u_a(R_n) = cos(k_a.R_n + phi_a) and sin(k_a.R_n + phi_a) at the centres of mass of the cells,
// by angle addition from the same functions at the reference positions R0_n (U0, Us0, formed
// once): with d = k_a.(R_n - R0_n), cos(t0 + d) = cos t0 cos d - sin t0 sin d and
// sin(t0 + d) = sin t0 cos d + cos t0 sin d. A cell moves ~4e-3 bohr per step and optical wave
// vectors are ~1e-4 / bohr, so d stays small: for |d| < 4e-3, cos d and sin d come from their
// Taylor series to d^4 and d^5 (truncation below 1e-17), otherwise from sincos. d is measured
// from the fixed reference every step, so nothing accumulates from step to step.
// Thread = cell (its centre summed over the cell's atoms in order), MF_MODES modes per thread.
constexpr int MF_MODES = 16;
constexpr double MF_SERIES_MAX = 4e-3;
__global__ void k_mode_functions_com(const double *__restrict__ k, const double *__restrict__ R0,
                                     const double *__restrict__ U0, const double *__restrict__ Us0,
                                     const double *__restrict__ r, const double *__restrict__ mass,
                                     const int *__restrict__ off, int M, int N, double *__restrict__ U,
                                     double *__restrict__ Us) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double mt = 0.0, x0 = 0.0, x1 = 0.0, x2 = 0.0;
    for (int j = off[n]; j < off[n + 1]; ++j) {
        const double m = mass[j];
        mt += m;
        x0 = fma(m, r[3 * j], x0);
        x1 = fma(m, r[3 * j + 1], x1);
        x2 = fma(m, r[3 * j + 2], x2);
    }
    const double d0 = x0 / mt - R0[3 * n], d1 = x1 / mt - R0[3 * n + 1], d2 = x2 / mt - R0[3 * n + 2];
    const int a1 = min(M, (int)(blockIdx.y + 1) * MF_MODES);
    for (int al = blockIdx.y * MF_MODES; al < a1; ++al) {
        const double d = fma(k[3 * al], d0, fma(k[3 * al + 1], d1, k[3 * al + 2] * d2));
        double sd, cd;
        if (fabs(d) < MF_SERIES_MAX) {
            const double d2s = d * d;
            cd = fma(d2s, fma(d2s, 1.0 / 24.0, -0.5), 1.0);
            sd = d * fma(d2s, fma(d2s, 1.0 / 120.0, -1.0 / 6.0), 1.0);
        } else {
            sincos(d, &sd, &cd);
        }
        const size_t e = (size_t)al * N + n;
        const double c0 = U0[e], s0 = Us0[e];
        U[e] = fma(c0, cd, -s0 * sd);
        Us[e] = fma(s0, cd, c0 * sd);
    }
}

// cos and sin of k_a.R_n + phi_a at given positions (the reference functions, once).
__global__ void k_mode_functions_pair(const double *__restrict__ k, const double *__restrict__ phi,
                                      const double *__restrict__ R, int M, int N, double *__restrict__ U,
                                      double *__restrict__ Us) {
    const size_t total = (size_t)M * N;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int al = (int)(e / N), n = (int)(e - (size_t)al * N);
        const double th = fma(k[3 * al], R[3 * n], fma(k[3 * al + 1], R[3 * n + 1], fma(k[3 * al + 2], R[3 * n + 2], phi[al])));
        double sn, cs;
        sincos(th, &sn, &cs);
        U[e] = cs;
        Us[e] = sn;
    }
}

// G_n = -sum_a W_a k_a Us[a][n] (thread per cell; evaluation read-back only).
__global__ void k_field_grad_only(const double *__restrict__ Us, const double *__restrict__ W,
                                  const double *__restrict__ k, int M, int N, double *__restrict__ G) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    for (int al = 0; al < M; ++al) {
        const double w = -W[al] * Us[(size_t)al * N + n];
        g0 = fma(w, k[3 * al], g0);
        g1 = fma(w, k[3 * al + 1], g1);
        g2 = fma(w, k[3 * al + 2], g2);
    }
    G[3 * n] = g0;
    G[3 * n + 1] = g1;
    G[3 * n + 2] = g2;
}

__global__ void k_field_only(const double *__restrict__ U, const double *__restrict__ W, int M, int N,
                             double *__restrict__ E) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double e = 0.0;
    for (int al = 0; al < M; ++al) e = fma(U[(size_t)al * N + n], W[al], e);
    E[n] = e;
}

}  // namespace

cudaError_t launch_mode_functions(const double *k, const double *phi, const double *R, int M, int N,
                                  double *U, cudaStream_t st) {
    const long long total = (long long)M * N;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_mode_functions<<<blocks, 256, 0, st>>>(k, phi, R, M, N, U);
    return cudaGetLastError();
}

cudaError_t launch_mode_functions_pair(const double *k, const double *phi, const double *R, int M, int N, double *U,
                                       double *Us, cudaStream_t st) {
    const long long total = (long long)M * N;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_mode_functions_pair<<<blocks, 256, 0, st>>>(k, phi, R, M, N, U, Us);
    return cudaGetLastError();
}

cudaError_t launch_mode_functions_com(const double *k, const double *R0, const double *U0, const double *Us0,
                                      const double *r, const double *mass, const int *cell_offset, int M, int N,
                                      double *U, double *Us, cudaStream_t st) {
    const dim3 grid((N + 127) / 128, (M + MF_MODES - 1) / MF_MODES);
    k_mode_functions_com<<<grid, 128, 0, st>>>(k, R0, U0, Us0, r, mass, cell_offset, M, N, U, Us);
    return cudaGetLastError();
}

cudaError_t launch_field_grad_only(const double *Us, const double *W, const double *k, int M, int N, double *G,
                                   cudaStream_t st) {
    k_field_grad_only<<<(N + 127) / 128, 128, 0, st>>>(Us, W, k, M, N, G);
    return cudaGetLastError();
}

cudaError_t launch_photon(const StepArgs &a, int flags, cudaStream_t st) {
    if (flags & PH_FORWARD)
        k_photon<<<a.M, PH_THREADS, 0, st>>>(a, flags);
    else
        k_photon_modes<<<(a.M + PHM_THREADS - 1) / PHM_THREADS, PHM_THREADS, 0, st>>>(a, flags);
    return cudaGetLastError();
}

int field_blocks(int N) { return (N + FLD_CELLS - 1) / FLD_CELLS; }   // >= the kick kernel's blocks

cudaError_t launch_field(const StepArgs &a, int flags, cudaStream_t st) {
    if (flags & FLD_E_GIVEN) {
        if (a.G1in) {
            k_kick<<<(a.N + KICK_THREADS - 1) / KICK_THREADS, KICK_THREADS, 0, st>>>(a, flags);
        } else {   // one resident wave at most (fewer block partials and last-block tickets), and at
                   // most field_blocks(N) blocks: the energy partials hold that many
            const long long need = (3LL * a.n_atoms + KA_THREADS - 1) / KA_THREADS;
            const int blocks = (int)std::max(1LL, std::min({need, (long long)KA_MAX_BLOCKS, (long long)field_blocks(a.N)}));
            k_kick_atoms<<<blocks, KA_THREADS, 0, st>>>(a, flags);
        }
    }
    else if (a.Us)
        k_field_moving<<<field_blocks(a.N), FLD_CELLS * FLD_SLICES, 0, st>>>(a, flags);
    else
        k_field<<<field_blocks(a.N), FLD_CELLS * FLD_SLICES, 0, st>>>(a, flags);
    return cudaGetLastError();
}

static __global__ void k_trial_positions(const double *__restrict__ r, const double *__restrict__ p,
                                  const double *__restrict__ inv_mass, double dt, int n, double *__restrict__ rt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    rt[i] = fma(dt * inv_mass[i / 3], p[i], r[i]);
}

cudaError_t launch_trial_positions(const double *r, const double *p, const double *inv_mass, double dt, int n_atoms,
                                   double *r_trial, cudaStream_t st) {
    k_trial_positions<<<(3 * n_atoms + 255) / 256, 256, 0, st>>>(r, p, inv_mass, dt, n_atoms, r_trial);
    return cudaGetLastError();
}

// Observables of the synchronised state packed for one device-to-host copy:
// out[0..7] the energy record, out[8] the largest SCC iteration count, out[9] the status word,
// then M (N), q, p, D (M each) from out[16]. Grid-stride copies over many blocks; the largest
// iteration count goes through an atomic maximum in scr[0] (order-independent), and the last block
// to finish (ticket in scr[1]) writes the scalars and resets both.
constexpr int PACK_THREADS = 256;
static __global__ void __launch_bounds__(PACK_THREADS) k_obs_pack(
    const double *__restrict__ hist_slot, const int *__restrict__ iters, int N, const unsigned *__restrict__ status,
    const double *__restrict__ Mc, const double *__restrict__ q, const double *__restrict__ p,
    const double *__restrict__ D, int M, int with_arrays, double *__restrict__ out, unsigned *__restrict__ scr) {
    __shared__ unsigned mx[PACK_THREADS / 32];
    __shared__ bool last;
    const int t = threadIdx.x;
    const long long g = (long long)blockIdx.x * PACK_THREADS + t, stride = (long long)gridDim.x * PACK_THREADS;
    unsigned m = 0u;
    for (long long n = g; n < N; n += stride) m = max(m, (unsigned)max(iters[n], 0));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(CAVMD_FULL_MASK, m, o));
    if ((t & 31) == 0) mx[t >> 5] = m;
    if (with_arrays) {
        for (long long n = g; n < N; n += stride) out[16 + n] = Mc[n];
        for (long long a = g; a < M; a += stride) {
            out[16 + N + a] = q[a];
            out[16 + N + M + a] = p[a];
            out[16 + N + 2 * M + a] = D[a];
        }
    }
    __syncthreads();
    if (t == 0) {
        unsigned r = 0u;
        for (int w = 0; w < PACK_THREADS / 32; ++w) r = max(r, mx[w]);
        atomicMax(scr, r);
        __threadfence();
        last = atomicAdd(scr + 1, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    if (t < 8) out[t] = hist_slot[t];
    if (t == 0) {
        __threadfence();
        out[8] = (double)atomicAdd(scr, 0u);
        out[9] = (double)*status;
        scr[0] = 0u;
        scr[1] = 0u;
    }
}

cudaError_t launch_obs_pack(const double *hist_slot, const int *iters, int N, const unsigned *status,
                            const double *Mc, const double *q, const double *p, const double *D, int M,
                            bool with_arrays, double *out, unsigned *scr, cudaStream_t st) {
    const long long work = std::max<long long>(N, M);
    const int grid = (int)std::max<long long>(1, std::min<long long>(1216, (work + 4 * PACK_THREADS - 1) / (4 * PACK_THREADS)));
    k_obs_pack<<<grid, PACK_THREADS, 0, st>>>(hist_slot, iters, N, status, Mc, q, p, D, M, with_arrays ? 1 : 0, out,
                                              scr);
    return cudaGetLastError();
}

cudaError_t launch_field_only(const double *U, const double *W, int M, int N, double *E,
                              cudaStream_t st) {
    k_field_only<<<(N + 127) / 128, 128, 0, st>>>(U, W, M, N, E);
    return cudaGetLastError();
}
