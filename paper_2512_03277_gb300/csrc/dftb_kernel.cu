// Batched second-order SCC-DFTB of small molecules, one group of NORB lanes per molecule.
//
// The paper evaluates -grad V_n, mu_n and the Mulliken charges of every cell on the fly with
// SCC-DFTB (section "Computational details"; Eq. dpj needs -grad V_n). This kernel evaluates
// many independent cells of one composition at once:
//
//   H0, S from Slater-Koster tables  ->  warm-started S-orthonormal basis C (Cholesky of C^T S C)
//   -> SCC loop: shifts eps_A = sum_B gamma_AB dq_B, H = H0 + 1/2 S o (eps_A + eps_B),
//      A = C^T H C, cyclic Jacobi on A (rotations applied to A and C), aufbau occupation,
//      P = 2 C_occ C_occ^T, Mulliken populations, Anderson-accelerated mixing
//   -> energy, analytic gradient (P dH0 + (P (eps_A+eps_B)/2 - W) dS + dgamma + dE_rep),
//      dipole M_n = pol . sum_A Q_A r_A and the Mulliken dipole derivative b_A = Q_A pol.
//
// Layout: lane j of a group owns column j of every NORB x NORB matrix, stored column-major in
// the group's shared-memory slot with an odd leading dimension. All groups of a warp advance in
// lock step (__syncwarp); a group whose charges have converged idles until the slowest group
// of its warp is done. The FP64 pipe bounds this kernel on GB300, so auxiliary quantities that
// only steer the iteration (rotation angles, mixing coefficients, convergence tests) are formed
// in FP32 or by integer comparisons, while every quantity that enters the result (rotations
// themselves, matrices, populations, energies, forces) is computed in FP64.
#include "cavmd_internal.cuh"

namespace {

constexpr int NHIST = 3;          // Anderson history (current + 2 previous iterates)
constexpr int MAX_SWEEPS = 24;    // default bound on the Jacobi sweeps of a cold start
constexpr double JACOBI_TOL = 1e-15;   // off-diagonal magnitude treated as converged (Hartree)
constexpr double MIN_GAP = 1e-3;       // closed-shell HOMO-LUMO threshold (Hartree)
constexpr double EIG_TOL = 1e-10;      // occupied-virtual coupling treated as converged (Hartree)
constexpr float KMAX_PERT = 1e-4f;     // largest generator entry for the second-order update

template <int NAT, int NORB>
struct MolShared {
    static constexpr int LD = (NORB % 2 == 0) ? NORB + 1 : NORB;   // odd column stride
    static constexpr int NPAIR = NAT * (NAT - 1) / 2;
    double S[NORB * LD];
    double H0[NORB * LD];
    double A[NORB * LD];
    double C[NORB * LD];
    double Y[NORB * LD];
    double P[NORB * LD];
    double pos[NAT][3];
    double gam[NAT][NAT];
    double zv[NAT];
    double q[NAT];
    double qout[NAT];
    double shift[NAT];
    double hq[NHIST][NAT];
    double hf[NHIST][NAT];
    double qstart[NAT];   // q(t) of the previous step, for the predictor
    double red[NORB];
    double cs[NORB / 2 + 1][2];
    double invd[NORB];
    double hsh[NORB];     // half shift of the atom of each orbital
    float diagf[NORB];    // diagonal of A in FP32 (generator denominators)
    double gpair[NPAIR > 0 ? NPAIR : 1][3];
    double gpart[2][NPAIR > 0 ? NPAIR : 1][3];   // H0 and S parts of the pair gradients
    double epair[NPAIR > 0 ? NPAIR : 1];
    double Hs[NORB * LD];   // H of the current SCC iteration
    int occ_list[NORB];
    int virt_list[NORB];
    int occf[NORB];       // orbital column j is occupied
    int eok[NORB];        // occupied-virtual couplings of column j were below EIG_TOL
    int orb_atom[NORB];
    int atom_off[NAT + 1];
    int spec[NAT];
    int pa[NPAIR > 0 ? NPAIR : 1];
    int pb[NPAIR > 0 ? NPAIR : 1];
    int flag;
    int conv;
    int iters;
    int nocc;
};

__device__ __forceinline__ void radial(const double *par, double r, const DevSK &sk, double &v,
                                       double &dv) {
    const double a = par[0], b = par[1], c1 = par[2], c2 = par[3];
    const double e = a * exp(-b * r);
    const double poly = fma(fma(c2, r, c1), r, 1.0);
    const double dpoly = fma(2.0 * c2, r, c1);
    const double x = (r - (sk.r_cut - sk.taper)) * sk.inv_taper;
    double f = 1.0, df = 0.0;
    if (x > 0.0) {
        if (x < 1.0) {
            double sn, cn;
            sincospi(x, &sn, &cn);
            f = 0.5 * (1.0 + cn);
            df = -0.5 * 3.141592653589793 * sk.inv_taper * sn;
        } else {
            f = 0.0;
        }
    }
    v = e * poly * f;
    dv = e * (fma(-b * poly, f, dpoly * f) + poly * df);
}

// Jacobi round-robin schedule for even n: in round r (0..n-2) index n-1 meets r and index j
// meets (2r - j) mod (n-1). Returns the partner of j and the pair slot (0 = the pair with n-1).
__device__ __forceinline__ int rr_partner(int j, int r, int n, int &slot) {
    const int m = n - 1;
    if (j == m) { slot = 0; return r; }
    if (j == r) { slot = 0; return m; }
    const int dlt = (j - r + m) % m;
    slot = min(dlt, m - dlt);
    return (r - dlt + m) % m;
}

__device__ __forceinline__ void rr_pair(int k, int r, int n, int &p, int &q) {
    const int m = n - 1;
    if (k == 0) { p = r; q = m; return; }
    const int x = (r + k) % m, y = (r - k + m) % m;
    p = min(x, y);
    q = max(x, y);
}

// Rotation (c, s) that annihilates a_pq: tan(phi) = t from the FP32 quadratic, then (c, s) made
// orthonormal in FP64 by two Newton steps on 1/sqrt(c^2 + s^2).
__device__ __forceinline__ void jacobi_cs(double app, double aqq, double apq, double &c, double &s) {
    const float d = d2f_steer(aqq - app);
    const float o = 2.0f * d2f_steer(apq);
    float t = 0.0f;
    if (o != 0.0f) t = o / (d + copysignf(sqrtf(fmaf(d, d, o * o)), d));
    const float cf = rsqrtf(fmaf(t, t, 1.0f));
    c = f2d_steer(cf);
    s = f2d_steer(t * cf);
    for (int it = 0; it < 2; ++it) {
        const double nrm = fma(c, c, s * s);
        const double f = fma(-0.5, nrm, 1.5);
        c *= f;
        s *= f;
    }
}

template <int NAT, int NORB>
__global__ void __launch_bounds__(256, 1) dftb_kernel(const DevSK *__restrict__ skp, const DftbArgs a, const int gpw) {
    const DevSK &sk = *skp;
    using SM = MolShared<NAT, NORB>;
    constexpr int LD = SM::LD;
    // gpw <= 32 / NORB molecules per warp (fewer spreads a small batch over more warps)
    constexpr int NPAIR = SM::NPAIR;
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int g = lane / NORB;
    const int j = lane - g * NORB;
    const bool act = g < gpw;
    SM &m = reinterpret_cast<SM *>(smem_raw)[warp * gpw + (act ? g : 0)];
    const bool disp = a.n_disp > 0;                       // finite-difference rows
    const int n_rows = disp ? a.n_cells * a.n_disp : a.n_cells;
    const int idx = (blockIdx.x * wpb + warp) * gpw + g;
    const bool valid = act && idx < n_rows;
    const int ridx = min(idx, n_rows - 1);
    const int cidx = disp ? ridx / a.n_disp : ridx;
    const int cell = a.cell_list ? a.cell_list[cidx] : cidx;
    const int a0 = a.cell_offset[cell];

    // ---------------------------------------------------------------- load geometry, layout
    const bool open = a.E_open != nullptr && !disp;
    double p_new[3], r_new[3];
    if (act && j < NAT) {
        m.spec[j] = a.species[a0 + j];
        m.pos[j][0] = a.r[3 * (a0 + j) + 0];
        m.pos[j][1] = a.r[3 * (a0 + j) + 1];
        m.pos[j][2] = a.r[3 * (a0 + j) + 2];
        if (open) {   // opening half-flow: kick by tau F + E_n b, then drift (stored after the warp sync)
            const int at = a0 + j;
            const double e1 = a.E_open[cell], im = a.inv_mass[at];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                p_new[k] = fma(a.tau, a.F[3 * at + k], fma(e1, a.b[3 * at + k], a.p_open[3 * at + k]));
                r_new[k] = fma(a.dt * im, p_new[k], m.pos[j][k]);
                m.pos[j][k] = r_new[k];
            }
        }
        if (disp) {   // displaced copy: atom da, component dc, by +h (forward) or +-h (central)
            const int k = ridx - cidx * a.n_disp;
            const int kk = a.fd_central ? k >> 1 : k;
            const int da = kk / 3, dc = kk - 3 * (kk / 3);
            const double sg = (a.fd_central && (k & 1)) ? -1.0 : 1.0;
            if (j == da) m.pos[j][dc] += sg * a.fd_h;
        }
    }
    __syncwarp();   // every lane of the warp has read the state it kicks before any is stored
    if (open && valid && j < NAT) {
        const int at = a0 + j;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            a.p_open[3 * at + k] = p_new[k];
            a.r_open[3 * at + k] = r_new[k];
        }
    }
    if (act && j == 0) {
        int o = 0;
        double nel = 0.0;
        for (int at = 0; at < NAT; ++at) {
            m.atom_off[at] = o;
            const int no = sk.norb[m.spec[at]];
            for (int k = 0; k < no; ++k) m.orb_atom[o + k] = at;
            o += no;
            m.zv[at] = sk.zval[m.spec[at]];
            nel += m.zv[at];
        }
        m.atom_off[NAT] = o;
        m.nocc = (int)(nel * 0.5f + 0.25f);
        int pi = 0;
        for (int x = 0; x < NAT; ++x)
            for (int y = x + 1; y < NAT; ++y) { m.pa[pi] = x; m.pb[pi] = y; ++pi; }
        m.flag = 0;
        m.conv = 0;
        m.iters = 0;
    }
    __syncwarp();

    // ---------------------------------------------------------------- H0, S, gamma
    if (act) {
        const int at = m.orb_atom[j];
        const int e = m.spec[at];
        const double eps = (j == m.atom_off[at]) ? sk.onsite[e][0] : sk.onsite[e][1];
        for (int i = 0; i < NORB; ++i) {
            m.S[j * LD + i] = (i == j) ? 1.0 : 0.0;
            m.H0[j * LD + i] = (i == j) ? eps : 0.0;
        }
    }
    __syncwarp();
    if (act) {
        // one (pair, table) task per lane: the H0 and the S integrals of a pair on two lanes
        for (int task = j; task < 2 * NPAIR; task += NORB) {
            const int pi = task % NPAIR, t = task / NPAIR;
            const int A = m.pa[pi], B = m.pb[pi];
            const int eA = m.spec[A], eB = m.spec[B];
            const int oA = m.atom_off[A], oB = m.atom_off[B];
            const int na = sk.norb[eA], nb = sk.norb[eB];
            const double dx = m.pos[B][0] - m.pos[A][0];
            const double dy = m.pos[B][1] - m.pos[A][1];
            const double dz = m.pos[B][2] - m.pos[A][2];
            const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
            const double ir = rsqrt_nr(r2);
            const double r = r2 * ir;
            const double ev[3] = {dx * ir, dy * ir, dz * ir};
            {
                const double (*tab)[CAVMD_MAX_ELEM][4][4] = t == 0 ? sk.h0 : sk.s;
                double *X = t == 0 ? m.H0 : m.S;
                double v, dv;
                radial(tab[eA][eB][CAVMD_SK_SS], r, sk, v, dv);
                X[oB * LD + oA] = v;
                X[oA * LD + oB] = v;
                if (nb == 4) {
                    radial(tab[eA][eB][CAVMD_SK_SP], r, sk, v, dv);
                    for (int i = 0; i < 3; ++i) {
                        X[(oB + 1 + i) * LD + oA] = ev[i] * v;
                        X[oA * LD + oB + 1 + i] = ev[i] * v;
                    }
                }
                if (na == 4) {
                    radial(tab[eB][eA][CAVMD_SK_SP], r, sk, v, dv);
                    for (int i = 0; i < 3; ++i) {
                        X[oB * LD + oA + 1 + i] = -ev[i] * v;
                        X[(oA + 1 + i) * LD + oB] = -ev[i] * v;
                    }
                }
                if (na == 4 && nb == 4) {
                    double vs, vp;
                    radial(tab[eA][eB][CAVMD_SK_PPS], r, sk, vs, dv);
                    radial(tab[eA][eB][CAVMD_SK_PPP], r, sk, vp, dv);
                    const double dl = vs - vp;
                    for (int i = 0; i < 3; ++i)
                        for (int k = 0; k < 3; ++k) {
                            const double val = fma(ev[i] * ev[k], dl, (i == k) ? vp : 0.0);
                            X[(oB + 1 + k) * LD + oA + 1 + i] = val;
                            X[(oA + 1 + i) * LD + oB + 1 + k] = val;
                        }
                }
            }
        }
        if (j < NAT) {
            for (int k = 0; k < NAT; ++k) {
                if (k == j) {
                    m.gam[j][k] = sk.hubbard[m.spec[j]];
                } else {
                    const double dx = m.pos[k][0] - m.pos[j][0];
                    const double dy = m.pos[k][1] - m.pos[j][1];
                    const double dz = m.pos[k][2] - m.pos[j][2];
                    m.gam[j][k] = rsqrt_nr(fma(dx, dx, fma(dy, dy, fma(dz, dz, sk.gamma_c2[m.spec[j]][m.spec[k]]))));
                }
            }
        }
    }
    __syncwarp();

    // ---------------------------------------------------------------- warm-started S-orthonormal basis
    if (act) {
        if (a.have_warm) {
            const double *cw = a.Cwarm + (a.Cwarm_off ? a.Cwarm_off[cell] : (long long)cell * NORB * NORB);
            for (int i = 0; i < NORB; ++i) m.C[j * LD + i] = cw[j * NORB + i];
            // linear predictor 2 q(t) - q(t - dt) of the populations (q_prev equals q after a
            // cold start, so the first warm step starts from q(t) itself)
            if (j < NAT) {
                const double qt = a.qpop[a0 + j];
                m.qstart[j] = qt;
                m.q[j] = disp ? qt : fma(2.0, qt, -a.qprev[a0 + j]);   // displaced rows start at q(r)
            }
        } else {
            for (int i = 0; i < NORB; ++i) m.C[j * LD + i] = (i == j) ? 1.0 : 0.0;
            if (j < NAT) m.q[j] = m.zv[j];
        }
    }
    __syncwarp();
    // G = C^T S C  (in A)
    if (act) {
        if (a.have_warm) {
            double y[NORB];
#pragma unroll
            for (int i = 0; i < NORB; ++i) y[i] = 0.0;
            for (int k = 0; k < NORB; ++k) {
                const double ckj = m.C[j * LD + k];
#pragma unroll
                for (int i = 0; i < NORB; ++i) y[i] = fma(m.S[k * LD + i], ckj, y[i]);
            }
#pragma unroll
            for (int i = 0; i < NORB; ++i) m.Y[j * LD + i] = y[i];
        }
    }
    __syncwarp();
    if (act) {
        if (a.have_warm) {
            for (int i = 0; i < NORB; ++i) {
                double s = 0.0;
#pragma unroll
                for (int k = 0; k < NORB; ++k) s = fma(m.C[i * LD + k], m.Y[j * LD + k], s);
                m.A[j * LD + i] = s;
            }
        } else {
            for (int i = 0; i < NORB; ++i) m.A[j * LD + i] = m.S[j * LD + i];
        }
    }
    __syncwarp();
    // Cholesky G = L L^T, right-looking, lane = column (L in the lower triangle of A)
    for (int k = 0; k < NORB; ++k) {
        if (act && j == k) {
            double d = m.A[k * LD + k];
            if (!(d > 1e-300)) {
                m.flag |= ERRBIT_S_NOT_PD;
                d = 1.0;
            }
            const double y = rsqrt_nr(d);
            m.invd[k] = y;
            m.A[k * LD + k] = d * y;
            for (int i = k + 1; i < NORB; ++i) m.A[k * LD + i] *= y;
        }
        __syncwarp();
        if (act && j > k) {
            const double ljk = m.A[k * LD + j];
            for (int i = j; i < NORB; ++i) m.A[j * LD + i] = fma(-m.A[k * LD + i], ljk, m.A[j * LD + i]);
        }
        __syncwarp();
    }
    // C <- C L^-T (lane = row)
    if (act) {
        const int i = j;
        for (int c = 0; c < NORB; ++c) {
            double x = m.C[c * LD + i];
            for (int k = 0; k < c; ++k) x = fma(-m.C[k * LD + i], m.A[k * LD + c], x);
            m.C[c * LD + i] = x * m.invd[c];
        }
    }
    __syncwarp();

    // ---------------------------------------------------------------- SCC loop
    // Each iteration builds H(q) and A = C^T H C in the current S-orthonormal basis C and moves C
    // towards the eigenvectors of H. When the occupied-virtual couplings are small, C takes the
    // second-order exponential V = I + K + K^2/2 of the first-order generator
    // K_kj = A_kj / (A_jj - A_kk) over occupied-virtual pairs: V is orthogonal to O(K^4) and, like
    // a Jacobi sweep, squares the remaining coupling, at a third of the cost. Otherwise (the first
    // iteration after a geometry change, a cold start, a large charge change) C takes Jacobi
    // sweeps: one per iteration when warm started, to full convergence in the first iteration of a
    // cold start. Only occupied-virtual mixing changes P, so occupied-occupied couplings are left
    // to the final energy-weighted density, which uses the whole occupied block. The charges count
    // as converged once |q_out - q| < tol and every occupied-virtual coupling was below EIG_TOL
    // before the update.
    int it = 0;
    for (it = 1; it <= a.max_iter; ++it) {
        const bool work = act && !m.conv;
        if (work && j < NAT) {
            double sh = 0.0;
            for (int k = 0; k < NAT; ++k) sh = fma(m.gam[j][k], m.q[k] - m.zv[k], sh);
            m.shift[j] = sh;
        }
        __syncwarp();
        if (work) m.hsh[j] = 0.5 * m.shift[m.orb_atom[j]];
        __syncwarp();
        if (work) {   // H column j: H0 + S o (eps_A + eps_B)/2 (halving is exact, so this equals the
                      // product with the halved sum bit for bit)
            const double hj = m.hsh[j];
            for (int i = 0; i < NORB; ++i)
                m.Hs[j * LD + i] = fma(m.S[j * LD + i], m.hsh[i] + hj, m.H0[j * LD + i]);
        }
        __syncwarp();
        if (work) {   // Y = H C
            double y[NORB];
#pragma unroll
            for (int i = 0; i < NORB; ++i) y[i] = 0.0;
            for (int k = 0; k < NORB; ++k) {
                const double ckj = m.C[j * LD + k];
#pragma unroll
                for (int i = 0; i < NORB; ++i) y[i] = fma(m.Hs[k * LD + i], ckj, y[i]);
            }
#pragma unroll
            for (int i = 0; i < NORB; ++i) m.Y[j * LD + i] = y[i];
        }
        __syncwarp();
        // A = C^T H C = C^T Y is formed only where the iteration needs it: its diagonal (aufbau,
        // denominators) and its occupied-virtual block (generator, convergence), the latter as
        // (occupied, virtual) pair tasks spread over the lanes and stored symmetric. The Jacobi
        // path adds the other entries when it runs.
        if (work) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < NORB; ++k) s = fma(m.C[j * LD + k], m.Y[j * LD + k], s);
            m.A[j * LD + j] = s;
        }
        __syncwarp();
        // aufbau occupation from the diagonal of A
        if (work) {
            m.diagf[j] = d2f_steer(m.A[j * LD + j]);
            const long long kj = order_key(m.A[j * LD + j]);
            int rank = 0;
            for (int i = 0; i < NORB; ++i) {
                const long long ki = order_key(m.A[i * LD + i]);
                rank += (ki < kj) || (ki == kj && i < j);
            }
            m.occf[j] = rank < m.nocc;
            if (rank < m.nocc) m.occ_list[rank] = j;
            else m.virt_list[rank - m.nocc] = j;
        }
        __syncwarp();
        if (work) {   // occupied-virtual block
            const int nv = NORB - m.nocc;
            for (int t = j; t < m.nocc * nv; t += NORB) {
                const int oi = t / nv;
                const int o = m.occ_list[oi], v = m.virt_list[t - oi * nv];
                double s = 0.0;
#pragma unroll
                for (int k = 0; k < NORB; ++k) s = fma(m.C[v * LD + k], m.Y[o * LD + k], s);
                m.A[o * LD + v] = s;
                m.A[v * LD + o] = s;
            }
        }
        __syncwarp();
        // first-order occupied-virtual generator, column j, into Y (FP32: it only steers)
        // Only the entries of the other block (virtual rows of an occupied column, and conversely)
        // are non-zero; the loop visits just those.
        float kmax = 0.0f;
        unsigned same_mask = 0u, other_mask = 0u;
        if (work) {
            unsigned om = 0u;
#pragma unroll
            for (int k = 0; k < NORB; ++k) om |= (m.occf[k] ? 1u : 0u) << k;
            same_mask = m.occf[j] ? om : (~om & ((1u << NORB) - 1u));
            other_mask = ~same_mask & ((1u << NORB) - 1u);
#pragma unroll
            for (int k = 0; k < NORB; ++k) m.P[j * LD + k] = 0.0;   // K column j (P is free until the density)
            const float dj = m.diagf[j];
            bool small = true;
            for (unsigned om = other_mask; om; om &= om - 1u) {
                const int k = __ffs(om) - 1;
                const double akj = m.A[j * LD + k];
                if (!abs_lt(akj, EIG_TOL)) small = false;
                float kf = d2f_steer(akj) / (dj - m.diagf[k]);
                if (!(fabsf(kf) <= 1e30f)) kf = 1e30f;   // degenerate or non-finite: Jacobi path
                m.P[j * LD + k] = f2d_steer(kf);
                kmax = fmaxf(kmax, fabsf(kf));
            }
            m.eok[j] = small;
        }
        const bool cold_first = !a.have_warm && it == 1;
        const bool perturb = __all_sync(CAVMD_FULL_MASK, !work || (kmax < KMAX_PERT && !cold_first));
        __syncwarp();
        if (perturb) {
            double cn[NORB];
            if (work) {   // V column j = e_j + K e_j + K (K e_j) / 2, then C <- C V
                // (K^2)(i, j) vanishes for rows i of the other block; for rows of j's own block it sums
                // over the other block only: n_occ n_virt products per column, in increasing index
                // order (the skipped terms are exact zeros). The row sums go to A, free here.
                for (unsigned sm = same_mask; sm; sm &= sm - 1u) {
                    const int i = __ffs(sm) - 1;
                    double acc = 0.0;
                    for (unsigned om = other_mask; om; om &= om - 1u) {
                        const int mm = __ffs(om) - 1;
                        acc = fma(m.P[mm * LD + i], m.P[j * LD + mm], acc);
                    }
                    m.A[j * LD + i] = acc;
                }
                // (K + K^2 / 2) e_j; the identity part of V is C's own column, the start of C V
                double v[NORB];
#pragma unroll
                for (int i = 0; i < NORB; ++i)
                    v[i] = fma(0.5, ((same_mask >> i) & 1u) ? m.A[j * LD + i] : 0.0, m.P[j * LD + i]);
#pragma unroll
                for (int i = 0; i < NORB; ++i) cn[i] = m.C[j * LD + i];
                for (int k = 0; k < NORB; ++k) {
                    const double vk = v[k];
#pragma unroll
                    for (int i = 0; i < NORB; ++i) cn[i] = fma(m.C[k * LD + i], vk, cn[i]);
                }
            }
            __syncwarp();
            if (work) {
#pragma unroll
                for (int i = 0; i < NORB; ++i) m.C[j * LD + i] = cn[i];
            }
            __syncwarp();
        } else {
            // the sweeps need all of A: add the off-diagonal entries inside the occupied and the
            // virtual blocks (Y still holds H C), one (a, b) pair per task, stored symmetric
            if (work) {
                for (int t = j; t < NORB * (NORB - 1) / 2; t += NORB) {
                    int pa_ = 0, rem = t;
                    while (rem >= NORB - 1 - pa_) {
                        rem -= NORB - 1 - pa_;
                        ++pa_;
                    }
                    const int pb_ = pa_ + 1 + rem;
                    if (m.occf[pa_] == m.occf[pb_]) {
                        double s = 0.0;
#pragma unroll
                        for (int k = 0; k < NORB; ++k) s = fma(m.C[pa_ * LD + k], m.Y[pb_ * LD + k], s);
                        m.A[pb_ * LD + pa_] = s;
                        m.A[pa_ * LD + pb_] = s;
                    }
                }
            }
            __syncwarp();
            // a cold start sweeps until the off-diagonal entries are below tolerance, at most `cap`
            // sweeps (then DEVICE_TIMEOUT); later iterations take one sweep
            const int cap = cold_first ? (a.max_sweeps > 0 ? a.max_sweeps : MAX_SWEEPS) : 1;
            for (int sweep = 0;; ++sweep) {
                bool small = true;
                if (work) {
                    for (int i = 0; i < NORB; ++i)
                        if (i != j && !abs_lt(m.A[j * LD + i], JACOBI_TOL)) small = false;
                }
                if (__all_sync(CAVMD_FULL_MASK, small)) break;
                if (sweep >= cap) {
                    if (cold_first && work && !small) m.flag |= ERRBIT_TIMEOUT;
                    break;
                }
                for (int rd = 0; rd < NORB - 1; ++rd) {
                    int slot = 0;
                    const int pj = rr_partner(j, rd, NORB, slot);
                    const int p = min(j, pj), q = max(j, pj);
                    double c = 1.0, s = 0.0;
                    double na[NORB], nc[NORB];
                    if (work) {
                        jacobi_cs(m.A[p * LD + p], m.A[q * LD + q], m.A[q * LD + p], c, s);
                        const double cp = (j == p) ? c : s;       // new col j = cp * col p + cq * col q
                        const double cq = (j == p) ? -s : c;
#pragma unroll
                        for (int i = 0; i < NORB; ++i) {
                            na[i] = fma(cp, m.A[p * LD + i], cq * m.A[q * LD + i]);
                            nc[i] = fma(cp, m.C[p * LD + i], cq * m.C[q * LD + i]);
                        }
                    }
                    __syncwarp();
                    if (work) {
#pragma unroll
                        for (int i = 0; i < NORB; ++i) {
                            m.A[j * LD + i] = na[i];
                            m.C[j * LD + i] = nc[i];
                        }
                        if (j == p) {
                            m.cs[slot][0] = c;
                            m.cs[slot][1] = s;
                        }
                    }
                    __syncwarp();
                    if (work) {
#pragma unroll
                        for (int k = 0; k < NORB / 2; ++k) {
                            int pk, qk;
                            rr_pair(k, rd, NORB, pk, qk);
                            const double ck = m.cs[k][0], sk_ = m.cs[k][1];
                            const double x = m.A[j * LD + pk], y = m.A[j * LD + qk];
                            m.A[j * LD + pk] = fma(ck, x, -sk_ * y);
                            m.A[j * LD + qk] = fma(sk_, x, ck * y);
                        }
                    }
                    __syncwarp();
                }
            }
            if (work) {   // occupation after the sweeps
                const long long kj = order_key(m.A[j * LD + j]);
                int rank = 0;
                for (int i = 0; i < NORB; ++i) {
                    const long long ki = order_key(m.A[i * LD + i]);
                    rank += (ki < kj) || (ki == kj && i < j);
                }
                m.occf[j] = rank < m.nocc;
                if (rank < m.nocc) m.occ_list[rank] = j;
            }
            __syncwarp();
        }

        if (work) {   // P = 2 C_occ C_occ^T, column j, and (P S)_jj
            double pc[NORB];
#pragma unroll
            for (int i = 0; i < NORB; ++i) pc[i] = 0.0;
            for (int o = 0; o < m.nocc; ++o) {
                const int col = m.occ_list[o];
                const double w = 2.0 * m.C[col * LD + j];
#pragma unroll
                for (int i = 0; i < NORB; ++i) pc[i] = fma(w, m.C[col * LD + i], pc[i]);
            }
            double qo = 0.0;
#pragma unroll
            for (int i = 0; i < NORB; ++i) {
                m.P[j * LD + i] = pc[i];
                qo = fma(pc[i], m.S[j * LD + i], qo);
            }
            m.red[j] = qo;
        }
        __syncwarp();
        const int hs = (it - 1) % NHIST;
        if (work && j < NAT) {
            double qa = 0.0;
            for (int o = m.atom_off[j]; o < m.atom_off[j + 1]; ++o) qa += m.red[o];
            m.qout[j] = qa;
            m.hq[hs][j] = m.q[j];
            m.hf[hs][j] = qa - m.q[j];
        }
        __syncwarp();
        if (work) {
            // convergence test and Anderson coefficients (FP32: they only steer the iteration)
            bool conv = true;
            for (int at = 0; at < NAT; ++at)
                if (!abs_lt(m.hf[hs][at], a.scc_tol)) conv = false;
            for (int c = 0; c < NORB; ++c) conv = conv && m.eok[c];
            float th1 = 0.0f, th2 = 0.0f;
            const int h = min(it, NHIST);
            if (!conv && h >= 2) {
                const int h1 = (hs + NHIST - 1) % NHIST, h2 = (hs + NHIST - 2) % NHIST;
                float a11 = 0.f, a12 = 0.f, a22 = 0.f, b1 = 0.f, b2 = 0.f;
                for (int at = 0; at < NAT; ++at) {
                    const float f0 = d2f_steer(m.hf[hs][at]);
                    const float d1 = d2f_steer(m.hf[h1][at]) - f0;
                    const float d2 = h >= 3 ? d2f_steer(m.hf[h2][at]) - f0 : 0.f;
                    a11 = fmaf(d1, d1, a11);
                    a12 = fmaf(d1, d2, a12);
                    a22 = fmaf(d2, d2, a22);
                    b1 = fmaf(-d1, f0, b1);
                    b2 = fmaf(-d2, f0, b2);
                }
                const float det = a11 * a22 - a12 * a12;
                if (h >= 3 && det > 1e-6f * a11 * a22 && det > 0.f) {
                    th1 = (b1 * a22 - b2 * a12) / det;
                    th2 = (a11 * b2 - a12 * b1) / det;
                } else if (a11 > 0.f) {
                    th1 = b1 / a11;
                }
                if (!(fabsf(th1) < 50.f) || !(fabsf(th2) < 50.f)) { th1 = 0.f; th2 = 0.f; }
            }
            if (j < NAT) {
                if (conv) {
                    m.q[j] = m.qout[j];
                } else {
                    const int h1 = (hs + NHIST - 1) % NHIST, h2 = (hs + NHIST - 2) % NHIST;
                    const double t1 = f2d_steer(th1), t2 = f2d_steer(th2);
                    const double q0 = m.hq[hs][j], f0 = m.hf[hs][j];
                    double qb = q0, fb = f0;
                    if (h >= 2) { qb = fma(t1, m.hq[h1][j] - q0, qb); fb = fma(t1, m.hf[h1][j] - f0, fb); }
                    if (h >= 3) { qb = fma(t2, m.hq[h2][j] - q0, qb); fb = fma(t2, m.hf[h2][j] - f0, fb); }
                    m.q[j] = fma(a.beta, fb, qb);
                }
            }
            if (j == 0 && conv) {
                m.conv = 1;
                m.iters = it;
            }
        }
        __syncwarp();
        if (__all_sync(CAVMD_FULL_MASK, !act || m.conv)) break;
    }
    if (act && j == 0 && !m.conv) {
        m.flag |= ERRBIT_SCC_NOCONV;
        m.iters = a.max_iter;
    }
    __syncwarp();

    if (disp) {   // finite-difference row: only the dipole of the converged charges
        if (valid && j == 0) {
            double mu[3] = {0.0, 0.0, 0.0};
            for (int at = 0; at < NAT; ++at) {
                const double Q = m.zv[at] - m.q[at];
                for (int k = 0; k < 3; ++k) mu[k] = fma(Q, m.pos[at][k] - m.pos[0][k], mu[k]);
            }
            a.M_disp[(long long)(a.fd_central ? 6 : 3) * a0 + (ridx - cidx * a.n_disp)] =
                fma(a.pol0, mu[0], fma(a.pol1, mu[1], a.pol2 * mu[2]));
            if (m.flag) atomicOr(a.status, (unsigned)m.flag);
        }
        return;
    }
    // ---------------------------------------------------------------- energy, forces, dipole
    if (act && j < NAT) {
        double sh = 0.0;
        for (int k = 0; k < NAT; ++k) sh = fma(m.gam[j][k], m.q[k] - m.zv[k], sh);
        m.shift[j] = sh;
    }
    __syncwarp();
    // energy-weighted density W = 2 C_o (C_o^T H C_o) C_o^T with the H of the last iteration and the
    // whole occupied block (basis independent inside the occupied subspace)
    if (act) {   // Y = H C
        double y[NORB];
#pragma unroll
        for (int i = 0; i < NORB; ++i) y[i] = 0.0;
        for (int k = 0; k < NORB; ++k) {
            const double ckj = m.C[j * LD + k];
#pragma unroll
            for (int i = 0; i < NORB; ++i) y[i] = fma(m.Hs[k * LD + i], ckj, y[i]);
        }
#pragma unroll
        for (int i = 0; i < NORB; ++i) m.Y[j * LD + i] = y[i];
    }
    __syncwarp();
    if (act) {   // A = C^T Y
        double y[NORB];
        for (int i = 0; i < NORB; ++i) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < NORB; ++k) s = fma(m.C[i * LD + k], m.Y[j * LD + k], s);
            y[i] = s;
        }
        for (int i = 0; i < NORB; ++i) m.A[j * LD + i] = y[i];
    }
    __syncwarp();
    if (act) {   // W column j, band energy partial, HOMO-LUMO gap
        double t[NORB];
        for (int o = 0; o < m.nocc; ++o) {
            const int co = m.occ_list[o];
            double x = 0.0;
            for (int o2 = 0; o2 < m.nocc; ++o2) {
                const int c2 = m.occ_list[o2];
                x = fma(m.A[c2 * LD + co], m.C[c2 * LD + j], x);
            }
            t[o] = 2.0 * x;
        }
        double wc[NORB];
#pragma unroll
        for (int i = 0; i < NORB; ++i) wc[i] = 0.0;
        for (int o = 0; o < m.nocc; ++o) {
            const int co = m.occ_list[o];
            const double w = t[o];
#pragma unroll
            for (int i = 0; i < NORB; ++i) wc[i] = fma(w, m.C[co * LD + i], wc[i]);
        }
        double eb = 0.0;
#pragma unroll
        for (int i = 0; i < NORB; ++i) {
            m.Y[j * LD + i] = wc[i];
            eb = fma(m.P[j * LD + i], m.H0[j * LD + i], eb);
        }
        m.red[j] = eb;
        if (j == 0 && m.nocc < NORB) {
            double homo = -1e300, lumo = 1e300;
            for (int i = 0; i < NORB; ++i) {
                const double ei = m.A[i * LD + i];
                if (m.occf[i]) homo = fmax(homo, ei); else lumo = fmin(lumo, ei);
            }
            if (!(lumo - homo > MIN_GAP)) m.flag |= ERRBIT_ZERO_GAP;
        }
    }
    __syncwarp();
    if (act) {
        // one (pair, table) task per lane: the H0 part of a pair's gradient on one lane, its S
        // part (with the second-order and repulsion terms) on another; combined below
        for (int task = j; task < 2 * NPAIR; task += NORB) {
            const int pi = task % NPAIR, t = task / NPAIR;
            const int A = m.pa[pi], B = m.pb[pi];
            const int eA = m.spec[A], eB = m.spec[B];
            const int oA = m.atom_off[A], oB = m.atom_off[B];
            const int na = sk.norb[eA], nb = sk.norb[eB];
            const double dx = m.pos[B][0] - m.pos[A][0];
            const double dy = m.pos[B][1] - m.pos[A][1];
            const double dz = m.pos[B][2] - m.pos[A][2];
            const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
            const double ir = rsqrt_nr(r2);
            const double r = r2 * ir;
            const double e[3] = {dx * ir, dy * ir, dz * ir};
            const double hshift = 0.5 * (m.shift[A] + m.shift[B]);
            double gk[3] = {0.0, 0.0, 0.0};
            {
                const double (*tab)[CAVMD_MAX_ELEM][4][4] = t == 0 ? sk.h0 : sk.s;
                // weights of the (A, B) block: P for H0, P (eps_A + eps_B)/2 - W for S
                auto wt = [&](int mu, int nu) -> double {
                    const double pv = m.P[nu * LD + mu];
                    return t == 0 ? pv : fma(pv, hshift, -m.Y[nu * LD + mu]);
                };
                double v, dv;
                radial(tab[eA][eB][CAVMD_SK_SS], r, sk, v, dv);
                {
                    const double w = wt(oA, oB) * dv;
                    for (int k = 0; k < 3; ++k) gk[k] = fma(w, e[k], gk[k]);
                }
                if (nb == 4) {
                    radial(tab[eA][eB][CAVMD_SK_SP], r, sk, v, dv);
                    double w[3], we = 0.0;
                    for (int i = 0; i < 3; ++i) { w[i] = wt(oA, oB + 1 + i); we = fma(w[i], e[i], we); }
                    for (int k = 0; k < 3; ++k)
                        gk[k] += fma(w[k] - we * e[k], v * ir, we * e[k] * dv);
                }
                if (na == 4) {
                    radial(tab[eB][eA][CAVMD_SK_SP], r, sk, v, dv);
                    double w[3], we = 0.0;
                    for (int i = 0; i < 3; ++i) { w[i] = wt(oA + 1 + i, oB); we = fma(w[i], e[i], we); }
                    for (int k = 0; k < 3; ++k)
                        gk[k] -= fma(w[k] - we * e[k], v * ir, we * e[k] * dv);
                }
                if (na == 4 && nb == 4) {
                    double vs, dvs, vp, dvp;
                    radial(tab[eA][eB][CAVMD_SK_PPS], r, sk, vs, dvs);
                    radial(tab[eA][eB][CAVMD_SK_PPP], r, sk, vp, dvp);
                    double Wm[3][3], We[3] = {0, 0, 0}, WTe[3] = {0, 0, 0}, tr = 0.0;
                    for (int i = 0; i < 3; ++i)
                        for (int k = 0; k < 3; ++k) Wm[i][k] = wt(oA + 1 + i, oB + 1 + k);
                    for (int i = 0; i < 3; ++i) {
                        tr += Wm[i][i];
                        for (int k = 0; k < 3; ++k) {
                            We[i] = fma(Wm[i][k], e[k], We[i]);
                            WTe[k] = fma(Wm[i][k], e[i], WTe[k]);
                        }
                    }
                    double eWe = 0.0;
                    for (int i = 0; i < 3; ++i) eWe = fma(e[i], We[i], eWe);
                    const double dl = vs - vp, ddl = dvs - dvp;
                    for (int k = 0; k < 3; ++k)
                        gk[k] += (We[k] + WTe[k] - 2.0 * eWe * e[k]) * dl * ir + eWe * e[k] * ddl +
                                 tr * e[k] * dvp;
                }
            }
            for (int k = 0; k < 3; ++k) m.gpart[t][pi][k] = gk[k];
            if (t == 1) {
                // second-order charge term and pair repulsion
                const double gi = rsqrt_nr(fma(r, r, sk.gamma_c2[eA][eB]));
                const double dgam = -r * gi * gi * gi;
                const double qq = (m.q[A] - m.zv[A]) * (m.q[B] - m.zv[B]) * dgam;
                const double arep = sk.rep[eA][eB][0], brep = sk.rep[eA][eB][1];
                double erep = 0.0, derep = 0.0;
                if (arep != 0.0) {
                    const double vr = arep * exp(-brep * r);
                    const double x = (r - (sk.r_cut - sk.taper)) * sk.inv_taper;
                    double f = 1.0, df = 0.0;
                    if (x > 0.0) {
                        if (x < 1.0) {
                            double sn, cn;
                            sincospi(x, &sn, &cn);
                            f = 0.5 * (1.0 + cn);
                            df = -0.5 * 3.141592653589793 * sk.inv_taper * sn;
                        } else {
                            f = 0.0;
                        }
                    }
                    erep = vr * f;
                    derep = vr * (df - brep * f);
                }
                for (int k = 0; k < 3; ++k) m.gpair[pi][k] = (qq + derep) * e[k];
                m.epair[pi] = erep;
            }
        }
    }
    __syncwarp();
    if (act && j < NPAIR)
        for (int k = 0; k < 3; ++k) m.gpair[j][k] = fma(2.0, m.gpart[0][j][k] + m.gpart[1][j][k], m.gpair[j][k]);
    __syncwarp();
    if (valid && j < NAT) {
        double f[3] = {0.0, 0.0, 0.0};
        for (int pi = 0; pi < NPAIR; ++pi) {
            const double sg = (m.pb[pi] == j) ? -1.0 : ((m.pa[pi] == j) ? 1.0 : 0.0);
            for (int k = 0; k < 3; ++k) f[k] = fma(sg, m.gpair[pi][k], f[k]);
        }
        const int at = a0 + j;
        for (int k = 0; k < 3; ++k) a.F[3 * at + k] = f[k];
        a.qprev[at] = a.have_warm ? m.qstart[j] : m.q[j];
        a.qpop[at] = m.q[j];
        if (a.Qout) a.Qout[at] = m.zv[j] - m.q[j];
        if (a.write_b) {
            const double Q = m.zv[j] - m.q[j];
            a.b[3 * at + 0] = Q * a.pol0;
            a.b[3 * at + 1] = Q * a.pol1;
            a.b[3 * at + 2] = Q * a.pol2;
        }
    }
    if (valid) {
        double *cw = a.Cwarm + (a.Cwarm_off ? a.Cwarm_off[cell] : (long long)cell * NORB * NORB);
        for (int i = 0; i < NORB; ++i) cw[j * NORB + i] = m.C[j * LD + i];
    }
    if (valid && j == 0) {
        double E = 0.0;
        for (int i = 0; i < NORB; ++i) E += m.red[i];
        double e2 = 0.0;
        for (int x = 0; x < NAT; ++x)
            for (int y = 0; y < NAT; ++y)
                e2 = fma(m.gam[x][y] * (m.q[x] - m.zv[x]), m.q[y] - m.zv[y], e2);
        E = fma(0.5, e2, E);
        for (int pi = 0; pi < NPAIR; ++pi) E += m.epair[pi];
        double mu[3] = {0.0, 0.0, 0.0};
        for (int at = 0; at < NAT; ++at) {
            const double Q = m.zv[at] - m.q[at];
            for (int k = 0; k < 3; ++k) mu[k] = fma(Q, m.pos[at][k] - m.pos[0][k], mu[k]);
        }
        a.E_cell[cell] = E;
        a.M_cell[cell] = fma(a.pol0, mu[0], fma(a.pol1, mu[1], a.pol2 * mu[2]));
        a.iters[cell] = m.iters;
        if (m.flag) atomicOr(a.status, (unsigned)m.flag);
    }
}

__global__ void k_born_assemble(int n_cells, const int *__restrict__ off, const double *__restrict__ M0,
                                const double *__restrict__ Md, int nd, int central, double h,
                                double *__restrict__ b) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_cells) return;
    const double ih = 1.0 / h;
    const double *md = Md + (size_t)(central ? 6 : 3) * off[n];
    for (int j = off[n]; j < off[n + 1]; ++j) {
        const int jl = j - off[n];
        for (int k = 0; k < 3; ++k) {
            const int r = 3 * jl + k;
            b[3 * j + k] = central ? (md[2 * r] - md[2 * r + 1]) * (0.5 * ih) : (md[r] - M0[n]) * ih;
        }
    }
}

}  // namespace

cudaError_t launch_born_assemble(int n_cells, const int *cell_offset, const double *M_cell,
                                 const double *M_disp, int n_disp, int central, double h, double *b,
                                 cudaStream_t st) {
    k_born_assemble<<<(n_cells + 127) / 128, 128, 0, st>>>(n_cells, cell_offset, M_cell, M_disp, n_disp,
                                                           central, h, b);
    return cudaGetLastError();
}

// warps per block (2, 4 or 8) and waters per warp (1..5). The warps per block never change a result;
// the waters per warp do at rounding level, because the choice between a Jacobi sweep and the
// second-order update is taken per warp.
cudaError_t launch_dftb_water(const DevSK *sk, const DftbArgs &a, cudaStream_t st, int warps, int per_warp) {
    constexpr int NAT = 3, NORB = 6;
    using SM = MolShared<NAT, NORB>;
    const int gpw = per_warp < 1 ? 1 : (per_warp > 32 / NORB ? 32 / NORB : per_warp);
    const int threads = 32 * warps;
    const int per_block = warps * gpw;
    const long long rows = (long long)a.n_cells * (a.n_disp > 0 ? a.n_disp : 1);
    const int blocks = (int)((rows + per_block - 1) / per_block);
    const size_t smem = sizeof(SM) * per_block;
    if (a.n_cells <= 0) return cudaSuccess;
    dftb_kernel<NAT, NORB><<<blocks, threads, smem, st>>>(sk, a, gpw);
    return cudaGetLastError();
}

cudaError_t prepare_dftb_water(int max_warps) {
    using SM = MolShared<3, 6>;
    return cudaFuncSetAttribute(dftb_kernel<3, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(SM) * max_warps * 5));
}
