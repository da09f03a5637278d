// Batched Gamma-point SCC-DFTB of periodic cells: the paper's per-molecule systems are cubic cells
// of 33 waters with periodic boundaries in all three directions and Gamma-point sampling (section
// "Computational details").
//
// What is computed (the textbook Gamma-point forms):
//   * H0 and S: the (A, B) block is the sum over lattice images T of the Slater-Koster block at
//     d = r_B + T - r_A, |d| < r_cut (for A = B the T = 0 term is the on-site block);
//   * gamma: Ewald lattice sum of 1/r (tin-foil boundary, neutralising background) plus the
//     Klopman-Ohno remainder 1/sqrt(r^2 + c^2) - 1/r over images with the cosine taper at r_cut,
//     and U_A on the diagonal. The real-space part is a matrix formed once per evaluation; the
//     reciprocal part acts on the charges through structure factors in every SCC iteration;
//   * the SCC loop, band + second-order + repulsion energy and its analytic gradient, every term
//     summed over the same images.
//
// Mapping to the machine. A 33-water cell has 198 orbitals: one 198 x 198 FP64 matrix is 313 KB,
// more than a block's shared memory, and GB300's FP64 pipe (2 FMA per clock per SM) is the only
// bottleneck. So each cell is one 256-thread block of a persistent grid (two per SM), its
// matrices live in a per-block global workspace (L2-resident while the cell runs), and every
// product stages k-chunks of its operands in shared memory and spreads its output entries
// evenly over the threads (8 per thread per pass, each summed over k in increasing order), so the
// results do not depend on the launch shape. Per SCC iteration only what the update needs is
// formed: H, Y = H C, the diagonal and the occupied-virtual block of C^T Y, and a rotation by the
// occupied-virtual generator K(v, o) = A_vo / (A_oo - A_vv): while some entry of K is 1e-4 or
// more, the Cayley rotation C <- C (I - K/2)^-1 (I + K/2), orthogonal to rounding for any K (two
// small Cholesky factorisations, I + X^T X / 4 and I + X X^T / 4, X = K_vo, and row solves);
// below that, C <- C (I + K + K^2/2), orthogonal to O(K^4), as two staged products. A cold start
// diagonalises C^T H C once by cyclic Jacobi sweeps; warm starts re-orthonormalise the previous
// step's C under the new overlap by a Cholesky factor of C^T S C, and their first iteration runs
// one Jacobi sweep inside the occupied and inside the virtual block: the diagonal denominators
// need those blocks nearly diagonal, and without the sweeps their off-diagonal part grows (a cold
// start leaves it large, then it drifts with every step; its norm over 132 nearly degenerate
// occupied orbitals reaches the gap) and the iteration count with it.
#include <algorithm>
#include <cmath>
#include <vector>

#include "cavmd_internal.cuh"

namespace {

constexpr int PT = 256;          // threads per block (one cell at a time)
constexpr int PE = 8;            // product entries per thread per pass
constexpr int KC = 24;           // contraction chunk staged in shared memory
constexpr int ZC = 80;           // columns of the second operand staged per pass
constexpr int PNMAX = 256;       // orbitals per cell
constexpr int PAMAX = 128;       // atoms per cell
constexpr int PHIST = 6;         // largest Anderson history
constexpr int P_MAX_SWEEPS = 40;   // default bound on the Jacobi sweeps of a cold start
constexpr double P_JACOBI_TOL = 1e-11;   // cold start: off-diagonal size where the sweeps stop
constexpr double P_MIN_GAP = 1e-3;
constexpr double P_EIG_TOL = 1e-10;
constexpr float P_KMAX_PERT = 1e-4f;      // generator size below which C (I + K + K^2/2) is used
constexpr int P_SWEEP_PERIOD = 1;         // warm steps between within-block Jacobi sweeps (every fourth
                                          // step measured slower: 13.6 SCC iterations instead of 11.9)
constexpr int P_SWEEP_ITERS = 12;         // or after an evaluation with more SCC iterations than this
constexpr double PI_D = 3.141592653589793;

// Shared memory of one block; PN is the largest problem dimension (the orbitals of a cell at the
// Gamma point, twice that for the real form of a complex k-point problem).
template <int PN>
struct PSharedT {
    double Xs[KC * PN];
    double Zs[KC * ZC];
    double pos[PAMAX][3];
    double zv[PAMAX], q[PAMAX], qout[PAMAX], qst[PAMAX], dq[PAMAX], shift[PAMAX];
    double hq[PHIST][PAMAX], hf[PHIST][PAMAX];
    double diag[PN], red[PN], invd[PN];
    double cs[PN];               // Jacobi (c, s) of the rotations of one round
    double qk[PNMAX];            // k-grid: populations summed over the k-points of one iteration
    double hl[2];                // k-grid: highest occupied and lowest empty level over the k-points
    double th[PHIST];
    double gred[PT / 32][3];
    int spec[PAMAX], atom_off[PAMAX + 1], orb_atom[PNMAX];
    int occ_list[PN], virt_list[PN], occf[PN];
    int pp[PN / 2], pq[PN / 2];
    int fl[8];                   // 0 error bits, 1 n, 2 iterations, 3 occupied orbitals
    int vote[PT / 32];
};
using PShared = PSharedT<PNMAX>;
using PSharedK = PSharedT<2 * PNMAX>;

__device__ __forceinline__ bool blk_all(bool p) { return __syncthreads_and(p) != 0; }

__device__ __forceinline__ void cutoff_fn(double r, const DevSK &sk, double &f, double &df) {
    const double x = (r - (sk.r_cut - sk.taper)) * sk.inv_taper;
    f = 1.0;
    df = 0.0;
    if (x > 0.0) {
        if (x < 1.0) {
            double sn, cn;
            sincospi(x, &sn, &cn);
            f = 0.5 * (1.0 + cn);
            df = -0.5 * PI_D * sk.inv_taper * sn;
        } else {
            f = 0.0;
        }
    }
}

// V(r) = a exp(-b r) (1 + c1 r + c2 r^2) f_cut(r) and dV/dr.
__device__ __forceinline__ void radial_p(const double *par, double r, const DevSK &sk, double &v, double &dv) {
    const double a = par[0], b = par[1], c1 = par[2], c2 = par[3];
    const double e = a * exp(-b * r);
    const double poly = fma(fma(c2, r, c1), r, 1.0);
    const double dpoly = fma(2.0 * c2, r, c1);
    double f, df;
    cutoff_fn(r, sk, f, df);
    v = e * poly * f;
    dv = e * (fma(-b * poly, f, dpoly * f) + poly * df);
}

// Column of entry e of the packed lower triangle of an m x m matrix, stored column by column
// (column c holds rows c..m-1 and starts at c m - c (c - 1) / 2).
__device__ __forceinline__ int lower_col(int e, int m) {
    const float b = 2.0f * (float)m + 1.0f;
    int c = (int)((b - sqrtf(fmaxf(b * b - 8.0f * (float)e, 0.0f))) * 0.5f);
    c = max(0, min(c, m - 1));
    while (c > 0 && c * m - c * (c - 1) / 2 > e) --c;
    while (c + 1 < m && (c + 1) * m - (c + 1) * c / 2 <= e) ++c;
    return c;
}

// Block-wide product: out(i, c) = sum_{k < K} xa(i, k) za(k, c) for the entries of an m x w
// matrix (LOWER: the entries i >= c of an m x m one), the sum taken in increasing k; epi(i, c, v)
// receives each entry once. Passes of up to PT * PE entries in column order; each k-chunk of the
// m rows of X and of the pass's columns of Z is staged in shared memory first.
// XK: consecutive k of X are adjacent in memory (else consecutive i); ZK: consecutive k of Z are
// adjacent (else consecutive c). They only choose the staging order, for coalesced loads.
template <bool LOWER, bool XK, bool ZK, class SH, class XA, class ZA, class EPI>
__device__ void pprod(SH &sh, int m, int w, int K, XA xa, ZA za, EPI epi) {
    const int tid = threadIdx.x;
    const int n_out = LOWER ? m * (m + 1) / 2 : m * w;
    const int pe = LOWER ? PT * PE : min(PT * PE, m * (ZC - 2));
    for (int e0 = 0; e0 < n_out; e0 += pe) {
        const int e1 = min(e0 + pe, n_out);
        const int c_lo = LOWER ? lower_col(e0, m) : e0 / m;
        const int c_hi = LOWER ? lower_col(e1 - 1, m) : (e1 - 1) / m;
        const int ncol = c_hi - c_lo + 1;
        int ii[PE], cc[PE];
        double acc[PE];
#pragma unroll
        for (int r = 0; r < PE; ++r) {
            const int e = min(e0 + tid + r * PT, e1 - 1);
            int i, c;
            if (LOWER) {
                c = lower_col(e, m);
                i = c + (e - (c * m - c * (c - 1) / 2));
            } else {
                c = e / m;
                i = e - c * m;
            }
            ii[r] = i;
            cc[r] = c - c_lo;
            acc[r] = 0.0;
        }
        for (int k0 = 0; k0 < K; k0 += KC) {
            const int kc = min(KC, K - k0);
            __syncthreads();
            for (int idx = tid; idx < kc * m; idx += PT) {
                int kk, i;
                if (XK) { i = idx / kc; kk = idx - i * kc; } else { kk = idx / m; i = idx - kk * m; }
                sh.Xs[kk * m + i] = xa(i, k0 + kk);
            }
            for (int idx = tid; idx < kc * ncol; idx += PT) {
                int kk, cl;
                if (ZK) { cl = idx / kc; kk = idx - cl * kc; } else { kk = idx / ncol; cl = idx - kk * ncol; }
                sh.Zs[kk * ZC + cl] = za(k0 + kk, c_lo + cl);
            }
            __syncthreads();
            for (int kk = 0; kk < kc; ++kk) {
#pragma unroll
                for (int r = 0; r < PE; ++r) acc[r] = fma(sh.Xs[kk * m + ii[r]], sh.Zs[kk * ZC + cc[r]], acc[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < PE; ++r)
            if (e0 + tid + r * PT < e1) epi(ii[r], cc[r] + c_lo, acc[r]);
    }
    __syncthreads();
}

// In-place lower Cholesky factor of the m x m matrix A (column-major, leading dimension m; the
// lower triangle is read and written), right-looking with one thread per trailing column.
// Returns false (in every thread) when a pivot is not positive.
template <class SH>
__device__ bool pchol(double *A, int m, SH &sh) {
    const int j = threadIdx.x;
    if (j == 0) sh.fl[4] = 0;
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        if (j == 0) {
            double d = A[k * m + k];
            if (!(d > 1e-300)) { sh.fl[4] = 1; d = 1.0; }
            const double y = rsqrt_nr(d);
            sh.invd[k] = y;
            A[k * m + k] = d * y;
        }
        __syncthreads();
        const double y = sh.invd[k];
        for (int i = k + 1 + j; i < m; i += PT) A[k * m + i] *= y;
        __syncthreads();
        for (int jj = k + 1 + j; jj < m; jj += PT) {
            const double ljk = A[k * m + jj];
            for (int i = jj; i < m; ++i) A[jj * m + i] = fma(-A[k * m + i], ljk, A[jj * m + i]);
        }
        __syncthreads();
    }
    const bool ok = sh.fl[4] == 0;
    __syncthreads();
    return ok;
}

// Row solve x L^T = z (forward substitution) for one row of length m with stride xs, in place.
__device__ __forceinline__ void row_solve_lt(const double *L, int m, const double *invd, double *x, int xs) {
    for (int c = 0; c < m; ++c) {
        double v = x[c * xs];
        for (int k = 0; k < c; ++k) v = fma(-x[k * xs], L[k * m + c], v);
        x[c * xs] = v * invd[c];
    }
}

// Row solve x L L^T = z for one row (z, x of length m, strides zs and xs), L the lower factor
// above: forward u L^T = z, then backward x L = u. x may alias z.
__device__ __forceinline__ void row_solve_llt(const double *L, int m, const double *invd, const double *z, int zs,
                                              double *x, int xs) {
    for (int c = 0; c < m; ++c) {   // u_c = (z_c - sum_{k<c} u_k L(c, k)) / L(c, c)
        double v = z[c * zs];
        for (int k = 0; k < c; ++k) v = fma(-x[k * xs], L[k * m + c], v);
        x[c * xs] = v * invd[c];
    }
    for (int c = m - 1; c >= 0; --c) {   // x_c = (u_c - sum_{k>c} x_k L(k, c)) / L(c, c)
        double v = x[c * xs];
        for (int k = c + 1; k < m; ++k) v = fma(-x[k * xs], L[c * m + k], v);
        x[c * xs] = v * invd[c];
    }
}

// Round-robin Jacobi schedule for even n: pair k of round r (0..n-2); index n-1 meets r.
__device__ __forceinline__ void p_pair(int k, int r, int n, int &p, int &q) {
    const int m = n - 1;
    if (k == 0) { p = r; q = m; return; }
    const int x = (r + k) % m, y = (r - k + m) % m;
    p = min(x, y);
    q = max(x, y);
}

// Rotation annihilating a_pq: angle from FP32, (c, s) normalised in FP64 by two Newton steps.
__device__ __forceinline__ void p_jacobi_cs(double app, double aqq, double apq, double &c, double &s) {
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


// Device view of the periodic plan (by value).
struct PbcDev {
    double lat[9], inv[9];       // lattice vectors as rows; fractional coordinates f = r inv
    double alpha, bg, self_e;    // Ewald alpha, -pi / (alpha^2 V), -2 alpha / sqrt(pi)
    double r_real2;              // real-space cutoff squared
    int n_img, n_img_sk, n_g, nmax, amax;
    const double *img;           // [n_img][3] lattice translations by increasing length; the first
                                 // n_img_sk reach every image within r_cut
    const double *gw;            // [n_g][4] half-space reciprocal vectors G and 2 w_G
    double *work;                // per-block workspaces
    long long work_stride;       // doubles per block
    int nk;                      // k-grid: irreducible k-points (0: Gamma-point kernel)
    const double *kpt;           // [nk][4] fractional k (units of the reciprocal rows) and weight
};

// One cell, evaluated by the whole block.
// One cell, or (disp_k >= 0) one finite-difference copy of it: atom disp_k / 3 (central: disp_k / 6)
// moved along x, y or z by +h (central: +h and -h in turn), warm started from the cell's converged
// basis in a private copy, and only its dipole written (M_disp, the layout of the water kernels).
//
// KG: the cell sampled on a k-grid (the paper's Gamma point of a folded supercell). Each k-point of
// the irreducible list (k and -k give complex-conjugate problems) is a complex Hermitian problem
// H(k) c = e S(k) c, H(k)_{mu nu} = sum_T exp(i 2 pi f_k . n_T) h_{mu nu}(r_B + T - r_A), solved in its
// real form of twice the size, [[Re, -Im], [Im, Re]] (every level appears twice, so twice the
// occupied count is occupied): the same products, factorisations, sweeps and rotations as the
// Gamma point. The SCC iteration runs every k-point's update in turn and joins the populations,
// sum_k w_k Re (P(k) S(k)*)_{mu mu}, before the mixing; the band energy is sum_k w_k Re Tr P(k) H0(k)*
// and the forces use the real-space densities rho(T) = sum_k w_k Re[P(k)_{nu mu} exp(i 2 pi f_k . n_T)]
// (and the same for the energy-weighted density) image by image.
template <bool DISP, bool KG, class SH>
__device__ void p_cell(const DevSK &sk, const DftbArgs &a, const PbcDev &pl, SH &sh, double *wk, int cell,
                       int disp_k) {
    const int j = threadIdx.x;
    const int a0 = a.cell_offset[cell];
    const int nat = a.cell_offset[cell + 1] - a0;
    const long long n2max = (KG ? 4LL : 1LL) * pl.nmax * pl.nmax;   // one problem matrix
    constexpr bool disp = DISP;
    const int NKP = KG ? pl.nk : 1;
    // Gamma: [H0][S][H][Y][P][Xg][Mo][Mv]; KG: [H][Y][P][Xg][Mo][Mv] and then H0(k), S(k) of every k
    double *H0 = wk, *S = wk + n2max;
    double *H = wk + (KG ? 0 : 2) * n2max, *Y = H + n2max, *P = H + 2 * n2max;
    double *Xg = H + 3 * n2max, *Mo = H + 4 * n2max, *Mv = H + 5 * n2max;
    double *const kbase = wk + 6 * n2max;
    double *gam = wk + (KG ? 6 + 2LL * NKP : 8) * n2max;
    double *csg = gam + (long long)pl.amax * pl.amax;     // [g][atom] (cos, sin)
    double *sgf = csg + 2LL * pl.amax * pl.n_g;           // [g] (S_c, S_s)
    double *pbuf = sgf + 2LL * pl.n_g;                    // [atom * nat + atom] gradient (3) + energy
    double *const C0 = a.Cwarm + a.Cwarm_off[cell];
    double *C = C0;

    if (j < nat) {
        sh.spec[j] = a.species[a0 + j];
        for (int k = 0; k < 3; ++k) sh.pos[j][k] = a.r[3 * (a0 + j) + k];
        if (disp) {
            const int kk = a.fd_central ? disp_k >> 1 : disp_k;
            const double sg = (a.fd_central && (disp_k & 1)) ? -1.0 : 1.0;
            if (j == kk / 3) sh.pos[j][kk % 3] += sg * a.fd_h;
        }
    }
    __syncthreads();
    if (j == 0) {
        int o = 0;
        double nel = 0.0;
        for (int at = 0; at < nat; ++at) {
            sh.atom_off[at] = o;
            const int no = sk.norb[sh.spec[at]];
            for (int k = 0; k < no; ++k) sh.orb_atom[o + k] = at;
            o += no;
            sh.zv[at] = sk.zval[sh.spec[at]];
            nel += sh.zv[at];
        }
        sh.atom_off[nat] = o;
        sh.fl[0] = 0;
        sh.fl[1] = o;
        sh.fl[2] = 0;
        sh.fl[3] = (int)(nel * 0.5 + 0.25);
    }
    __syncthreads();
    const int n = sh.fl[1], nocc = sh.fl[3];
    const int nv = n - nocc, nn = n * n;
    // the problem: orbitals (Gamma), or the real form of a k-point problem (KG)
    const int m = KG ? 2 * n : n, mo = KG ? 2 * nocc : nocc, mv = m - mo, mm = m * m;
    double *Cb = C0;   // the bases of the k-points, mm apart
    if (disp) {   // a private copy of the cell's basis: the cell and its other copies read the original
        double *Cd = pbuf + 4LL * pl.amax * pl.amax;
        for (long long e = j; e < (long long)NKP * mm; e += PT) Cd[e] = C0[e];
        Cb = Cd;
        C = Cd;
        __syncthreads();
    }
    // point the problem's matrices at k-point kp
    auto set_k = [&](int kp) {
        if (KG) {
            H0 = kbase + 2LL * kp * n2max;
            S = H0 + n2max;
            C = Cb + (long long)kp * mm;
        }
    };

    // ---------------------------------------------------------------- H0, S, real-space gamma
    if constexpr (KG) {
        // every k-point: H0(k), S(k) in real form; gamma (k-independent) with the first k-point
        const double rc2 = sk.r_cut * sk.r_cut;
        for (int kp = 0; kp < NKP; ++kp) {
            set_k(kp);
            const bool first = kp == 0;
            const double fk[3] = {pl.kpt[4 * kp], pl.kpt[4 * kp + 1], pl.kpt[4 * kp + 2]};
            for (int e = j; e < mm; e += PT) {
                const int c = e / m, i = e - c * m;
                double h = 0.0, s = 0.0;
                if (i == c) {
                    const int io = i < n ? i : i - n;
                    const int at = sh.orb_atom[io], el = sh.spec[at];
                    h = (io == sh.atom_off[at]) ? sk.onsite[el][0] : sk.onsite[el][1];
                    s = 1.0;
                }
                H0[e] = h;
                S[e] = s;
            }
            __syncthreads();
            for (int t = j; t < nat * (nat + 1) / 2; t += PT) {   // pairs A <= B, packed by A
                const int A = lower_col(t, nat), B = A + (t - (A * nat - A * (A - 1) / 2));
                const int eA = sh.spec[A], eB = sh.spec[B];
                const int oA = sh.atom_off[A], oB = sh.atom_off[B];
                const int na = sk.norb[eA], nb = sk.norb[eB];
                double d[3], f[3], dw[3];
                for (int k = 0; k < 3; ++k) d[k] = sh.pos[B][k] - sh.pos[A][k];
                for (int k = 0; k < 3; ++k) f[k] = rint(fma(d[0], pl.inv[k], fma(d[1], pl.inv[3 + k], d[2] * pl.inv[6 + k])));
                for (int k = 0; k < 3; ++k) dw[k] = d[k] - fma(f[0], pl.lat[k], fma(f[1], pl.lat[3 + k], f[2] * pl.lat[6 + k]));
                double hr[16], hi[16], sr[16], si[16];
                for (int u = 0; u < 16; ++u) { hr[u] = 0.0; hi[u] = 0.0; sr[u] = 0.0; si[u] = 0.0; }
                double g_re = 0.0, g_sr = 0.0;
                const double c2 = sk.gamma_c2[eA][eB];
                if (first) {
                    for (int im = 0; im < pl.n_img; ++im) {   // real-space Ewald sum
                        const double x0 = dw[0] + pl.img[3 * im], x1 = dw[1] + pl.img[3 * im + 1], x2 = dw[2] + pl.img[3 * im + 2];
                        const double r2 = fma(x0, x0, fma(x1, x1, x2 * x2));
                        if (!(r2 < pl.r_real2) || r2 == 0.0) continue;
                        const double ir = rsqrt_nr(r2);
                        g_re = fma(erfc(pl.alpha * (r2 * ir)), ir, g_re);
                    }
                }
                for (int im = 0; im < pl.n_img_sk; ++im) {   // images within r_cut
                    const double x0 = dw[0] + pl.img[3 * im], x1 = dw[1] + pl.img[3 * im + 1], x2 = dw[2] + pl.img[3 * im + 2];
                    const double r2 = fma(x0, x0, fma(x1, x1, x2 * x2));
                    if (!(r2 < rc2) || r2 == 0.0) continue;
                    const double ir = rsqrt_nr(r2);
                    const double r = r2 * ir;
                    const double e[3] = {x0 * ir, x1 * ir, x2 * ir};
                    // the image's translation n_T = (its lattice coordinates) - f, and its phase
                    double ph = 0.0;
                    for (int k = 0; k < 3; ++k) {
                        const double nk_ = rint(fma(pl.img[3 * im], pl.inv[k], fma(pl.img[3 * im + 1], pl.inv[3 + k],
                                                                                     pl.img[3 * im + 2] * pl.inv[6 + k]))) - f[k];
                        ph = fma(fk[k], nk_, ph);
                    }
                    double sn, cs;
                    sincospi(2.0 * ph, &sn, &cs);
                    for (int tb = 0; tb < 2; ++tb) {
                        const double(*tab)[CAVMD_MAX_ELEM][4][4] = tb == 0 ? sk.h0 : sk.s;
                        double blk[16];
                        for (int u = 0; u < 16; ++u) blk[u] = 0.0;
                        double v, dv;
                        radial_p(tab[eA][eB][CAVMD_SK_SS], r, sk, v, dv);
                        blk[0] = v;
                        if (nb == 4) {
                            radial_p(tab[eA][eB][CAVMD_SK_SP], r, sk, v, dv);
                            for (int i = 0; i < 3; ++i) blk[1 + i] = e[i] * v;
                        }
                        if (na == 4) {
                            radial_p(tab[eB][eA][CAVMD_SK_SP], r, sk, v, dv);
                            for (int i = 0; i < 3; ++i) blk[4 * (1 + i)] = -e[i] * v;
                        }
                        if (na == 4 && nb == 4) {
                            double vs, vp;
                            radial_p(tab[eA][eB][CAVMD_SK_PPS], r, sk, vs, dv);
                            radial_p(tab[eA][eB][CAVMD_SK_PPP], r, sk, vp, dv);
                            const double dl = vs - vp;
                            for (int i = 0; i < 3; ++i)
                                for (int k = 0; k < 3; ++k) blk[4 * (1 + i) + 1 + k] = fma(e[i] * e[k], dl, (i == k) ? vp : 0.0);
                        }
                        double *re = tb == 0 ? hr : sr, *imv = tb == 0 ? hi : si;
                        for (int u = 0; u < 16; ++u) {
                            re[u] = fma(cs, blk[u], re[u]);
                            imv[u] = fma(sn, blk[u], imv[u]);
                        }
                    }
                    if (first) {
                        double fc, dfc;
                        cutoff_fn(r, sk, fc, dfc);
                        g_sr = fma(rsqrt_nr(r2 + c2) - ir, fc, g_sr);
                    }
                }
                // complex block z (mu of A, nu of B) at row oA + mu, column oB + nu of [[Re, -Im], [Im, Re]],
                // and its Hermitian transpose; a block of an atom with its own images is Hermitian,
                // written as the mean of z and the conjugate transpose
                for (int mu = 0; mu < na; ++mu)
                    for (int nu = 0; nu < nb; ++nu) {
                        const int u = 4 * mu + nu, ut = 4 * nu + mu;
                        for (int tb = 0; tb < 2; ++tb) {
                            const double *re = tb == 0 ? hr : sr, *imv = tb == 0 ? hi : si;
                            double *M_ = tb == 0 ? H0 : S;
                            const double zr = A == B ? 0.5 * (re[u] + re[ut]) : re[u];
                            const double zi = A == B ? 0.5 * (imv[u] - imv[ut]) : imv[u];
                            const int row = oA + mu, col = oB + nu;
                            if (A == B) {
                                M_[(long long)col * m + row] += zr;
                                M_[(long long)(col + n) * m + row] -= zi;
                                M_[(long long)col * m + row + n] += zi;
                                M_[(long long)(col + n) * m + row + n] += zr;
                            } else {
                                M_[(long long)col * m + row] = zr;
                                M_[(long long)(col + n) * m + row] = -zi;
                                M_[(long long)col * m + row + n] = zi;
                                M_[(long long)(col + n) * m + row + n] = zr;
                                M_[(long long)row * m + col] = zr;
                                M_[(long long)(row + n) * m + col] = zi;
                                M_[(long long)row * m + col + n] = -zi;
                                M_[(long long)(row + n) * m + col + n] = zr;
                            }
                        }
                    }
                if (first) {
                    double gv = g_re + g_sr + pl.bg;
                    if (A == B) gv += sk.hubbard[eA] + pl.self_e;
                    gam[A * pl.amax + B] = gv;
                    gam[B * pl.amax + A] = gv;
                }
            }
            __syncthreads();
        }
    } else {
        for (int e = j; e < nn; e += PT) {
            const int c = e / n, i = e - c * n;
            double h = 0.0, s = 0.0;
            if (i == c) {
                const int at = sh.orb_atom[c], el = sh.spec[at];
                h = (c == sh.atom_off[at]) ? sk.onsite[el][0] : sk.onsite[el][1];
                s = 1.0;
            }
            H0[e] = h;
            S[e] = s;
        }
        __syncthreads();
        for (int t = j; t < nat * (nat + 1) / 2; t += PT) {   // pairs A <= B, packed by A
            const int A = lower_col(t, nat), B = A + (t - (A * nat - A * (A - 1) / 2));
            const int eA = sh.spec[A], eB = sh.spec[B];
            const int oA = sh.atom_off[A], oB = sh.atom_off[B];
            const int na = sk.norb[eA], nb = sk.norb[eB];
            double d[3], f[3], dw[3];
            for (int k = 0; k < 3; ++k) d[k] = sh.pos[B][k] - sh.pos[A][k];
            for (int k = 0; k < 3; ++k) f[k] = rint(fma(d[0], pl.inv[k], fma(d[1], pl.inv[3 + k], d[2] * pl.inv[6 + k])));
            for (int k = 0; k < 3; ++k) dw[k] = d[k] - fma(f[0], pl.lat[k], fma(f[1], pl.lat[3 + k], f[2] * pl.lat[6 + k]));
            double hb[16], sb[16];
            for (int u = 0; u < 16; ++u) { hb[u] = 0.0; sb[u] = 0.0; }
            double g_re = 0.0, g_sr = 0.0;
            const double c2 = sk.gamma_c2[eA][eB];
            const double rc2 = sk.r_cut * sk.r_cut;
            for (int im = 0; im < pl.n_img; ++im) {   // real-space Ewald sum
                const double x0 = dw[0] + pl.img[3 * im], x1 = dw[1] + pl.img[3 * im + 1], x2 = dw[2] + pl.img[3 * im + 2];
                const double r2 = fma(x0, x0, fma(x1, x1, x2 * x2));
                if (!(r2 < pl.r_real2) || r2 == 0.0) continue;
                const double ir = rsqrt_nr(r2);
                g_re = fma(erfc(pl.alpha * (r2 * ir)), ir, g_re);
            }
            for (int im = 0; im < pl.n_img_sk; ++im) {   // images within r_cut
                const double x0 = dw[0] + pl.img[3 * im], x1 = dw[1] + pl.img[3 * im + 1], x2 = dw[2] + pl.img[3 * im + 2];
                const double r2 = fma(x0, x0, fma(x1, x1, x2 * x2));
                if (!(r2 < rc2) || r2 == 0.0) continue;
                const double ir = rsqrt_nr(r2);
                const double r = r2 * ir;
                const double e[3] = {x0 * ir, x1 * ir, x2 * ir};
                for (int tb = 0; tb < 2; ++tb) {
                    const double(*tab)[CAVMD_MAX_ELEM][4][4] = tb == 0 ? sk.h0 : sk.s;
                    double *acc = tb == 0 ? hb : sb;
                    double v, dv;
                    radial_p(tab[eA][eB][CAVMD_SK_SS], r, sk, v, dv);
                    acc[0] += v;
                    if (nb == 4) {
                        radial_p(tab[eA][eB][CAVMD_SK_SP], r, sk, v, dv);
                        for (int i = 0; i < 3; ++i) acc[1 + i] = fma(e[i], v, acc[1 + i]);
                    }
                    if (na == 4) {
                        radial_p(tab[eB][eA][CAVMD_SK_SP], r, sk, v, dv);
                        for (int i = 0; i < 3; ++i) acc[4 * (1 + i)] = fma(-e[i], v, acc[4 * (1 + i)]);
                    }
                    if (na == 4 && nb == 4) {
                        double vs, vp;
                        radial_p(tab[eA][eB][CAVMD_SK_PPS], r, sk, vs, dv);
                        radial_p(tab[eA][eB][CAVMD_SK_PPP], r, sk, vp, dv);
                        const double dl = vs - vp;
                        for (int i = 0; i < 3; ++i)
                            for (int k = 0; k < 3; ++k)
                                acc[4 * (1 + i) + 1 + k] += fma(e[i] * e[k], dl, (i == k) ? vp : 0.0);
                    }
                }
                double fc, dfc;
                cutoff_fn(r, sk, fc, dfc);
                g_sr = fma(rsqrt_nr(r2 + c2) - ir, fc, g_sr);
            }
            // block (mu of A, nu of B) at column oB + nu, row oA + mu, and its transpose; a block of an
            // atom with its own images is symmetric, written as the mean of the two halves
            for (int mu = 0; mu < na; ++mu)
                for (int nu = 0; nu < nb; ++nu) {
                    const double hv = A == B ? 0.5 * (hb[4 * mu + nu] + hb[4 * nu + mu]) : hb[4 * mu + nu];
                    const double sv = A == B ? 0.5 * (sb[4 * mu + nu] + sb[4 * nu + mu]) : sb[4 * mu + nu];
                    H0[(oB + nu) * n + oA + mu] += hv;
                    S[(oB + nu) * n + oA + mu] += sv;
                    if (A != B) {
                        H0[(oA + mu) * n + oB + nu] = hv;
                        S[(oA + mu) * n + oB + nu] = sv;
                    }
                }
            double gv = g_re + g_sr + pl.bg;
            if (A == B) gv += sk.hubbard[eA] + pl.self_e;
            gam[A * pl.amax + B] = gv;
            gam[B * pl.amax + A] = gv;
        }
    }
    // cos and sin of G . (r_A - r_0) for the reciprocal sum
    for (int e = j; e < nat * pl.n_g; e += PT) {
        const int g = e / nat, at = e - g * nat;
        const double *G = pl.gw + 4 * g;
        const double ph = fma(G[0], sh.pos[at][0] - sh.pos[0][0],
                              fma(G[1], sh.pos[at][1] - sh.pos[0][1], G[2] * (sh.pos[at][2] - sh.pos[0][2])));
        double sn, cn;
        sincos(ph, &sn, &cn);
        csg[2LL * e] = cn;
        csg[2LL * e + 1] = sn;
    }
    __syncthreads();

    // atomic shifts eps_A = sum_B gamma_AB dq_B + reciprocal part, from sh.dq
    auto shifts = [&]() {
        for (int g = j; g < pl.n_g; g += PT) {
            double sc = 0.0, ss = 0.0;
            const double *t = csg + 2LL * g * nat;
            for (int at = 0; at < nat; ++at) {
                sc = fma(sh.dq[at], t[2 * at], sc);
                ss = fma(sh.dq[at], t[2 * at + 1], ss);
            }
            sgf[2 * g] = sc;
            sgf[2 * g + 1] = ss;
        }
        __syncthreads();
        if (j < nat) {
            double v = 0.0;
            for (int k = 0; k < nat; ++k) v = fma(gam[j * pl.amax + k], sh.dq[k], v);
            double rr = 0.0;
            for (int g = 0; g < pl.n_g; ++g) {
                const double *t = csg + 2LL * (g * nat + j);
                rr = fma(pl.gw[4 * g + 3], fma(t[0], sgf[2 * g], t[1] * sgf[2 * g + 1]), rr);
            }
            sh.shift[j] = v + rr;
        }
        __syncthreads();
    };
    auto build_h = [&]() {
        for (int e = j; e < mm; e += PT) {
            const int c = e / m, i = e - c * m;
            const int io = (KG && i >= n) ? i - n : i, co = (KG && c >= n) ? c - n : c;
            H[e] = fma(0.5 * S[e], sh.shift[sh.orb_atom[io]] + sh.shift[sh.orb_atom[co]], H0[e]);
        }
        __syncthreads();
    };
    auto rank_occupation = [&]() {
        for (int r = j; r < m; r += PT) {
            const long long kj = order_key(sh.diag[r]);
            int rank = 0;
            for (int i = 0; i < m; ++i) {
                const long long ki = order_key(sh.diag[i]);
                rank += (ki < kj) || (ki == kj && i < r);
            }
            sh.occf[r] = rank < mo;
            if (rank < mo) sh.occ_list[rank] = r; else sh.virt_list[rank - mo] = r;
        }
        __syncthreads();
    };
    auto Cat = [&](int i, int c) -> double { return C[c * m + i]; };
    // One cyclic Jacobi sweep on the block Ab = C_b^T Y_b of the columns list[0..m-1] (occupied or
    // virtual). It keeps the diagonal blocks of C^T H C diagonal, which the generator's diagonal
    // denominators need (the occupied-virtual rotations leave them alone, and within a block they
    // drift with every step). The rounds rotate Ab and accumulate the rotations in Vb (m x m,
    // starting from I); then C_b <- C_b Vb and Y_b <- Y_b Vb as staged products through H, which
    // is free until the next iteration builds it.
    // Workspaces it overwrites: Vb (the caller passes the density buffer P, free at this point:
    // P = 2 C_o C_o^T is formed later in the same iteration) and H (rebuilt at the start of the
    // next iteration). Neither may be read after a sweep before it is formed again.
    auto block_sweep = [&](const int *list, int mb, double *Ab, double *Vb) {
        pprod<false, true, true>(sh, mb, mb, m, [&](int i, int k) { return C[list[i] * m + k]; },
                                 [&](int k, int c) { return Y[list[c] * m + k]; },
                                 [&](int i, int c, double v) { Ab[c * mb + i] = v; });
        for (int e = j; e < mb * mb; e += PT) Vb[e] = (e / mb == e % mb) ? 1.0 : 0.0;
        __syncthreads();
        const int me = mb + (mb & 1), half = me / 2, span = 2 * mb;
        for (int rd = 0; rd < me - 1; ++rd) {
            if (j < half) {
                int p, qq;
                p_pair(j, rd, me, p, qq);
                double c = 1.0, s = 0.0;
                if (qq < mb) p_jacobi_cs(Ab[p * mb + p], Ab[qq * mb + qq], Ab[qq * mb + p], c, s);
                sh.pp[j] = p;
                sh.pq[j] = qq;
                sh.cs[2 * j] = c;
                sh.cs[2 * j + 1] = s;
            }
            __syncthreads();
            for (int e = j; e < half * span; e += PT) {   // columns p, q of Ab and Vb
                const int k = e / span, r = e - k * span;
                const int p = sh.pp[k], qq = sh.pq[k];
                if (qq >= mb) continue;
                const double c = sh.cs[2 * k], s = sh.cs[2 * k + 1];
                double *base = r < mb ? Ab : Vb;
                const int rr = r < mb ? r : r - mb;
                const double xp = base[p * mb + rr], yq = base[qq * mb + rr];
                base[p * mb + rr] = fma(c, xp, -s * yq);
                base[qq * mb + rr] = fma(s, xp, c * yq);
            }
            __syncthreads();
            for (int e = j; e < half * mb; e += PT) {   // rows p, q of Ab
                const int k = e / mb, cc = e - k * mb;
                const int p = sh.pp[k], qq = sh.pq[k];
                if (qq >= mb) continue;
                const double ck = sh.cs[2 * k], sk_ = sh.cs[2 * k + 1];
                const double x = Ab[cc * mb + p], y = Ab[cc * mb + qq];
                Ab[cc * mb + p] = fma(ck, x, -sk_ * y);
                Ab[cc * mb + qq] = fma(sk_, x, ck * y);
            }
            __syncthreads();
        }
        for (int t = 0; t < 2; ++t) {   // C_b <- C_b Vb, then Y_b <- Y_b Vb
            double *M_ = t == 0 ? C : Y;
            pprod<false, false, true>(sh, m, mb, mb, [&](int i, int k) { return M_[list[k] * m + i]; },
                                      [&](int k, int c) { return Vb[c * mb + k]; },
                                      [&](int i, int c, double v) { H[c * m + i] = v; });
            for (int e = j; e < m * mb; e += PT) {
                const int c = e / m, i = e - c * m;
                M_[list[c] * m + i] = H[e];
            }
            __syncthreads();
        }
        for (int r = j; r < mb; r += PT) sh.diag[list[r]] = Ab[r * mb + r];
        __syncthreads();
    };

    // ---------------------------------------------------------------- S-orthonormal start
    if (j < nat) {
        if (a.have_warm) {   // predictor 2 q(t) - q(t - dt); a displaced copy starts from q(r)
            const double qt = a.qpop[a0 + j];
            sh.qst[j] = qt;
            sh.q[j] = disp ? qt : fma(2.0, qt, -a.qprev[a0 + j]);
        } else {
            sh.q[j] = sh.zv[j];
        }
    }
    __syncthreads();
    // Mo <- lower of C^T S C (Y = S C first), its Cholesky factor L, then C <- C L^-T (every k-point)
    for (int kp = 0; kp < NKP; ++kp) {
        set_k(kp);
        if (!a.have_warm)
            for (int e = j; e < mm; e += PT) C[e] = (e / m == e % m) ? 1.0 : 0.0;
        pprod<false, false, true>(sh, m, m, m, [&](int i, int k) { return S[k * m + i]; }, Cat,
                                  [&](int i, int c, double v) { Y[c * m + i] = v; });
        pprod<true, true, true>(sh, m, m, m, [&](int i, int k) { return C[i * m + k]; },
                                [&](int k, int c) { return Y[c * m + k]; }, [&](int i, int c, double v) { Mo[c * m + i] = v; });
        if (!pchol(Mo, m, sh) && j == 0) sh.fl[0] |= ERRBIT_S_NOT_PD;
        for (int r = j; r < m; r += PT) row_solve_lt(Mo, m, sh.invd, C + r, m);
        __syncthreads();
    }

    // Warm steps re-diagonalise the occupied and virtual blocks every P_SWEEP_PERIOD steps, and
    // after an evaluation that needed more than P_SWEEP_ITERS iterations (a cold start, or drift).
    const bool sweep_now = a.have_warm && ((a.step_counter && (*a.step_counter % P_SWEEP_PERIOD) == 0) ||
                                           a.iters[cell] > P_SWEEP_ITERS);

    // ---------------------------------------------------------------- SCC loop
    // Per iteration: shifts, H, Y = H C, the diagonal of C^T Y and the occupation by rank; then the
    // occupied-virtual block A_vo, the generator X(v, o) = A_vo / (A_oo - A_vv) (FP32: it only
    // steers) and the Cayley rotation
    //   C_o <- (2 C_o + C_v X) (I + X^T X / 4)^-1 - C_o,  C_v <- (2 C_v - C_o X^T) (I + X X^T / 4)^-1 - C_v,
    // which is C (I - K/2)^-1 (I + K/2) for the antisymmetric K with K_vo = X. A cold start instead
    // forms all of C^T H C and runs Jacobi sweeps on its first iteration. Then P = 2 C_o C_o^T,
    // the Mulliken populations and Anderson mixing.
    int it;
    for (it = 1; it <= a.max_iter; ++it) {
        if (j < nat) sh.dq[j] = sh.q[j] - sh.zv[j];
        __syncthreads();
        shifts();
        bool eok_all = true;
        if (KG) {
            for (int r = j; r < n; r += PT) sh.qk[r] = 0.0;
            if (j == 0) {
                sh.hl[0] = -1e300;
                sh.hl[1] = 1e300;
            }
        }
        for (int kp = 0; kp < NKP; ++kp) {   // each k-point's update (Gamma: the one problem)
        set_k(kp);
        build_h();
        pprod<false, false, true>(sh, m, m, m, [&](int i, int k) { return H[k * m + i]; }, Cat,
                                  [&](int i, int c, double v) { Y[c * m + i] = v; });
        for (int r = j; r < m; r += PT) {
            double dg = 0.0;
            for (int k = 0; k < m; ++k) dg = fma(C[r * m + k], Y[r * m + k], dg);
            sh.diag[r] = dg;
        }
        __syncthreads();
        bool eok = false;
        const bool cold_first = !a.have_warm && it == 1;
        if (cold_first) {
            // all of A = C^T H C into P, then Jacobi sweeps on A accumulated into C
            pprod<false, true, true>(sh, m, m, m, [&](int i, int k) { return C[i * m + k]; },
                                     [&](int k, int c) { return Y[c * m + k]; },
                                     [&](int i, int c, double v) { P[c * m + i] = v; });
            double *Am = P;
            const int cap = a.max_sweeps > 0 ? a.max_sweeps : P_MAX_SWEEPS;
            for (int sweep = 0;; ++sweep) {
                bool off_small = true;
                for (int e = j; e < mm; e += PT) {
                    const int c = e / m, i = e - c * m;
                    if (i != c && !abs_lt(Am[c * m + i], P_JACOBI_TOL)) off_small = false;
                }
                if (blk_all(off_small)) break;
                if (sweep >= cap) {   // the cold start's sweeps ran out: DEVICE_TIMEOUT
                    if (j == 0) sh.fl[0] |= ERRBIT_TIMEOUT;
                    break;
                }
                for (int rd = 0; rd < m - 1; ++rd) {
                    if (j < m / 2) {
                        int p, qq;
                        p_pair(j, rd, m, p, qq);
                        double c, s;
                        p_jacobi_cs(Am[p * m + p], Am[qq * m + qq], Am[qq * m + p], c, s);
                        sh.pp[j] = p;
                        sh.pq[j] = qq;
                        sh.cs[2 * j] = c;
                        sh.cs[2 * j + 1] = s;
                    }
                    __syncthreads();
                    for (int e = j; e < m * (m / 2); e += PT) {   // columns p, q of A and C, row i
                        const int k = e / m, i = e - k * m;
                        const int p = sh.pp[k], qq = sh.pq[k];
                        const double c = sh.cs[2 * k], s = sh.cs[2 * k + 1];
                        const double ap = Am[p * m + i], aq = Am[qq * m + i];
                        Am[p * m + i] = fma(c, ap, -s * aq);
                        Am[qq * m + i] = fma(s, ap, c * aq);
                        const double cp = C[p * m + i], cq = C[qq * m + i];
                        C[p * m + i] = fma(c, cp, -s * cq);
                        C[qq * m + i] = fma(s, cp, c * cq);
                    }
                    __syncthreads();
                    for (int e = j; e < m * (m / 2); e += PT) {   // rows p, q of A, column c
                        const int k = e / m, c = e - k * m;
                        const int p = sh.pp[k], qq = sh.pq[k];
                        const double ck = sh.cs[2 * k], sk_ = sh.cs[2 * k + 1];
                        const double x = Am[c * m + p], y = Am[c * m + qq];
                        Am[c * m + p] = fma(ck, x, -sk_ * y);
                        Am[c * m + qq] = fma(sk_, x, ck * y);
                    }
                    __syncthreads();
                }
            }
            for (int r = j; r < m; r += PT) sh.diag[r] = Am[r * m + r];
            __syncthreads();
            rank_occupation();
        } else {
            rank_occupation();
            if (sweep_now && it == 1) {   // first iteration after a geometry change
                double *const sweep_V = P;   // the rotation accumulator: P is formed later this iteration
                block_sweep(sh.occ_list, mo, Mo, sweep_V);
                block_sweep(sh.virt_list, mv, Mv, sweep_V);
            }
            bool small = true;
            float kmax = 0.0f;
            // A_vo (entry (v, o), v fastest) and the generator, stored X[o nv + v]
            pprod<false, true, true>(sh, mv, mo, m, [&](int v, int k) { return C[sh.virt_list[v] * m + k]; },
                                     [&](int k, int o) { return Y[sh.occ_list[o] * m + k]; },
                                     [&](int v, int o, double val) {
                                         if (!abs_lt(val, P_EIG_TOL)) small = false;
                                         const float den = d2f_steer(sh.diag[sh.occ_list[o]] - sh.diag[sh.virt_list[v]]);
                                         float kf = d2f_steer(val) / den;
                                         if (!(fabsf(kf) <= 1e3f)) kf = copysignf(1e3f, kf);
                                         kmax = fmaxf(kmax, fabsf(kf));
                                         Xg[o * mv + v] = f2d_steer(kf);
                                     });
            eok = blk_all(small);
            // X^T X and X X^T (lower triangles)
            pprod<true, true, true>(sh, mo, mo, mv, [&](int o1, int v) { return Xg[o1 * mv + v]; },
                                    [&](int v, int o2) { return Xg[o2 * mv + v]; },
                                    [&](int i, int c, double v) { Mo[c * mo + i] = v; });
            pprod<true, false, false>(sh, mv, mv, mo, [&](int v1, int o) { return Xg[o * mv + v1]; },
                                      [&](int o, int v2) { return Xg[o * mv + v2]; },
                                      [&](int i, int c, double v) { Mv[c * mv + i] = v; });
            if (blk_all(kmax < P_KMAX_PERT)) {
                // small generator: C <- C (I + K + K^2/2), orthogonal to O(K^4) (below 1e-16 here):
                //   C_o <- C_o (I - X^T X / 2) + C_v X,  C_v <- C_v (I - X X^T / 2) - C_o X^T,
                // each one staged product over the columns [C_o | C_v], into Y
                pprod<false, false, true>(
                    sh, m, mo, m,
                    [&](int i, int k) { return C[(k < mo ? sh.occ_list[k] : sh.virt_list[k - mo]) * m + i]; },
                    [&](int k, int o) {
                        if (k >= mo) return Xg[o * mv + (k - mo)];
                        return fma(-0.5, Mo[min(k, o) * mo + max(k, o)], k == o ? 1.0 : 0.0);
                    },
                    [&](int i, int o, double v) { Y[o * m + i] = v; });
                pprod<false, false, false>(
                    sh, m, mv, m,
                    [&](int i, int k) { return C[(k < mv ? sh.virt_list[k] : sh.occ_list[k - mv]) * m + i]; },
                    [&](int k, int v) {
                        if (k >= mv) return -Xg[(k - mv) * mv + v];
                        return fma(-0.5, Mv[min(k, v) * mv + max(k, v)], k == v ? 1.0 : 0.0);
                    },
                    [&](int i, int v, double val) { Y[(mo + v) * m + i] = val; });
                for (int e = j; e < mm; e += PT) {
                    const int c = e / m, i = e - c * m;
                    const int col = c < mo ? sh.occ_list[c] : sh.virt_list[c - mo];
                    C[col * m + i] = Y[e];
                }
                __syncthreads();
            } else {
            // I + X^T X / 4 and I + X X^T / 4 in place
            for (int e = j; e < mo * mo; e += PT) {
                const int c = e / mo, i = e - c * mo;
                if (i >= c) Mo[e] = fma(0.25, Mo[e], i == c ? 1.0 : 0.0);
            }
            for (int e = j; e < mv * mv; e += PT) {
                const int c = e / mv, i = e - c * mv;
                if (i >= c) Mv[e] = fma(0.25, Mv[e], i == c ? 1.0 : 0.0);
            }
            __syncthreads();
            // Z1 = 2 C_o + C_v X into Y[o n + i]; Z2 = 2 C_v - C_o X^T into Y[(nocc + v) n + i]
            pprod<false, false, true>(sh, m, mo, mv, [&](int i, int v) { return C[sh.virt_list[v] * m + i]; },
                                      [&](int v, int o) { return Xg[o * mv + v]; },
                                      [&](int i, int o, double v) { Y[o * m + i] = fma(2.0, C[sh.occ_list[o] * m + i], v); });
            pprod<false, false, false>(sh, m, mv, mo, [&](int i, int o) { return C[sh.occ_list[o] * m + i]; },
                                       [&](int o, int v) { return Xg[o * mv + v]; },
                                       [&](int i, int v, double val) {
                                           Y[(mo + v) * m + i] = fma(2.0, C[sh.virt_list[v] * m + i], -val);
                                       });
            pchol(Mo, mo, sh);
            for (int r = j; r < m; r += PT) row_solve_llt(Mo, mo, sh.invd, Y + r, m, Y + r, m);
            __syncthreads();
            if (mv > 0) {
                pchol(Mv, mv, sh);
                for (int r = j; r < m; r += PT) row_solve_llt(Mv, mv, sh.invd, Y + mo * m + r, m, Y + mo * m + r, m);
            }
            __syncthreads();
            for (int e = j; e < mm; e += PT) {
                const int c = e / m, i = e - c * m;   // c < mo: occupied column c, else virtual c - mo
                const int col = c < mo ? sh.occ_list[c] : sh.virt_list[c - mo];
                C[col * m + i] = Y[e] - C[col * m + i];
            }
            __syncthreads();
            }
        }
        // P = 2 C_o C_o^T (lower triangle) and the Mulliken populations
        pprod<true, false, false>(sh, m, m, mo, [&](int i, int o) { return C[sh.occ_list[o] * m + i]; },
                                  [&](int o, int c) { return C[sh.occ_list[o] * m + c]; },
                                  [&](int i, int c, double v) { P[c * m + i] = 2.0 * v; });
        for (int r = j; r < m; r += PT) {
            double qo = 0.0;
            for (int k = 0; k < m; ++k) {
                const int lo = min(r, k), hi = max(r, k);
                qo = fma(P[lo * m + hi], S[k * m + r], qo);
            }
            sh.red[r] = qo;
        }
        __syncthreads();
        if (KG) {   // the k-point's populations (both halves of the real form) and its frontier levels
            const double w = pl.kpt[4 * kp + 3];
            for (int r = j; r < n; r += PT) sh.qk[r] = fma(0.5 * w, sh.red[r] + sh.red[r + n], sh.qk[r]);
            if (j == 0 && mo < m) {
                double homo = -1e300, lumo = 1e300;
                for (int c = 0; c < m; ++c) {
                    if (sh.occf[c]) homo = fmax(homo, sh.diag[c]); else lumo = fmin(lumo, sh.diag[c]);
                }
                sh.hl[0] = fmax(sh.hl[0], homo);
                sh.hl[1] = fmin(sh.hl[1], lumo);
            }
            __syncthreads();
        }
        eok_all = eok_all && eok;
        }
        const int NH = a.hist;
        const int hs = (it - 1) % NH;
        if (j < nat) {
            double qa = 0.0;
            for (int o = sh.atom_off[j]; o < sh.atom_off[j + 1]; ++o) qa += KG ? sh.qk[o] : sh.red[o];
            sh.qout[j] = qa;
            sh.hq[hs][j] = sh.q[j];
            sh.hf[hs][j] = qa - sh.q[j];
        }
        __syncthreads();
        bool conv = eok_all;
        for (int at = 0; at < nat; ++at)
            if (!abs_lt(sh.hf[hs][at], a.scc_tol)) conv = false;
        const int h = min(it, NH);
        if (!conv && j == 0) {
            // Anderson coefficients over the h - 1 previous iterates: normal equations in FP32 with
            // a small diagonal shift, solved by Cholesky (they only steer the iteration)
            float Mx[PHIST - 1][PHIST - 1], bv[PHIST - 1], x[PHIST - 1];
            const int mh = h - 1;
            for (int u = 0; u < mh; ++u) {
                const int hu = (hs + NH - 1 - u) % NH;
                float b = 0.f;
                for (int w = 0; w <= u; ++w) {
                    const int hw = (hs + NH - 1 - w) % NH;
                    float sacc = 0.f;
                    for (int at = 0; at < nat; ++at) {
                        const float du = d2f_steer(sh.hf[hu][at] - sh.hf[hs][at]);
                        const float dw = d2f_steer(sh.hf[hw][at] - sh.hf[hs][at]);
                        sacc = fmaf(du, dw, sacc);
                    }
                    Mx[u][w] = sacc;
                }
                for (int at = 0; at < nat; ++at)
                    b = fmaf(-d2f_steer(sh.hf[hu][at] - sh.hf[hs][at]), d2f_steer(sh.hf[hs][at]), b);
                bv[u] = b;
            }
            float dmax = 0.f;
            for (int u = 0; u < mh; ++u) dmax = fmaxf(dmax, Mx[u][u]);
            bool ok = mh > 0 && dmax > 0.f;
            for (int u = 0; u < mh && ok; ++u) {
                for (int w = 0; w <= u && ok; ++w) {
                    float sacc = Mx[u][w] + (u == w ? 1e-6f * dmax : 0.f);
                    for (int l = 0; l < w; ++l) sacc -= Mx[u][l] * Mx[w][l];
                    if (u == w) {
                        if (!(sacc > 0.f)) ok = false; else Mx[u][u] = sqrtf(sacc);
                    } else {
                        Mx[u][w] = sacc / Mx[w][w];
                    }
                }
            }
            if (ok) {
                for (int u = 0; u < mh; ++u) {
                    float sacc = bv[u];
                    for (int l = 0; l < u; ++l) sacc -= Mx[u][l] * x[l];
                    x[u] = sacc / Mx[u][u];
                }
                for (int u = mh - 1; u >= 0; --u) {
                    float sacc = x[u];
                    for (int l = u + 1; l < mh; ++l) sacc -= Mx[l][u] * x[l];
                    x[u] = sacc / Mx[u][u];
                }
                for (int u = 0; u < mh; ++u)
                    if (!(fabsf(x[u]) < 50.f)) ok = false;
            }
            for (int u = 0; u < PHIST - 1; ++u) sh.th[u] = (ok && u < mh) ? f2d_steer(x[u]) : 0.0;
        }
        __syncthreads();
        if (j < nat) {
            if (conv) {
                sh.q[j] = sh.qout[j];
            } else {
                const double q0 = sh.hq[hs][j], f0 = sh.hf[hs][j];
                double qb = q0, fb = f0;
                for (int u = 0; u < h - 1; ++u) {
                    const int hu = (hs + NH - 1 - u) % NH;
                    qb = fma(sh.th[u], sh.hq[hu][j] - q0, qb);
                    fb = fma(sh.th[u], sh.hf[hu][j] - f0, fb);
                }
                sh.q[j] = fma(a.beta, fb, qb);
            }
        }
        __syncthreads();
        if (conv) {
            if (j == 0) sh.fl[2] = it;
            break;
        }
    }
    __syncthreads();
    if (j == 0 && it > a.max_iter) {
        sh.fl[0] |= ERRBIT_SCC_NOCONV;
        sh.fl[2] = a.max_iter;
    }
    __syncthreads();
    if (disp) {   // a finite-difference copy: only its dipole
        if (j == 0) {
            double mu[3] = {0.0, 0.0, 0.0};
            for (int at = 0; at < nat; ++at) {
                const double Q = sh.zv[at] - sh.q[at];
                for (int k = 0; k < 3; ++k) mu[k] = fma(Q, sh.pos[at][k] - sh.pos[0][k], mu[k]);
            }
            a.M_disp[(long long)(a.fd_central ? 6 : 3) * a0 + disp_k] =
                fma(a.pol0, mu[0], fma(a.pol1, mu[1], a.pol2 * mu[2]));
            if (sh.fl[0]) atomicOr(a.status, (unsigned)sh.fl[0]);
        }
        __syncthreads();
        return;
    }

    // ---------------------------------------------------------------- energy and forces
    if constexpr (KG) {
        // per k-point: H; Y = H C and the occupation by rank; Aoo = C_o^T Y_o (lower) into Mo;
        // t = 2 Aoo C_o^T into Mv; W = C_o t (lower) into H; P = 2 C_o C_o^T (lower) into P; then the
        // pair tasks with the k-point's phases, accumulated over the k-points (the k-independent
        // terms, second order and repulsion, with the first)
        if (j < nat) sh.dq[j] = sh.q[j] - sh.zv[j];
        __syncthreads();
        shifts();
        if (j == 0) {
            sh.hl[0] = -1e300;
            sh.hl[1] = 1e300;
        }
        double eb_t = 0.0;   // this thread's part of the band energy sum_k w_k Re Tr P(k) H0(k)*
        const double rc2 = sk.r_cut * sk.r_cut;
        for (int kp = 0; kp < NKP; ++kp) {
            set_k(kp);
            const bool first = kp == 0;
            const double wkp = pl.kpt[4 * kp + 3];
            const double fk[3] = {pl.kpt[4 * kp], pl.kpt[4 * kp + 1], pl.kpt[4 * kp + 2]};
            build_h();
            pprod<false, false, true>(sh, m, m, m, [&](int i, int k) { return H[k * m + i]; }, Cat,
                                      [&](int i, int c, double v) { Y[c * m + i] = v; });
            for (int r = j; r < m; r += PT) {
                double dg = 0.0;
                for (int k = 0; k < m; ++k) dg = fma(C[r * m + k], Y[r * m + k], dg);
                sh.diag[r] = dg;
            }
            __syncthreads();
            rank_occupation();
            if (j == 0) {
                for (int c = 0; c < m; ++c) {
                    if (sh.occf[c]) sh.hl[0] = fmax(sh.hl[0], sh.diag[c]); else sh.hl[1] = fmin(sh.hl[1], sh.diag[c]);
                }
            }
            pprod<true, true, true>(sh, mo, mo, m, [&](int o1, int k) { return C[sh.occ_list[o1] * m + k]; },
                                    [&](int k, int o2) { return Y[sh.occ_list[o2] * m + k]; },
                                    [&](int i, int c, double v) { Mo[c * mo + i] = v; });
            pprod<false, false, false>(sh, mo, m, mo,
                                       [&](int o, int o2) { return Mo[min(o, o2) * mo + max(o, o2)]; },
                                       [&](int o2, int c) { return C[sh.occ_list[o2] * m + c]; },
                                       [&](int o, int c, double v) { Mv[c * mo + o] = 2.0 * v; });
            pprod<true, false, true>(sh, m, m, mo, [&](int i, int o) { return C[sh.occ_list[o] * m + i]; },
                                     [&](int o, int c) { return Mv[c * mo + o]; },
                                     [&](int i, int c, double v) { H[c * m + i] = v; });
            pprod<true, false, false>(sh, m, m, mo, [&](int i, int o) { return C[sh.occ_list[o] * m + i]; },
                                      [&](int o, int c) { return C[sh.occ_list[o] * m + c]; },
                                      [&](int i, int c, double v) { P[c * m + i] = 2.0 * v; });
            for (int r = j; r < m; r += PT) {   // sum over the real form: 2 Re Tr P(k) H0(k)*
                double eb = 0.0;
                for (int i = r; i < m; ++i) eb = fma((i == r ? 1.0 : 2.0) * P[r * m + i], H0[r * m + i], eb);
                eb_t = fma(0.5 * wkp, eb, eb_t);
            }
            __syncthreads();
            const double *W = H;
            for (int t = j; t < nat * (nat + 1) / 2; t += PT) {   // pairs A <= B, packed by A
                const int A = lower_col(t, nat), B = A + (t - (A * nat - A * (A - 1) / 2));
                const int eA = sh.spec[A], eB = sh.spec[B];
                const int oA = sh.atom_off[A], oB = sh.atom_off[B];
                const int na = sk.norb[eA], nb = sk.norb[eB];
                double d[3], f[3], dw[3];
                for (int k = 0; k < 3; ++k) d[k] = sh.pos[B][k] - sh.pos[A][k];
                for (int k = 0; k < 3; ++k) f[k] = rint(fma(d[0], pl.inv[k], fma(d[1], pl.inv[3 + k], d[2] * pl.inv[6 + k])));
                for (int k = 0; k < 3; ++k) dw[k] = d[k] - fma(f[0], pl.lat[k], fma(f[1], pl.lat[3 + k], f[2] * pl.lat[6 + k]));
                const double hshift = 0.5 * (sh.shift[A] + sh.shift[B]);
                const double qq = sh.dq[A] * sh.dq[B];
                const double c2 = sk.gamma_c2[eA][eB];
                const double arep = sk.rep[eA][eB][0], brep = sk.rep[eA][eB][1];
                const double two_a_spi = 2.0 * pl.alpha * 0.5641895835477563;   // 2 alpha / sqrt(pi)
                double gk[3] = {0.0, 0.0, 0.0};
                double erep = 0.0;
                if (A != B && first) {
                    for (int im = 0; im < pl.n_img; ++im) {   // real-space Ewald gradient
                        const double x0 = dw[0] + pl.img[3 * im], x1 = dw[1] + pl.img[3 * im + 1], x2 = dw[2] + pl.img[3 * im + 2];
                        const double r2 = fma(x0, x0, fma(x1, x1, x2 * x2));
                        if (!(r2 < pl.r_real2) || r2 == 0.0) continue;
                        const double ir = rsqrt_nr(r2);
                        const double ar = pl.alpha * (r2 * ir);
                        const double rad = -qq * (erfc(ar) * ir + two_a_spi * exp(-ar * ar)) * ir * ir;
                        gk[0] = fma(rad, x0, gk[0]);
                        gk[1] = fma(rad, x1, gk[1]);
                        gk[2] = fma(rad, x2, gk[2]);
                    }
                }
                for (int im = 0; im < pl.n_img_sk; ++im) {   // images within r_cut
                    const double x0 = dw[0] + pl.img[3 * im], x1 = dw[1] + pl.img[3 * im + 1], x2 = dw[2] + pl.img[3 * im + 2];
                    const double r2 = fma(x0, x0, fma(x1, x1, x2 * x2));
                    if (!(r2 < rc2) || r2 == 0.0) continue;
                    const double ir = rsqrt_nr(r2);
                    const double r = r2 * ir;
                    const double e[3] = {x0 * ir, x1 * ir, x2 * ir};
                    double rad = 0.0;   // d/dr of the radial terms, along e
                    double fc, dfc;
                    cutoff_fn(r, sk, fc, dfc);
                    if (first) {
                        if (arep != 0.0) {
                            const double vr = arep * exp(-brep * r);
                            erep = fma(vr, fc, erep);
                            if (A != B) rad = fma(vr, dfc - brep * fc, rad);
                        }
                        if (A != B) {
                            const double gi = rsqrt_nr(r2 + c2);
                            const double s_ = gi - ir;
                            const double ds = fma(-r * gi, gi * gi, ir * ir);
                            rad = fma(qq, fma(ds, fc, s_ * dfc), rad);
                        }
                    }
                    if (A != B) {
                        double ph = 0.0;   // the image's phase 2 pi f_k . n_T
                        for (int k = 0; k < 3; ++k) {
                            const double nk_ = rint(fma(pl.img[3 * im], pl.inv[k], fma(pl.img[3 * im + 1], pl.inv[3 + k],
                                                                                         pl.img[3 * im + 2] * pl.inv[6 + k]))) - f[k];
                            ph = fma(fk[k], nk_, ph);
                        }
                        double sn, cs;
                        sincospi(2.0 * ph, &sn, &cs);
                        // band and overlap terms: weights rho(T) and rho(T) (eps_A + eps_B) / 2 - w(T) of the
                        // block, rho(T)_{mu nu} = w_k Re[P(k)_{nu mu} e^{i ph}] (mu of A < nu of B)
                        double g[3] = {0.0, 0.0, 0.0};
                        for (int tb = 0; tb < 2; ++tb) {
                            const double(*tab)[CAVMD_MAX_ELEM][4][4] = tb == 0 ? sk.h0 : sk.s;
                            auto wt = [&](int mu, int nu) -> double {
                                const double pr = P[(long long)mu * m + nu], pim = P[(long long)mu * m + n + nu];
                                const double rho = wkp * fma(pr, cs, -pim * sn);
                                if (tb == 0) return rho;
                                const double wr = W[(long long)mu * m + nu], wim = W[(long long)mu * m + n + nu];
                                return fma(rho, hshift, -wkp * fma(wr, cs, -wim * sn));
                            };
                            double v, dv;
                            radial_p(tab[eA][eB][CAVMD_SK_SS], r, sk, v, dv);
                            {
                                const double w = wt(oA, oB) * dv;
                                for (int k = 0; k < 3; ++k) g[k] = fma(w, e[k], g[k]);
                            }
                            if (nb == 4) {
                                radial_p(tab[eA][eB][CAVMD_SK_SP], r, sk, v, dv);
                                double w[3], we = 0.0;
                                for (int i = 0; i < 3; ++i) { w[i] = wt(oA, oB + 1 + i); we = fma(w[i], e[i], we); }
                                for (int k = 0; k < 3; ++k) g[k] += fma(w[k] - we * e[k], v * ir, we * e[k] * dv);
                            }
                            if (na == 4) {
                                radial_p(tab[eB][eA][CAVMD_SK_SP], r, sk, v, dv);
                                double w[3], we = 0.0;
                                for (int i = 0; i < 3; ++i) { w[i] = wt(oA + 1 + i, oB); we = fma(w[i], e[i], we); }
                                for (int k = 0; k < 3; ++k) g[k] -= fma(w[k] - we * e[k], v * ir, we * e[k] * dv);
                            }
                            if (na == 4 && nb == 4) {
                                double vs, dvs, vp, dvp;
                                radial_p(tab[eA][eB][CAVMD_SK_PPS], r, sk, vs, dvs);
                                radial_p(tab[eA][eB][CAVMD_SK_PPP], r, sk, vp, dvp);
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
                                    g[k] += (We[k] + WTe[k] - 2.0 * eWe * e[k]) * dl * ir + eWe * e[k] * ddl + tr * e[k] * dvp;
                            }
                        }
                        for (int k = 0; k < 3; ++k) gk[k] = fma(2.0, g[k], gk[k]);
                    }
                    for (int k = 0; k < 3; ++k) gk[k] = fma(rad, e[k], gk[k]);
                }
                double *pb = pbuf + 4LL * (A * nat + B);
                if (first) {
                    pb[0] = gk[0];
                    pb[1] = gk[1];
                    pb[2] = gk[2];
                    pb[3] = A == B ? 0.5 * erep : erep;
                } else {
                    pb[0] += gk[0];
                    pb[1] += gk[1];
                    pb[2] += gk[2];
                }
            }
            __syncthreads();
        }
        if (j == 0 && mo < m && !(sh.hl[1] - sh.hl[0] > P_MIN_GAP)) sh.fl[0] |= ERRBIT_ZERO_GAP;
        // the band energy into sh.red[0] (the rest of the n entries zero), summed in thread order
        sh.cs[j] = eb_t;
        __syncthreads();
        if (j == 0) {
            double eb = 0.0;
            for (int t = 0; t < PT; ++t) eb += sh.cs[t];
            sh.red[0] = eb;
        }
        for (int r = j; r < n; r += PT)
            if (r > 0) sh.red[r] = 0.0;
        __syncthreads();
    } else {
        // Shifts of the converged charges; H; T = H C_o into Y; Aoo = C_o^T T (lower) into Mo;
        // t = 2 Aoo C_o^T into Mv; W = C_o t (lower) into H; P = 2 C_o C_o^T (lower) into P.
        if (j < nat) sh.dq[j] = sh.q[j] - sh.zv[j];
        __syncthreads();
        shifts();
        build_h();
        pprod<false, false, true>(sh, n, nocc, n, [&](int i, int k) { return H[k * n + i]; },
                                  [&](int k, int o) { return C[sh.occ_list[o] * n + k]; },
                                  [&](int i, int o, double v) { Y[o * n + i] = v; });
        pprod<true, true, true>(sh, nocc, nocc, n, [&](int o1, int k) { return C[sh.occ_list[o1] * n + k]; },
                                [&](int k, int o2) { return Y[o2 * n + k]; },
                                [&](int i, int c, double v) { Mo[c * nocc + i] = v; });
        pprod<false, false, false>(sh, nocc, n, nocc,
                                   [&](int o, int o2) { return Mo[min(o, o2) * nocc + max(o, o2)]; },
                                   [&](int o2, int c) { return C[sh.occ_list[o2] * n + c]; },
                                   [&](int o, int c, double v) { Mv[c * nocc + o] = 2.0 * v; });
        pprod<true, false, true>(sh, n, n, nocc, [&](int i, int o) { return C[sh.occ_list[o] * n + i]; },
                                 [&](int o, int c) { return Mv[c * nocc + o]; },
                                 [&](int i, int c, double v) { H[c * n + i] = v; });
        pprod<true, false, false>(sh, n, n, nocc, [&](int i, int o) { return C[sh.occ_list[o] * n + i]; },
                                  [&](int o, int c) { return C[sh.occ_list[o] * n + c]; },
                                  [&](int i, int c, double v) { P[c * n + i] = 2.0 * v; });
        if (j == 0 && nocc < n) {   // HOMO-LUMO gap of the last iteration
            double homo = -1e300, lumo = 1e300;
            for (int c = 0; c < n; ++c) {
                if (sh.occf[c]) homo = fmax(homo, sh.diag[c]); else lumo = fmin(lumo, sh.diag[c]);
            }
            if (!(lumo - homo > P_MIN_GAP)) sh.fl[0] |= ERRBIT_ZERO_GAP;
        }
        if (j < n) {   // band energy sum P H0, by column of the lower triangle
            double eb = 0.0;
            for (int i = j; i < n; ++i) eb = fma((i == j ? 1.0 : 2.0) * P[j * n + i], H0[j * n + i], eb);
            sh.red[j] = eb;
        }
        __syncthreads();
        const double *W = H;
        // pair tasks A <= B: d/dr_B of every image term (band, overlap, second order, repulsion), and
        // the repulsion energy (an atom with its own images counts each image pair once)
        for (int t = j; t < nat * (nat + 1) / 2; t += PT) {   // pairs A <= B, packed by A
            const int A = lower_col(t, nat), B = A + (t - (A * nat - A * (A - 1) / 2));
            const int eA = sh.spec[A], eB = sh.spec[B];
            const int oA = sh.atom_off[A], oB = sh.atom_off[B];
            const int na = sk.norb[eA], nb = sk.norb[eB];
            double d[3], f[3], dw[3];
            for (int k = 0; k < 3; ++k) d[k] = sh.pos[B][k] - sh.pos[A][k];
            for (int k = 0; k < 3; ++k) f[k] = rint(fma(d[0], pl.inv[k], fma(d[1], pl.inv[3 + k], d[2] * pl.inv[6 + k])));
            for (int k = 0; k < 3; ++k) dw[k] = d[k] - fma(f[0], pl.lat[k], fma(f[1], pl.lat[3 + k], f[2] * pl.lat[6 + k]));
            const double hshift = 0.5 * (sh.shift[A] + sh.shift[B]);
            const double qq = sh.dq[A] * sh.dq[B];
            const double c2 = sk.gamma_c2[eA][eB];
            const double rc2 = sk.r_cut * sk.r_cut;
            const double arep = sk.rep[eA][eB][0], brep = sk.rep[eA][eB][1];
            const double two_a_spi = 2.0 * pl.alpha * 0.5641895835477563;   // 2 alpha / sqrt(pi)
            double gk[3] = {0.0, 0.0, 0.0};
            double erep = 0.0;
            if (A != B) {
                for (int im = 0; im < pl.n_img; ++im) {   // real-space Ewald gradient
                    const double x0 = dw[0] + pl.img[3 * im], x1 = dw[1] + pl.img[3 * im + 1], x2 = dw[2] + pl.img[3 * im + 2];
                    const double r2 = fma(x0, x0, fma(x1, x1, x2 * x2));
                    if (!(r2 < pl.r_real2) || r2 == 0.0) continue;
                    const double ir = rsqrt_nr(r2);
                    const double ar = pl.alpha * (r2 * ir);
                    const double rad = -qq * (erfc(ar) * ir + two_a_spi * exp(-ar * ar)) * ir * ir;
                    gk[0] = fma(rad, x0, gk[0]);
                    gk[1] = fma(rad, x1, gk[1]);
                    gk[2] = fma(rad, x2, gk[2]);
                }
            }
            for (int im = 0; im < pl.n_img_sk; ++im) {   // images within r_cut
                const double x0 = dw[0] + pl.img[3 * im], x1 = dw[1] + pl.img[3 * im + 1], x2 = dw[2] + pl.img[3 * im + 2];
                const double r2 = fma(x0, x0, fma(x1, x1, x2 * x2));
                if (!(r2 < rc2) || r2 == 0.0) continue;
                const double ir = rsqrt_nr(r2);
                const double r = r2 * ir;
                const double e[3] = {x0 * ir, x1 * ir, x2 * ir};
                double rad = 0.0;   // d/dr of the radial terms, along e
                {
                    double fc, dfc;
                    cutoff_fn(r, sk, fc, dfc);
                    if (arep != 0.0) {
                        const double vr = arep * exp(-brep * r);
                        erep = fma(vr, fc, erep);
                        if (A != B) rad = fma(vr, dfc - brep * fc, rad);
                    }
                    if (A != B) {
                        const double gi = rsqrt_nr(r2 + c2);
                        const double s_ = gi - ir;
                        const double ds = fma(-r * gi, gi * gi, ir * ir);
                        rad = fma(qq, fma(ds, fc, s_ * dfc), rad);
                        // band and overlap terms: weights P and P (eps_A + eps_B) / 2 - W of the block
                        double g[3] = {0.0, 0.0, 0.0};
                        for (int tb = 0; tb < 2; ++tb) {
                            const double(*tab)[CAVMD_MAX_ELEM][4][4] = tb == 0 ? sk.h0 : sk.s;
                            auto wt = [&](int mu, int nu) -> double {   // mu of A < nu of B: lower entry (nu, mu)
                                const double pv = P[mu * n + nu];
                                return tb == 0 ? pv : fma(pv, hshift, -W[mu * n + nu]);
                            };
                            double v, dv;
                            radial_p(tab[eA][eB][CAVMD_SK_SS], r, sk, v, dv);
                            {
                                const double w = wt(oA, oB) * dv;
                                for (int k = 0; k < 3; ++k) g[k] = fma(w, e[k], g[k]);
                            }
                            if (nb == 4) {
                                radial_p(tab[eA][eB][CAVMD_SK_SP], r, sk, v, dv);
                                double w[3], we = 0.0;
                                for (int i = 0; i < 3; ++i) { w[i] = wt(oA, oB + 1 + i); we = fma(w[i], e[i], we); }
                                for (int k = 0; k < 3; ++k) g[k] += fma(w[k] - we * e[k], v * ir, we * e[k] * dv);
                            }
                            if (na == 4) {
                                radial_p(tab[eB][eA][CAVMD_SK_SP], r, sk, v, dv);
                                double w[3], we = 0.0;
                                for (int i = 0; i < 3; ++i) { w[i] = wt(oA + 1 + i, oB); we = fma(w[i], e[i], we); }
                                for (int k = 0; k < 3; ++k) g[k] -= fma(w[k] - we * e[k], v * ir, we * e[k] * dv);
                            }
                            if (na == 4 && nb == 4) {
                                double vs, dvs, vp, dvp;
                                radial_p(tab[eA][eB][CAVMD_SK_PPS], r, sk, vs, dvs);
                                radial_p(tab[eA][eB][CAVMD_SK_PPP], r, sk, vp, dvp);
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
                                    g[k] += (We[k] + WTe[k] - 2.0 * eWe * e[k]) * dl * ir + eWe * e[k] * ddl + tr * e[k] * dvp;
                            }
                        }
                        for (int k = 0; k < 3; ++k) gk[k] = fma(2.0, g[k], gk[k]);
                    }
                }
                for (int k = 0; k < 3; ++k) gk[k] = fma(rad, e[k], gk[k]);
            }
            double *pb = pbuf + 4LL * (A * nat + B);
            pb[0] = gk[0];
            pb[1] = gk[1];
            pb[2] = gk[2];
            pb[3] = A == B ? 0.5 * erep : erep;
        }
        __syncthreads();
    }
    if (j < nat) {
        // reciprocal part: d/dr_A of 1/2 sum_G w_G |S(G)|^2 = dq_A sum_G w_G G (c_A S_s - s_A S_c)
        double gr[3] = {0.0, 0.0, 0.0};
        for (int g = 0; g < pl.n_g; ++g) {
            const double *t = csg + 2LL * (g * nat + j);
            const double amp = pl.gw[4 * g + 3] * fma(t[0], sgf[2 * g + 1], -t[1] * sgf[2 * g]);
            for (int k = 0; k < 3; ++k) gr[k] = fma(amp, pl.gw[4 * g + k], gr[k]);
        }
        double G[3];
        for (int k = 0; k < 3; ++k) G[k] = sh.dq[j] * gr[k];
        for (int A = 0; A < nat; ++A) {
            if (A == j) continue;
            const double *pb = pbuf + 4LL * (A < j ? A * nat + j : j * nat + A);
            const double sg = A < j ? 1.0 : -1.0;
            for (int k = 0; k < 3; ++k) G[k] = fma(sg, pb[k], G[k]);
        }
        const int at = a0 + j;
        for (int k = 0; k < 3; ++k) a.F[3 * at + k] = -G[k];
        a.qprev[at] = a.have_warm ? sh.qst[j] : sh.q[j];
        a.qpop[at] = sh.q[j];
        if (a.Qout) a.Qout[at] = sh.zv[j] - sh.q[j];
        if (a.write_b) {
            const double Q = sh.zv[j] - sh.q[j];
            a.b[3 * at + 0] = Q * a.pol0;
            a.b[3 * at + 1] = Q * a.pol1;
            a.b[3 * at + 2] = Q * a.pol2;
        }
    }
    if (j == 0) {
        double E = 0.0;
        for (int i = 0; i < n; ++i) E += sh.red[i];
        double e2 = 0.0;
        for (int x = 0; x < nat; ++x) e2 = fma(sh.dq[x], sh.shift[x], e2);
        E = fma(0.5, e2, E);
        for (int A = 0; A < nat; ++A)
            for (int B = A; B < nat; ++B) E += pbuf[4LL * (A * nat + B) + 3];
        double mu[3] = {0.0, 0.0, 0.0};
        for (int at = 0; at < nat; ++at) {
            const double Q = sh.zv[at] - sh.q[at];
            for (int k = 0; k < 3; ++k) mu[k] = fma(Q, sh.pos[at][k] - sh.pos[0][k], mu[k]);
        }
        a.E_cell[cell] = E;
        a.M_cell[cell] = fma(a.pol0, mu[0], fma(a.pol1, mu[1], a.pol2 * mu[2]));
        a.iters[cell] = sh.fl[2];
        if (sh.fl[0]) atomicOr(a.status, (unsigned)sh.fl[0]);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(PT, 2) k_dftb_periodic(const DevSK *__restrict__ skp, const DftbArgs a, const PbcDev pl) {
    extern __shared__ __align__(16) unsigned char p_smem[];
    PShared &sh = *reinterpret_cast<PShared *>(p_smem);
    const DevSK &sk = *skp;
    double *wk = pl.work + (long long)blockIdx.x * pl.work_stride;
    for (int cell = blockIdx.x; cell < a.n_cells; cell += gridDim.x) p_cell<false, false>(sk, a, pl, sh, wk, cell, -1);
}

// k-grid sampling: one cell at a time per block, its k-points in turn (one block per SM: the real
// forms of the k-point problems need twice the shared staging of the Gamma point).
__global__ void __launch_bounds__(PT, 1) k_dftb_periodic_kg(const DevSK *__restrict__ skp, const DftbArgs a,
                                                            const PbcDev pl) {
    extern __shared__ __align__(16) unsigned char p_smem[];
    PSharedK &sh = *reinterpret_cast<PSharedK *>(p_smem);
    const DevSK &sk = *skp;
    double *wk = pl.work + (long long)blockIdx.x * pl.work_stride;
    for (int cell = blockIdx.x; cell < a.n_cells; cell += gridDim.x) p_cell<false, true>(sk, a, pl, sh, wk, cell, -1);
}

// Finite-difference copies of every cell: (cell, row) items, rows_max = 3 (central: 6) x the
// largest atom count per cell.
__global__ void __launch_bounds__(PT, 2) k_dftb_periodic_disp(const DevSK *__restrict__ skp, const DftbArgs a,
                                                             const PbcDev pl) {
    extern __shared__ __align__(16) unsigned char p_smem[];
    PShared &sh = *reinterpret_cast<PShared *>(p_smem);
    const DevSK &sk = *skp;
    double *wk = pl.work + (long long)blockIdx.x * pl.work_stride;
    const int per_atom = a.fd_central ? 6 : 3;
    const long long rows_max = (long long)per_atom * pl.amax, items = rows_max * a.n_cells;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int cell = (int)(it / rows_max), k = (int)(it - (long long)cell * rows_max);
        if (k < per_atom * (a.cell_offset[cell + 1] - a.cell_offset[cell])) p_cell<true, false>(sk, a, pl, sh, wk, cell, k);
    }
}

__global__ void __launch_bounds__(PT, 1) k_dftb_periodic_kg_disp(const DevSK *__restrict__ skp, const DftbArgs a,
                                                                 const PbcDev pl) {
    extern __shared__ __align__(16) unsigned char p_smem[];
    PSharedK &sh = *reinterpret_cast<PSharedK *>(p_smem);
    const DevSK &sk = *skp;
    double *wk = pl.work + (long long)blockIdx.x * pl.work_stride;
    const int per_atom = a.fd_central ? 6 : 3;
    const long long rows_max = (long long)per_atom * pl.amax, items = rows_max * a.n_cells;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int cell = (int)(it / rows_max), k = (int)(it - (long long)cell * rows_max);
        if (k < per_atom * (a.cell_offset[cell + 1] - a.cell_offset[cell])) p_cell<true, true>(sk, a, pl, sh, wk, cell, k);
    }
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// Host side

size_t pbc_workspace_doubles(int nmax, int amax, int n_g, int nk) {
    if (nk > 0) {   // k-grid: six work matrices and H0(k), S(k) of every k-point, in real form (2 nmax)^2;
                    // the last nk of them: a finite-difference copy's bases
        const size_t m2 = 4 * (size_t)nmax * nmax;
        return (6 + 3 * (size_t)nk) * m2 + (size_t)amax * amax + 2 * (size_t)amax * n_g + 2 * (size_t)n_g +
               4 * (size_t)amax * amax + 32;
    }
    const size_t n2 = (size_t)nmax * nmax;   // the last n2: a finite-difference copy's basis
    return 9 * n2 + (size_t)amax * amax + 2 * (size_t)amax * n_g + 2 * (size_t)n_g + 4 * (size_t)amax * amax + 32;
}

// The irreducible points of a Gamma-centred n1 x n2 x n3 grid: k and -k (modulo the reciprocal
// lattice) give complex-conjugate problems with the same populations and band energy, so each
// pair is kept once with weight 2 / (n1 n2 n3) (self-conjugate points: 1 / (n1 n2 n3)), the
// member with the smaller grid index. Rows: f1, f2, f3, weight.
std::vector<double> pbc_kpoints(const int *kgrid) {
    const int n1 = kgrid[0], n2 = kgrid[1], n3 = kgrid[2], N = n1 * n2 * n3;
    std::vector<double> out;
    for (int i = 0; i < n1; ++i)
        for (int j = 0; j < n2; ++j)
            for (int l = 0; l < n3; ++l) {
                const int ii = (n1 - i) % n1, jj = (n2 - j) % n2, ll = (n3 - l) % n3;   // -k on the grid
                const int idx = (i * n2 + j) * n3 + l, midx = (ii * n2 + jj) * n3 + ll;
                if (midx < idx) continue;
                out.push_back((double)i / n1);
                out.push_back((double)j / n2);
                out.push_back((double)l / n3);
                out.push_back((midx == idx ? 1.0 : 2.0) / N);
            }
    return out;
}

// Lattice images and reciprocal vectors for one lattice (rows a_i), and the Ewald constants. The
// splitting parameter is chosen so the half-space reciprocal list holds about 1000 vectors; every
// term left out of either sum is below 1e-18 (erfc(6.5) and exp(-6.5^2)).
void plan_dftb_periodic(const double *lat, double r_cut, PbcPlan &p, std::vector<double> &img,
                        std::vector<double> &gw) {
    for (int k = 0; k < 9; ++k) p.lat[k] = lat[k];
    const double a0 = lat[0], a1 = lat[1], a2 = lat[2], b0 = lat[3], b1 = lat[4], b2 = lat[5], c0 = lat[6],
                 c1 = lat[7], c2 = lat[8];
    const double det = a0 * (b1 * c2 - b2 * c1) - a1 * (b0 * c2 - b2 * c0) + a2 * (b0 * c1 - b1 * c0);
    // inverse (f = r inv with r a row vector): inv = lat^-1
    double inv[9];
    inv[0] = (b1 * c2 - b2 * c1) / det; inv[1] = (a2 * c1 - a1 * c2) / det; inv[2] = (a1 * b2 - a2 * b1) / det;
    inv[3] = (b2 * c0 - b0 * c2) / det; inv[4] = (a0 * c2 - a2 * c0) / det; inv[5] = (a2 * b0 - a0 * b2) / det;
    inv[6] = (b0 * c1 - b1 * c0) / det; inv[7] = (a1 * c0 - a0 * c1) / det; inv[8] = (a0 * b1 - a1 * b0) / det;
    for (int k = 0; k < 9; ++k) p.inv[k] = inv[k];
    const double V = std::fabs(det);
    const double EX = 6.5;
    const double pi = 3.141592653589793;
    // half-space count N ~ (4 pi / 3) (2 alpha EX)^3 V / (2 (2 pi)^3)  ->  alpha for N = 1000
    const double g_cube = 1000.0 * 2.0 * std::pow(2.0 * pi, 3) * 3.0 / (4.0 * pi * V);
    const double alpha = std::cbrt(g_cube) / (2.0 * EX);
    p.alpha = alpha;
    p.bg = -pi / (alpha * alpha * V);
    p.self_e = -2.0 * alpha / std::sqrt(pi);
    const double r_real = std::max(EX / alpha, r_cut);
    p.r_real = r_real;
    // farthest point of a wrapped separation (fractional coordinates in [-1/2, 1/2]): a corner
    double hmax = 0.0;
    for (int s = 0; s < 8; ++s) {
        const double f0 = (s & 1) ? 0.5 : -0.5, f1 = (s & 2) ? 0.5 : -0.5, f2 = (s & 4) ? 0.5 : -0.5;
        double x[3];
        for (int k = 0; k < 3; ++k) x[k] = f0 * lat[k] + f1 * lat[3 + k] + f2 * lat[6 + k];
        hmax = std::max(hmax, std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]));
    }
    // heights across the faces: h_i = 1 / |column i of inv|
    int N[3];
    for (int i = 0; i < 3; ++i) {
        const double h = 1.0 / std::sqrt(inv[i] * inv[i] + inv[3 + i] * inv[3 + i] + inv[6 + i] * inv[6 + i]);
        N[i] = (int)std::ceil((r_real + hmax) / h) + 1;
    }
    // translations by increasing length (ties in the order generated); a wrapped separation
    // reaches an image within r_cut only through a translation shorter than r_cut + hmax
    struct Tr { double len, t[3]; };
    std::vector<Tr> trs;
    const double reach = r_real + hmax;
    for (int n0 = -N[0]; n0 <= N[0]; ++n0)
        for (int n1 = -N[1]; n1 <= N[1]; ++n1)
            for (int n2 = -N[2]; n2 <= N[2]; ++n2) {
                Tr t;
                for (int k = 0; k < 3; ++k) t.t[k] = n0 * lat[k] + n1 * lat[3 + k] + n2 * lat[6 + k];
                t.len = std::sqrt(t.t[0] * t.t[0] + t.t[1] * t.t[1] + t.t[2] * t.t[2]);
                if (t.len < reach) trs.push_back(t);
            }
    std::stable_sort(trs.begin(), trs.end(), [](const Tr &a, const Tr &b) { return a.len < b.len; });
    img.clear();
    p.n_img_sk = 0;
    for (const Tr &t : trs) {
        img.insert(img.end(), t.t, t.t + 3);
        if (t.len < r_cut + hmax) ++p.n_img_sk;
    }
    p.n_img = (int)(img.size() / 3);
    // reciprocal rows b_j = 2 pi (column j of inv), G = m b; half space: first nonzero m positive
    double B[9];
    for (int jx = 0; jx < 3; ++jx)
        for (int k = 0; k < 3; ++k) B[3 * jx + k] = 2.0 * pi * inv[3 * k + jx];
    const double g_max = 2.0 * alpha * EX;
    int M[3];
    for (int i = 0; i < 3; ++i) {   // heights of the reciprocal cell: 2 pi / |a_i|
        const double an = std::sqrt(lat[3 * i] * lat[3 * i] + lat[3 * i + 1] * lat[3 * i + 1] + lat[3 * i + 2] * lat[3 * i + 2]);
        M[i] = (int)std::ceil(g_max * an / (2.0 * pi)) + 1;
    }
    gw.clear();
    for (int m0 = -M[0]; m0 <= M[0]; ++m0)
        for (int m1 = -M[1]; m1 <= M[1]; ++m1)
            for (int m2 = -M[2]; m2 <= M[2]; ++m2) {
                const bool pos = m0 > 0 || (m0 == 0 && (m1 > 0 || (m1 == 0 && m2 > 0)));
                if (!pos) continue;
                double G[3];
                for (int k = 0; k < 3; ++k) G[k] = m0 * B[k] + m1 * B[3 + k] + m2 * B[6 + k];
                const double g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
                if (!(g2 < g_max * g_max)) continue;
                const double w = 4.0 * pi / V * std::exp(-g2 / (4.0 * alpha * alpha)) / g2;
                gw.push_back(G[0]);
                gw.push_back(G[1]);
                gw.push_back(G[2]);
                gw.push_back(2.0 * w);
            }
    p.n_g = (int)(gw.size() / 4);
}

size_t pbc_smem(bool kgrid) { return kgrid ? sizeof(PSharedK) : sizeof(PShared); }

cudaError_t prepare_dftb_periodic() {
    cudaError_t e = cudaFuncSetAttribute(k_dftb_periodic, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PShared));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_dftb_periodic_disp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PShared));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_dftb_periodic_kg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PSharedK));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_dftb_periodic_kg_disp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(PSharedK));
    return e;
}

cudaError_t launch_dftb_periodic(const DevSK *sk_dev, const DftbArgs &a, const PbcPlan &p, cudaStream_t st) {
    if (a.n_cells <= 0) return cudaSuccess;
    PbcDev d;
    for (int k = 0; k < 9; ++k) { d.lat[k] = p.lat[k]; d.inv[k] = p.inv[k]; }
    d.alpha = p.alpha;
    d.bg = p.bg;
    d.self_e = p.self_e;
    d.r_real2 = p.r_real * p.r_real;
    d.n_img = p.n_img;
    d.n_img_sk = p.n_img_sk;
    d.n_g = p.n_g;
    d.nmax = p.nmax;
    d.amax = p.amax;
    d.img = p.d_img;
    d.gw = p.d_gw;
    d.work = p.work;
    d.work_stride = (long long)pbc_workspace_doubles(p.nmax, p.amax, p.n_g, p.nk);
    d.nk = p.nk;
    d.kpt = p.d_kpt;
    const long long items = a.n_disp > 0 ? (long long)a.n_cells * (a.fd_central ? 6 : 3) * p.amax : a.n_cells;
    const int grid = (int)std::min<long long>(items, p.blocks);
    if (p.nk > 0) {
        if (a.n_disp > 0) k_dftb_periodic_kg_disp<<<grid, PT, sizeof(PSharedK), st>>>(sk_dev, a, d);
        else k_dftb_periodic_kg<<<grid, PT, sizeof(PSharedK), st>>>(sk_dev, a, d);
    } else if (a.n_disp > 0) {
        k_dftb_periodic_disp<<<grid, PT, sizeof(PShared), st>>>(sk_dev, a, d);
    } else {
        k_dftb_periodic<<<grid, PT, sizeof(PShared), st>>>(sk_dev, a, d);
    }
    return cudaGetLastError();
}
