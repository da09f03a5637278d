// Batched SCC-DFTB for cells of any composition up to 64 orbitals, e.g. water clusters (H2O)_n
// with n <= 10 (6n orbitals), in one persistent launch per evaluation.
//
// The method is the one of the water kernel in dftb_kernel.cu (second-order SCC-DFTB, section
// "Computational details"): warm-started S-orthonormal basis, SCC iterations with Jacobi sweeps or
// the second-order occupied-virtual update, Anderson mixing, analytic forces. What differs is the
// mapping to the machine, made for matrices too large for a lane group:
//   * work items: a cell of more than 32 orbitals takes a whole 64-thread block (thread j owns
//     orbital column j); smaller cells take one warp each, two per block. A persistent grid pulls
//     items from a queue ordered by decreasing size, so large cells start first and small ones
//     fill the tail (the item lists are built once on the host);
//   * four n x n matrices per cell in shared memory, sized for the largest cell of each class:
//     SH (the symmetric S in the strict lower triangle, the symmetric H0 in the upper triangle and
//     on the diagonal, since S_ii = 1), C, A and Y. Every matrix product is a column product with
//     eight independent row accumulators, one operand broadcast from shared memory;
//   * the final stage reuses the four buffers for H, C_occ, C_occ^T H C_occ, P, W and the pair
//     gradients, so the energy-weighted density needs no further storage. A (H2O)_8 cell (48
//     orbitals) takes 87 KB, so two large cells share an SM.
#include <algorithm>
#include <vector>

#include "cavmd_internal.cuh"

namespace {

constexpr int GNHIST = 3;
constexpr int G_MAX_SWEEPS = 40;
constexpr double G_JACOBI_TOL = 1e-15;
constexpr double G_MIN_GAP = 1e-3;
constexpr double G_EIG_TOL = 1e-10;
constexpr float G_KMAX_PERT = 1e-4f;
constexpr int CH = 8;       // rows per register block
constexpr int GTPB = 64;    // threads per block

// Shared-memory layout of one cell (byte offsets) for cells of at most nmax orbitals, amax atoms.
struct GLayout {
    int nmax, amax, pmax;
    unsigned SH, C, A, Y, pos, gam, zv, q, qout, qst, shift, shl, hq, hf, red, diag, cs, invd, ints, total;
};

__host__ __device__ inline GLayout g_layout(int nmax, int amax) {
    GLayout L;
    L.nmax = nmax;
    L.amax = amax;
    L.pmax = amax * (amax - 1) / 2 > 0 ? amax * (amax - 1) / 2 : 1;
    const int ld = (nmax % 2 == 0) ? nmax + 1 : nmax;
    const unsigned mat = (unsigned)(nmax * ld + 8) * 8;   // 8 doubles of slack for clamped reads
    const unsigned ymat = mat > (unsigned)L.pmax * 32u ? mat : (unsigned)L.pmax * 32u;   // Y also holds pair gradients
    unsigned o = 0;
    L.SH = o; o += mat;
    L.C = o; o += mat;
    L.A = o; o += mat;
    L.Y = o; o += ymat;
    L.pos = o; o += amax * 3 * 8;
    L.gam = o; o += amax * amax * 8;
    L.zv = o; o += amax * 8;
    L.q = o; o += amax * 8;
    L.qout = o; o += amax * 8;
    L.qst = o; o += amax * 8;
    L.shift = o; o += amax * 8;
    L.shl = o; o += amax * 8;
    L.hq = o; o += GNHIST * amax * 8;
    L.hf = o; o += GNHIST * amax * 8;
    L.red = o; o += nmax * 8;
    L.diag = o; o += nmax * 8;
    L.cs = o; o += (nmax / 2 + 1) * 16;
    L.invd = o; o += nmax * 8;
    L.ints = o;
    // ints: spec[amax], atom_off[amax+1], orb_atom[nmax], occ_list[nmax], occf[nmax], eok[nmax],
    //       pa[pmax], pb[pmax], fl[8]
    o += (unsigned)(2 * amax + 1 + 4 * nmax + 2 * L.pmax + 8) * 4;
    L.total = (o + 15u) & ~15u;
    return L;
}

__device__ __forceinline__ void radial_g(const double *par, double r, const DevSK &sk, double &v, double &dv) {
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

// Round-robin Jacobi schedule for even n (rounds r = 0..n-2; index n-1 meets r).
__device__ __forceinline__ int g_partner(int j, int r, int n, int &slot) {
    const int m = n - 1;
    if (j == m) { slot = 0; return r; }
    if (j == r) { slot = 0; return m; }
    const int dlt = (j - r + m) % m;
    slot = min(dlt, m - dlt);
    return (r - dlt + m) % m;
}

__device__ __forceinline__ void g_pair(int k, int r, int n, int &p, int &q) {
    const int m = n - 1;
    if (k == 0) { p = r; q = m; return; }
    const int x = (r + k) % m, y = (r - k + m) % m;
    p = min(x, y);
    q = max(x, y);
}

// Rotation annihilating a_pq: angle from FP32, (c, s) normalised in FP64 by two Newton steps.
__device__ __forceinline__ void g_jacobi_cs(double app, double aqq, double apq, double &c, double &s) {
    const float d = (float)(aqq - app);
    const float o = 2.0f * (float)apq;
    float t = 0.0f;
    if (o != 0.0f) t = o / (d + copysignf(sqrtf(fmaf(d, d, o * o)), d));
    const float cf = rsqrtf(fmaf(t, t, 1.0f));
    c = (double)cf;
    s = (double)(t * cf);
    for (int it = 0; it < 2; ++it) {
        const double nrm = fma(c, c, s * s);
        const double f = fma(-0.5, nrm, 1.5);
        c *= f;
        s *= f;
    }
}

template <int T>
__device__ __forceinline__ void gsync() {
    if (T == 32) __syncwarp(); else __syncthreads();
}

template <int T>
__device__ __forceinline__ bool gall(bool p) {
    if (T == 32) {
        __syncwarp();
        return __all_sync(CAVMD_FULL_MASK, p);
    }
    return __syncthreads_and(p) != 0;
}

// Column product: for rows i < n_out, epi(i, sum_{k < n_k} X(i, k) Z(k)), with
//   X(i, k) = X[k * xs_k + i * xs_i] (a broadcast read: the same for every thread) and
//   Z(k) = Z[k * zs] (this thread's operand). Rows are done CH at a time with independent
// accumulators; rows past n_out read row n_out - 1 and are dropped.
template <typename Epi>
__device__ __forceinline__ void col_product(int n_out, int n_k, const double *X, int xs_i, int xs_k,
                                            const double *Z, int zs, Epi epi) {
    for (int i0 = 0; i0 < n_out; i0 += CH) {
        int ro[CH];
#pragma unroll
        for (int t = 0; t < CH; ++t) ro[t] = min(i0 + t, n_out - 1) * xs_i;
        double acc[CH];
#pragma unroll
        for (int t = 0; t < CH; ++t) acc[t] = 0.0;
        for (int k = 0; k < n_k; ++k) {
            const double z = Z[k * zs];
            const double *xk = X + k * xs_k;
#pragma unroll
            for (int t = 0; t < CH; ++t) acc[t] = fma(xk[ro[t]], z, acc[t]);
        }
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (i0 + t < n_out) epi(i0 + t, acc[t]);
    }
}

// The same with the occupied columns of C as X and Z: for rows i < n_out,
// epi(i, sum_o C(i, occ[o]) C(jz, occ[o])).
template <typename Epi>
__device__ __forceinline__ void col_product_occ(int n_out, int nocc, const double *C, int LD, const int *occ,
                                                int jz, Epi epi) {
    for (int i0 = 0; i0 < n_out; i0 += CH) {
        int ro[CH];
#pragma unroll
        for (int t = 0; t < CH; ++t) ro[t] = min(i0 + t, n_out - 1);
        double acc[CH];
#pragma unroll
        for (int t = 0; t < CH; ++t) acc[t] = 0.0;
        for (int o = 0; o < nocc; ++o) {
            const double *co = C + occ[o] * LD;
            const double z = co[jz];
#pragma unroll
            for (int t = 0; t < CH; ++t) acc[t] = fma(co[ro[t]], z, acc[t]);
        }
#pragma unroll
        for (int t = 0; t < CH; ++t)
            if (i0 + t < n_out) epi(i0 + t, acc[t]);
    }
}

// One cell (main evaluation, kd < 0) or one displaced copy of it (kd = displacement index),
// evaluated by T threads; j = this thread's index among them.
template <int T>
__device__ void g_molecule(const DevSK &sk, const DftbArgs &a, const GLayout &L, unsigned char *sm, int cell,
                           int kd, int j) {
    const bool disp = kd >= 0;
    const int a0 = a.cell_offset[cell];
    const int nat = a.cell_offset[cell + 1] - a0;
    double *SH = (double *)(sm + L.SH), *C = (double *)(sm + L.C);
    double *A = (double *)(sm + L.A), *Y = (double *)(sm + L.Y);
    double(*pos)[3] = (double(*)[3])(sm + L.pos);
    double *gam = (double *)(sm + L.gam), *zv = (double *)(sm + L.zv), *q = (double *)(sm + L.q);
    double *qout = (double *)(sm + L.qout), *qst = (double *)(sm + L.qst);
    double *shift = (double *)(sm + L.shift), *shl = (double *)(sm + L.shl);
    double *hq = (double *)(sm + L.hq), *hf = (double *)(sm + L.hf), *red = (double *)(sm + L.red);
    double *diag = (double *)(sm + L.diag), *cs = (double *)(sm + L.cs), *invd = (double *)(sm + L.invd);
    int *spec = (int *)(sm + L.ints);
    int *atom_off = spec + L.amax;
    int *orb_atom = atom_off + L.amax + 1;
    int *occ_list = orb_atom + L.nmax;
    int *occf = occ_list + L.nmax;
    int *eok = occf + L.nmax;
    int *pa = eok + L.nmax;
    int *pb = pa + L.pmax;
    int *fl = pb + L.pmax;   // 0 error bits, 2 iterations, 3 occupied orbitals, 4 orbitals, 5 pairs
    const int AM = L.amax;

    if (j < nat) {
        spec[j] = a.species[a0 + j];
        for (int k = 0; k < 3; ++k) pos[j][k] = a.r[3 * (a0 + j) + k];
        if (disp) {   // atom da, component dc, by +h (forward) or +-h (central pairs)
            const int kk = a.fd_central ? kd >> 1 : kd;
            const int da = kk / 3, dc = kk - 3 * (kk / 3);
            const double sg = (a.fd_central && (kd & 1)) ? -1.0 : 1.0;
            if (j == da) pos[j][dc] += sg * a.fd_h;
        }
    }
    gsync<T>();
    if (j == 0) {
        int o = 0;
        double nel = 0.0;
        for (int at = 0; at < nat; ++at) {
            atom_off[at] = o;
            const int no = sk.norb[spec[at]];
            for (int k = 0; k < no; ++k) orb_atom[o + k] = at;
            o += no;
            zv[at] = sk.zval[spec[at]];
            nel += zv[at];
        }
        atom_off[nat] = o;
        fl[0] = 0;
        fl[2] = 0;
        fl[3] = (int)(nel * 0.5 + 0.25);
        fl[4] = o;
        int pi = 0;
        for (int x = 0; x < nat; ++x)
            for (int y = x + 1; y < nat; ++y) { pa[pi] = x; pb[pi] = y; ++pi; }
        fl[5] = pi;
    }
    gsync<T>();
    const int n = fl[4], nocc = fl[3], npair = fl[5];
    const int LD = n + 1;   // n is even (closed shell), so the stride is odd
    const bool act = j < n;
    // S(i, j) and H0(i, j) from the shared buffer: column j below the diagonal, row j above it
    auto s_ij = [&](int i) -> double {
        const double lo = SH[j * LD + i], up = SH[i * LD + j];
        return i == j ? 1.0 : (i > j ? lo : up);
    };
    auto h0_ij = [&](int i) -> double {
        const double lo = SH[j * LD + i], up = SH[i * LD + j];
        return i <= j ? lo : up;
    };

    // ---------------------------------------------------------------- H0, S, gamma
    if (act) {
        const int at = orb_atom[j];
        const int e = spec[at];
        const double eps = (j == atom_off[at]) ? sk.onsite[e][0] : sk.onsite[e][1];
        for (int i = 0; i < n; ++i) SH[j * LD + i] = (i == j) ? eps : 0.0;
    }
    gsync<T>();
    for (int pi = j; pi < npair; pi += T) {
        const int PA = pa[pi], PB = pb[pi];
        const int eA = spec[PA], eB = spec[PB];
        const int oA = atom_off[PA], oB = atom_off[PB];
        const int na = sk.norb[eA], nb = sk.norb[eB];
        const double dx = pos[PB][0] - pos[PA][0], dy = pos[PB][1] - pos[PA][1], dz = pos[PB][2] - pos[PA][2];
        const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
        const double ir = rsqrt_nr(r2);
        const double r = r2 * ir;
        const double ev[3] = {dx * ir, dy * ir, dz * ir};
        for (int t = 0; t < 2; ++t) {
            const double(*tab)[CAVMD_MAX_ELEM][4][4] = t == 0 ? sk.h0 : sk.s;
            // element (mu of A, nu of B), mu < nu: H0 in column nu, S in column mu
            auto put = [&](int mu, int nu, double v) {
                if (t == 0) SH[nu * LD + mu] = v; else SH[mu * LD + nu] = v;
            };
            double v, dv;
            radial_g(tab[eA][eB][CAVMD_SK_SS], r, sk, v, dv);
            put(oA, oB, v);
            if (nb == 4) {
                radial_g(tab[eA][eB][CAVMD_SK_SP], r, sk, v, dv);
                for (int i = 0; i < 3; ++i) put(oA, oB + 1 + i, ev[i] * v);
            }
            if (na == 4) {
                radial_g(tab[eB][eA][CAVMD_SK_SP], r, sk, v, dv);
                for (int i = 0; i < 3; ++i) put(oA + 1 + i, oB, -ev[i] * v);
            }
            if (na == 4 && nb == 4) {
                double vs, vp;
                radial_g(tab[eA][eB][CAVMD_SK_PPS], r, sk, vs, dv);
                radial_g(tab[eA][eB][CAVMD_SK_PPP], r, sk, vp, dv);
                const double dl = vs - vp;
                for (int i = 0; i < 3; ++i)
                    for (int k = 0; k < 3; ++k) put(oA + 1 + i, oB + 1 + k, fma(ev[i] * ev[k], dl, (i == k) ? vp : 0.0));
            }
        }
    }
    for (int e2 = j; e2 < nat * nat; e2 += T) {
        const int x = e2 / nat, y = e2 - x * nat;
        const double Ua = sk.hubbard[spec[x]], Ub = sk.hubbard[spec[y]];
        if (x == y) {
            gam[x * AM + y] = Ua;
        } else {
            const double dx = pos[y][0] - pos[x][0], dy = pos[y][1] - pos[x][1], dz = pos[y][2] - pos[x][2];
            const double cc = 2.0 / (Ua + Ub);
            gam[x * AM + y] = rsqrt_nr(fma(dx, dx, fma(dy, dy, fma(dz, dz, cc * cc))));
        }
    }

    // ---------------------------------------------------------------- warm-started S-orthonormal basis
    const long long coff = a.Cwarm_off ? a.Cwarm_off[cell] : (long long)cell * 36;
    const double *cw = a.Cwarm + coff;
    if (a.have_warm) {
        for (int e2 = j; e2 < n * n; e2 += T) {   // coalesced copy of the previous eigenvectors
            const int c = e2 / n;
            C[c * LD + (e2 - c * n)] = cw[e2];
        }
    } else if (act) {
        for (int i = 0; i < n; ++i) C[j * LD + i] = (i == j) ? 1.0 : 0.0;
    }
    if (j < nat) {
        if (a.have_warm) {   // predictor 2 q(t) - q(t - dt); displaced copies start from q(t)
            const double qt = a.qpop[a0 + j];
            qst[j] = qt;
            q[j] = disp ? qt : fma(2.0, qt, -a.qprev[a0 + j]);
        } else {
            q[j] = zv[j];
        }
    }
    gsync<T>();
    if (act)   // S, full, into A
        for (int i = 0; i < n; ++i) A[j * LD + i] = s_ij(i);
    if (a.have_warm) {
        gsync<T>();
        if (act)   // Y = S C
            col_product(n, n, A, 1, LD, C + j * LD, 1, [&](int i, double v) { Y[j * LD + i] = v; });
        gsync<T>();
        if (act)   // A = C^T Y
            col_product(n, n, C, LD, 1, Y + j * LD, 1, [&](int i, double v) { A[j * LD + i] = v; });
    }
    gsync<T>();
    for (int k = 0; k < n; ++k) {   // Cholesky A = L L^T, right-looking, thread = column
        if (j == k) {
            double d = A[k * LD + k];
            if (!(d > 1e-300)) { atomicOr(&fl[0], ERRBIT_S_NOT_PD); d = 1.0; }
            const double y = rsqrt_nr(d);
            invd[k] = y;
            A[k * LD + k] = d * y;
            for (int i = k + 1; i < n; ++i) A[k * LD + i] *= y;
        }
        gsync<T>();
        if (act && j > k) {
            const double ljk = A[k * LD + j];
            for (int i = j; i < n; ++i) A[j * LD + i] = fma(-A[k * LD + i], ljk, A[j * LD + i]);
        }
        gsync<T>();
    }
    if (act) {   // C <- C L^-T, thread = row
        const int i = j;
        for (int c = 0; c < n; ++c) {
            double x = C[c * LD + i];
            for (int k = 0; k < c; ++k) x = fma(-C[k * LD + i], A[k * LD + c], x);
            C[c * LD + i] = x * invd[c];
        }
    }
    gsync<T>();

    // ---------------------------------------------------------------- SCC loop
    int it;
    for (it = 1; it <= a.max_iter; ++it) {
        if (j < nat) {
            double sh = 0.0;
            for (int k = 0; k < nat; ++k) sh = fma(gam[j * AM + k], q[k] - zv[k], sh);
            shift[j] = sh;
        }
        gsync<T>();
        if (act) {   // H column j into A
            const double shj = shift[orb_atom[j]];
            for (int i = 0; i < n; ++i) A[j * LD + i] = fma(0.5 * s_ij(i), shift[orb_atom[i]] + shj, h0_ij(i));
        }
        gsync<T>();
        if (act)   // Y = H C
            col_product(n, n, A, 1, LD, C + j * LD, 1, [&](int i, double v) { Y[j * LD + i] = v; });
        gsync<T>();
        if (act)   // A = C^T Y
            col_product(n, n, C, LD, 1, Y + j * LD, 1, [&](int i, double v) { A[j * LD + i] = v; });
        gsync<T>();
        if (act) {   // aufbau occupation from the diagonal
            const double ajj = A[j * LD + j];
            diag[j] = ajj;
            const long long kj = order_key(ajj);
            int rank = 0;
            for (int i = 0; i < n; ++i) {
                const long long ki = order_key(A[i * LD + i]);
                rank += (ki < kj) || (ki == kj && i < j);
            }
            occf[j] = rank < nocc;
            if (rank < nocc) occ_list[rank] = j;
        }
        gsync<T>();
        float kmax = 0.0f;
        if (act) {   // occupied-virtual generator, column j, into Y (FP32: it only steers)
            const int oj = occf[j];
            const double ajj = A[j * LD + j];
            bool small = true;
            for (int k = 0; k < n; ++k) {
                double kv = 0.0;
                if (occf[k] != oj) {
                    const double akj = A[j * LD + k];
                    if (!abs_lt(akj, G_EIG_TOL)) small = false;
                    float kf = (float)akj / (float)(ajj - A[k * LD + k]);
                    if (!(fabsf(kf) <= 1e30f)) kf = 1e30f;
                    kv = (double)kf;
                    kmax = fmaxf(kmax, fabsf(kf));
                }
                Y[j * LD + k] = kv;
            }
            eok[j] = small;
        }
        const bool cold_first = !a.have_warm && it == 1;
        const bool perturb = gall<T>(!act || (kmax < G_KMAX_PERT && !cold_first));
        if (perturb) {
            if (act)   // V = I + K + K^2 / 2, column j, into A
                col_product(n, n, Y, 1, LD, Y + j * LD, 1, [&](int i, double v) {
                    A[j * LD + i] = fma(0.5, v, Y[j * LD + i] + (i == j ? 1.0 : 0.0));
                });
            gsync<T>();
            if (act)   // C V into Y
                col_product(n, n, C, 1, LD, A + j * LD, 1, [&](int i, double v) { Y[j * LD + i] = v; });
            gsync<T>();
            if (act)
                for (int i = 0; i < n; ++i) C[j * LD + i] = Y[j * LD + i];
            gsync<T>();
        } else {
            const int sweeps = cold_first ? G_MAX_SWEEPS : 1;
            for (int sweep = 0; sweep < G_MAX_SWEEPS; ++sweep) {
                bool small = true;
                if (act)
                    for (int i = 0; i < n; ++i)
                        if (i != j && !abs_lt(A[j * LD + i], G_JACOBI_TOL)) small = false;
                if (gall<T>(small)) break;
                if (sweep >= sweeps) break;
                if (sweep == G_MAX_SWEEPS - 1) {
                    if (act && !small) atomicOr(&fl[0], ERRBIT_TIMEOUT);
                    break;
                }
                for (int rd = 0; rd < n - 1; ++rd) {
                    int p = 0, qq = 0;
                    double cp = 0.0, cq = 0.0;
                    if (act) {
                        int slot;
                        const int pj = g_partner(j, rd, n, slot);
                        p = min(j, pj);
                        qq = max(j, pj);
                        double c, s;
                        g_jacobi_cs(A[p * LD + p], A[qq * LD + qq], A[qq * LD + p], c, s);
                        cp = (j == p) ? c : s;     // new column j = cp col p + cq col q
                        cq = (j == p) ? -s : c;
                        if (j == p) { cs[2 * slot] = c; cs[2 * slot + 1] = s; }
                    }
                    // columns in blocks of CH rows: read the pair's block, wait, write column j's
                    for (int i0 = 0; i0 < n; i0 += CH) {
                        double na[CH], nc[CH];
                        if (act) {
#pragma unroll
                            for (int t = 0; t < CH; ++t) {
                                const int i = min(i0 + t, n - 1);
                                na[t] = fma(cp, A[p * LD + i], cq * A[qq * LD + i]);
                                nc[t] = fma(cp, C[p * LD + i], cq * C[qq * LD + i]);
                            }
                        }
                        gsync<T>();
                        if (act) {
#pragma unroll
                            for (int t = 0; t < CH; ++t) {
                                if (i0 + t < n) {
                                    A[j * LD + i0 + t] = na[t];
                                    C[j * LD + i0 + t] = nc[t];
                                }
                            }
                        }
                    }
                    if (act) {   // rows of column j, for every pair of the round
                        for (int k = 0; k < n / 2; ++k) {
                            int pk, qk;
                            g_pair(k, rd, n, pk, qk);
                            const double ck = cs[2 * k], sk_ = cs[2 * k + 1];
                            const double x = A[j * LD + pk], y = A[j * LD + qk];
                            A[j * LD + pk] = fma(ck, x, -sk_ * y);
                            A[j * LD + qk] = fma(sk_, x, ck * y);
                        }
                    }
                    gsync<T>();
                }
            }
            if (act) {
                const double ajj = A[j * LD + j];
                diag[j] = ajj;
                const long long kj = order_key(ajj);
                int rank = 0;
                for (int i = 0; i < n; ++i) {
                    const long long ki = order_key(A[i * LD + i]);
                    rank += (ki < kj) || (ki == kj && i < j);
                }
                occf[j] = rank < nocc;
                if (rank < nocc) occ_list[rank] = j;
            }
            gsync<T>();
        }
        if (act) {   // Mulliken population of orbital j: (P S)_jj, P = 2 C_occ C_occ^T
            double qo = 0.0;
            col_product_occ(n, nocc, C, LD, occ_list, j, [&](int i, double v) { qo = fma(2.0 * v, s_ij(i), qo); });
            red[j] = qo;
        }
        gsync<T>();
        const int hs = (it - 1) % GNHIST;
        if (j < nat) {
            double qa = 0.0;
            for (int o = atom_off[j]; o < atom_off[j + 1]; ++o) qa += red[o];
            qout[j] = qa;
            shl[j] = shift[j];
            hq[hs * AM + j] = q[j];
            hf[hs * AM + j] = qa - q[j];
        }
        gsync<T>();
        bool conv = true;
        for (int at = 0; at < nat; ++at)
            if (!abs_lt(hf[hs * AM + at], a.scc_tol)) conv = false;
        for (int c = 0; c < n; ++c) conv = conv && eok[c];
        if (j < nat) {
            if (conv) {
                q[j] = qout[j];
            } else {   // Anderson mixing over the last GNHIST iterates (coefficients in FP32)
                float th1 = 0.0f, th2 = 0.0f;
                const int h = min(it, GNHIST);
                const int h1 = (hs + GNHIST - 1) % GNHIST, h2 = (hs + GNHIST - 2) % GNHIST;
                if (h >= 2) {
                    float a11 = 0.f, a12 = 0.f, a22 = 0.f, b1 = 0.f, b2 = 0.f;
                    for (int at = 0; at < nat; ++at) {
                        const float f0 = (float)hf[hs * AM + at];
                        const float d1 = (float)(hf[h1 * AM + at] - hf[hs * AM + at]);
                        const float d2 = h >= 3 ? (float)(hf[h2 * AM + at] - hf[hs * AM + at]) : 0.f;
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
                const double t1 = th1, t2 = th2;
                const double q0 = hq[hs * AM + j], f0 = hf[hs * AM + j];
                double qb = q0, fb = f0;
                if (h >= 2) { qb = fma(t1, hq[h1 * AM + j] - q0, qb); fb = fma(t1, hf[h1 * AM + j] - f0, fb); }
                if (h >= 3) { qb = fma(t2, hq[h2 * AM + j] - q0, qb); fb = fma(t2, hf[h2 * AM + j] - f0, fb); }
                q[j] = fma(a.beta, fb, qb);
            }
        }
        gsync<T>();   // the next iteration's shifts read every atom's charge
        if (conv) {   // the same value in every thread: all leave together
            if (j == 0) fl[2] = it;
            break;
        }
    }
    gsync<T>();
    if (j == 0 && it > a.max_iter) {
        atomicOr(&fl[0], ERRBIT_SCC_NOCONV);
        fl[2] = a.max_iter;
    }
    gsync<T>();

    if (disp) {   // displaced copy: only the dipole of the converged charges
        if (j == 0) {
            double mu[3] = {0.0, 0.0, 0.0};
            for (int at = 0; at < nat; ++at) {
                const double Q = zv[at] - q[at];
                for (int k = 0; k < 3; ++k) mu[k] = fma(Q, pos[at][k] - pos[0][k], mu[k]);
            }
            a.M_disp[(long long)(a.fd_central ? 6 : 3) * a0 + kd] = fma(a.pol0, mu[0], fma(a.pol1, mu[1], a.pol2 * mu[2]));
            if (fl[0]) atomicOr(a.status, (unsigned)fl[0]);
        }
        gsync<T>();
        return;
    }

    // ---------------------------------------------------------------- energy, forces, dipole
    {   // eigenvectors for the next warm start
        double *cwo = a.Cwarm + coff;
        for (int e2 = j; e2 < n * n; e2 += T) {
            const int c = e2 / n;
            cwo[e2] = C[c * LD + (e2 - c * n)];
        }
    }
    if (j < nat) {
        double sh = 0.0;
        for (int k = 0; k < nat; ++k) sh = fma(gam[j * AM + k], q[k] - zv[k], sh);
        shift[j] = sh;
    }
    // W = 2 C_occ (C_occ^T H C_occ) C_occ^T with the H of the last iteration and the whole occupied
    // block; buffers: A <- H; Y <- T = H C_occ; A <- C_occ; C <- Aoo = C_occ^T T;
    // Y <- t = 2 Aoo C_occ^T; C <- P (band energy with H0); SH <- W = C_occ t; Y <- pair gradients
    if (act) {
        const double shj = shl[orb_atom[j]];
        for (int i = 0; i < n; ++i) A[j * LD + i] = fma(0.5 * s_ij(i), shl[orb_atom[i]] + shj, h0_ij(i));
    }
    gsync<T>();
    if (j < nocc)
        col_product(n, n, A, 1, LD, C + occ_list[j] * LD, 1, [&](int i, double v) { Y[j * LD + i] = v; });
    gsync<T>();
    if (j < nocc)
        for (int i = 0; i < n; ++i) A[j * LD + i] = C[occ_list[j] * LD + i];
    gsync<T>();
    if (j < nocc)
        col_product(nocc, n, A, LD, 1, Y + j * LD, 1, [&](int i, double v) { C[j * LD + i] = v; });
    gsync<T>();
    if (act)
        col_product(nocc, nocc, C, 1, LD, A + j, LD, [&](int i, double v) { Y[j * LD + i] = 2.0 * v; });
    if (j == 0 && nocc < n) {   // HOMO-LUMO gap of the last iteration
        double homo = -1e300, lumo = 1e300;
        for (int c = 0; c < n; ++c) {
            if (occf[c]) homo = fmax(homo, diag[c]); else lumo = fmin(lumo, diag[c]);
        }
        if (!(lumo - homo > G_MIN_GAP)) atomicOr(&fl[0], ERRBIT_ZERO_GAP);
    }
    gsync<T>();
    if (act) {
        double eb = 0.0;
        col_product(n, nocc, A, 1, LD, A + j, LD, [&](int i, double v) {
            C[j * LD + i] = 2.0 * v;
            eb = fma(2.0 * v, h0_ij(i), eb);
        });
        red[j] = eb;
    }
    gsync<T>();
    if (act)
        col_product(n, nocc, A, 1, LD, Y + j * LD, 1, [&](int i, double v) { SH[j * LD + i] = v; });
    gsync<T>();
    const double *P = C, *W = SH;
    double *gp = Y, *ep = Y + 3 * L.pmax;
    for (int pi = j; pi < npair; pi += T) {
        const int PA = pa[pi], PB = pb[pi];
        const int eA = spec[PA], eB = spec[PB];
        const int oA = atom_off[PA], oB = atom_off[PB];
        const int na = sk.norb[eA], nb = sk.norb[eB];
        const double dx = pos[PB][0] - pos[PA][0], dy = pos[PB][1] - pos[PA][1], dz = pos[PB][2] - pos[PA][2];
        const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
        const double ir = rsqrt_nr(r2);
        const double r = r2 * ir;
        const double e[3] = {dx * ir, dy * ir, dz * ir};
        const double hshift = 0.5 * (shl[PA] + shl[PB]);
        double gk[3] = {0.0, 0.0, 0.0};
        for (int t = 0; t < 2; ++t) {
            const double(*tab)[CAVMD_MAX_ELEM][4][4] = t == 0 ? sk.h0 : sk.s;
            // weights of the (A, B) block: P for H0, P (eps_A + eps_B)/2 - W for S
            auto wt = [&](int mu, int nu) -> double {
                const double pv = P[nu * LD + mu];
                return t == 0 ? pv : fma(pv, hshift, -W[nu * LD + mu]);
            };
            double v, dv;
            radial_g(tab[eA][eB][CAVMD_SK_SS], r, sk, v, dv);
            {
                const double w = wt(oA, oB) * dv;
                for (int k = 0; k < 3; ++k) gk[k] = fma(w, e[k], gk[k]);
            }
            if (nb == 4) {
                radial_g(tab[eA][eB][CAVMD_SK_SP], r, sk, v, dv);
                double w[3], we = 0.0;
                for (int i = 0; i < 3; ++i) { w[i] = wt(oA, oB + 1 + i); we = fma(w[i], e[i], we); }
                for (int k = 0; k < 3; ++k) gk[k] += fma(w[k] - we * e[k], v * ir, we * e[k] * dv);
            }
            if (na == 4) {
                radial_g(tab[eB][eA][CAVMD_SK_SP], r, sk, v, dv);
                double w[3], we = 0.0;
                for (int i = 0; i < 3; ++i) { w[i] = wt(oA + 1 + i, oB); we = fma(w[i], e[i], we); }
                for (int k = 0; k < 3; ++k) gk[k] -= fma(w[k] - we * e[k], v * ir, we * e[k] * dv);
            }
            if (na == 4 && nb == 4) {
                double vs, dvs, vp, dvp;
                radial_g(tab[eA][eB][CAVMD_SK_PPS], r, sk, vs, dvs);
                radial_g(tab[eA][eB][CAVMD_SK_PPP], r, sk, vp, dvp);
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
                    gk[k] += (We[k] + WTe[k] - 2.0 * eWe * e[k]) * dl * ir + eWe * e[k] * ddl + tr * e[k] * dvp;
            }
        }
        for (int k = 0; k < 3; ++k) gk[k] *= 2.0;
        const double Ua = sk.hubbard[eA], Ub = sk.hubbard[eB];
        const double cc = 2.0 / (Ua + Ub);
        const double gi = rsqrt_nr(fma(r, r, cc * cc));
        const double dgam = -r * gi * gi * gi;
        const double qq = (q[PA] - zv[PA]) * (q[PB] - zv[PB]) * dgam;
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
        for (int k = 0; k < 3; ++k) gp[3 * pi + k] = gk[k] + (qq + derep) * e[k];
        ep[pi] = erep;
    }
    gsync<T>();
    if (j < nat) {
        double f[3] = {0.0, 0.0, 0.0};
        for (int pi = 0; pi < npair; ++pi) {
            const double sg = (pb[pi] == j) ? -1.0 : ((pa[pi] == j) ? 1.0 : 0.0);
            if (sg != 0.0)
                for (int k = 0; k < 3; ++k) f[k] = fma(sg, gp[3 * pi + k], f[k]);
        }
        const int at = a0 + j;
        for (int k = 0; k < 3; ++k) a.F[3 * at + k] = f[k];
        a.qprev[at] = a.have_warm ? qst[j] : q[j];
        a.qpop[at] = q[j];
        if (a.Qout) a.Qout[at] = zv[j] - q[j];
        if (a.write_b) {
            const double Q = zv[j] - q[j];
            a.b[3 * at + 0] = Q * a.pol0;
            a.b[3 * at + 1] = Q * a.pol1;
            a.b[3 * at + 2] = Q * a.pol2;
        }
    }
    if (j == 0) {
        double E = 0.0;
        for (int i = 0; i < n; ++i) E += red[i];
        double e2 = 0.0;
        for (int x = 0; x < nat; ++x)
            for (int y = 0; y < nat; ++y) e2 = fma(gam[x * AM + y] * (q[x] - zv[x]), q[y] - zv[y], e2);
        E = fma(0.5, e2, E);
        for (int pi = 0; pi < npair; ++pi) E += ep[pi];
        double mu[3] = {0.0, 0.0, 0.0};
        for (int at = 0; at < nat; ++at) {
            const double Q = zv[at] - q[at];
            for (int k = 0; k < 3; ++k) mu[k] = fma(Q, pos[at][k] - pos[0][k], mu[k]);
        }
        a.E_cell[cell] = E;
        a.M_cell[cell] = fma(a.pol0, mu[0], fma(a.pol1, mu[1], a.pol2 * mu[2]));
        a.iters[cell] = fl[2];
        if (fl[0]) atomicOr(a.status, (unsigned)fl[0]);
    }
    gsync<T>();
}

// Persistent grid over a queue of work units: units [0, n_big) are one large item each (whole
// block), the rest take two small items (one per warp).
__global__ void __launch_bounds__(GTPB) k_dftb_generic(const DevSK *__restrict__ skp, const DftbArgs a,
                                                       const int2 *__restrict__ items, int n_big, int n_small,
                                                       unsigned *__restrict__ queue, int nmax_b, int amax_b,
                                                       int nmax_s, int amax_s) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int next;
    const DevSK &sk = *skp;
    const GLayout Lb = g_layout(nmax_b, amax_b);
    const GLayout Ls = g_layout(nmax_s, amax_s);
    const int n_units = n_big + (n_small + 1) / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) next = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int w = next;
        __syncthreads();
        if (w >= n_units) break;
        if (w < n_big) {
            const int2 it = items[w];
            g_molecule<GTPB>(sk, a, Lb, smem, it.x, it.y, threadIdx.x);
        } else {
            const int s = 2 * (w - n_big) + warp;
            if (s < n_small) {
                const int2 it = items[n_big + s];
                g_molecule<32>(sk, a, Ls, smem + warp * Ls.total, it.x, it.y, lane);
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t dftb_generic_smem(int nmax_b, int amax_b, int nmax_s, int amax_s) {
    const size_t b = nmax_b > 0 ? g_layout(nmax_b, amax_b).total : 0;
    const size_t s = nmax_s > 0 ? 2 * (size_t)g_layout(nmax_s, amax_s).total : 0;
    return std::max(b, s);
}

void plan_dftb_generic(const int *cell_offset, const int *species, const int *norb_of_elem, int n_cells,
                       int n_disp_per_atom, GenericPlan &p, std::vector<int2> &items,
                       std::vector<int2> &disp_items) {
    std::vector<int> order(n_cells), norb(n_cells);
    for (int c = 0; c < n_cells; ++c) {
        int o = 0;
        for (int i = cell_offset[c]; i < cell_offset[c + 1]; ++i) o += norb_of_elem[species[i]];
        norb[c] = o;
        order[c] = c;
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return norb[x] > norb[y]; });
    p.nmax_b = p.amax_b = p.nmax_s = p.amax_s = 0;
    p.n_big = p.n_small = p.n_disp_big = p.n_disp_small = 0;
    items.clear();
    disp_items.clear();
    for (int c : order) {
        const int nat = cell_offset[c + 1] - cell_offset[c];
        const bool big = norb[c] > 32;
        int &nmax = big ? p.nmax_b : p.nmax_s, &amax = big ? p.amax_b : p.amax_s;
        nmax = std::max(nmax, norb[c]);
        amax = std::max(amax, nat);
        (big ? p.n_big : p.n_small) += 1;
        (big ? p.n_disp_big : p.n_disp_small) += n_disp_per_atom * nat;
        items.push_back(make_int2(c, -1));
        for (int k = 0; k < n_disp_per_atom * nat; ++k) disp_items.push_back(make_int2(c, k));
    }
    p.smem = dftb_generic_smem(p.nmax_b, p.amax_b, p.nmax_s, p.amax_s);
}

cudaError_t prepare_dftb_generic(GenericPlan &p) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p.n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_dftb_generic, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p.blocks_per_sm, k_dftb_generic, GTPB, p.smem);
    return e;
}

// Evaluates the items of the plan: the cells, or their displaced copies when a.n_disp > 0.
cudaError_t launch_dftb_generic(const DevSK *sk, const DftbArgs &a, const GenericPlan &p, cudaStream_t st) {
    const bool disp = a.n_disp > 0;
    const int2 *items = disp ? p.disp_items : p.items;
    const int nb = disp ? p.n_disp_big : p.n_big, ns = disp ? p.n_disp_small : p.n_small;
    const int units = nb + (ns + 1) / 2;
    if (units <= 0) return cudaSuccess;
    unsigned *queue = p.queue + (disp ? 1 : 0);
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const int grid = std::min(units, p.n_sm * std::max(p.blocks_per_sm, 1));
    k_dftb_generic<<<grid, GTPB, p.smem, st>>>(sk, a, items, nb, ns, queue, p.nmax_b, p.amax_b, p.nmax_s,
                                               p.amax_s);
    return cudaGetLastError();
}
