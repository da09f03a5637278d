// Batched SCC-DFTB for cells of any composition up to 64 orbitals, e.g. water clusters (H2O)_n
// with n <= 10 (6n orbitals), in one persistent launch per evaluation.
//
// The method is the one of the water kernel in dftb_kernel.cu (second-order SCC-DFTB, section
// "Computational details"): warm-started S-orthonormal basis, SCC iterations with Jacobi sweeps or
// the second-order occupied-virtual update, Anderson mixing, analytic forces. The mapping to the
// machine is made for matrices too large for a lane group, on a GPU whose FP64 pipe (2 FMA per
// clock per SM) is the only bottleneck, so what counts is the number of FP64 warp instructions:
//   * work items: a cell of more than 32 orbitals takes a whole 128-thread block, smaller cells
//     take 64 threads each, two per block. A persistent grid pulls items from a queue ordered by
//     decreasing size, so large cells start first and small ones fill the tail;
//   * every matrix product spreads its output entries evenly over the cell's threads (R entries
//     per thread per pass, each summed over k in increasing order), so nearly every lane of
//     every FP64 instruction does useful work whatever the orbital count; the results do not
//     depend on R or on the grid size;
//   * per SCC iteration only what the update needs is formed: H C, the diagonal and the
//     occupied-virtual block of C^T H C, K^2 in its two diagonal blocks from the compact
//     occupied-virtual generator, C V, and S C_occ for the Mulliken populations;
//   * four n x n matrices per cell in shared memory: SH (the symmetric S in the strict lower
//     triangle, the symmetric H0 in the upper triangle and on the diagonal, since S_ii = 1),
//     C, A and Y, plus the compact generator. A (H2O)_8 cell (48 orbitals) takes about 92 KB, so
//     two large cells share an SM.
#include <algorithm>
#include <vector>

#include "cavmd_internal.cuh"

namespace {

constexpr int GNHIST = 6;              // largest Anderson history (current + 5 previous iterates)
constexpr int G_MAX_SWEEPS = 40;            // default bound on the Jacobi sweeps of a cold start
constexpr double G_JACOBI_TOL = 1e-15;
constexpr double G_MIN_GAP = 1e-3;
constexpr double G_EIG_TOL = 1e-10;
constexpr float G_KMAX_PERT = 1e-4f;
constexpr int BT = 128;                // threads per block
constexpr int TB = 128;                // threads per large cell
constexpr int TS = 64;                 // threads per small cell (two per block)

// Shared-memory layout of one cell (byte offsets) for cells of at most nmax orbitals, amax atoms.
struct GLayout {
    int nmax, amax, pmax;
    unsigned SH, C, A, Y, Kc, pos, gam, zv, q, qout, qst, shift, shl, hq, hf, red, diag, cs, invd, th, ints,
        total;
};

__host__ __device__ inline GLayout g_layout(int nmax, int amax) {
    GLayout L;
    L.nmax = nmax;
    L.amax = amax;
    L.pmax = amax * (amax - 1) / 2 > 0 ? amax * (amax - 1) / 2 : 1;
    const int ld = nmax + 1;
    const unsigned mat = (unsigned)(nmax * ld + 8) * 8;   // 8 doubles of slack for clamped reads
    const unsigned ymat = mat > (unsigned)L.pmax * 32u ? mat : (unsigned)L.pmax * 32u;   // pair gradients fit too
    unsigned o = 0;
    L.SH = o; o += mat;
    L.C = o; o += ymat;   // C and Y swap roles: both can hold the pair gradients
    L.A = o; o += mat;
    L.Y = o; o += ymat;
    L.Kc = o; o += (unsigned)((nmax / 2) * ((nmax + 1) / 2) + 8) * 8;   // n_occ x n_virt <= n^2 / 4
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
    L.th = o; o += GNHIST * 8;
    L.ints = o;
    // ints: spec[amax], atom_off[amax+1], orb_atom[nmax], occ_list[nmax], virt_list[nmax],
    //       occf[nmax], pp[nmax/2+1], pq[nmax/2+1], pa[pmax], pb[pmax], fl[8]
    o += (unsigned)(2 * amax + 1 + 4 * nmax + 2 * (nmax / 2 + 1) + 2 * L.pmax + 8) * 4;
    L.total = (o + 15u) & ~15u;
    return L;
}

// A group of T threads evaluating one cell: the whole block (T = BT), or one half of it
// (T = 64, named barrier 1 or 2).
template <int T>
struct Grp {
    int tid;
    int bar;
    int *vote;   // T/32 ints of shared scratch (halves only)
    __device__ __forceinline__ void sync() const {
        if (T == BT) __syncthreads();
        else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(T) : "memory");
    }
    __device__ __forceinline__ bool all(bool p) const {
        if (T == BT) return __syncthreads_and(p) != 0;
        const bool w = __all_sync(CAVMD_FULL_MASK, p);
        sync();   // earlier readers of vote are done
        if ((tid & 31) == 0) vote[tid >> 5] = w;
        sync();
        bool r = true;
#pragma unroll
        for (int i = 0; i < T / 32; ++i) r = r && vote[i];
        return r;
    }
};

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

// Round-robin Jacobi schedule for even n: pair k of round r (0..n-2); index n-1 meets r.
__device__ __forceinline__ void g_pair(int k, int r, int n, int &p, int &q) {
    const int m = n - 1;
    if (k == 0) { p = r; q = m; return; }
    const int x = (r + k) % m, y = (r - k + m) % m;
    p = min(x, y);
    q = max(x, y);
}

// Rotation annihilating a_pq: angle from FP32, (c, s) normalised in FP64 by two Newton steps.
__device__ __forceinline__ void g_jacobi_cs(double app, double aqq, double apq, double &c, double &s) {
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

// Flattened dot products: for every entry e < n_out of this thread (e = tid, tid + T, ...),
// epi(e, sum_{k < nk} xb(e)[k xs] zb(e)[k zs]), the sum taken in increasing k. R entries per pass
// with independent accumulators; the last pass clamps its surplus entries to n_out - 1 and drops
// them.
template <int T, int R, typename XB, typename ZB, typename EPI>
__device__ __forceinline__ void flat(int tid, int n_out, int nk, int xs, int zs, XB xb, ZB zb, EPI epi) {
    for (int e0 = tid; e0 < n_out; e0 += T * R) {
        const double *xp[R];
        const double *zp[R];
        double acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = min(e0 + r * T, n_out - 1);
            xp[r] = xb(e);
            zp[r] = zb(e);
            acc[r] = 0.0;
        }
        for (int k = 0; k < nk; ++k) {
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = fma(xp[r][k * xs], zp[r][k * zs], acc[r]);
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (e0 + r * T < n_out) epi(e0 + r * T, acc[r]);
    }
}

// One cell (main evaluation, kd < 0) or one displaced copy of it (kd = displacement index),
// evaluated by the T threads of group g.
template <int T, int R>
__device__ void g_molecule(const DevSK &sk, const DftbArgs &a, const GLayout &L, unsigned char *sm, int cell,
                           int kd, const Grp<T> &g) {
    const int j = g.tid;
    const bool disp = kd >= 0;
    const int a0 = a.cell_offset[cell];
    const int nat = a.cell_offset[cell + 1] - a0;
    double *SH = (double *)(sm + L.SH), *A = (double *)(sm + L.A), *Kc = (double *)(sm + L.Kc);
    double *C = (double *)(sm + L.C), *Y = (double *)(sm + L.Y);   // swapped by the second-order update
    double(*pos)[3] = (double(*)[3])(sm + L.pos);
    double *gam = (double *)(sm + L.gam), *zv = (double *)(sm + L.zv), *q = (double *)(sm + L.q);
    double *qout = (double *)(sm + L.qout), *qst = (double *)(sm + L.qst);
    double *shift = (double *)(sm + L.shift), *shl = (double *)(sm + L.shl);
    double *hq = (double *)(sm + L.hq), *hf = (double *)(sm + L.hf), *red = (double *)(sm + L.red);
    double *diag = (double *)(sm + L.diag), *cs = (double *)(sm + L.cs), *invd = (double *)(sm + L.invd);
    double *th = (double *)(sm + L.th);
    int *spec = (int *)(sm + L.ints);
    int *atom_off = spec + L.amax;
    int *orb_atom = atom_off + L.amax + 1;
    int *occ_list = orb_atom + L.nmax;
    int *virt_list = occ_list + L.nmax;
    int *occf = virt_list + L.nmax;
    int *pp = occf + L.nmax;
    int *pq = pp + (L.nmax / 2 + 1);
    int *pa = pq + (L.nmax / 2 + 1);
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
    g.sync();
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
    g.sync();
    const int n = fl[4], nocc = fl[3], npair = fl[5];
    const int nv = n - nocc;
    const int LD = n + 1;   // n is even (closed shell), so the stride is odd
    const int nn = n * n;
    // S(i, k) and H0(i, k) from the shared buffer: column k below the diagonal, row k above it
    auto s_at = [&](int i, int k) -> double {
        const double lo = SH[k * LD + i], up = SH[i * LD + k];
        return i == k ? 1.0 : (i > k ? lo : up);
    };
    auto h0_at = [&](int i, int k) -> double {
        const double lo = SH[k * LD + i], up = SH[i * LD + k];
        return i <= k ? lo : up;
    };

    // ---------------------------------------------------------------- H0, S, gamma
    for (int e = j; e < nn; e += T) {
        const int c = e / n, i = e - c * n;
        double v = 0.0;
        if (i == c) {
            const int at = orb_atom[c], el = spec[at];
            v = (c == atom_off[at]) ? sk.onsite[el][0] : sk.onsite[el][1];
        }
        SH[c * LD + i] = v;
    }
    g.sync();
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
        if (x == y) {
            gam[x * AM + y] = sk.hubbard[spec[x]];
        } else {
            const double dx = pos[y][0] - pos[x][0], dy = pos[y][1] - pos[x][1], dz = pos[y][2] - pos[x][2];
            gam[x * AM + y] = rsqrt_nr(fma(dx, dx, fma(dy, dy, fma(dz, dz, sk.gamma_c2[spec[x]][spec[y]]))));
        }
    }

    // ---------------------------------------------------------------- warm-started S-orthonormal basis
    const long long coff = a.Cwarm_off ? a.Cwarm_off[cell] : (long long)cell * 36;
    const double *cw = a.Cwarm + coff;
    for (int e = j; e < nn; e += T) {   // coalesced copy of the previous eigenvectors
        const int c = e / n, i = e - c * n;
        C[c * LD + i] = a.have_warm ? cw[e] : (i == c ? 1.0 : 0.0);
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
    g.sync();
    for (int e = j; e < nn; e += T) {   // S, full, into A
        const int c = e / n, i = e - c * n;
        A[c * LD + i] = s_at(i, c);
    }
    if (a.have_warm) {   // A = C^T S C
        g.sync();
        flat<T, R>(j, nn, n, LD, 1, [&](int e) { return A + (e % n); }, [&](int e) { return C + (e / n) * LD; },
                   [&](int e, double v) { Y[(e / n) * LD + e % n] = v; });
        g.sync();
        flat<T, R>(j, nn, n, 1, 1, [&](int e) { return C + (e % n) * LD; }, [&](int e) { return Y + (e / n) * LD; },
                   [&](int e, double v) { A[(e / n) * LD + e % n] = v; });
    }
    g.sync();
    for (int k = 0; k < n; ++k) {   // Cholesky A = L L^T, right-looking, thread = column
        if (j == k) {
            double d = A[k * LD + k];
            if (!(d > 1e-300)) { atomicOr(&fl[0], ERRBIT_S_NOT_PD); d = 1.0; }
            const double y = rsqrt_nr(d);
            invd[k] = y;
            A[k * LD + k] = d * y;
            for (int i = k + 1; i < n; ++i) A[k * LD + i] *= y;
        }
        g.sync();
        if (j > k && j < n) {
            const double ljk = A[k * LD + j];
            for (int i = j; i < n; ++i) A[j * LD + i] = fma(-A[k * LD + i], ljk, A[j * LD + i]);
        }
        g.sync();
    }
    if (j < n) {   // C <- C L^-T, thread = row
        const int i = j;
        for (int c = 0; c < n; ++c) {
            double x = C[c * LD + i];
            for (int k = 0; k < c; ++k) x = fma(-C[k * LD + i], A[k * LD + c], x);
            C[c * LD + i] = x * invd[c];
        }
    }
    g.sync();

    // aufbau occupation from diag[]: occupied and virtual index lists in order of rank
    auto rank_occupation = [&]() {
        if (j < n) {
            const long long kj = order_key(diag[j]);
            int rank = 0;
            for (int i = 0; i < n; ++i) {
                const long long ki = order_key(diag[i]);
                rank += (ki < kj) || (ki == kj && i < j);
            }
            occf[j] = rank < nocc;
            if (rank < nocc) occ_list[rank] = j; else virt_list[rank - nocc] = j;
        }
    };

    // ---------------------------------------------------------------- SCC loop
    // Per iteration: H(q) into A; Y = H C; the diagonal of C^T Y, the occupation, the occupied-
    // virtual block of C^T Y and the compact generator K(v, o) = A_vo / (A_oo - A_vv). When every
    // generator entry is below KMAX the basis takes C <- C (I + K + K^2/2) (orthogonal to O(K^4));
    // otherwise the rest of A = C^T H C is formed and Jacobi sweeps move C (one per iteration when
    // warm started, to convergence on a cold start).
    int it;
    for (it = 1; it <= a.max_iter; ++it) {
        if (j < nat) {
            double sh = 0.0;
            for (int k = 0; k < nat; ++k) sh = fma(gam[j * AM + k], q[k] - zv[k], sh);
            shift[j] = sh;
        }
        g.sync();
        for (int e = j; e < nn; e += T) {   // H into A
            const int c = e / n, i = e - c * n;
            A[c * LD + i] = fma(0.5 * s_at(i, c), shift[orb_atom[i]] + shift[orb_atom[c]], h0_at(i, c));
        }
        g.sync();
        flat<T, R>(j, nn, n, LD, 1, [&](int e) { return A + (e % n); }, [&](int e) { return C + (e / n) * LD; },
                   [&](int e, double v) { Y[(e / n) * LD + e % n] = v; });
        g.sync();
        flat<T, R>(j, n, n, 1, 1, [&](int e) { return C + e * LD; }, [&](int e) { return Y + e * LD; },
                   [&](int e, double v) { diag[e] = v; });
        g.sync();
        rank_occupation();
        g.sync();
        // occupied-virtual block of C^T H C (entry e: virtual index e % nv, occupied e / nv)
        bool small = true;
        float kmax = 0.0f;
        flat<T, R>(j, nocc * nv, n, 1, 1, [&](int e) { return C + virt_list[e % nv] * LD; },
                   [&](int e) { return Y + occ_list[e / nv] * LD; }, [&](int e, double v) {
                       const int vi = virt_list[e % nv], oi = occ_list[e / nv];
                       A[oi * LD + vi] = v;
                       A[vi * LD + oi] = v;
                       if (!abs_lt(v, G_EIG_TOL)) small = false;
                       float kf = d2f_steer(v) / d2f_steer(diag[oi] - diag[vi]);
                       if (!(fabsf(kf) <= 1e30f)) kf = 1e30f;   // degenerate or non-finite: Jacobi path
                       kmax = fmaxf(kmax, fabsf(kf));
                       Kc[e] = f2d_steer(kf);   // K(v, o) at [o][v]
                   });
        const bool eok = g.all(small);
        const bool cold_first = !a.have_warm && it == 1;
        const bool perturb = g.all(kmax < G_KMAX_PERT && !cold_first);
        if (perturb) {
            // V = I + K + K^2/2 into A: K(v, o) = Kc[o][v], K(o, v) = -Kc[o][v];
            // (K^2)(o1, o2) = -sum_v Kc[o1][v] Kc[o2][v], (K^2)(v1, v2) = -sum_o Kc[o][v1] Kc[o][v2]
            flat<T, R>(j, nocc * nocc, nv, 1, 1, [&](int e) { return Kc + (e % nocc) * nv; },
                       [&](int e) { return Kc + (e / nocc) * nv; }, [&](int e, double v) {
                           const int o1 = e % nocc, o2 = e / nocc;
                           A[occ_list[o2] * LD + occ_list[o1]] = fma(-0.5, v, o1 == o2 ? 1.0 : 0.0);
                       });
            flat<T, R>(j, nv * nv, nocc, nv, nv, [&](int e) { return Kc + (e % nv); },
                       [&](int e) { return Kc + (e / nv); }, [&](int e, double v) {
                           const int v1 = e % nv, v2 = e / nv;
                           A[virt_list[v2] * LD + virt_list[v1]] = fma(-0.5, v, v1 == v2 ? 1.0 : 0.0);
                       });
            for (int e = j; e < nocc * nv; e += T) {
                const int vi = virt_list[e % nv], oi = occ_list[e / nv];
                const double k = Kc[e];
                A[oi * LD + vi] = k;    // V(v, o) = K(v, o)
                A[vi * LD + oi] = -k;   // V(o, v) = K(o, v)
            }
            g.sync();
            flat<T, R>(j, nn, n, LD, 1, [&](int e) { return C + (e % n); }, [&](int e) { return A + (e / n) * LD; },
                       [&](int e, double v) { Y[(e / n) * LD + e % n] = v; });
            g.sync();
            double *t = C;
            C = Y;
            Y = t;
        } else {
            // the rest of C^T H C: the occupied and virtual diagonal blocks
            flat<T, R>(j, nocc * nocc, n, 1, 1, [&](int e) { return C + occ_list[e % nocc] * LD; },
                       [&](int e) { return Y + occ_list[e / nocc] * LD; },
                       [&](int e, double v) { A[occ_list[e / nocc] * LD + occ_list[e % nocc]] = v; });
            flat<T, R>(j, nv * nv, n, 1, 1, [&](int e) { return C + virt_list[e % nv] * LD; },
                       [&](int e) { return Y + virt_list[e / nv] * LD; },
                       [&](int e, double v) { A[virt_list[e / nv] * LD + virt_list[e % nv]] = v; });
            g.sync();
            // a cold start sweeps until the off-diagonal entries are below tolerance, at most `cap`
            // sweeps (then DEVICE_TIMEOUT); later iterations take one sweep
            const int cap = cold_first ? (a.max_sweeps > 0 ? a.max_sweeps : G_MAX_SWEEPS) : 1;
            for (int sweep = 0;; ++sweep) {
                bool off_small = true;
                for (int e = j; e < nn; e += T) {
                    const int c = e / n, i = e - c * n;
                    if (i != c && !abs_lt(A[c * LD + i], G_JACOBI_TOL)) off_small = false;
                }
                if (g.all(off_small)) break;
                if (sweep >= cap) {
                    if (cold_first && j == 0) atomicOr(&fl[0], ERRBIT_TIMEOUT);
                    break;
                }
                for (int rd = 0; rd < n - 1; ++rd) {
                    if (j < n / 2) {   // the rotations of this round
                        int p, qq;
                        g_pair(j, rd, n, p, qq);
                        double c, s;
                        g_jacobi_cs(A[p * LD + p], A[qq * LD + qq], A[qq * LD + p], c, s);
                        pp[j] = p;
                        pq[j] = qq;
                        cs[2 * j] = c;
                        cs[2 * j + 1] = s;
                    }
                    g.sync();
                    for (int e = j; e < n * (n / 2); e += T) {   // columns p, q of A and C, row i
                        const int k = e / n, i = e - k * n;
                        const int p = pp[k], qq = pq[k];
                        const double c = cs[2 * k], s = cs[2 * k + 1];
                        const double ap = A[p * LD + i], aq = A[qq * LD + i];
                        A[p * LD + i] = fma(c, ap, -s * aq);
                        A[qq * LD + i] = fma(s, ap, c * aq);
                        const double cp = C[p * LD + i], cq = C[qq * LD + i];
                        C[p * LD + i] = fma(c, cp, -s * cq);
                        C[qq * LD + i] = fma(s, cp, c * cq);
                    }
                    g.sync();
                    for (int e = j; e < n * (n / 2); e += T) {   // rows p, q of A, column c
                        const int k = e / n, c = e - k * n;
                        const int p = pp[k], qq = pq[k];
                        const double ck = cs[2 * k], sk_ = cs[2 * k + 1];
                        const double x = A[c * LD + p], y = A[c * LD + qq];
                        A[c * LD + p] = fma(ck, x, -sk_ * y);
                        A[c * LD + qq] = fma(sk_, x, ck * y);
                    }
                    g.sync();
                }
            }
            if (j < n) diag[j] = A[j * LD + j];
            g.sync();
            rank_occupation();
            g.sync();
        }
        // Mulliken populations: (P S)_ii = 2 sum_o C(i, o) (S C)(i, o); S C_occ into A
        for (int e = j; e < n * nocc; e += T) {
            const int o = e / n, i = e - o * n;
            const double *co = C + occ_list[o] * LD;
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc = fma(s_at(i, k), co[k], acc);
            A[o * LD + i] = acc;
        }
        g.sync();
        if (j < n) {
            double qo = 0.0;
            for (int o = 0; o < nocc; ++o) qo = fma(C[occ_list[o] * LD + j], A[o * LD + j], qo);
            red[j] = 2.0 * qo;
        }
        g.sync();
        const int NH = a.hist;   // ring of the last NH iterates
        const int hs = (it - 1) % NH;
        if (j < nat) {
            double qa = 0.0;
            for (int o = atom_off[j]; o < atom_off[j + 1]; ++o) qa += red[o];
            qout[j] = qa;
            shl[j] = shift[j];
            hq[hs * AM + j] = q[j];
            hf[hs * AM + j] = qa - q[j];
        }
        g.sync();
        bool conv = eok;
        for (int at = 0; at < nat; ++at)
            if (!abs_lt(hf[hs * AM + at], a.scc_tol)) conv = false;
        const int h = min(it, NH);
        if (!conv && j == 0) {
            // Anderson coefficients over the h - 1 previous iterates: normal equations in FP32 with
            // a small diagonal shift, solved by Cholesky (they only steer the iteration)
            float Mx[GNHIST - 1][GNHIST - 1], bv[GNHIST - 1], x[GNHIST - 1];
            const int m = h - 1;
            for (int u = 0; u < m; ++u) {
                const int hu = (hs + NH - 1 - u) % NH;
                float b = 0.f;
                for (int w = 0; w <= u; ++w) {
                    const int hw = (hs + NH - 1 - w) % NH;
                    float s = 0.f;
                    for (int at = 0; at < nat; ++at) {
                        const float du = d2f_steer(hf[hu * AM + at] - hf[hs * AM + at]);
                        const float dw = d2f_steer(hf[hw * AM + at] - hf[hs * AM + at]);
                        s = fmaf(du, dw, s);
                    }
                    Mx[u][w] = s;
                }
                for (int at = 0; at < nat; ++at)
                    b = fmaf(-d2f_steer(hf[hu * AM + at] - hf[hs * AM + at]), d2f_steer(hf[hs * AM + at]), b);
                bv[u] = b;
            }
            float dmax = 0.f;
            for (int u = 0; u < m; ++u) dmax = fmaxf(dmax, Mx[u][u]);
            bool ok = m > 0 && dmax > 0.f;
            for (int u = 0; u < m && ok; ++u) {   // lower Cholesky factor of M + 1e-6 max(diag) I, in place
                for (int w = 0; w <= u && ok; ++w) {
                    float s = Mx[u][w] + (u == w ? 1e-6f * dmax : 0.f);
                    for (int l = 0; l < w; ++l) s -= Mx[u][l] * Mx[w][l];
                    if (u == w) {
                        if (!(s > 0.f)) ok = false; else Mx[u][u] = sqrtf(s);
                    } else {
                        Mx[u][w] = s / Mx[w][w];
                    }
                }
            }
            if (ok) {
                for (int u = 0; u < m; ++u) {
                    float s = bv[u];
                    for (int l = 0; l < u; ++l) s -= Mx[u][l] * x[l];
                    x[u] = s / Mx[u][u];
                }
                for (int u = m - 1; u >= 0; --u) {
                    float s = x[u];
                    for (int l = u + 1; l < m; ++l) s -= Mx[l][u] * x[l];
                    x[u] = s / Mx[u][u];
                }
                for (int u = 0; u < m; ++u)
                    if (!(fabsf(x[u]) < 50.f)) ok = false;
            }
            for (int u = 0; u < GNHIST - 1; ++u) th[u] = (ok && u < m) ? f2d_steer(x[u]) : 0.0;
        }
        g.sync();
        if (j < nat) {
            if (conv) {
                q[j] = qout[j];
            } else {
                const double q0 = hq[hs * AM + j], f0 = hf[hs * AM + j];
                double qb = q0, fb = f0;
                for (int u = 0; u < h - 1; ++u) {
                    const int hu = (hs + NH - 1 - u) % NH;
                    qb = fma(th[u], hq[hu * AM + j] - q0, qb);
                    fb = fma(th[u], hf[hu * AM + j] - f0, fb);
                }
                q[j] = fma(a.beta, fb, qb);
            }
        }
        g.sync();   // the next iteration's shifts read every atom's charge
        if (conv) {   // the same value in every thread: all leave together
            if (j == 0) fl[2] = it;
            break;
        }
    }
    g.sync();
    if (j == 0 && it > a.max_iter) {
        atomicOr(&fl[0], ERRBIT_SCC_NOCONV);
        fl[2] = a.max_iter;
    }
    g.sync();

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
        g.sync();
        return;
    }

    // ---------------------------------------------------------------- energy, forces, dipole
    {   // eigenvectors for the next warm start
        double *cwo = a.Cwarm + coff;
        for (int e = j; e < nn; e += T) {
            const int c = e / n;
            cwo[e] = C[c * LD + (e - c * n)];
        }
    }
    if (j < nat) {
        double sh = 0.0;
        for (int k = 0; k < nat; ++k) sh = fma(gam[j * AM + k], q[k] - zv[k], sh);
        shift[j] = sh;
    }
    // W = 2 C_occ (C_occ^T H C_occ) C_occ^T with the H of the last iteration and the whole occupied
    // block. Buffers: A <- H; Y <- T = H C_occ; A <- C_occ; C <- Aoo = C_occ^T T;
    // Y <- t = 2 Aoo C_occ^T; C <- P; SH <- W = C_occ t; Y <- pair gradients
    for (int e = j; e < nn; e += T) {
        const int c = e / n, i = e - c * n;
        A[c * LD + i] = fma(0.5 * s_at(i, c), shl[orb_atom[i]] + shl[orb_atom[c]], h0_at(i, c));
    }
    g.sync();
    flat<T, R>(j, n * nocc, n, LD, 1, [&](int e) { return A + (e % n); },
               [&](int e) { return C + occ_list[e / n] * LD; }, [&](int e, double v) { Y[(e / n) * LD + e % n] = v; });
    g.sync();
    for (int e = j; e < n * nocc; e += T) {
        const int o = e / n, i = e - o * n;
        A[o * LD + i] = C[occ_list[o] * LD + i];
    }
    g.sync();
    flat<T, R>(j, nocc * nocc, n, 1, 1, [&](int e) { return A + (e % nocc) * LD; },
               [&](int e) { return Y + (e / nocc) * LD; }, [&](int e, double v) { C[(e / nocc) * LD + e % nocc] = v; });
    g.sync();
    // t(o, i) = 2 sum_o2 Aoo(o, o2) C_occ(i, o2) into Y[i * LD + o]
    flat<T, R>(j, nocc * n, nocc, LD, LD, [&](int e) { return C + (e % nocc); }, [&](int e) { return A + (e / nocc); },
               [&](int e, double v) { Y[(e / nocc) * LD + e % nocc] = 2.0 * v; });
    if (j == 0 && nocc < n) {   // HOMO-LUMO gap of the last iteration
        double homo = -1e300, lumo = 1e300;
        for (int c = 0; c < n; ++c) {
            if (occf[c]) homo = fmax(homo, diag[c]); else lumo = fmin(lumo, diag[c]);
        }
        if (!(lumo - homo > G_MIN_GAP)) atomicOr(&fl[0], ERRBIT_ZERO_GAP);
    }
    g.sync();
    // P = 2 C_occ C_occ^T into C
    flat<T, R>(j, nn, nocc, LD, LD, [&](int e) { return A + (e % n); }, [&](int e) { return A + (e / n); },
               [&](int e, double v) { C[(e / n) * LD + e % n] = 2.0 * v; });
    g.sync();
    if (j < n) {   // band energy, per column in a fixed order
        double eb = 0.0;
        for (int i = 0; i < n; ++i) eb = fma(C[j * LD + i], h0_at(i, j), eb);
        red[j] = eb;
    }
    g.sync();
    // W(i, c) = sum_o C_occ(i, o) t(o, c) into SH
    flat<T, R>(j, nn, nocc, LD, 1, [&](int e) { return A + (e % n); }, [&](int e) { return Y + (e / n) * LD; },
               [&](int e, double v) { SH[(e / n) * LD + e % n] = v; });
    g.sync();
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
        const double gi = rsqrt_nr(fma(r, r, sk.gamma_c2[eA][eB]));
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
    g.sync();
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
    g.sync();
}

// Persistent grid over a queue of work units: units [0, n_big) are one large item each (the whole
// block), the rest take two small items (one per half of the block).
template <int R>
__global__ void __launch_bounds__(BT, 2) k_dftb_generic(const DevSK *__restrict__ skp, const DftbArgs a,
                                                     const int2 *__restrict__ items, int n_big, int n_small,
                                                     unsigned *__restrict__ queue, int nmax_b, int amax_b,
                                                     int nmax_s, int amax_s) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int next;
    __shared__ int vote[2][2];
    const DevSK &sk = *skp;
    const GLayout Lb = g_layout(nmax_b, amax_b);
    const GLayout Ls = g_layout(nmax_s, amax_s);
    const int n_units = n_big + (n_small + 1) / 2;
    const int half = threadIdx.x / TS;
    for (;;) {
        if (threadIdx.x == 0) next = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int w = next;
        __syncthreads();
        if (w >= n_units) break;
        if (w < n_big) {
            const int2 it = items[w];
            const Grp<TB> g{(int)threadIdx.x, 0, nullptr};
            g_molecule<TB, R>(sk, a, Lb, smem, it.x, it.y, g);
        } else {
            const int s = 2 * (w - n_big) + half;
            if (s < n_small) {
                const int2 it = items[n_big + s];
                const Grp<TS> g{(int)threadIdx.x - half * TS, 1 + half, vote[half]};
                g_molecule<TS, R>(sk, a, Ls, smem + half * Ls.total, it.x, it.y, g);
            }
        }
        __syncthreads();
    }
}

template <int R>
cudaError_t set_attr(size_t smem, int &blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_dftb_generic<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_dftb_generic<R>, BT, smem);
    return e;
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
    p.r_entries = 4;
    p.blocks_per_sm = 0;
}

cudaError_t prepare_dftb_generic(GenericPlan &p) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p.n_sm, cudaDevAttrMultiProcessorCount, dev);
    int b2 = 0, b4 = 0;
    if (e == cudaSuccess) e = set_attr<2>(p.smem, b2);
    if (e == cudaSuccess) e = set_attr<4>(p.smem, b4);
    p.max_blocks_per_sm = std::max(1, std::min(b2, b4));
    if (p.blocks_per_sm <= 0 || p.blocks_per_sm > p.max_blocks_per_sm) p.blocks_per_sm = p.max_blocks_per_sm;
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
    if (p.r_entries == 2)
        k_dftb_generic<2><<<grid, BT, p.smem, st>>>(sk, a, items, nb, ns, queue, p.nmax_b, p.amax_b, p.nmax_s,
                                                   p.amax_s);
    else
        k_dftb_generic<4><<<grid, BT, p.smem, st>>>(sk, a, items, nb, ns, queue, p.nmax_b, p.amax_b, p.nmax_s,
                                                   p.amax_s);
    return cudaGetLastError();
}
