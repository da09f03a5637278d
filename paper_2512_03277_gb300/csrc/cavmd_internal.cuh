// Internal declarations shared by the CUDA translation units of the cavity-MD library.
// Nothing here is part of the public ABI (include/cavmd.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cavmd.h"

#define CAVMD_FULL_MASK 0xffffffffu

// Device copy of the Slater-Koster set (kept in global memory, read through the L1 cache).
struct DevSK {
    double onsite[CAVMD_MAX_ELEM][2];
    double hubbard[CAVMD_MAX_ELEM];
    double zval[CAVMD_MAX_ELEM];
    double h0[CAVMD_MAX_ELEM][CAVMD_MAX_ELEM][4][4];
    double s[CAVMD_MAX_ELEM][CAVMD_MAX_ELEM][4][4];
    double rep[CAVMD_MAX_ELEM][CAVMD_MAX_ELEM][2];
    double gamma_c2[CAVMD_MAX_ELEM][CAVMD_MAX_ELEM];   // (2 / (U_A + U_B))^2 of the Klopman-Ohno gamma
    int norb[CAVMD_MAX_ELEM];
    double r_cut, taper, inv_taper;
};

// Error bits OR-ed into the context's device status word by any kernel.
enum {
    ERRBIT_SCC_NOCONV = 1,
    ERRBIT_S_NOT_PD = 2,
    ERRBIT_ZERO_GAP = 4,
    ERRBIT_NONFINITE = 8,
    ERRBIT_TIMEOUT = 16,
};

// Arguments of one batched SCC-DFTB evaluation (cells of one composition).
struct DftbArgs {
    int n_cells;               // cells in this launch
    const int *cell_list;      // [n_cells] cell ids, or NULL for 0..n_cells-1
    const int *cell_offset;    // [N+1] first atom of each cell
    const int *species;        // [n_atoms]
    const double *r;           // [3 n_atoms]
    double *F;                 // [3 n_atoms] out: -dE/dr
    double *b;                 // [3 n_atoms] out: Mulliken b_j = Q_j pol (charge_model 0)
    double *qpop;              // [n_atoms] in/out: Mulliken populations (warm start)
    double *qprev;             // [n_atoms] in/out: populations of the step before (predictor)
    double *Cwarm;             // in/out eigenvectors of every cell (column-major, n_c x n_c each)
    const long long *Cwarm_off;   // [N] first element of each cell's block in Cwarm (NULL: 36 per cell)
    double *E_cell;            // [N] out
    double *M_cell;            // [N] out
    int *iters;                // [N] out
    unsigned *status;          // device error word
    double pol0, pol1, pol2;
    double scc_tol;
    double beta;
    int max_iter;
    int hist;                  // Anderson history (cluster kernel): current + hist-1 previous iterates
    int have_warm;             // 1: Cwarm and qpop hold a previous solution
    int max_sweeps;            // bound on the Jacobi sweeps of a cold start (0: the kernel's default)
    int write_b;               // 1: write Mulliken b
    // finite-difference rows: n_disp > 0 turns every cell into displaced copies that only compute
    // their dipole (3 per atom forward, or 6 per atom central in +h, -h pairs)
    int n_disp;
    int fd_central;
    double fd_h;
    double *M_disp;            // [3 or 6 per atom] out: row k of the cell starting at atom a0 at 3 a0 + k (6 a0 + k)
    double *Qout;              // [n_atoms] out: Mulliken net charges (may be NULL)
    // Opening half-flow of a call's first step, applied by the water kernel to the atoms of its
    // cells before it reads their positions: p += tau F + E_n b, then r += dt p / m (the same
    // arithmetic as the kick kernel). E_open = NULL: none.
    const double *E_open;      // [N] field of the opening half-flow
    double *p_open;            // [3 n_atoms] momenta, kicked in place
    double *r_open;            // [3 n_atoms] positions, drifted in place (the array r points to)
    const double *inv_mass;    // [n_atoms]
    double tau, dt;
    const long long *step_counter;   // device step counter (periodic kernel: which steps re-diagonalise)
};

// Arguments of the coupling / integrator kernels.
struct StepArgs {
    int N, M, n_atoms;
    const int *cell_offset;
    const double *U;           // [M][N] u_a(R_n), row-major
    const double *M_cell;      // [N]
    const double *E_cell;      // [N]
    const double *inv_mass;    // [n_atoms]
    const double *mass;        // [n_atoms]
    const double *F;           // [3 n_atoms]
    const double *b;           // [3 n_atoms]
    double *r, *p;             // [3 n_atoms]
    // photons
    const double *omega, *lam, *inv_omega;
    const double *cos_h, *sin_h, *omc_h;   // cos(w tau), sin(w tau), (1 - cos(w tau)) / w, tau = dt/2
    double *q, *pq;            // running photon state (mid-step when a first half-flow is applied)
    double *q_sync, *pq_sync;  // photon state at the last full step
    double *D;                 // [M]
    double *W1, *W2;           // [M] field weights of the first / second half-flow
    double *e_mode;            // [M][4] photon, coupling, dse, free-photon energy of each mode
    double *e_kin_part;        // [n_blocks] partial kinetic energies
    double *e_dftb_part;       // [n_blocks]
    unsigned *done_counter;    // last-block counter of the field kernel
    double *hist;              // [hist_cap][8] energy history
    int hist_cap;
    long long *step_counter;   // device step counter
    unsigned *status;
    double dt, tau;
    // mixed-precision coupling (modes on a grid): Gram matrix in, weight matrices and fields out
    const double *G;           // [128][KY] forward Gram matrix (PH_FORWARD_G)
    float *Wt2, *Wt1;          // [128][KY] back-product weights written by the photon kernel
    const double *E2in, *E1in; // [N] fields from the back product (FLD_E_GIVEN)
    double *E1store;           // [N] the next first half-flow's field, kept for the next call (FLD_E1_STORE)
    int Kx, Ky2, KY;
    // moving mode positions (Us != NULL): u_a at the cell centres of mass, their sines, and the
    // position term of the kicks, (m_j / m_n) M_n G_n with G_n = sum_a Wk_a sin(k_a.R_n + phi_a)
    const double *Us;          // [M][N] sin(k_a.R_n + phi_a), row-major
    const double *kvec;        // [M][3] wave vectors
    double *Wk2, *Wk1;         // [M][3] -W_a k_a of the second / first half-flow (written by k_photon)
    const double *w_atom;      // [n_atoms] m_j / m_n
    const int *atom_cell;      // [n_atoms] the cell of each atom
    double *G1store;           // [N][3] G_n of the next first half-flow, kept for the next call
    const double *G1in;        // [N][3] G_n of the opening first half-flow (FLD_E_GIVEN)
    const double *G2in;        // [N][3] G_n of the second half-flow (FLD_E_GIVEN, tensor-core coupling)
    int paper;                 // 1: kicks with the instantaneous force (CAVMD_SPLIT_PAPER or STRANG), 0: exact half-flows
    int strang;                // 1: the modes turn between the two kicks (CAVMD_SPLIT_STRANG)
};

// The paper's real-space photon scheme (CAVMD_SPLIT_REAL_SPACE, realspace.cu).
struct RsArgs {
    double eta, eta2_w0sq, inv_w0sq;   // eta = sqrt(2N) g0 omega_0; eta^2 / omega_0^2; 1 / omega_0^2
    double sq, isq, inv_sq, inv_isq;   // sqrt(omega_0 / 2), 1 / sqrt(2 omega_0) and their inverses
    const double *w, *cdt, *sdt;       // [M] lambda_a^2 / (2 N g0^2), cos and sin of omega_a dt
    double *x, *y;                     // [N] amplitude parts of the cells
    double *Xw, *Yw;                   // [M] weighted, turned mode amplitudes
    double *E1, *E2;                   // [N] fields of the first and second half-kicks (times dt/2)
};
// RS_INIT flags: 0 keep the synchronised photons, 1 relaxed (q_n = -eta M_n / omega_0^2), 2 zero;
// RS_FORWARD flags: 1 = turn by omega_a dt; RS_BACK flags: bit 0 = map back, bit 1 = first half-kick
enum { RS_INIT = 0, RS_OPEN = 1, RS_SECOND = 2, RS_FORWARD = 3, RS_BACK = 4 };
cudaError_t launch_rs(const RsArgs &r, const StepArgs &a, int what, int flags, cudaStream_t st);

// Plan of the tensor-core coupling contraction for modes on a uniform in-plane grid.
struct TcPlan {
    int N, Npad, Kx, Ky2, KY, n_fwd_cta, n_sm;
    double dkx, dky;
    __nv_bfloat16 *Ahi, *Alo, *Yhi, *Ylo;   // phase panels (bfloat16 hi / lo, core-matrix order)
    float *Af, *Bsrc;                       // FP32 panels
    double *partial;                        // split-K partial Gram matrices [n_fwd_cta][128][KY]
};
size_t tc_fwd_smem(int KY);
int tc_fwd_stage_cells();         // cells per stage of the forward product
size_t tc_back_smem(int KY);
cudaError_t tc_prepare(int KY);   // kernel attributes (shared-memory size), once per plan
cudaError_t launch_tc_panels(const TcPlan &p, const double *R, cudaStream_t st);
cudaError_t launch_tc_forward(const TcPlan &p, const double *Mc, double *G, unsigned *status, cudaStream_t st);
// Back product: E2 (and E1 when Wt1 is given) from the weight matrices; with G (moving mode
// positions, Wt1 = NULL, E1 = NULL) also the gradients G[3n + k] of E2 at the cells' centres.
cudaError_t launch_tc_back(const TcPlan &p, const float *Wt2, const float *Wt1, double *E2, double *E1,
                           unsigned *status, cudaStream_t st, double *G = nullptr);
// Phase panels at the cells' centres of mass (moving mode positions), every step.
cudaError_t launch_tc_panels_com(const TcPlan &p, const double *r, const double *mass, const int *cell_offset,
                                 cudaStream_t st);

// Conversions between FP64 and FP32 on the integer pipe, for quantities that only steer an
// iteration (generator entries, rotation angles, mixing coefficients): on GB300 the hardware
// conversions issue to the FP64 pipe, the bottleneck of the SCC kernels. d2f_steer truncates the
// significand (magnitudes below 2^-126 give a signed zero, above the FP32 range a signed
// infinity, and so do NaNs); f2d_steer is exact for zero, normal numbers, infinities and NaNs
// (subnormals give a signed zero).
__device__ __forceinline__ float d2f_steer(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32);
    const unsigned sgn = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu) - 896;   // rebias 1023 -> 127
    if (e <= 0) return __uint_as_float(sgn);
    if (e >= 255) return __uint_as_float(sgn | 0x7f800000u);
    return __uint_as_float(sgn | ((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7fffffull));
}
__device__ __forceinline__ double f2d_steer(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
    if (e == 0) return __longlong_as_double((long long)sgn);
    const unsigned long long ee = e == 255u ? 0x7ffull : (unsigned long long)(e + 896u);
    return __longlong_as_double((long long)(sgn | (ee << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}

// |x| < y for finite doubles and y > 0, by the ordering of the IEEE bit patterns: an integer
// comparison that leaves the FP64 pipe free.
__device__ __forceinline__ bool abs_lt(double x, double y) {
    return (__double_as_longlong(x) & 0x7fffffffffffffffLL) < __double_as_longlong(y);
}

// Total order key of a double (same order as the numeric value for non-NaN inputs).
__device__ __forceinline__ long long order_key(double x) {
    long long b = __double_as_longlong(x);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}

// 1/sqrt(d) for d > 0 within FP64 rounding: single-precision seed, then two Newton-Raphson
// steps y <- y (3 - d y^2) / 2, each of which doubles the number of correct bits (24 -> 48 -> 96).
__device__ __forceinline__ double rsqrt_nr(double d) {
    double y = (double)rsqrtf((float)d);
    y = y * fma(-0.5 * d * y, y, 1.5);
    y = y * fma(-0.5 * d * y, y, 1.5);
    return y;
}

#include <string>
#include <vector>
// Records the message returned by cavmd_last_error(NULL) (calls without a context).
void cavmd_set_global_error(const std::string &msg);

// On-device autocorrelation accumulators (channels: M photon coordinates, then the total dipole).
struct AcfArgs {
    int M, C, L;                 // modes, channels (M + 1), lags
    int B;                       // samples folded into the lag products at a time
    double *ring;                // [C][L + B] the last L + B samples
    double *head, *acc;          // [C][L]: first L samples, lag products
    double *sum;                 // [C] running sums
    long long *n;                // samples so far
    unsigned *ticket;            // last-block counter
    int G;                       // blocks per sample (>= M / 8, a warp per photon channel): each also
                                 // sums a slice of the cell dipoles
    double *part;                // [G] those slice sums
};
cudaError_t launch_acf(const AcfArgs &a, const double *q_sync, const double *M_cell, int N, cudaStream_t st);
cudaError_t launch_acf_finalize(const AcfArgs &a, double *out, cudaStream_t st);

// Host-side launchers (defined in the .cu files).
cudaError_t launch_dftb_water(const DevSK *sk_dev, const DftbArgs &a, cudaStream_t st, int warps = 2,
                              int per_warp = 5);
cudaError_t prepare_dftb_water(int max_warps);   // shared-memory attribute for up to max_warps per block
// r_trial = r + dt p / m: positions one drift ahead, for timing trial evaluations
cudaError_t launch_trial_positions(const double *r, const double *p, const double *inv_mass, double dt, int n_atoms,
                                   double *r_trial, cudaStream_t st);

// Plan of the persistent SCC-DFTB launch over cells of any composition (up to 64 orbitals).
struct GenericPlan {
    int nmax_b, amax_b, nmax_s, amax_s;          // largest cell of the large (> 32 orbitals) and small classes
    int n_big, n_small, n_disp_big, n_disp_small;
    int n_sm, blocks_per_sm, max_blocks_per_sm;  // persistent grid: n_sm x blocks_per_sm blocks
    int r_entries;                               // product entries per thread per pass (2 or 4)
    size_t smem;                                 // dynamic shared memory per block
    int2 *items, *disp_items;                    // device: (cell, -1) and (cell, displacement), largest first
    unsigned *queue;                             // device: [2] work counters
};
// Host: item lists (largest first) and shared-memory size from the cell sizes.
void plan_dftb_generic(const int *cell_offset, const int *species, const int *norb_of_elem, int n_cells,
                       int n_disp_per_atom, GenericPlan &p, std::vector<int2> &items,
                       std::vector<int2> &disp_items);
cudaError_t prepare_dftb_generic(GenericPlan &p);   // kernel attribute and occupancy, once per plan
cudaError_t launch_dftb_generic(const DevSK *sk_dev, const DftbArgs &a, const GenericPlan &p, cudaStream_t st);
// Plan of the Gamma-point SCC-DFTB launch over periodic cells (one lattice for all cells).
struct PbcPlan {
    double lat[9], inv[9];                // lattice vectors as rows; inverse (f = r inv)
    double alpha, bg, self_e, r_real;     // Ewald splitting, background and self terms, real-space cutoff
    int n_img, n_img_sk, n_g;             // lattice translations (by length; the first n_img_sk reach
                                          // r_cut); half-space reciprocal vectors
    int nmax, amax, blocks;               // largest cell; persistent blocks (2 per SM, k-grid 1)
    double *d_img, *d_gw;                 // device: [n_img][3], [n_g][4] (G, 2 w_G)
    double *work;                         // device: per-block workspaces
    int nk;                               // k-grid: irreducible k-points (0: Gamma point only)
    double *d_kpt;                        // device: [nk][4] fractional k and weight
};
size_t pbc_workspace_doubles(int nmax, int amax, int n_g, int nk);
std::vector<double> pbc_kpoints(const int *kgrid);
size_t pbc_smem(bool kgrid);
void plan_dftb_periodic(const double *lat, double r_cut, PbcPlan &p, std::vector<double> &img,
                        std::vector<double> &gw);
cudaError_t prepare_dftb_periodic();
cudaError_t launch_dftb_periodic(const DevSK *sk_dev, const DftbArgs &a, const PbcPlan &p, cudaStream_t st);
// b_j = dM/dr_j from the displaced dipoles (forward or central differences)
cudaError_t launch_born_assemble(int n_cells, const int *cell_offset, const double *M_cell,
                                 const double *M_disp, int n_disp, int central, double h, double *b,
                                 cudaStream_t st);
// Born-charge network pieces used by a time step
cudaError_t launch_mlp_features(int n_cells, const int *off, const int *species, const double *r, float *X,
                                float *R, unsigned *status, cudaStream_t st, int atoms_per_cell = 0);
cudaError_t launch_mlp_forward(int n_atoms, const float *X, const float *R, const void *w_bf16, float *Zl,
                               unsigned *status, cudaStream_t st);
cudaError_t prepare_mlp_forward();   // shared-memory attribute of the inference forward, once per process
cudaError_t launch_mlp_born(int n_cells, const int *off, const float *Zl, const float *R, const double *Q,
                            double pol0, double pol1, double pol2, double *b, cudaStream_t st);
cudaError_t launch_to_bf16(const float *src, void *dst, int n, cudaStream_t st);
cudaError_t launch_mode_functions(const double *k, const double *phi, const double *R, int M, int N,
                                  double *U, cudaStream_t st);
// cos and sin of k_a.R_n + phi_a at given positions (moving mode positions: the reference functions)
cudaError_t launch_mode_functions_pair(const double *k, const double *phi, const double *R, int M, int N, double *U,
                                       double *Us, cudaStream_t st);
// u_a and sin(k_a.R + phi_a) at the centres of mass of the cells, by angle addition from the
// reference functions U0, Us0 at the positions R0 (moving mode positions)
cudaError_t launch_mode_functions_com(const double *k, const double *R0, const double *U0, const double *Us0,
                                      const double *r, const double *mass, const int *cell_offset, int M, int N,
                                      double *U, double *Us, cudaStream_t st);
// G_n = -sum_a W_a k_a Us[a][n] for a given W (evaluation read-back)
cudaError_t launch_field_grad_only(const double *Us, const double *W, const double *k, int M, int N, double *G,
                                   cudaStream_t st);
// forward contraction of M_cell into D plus the photon half-flows (flags below)
// PH_W1: weights of the next first half-flow from the synchronised state, without rotating
// PH_OPEN (with PH_SECOND): apply the opening first half-flow of a call from the synchronised
// state before the second, instead of a PH_FIRST launch of its own
enum { PH_FORWARD = 1, PH_SECOND = 2, PH_FIRST = 4, PH_INIT_RELAXED = 8, PH_INIT_ZERO = 16,
       PH_ENERGY = 32, PH_FORWARD_G = 64, PH_W1 = 128, PH_OPEN = 256 };
cudaError_t launch_photon(const StepArgs &a, int flags, cudaStream_t st);
// field on the cells with weights W2 (second half-flow kick) and/or W1 (first half-flow kick +
// drift); always records the energies of the synchronised state when FLD_ENERGY is set
// FLD_E1_STORE: form the next first half-flow's field from W1 and store it, without that kick
enum { FLD_SECOND = 1, FLD_FIRST = 2, FLD_ENERGY = 4, FLD_E_GIVEN = 8, FLD_E1_STORE = 16 };
cudaError_t launch_field(const StepArgs &a, int flags, cudaStream_t st);
int field_blocks(int N);
// instantaneous field E_n = sum_a u_a(R_n) W_a for a caller-supplied weight vector
// the observables of the synchronised state packed into one buffer (see couple_kernels.cu)
cudaError_t launch_obs_pack(const double *hist_slot, const int *iters, int N, const unsigned *status,
                            const double *Mc, const double *q, const double *p, const double *D, int M,
                            bool with_arrays, double *out, unsigned *scr, cudaStream_t st);   // scr: 2 zeroed words
cudaError_t launch_field_only(const double *U, const double *W, int M, int N, double *E,
                              cudaStream_t st);
