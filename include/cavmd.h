/*
 * cavmd.h - C ABI of the GB300 cavity molecular-dynamics hot path.
 *
 * One context propagates N independent cells (molecules or clusters, the batch
 * dimension; the paper's non-interacting cells of Eq. hm) coupled to M cavity
 * modes through the multimode dipole-gauge Hamiltonian beyond the long-wavelength
 * approximation (Eq. hlm_bigin / hlm2, written with real modes). Every time step
 * runs, on one GPU:
 *   - an SCC-DFTB evaluation of every cell (Slater-Koster H0/S, self-consistent
 *     charges, generalised eigensolve, Mulliken charges, analytic forces; the
 *     method the paper's "Computational details" names, second-order SCC-DFTB);
 *   - the cell dipoles M_n = pol . mu_n and their derivatives b_j = dM_n/dr_j
 *     (Mulliken charges or finite-difference Born charges, Results section);
 *   - the forward contraction D_a = lambda_a sum_n u_a(R_n) M_n and the field on
 *     every cell E_n = sum_a lambda_a u_a(R_n) Y_a (k-space form of Eq. dpj);
 *   - one symmetric velocity-Verlet-like step with the analytic photon rotation
 *     of Eq. qknk (Step 3), integrated as described for CAVMD_SPLIT_PHOTON_EXACT.
 *
 * Units: atomic units throughout (bohr, Hartree, electron masses, a.u. of time).
 *
 * Conventions shared by every entry point:
 *   - Every pointer in the structs below is a HOST pointer unless its comment
 *     says otherwise. The library copies what it reads during the call; the
 *     caller keeps ownership of all its arrays.
 *   - Arrays of 3-vectors are atom-major: x[3*i + k] is component k of atom i.
 *   - Return value: CAVMD_OK (0) or a negative CAVMD_ERR_* code. The message of
 *     the last failure is available from cavmd_last_error(ctx) (or
 *     cavmd_last_error(NULL) when cavmd_init itself failed). No exception or
 *     abort crosses the ABI.
 *   - One context belongs to one GPU and one CUDA stream. A context is not
 *     thread safe; distinct contexts are independent.
 */
#ifndef CAVMD_H
#define CAVMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CAVMD_OK 0
#define CAVMD_ERR_INVALID_ARG -1   /* a size, pointer or option is out of range            */
#define CAVMD_ERR_CUDA -2          /* a CUDA runtime call failed (message has the name)    */
#define CAVMD_ERR_SCC_NOCONV -3    /* a cell's charges did not converge in scc_max_iter    */
#define CAVMD_ERR_NONFINITE -4     /* a NaN or Inf appeared in the state                   */
#define CAVMD_ERR_S_NOT_PD -5      /* an overlap matrix was not positive definite          */
#define CAVMD_ERR_ZERO_GAP -6      /* HOMO-LUMO gap below the closed-shell threshold       */
#define CAVMD_ERR_DEVICE_TIMEOUT -7/* a bounded device loop ran out of iterations          */
#define CAVMD_ERR_UNSUPPORTED -8   /* valid request that this build does not implement     */
#define CAVMD_ERR_NOMEM -9         /* device allocation failed                             */

#define CAVMD_MAX_ELEM 4           /* element ids 0..3                                    */
#define CAVMD_MAX_CELL_ORBITALS 64 /* orbitals per cell (an even count); more, or cells  */
                                   /* whose on-chip storage exceeds 227 KB, return        */
                                   /* CAVMD_ERR_UNSUPPORTED. Cells of 3 atoms and 6       */
                                   /* orbitals take a lane-group kernel; any other mix of  */
                                   /* cells takes the persistent cluster kernel.           */
#define CAVMD_MAX_PERIODIC_ORBITALS 256 /* periodic cells (cavmd_system.lattice): orbitals  */
#define CAVMD_MAX_PERIODIC_ATOMS 128    /* and atoms per cell                             */
/* Dipole derivative b_j = dM_n/dr_j used by the coupling force:
 *   MULLIKEN     b_j = Q_j pol (the paper's cheap replacement; not conservative);
 *   BORN_FD      forward differences [M(r + h e) - M(r)] / h, the paper's choice, from 3 N_at
 *                displaced SCC solves per cell (warm started from the cell's solution);
 *   BORN_CENTRAL central differences from 6 N_at displaced solves (for tests and conservation);
 *   BORN_MLP     the per-atom network of cavmd_load_born_mlp (below).                        */

/* Integral kinds of a Slater-Koster table entry [eA][eB][kind]: SP means an s
 * orbital on the first element and a p orbital on the second. */
enum { CAVMD_SK_SS = 0, CAVMD_SK_SP = 1, CAVMD_SK_PPS = 2, CAVMD_SK_PPP = 3 };

enum { CAVMD_PREC_FP64 = 0, CAVMD_PREC_MIXED_TF32 = 1, CAVMD_PREC_MIXED_BF16X3 = 2 };
enum { CAVMD_CHARGE_MULLIKEN = 0, CAVMD_CHARGE_BORN_FD = 1, CAVMD_CHARGE_BORN_CENTRAL = 2,
       CAVMD_CHARGE_BORN_MLP = 3 };
/* Time step. PHOTON_EXACT: H_2(dt/2), drift(dt), H_2(dt/2), with H_2 = V + H_ph solved exactly at
 * frozen nuclei (each mode turns about its displaced centre; the nuclei take the time-integrated
 * force). PAPER: the paper's order, Eq. pj1 then Step 3: half-kick the nuclei and the photon
 * momenta with the instantaneous force (p_a += dt/2 omega_a D_a), drift, evaluate, half-kick again,
 * then turn every mode freely by omega_a dt (Eq. qknk). With cells on a line lattice, modes on its
 * DFT grid and a flat dispersion, PAPER reproduces the paper's real-space / reciprocal-space
 * Steps 1-4 exactly. STRANG: kick(dt/2) with the instantaneous force, then the free flow of the
 * nuclei (drift) and of every mode (turn by omega_a dt) over dt, evaluate, kick(dt/2): the
 * textbook split of H into the free part and V - sum_a omega_a q_a D_a + 1/2 sum_a D_a^2. Like
 * PAPER it needs omega_a dt below about 1 for stability. */
/* REAL_SPACE: the paper's real-space / reciprocal-space scheme as printed (Eq. hlm3; Step 1,
 * Eq. pj1; Steps 2-4, Eqs. qkink_ak, qknk, qkink_an). Each cell n carries a real-space photon
 * coordinate q_n and momentum p_n; the coupling takes sqrt(omega_k) ~ sqrt(omega_0) and is local,
 * eta q_n M_n + eta^2 M_n^2 / (2 omega_0^2) with eta = sqrt(2N) g0 omega_0 (options.real_space_g0,
 * real_space_omega0); Step 1 kicks p_n by -eta M_n and the nuclei by -(eta q_n + eta^2 M_n /
 * omega_0^2) dM_n/dr_j around the drift, then the omega_0-normalised amplitudes sqrt(omega_0/2) q_n
 * + i p_n / sqrt(2 omega_0) go to the modes, turn by omega_a dt each (any dispersion), and come
 * back. It is the paper's scheme when the cells sit on a lattice and the modes are the real modes
 * of its wave-vector grid (cos and sin of each +-k pair with lambda = 2 g0, single modes sqrt(2) g0);
 * it needs as many modes as cells, the FP64 coupling and fixed mode positions. In cavmd_obs and
 * cavmd_state the arrays q and p (pq) then hold q_n and p_n of the cells (D is zero), and the
 * energy record's free-photon term is the k-space sum_a omega_a |a_a|^2. */
enum { CAVMD_SPLIT_PHOTON_EXACT = 0, CAVMD_SPLIT_STRANG = 1, CAVMD_SPLIT_PAPER = 2, CAVMD_SPLIT_REAL_SPACE = 3 };
enum { CAVMD_PHOTON_RELAXED = 0, CAVMD_PHOTON_ZERO = 1 };
/* Where the mode functions u_a are evaluated. FIXED: at the cells' reference positions R_n (the
 * paper's boxes sit at fixed positions, Eq. hlm2). CENTRE_OF_MASS: at every cell's instantaneous
 * centre of mass R_n(t) = sum_j m_j r_j / m_n, regenerated after every drift. Then D_a also
 * depends on the positions through u_a(R_n), and each nucleus j of cell n feels the extra force
 * (m_j / m_n) M_n sum_a lambda_a (omega_a q_a - D_a) grad u_a(R_n). This extends the paper,
 * whose boxes do not move. With the FP64 coupling each step regenerates M x N mode functions and
 * their sines (FP64, by angle addition from the reference positions). With
 * CAVMD_PREC_MIXED_BF16X3 each step rebuilds the factorised phase panels at the centres of mass
 * (FP32 phases from an exact fixed-point reduction of the angle, relative error about 3 * 2^-24)
 * and the back product runs once per half-flow, also forming the gradients of the field.
 * Only with CAVMD_SPLIT_PHOTON_EXACT: other splittings return CAVMD_ERR_UNSUPPORTED. */
enum { CAVMD_MODES_FIXED = 0, CAVMD_MODES_CENTRE_OF_MASS = 1 };

/* The cells. Cell c owns atoms cell_offset[c] .. cell_offset[c+1]-1. Cells are
 * neutral and closed shell (sum of valence charges even). */
typedef struct {
    int32_t n_cells;
    int32_t n_atoms;
    const int32_t *cell_offset; /* [n_cells + 1], non-decreasing, [0] = 0, [n_cells] = n_atoms */
    const int32_t *species;     /* [n_atoms] element ids < n_elem of the tables                */
    const double *r;            /* [3 n_atoms] positions, bohr                                  */
    const double *p;            /* [3 n_atoms] momenta                                          */
    const double *R_ref;        /* [3 n_cells] fixed mode-function centres R_n, or NULL for the
                                   initial centre of mass of each cell                           */
    const double *lattice;      /* NULL: isolated cells. Otherwise [9] lattice vectors a_1, a_2,
                                   a_3 as rows (bohr), shared by every cell, and each cell is
                                   periodic (the paper's cubic 33-water cells, section
                                   "Computational details") and evaluated at the Gamma point:
                                   H0 and S summed over lattice images within r_cut, gamma as the
                                   Ewald sum of 1/r (tin-foil boundary) plus the Klopman-Ohno
                                   remainder over images with the cosine taper at r_cut. Positions
                                   are unwrapped (molecules stay whole); the cell dipole is
                                   sum_j Q_j r_j. Cells up to CAVMD_MAX_PERIODIC_ORBITALS orbitals
                                   and CAVMD_MAX_PERIODIC_ATOMS atoms; Mulliken or finite-difference
                                   Born charges (the network returns CAVMD_ERR_UNSUPPORTED); the
                                   Brillouin zone sampled at Gamma or on cavmd_options.kgrid      */
} cavmd_system;

/* Slater-Koster parameter set. Every radial integral is
 *   V(r) = a exp(-b r) (1 + c1 r + c2 r^2) f_cut(r)   with params {a, b, c1, c2},
 * f_cut = 1 below r_cut - taper, then 1/2 (1 + cos(pi x)), x = (r - r_cut + taper)/taper,
 * and 0 from r_cut on. Entries of kinds that do not exist for a pair (p orbitals
 * on an s-only element) are ignored. Klopman-Ohno gamma uses hubbard[]. */
typedef struct {
    int32_t n_elem;                                       /* 1..CAVMD_MAX_ELEM                */
    int32_t norb[CAVMD_MAX_ELEM];                         /* 1 (s) or 4 (s, px, py, pz)       */
    double onsite[CAVMD_MAX_ELEM][2];                     /* eps_s, eps_p, Hartree            */
    double hubbard[CAVMD_MAX_ELEM];                       /* U, Hartree                       */
    double zval[CAVMD_MAX_ELEM];                          /* valence electrons                */
    double mass[CAVMD_MAX_ELEM];                          /* electron masses                  */
    double h0[CAVMD_MAX_ELEM][CAVMD_MAX_ELEM][4][4];      /* [eA][eB][kind][a,b,c1,c2]        */
    double s[CAVMD_MAX_ELEM][CAVMD_MAX_ELEM][4][4];       /* same layout, overlap             */
    double rep[CAVMD_MAX_ELEM][CAVMD_MAX_ELEM][2];        /* pair repulsion a exp(-b r) f_cut */
    double r_cut;                                         /* bohr                             */
    double taper;                                         /* bohr, > 0                        */
} cavmd_sk_tables;

/* Real cavity modes u_a(R) = cos(k_a . R + phi_a) with frequency omega_a > 0 and
 * amplitude lambda_a (2 g0 for each real member of a travelling +-k pair,
 * sqrt(2) g0 for a single real mode; see Eq. hlm2). */
typedef struct {
    int32_t n_modes;            /* M >= 1                                   */
    const double *k;            /* [3 M] wave vectors, 1/bohr               */
    const double *omega;        /* [M]                                      */
    const double *lambda;       /* [M]                                      */
    const double *phi;          /* [M]                                      */
    double pol[3];              /* polarisation, the same for every mode    */
} cavmd_modes;

typedef void *(*cavmd_alloc_fn)(size_t bytes, void *user);
typedef void (*cavmd_free_fn)(void *device_ptr, void *user);

typedef struct {
    double dt;                  /* time step, a.u.                                            */
    int32_t precision;          /* CAVMD_PREC_*                                               */
    int32_t charge_model;       /* CAVMD_CHARGE_*                                             */
    int32_t born_interval;      /* refresh finite-difference Born charges on every evaluation whose
                                   index (0 = the initial one, then the step number) is a multiple
                                   of this; the paper refreshes every 3 steps. Stale in between.  */
    double fd_step;             /* finite-difference displacement, bohr                      */
    double scc_tol;             /* max |q_out - q_in| per atom at convergence                */
    int32_t scc_max_iter;
    double mixing;              /* linear part of the charge mixing                           */
    int32_t splitting;          /* CAVMD_SPLIT_*                                              */
    int32_t photon_init;        /* CAVMD_PHOTON_*                                             */
    int32_t graph_chunk;        /* steps per captured CUDA graph; 0 = no graph                */
    int32_t device;             /* CUDA device ordinal                                        */
    void *stream;               /* cudaStream_t to run on, or NULL for a library-owned stream */
    cavmd_alloc_fn dev_alloc;   /* optional device allocator (e.g. a framework's); NULL = cudaMalloc */
    cavmd_free_fn dev_free;     /* its matching free                                          */
    void *alloc_user;           /* passed back to dev_alloc / dev_free                        */
    int32_t energy_history;     /* steps of energy history kept on the device (>= 1)          */
    int32_t acf_lags;           /* on-device autocorrelation of the photon coordinates and of the
                                   total dipole, lags 0 .. acf_lags-1 (0 = off; see
                                   cavmd_autocorrelation)                                        */
    int32_t autotune;           /* 1: cavmd_init times candidate launch shapes of the SCC-DFTB
                                   kernel on a trial step and keeps the fastest (all candidates
                                   give bitwise identical results); 0: fixed defaults            */
    int32_t scc_history;        /* Anderson mixing history of the cluster kernel: the current and
                                   up to scc_history-1 previous iterates (1..6; 1 = linear mixing).
                                   Cells of 3 atoms / 6 orbitals use a fixed history of 3.        */
    int32_t mode_positions;     /* CAVMD_MODES_FIXED (default) or CAVMD_MODES_CENTRE_OF_MASS    */
    int32_t jacobi_max_sweeps;  /* bound on the Jacobi sweeps of a cold start (the first evaluation,
                                   and the first SCC iteration after cavmd_set_state): 0 = the
                                   kernels' defaults (24 for waters, 40 for clusters and periodic
                                   cells), else 1..1000. A cell whose off-diagonal elements are
                                   still above tolerance at the bound makes the call report
                                   CAVMD_ERR_DEVICE_TIMEOUT. Later SCC iterations take one sweep. */
    double real_space_g0;       /* CAVMD_SPLIT_REAL_SPACE: the coupling constant g0 (> 0)         */
    double real_space_omega0;   /* CAVMD_SPLIT_REAL_SPACE: the reference frequency omega_0 (> 0)  */
    int32_t kgrid[3];           /* periodic cells: Gamma-centred k-grid n1 x n2 x n3 sampling the
                                   Brillouin zone (the paper's "Gamma point of a 3 x 3 x 3 folded
                                   supercell" is {3, 3, 3}). {1, 1, 1} (the default; {0, 0, 0}
                                   means the same) is the Gamma point. Each entry 1..8. k and -k
                                   are solved once (weight 2 / (n1 n2 n3)); each remaining point is
                                   a complex Hermitian problem, solved in its real form of twice
                                   the size, so a step costs about 8 x the irreducible count x the
                                   Gamma point's work (3 x 3 x 3: 14 points). Isolated cells:
                                   must be {1, 1, 1} or {0, 0, 0}.                               */
} cavmd_options;

/* Observables at the current (synchronised) time. Optional arrays may be NULL. */
typedef struct {
    double e_kin, e_dftb, e_photon, e_coupling, e_dse, e_photon_free, e_total, temperature;
    int64_t step;               /* steps taken since cavmd_init                   */
    int32_t scc_iter_max;       /* largest SCC iteration count of the last step   */
    double *M;                  /* out [n_cells] projected cell dipoles, or NULL  */
    double *q;                  /* out [M] photon coordinates, or NULL            */
    double *p;                  /* out [M] photon momenta, or NULL                */
    double *D;                  /* out [M] D_a, or NULL                           */
} cavmd_obs;

/* The propagated state. All arrays host, caller-owned, sized as noted. */
typedef struct {
    double *r;                  /* [3 n_atoms] */
    double *p;                  /* [3 n_atoms] */
    double *q;                  /* [M]         */
    double *pq;                 /* [M]         */
    int64_t step;
} cavmd_state;

/* The last evaluation (at the current positions). Optional arrays may be NULL. */
typedef struct {
    double *F_dftb;             /* [3 n_atoms] -dE_DFTB/dr                                */
    double *F_total;            /* [3 n_atoms] F_dftb + E_n b_j with the instantaneous
                                   field E_n = sum_a lambda_a u_a(R_n)(omega_a q_a - D_a) */
    double *b;                  /* [3 n_atoms] dM_n/dr_j used by the step                 */
    double *q_pop;              /* [n_atoms] Mulliken populations                         */
    double *E_cell;             /* [n_cells] E_DFTB of every cell                         */
    double *M;                  /* [n_cells] projected dipoles                            */
    int32_t *scc_iters;         /* [n_cells] SCC iterations of the last evaluation        */
} cavmd_eval;

/* Opaque context: one propagated system on one GPU. */
typedef struct cavmd_ctx cavmd_ctx;

/* Fills *opt with the defaults: dt = 0.5 fs, FP64, Mulliken, born_interval 3, fd_step 1e-3,
 * scc_tol 1e-12, scc_max_iter 200, mixing 0.7, PHOTON_EXACT, relaxed photons, graph_chunk 50,
 * device 0, library stream, cudaMalloc, energy_history 1024. */
void cavmd_default_options(cavmd_options *opt);

/* Creates a context: validates and copies the inputs to the device, evaluates every cell at
 * the initial positions, initialises the photons (CAVMD_PHOTON_RELAXED: p_a = 0,
 * q_a = D_a / omega_a, the minimum of the photon energy at the initial matter, the
 * zero-temperature end point of the paper's Step 0) and records the energies of step 0.
 * On success *ctx owns its device memory until cavmd_destroy. Blocks until done. */
int cavmd_init(cavmd_ctx **ctx, const cavmd_system *sys, const cavmd_sk_tables *sk,
               const cavmd_modes *modes, const cavmd_options *opt);

/* Advances nsteps >= 0 time steps (Steps 1-4 of the paper's loop, in k-space form). The work is
 * queued on the context's stream and the call returns once it is queued, without waiting for
 * earlier work. It returns the status of earlier work that has already finished (a
 * non-convergence or a non-finite value found there). An error in work still running stays in the
 * device status word: a later cavmd_step, cavmd_observables or cavmd_observables_wait reports it. */
int cavmd_step(cavmd_ctx *ctx, int64_t nsteps);

/* Waits for the queued work and copies the observables of the current time into *out. */
int cavmd_observables(cavmd_ctx *ctx, cavmd_obs *out);

/* The same read-out in two halves, so that the host reads step t while the GPU runs step t + 1.
 * cavmd_observables_async queues, behind every step queued so far, the packing of the current
 * observables (with the arrays M, q, p, D when with_arrays != 0) and their copy into the
 * context's pinned staging slot `slot` (0 or 1), and returns at once. cavmd_observables_wait
 * waits for that copy and fills *out as cavmd_observables does (out->step is the step at which the
 * read-out was queued; array pointers must be NULL if the slot was queued without arrays).
 * Alternate the two slots: queue slot s % 2 after step s, then wait for slot (s - 1) % 2.
 * cavmd_observables itself uses slot 0. Errors: CAVMD_ERR_INVALID_ARG for a bad slot, a wait
 * with nothing queued in the slot, or arrays requested from a slot queued without them. */
int cavmd_observables_async(cavmd_ctx *ctx, int32_t slot, int32_t with_arrays);
int cavmd_observables_wait(cavmd_ctx *ctx, int32_t slot, cavmd_obs *out);

/* Copies the energy history: up to n most recent steps, 8 doubles each
 * (e_kin, e_dftb, e_photon, e_coupling, e_dse, e_photon_free, e_total, step), oldest first.
 * *n_out receives the number written. Waits for the queued work. */
int cavmd_energy_history(cavmd_ctx *ctx, double *out, int32_t n, int32_t *n_out);

/* Autocorrelation functions accumulated on the device (options.acf_lags > 0), the correlation
 * functions behind the paper's molecular spectrum <mu_x(t) mu_x(0)> and angle-resolved photonic
 * spectrum <q_k(t) q_k(0)> (Results). One sample per synchronised state: the state after
 * cavmd_init (or cavmd_set_state, which restarts the accumulation) and the state after every
 * step. Channels c = 0..M-1 are the photon coordinates q_c, channel M the total projected dipole
 * sum_n M_n. out (HOST, (M + 1) * n_lags doubles, channel-major) receives the mean-removed
 * unbiased estimator
 *     C_c(l) = 1/(n - l) sum_{t=l}^{n-1} (x_t - xbar)(x_{t-l} - xbar),  xbar = mean of the n samples,
 * for lag l (in steps) < n, and 0 for l >= n. *n_samples (may be NULL) receives n. reset != 0
 * clears the accumulation after reading. Waits for the queued work. Errors: INVALID_ARG when the
 * context was made with acf_lags = 0 or n_lags differs from it. */
int cavmd_autocorrelation(cavmd_ctx *ctx, double *out, int32_t n_lags, int64_t *n_samples, int32_t reset);

/* A one-line report of the launch shapes in use: with options.autotune = 1, the candidates timed
 * by cavmd_init on a trial step and the one kept. buf is a HOST buffer of len bytes; the report
 * is truncated to fit and always NUL-terminated. */
int cavmd_tuning(cavmd_ctx *ctx, char *buf, int32_t len);

/* Waits, then copies the state into / out of the caller's host buffers. cavmd_set_state
 * re-evaluates every cell at the new positions (as cavmd_init does, without touching the
 * photons), so a run resumed from a saved state repeats the original one exactly. */
int cavmd_get_state(cavmd_ctx *ctx, cavmd_state *st);
int cavmd_set_state(cavmd_ctx *ctx, const cavmd_state *st);

/* Waits, then copies the last evaluation into the caller's host buffers. */
int cavmd_get_eval(cavmd_ctx *ctx, cavmd_eval *out);

/* Per-phase device timers. enable = 1 starts recording CUDA events around every kernel
 * phase of later steps (on the context's stream); enable = 2 only around the SCC-DFTB launches
 * (phase 0: two events per step, which barely perturb a step's timing); enable = 0 stops.
 * Recording disables CUDA-graph replay. ms_out[CAVMD_N_PHASES] receives the summed durations and
 * counts[CAVMD_N_PHASES] the launches since the last reset (reset = 1 clears both after
 * reading). Either output may be NULL. */
#define CAVMD_N_PHASES 4        /* 0: SCC-DFTB, 1: forward contraction + photons,
                                   2: field + kicks + drift, 3: finite-difference Born rows */
int cavmd_phase_times(cavmd_ctx *ctx, int32_t enable, double *ms_out, int64_t *counts,
                      int32_t reset);

/* Message of the last failure on ctx (or, when ctx is NULL, of the last failed cavmd_init or
 * context-free call on this thread).
 * The string stays valid until the next call on the same context. */
const char *cavmd_last_error(const cavmd_ctx *ctx);

/* Frees every device buffer and the context itself. NULL is allowed. */
void cavmd_destroy(cavmd_ctx *ctx);

/* ------------------------------------------------------------------------------------------
 * Born-charge network (CAVMD_CHARGE_BORN_MLP).
 *
 * Stands in for the finite-difference Born charges the paper calls its computational bottleneck
 * (Results), against which it is trained. Per atom j of a cell: 32 invariant features of the
 * other atoms of its cell within 8 bohr (11 Gaussian radial terms per neighbour element, 8
 * angular terms, the element one-hot; elements 0 and 1 only), a local frame R_j (nearest
 * neighbour, second-nearest orthogonalised, their cross product), and a 32-128-128-9 network
 * with SiLU activations and bfloat16 weights evaluated in FP32. Its 9 outputs T_j, read as a
 * 3 x 3 tensor in the local frame, give the Born tensor
 *     Z_j = Q_j I + R_j^T T_j R_j - (mean over the cell of R^T T R),
 * Q_j the Mulliken net charge, so sum_j Z_j = Q_cell I exactly and the zero network is the
 * Mulliken model; b_j = pol^T Z_j. Parameters are one float array of CAVMD_MLP_NPARAMS values,
 * in order W1[128][32], b1[128], W2[128][128], b2[128], W3[9][128], b3[9] (row-major); they are
 * rounded to bfloat16 (nearest even) when loaded.
 * Training minimises sum_j |Z_j - Z_ref_j|^2 / (9 n_atoms) with AdamW (beta 0.9, 0.999, eps
 * 1e-8) on FP32 master weights, on the GPU. Data: water cells (O, H, H); all arrays host. */
#define CAVMD_MLP_NFEAT 32
#define CAVMD_MLP_HIDDEN 128
#define CAVMD_MLP_NPARAMS 21897
typedef struct cavmd_mlp cavmd_mlp;
/* Creates a network with the given parameters on `device` (its own stream and memory). */
int cavmd_mlp_create(cavmd_mlp **mlp, const float *params, int32_t n_params, int32_t device);
/* Loads n_cells water cells: species [3 n_cells], positions r [9 n_cells] (bohr), Mulliken net
 * charges Q [3 n_cells] and, for training, reference Born tensors Z_ref [27 n_cells]
 * (Z_ref[9 j + 3 alpha + beta] = d mu_alpha / d r_j,beta), or NULL. Computes the features. */
int cavmd_mlp_set_data(cavmd_mlp *mlp, int32_t n_cells, const int32_t *species, const double *r,
                       const double *Q, const double *Z_ref);
/* Loss and its gradient (FP32, [CAVMD_MLP_NPARAMS], may be NULL) over all loaded cells at the
 * current bfloat16 weights. */
int cavmd_mlp_loss_grad(cavmd_mlp *mlp, double *loss, float *grad);
/* AdamW over `epochs` passes of shuffled mini-batches of batch_cells cells (shuffle seeded by
 * seed); epoch_loss [epochs] (may be NULL) receives the mean batch loss of every epoch. */
int cavmd_mlp_train(cavmd_mlp *mlp, int32_t epochs, int32_t batch_cells, float lr, float weight_decay,
                    uint64_t seed, double *epoch_loss);
/* Predicted Born tensors [27 n_cells] of the loaded cells. */
int cavmd_mlp_predict(cavmd_mlp *mlp, double *Z_out);
/* Current parameters (the bfloat16 values, as floats). */
int cavmd_mlp_get_params(cavmd_mlp *mlp, float *params);
void cavmd_mlp_destroy(cavmd_mlp *mlp);
/* Loads network parameters into a context created with CAVMD_CHARGE_BORN_MLP and recomputes b
 * at the current positions (before a load the network is zero, i.e. Mulliken charges). */
int cavmd_load_born_mlp(cavmd_ctx *ctx, const float *params, int32_t n_params);

/* Allocation-free field and kick (no counterpart in the paper; an addition for embedding).
 *
 * For callers that cannot allocate device memory while they run: a framework that owns all of
 * the GPU's memory through its own pool, a latency-critical loop where cudaMalloc / cudaFree
 * would synchronise the device, or a plug-in whose host code may not allocate. The call performs
 * one half-step kick of the time step without any allocation, on caller-owned DEVICE arrays:
 *   E_n = sum_a U[a * n_cells + n] W[a]                  (field on cell n; U row-major [n_modes][n_cells])
 *   p_j += tau F_j + E_n b_j   for every atom j of cell n (cell_offset as in cavmd_system)
 *   *e_kin_out = sum_j |p_j|^2 inv_mass[j] / 2             (after the kick, summed in a fixed order)
 * E_out [n_cells] receives E_n and may be NULL. p is updated in place. All pointers are device
 * pointers; stream is a cudaStream_t (NULL = the legacy default stream); the work is queued and
 * the call returns without waiting.
 *
 * Scratch: the per-block energy partials and a counter live in one file-scope device array of
 * fixed size inside the library (about 256 KB, held by every GPU that loads the library until the
 * process exits). Hence the limit 1 <= n_cells <= CAVMD_NOALLOC_MAX_CELLS; larger sizes return
 * CAVMD_ERR_INVALID_ARG with a message from cavmd_last_error(NULL). The call never allocates and
 * never calls cudaMalloc or cudaFree. Every call made outside a stream capture looks up the array's
 * device address (cudaGetSymbolAddress) on the current device; a call made while `stream` is being
 * captured uses the address of the last such lookup on that device, so make one call on each device
 * before any capture (a captured call with no earlier lookup returns CAVMD_ERR_INVALID_ARG). After
 * cudaDeviceReset the next call outside a capture looks the address up again. Every call clears the
 * counter it needs, but all calls share the one array, which keeps
 * the last call's contents: calls that may overlap on the GPU (other streams, other host threads)
 * race and give wrong totals; serialise them. */
#define CAVMD_NOALLOC_MAX_CELLS 1048576
int cavmd_field_kick_noalloc(int32_t n_cells, int32_t n_modes, const int32_t *cell_offset,
                             const double *U, const double *W, const double *F, const double *b,
                             const double *inv_mass, double tau, double *p, double *E_out,
                             double *e_kin_out, void *stream);

/* Diagnostic of the tensor-core building block used by the mixed-precision coupling (no paper
 * counterpart): C[128][N] = A[128][K] B[N][K]^T with A, B bfloat16 bit patterns (host, row-major,
 * K contiguous) multiplied on the fifth-generation tensor cores with FP32 accumulation; C host,
 * row-major. K a positive multiple of 64, N = 128 or 256. Allocates its own device buffers. */
int cavmd_tc_selftest(const uint16_t *A, const uint16_t *B, int32_t K, int32_t N, float *C);

/* Size of one of the library's structs, for bindings that lay them out by hand. */
size_t cavmd_struct_size(int32_t which); /* 0 system, 1 sk_tables, 2 modes, 3 options,
                                            4 obs, 5 state, 6 eval */

#ifdef __cplusplus
}
#endif
#endif /* CAVMD_H */
