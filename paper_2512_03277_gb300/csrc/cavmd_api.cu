// Host implementation of the C ABI declared in include/cavmd.h.
//
// One step of the loop (the paper's Steps 1-4 in k-space form) is three kernels:
//   dftb      SCC-DFTB of every cell at the drifted positions (forces, charges, dipoles);
//   photon    D_a from the new dipoles, second half-flow of every mode, energies, and the first
//             half-flow of the next step;
//   field     E_n for both half-flows in one pass over u_a(R_n), the two nuclear kicks and the
//             drift to the next positions, and the energy record of the synchronised state.
// A call of cavmd_step(n) opens with the first half-flow (photon + field kernels without the
// forward contraction) and closes with a second half-flow only, so the state between calls is
// synchronised. Chunks of graph_chunk steps are captured once as a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "cavmd_internal.cuh"

namespace {
thread_local std::string g_init_error;
}

void cavmd_set_global_error(const std::string &msg) { g_init_error = msg; }

struct cavmd_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cavmd_options opt{};
    int N = 0, n_atoms = 0, M = 0;
    std::vector<int> h_off, h_species;
    double pol[3] = {1, 0, 0};
    // device buffers
    DevSK *d_sk = nullptr;
    int *d_off = nullptr, *d_species = nullptr, *d_iters = nullptr, *d_acell = nullptr;
    double *d_r = nullptr, *d_p = nullptr, *d_F = nullptr, *d_b = nullptr, *d_qpop = nullptr, *d_qprev = nullptr;
    double *d_C = nullptr, *d_E = nullptr, *d_Mc = nullptr, *d_mass = nullptr, *d_imass = nullptr;
    double *d_U = nullptr, *d_k = nullptr, *d_phi = nullptr, *d_R = nullptr;
    double *d_omega = nullptr, *d_lam = nullptr, *d_iomega = nullptr;
    double *d_cos = nullptr, *d_sin = nullptr, *d_omc = nullptr;
    double *d_q = nullptr, *d_pq = nullptr, *d_qs = nullptr, *d_pqs = nullptr, *d_D = nullptr;
    double *d_W1 = nullptr, *d_W2 = nullptr, *d_emode = nullptr, *d_Einst = nullptr;
    double *d_ekp = nullptr, *d_edp = nullptr, *d_hist = nullptr, *d_Mdisp = nullptr, *d_Q = nullptr;
    float *d_mlpX = nullptr, *d_mlpR = nullptr, *d_mlpZl = nullptr, *d_mlpf = nullptr;
    void *d_mlpw = nullptr;                  // bfloat16 network parameters
    bool mixed = false;                      // tensor-core coupling (modes on a grid)
    bool generic = false;                    // cells other than 3-atom, 6-orbital ones: persistent kernel
    bool moving = false;                     // mode functions at the cells' centres of mass
    bool periodic = false;                   // periodic cells (Gamma point): their own kernel
    bool rs = false;                         // the paper's real-space photon scheme
    RsArgs rsa{};
    PbcPlan pplan{};
    double *d_Us = nullptr, *d_Wk2 = nullptr, *d_Wk1 = nullptr, *d_watom = nullptr;
    double *d_G1 = nullptr, *d_Ginst = nullptr, *d_G2 = nullptr;   // [N][3] position-term gradients
    double *d_U0 = nullptr, *d_Us0 = nullptr;   // mode functions and sines at the reference positions
    std::vector<double> h_watom;             // m_j / m_n
    GenericPlan gplan{};
    long long *d_Coff = nullptr;             // eigenvector block of each cell (generic kernel)
    int water_warps = 2, water_per_warp = 5; // launch shape of the water kernel
    long long n_cwarm = 0;                   // doubles in the warm-start eigenvector blocks
    std::string tuning = "not tuned (options.autotune = 0): default launch shapes";
    AcfArgs acf{};                           // on-device autocorrelation (acf.L > 0)
    double *d_acf_out = nullptr;
    TcPlan tc{};
    double *d_G = nullptr, *d_E2 = nullptr, *d_E1 = nullptr;
    float *d_Wt2 = nullptr, *d_Wt1 = nullptr;
    unsigned *d_done = nullptr, *d_status = nullptr;
    long long *d_step = nullptr;
    unsigned *d_pack = nullptr;                // read-out packing: iteration maximum and ticket
    std::vector<void *> allocs;
    // host-side bookkeeping
    unsigned *h_status = nullptr;   // pinned
    double *d_obs = nullptr, *h_obs = nullptr;   // packed observables, device and pinned host
    // the second read-out slot and the state of both (cavmd_observables_async / _wait)
    double *d_obs1 = nullptr, *h_obs1 = nullptr;
    cudaEvent_t obs_ev[2] = {nullptr, nullptr};   // a slot's copy has landed
    cudaEvent_t obs_packed[2] = {nullptr, nullptr};   // a slot's snapshot is packed on the device
    cudaStream_t copy_stream = nullptr;             // device-to-host copies of the read-out
    bool obs_queued[2] = {false, false}, obs_arrays[2] = {false, false};
    int64_t obs_step[2] = {0, 0};
    cudaEvent_t status_ev = nullptr;
    bool status_pending = false;
    std::map<int, cudaGraphExec_t> graphs;   // keyed by the Born refresh phase of the first step
    int graph_steps = 0;
    int n_disp = 0;                          // finite-difference rows per cell (0: Mulliken)
    int64_t step = 0;
    std::string err;
    // phase timers
    bool timing = false;
    bool timing_all = true;                  // events around every phase (else only phase 0)
    struct Pending { cudaEvent_t a, b; int phase; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> ev_free;
    double phase_ms[CAVMD_N_PHASES] = {0, 0, 0, 0};
    int64_t phase_cnt[CAVMD_N_PHASES] = {0, 0, 0, 0};
    StepArgs sa{};
    DftbArgs da{};
};

namespace {

int fail(cavmd_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg; else g_init_error = msg;
    return code;
}

int cuda_fail(cavmd_ctx *c, cudaError_t e, const char *what) {
    return fail(c, CAVMD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                                       cudaGetErrorString(e) + ")");
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);     \
    } while (0)

int dalloc(cavmd_ctx *c, void **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void *q = nullptr;
    if (c->opt.dev_alloc) {
        q = c->opt.dev_alloc(bytes, c->opt.alloc_user);
        if (!q) return fail(c, CAVMD_ERR_NOMEM, "device allocator callback returned NULL");
    } else {
        cudaError_t e = cudaMalloc(&q, bytes);
        if (e != cudaSuccess) return fail(c, CAVMD_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    c->allocs.push_back(q);
    *p = q;
    return CAVMD_OK;
}

template <typename T>
int dalloc_n(cavmd_ctx *c, T **p, size_t n) {
    return dalloc(c, reinterpret_cast<void **>(p), n * sizeof(T));
}

// Frees a buffer of dalloc before the context ends (scratch of the tuner).
void dfree(cavmd_ctx *c, void *p) {
    if (!p) return;
    auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
    if (it != c->allocs.end()) c->allocs.erase(it);
    if (c->opt.dev_free) c->opt.dev_free(p, c->opt.alloc_user);
    else cudaFree(p);
}

#define AL(ptr, n)                                   \
    do {                                             \
        int rc_ = dalloc_n(c, &(ptr), (size_t)(n));  \
        if (rc_) return rc_;                         \
    } while (0)

int status_to_code(cavmd_ctx *c, unsigned st) {
    if (!st) return CAVMD_OK;
    if (st & ERRBIT_NONFINITE) return fail(c, CAVMD_ERR_NONFINITE, "non-finite energy in the state");
    if (st & ERRBIT_S_NOT_PD) return fail(c, CAVMD_ERR_S_NOT_PD, "an overlap matrix is not positive definite");
    if (st & ERRBIT_ZERO_GAP) return fail(c, CAVMD_ERR_ZERO_GAP, "HOMO-LUMO gap below threshold");
    // a bounded loop that ran out is the cause of any non-convergence that follows it
    if (st & ERRBIT_TIMEOUT)
        return fail(c, CAVMD_ERR_DEVICE_TIMEOUT,
                    "a bounded device loop ran out (the Jacobi sweeps of a cold start, or a tensor-core wait)");
    if (st & ERRBIT_SCC_NOCONV) return fail(c, CAVMD_ERR_SCC_NOCONV, "SCC charges did not converge within scc_max_iter");
    return fail(c, CAVMD_ERR_CUDA, "unknown device status");
}

// Waits for the queued work, reads and clears the device status word.
int sync_status(cavmd_ctx *c) {
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(c->h_status, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    const unsigned st = *c->h_status;
    c->status_pending = false;
    if (st) {
        CK(cudaMemset(c->d_status, 0, sizeof(unsigned)));
        return status_to_code(c, st);
    }
    return CAVMD_OK;
}

cudaEvent_t get_event(cavmd_ctx *c) {
    if (!c->ev_free.empty()) {
        cudaEvent_t e = c->ev_free.back();
        c->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

struct PhaseScope {
    cavmd_ctx *c;
    cavmd_ctx::Pending pd{};
    bool on;
    PhaseScope(cavmd_ctx *c_, int phase) : c(c_), on(c_->timing && (c_->timing_all || phase == 0)) {
        if (on) {
            pd.a = get_event(c);
            pd.b = get_event(c);
            pd.phase = phase;
            cudaEventRecord(pd.a, c->stream);
        }
    }
    ~PhaseScope() {
        if (on) {
            cudaEventRecord(pd.b, c->stream);
            c->pending.push_back(pd);
        }
    }
};

void collect_phase_times(cavmd_ctx *c) {
    for (auto &pd : c->pending) {
        float ms = 0.f;
        cudaEventSynchronize(pd.b);
        cudaEventElapsedTime(&ms, pd.a, pd.b);
        c->phase_ms[pd.phase] += ms;
        c->phase_cnt[pd.phase] += 1;
        c->ev_free.push_back(pd.a);
        c->ev_free.push_back(pd.b);
    }
    c->pending.clear();
}

cudaError_t run_dftb(cavmd_ctx *c, int have_warm) {
    PhaseScope ps(c, 0);
    c->da.have_warm = have_warm;
    if (c->periodic) return launch_dftb_periodic(c->d_sk, c->da, c->pplan, c->stream);
    if (c->generic) return launch_dftb_generic(c->d_sk, c->da, c->gplan, c->stream);
    return launch_dftb_water(c->d_sk, c->da, c->stream, c->water_warps, c->water_per_warp);
}

// Finite-difference dipole derivatives at the current positions (after the cell evaluation).
cudaError_t run_born(cavmd_ctx *c) {
    PhaseScope ps(c, 3);
    DftbArgs d = c->da;
    d.have_warm = 1;
    d.n_disp = c->n_disp;
    d.fd_central = c->opt.charge_model == CAVMD_CHARGE_BORN_CENTRAL;
    d.fd_h = c->opt.fd_step;
    d.M_disp = c->d_Mdisp;
    cudaError_t e = c->periodic ? launch_dftb_periodic(c->d_sk, d, c->pplan, c->stream)
                    : c->generic ? launch_dftb_generic(c->d_sk, d, c->gplan, c->stream)
                                 : launch_dftb_water(c->d_sk, d, c->stream, c->water_warps, c->water_per_warp);
    if (e != cudaSuccess) return e;
    return launch_born_assemble(c->N, c->d_off, c->d_Mc, c->d_Mdisp, c->n_disp, d.fd_central, d.fd_h, c->d_b,
                                c->stream);
}

// Network dipole derivatives at the current positions (after the cell evaluation).
cudaError_t run_mlp(cavmd_ctx *c) {
    PhaseScope ps(c, 3);
    // the water kernel's cells hold 3 atoms each, at 3 n .. 3 n + 2
    cudaError_t e = launch_mlp_features(c->N, c->d_off, c->d_species, c->d_r, c->d_mlpX, c->d_mlpR, c->d_status,
                                        c->stream, (c->generic || c->periodic) ? 0 : 3);
    if (e == cudaSuccess) e = launch_mlp_forward(c->n_atoms, c->d_mlpX, c->d_mlpR, c->d_mlpw, c->d_mlpZl, c->d_status, c->stream);
    if (e == cudaSuccess)
        e = launch_mlp_born(c->N, c->d_off, c->d_mlpZl, c->d_mlpR, c->d_Q, c->pol[0], c->pol[1], c->pol[2], c->d_b,
                            c->stream);
    return e;
}

bool born_refresh(const cavmd_ctx *c, int64_t eval_index) {
    return c->n_disp > 0 && (eval_index % c->opt.born_interval) == 0;
}

cudaError_t run_tc_forward(cavmd_ctx *c) {
    PhaseScope ps(c, 1);
    return launch_tc_forward(c->tc, c->d_Mc, c->d_G, c->d_status, c->stream);
}

// Back product for the second half-flow (Wt2 -> E2) and, when `first`, the next first half-flow
// (Wt1 -> E1); with second = false only Wt1 -> E1. Moving mode positions take one launch per
// half-flow, each with the gradients (G2, G1).
cudaError_t run_tc_back(cavmd_ctx *c, bool second, bool first) {
    PhaseScope ps(c, 2);
    if (c->moving) {
        cudaError_t e = cudaSuccess;
        if (second) e = launch_tc_back(c->tc, c->d_Wt2, nullptr, c->d_E2, nullptr, c->d_status, c->stream, c->d_G2);
        if (e == cudaSuccess && first)
            e = launch_tc_back(c->tc, c->d_Wt1, nullptr, c->d_E1, nullptr, c->d_status, c->stream, c->d_G1);
        return e;
    }
    if (second)
        return launch_tc_back(c->tc, c->d_Wt2, first ? c->d_Wt1 : nullptr, c->d_E2, first ? c->d_E1 : nullptr,
                              c->d_status, c->stream);
    return launch_tc_back(c->tc, c->d_Wt1, nullptr, c->d_E1, nullptr, c->d_status, c->stream);
}

cudaError_t run_photon(cavmd_ctx *c, int flags) {
    PhaseScope ps(c, 1);
    return launch_photon(c->sa, flags, c->stream);
}

// Mode functions and their sines at the current cell centres of mass (moving mode positions); with
// the tensor-core coupling, its phase panels.
cudaError_t run_modes(cavmd_ctx *c) {
    PhaseScope ps(c, 1);
    if (c->mixed) return launch_tc_panels_com(c->tc, c->d_r, c->d_mass, c->d_off, c->stream);
    return launch_mode_functions_com(c->d_k, c->d_R, c->d_U0, c->d_Us0, c->d_r, c->d_mass, c->d_off, c->M, c->N,
                                     c->d_U, c->d_Us, c->stream);
}

cudaError_t run_rs(cavmd_ctx *c, int what, int flags) {
    PhaseScope ps(c, 1);
    return launch_rs(c->rsa, c->sa, what, flags, c->stream);
}

cudaError_t run_field(cavmd_ctx *c, int flags) {
    PhaseScope ps(c, 2);
    return launch_field(c->sa, flags, c->stream);
}

// One autocorrelation sample of the synchronised state (after the energy record).
cudaError_t run_acf(cavmd_ctx *c) {
    if (c->acf.L <= 0) return cudaSuccess;
    PhaseScope ps(c, 2);
    return launch_acf(c->acf, c->d_qs, c->d_Mc, c->N, c->stream);
}

cudaError_t reset_acf(cavmd_ctx *c) {
    if (c->acf.L <= 0) return cudaSuccess;
    const size_t cl = (size_t)c->acf.C * c->acf.L;
    cudaError_t e = cudaMemsetAsync(c->acf.ring, 0, sizeof(double) * (size_t)c->acf.C * (c->acf.L + c->acf.B),
                                    c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->acf.head, 0, sizeof(double) * cl, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->acf.acc, 0, sizeof(double) * cl, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->acf.sum, 0, sizeof(double) * c->acf.C, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->acf.n, 0, sizeof(long long), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->acf.ticket, 0, sizeof(unsigned), c->stream);
    return e;
}

// Queues n >= 1 steps starting and ending at a synchronised state; the first queued step is
// step number first_step (evaluation index = step number, init being evaluation 0).
cudaError_t enqueue_steps(cavmd_ctx *c, int64_t n, int64_t first_step) {
    cudaError_t e;
    // The opening first half-flow: its field E1 was formed at the end of the previous call (or by
    // cavmd_init / cavmd_set_state) from the same synchronised state, so only the photon rotation
    // and the kick and drift remain. Water systems fold them into the first step's launches: the
    // SCC-DFTB kernel kicks and drifts the atoms of its cells before reading their positions, and
    // the photon kernel rotates the modes before their second half-flow. The cluster kernel takes
    // two launches of their own.
    const bool fold = !c->generic && !c->moving && !c->periodic && !c->rs;
    if (c->rs) {
        if ((e = run_rs(c, RS_OPEN, 0)) != cudaSuccess) return e;
        if ((e = run_field(c, FLD_FIRST | FLD_E_GIVEN)) != cudaSuccess) return e;
    } else if (!fold) {
        if ((e = run_photon(c, PH_FIRST)) != cudaSuccess) return e;
        if ((e = run_field(c, FLD_FIRST | FLD_E_GIVEN)) != cudaSuccess) return e;
    }
    for (int64_t s = 0; s < n; ++s) {
        const bool last = (s == n - 1);
        const int open = (fold && s == 0) ? PH_OPEN : 0;
        c->da.E_open = open ? c->d_E1 : nullptr;
        e = run_dftb(c, 1);
        c->da.E_open = nullptr;
        if (e != cudaSuccess) return e;
        if (c->moving && (e = run_modes(c)) != cudaSuccess) return e;   // positions of this step
        if (born_refresh(c, first_step + s) && (e = run_born(c)) != cudaSuccess) return e;
        if (c->d_mlpw && (e = run_mlp(c)) != cudaSuccess) return e;
        if (c->rs) {   // Step 1's second half-kick, Steps 2-4, the next first half-kick
            if ((e = run_rs(c, RS_SECOND, 0)) != cudaSuccess) return e;
            if ((e = run_rs(c, RS_FORWARD, 1)) != cudaSuccess) return e;
            if ((e = run_rs(c, RS_BACK, 1 | (last ? 0 : 2))) != cudaSuccess) return e;
            if ((e = run_field(c, FLD_SECOND | FLD_ENERGY | FLD_E_GIVEN | (last ? 0 : FLD_FIRST))) != cudaSuccess)
                return e;
        } else if (c->mixed) {
            if ((e = run_tc_forward(c)) != cudaSuccess) return e;
            if ((e = run_photon(c, open | PH_FORWARD_G | PH_SECOND | PH_ENERGY | (last ? PH_W1 : PH_FIRST))) !=
                cudaSuccess)
                return e;
            if ((e = run_tc_back(c, true, true)) != cudaSuccess) return e;   // E1 also for the next call
            if ((e = run_field(c, FLD_SECOND | FLD_ENERGY | FLD_E_GIVEN | (last ? 0 : FLD_FIRST))) != cudaSuccess)
                return e;
        } else {
            if ((e = run_photon(c, open | PH_FORWARD | PH_SECOND | PH_ENERGY | (last ? PH_W1 : PH_FIRST))) != cudaSuccess)
                return e;
            if ((e = run_field(c, FLD_SECOND | FLD_ENERGY | (last ? FLD_E1_STORE : FLD_FIRST))) != cudaSuccess) return e;
        }
        if ((e = run_acf(c)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Launch-shape tuner. Candidates differ only in how work is mapped to threads and blocks, never in
// arithmetic, so every candidate gives bitwise identical results:
//   cluster kernel: product entries per thread per pass (2 or 4) x persistent blocks per SM;
//   water kernel: warps per block (2, 4 or 8), five waters per warp. (Fewer waters per warp would
//   change which waters share a warp, and the warp-wide choice between a Jacobi sweep and the
//   second-order update couples them, so it is not a candidate; it was never faster either.)
// Each candidate evaluates a trial step (positions drifted by dt p / m, warm started from a copy of
// the converged state) twice, timed with CUDA events on the context's stream; the fastest is kept.
// The context's own state is not touched.
int autotune(cavmd_ctx *c) {
    if (c->periodic) {
        c->tuning = c->pplan.nk > 0 ? "k_dftb_periodic_kg: one 256-thread block per cell, one per SM (no candidates)"
                                    : "k_dftb_periodic: one 256-thread block per cell, two per SM (no candidates)";
        return CAVMD_OK;
    }
    const int NA = c->n_atoms, N = c->N;
    cudaStream_t st = c->stream;
    const long long ncw = c->n_cwarm;
    double *r_t = nullptr, *F_t = nullptr, *b_t = nullptr, *qp_t = nullptr, *qv_t = nullptr, *C_t = nullptr;
    double *E_t = nullptr, *M_t = nullptr, *Q_t = nullptr;
    int *it_t = nullptr;
    unsigned *st_t = nullptr;
    AL(r_t, 3 * NA); AL(F_t, 3 * NA); AL(b_t, 3 * NA); AL(qp_t, NA); AL(qv_t, NA); AL(C_t, ncw);
    AL(E_t, N); AL(M_t, N); AL(Q_t, NA); AL(it_t, N); AL(st_t, 1);
    CK(launch_trial_positions(c->d_r, c->d_p, c->d_imass, c->opt.dt, NA, r_t, st));
    DftbArgs t = c->da;
    t.r = r_t; t.F = F_t; t.b = b_t; t.qpop = qp_t; t.qprev = qv_t; t.Cwarm = C_t; t.E_cell = E_t;
    t.M_cell = M_t; t.iters = it_t; t.status = st_t; t.Qout = Q_t; t.have_warm = 1; t.n_disp = 0;
    t.M_disp = nullptr;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    struct Cand { int a, b; float ms; };
    std::vector<Cand> cands;
    if (c->generic) {
        for (int r : {2, 4})
            for (int b = 1; b <= c->gplan.max_blocks_per_sm; ++b) cands.push_back({r, b, 0.f});
    } else {
        for (int w : {2, 4, 8}) cands.push_back({w, 5, 0.f});
    }
    for (auto &cd : cands) {
        cd.ms = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            CK(cudaMemcpyAsync(qp_t, c->d_qpop, sizeof(double) * NA, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(qv_t, c->d_qprev, sizeof(double) * NA, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(C_t, c->d_C, sizeof(double) * ncw, cudaMemcpyDeviceToDevice, st));
            CK(cudaEventRecord(e0, st));
            if (c->generic) {
                GenericPlan g = c->gplan;
                g.r_entries = cd.a;
                g.blocks_per_sm = cd.b;
                CK(launch_dftb_generic(c->d_sk, t, g, st));
            } else {
                CK(launch_dftb_water(c->d_sk, t, st, cd.a, cd.b));
            }
            CK(cudaEventRecord(e1, st));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            cd.ms = std::min(cd.ms, ms);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const Cand *best = &cands[0];
    for (auto &cd : cands)
        if (cd.ms < best->ms) best = &cd;
    char buf[160];
    std::string rep;
    if (c->generic) {
        c->gplan.r_entries = best->a;
        c->gplan.blocks_per_sm = best->b;
        std::snprintf(buf, sizeof(buf), "k_dftb_generic: r_entries=%d blocks_per_sm=%d (%.3f ms); candidates:",
                      best->a, best->b, best->ms);
        rep = buf;
        for (auto &cd : cands) {
            std::snprintf(buf, sizeof(buf), " r%d/b%d %.3f ms", cd.a, cd.b, cd.ms);
            rep += buf;
        }
    } else {
        c->water_warps = best->a;
        c->water_per_warp = best->b;
        std::snprintf(buf, sizeof(buf), "dftb_kernel<3,6>: warps_per_block=%d waters_per_warp=%d (%.3f ms); candidates:",
                      best->a, best->b, best->ms);
        rep = buf;
        for (auto &cd : cands) {
            std::snprintf(buf, sizeof(buf), " w%d/g%d %.3f ms", cd.a, cd.b, cd.ms);
            rep += buf;
        }
    }
    c->tuning = rep;
    for (void *p : {(void *)r_t, (void *)F_t, (void *)b_t, (void *)qp_t, (void *)qv_t, (void *)C_t, (void *)E_t,
                    (void *)M_t, (void *)Q_t, (void *)it_t, (void *)st_t})
        dfree(c, p);
    return CAVMD_OK;
}

int initial_evaluation(cavmd_ctx *c, bool init_photons) {
    CK(run_dftb(c, 0));
    if (c->moving) CK(run_modes(c));
    if (c->n_disp > 0) CK(run_born(c));
    if (c->d_mlpw) CK(run_mlp(c));
    if (c->rs) {   // the synchronised photons, their energies and the next first half-kick's field
        const int mode = !init_photons ? 0 : (c->opt.photon_init == CAVMD_PHOTON_ZERO ? 2 : 1);
        CK(run_rs(c, RS_INIT, mode));
        CK(run_rs(c, RS_FORWARD, 0));
        CK(run_rs(c, RS_BACK, 0));
        CK(run_field(c, FLD_ENERGY | FLD_E_GIVEN));
        return sync_status(c);
    }
    int fwd = PH_FORWARD;
    if (c->mixed) {
        CK(run_tc_forward(c));
        fwd = PH_FORWARD_G;
    }
    // energies of the synchronised state, and the field of the next first half-flow (kept for the
    // opening of the next cavmd_step call)
    if (init_photons) {
        const int pf = (c->opt.photon_init == CAVMD_PHOTON_ZERO) ? PH_INIT_ZERO : PH_INIT_RELAXED;
        CK(run_photon(c, fwd | pf | PH_ENERGY | PH_W1));
    } else {
        CK(run_photon(c, fwd | PH_ENERGY | PH_W1));   // keeps q_sync / pq_sync
    }
    if (c->mixed) CK(run_tc_back(c, false, true));
    CK(run_field(c, FLD_ENERGY | (c->mixed ? 0 : FLD_E1_STORE)));
    return sync_status(c);
}

void fill_devsk(const cavmd_sk_tables *t, DevSK *d) {
    std::memset(d, 0, sizeof(*d));
    for (int e = 0; e < CAVMD_MAX_ELEM; ++e) {
        d->onsite[e][0] = t->onsite[e][0];
        d->onsite[e][1] = t->onsite[e][1];
        d->hubbard[e] = t->hubbard[e];
        d->zval[e] = t->zval[e];
        d->norb[e] = t->norb[e];
    }
    std::memcpy(d->h0, t->h0, sizeof(d->h0));
    std::memcpy(d->s, t->s, sizeof(d->s));
    std::memcpy(d->rep, t->rep, sizeof(d->rep));
    for (int x = 0; x < CAVMD_MAX_ELEM; ++x)   // host IEEE division and product: the device's bits
        for (int y = 0; y < CAVMD_MAX_ELEM; ++y) {
            const double s2 = t->hubbard[x] + t->hubbard[y];
            const double cc = s2 != 0.0 ? 2.0 / s2 : 0.0;
            d->gamma_c2[x][y] = cc * cc;
        }
    d->r_cut = t->r_cut;
    d->taper = t->taper;
    d->inv_taper = 1.0 / t->taper;
}

// Modes on a uniform in-plane grid in the order a = s + 2 (jy + Ky2 jx), k = (jx dkx, jy dky, 0),
// phase 0 (s = 0) or -pi/2 (s = 1): the structure the tensor-core contraction factorises.
bool detect_grid(const cavmd_modes *md, int &Kx, int &Ky2, double &dkx, double &dky, std::string &why) {
    const int M = md->n_modes;
    dkx = 0.0;
    dky = 0.0;
    for (int a = 0; a < M; ++a) {
        const double kx = md->k[3 * a], ky = md->k[3 * a + 1], kz = md->k[3 * a + 2];
        if (kz != 0.0 || kx < 0.0 || ky < 0.0) { why = "modes need k_z = 0 and k_x, k_y >= 0"; return false; }
        if (kx > 0.0 && (dkx == 0.0 || kx < dkx)) dkx = kx;
        if (ky > 0.0 && (dky == 0.0 || ky < dky)) dky = ky;
    }
    int mx = 0, my = 0;
    std::vector<int> jxs(M), jys(M);
    for (int a = 0; a < M; ++a) {
        const double kx = md->k[3 * a], ky = md->k[3 * a + 1];
        const long jx = dkx > 0.0 ? std::lround(kx / dkx) : 0, jy = dky > 0.0 ? std::lround(ky / dky) : 0;
        if (std::fabs(kx - jx * dkx) > 1e-9 * dkx || std::fabs(ky - jy * dky) > 1e-9 * dky) {
            why = "mode wave vectors are not on a uniform grid";
            return false;
        }
        jxs[a] = (int)jx;
        jys[a] = (int)jy;
        mx = std::max(mx, (int)jx);
        my = std::max(my, (int)jy);
    }
    Kx = mx + 1;
    Ky2 = my + 1;
    if (M != 2 * Kx * Ky2) { why = "mode count is not 2 Kx Ky2"; return false; }
    for (int a = 0; a < M; ++a) {
        const int s = a & 1, rem = a >> 1;
        if (jxs[a] != rem / Ky2 || jys[a] != rem % Ky2) { why = "modes are not ordered a = s + 2 (jy + Ky2 jx)"; return false; }
        const double ph = s == 0 ? 0.0 : -1.5707963267948966;
        if (std::fabs(md->phi[a] - ph) > 1e-12) { why = "mode phases must be 0 (cos) and -pi/2 (sin)"; return false; }
    }
    if (2 * Kx > 128) { why = "2 Kx must not exceed 128"; return false; }
    return true;
}

int padded_ky(int Ky2) {
    const int need = 2 * Ky2;
    const int sizes[] = {16, 32, 48, 64, 96, 128};
    for (int v : sizes)
        if (v >= need) return v;
    return 0;
}

// Grid points of the k-grid option (1: the Gamma point).
int kgrid_points(const cavmd_options *o) {
    if (o->kgrid[0] == 0 && o->kgrid[1] == 0 && o->kgrid[2] == 0) return 1;
    return o->kgrid[0] * o->kgrid[1] * o->kgrid[2];
}

int validate(const cavmd_system *sys, const cavmd_sk_tables *sk, const cavmd_modes *md,
             const cavmd_options *o) {
    cavmd_ctx *c = nullptr;
    if (!sys || !sk || !md || !o) return fail(c, CAVMD_ERR_INVALID_ARG, "NULL argument");
    if (sys->n_cells < 1 || sys->n_atoms < 1) return fail(c, CAVMD_ERR_INVALID_ARG, "need n_cells >= 1 and n_atoms >= 1");
    if (!sys->cell_offset || !sys->species || !sys->r || !sys->p) return fail(c, CAVMD_ERR_INVALID_ARG, "NULL system array");
    if (sk->n_elem < 1 || sk->n_elem > CAVMD_MAX_ELEM) return fail(c, CAVMD_ERR_INVALID_ARG, "n_elem out of range");
    for (int e = 0; e < sk->n_elem; ++e)
        if (sk->norb[e] != 1 && sk->norb[e] != 4) return fail(c, CAVMD_ERR_INVALID_ARG, "norb must be 1 or 4");
    if (!(sk->taper > 0.0) || !(sk->r_cut > sk->taper)) return fail(c, CAVMD_ERR_INVALID_ARG, "need r_cut > taper > 0");
    if (sys->cell_offset[0] != 0 || sys->cell_offset[sys->n_cells] != sys->n_atoms)
        return fail(c, CAVMD_ERR_INVALID_ARG, "cell_offset must start at 0 and end at n_atoms");
    for (int i = 0; i < sys->n_atoms; ++i)
        if (sys->species[i] < 0 || sys->species[i] >= sk->n_elem) return fail(c, CAVMD_ERR_INVALID_ARG, "species id out of range");
    for (int i = 0; i < 3 * sys->n_atoms; ++i)
        if (!std::isfinite(sys->r[i]) || !std::isfinite(sys->p[i])) return fail(c, CAVMD_ERR_INVALID_ARG, "non-finite position or momentum");
    const bool per = sys->lattice != nullptr;
    if (per) {
        const double *L = sys->lattice;
        for (int k = 0; k < 9; ++k)
            if (!std::isfinite(L[k])) return fail(c, CAVMD_ERR_INVALID_ARG, "non-finite lattice vector");
        const double det = L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                           L[2] * (L[3] * L[7] - L[4] * L[6]);
        if (!(std::fabs(det) > 1e-6)) return fail(c, CAVMD_ERR_INVALID_ARG, "lattice vectors are linearly dependent");
        if (o->charge_model == CAVMD_CHARGE_BORN_MLP)
            return fail(c, CAVMD_ERR_UNSUPPORTED, "periodic cells take Mulliken or finite-difference Born charges");
    }
    for (int n = 0; n < sys->n_cells; ++n) {
        const int a0 = sys->cell_offset[n], a1 = sys->cell_offset[n + 1];
        if (a1 <= a0) return fail(c, CAVMD_ERR_INVALID_ARG, "every cell needs at least one atom");
        int norb = 0;
        double nel = 0;
        for (int i = a0; i < a1; ++i) { norb += sk->norb[sys->species[i]]; nel += sk->zval[sys->species[i]]; }
        const long ne = std::lround(nel);
        if (std::fabs(nel - ne) > 1e-12 || (ne & 1) || ne <= 0 || ne > 2 * norb)
            return fail(c, CAVMD_ERR_INVALID_ARG, "cells must be neutral and closed shell");
        if (per) {
            if (norb > CAVMD_MAX_PERIODIC_ORBITALS || (norb & 1) || a1 - a0 > CAVMD_MAX_PERIODIC_ATOMS)
                return fail(c, CAVMD_ERR_UNSUPPORTED, "periodic cells need an even number of orbitals, at most 256, "
                                                      "and at most 128 atoms");
            if (ne / 2 >= norb) return fail(c, CAVMD_ERR_UNSUPPORTED, "periodic cells need an empty orbital");
        } else if (norb > CAVMD_MAX_CELL_ORBITALS || (norb & 1)) {
            return fail(c, CAVMD_ERR_UNSUPPORTED, "cells need an even number of orbitals, at most 64");
        }
    }
    if (!per) {   // shared memory of the persistent kernel for the largest cells
        std::vector<int> norb_e(sk->norb, sk->norb + sk->n_elem);
        GenericPlan gp{};
        std::vector<int2> it, dit;
        plan_dftb_generic(sys->cell_offset, sys->species, norb_e.data(), sys->n_cells, 0, gp, it, dit);
        if (gp.smem > 227 * 1024 - 256)   // the opt-in limit per block, less the kernel's static bytes
            return fail(c, CAVMD_ERR_UNSUPPORTED, "cells too large for on-chip storage (" +
                        std::to_string(gp.smem) + " bytes of shared memory per block)");
    }
    if (md->n_modes < 1 || !md->k || !md->omega || !md->lambda || !md->phi)
        return fail(c, CAVMD_ERR_INVALID_ARG, "need n_modes >= 1 and all mode arrays");
    for (int a = 0; a < md->n_modes; ++a)
        if (!(md->omega[a] > 0.0) || !std::isfinite(md->omega[a]) || !std::isfinite(md->lambda[a]) ||
            !std::isfinite(md->phi[a]))
            return fail(c, CAVMD_ERR_INVALID_ARG, "mode frequencies must be positive and finite");
    if (!(o->dt > 0.0) || !std::isfinite(o->dt)) return fail(c, CAVMD_ERR_INVALID_ARG, "dt must be positive");
    if (!(o->scc_tol > 0.0) || o->scc_max_iter < 1) return fail(c, CAVMD_ERR_INVALID_ARG, "bad SCC tolerance or iteration limit");
    if (!(o->mixing > 0.0 && o->mixing <= 1.0)) return fail(c, CAVMD_ERR_INVALID_ARG, "mixing must be in (0, 1]");
    if (o->precision == CAVMD_PREC_MIXED_TF32)
        return fail(c, CAVMD_ERR_UNSUPPORTED, "CAVMD_PREC_MIXED_TF32 is not built; use CAVMD_PREC_MIXED_BF16X3");
    if (o->precision != CAVMD_PREC_FP64 && o->precision != CAVMD_PREC_MIXED_BF16X3)
        return fail(c, CAVMD_ERR_INVALID_ARG, "bad precision");
    if (o->charge_model < CAVMD_CHARGE_MULLIKEN || o->charge_model > CAVMD_CHARGE_BORN_MLP)
        return fail(c, CAVMD_ERR_INVALID_ARG, "bad charge_model");
    if (o->charge_model != CAVMD_CHARGE_MULLIKEN && (o->born_interval < 1 || !(o->fd_step > 0.0)))
        return fail(c, CAVMD_ERR_INVALID_ARG, "Born charges need born_interval >= 1 and fd_step > 0");
    if (o->splitting != CAVMD_SPLIT_PHOTON_EXACT && o->splitting != CAVMD_SPLIT_PAPER &&
        o->splitting != CAVMD_SPLIT_STRANG && o->splitting != CAVMD_SPLIT_REAL_SPACE)
        return fail(c, CAVMD_ERR_INVALID_ARG, "bad splitting");
    if (o->splitting == CAVMD_SPLIT_REAL_SPACE) {
        if (!(o->real_space_g0 > 0.0) || !(o->real_space_omega0 > 0.0) || !std::isfinite(o->real_space_g0) ||
            !std::isfinite(o->real_space_omega0))
            return fail(c, CAVMD_ERR_INVALID_ARG, "CAVMD_SPLIT_REAL_SPACE needs real_space_g0 > 0 and real_space_omega0 > 0");
        if (md->n_modes != sys->n_cells)
            return fail(c, CAVMD_ERR_INVALID_ARG, "CAVMD_SPLIT_REAL_SPACE needs as many modes as cells");
        if (o->precision != CAVMD_PREC_FP64 || o->mode_positions != CAVMD_MODES_FIXED)
            return fail(c, CAVMD_ERR_UNSUPPORTED, "CAVMD_SPLIT_REAL_SPACE takes the FP64 coupling and fixed mode positions");
    }
    if (o->photon_init != CAVMD_PHOTON_RELAXED && o->photon_init != CAVMD_PHOTON_ZERO)
        return fail(c, CAVMD_ERR_INVALID_ARG, "bad photon_init");
    if (o->graph_chunk < 0 || o->energy_history < 1) return fail(c, CAVMD_ERR_INVALID_ARG, "bad graph_chunk or energy_history");
    if ((o->dev_alloc == nullptr) != (o->dev_free == nullptr)) return fail(c, CAVMD_ERR_INVALID_ARG, "dev_alloc and dev_free go together");
    if (o->acf_lags < 0 || (o->autotune != 0 && o->autotune != 1))
        return fail(c, CAVMD_ERR_INVALID_ARG, "acf_lags must be >= 0 and autotune 0 or 1");
    if (o->scc_history < 1 || o->scc_history > 6) return fail(c, CAVMD_ERR_INVALID_ARG, "scc_history must be 1..6");
    if (o->jacobi_max_sweeps < 0 || o->jacobi_max_sweeps > 1000)
        return fail(c, CAVMD_ERR_INVALID_ARG, "jacobi_max_sweeps must be 0..1000");
    if (o->mode_positions != CAVMD_MODES_FIXED && o->mode_positions != CAVMD_MODES_CENTRE_OF_MASS)
        return fail(c, CAVMD_ERR_INVALID_ARG, "bad mode_positions");
    if (o->mode_positions == CAVMD_MODES_CENTRE_OF_MASS && o->splitting != CAVMD_SPLIT_PHOTON_EXACT)
        return fail(c, CAVMD_ERR_UNSUPPORTED, "moving mode positions take the photon-exact splitting");
    {
        const bool zero = o->kgrid[0] == 0 && o->kgrid[1] == 0 && o->kgrid[2] == 0;
        for (int k = 0; k < 3; ++k)
            if (!zero && (o->kgrid[k] < 1 || o->kgrid[k] > 8))
                return fail(c, CAVMD_ERR_INVALID_ARG, "kgrid entries must be 1..8 (or all 0)");
        if (kgrid_points(o) > 1 && !sys->lattice)
            return fail(c, CAVMD_ERR_INVALID_ARG, "a k-grid needs periodic cells (cavmd_system.lattice)");
    }
    if (o->precision == CAVMD_PREC_MIXED_BF16X3) {
        int Kx, Ky2;
        double dkx, dky;
        std::string why;
        if (!detect_grid(md, Kx, Ky2, dkx, dky, why))
            return fail(c, CAVMD_ERR_UNSUPPORTED, "mixed-precision coupling needs modes on a grid: " + why);
        if (!padded_ky(Ky2)) return fail(c, CAVMD_ERR_UNSUPPORTED, "2 Ky2 must not exceed 128");
    }
    return CAVMD_OK;
}

void release(cavmd_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    for (auto &pd : c->pending) { cudaEventDestroy(pd.a); cudaEventDestroy(pd.b); }
    for (auto e : c->ev_free) cudaEventDestroy(e);
    for (void *p : c->allocs) {
        if (c->opt.dev_free) c->opt.dev_free(p, c->opt.alloc_user);
        else cudaFree(p);
    }
    if (c->status_ev) cudaEventDestroy(c->status_ev);
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->h_obs) cudaFreeHost(c->h_obs);
    if (c->h_obs1) cudaFreeHost(c->h_obs1);
    for (auto e : c->obs_ev)
        if (e) cudaEventDestroy(e);
    for (auto e : c->obs_packed)
        if (e) cudaEventDestroy(e);
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
    }
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int build_context(cavmd_ctx *c, const cavmd_system *sys, const cavmd_sk_tables *sk, const cavmd_modes *md) {
    const int N = c->N, NA = c->n_atoms, M = c->M;
    CK(cudaSetDevice(c->device));
    if (c->opt.stream) {
        c->stream = (cudaStream_t)c->opt.stream;
    } else {
        CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    CK(cudaMallocHost(&c->h_status, sizeof(unsigned)));
    CK(cudaMallocHost(&c->h_obs, sizeof(double) * (16 + (size_t)c->N + 3 * (size_t)c->M)));
    CK(cudaMallocHost(&c->h_obs1, sizeof(double) * (16 + (size_t)c->N + 3 * (size_t)c->M)));
    CK(cudaEventCreateWithFlags(&c->status_ev, cudaEventDisableTiming));
    for (auto &e : c->obs_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    for (auto &e : c->obs_packed) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));

    // host-side derived arrays
    std::vector<double> mass(NA), imass(NA), R(3 * N);
    for (int i = 0; i < NA; ++i) { mass[i] = sk->mass[sys->species[i]]; imass[i] = 1.0 / mass[i]; }
    for (int n = 0; n < N; ++n) {
        if (sys->R_ref) {
            for (int k = 0; k < 3; ++k) R[3 * n + k] = sys->R_ref[3 * n + k];
        } else {
            double mt = 0, x[3] = {0, 0, 0};
            for (int i = sys->cell_offset[n]; i < sys->cell_offset[n + 1]; ++i) {
                mt += mass[i];
                for (int k = 0; k < 3; ++k) x[k] += mass[i] * sys->r[3 * i + k];
            }
            for (int k = 0; k < 3; ++k) R[3 * n + k] = x[k] / mt;
        }
    }
    std::vector<double> iw(M), cw(M), sw(M), omc(M);
    const double tau = 0.5 * c->opt.dt;
    for (int a = 0; a < M; ++a) {
        const double w = md->omega[a];
        iw[a] = 1.0 / w;
        cw[a] = std::cos(w * tau);
        sw[a] = std::sin(w * tau);
        omc[a] = (1.0 - cw[a]) / w;
    }
    DevSK hsk;
    fill_devsk(sk, &hsk);

    AL(c->d_sk, 1);
    AL(c->d_off, N + 1); AL(c->d_species, NA); AL(c->d_iters, N); AL(c->d_acell, NA);
    AL(c->d_r, 3 * NA); AL(c->d_p, 3 * NA); AL(c->d_F, 3 * NA); AL(c->d_b, 3 * NA);
    // eigenvector blocks: n_c^2 per cell; the water kernel takes every cell when all are 3-atom,
    // 6-orbital cells, the persistent generic kernel otherwise
    std::vector<long long> coff(N + 1, 0);
    c->generic = false;
    // k-grid: a basis per irreducible k-point, each the real form of twice the orbitals
    std::vector<double> kpts;
    if (sys->lattice && kgrid_points(&c->opt) > 1) kpts = pbc_kpoints(c->opt.kgrid);
    const int nk = (int)(kpts.size() / 4);
    for (int n = 0; n < N; ++n) {
        int no = 0;
        for (int i = sys->cell_offset[n]; i < sys->cell_offset[n + 1]; ++i) no += sk->norb[sys->species[i]];
        if (!sys->lattice && (no != 6 || sys->cell_offset[n + 1] - sys->cell_offset[n] != 3)) c->generic = true;
        coff[n + 1] = coff[n] + (nk > 0 ? 4LL * nk : 1LL) * no * no;
    }
    c->n_cwarm = coff[N];
    AL(c->d_qpop, NA); AL(c->d_qprev, NA); AL(c->d_C, (size_t)coff[N]); AL(c->d_E, N); AL(c->d_Mc, N);
    c->periodic = sys->lattice != nullptr;
    if (!c->generic && !c->periodic) CK(prepare_dftb_water(8));
    AL(c->d_mass, NA); AL(c->d_imass, NA); AL(c->d_Einst, N); AL(c->d_E1, N);
    c->mixed = c->opt.precision == CAVMD_PREC_MIXED_BF16X3;
    if (!c->mixed) AL(c->d_U, (size_t)M * N);
    c->moving = c->opt.mode_positions == CAVMD_MODES_CENTRE_OF_MASS;
    if (c->moving) {
        if (!c->mixed) {   // FP64 mode functions and sines (the tensor-core path forms phase panels)
            AL(c->d_Us, (size_t)M * N); AL(c->d_Wk2, 3 * M); AL(c->d_Wk1, 3 * M);
            AL(c->d_U0, (size_t)M * N); AL(c->d_Us0, (size_t)M * N);
        } else {
            AL(c->d_G2, 3 * N);
        }
        AL(c->d_watom, NA); AL(c->d_G1, 3 * N); AL(c->d_Ginst, 3 * N);
        c->h_watom.assign(NA, 0.0);
        for (int n = 0; n < N; ++n) {
            double mt = 0.0;
            for (int i = sys->cell_offset[n]; i < sys->cell_offset[n + 1]; ++i) mt += mass[i];
            for (int i = sys->cell_offset[n]; i < sys->cell_offset[n + 1]; ++i) c->h_watom[i] = mass[i] / mt;
        }
    }
    AL(c->d_k, 3 * M); AL(c->d_phi, M); AL(c->d_R, 3 * N);
    AL(c->d_omega, M); AL(c->d_lam, M); AL(c->d_iomega, M); AL(c->d_cos, M); AL(c->d_sin, M); AL(c->d_omc, M);
    AL(c->d_q, M); AL(c->d_pq, M); AL(c->d_qs, M); AL(c->d_pqs, M); AL(c->d_D, M);
    AL(c->d_W1, M); AL(c->d_W2, M); AL(c->d_emode, 4 * M);
    const int fb = field_blocks(N);
    AL(c->d_ekp, fb); AL(c->d_edp, fb); AL(c->d_hist, 8 * (size_t)c->opt.energy_history);
    AL(c->d_done, 1); AL(c->d_status, 1); AL(c->d_step, 1); AL(c->d_pack, 2);
    AL(c->d_obs, 16 + (size_t)N + 3 * (size_t)M);
    AL(c->d_obs1, 16 + (size_t)N + 3 * (size_t)M);
    // finite-difference copies: 3 per atom (forward) or 6 (central); n_disp counts them per water
    // cell for the water kernel, the generic kernel walks its own item list
    int disp_per_atom = 0;
    if (c->opt.charge_model == CAVMD_CHARGE_BORN_FD) disp_per_atom = 3;
    if (c->opt.charge_model == CAVMD_CHARGE_BORN_CENTRAL) disp_per_atom = 6;
    c->n_disp = 3 * disp_per_atom;
    if (c->n_disp) AL(c->d_Mdisp, (size_t)disp_per_atom * NA);
    if (c->opt.charge_model == CAVMD_CHARGE_BORN_MLP) {
        CK(prepare_mlp_forward());
        AL(c->d_Q, NA);
        AL(c->d_mlpX, (size_t)NA * CAVMD_MLP_NFEAT);
        AL(c->d_mlpR, (size_t)NA * 9);
        AL(c->d_mlpZl, (size_t)NA * 9);
        AL(c->d_mlpf, CAVMD_MLP_NPARAMS);
        void *w = nullptr;
        int rc = dalloc(c, &w, (size_t)CAVMD_MLP_NPARAMS * 2);
        if (rc) return rc;
        c->d_mlpw = w;
        CK(cudaMemsetAsync(c->d_mlpw, 0, (size_t)CAVMD_MLP_NPARAMS * 2, c->stream));   // zero network
    }

    cudaStream_t st = c->stream;
    CK(cudaMemcpyAsync(c->d_sk, &hsk, sizeof(DevSK), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_off, sys->cell_offset, sizeof(int) * (N + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_species, sys->species, sizeof(int) * NA, cudaMemcpyHostToDevice, st));
    {
        std::vector<int> acell(NA);
        for (int n = 0; n < N; ++n)
            for (int i = sys->cell_offset[n]; i < sys->cell_offset[n + 1]; ++i) acell[i] = n;
        CK(cudaMemcpyAsync(c->d_acell, acell.data(), sizeof(int) * NA, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));   // acell is pageable and local
    }
    CK(cudaMemcpyAsync(c->d_r, sys->r, sizeof(double) * 3 * NA, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_p, sys->p, sizeof(double) * 3 * NA, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_mass, mass.data(), sizeof(double) * NA, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_imass, imass.data(), sizeof(double) * NA, cudaMemcpyHostToDevice, st));
    if (c->moving)
        CK(cudaMemcpyAsync(c->d_watom, c->h_watom.data(), sizeof(double) * NA, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_R, R.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_k, md->k, sizeof(double) * 3 * M, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_phi, md->phi, sizeof(double) * M, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_omega, md->omega, sizeof(double) * M, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_lam, md->lambda, sizeof(double) * M, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_iomega, iw.data(), sizeof(double) * M, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_cos, cw.data(), sizeof(double) * M, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_sin, sw.data(), sizeof(double) * M, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_omc, omc.data(), sizeof(double) * M, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(c->d_done, 0, sizeof(unsigned), st));
    CK(cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), st));
    CK(cudaMemsetAsync(c->d_step, 0, sizeof(long long), st));
    CK(cudaMemsetAsync(c->d_pack, 0, 2 * sizeof(unsigned), st));
    CK(cudaMemsetAsync(c->d_hist, 0, sizeof(double) * 8 * c->opt.energy_history, st));
    CK(cudaMemsetAsync(c->d_q, 0, sizeof(double) * M, st));
    CK(cudaMemsetAsync(c->d_pq, 0, sizeof(double) * M, st));
    if (c->moving && !c->mixed) {
        CK(launch_mode_functions_pair(c->d_k, c->d_phi, c->d_R, M, N, c->d_U0, c->d_Us0, st));
        CK(cudaMemcpyAsync(c->d_U, c->d_U0, sizeof(double) * M * N, cudaMemcpyDeviceToDevice, st));
    } else if (!c->mixed) {
        CK(launch_mode_functions(c->d_k, c->d_phi, c->d_R, M, N, c->d_U, st));
    } else {
        TcPlan &p = c->tc;
        std::string why;
        detect_grid(md, p.Kx, p.Ky2, p.dkx, p.dky, why);
        p.KY = padded_ky(p.Ky2);
        p.N = N;
        p.Npad = ((N + 127) / 128) * 128;
        CK(cudaDeviceGetAttribute(&p.n_sm, cudaDevAttrMultiProcessorCount, c->device));
        p.n_fwd_cta = std::min(p.Npad / tc_fwd_stage_cells(), p.n_sm);
        const size_t np = (size_t)p.Npad;
        AL(p.Ahi, 128 * np); AL(p.Alo, 128 * np); AL(p.Af, 128 * np); AL(p.Bsrc, (size_t)p.KY * np);
        AL(p.Yhi, (size_t)p.KY * np); AL(p.Ylo, (size_t)p.KY * np);
        AL(p.partial, (size_t)p.n_fwd_cta * 128 * p.KY);
        AL(c->d_G, 128 * (size_t)p.KY); AL(c->d_Wt2, 128 * (size_t)p.KY); AL(c->d_Wt1, 128 * (size_t)p.KY);
        AL(c->d_E2, N);
        CK(cudaMemsetAsync(c->d_Wt2, 0, sizeof(float) * 128 * p.KY, st));
        CK(cudaMemsetAsync(c->d_Wt1, 0, sizeof(float) * 128 * p.KY, st));
        CK(tc_prepare(p.KY));
        CK(launch_tc_panels(p, c->d_R, st));   // moving positions: the zero padding; run_modes fills the rest
    }

    c->rs = c->opt.splitting == CAVMD_SPLIT_REAL_SPACE;
    if (c->rs) {
        RsArgs &r = c->rsa;
        const double g0 = c->opt.real_space_g0, w0 = c->opt.real_space_omega0;
        r.eta = std::sqrt(2.0 * N) * g0 * w0;
        r.eta2_w0sq = r.eta * r.eta / (w0 * w0);
        r.inv_w0sq = 1.0 / (w0 * w0);
        r.sq = std::sqrt(0.5 * w0);
        r.isq = 1.0 / std::sqrt(2.0 * w0);
        r.inv_sq = 1.0 / r.sq;
        r.inv_isq = 1.0 / r.isq;
        std::vector<double> wa(M), cd(M), sd(M);
        for (int a = 0; a < M; ++a) {
            wa[a] = md->lambda[a] * md->lambda[a] / (2.0 * N * g0 * g0);
            cd[a] = std::cos(md->omega[a] * c->opt.dt);
            sd[a] = std::sin(md->omega[a] * c->opt.dt);
        }
        double *w_ = nullptr, *c_ = nullptr, *s_ = nullptr;
        AL(w_, M); AL(c_, M); AL(s_, M);
        AL(r.x, N); AL(r.y, N); AL(r.Xw, M); AL(r.Yw, M); AL(r.E2, N);
        r.E1 = c->d_E1;
        r.w = w_;
        r.cdt = c_;
        r.sdt = s_;
        CK(cudaMemcpyAsync(w_, wa.data(), sizeof(double) * M, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(c_, cd.data(), sizeof(double) * M, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(s_, sd.data(), sizeof(double) * M, cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(c->d_D, 0, sizeof(double) * M, st));
        CK(cudaMemsetAsync(c->d_emode, 0, sizeof(double) * 4 * M, st));
        CK(cudaStreamSynchronize(st));   // the host vectors must outlive the copies
    }

    if (c->opt.acf_lags > 0) {
        AcfArgs &a = c->acf;
        a.M = M;
        a.C = M + 1;
        a.L = c->opt.acf_lags;
        a.B = 16;
        const size_t cl = (size_t)a.C * a.L;
        AL(a.ring, (size_t)a.C * (a.L + a.B)); AL(a.head, cl); AL(a.acc, cl); AL(a.sum, a.C); AL(a.n, 1);
        AL(a.ticket, 1);
        a.G = std::max((a.M + 7) / 8, std::min(2048, (c->N + 255) / 256));   // 8 channels (warps) per block
        AL(a.part, a.G);
        AL(c->d_acf_out, cl);
        CK(reset_acf(c));
    }
    if (c->generic) {
        GenericPlan &g = c->gplan;
        std::vector<int> norb_e(sk->norb, sk->norb + sk->n_elem);
        std::vector<int2> items, disp_items;
        plan_dftb_generic(sys->cell_offset, sys->species, norb_e.data(), N, disp_per_atom, g, items, disp_items);
        AL(g.items, items.size());
        AL(g.queue, 2);
        CK(cudaMemcpyAsync(g.items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, st));
        if (!disp_items.empty()) {
            AL(g.disp_items, disp_items.size());
            CK(cudaMemcpyAsync(g.disp_items, disp_items.data(), sizeof(int2) * disp_items.size(),
                               cudaMemcpyHostToDevice, st));
        }
        AL(c->d_Coff, N);
        CK(cudaMemcpyAsync(c->d_Coff, coff.data(), sizeof(long long) * N, cudaMemcpyHostToDevice, st));
        CK(prepare_dftb_generic(g));
        // the host vectors must outlive the copies
        CK(cudaStreamSynchronize(st));
    }

    if (c->periodic) {
        PbcPlan &pp = c->pplan;
        std::vector<double> img, gw;
        plan_dftb_periodic(sys->lattice, sk->r_cut, pp, img, gw);
        if (pp.n_img > 200000 || pp.n_g > 20000)
            return fail(c, CAVMD_ERR_UNSUPPORTED, "lattice too thin: " + std::to_string(pp.n_img) + " lattice images");
        pp.nmax = 0;
        pp.amax = 0;
        pp.nk = nk;
        for (int n = 0; n < N; ++n) {
            pp.nmax = std::max(pp.nmax, (int)std::lround(std::sqrt((double)(coff[n + 1] - coff[n]) /
                                                                   (nk > 0 ? 4.0 * nk : 1.0))));
            pp.amax = std::max(pp.amax, sys->cell_offset[n + 1] - sys->cell_offset[n]);
        }
        int nsm = 0;
        CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
        pp.blocks = std::max(1, std::min(N, (nk > 0 ? 1 : 2) * nsm));
        AL(pp.d_img, img.size());
        AL(pp.d_gw, gw.size());
        AL(pp.work, pbc_workspace_doubles(pp.nmax, pp.amax, pp.n_g, nk) * (size_t)pp.blocks);
        if (nk > 0) {
            AL(pp.d_kpt, kpts.size());
            CK(cudaMemcpyAsync(pp.d_kpt, kpts.data(), sizeof(double) * kpts.size(), cudaMemcpyHostToDevice, st));
        }
        CK(cudaMemcpyAsync(pp.d_img, img.data(), sizeof(double) * img.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(pp.d_gw, gw.data(), sizeof(double) * gw.size(), cudaMemcpyHostToDevice, st));
        AL(c->d_Coff, N);
        CK(cudaMemcpyAsync(c->d_Coff, coff.data(), sizeof(long long) * N, cudaMemcpyHostToDevice, st));
        CK(prepare_dftb_periodic());
        CK(cudaStreamSynchronize(st));   // the host vectors must outlive the copies
    }

    DftbArgs &d = c->da;
    d.n_cells = N;
    d.cell_list = nullptr;
    d.cell_offset = c->d_off;
    d.species = c->d_species;
    d.r = c->d_r;
    d.F = c->d_F;
    d.b = c->d_b;
    d.qpop = c->d_qpop;
    d.qprev = c->d_qprev;
    d.Cwarm = c->d_C;
    d.Cwarm_off = c->d_Coff;
    d.E_cell = c->d_E;
    d.M_cell = c->d_Mc;
    d.iters = c->d_iters;
    d.status = c->d_status;
    d.pol0 = c->pol[0];
    d.pol1 = c->pol[1];
    d.pol2 = c->pol[2];
    d.scc_tol = c->opt.scc_tol;
    d.beta = c->opt.mixing;
    d.max_iter = c->opt.scc_max_iter;
    d.hist = c->opt.scc_history;
    d.have_warm = 0;
    d.max_sweeps = c->opt.jacobi_max_sweeps;
    d.write_b = c->opt.charge_model == CAVMD_CHARGE_MULLIKEN;
    d.n_disp = 0;
    d.fd_central = 0;
    d.fd_h = c->opt.fd_step;
    d.M_disp = nullptr;
    d.Qout = c->d_Q;

    StepArgs &s = c->sa;
    s.N = N; s.M = M; s.n_atoms = NA;
    s.cell_offset = c->d_off; s.U = c->d_U; s.M_cell = c->d_Mc; s.E_cell = c->d_E;
    s.inv_mass = c->d_imass; s.mass = c->d_mass; s.F = c->d_F; s.b = c->d_b; s.r = c->d_r; s.p = c->d_p;
    s.omega = c->d_omega; s.lam = c->d_lam; s.inv_omega = c->d_iomega;
    s.cos_h = c->d_cos; s.sin_h = c->d_sin; s.omc_h = c->d_omc;
    s.q = c->d_q; s.pq = c->d_pq; s.q_sync = c->d_qs; s.pq_sync = c->d_pqs; s.D = c->d_D;
    s.W1 = c->d_W1; s.W2 = c->d_W2; s.e_mode = c->d_emode; s.e_kin_part = c->d_ekp; s.e_dftb_part = c->d_edp;
    s.done_counter = c->d_done; s.hist = c->d_hist; s.hist_cap = c->opt.energy_history;
    s.step_counter = c->d_step; s.status = c->d_status; s.dt = c->opt.dt; s.tau = tau;
    s.G = c->d_G; s.Wt2 = c->d_Wt2; s.Wt1 = c->d_Wt1; s.E2in = c->rs ? c->rsa.E2 : c->d_E2; s.E1in = c->d_E1;
    s.E1store = c->d_E1;
    s.Kx = c->tc.Kx; s.Ky2 = c->tc.Ky2; s.KY = c->tc.KY;
    s.Us = c->d_Us; s.kvec = c->d_k; s.Wk2 = c->d_Wk2; s.Wk1 = c->d_Wk1; s.w_atom = c->d_watom;
    s.atom_cell = c->d_acell;
    s.G1store = c->d_G1; s.G1in = c->d_G1;   // all NULL with fixed mode positions
    s.G2in = c->d_G2;                          // tensor-core coupling with moving mode positions only
    s.paper = c->opt.splitting == CAVMD_SPLIT_PAPER || c->opt.splitting == CAVMD_SPLIT_STRANG;
    s.strang = c->opt.splitting == CAVMD_SPLIT_STRANG;
    d.E_open = nullptr;   // set for the first evaluation of a call (water kernel)
    d.p_open = c->d_p; d.r_open = c->d_r; d.inv_mass = c->d_imass; d.tau = tau; d.dt = c->opt.dt;
    d.step_counter = c->d_step;
    return CAVMD_OK;
}

}  // namespace

extern "C" {

void cavmd_default_options(cavmd_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->dt = 0.5 * 41.341373335;
    o->precision = CAVMD_PREC_FP64;
    o->charge_model = CAVMD_CHARGE_MULLIKEN;
    o->born_interval = 3;
    o->fd_step = 1e-3;
    o->scc_tol = 1e-12;
    o->scc_max_iter = 200;
    o->mixing = 0.7;
    o->splitting = CAVMD_SPLIT_PHOTON_EXACT;
    o->photon_init = CAVMD_PHOTON_RELAXED;
    o->graph_chunk = 50;
    o->device = 0;
    o->energy_history = 1024;
    o->scc_history = 3;
    o->kgrid[0] = o->kgrid[1] = o->kgrid[2] = 1;
}

int cavmd_init(cavmd_ctx **out, const cavmd_system *sys, const cavmd_sk_tables *sk,
               const cavmd_modes *md, const cavmd_options *opt) {
    if (!out) return fail(nullptr, CAVMD_ERR_INVALID_ARG, "ctx pointer is NULL");
    *out = nullptr;
    int rc = validate(sys, sk, md, opt);
    if (rc) return rc;
    cavmd_ctx *c = new cavmd_ctx();
    c->opt = *opt;
    c->device = opt->device;
    c->N = sys->n_cells;
    c->n_atoms = sys->n_atoms;
    c->M = md->n_modes;
    c->h_off.assign(sys->cell_offset, sys->cell_offset + sys->n_cells + 1);
    c->h_species.assign(sys->species, sys->species + sys->n_atoms);
    for (int k = 0; k < 3; ++k) c->pol[k] = md->pol[k];
    rc = build_context(c, sys, sk, md);
    if (!rc) rc = initial_evaluation(c, true);
    if (!rc && c->opt.autotune) rc = autotune(c);
    if (!rc) {
        const cudaError_t e = run_acf(c);
        if (e != cudaSuccess) rc = cuda_fail(c, e, "autocorrelation sample");
    }
    if (rc) {
        g_init_error = c->err;
        release(c);
        return rc;
    }
    *out = c;
    return CAVMD_OK;
}

int cavmd_step(cavmd_ctx *c, int64_t nsteps) {
    if (!c) return fail(nullptr, CAVMD_ERR_INVALID_ARG, "NULL context");
    if (nsteps < 0) return fail(c, CAVMD_ERR_INVALID_ARG, "nsteps < 0");
    int rc = CAVMD_OK;
    if (c->status_pending) {   // the status of earlier work, only if it has finished: no wait here
        const cudaError_t q = cudaEventQuery(c->status_ev);
        if (q == cudaSuccess) {
            c->status_pending = false;
            const unsigned st = *c->h_status;
            if (st) {
                CK(cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream));
                rc = status_to_code(c, st);
            }
        } else if (q != cudaErrorNotReady) {
            return cuda_fail(c, q, "cudaEventQuery");
        }
    }
    if (nsteps == 0) return rc;
    CK(cudaSetDevice(c->device));
    int64_t left = nsteps;
    int64_t next = c->step + 1;                      // step number of the next queued step
    int G = c->opt.graph_chunk;
    if (c->n_disp > 0 && G > 0) G = ((G + c->opt.born_interval - 1) / c->opt.born_interval) * c->opt.born_interval;
    if (G > 0 && !c->timing && left >= G) {
        const int phase = c->n_disp > 0 ? (int)(next % c->opt.born_interval) : 0;
        auto it = c->graphs.find(phase);
        if (it == c->graphs.end()) {
            cudaGraph_t g;
            cudaGraphExec_t ge;
            CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = enqueue_steps(c, G, next);
            cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
            if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch during graph capture");
            if (e2 != cudaSuccess) return cuda_fail(c, e2, "cudaStreamEndCapture");
            CK(cudaGraphInstantiate(&ge, g, 0));
            cudaGraphDestroy(g);
            it = c->graphs.emplace(phase, ge).first;
            c->graph_steps = G;
        }
        while (left >= G) {   // G is a multiple of born_interval: every chunk starts at this phase
            CK(cudaGraphLaunch(it->second, c->stream));
            left -= G;
            next += G;
        }
    }
    if (left > 0) {
        cudaError_t e = enqueue_steps(c, left, next);
        if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
    }
    c->step += nsteps;
    CK(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaEventRecord(c->status_ev, c->stream));
    c->status_pending = true;
    return rc;
}

int cavmd_observables_async(cavmd_ctx *c, int32_t slot, int32_t with_arrays) {
    if (!c || slot < 0 || slot > 1) return fail(c, CAVMD_ERR_INVALID_ARG, "slot must be 0 or 1");
    // one packing kernel and one copy into the slot's pinned buffer, both queued behind the steps
    const int hs = (int)(c->step % c->opt.energy_history);
    const bool arrays = with_arrays != 0;
    const size_t cnt = 16 + (arrays ? (size_t)c->N + 3 * (size_t)c->M : 0);
    double *d = slot ? c->d_obs1 : c->d_obs, *h = slot ? c->h_obs1 : c->h_obs;
    // the snapshot is packed in stream order (the next step overwrites what it reads); its copy to
    // the host runs on a side stream, overlapping the next step. The slot's previous copy must have
    // left the device buffer before it is packed again.
    CK(cudaStreamWaitEvent(c->stream, c->obs_ev[slot], 0));
    CK(launch_obs_pack(c->d_hist + 8 * (size_t)hs, c->d_iters, c->N, c->d_status, c->d_Mc, c->d_qs, c->d_pqs,
                       c->d_D, c->M, arrays, d, c->d_pack, c->stream));
    CK(cudaEventRecord(c->obs_packed[slot], c->stream));
    CK(cudaStreamWaitEvent(c->copy_stream, c->obs_packed[slot], 0));
    CK(cudaMemcpyAsync(h, d, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->copy_stream));
    CK(cudaEventRecord(c->obs_ev[slot], c->copy_stream));
    c->obs_queued[slot] = true;
    c->obs_arrays[slot] = arrays;
    c->obs_step[slot] = c->step;
    return CAVMD_OK;
}

int cavmd_observables_wait(cavmd_ctx *c, int32_t slot, cavmd_obs *o) {
    if (!c || !o || slot < 0 || slot > 1) return fail(c, CAVMD_ERR_INVALID_ARG, "NULL argument or bad slot");
    if (!c->obs_queued[slot]) return fail(c, CAVMD_ERR_INVALID_ARG, "no read-out queued in this slot");
    if ((o->M || o->q || o->p || o->D) && !c->obs_arrays[slot])
        return fail(c, CAVMD_ERR_INVALID_ARG, "the read-out of this slot was queued without arrays");
    CK(cudaEventSynchronize(c->obs_ev[slot]));
    c->obs_queued[slot] = false;
    const double *h = slot ? c->h_obs1 : c->h_obs;
    int rc = CAVMD_OK;
    const unsigned st = (unsigned)h[9];
    if (st) {
        CK(cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream));
        rc = status_to_code(c, st);
    }
    o->e_kin = h[0];
    o->e_dftb = h[1];
    o->e_photon = h[2];
    o->e_coupling = h[3];
    o->e_dse = h[4];
    o->e_photon_free = h[5];
    o->e_total = h[6];
    o->temperature = 2.0 * h[0] / (3.0 * c->n_atoms * 3.166811563e-6);
    o->step = c->obs_step[slot];
    o->scc_iter_max = (int32_t)h[8];
    const size_t N = c->N, M = c->M;
    if (o->M) std::memcpy(o->M, h + 16, sizeof(double) * N);
    if (o->q) std::memcpy(o->q, h + 16 + N, sizeof(double) * M);
    if (o->p) std::memcpy(o->p, h + 16 + N + M, sizeof(double) * M);
    if (o->D) std::memcpy(o->D, h + 16 + N + 2 * M, sizeof(double) * M);
    return rc;
}

int cavmd_observables(cavmd_ctx *c, cavmd_obs *o) {
    if (!c || !o) return fail(c, CAVMD_ERR_INVALID_ARG, "NULL argument");
    int rc = cavmd_observables_async(c, 0, (o->M || o->q || o->p || o->D) ? 1 : 0);
    if (rc) return rc;
    rc = cavmd_observables_wait(c, 0, o);
    return rc;
}

int cavmd_energy_history(cavmd_ctx *c, double *out, int32_t n, int32_t *n_out) {
    if (!c || !out || n < 0) return fail(c, CAVMD_ERR_INVALID_ARG, "bad argument");
    int rc = sync_status(c);
    const int64_t cap = c->opt.energy_history;
    const int64_t avail = (c->step + 1 < cap) ? c->step + 1 : cap;
    const int64_t cnt = n < avail ? n : avail;
    std::vector<double> all(8 * (size_t)cap);
    CK(cudaMemcpy(all.data(), c->d_hist, sizeof(double) * 8 * cap, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < cnt; ++i) {
        const int64_t stp = c->step - cnt + 1 + i;
        std::memcpy(out + 8 * i, all.data() + 8 * (stp % cap), 8 * sizeof(double));
    }
    if (n_out) *n_out = (int32_t)cnt;
    return rc;
}

int cavmd_autocorrelation(cavmd_ctx *c, double *out, int32_t n_lags, int64_t *n_samples, int32_t reset) {
    if (!c || !out) return fail(c, CAVMD_ERR_INVALID_ARG, "NULL argument");
    if (c->acf.L <= 0) return fail(c, CAVMD_ERR_INVALID_ARG, "the context was made with acf_lags = 0");
    if (n_lags != c->acf.L) return fail(c, CAVMD_ERR_INVALID_ARG, "n_lags differs from the context's acf_lags");
    int rc = sync_status(c);
    CK(launch_acf_finalize(c->acf, c->d_acf_out, c->stream));
    long long n = 0;
    CK(cudaMemcpyAsync(&n, c->acf.n, sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(out, c->d_acf_out, sizeof(double) * (size_t)c->acf.C * c->acf.L, cudaMemcpyDeviceToHost,
                       c->stream));
    if (reset) CK(reset_acf(c));
    CK(cudaStreamSynchronize(c->stream));
    if (n_samples) *n_samples = n;
    return rc;
}

int cavmd_tuning(cavmd_ctx *c, char *buf, int32_t len) {
    if (!c || !buf || len < 1) return fail(c, CAVMD_ERR_INVALID_ARG, "bad argument");
    std::snprintf(buf, (size_t)len, "%s", c->tuning.c_str());
    return CAVMD_OK;
}

int cavmd_get_state(cavmd_ctx *c, cavmd_state *s) {
    if (!c || !s) return fail(c, CAVMD_ERR_INVALID_ARG, "NULL argument");
    int rc = sync_status(c);
    if (s->r) CK(cudaMemcpy(s->r, c->d_r, sizeof(double) * 3 * c->n_atoms, cudaMemcpyDeviceToHost));
    if (s->p) CK(cudaMemcpy(s->p, c->d_p, sizeof(double) * 3 * c->n_atoms, cudaMemcpyDeviceToHost));
    if (s->q) CK(cudaMemcpy(s->q, c->d_qs, sizeof(double) * c->M, cudaMemcpyDeviceToHost));
    if (s->pq) CK(cudaMemcpy(s->pq, c->d_pqs, sizeof(double) * c->M, cudaMemcpyDeviceToHost));
    s->step = c->step;
    return rc;
}

int cavmd_set_state(cavmd_ctx *c, const cavmd_state *s) {
    if (!c || !s || !s->r || !s->p || !s->q || !s->pq) return fail(c, CAVMD_ERR_INVALID_ARG, "NULL argument");
    int rc = sync_status(c);
    if (rc) return rc;
    for (int i = 0; i < 3 * c->n_atoms; ++i)
        if (!std::isfinite(s->r[i]) || !std::isfinite(s->p[i])) return fail(c, CAVMD_ERR_INVALID_ARG, "non-finite state");
    CK(cudaMemcpy(c->d_r, s->r, sizeof(double) * 3 * c->n_atoms, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_p, s->p, sizeof(double) * 3 * c->n_atoms, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_qs, s->q, sizeof(double) * c->M, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_pqs, s->pq, sizeof(double) * c->M, cudaMemcpyHostToDevice));
    long long stp = s->step;
    CK(cudaMemcpy(c->d_step, &stp, sizeof(long long), cudaMemcpyHostToDevice));
    c->step = s->step;
    rc = initial_evaluation(c, false);   // Born charges, if any, are refreshed here as well
    if (rc) return rc;
    CK(reset_acf(c));                      // a new trajectory segment: its own correlation functions
    CK(run_acf(c));
    return sync_status(c);
}

int cavmd_get_eval(cavmd_ctx *c, cavmd_eval *o) {
    if (!c || !o) return fail(c, CAVMD_ERR_INVALID_ARG, "NULL argument");
    int rc = sync_status(c);
    const size_t NA = c->n_atoms, N = c->N;
    if (o->F_dftb) CK(cudaMemcpy(o->F_dftb, c->d_F, sizeof(double) * 3 * NA, cudaMemcpyDeviceToHost));
    if (o->b) CK(cudaMemcpy(o->b, c->d_b, sizeof(double) * 3 * NA, cudaMemcpyDeviceToHost));
    if (o->q_pop) CK(cudaMemcpy(o->q_pop, c->d_qpop, sizeof(double) * NA, cudaMemcpyDeviceToHost));
    if (o->E_cell) CK(cudaMemcpy(o->E_cell, c->d_E, sizeof(double) * N, cudaMemcpyDeviceToHost));
    if (o->M) CK(cudaMemcpy(o->M, c->d_Mc, sizeof(double) * N, cudaMemcpyDeviceToHost));
    if (o->scc_iters) CK(cudaMemcpy(o->scc_iters, c->d_iters, sizeof(int) * N, cudaMemcpyDeviceToHost));
    if (o->F_total) {
        // instantaneous field with W_a = lambda_a (omega_a q_a - D_a), on the device
        std::vector<double> q(c->M), D(c->M), w(c->M), lam(c->M), W(c->M);
        CK(cudaMemcpy(q.data(), c->d_qs, sizeof(double) * c->M, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(D.data(), c->d_D, sizeof(double) * c->M, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(w.data(), c->d_omega, sizeof(double) * c->M, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(lam.data(), c->d_lam, sizeof(double) * c->M, cudaMemcpyDeviceToHost));
        for (int a = 0; a < c->M; ++a) W[a] = lam[a] * (w[a] * q[a] - D[a]);
        if (c->rs) {   // the local field -(eta q_n + eta^2 M_n / omega_0^2) of the real-space scheme
            std::vector<double> Mn(N), F(3 * NA), b(3 * NA);
            CK(cudaMemcpy(Mn.data(), c->d_Mc, sizeof(double) * N, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(F.data(), c->d_F, sizeof(double) * 3 * NA, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(b.data(), c->d_b, sizeof(double) * 3 * NA, cudaMemcpyDeviceToHost));
            for (size_t n = 0; n < N; ++n) {
                const double En = -(c->rsa.eta * q[n] + c->rsa.eta2_w0sq * Mn[n]);
                for (int i = c->h_off[n]; i < c->h_off[n + 1]; ++i)
                    for (int k = 0; k < 3; ++k) o->F_total[3 * i + k] = F[3 * i + k] + En * b[3 * i + k];
            }
            return rc;
        }
        if (c->mixed) {   // same arrangement of the weights as the photon kernel writes
            const TcPlan &p = c->tc;
            std::vector<float> Wt((size_t)128 * p.KY, 0.0f);
            for (int a = 0; a < c->M; ++a) {
                const int jx = a / (2 * p.Ky2), rem = a - jx * 2 * p.Ky2, jy = rem >> 1, sm = rem & 1;
                if (sm == 0) {
                    Wt[jx * p.KY + jy] = (float)W[a];
                    Wt[(p.Kx + jx) * p.KY + p.Ky2 + jy] = (float)(-W[a]);
                } else {
                    Wt[jx * p.KY + p.Ky2 + jy] = (float)W[a];
                    Wt[(p.Kx + jx) * p.KY + jy] = (float)W[a];
                }
            }
            CK(cudaMemcpy(c->d_Wt1, Wt.data(), sizeof(float) * Wt.size(), cudaMemcpyHostToDevice));
            CK(launch_tc_back(p, c->d_Wt1, nullptr, c->d_Einst, nullptr, c->d_status, c->stream,
                              c->moving ? c->d_Ginst : nullptr));
        } else {
            CK(cudaMemcpy(c->d_W1, W.data(), sizeof(double) * c->M, cudaMemcpyHostToDevice));
            CK(launch_field_only(c->d_U, c->d_W1, c->M, c->N, c->d_Einst, c->stream));
        }
        CK(cudaStreamSynchronize(c->stream));
        std::vector<double> E(N), F(3 * NA), b(3 * NA), G, Mn;
        if (c->moving) {   // position term: (m_j / m_n) M_n sum_a W_a grad u_a(R_n)
            if (!c->mixed) CK(launch_field_grad_only(c->d_Us, c->d_W1, c->d_k, c->M, c->N, c->d_Ginst, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            G.resize(3 * N);
            Mn.resize(N);
            CK(cudaMemcpy(G.data(), c->d_Ginst, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(Mn.data(), c->d_Mc, sizeof(double) * N, cudaMemcpyDeviceToHost));
        }
        CK(cudaMemcpy(E.data(), c->d_Einst, sizeof(double) * N, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(F.data(), c->d_F, sizeof(double) * 3 * NA, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(b.data(), c->d_b, sizeof(double) * 3 * NA, cudaMemcpyDeviceToHost));
        for (size_t n = 0; n < N; ++n)
            for (int i = c->h_off[n]; i < c->h_off[n + 1]; ++i)
                for (int k = 0; k < 3; ++k) {
                    o->F_total[3 * i + k] = F[3 * i + k] + E[n] * b[3 * i + k];
                    if (c->moving) o->F_total[3 * i + k] += c->h_watom[i] * Mn[n] * G[3 * n + k];
                }
    }
    return rc;
}

int cavmd_load_born_mlp(cavmd_ctx *c, const float *params, int32_t n_params) {
    if (!c) return fail(nullptr, CAVMD_ERR_INVALID_ARG, "NULL context");
    if (!params || n_params != CAVMD_MLP_NPARAMS) return fail(c, CAVMD_ERR_INVALID_ARG, "need CAVMD_MLP_NPARAMS parameters");
    if (!c->d_mlpw) return fail(c, CAVMD_ERR_INVALID_ARG, "context was not created with CAVMD_CHARGE_BORN_MLP");
    int rc = sync_status(c);
    if (rc) return rc;
    for (int i = 0; i < n_params; ++i)
        if (!std::isfinite(params[i])) return fail(c, CAVMD_ERR_INVALID_ARG, "non-finite network parameter");
    CK(cudaMemcpy(c->d_mlpf, params, sizeof(float) * n_params, cudaMemcpyHostToDevice));
    CK(launch_to_bf16(c->d_mlpf, c->d_mlpw, n_params, c->stream));
    CK(run_mlp(c));
    return sync_status(c);
}

int cavmd_phase_times(cavmd_ctx *c, int32_t enable, double *ms, int64_t *cnt, int32_t reset) {
    if (!c) return fail(nullptr, CAVMD_ERR_INVALID_ARG, "NULL context");
    CK(cudaStreamSynchronize(c->stream));
    collect_phase_times(c);
    for (int i = 0; i < CAVMD_N_PHASES; ++i) {
        if (ms) ms[i] = c->phase_ms[i];
        if (cnt) cnt[i] = c->phase_cnt[i];
        if (reset) { c->phase_ms[i] = 0; c->phase_cnt[i] = 0; }
    }
    if (enable < 0 || enable > 2) return fail(c, CAVMD_ERR_INVALID_ARG, "enable must be 0, 1 or 2");
    c->timing = enable != 0;
    c->timing_all = enable != 2;
    return CAVMD_OK;
}

const char *cavmd_last_error(const cavmd_ctx *c) {
    return c ? c->err.c_str() : g_init_error.c_str();
}

void cavmd_destroy(cavmd_ctx *c) { release(c); }

size_t cavmd_struct_size(int32_t which) {
    switch (which) {
        case 0: return sizeof(cavmd_system);
        case 1: return sizeof(cavmd_sk_tables);
        case 2: return sizeof(cavmd_modes);
        case 3: return sizeof(cavmd_options);
        case 4: return sizeof(cavmd_obs);
        case 5: return sizeof(cavmd_state);
        case 6: return sizeof(cavmd_eval);
        default: return 0;
    }
}

}  // extern "C"
