"""Benchmark: molecule-steps/s of the cavity-MD hot path on one GB300 (or N replicas).

Workload (default "c2"): 4096 synthetic waters (12,288 atoms) in a 919 x 30 x 30 bohr slab at
liquid density, 512 real cavity modes on an in-plane line of wave vectors, g = 0.001 a.u.,
dt = 0.5 fs, FP64 SCC-DFTB with Mulliken charges, photons initially at rest.

One timed step = one cavmd_step(ctx, 1) call: the whole hot path (SCC-DFTB of every cell,
dipoles, forward contraction, photon half-flows, field on every cell, kicks and drift,
energies). Each step is bracketed by CUDA events on the library's stream; a 256 MB buffer
(larger than the 129 MB L2) is rewritten between steps, outside the events.

Multi-GPU (torchrun): every rank propagates its own independent replica (its own velocities),
no data-path collective; value = all ranks' molecule-steps / max-over-ranks time (weak scaling).

--impl reference times the FP64 oracle (oracle/) on the host cores instead: each step runs the
oracle's full time step on a bounded sample of the same workload (its first 512 cells).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

FP64_FLOPS_PER_CLK_SM = 4.0      # 2 FP64 FMA per clock per SM (1.25 TFLOP/s nominal at 2.07 GHz)
N_SM = 152
SM_MAX_MHZ = 2070.0
FLUSH_BYTES = 256 << 20
# DRAM bytes (read + write) of one dftb_kernel<3,6> launch on this workload, from one ncu capture
# (profiles/dftb_kernel_c2_4096x512.md); None once the kernel has changed since that capture.
DFTB_DRAM_BYTES_PER_LAUNCH = (2908928 + 2905856 + 2907904 + 256) // 3   # mean of three in-step launches


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _reduce_max(x, ws, device):
    """The largest x over the ranks of the process group (x itself on one process)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _whole_job_value(n_mol_per_rank, steps, ws, max_ms):
    """Molecule-steps per second of the whole job: every rank's replica over the slowest rank's
    time (each rank runs the same workload)."""
    return n_mol_per_rank * steps * ws / (max_ms * 1e-3)


def _dftb_flops_per_cell(iters, n=6, nocc=4, npair=3):
    """Algorithmic FP64 flops of one cell (n orbitals, n_occ occupied, npair atom pairs) per time
    step: per SCC iteration 2n^3 (basis transform) + 9n^3 (symmetric eigensolve with vectors)
    + 2 n^2 n_occ (density) + 2 n^2 (Mulliken), plus 1000 per atom pair for the Slater-Koster
    build and the analytic forces. A water: 2736 per iteration + 3000."""
    n, nocc, npair = (np.asarray(x, float) for x in (n, nocc, npair))
    per_iter = 2 * n ** 3 + 9 * n ** 3 + 2 * n * n * nocc + 2 * n * n
    return per_iter * np.asarray(iters, float) + 1000.0 * npair


def _periodic_flops_per_cell(iters, n, nocc):
    """FP64 flops of the products one periodic cell needs per time step in the warm-started Gamma-point
    SCC (n orbitals, o = n_occ occupied, v = n - o virtual):
      start, once: S C (2n^3), C^T S C lower (n^3), its Cholesky (n^3/3), C L^-T (n^3);
      every SCC iteration: H C (2n^3), the occupied-virtual block of C^T H C (2 n o v), X^T X and X X^T
        lower (o^2 v + v^2 o), P lower (n^2 o), H, the diagonal and Mulliken (7 n^2);
      the rotation: on the first iteration the Cayley form, C_v X and C_o X^T (4 n o v), two Cholesky
        factors (o^3/3 + v^3/3) and their row solves (2 n (o^2 + v^2)); on the others
        C (I + K + K^2/2) as products over [C_o | C_v] (2 n^3);
      every step, one Jacobi sweep inside each block of m columns: the block C_b^T Y_b (2 n m^2),
        its rotations accumulated in V (9 m^3), and C_b V, Y_b V (4 n m^2);
      forces, once: H C_o (2 n^2 o), C_o^T H C_o lower (n o^2), t = 2 Aoo C_o^T (2 n o^2),
        W and P lower (2 n^2 o).
    A full eigensolve per iteration (the 9 n^3 of the isolated-cell count) is never done."""
    n = float(n)
    o = float(nocc)
    v = n - o
    it = np.asarray(iters, float)
    start = (2.0 + 1.0 + 1.0 / 3.0 + 1.0) * n ** 3
    common = 2 * n ** 3 + 2 * n * o * v + o * o * v + v * v * o + n * n * o + 7 * n * n
    cayley = 4 * n * o * v + (o ** 3 + v ** 3) / 3 + 2 * n * (o * o + v * v)
    second = 2 * n ** 3
    sweep = sum(6 * n * m * m + 9 * m ** 3 for m in (o, v))
    forces = 2 * n * n * o + n * o * o + 2 * n * o * o + 2 * n * n * o
    return start + common * it + cayley + second * np.maximum(it - 1, 0) + sweep + forces


def _cell_shapes(system):
    """Orbitals, occupied orbitals and atom pairs of every cell of a water or cluster system."""
    nat = np.diff(system.cell_offset)
    nw = nat // 3
    return 6 * nw, 4 * nw, nat * (nat - 1) // 2


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_matter(w):
    from oracle import cavity as OC
    from oracle import periodic as PR
    if w.get("lattice") is not None:
        return PR.PeriodicDFTBMatter(w["params"], w["system"], w["lattice"])
    return OC.DFTBMatter(w["params"], w["system"])


def cpu_baseline(workload, seconds=12.0, n_sample=None):
    """The oracle as it stands, on a bounded sample of the workload, on this host."""
    import cavmd_synth as cs
    from oracle import cavity as OC
    w = cs.make_workload(workload, n_cells=n_sample)
    sy, mo, pa = w["system"], w["modes"], w["params"]
    mat = _oracle_matter(w)
    md = OC.CavityMD(mat, sy.r, sy.p, mo.k, mo.omega, mo.lam, mo.phi, sy.R_ref, w["options"]["dt"])
    md.step()                                   # warm start of the charges
    t0 = time.perf_counter()
    n = 0
    while True:
        md.step()
        n += 1
        el = time.perf_counter() - t0
        if (el >= seconds and n >= 3) or n >= 1000:
            break
    return {"value": (sy.n_atoms // 3) * n / el, "unit": "molecule-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{sy.n_cells} cells x {mo.n_modes} modes of workload {workload}, {n} oracle time "
                      f"steps after one warm-up step ({el:.1f} s, NumPy, one thread)"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import cavmd_synth as cs
    from oracle import cavity as OC
    n_sample = 1 if args.workload == "p33" else 512
    w = cs.make_workload(args.workload)
    sub = cs.make_workload(args.workload, n_cells=n_sample)
    sy, mo, pa = sub["system"], w["modes"], sub["params"]
    mat = _oracle_matter(sub)
    md = OC.CavityMD(mat, sy.r, sy.p, mo.k, mo.omega, mo.lam, mo.phi, sy.R_ref, w["options"]["dt"])
    for _ in range(args.warmup):
        md.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        md.step()
    el = time.perf_counter() - t0
    value = (sy.n_atoms // 3) * args.steps / el
    line = {
        "impl": "reference", "metric": "molecule-steps/s", "value": value, "unit": "molecule-steps/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(args.workload, w),
        "cpu_baseline": {"value": value, "unit": "molecule-steps/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {n_sample} of {w['system'].n_cells} cells, all {mo.n_modes} modes, "
                                   f"one oracle time step per step (NumPy FP64, one thread)"},
        "e2e": {"value": value, "unit": "molecule-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _config(workload, w, charge_model="mulliken", precision="fp64", mode_positions="fixed"):
    sy, mo = w["system"], w["modes"]
    nw = sy.n_atoms // 3
    cells = (f"{nw} water" if nw == sy.n_cells else
             f"{sy.n_cells} clusters (H2O)_n, n = 1..8 ({nw} water molecules, up to 48 orbitals)")
    if w.get("lattice") is not None:
        cells = (f"{sy.n_cells} periodic cells of {nw // sy.n_cells} water (10 Angstrom cubes, Gamma point, "
                 f"{nw} water molecules, {2 * nw // sy.n_cells * 3} orbitals per cell)")
    cm = {"mulliken": "Mulliken", "born_fd": "forward-FD Born every 3 steps",
          "born_central": "central-FD Born every 3 steps", "born_mlp": "network Born charges"}[charge_model]
    cp = "FP64 coupling" if precision == "fp64" else "BF16x3 tensor-core coupling"
    mp = ", mode functions at the moving cell centres of mass" if mode_positions == "com" else ""
    return {"workload": f"{workload}: {cells} x {mo.n_modes} modes, FP64 SCC-DFTB, {cm}, {cp}{mp}, dt 0.5 fs",
            "n_cells": sy.n_cells, "n_molecules": nw, "n_atoms": sy.n_atoms, "n_modes": mo.n_modes, "precision": precision,
            "charge_model": charge_model, "l2": "256 MB buffer rewritten between timed steps (L2 flush)",
            "parallelism": "replicas"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mixing", type=float, default=None, help="charge mixing (default: the library's)")
    ap.add_argument("--charge-model", default="mulliken", choices=["mulliken", "born_fd", "born_central", "born_mlp"],
                    help="dipole derivative (default: Mulliken charges)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="coupling contraction: FP64, or BF16x3 on the tensor cores (grid modes)")
    ap.add_argument("--n-cells", type=int, default=None, help="trim the workload to this many cells")
    ap.add_argument("--phase-events", default="dftb", choices=["dftb", "all", "off"],
                    help="CUDA events inside the timed region: around the SCC-DFTB launches only (default; "
                         "the roofline's kernel time), around every launch, or none (kernel times from a "
                         "second pass); phase shares always come from a second pass with every launch timed")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes instead of timing candidates at init")
    ap.add_argument("--scc-history", type=int, default=None,
                    help="Anderson history of the cluster kernel (default: the library's)")
    ap.add_argument("--mode-positions", default="fixed", choices=["fixed", "com"],
                    help="mode functions at the reference cell positions, or at the moving cell centres of mass")
    ap.add_argument("--acf-lags", type=int, default=None,
                    help="on-device autocorrelation lags (default: 1024 for c5, whose configuration asks for "
                         "it, else off)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    import cavmd_synth as cs
    import paper_2512_03277_gb300 as P
    from paper_2512_03277_gb300 import build
    from paper_2512_03277_gb300 import cavmd as B

    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    build.build()
    w = cs.make_workload(args.workload, n_cells=args.n_cells)
    if rank > 0:   # independent replica: its own Maxwell-Boltzmann velocities
        w["system"].p = cs.mb_momenta(np.random.default_rng(1000 + rank), w["system"])
    opt = P.default_options()
    opt.device = local
    if args.mixing is not None:
        opt.mixing = args.mixing
    opt.charge_model = {"mulliken": 0, "born_fd": 1, "born_central": 2, "born_mlp": 3}[args.charge_model]
    opt.precision = {"fp64": 0, "mixed": 2}[args.precision]
    if args.scc_history is not None:
        opt.scc_history = args.scc_history
    opt.autotune = 0 if args.no_autotune else 1
    opt.mode_positions = 1 if args.mode_positions == "com" else 0
    if args.acf_lags is None:
        args.acf_lags = 1024 if args.workload == "c5" else 0
    opt.acf_lags = args.acf_lags
    ctx = P.Context(w["system"], w["params"], w["modes"], opt, lattice=w.get("lattice"))
    if args.charge_model == "born_mlp":
        # a seeded network: the cost of a time step does not depend on the weight values
        rng = np.random.default_rng(4)
        sizes = [(128, 32), (128,), (128, 128), (128,), (9, 128), (9,)]
        params = np.concatenate([rng.uniform(-1, 1, s_).ravel() / np.sqrt(s_[-1]) * (len(s_) == 2) for s_ in sizes])
        ctx.cavmd_load_born_mlp(params.astype(np.float32))
    stream = ctx.stream
    N = w["system"].n_cells
    n_mol = w["system"].n_atoms // 3          # water molecules (cells of the water workloads)
    for _ in range(args.warmup):
        ctx.cavmd_step(1)
    ctx.cavmd_observables(want_arrays=False)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{local}")
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    ctx.cavmd_phase_times({"dftb": 2, "all": 1, "off": 0}[args.phase_events], reset=True)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    t_wall = time.perf_counter()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            ctx.cavmd_step(1)
            ends[k].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    timed_ms, timed_cnt = ctx.cavmd_phase_times(0, reset=True)
    # phase shares and launch counts from a second pass of the same steps, every launch timed
    ctx.cavmd_phase_times(1, reset=True)
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()
            ctx.cavmd_step(1)
    torch.cuda.synchronize()
    phase_ms, phase_cnt = ctx.cavmd_phase_times(0, reset=True)
    obs = ctx.cavmd_observables(want_arrays=False)
    ev = ctx.cavmd_get_eval()
    step_ms = np.array([s.elapsed_time(e) for s, e in zip(starts, ends)])
    total_ms = float(step_ms.sum())
    total_ms = _reduce_max(total_ms, ws, f"cuda:{local}")
    value = _whole_job_value(n_mol, args.steps, ws, total_ms)

    # roofline of the dominant kernel (SCC-DFTB, FP64-ALU bound)
    if args.phase_events == "off":
        dftb_ms = phase_ms[0] / max(phase_cnt[0], 1)
    else:   # measured inside the timed region
        dftb_ms = timed_ms[0] / max(timed_cnt[0], 1)
    periodic = w.get("lattice") is not None
    if periodic:
        n_orb = 2 * np.diff(w["system"].cell_offset)          # 6 per water: 2 per atom
        flops = float(sum(_periodic_flops_per_cell(i, n, n * 2 // 3) for i, n in zip(ev["scc_iters"], n_orb)))
    else:
        flops = float(_dftb_flops_per_cell(ev["scc_iters"], *_cell_shapes(w["system"])).sum())
    generic = not np.all(np.diff(w["system"].cell_offset) == 3)
    achieved = flops / (dftb_ms * 1e-3) / 1e12
    peak = N_SM * FP64_FLOPS_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12
    shares = {name: float(phase_ms[i] / max(phase_ms.sum(), 1e-30))
              for i, name in enumerate(["dftb", "photon_forward", "field_kick_drift", "born_fd_rows"])}

    # end to end through the C ABI: step + observables into pinned host buffers, wall clock
    pin = {k: torch.empty(n, dtype=torch.float64, pin_memory=True)
           for k, n in (("M", N), ("q", ctx.n_modes), ("p", ctx.n_modes), ("D", ctx.n_modes))}
    o = B.cavmd_obs()
    import ctypes as C
    for k, t in pin.items():
        setattr(o, k, C.cast(t.data_ptr(), C.POINTER(C.c_double)))
    ctx.cavmd_step(1)
    ctx.cavmd_observables_into(o)
    # double-buffered read-out: step s's observables are queued into slot s % 2 behind the step and
    # collected after step s + 1 has been queued, so the host reads step s while the GPU runs s + 1
    t0 = time.perf_counter()
    for s in range(args.e2e_steps):
        ctx.cavmd_step(1)
        ctx.cavmd_observables_async(s % 2)
        if s > 0:
            ctx.cavmd_observables_wait_into((s - 1) % 2, o)
    ctx.cavmd_observables_wait_into((args.e2e_steps - 1) % 2, o)
    e2e_s = time.perf_counter() - t0
    d2h = 8 * (16 + N + 3 * ctx.n_modes)   # one packed copy: energies, max SCC iterations, status, M, q, p, D
    e2e = {"value": n_mol * args.e2e_steps * ws / e2e_s, "unit": "molecule-steps/s", "h2d_bytes_per_step": 0,
           "d2h_bytes_per_step": d2h,
           "note": "cavmd_step(1) + cavmd_observables_async / _wait (energies, per-cell dipoles, photon q/p/D) "
                   "every step, double-buffered so the host reads step s while step s + 1 runs; the MD state "
                   "stays on the device between steps, so no host input is copied per step"}

    line = {
        "metric": "molecule-steps/s", "value": value, "unit": "molecule-steps/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(args.workload, w, args.charge_model, args.precision, args.mode_positions),
        "roofline": {"bound": "alu",
                     "kernel": "k_dftb_periodic" if periodic else ("k_dftb_generic" if generic else "dftb_kernel<3,6>"),
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": DFTB_DRAM_BYTES_PER_LAUNCH if (args.workload == "c2" and args.n_cells is None) else None,
                     "flops_per_launch": flops, "avg_launch_ms": dftb_ms,
                     "mean_scc_iters": float(np.mean(ev["scc_iters"])),
                     "peak_note": "FP64 ALU: 152 SMs x 4 FP64 flop/clk x 2070 MHz (derived, 1.26 TFLOP/s)",
                     "launch_time_source": "CUDA events in a second pass of the same steps"
                     if args.phase_events == "off" else "CUDA events around each SCC-DFTB launch in the timed region"},
        "phase_share": shares,
        "e2e": e2e,
        "gpu_launches": int(phase_cnt.sum()) + (int(phase_cnt[3]) if args.charge_model in ("born_fd", "born_central") else 0)
                        + 2 * (int(phase_cnt[3]) if args.charge_model == "born_mlp" else 0)
                        + (int(phase_cnt[0]) if args.precision == "mixed" else 0),
        "acf_lags": args.acf_lags,
        "mode_positions": args.mode_positions,
        "clocks": clk,
        "tuning": ctx.cavmd_tuning(),
        "wall_s_timed_region": t_wall,
        "energy_total": obs["e_total"], "temperature_K": obs["temperature"],
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        n_sample = None if w["system"].n_cells <= 4096 else (1024 if generic else 4096)
        if periodic:
            n_sample = 1
        line["cpu_baseline"] = cpu_baseline(args.workload, n_sample=n_sample)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.cavmd_destroy()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
