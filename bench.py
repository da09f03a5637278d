"""Benchmark: molecule-steps/s of the cavity-MD hot path on one GB300 (or N replicas), the
surrogate/mixed form against the plain FP64 form on the same workload.

Workload (default "c5"): 262,144 synthetic waters (786,432 atoms) in a 30 bohr slab at liquid
density, 8192 real cavity modes on a 64 x 128 in-plane wave-vector grid, g = 0.001 a.u.,
dt = 0.5 fs, FP64 SCC-DFTB, photons initially at rest, on-device autocorrelation of the photon
coordinates and the total dipole (1024 lags). Two arms run on it, one after the other:
  surrogate/mixed (the headline): network Born charges, BF16x3 coupling on the tensor cores;
  plain FP64: forward finite-difference Born charges refreshed every 3 steps (the paper's scheme),
              FP64 coupling.
Both keep the SCC, the charge mixing and the Verlet update in FP64.

One timed step = one cavmd_step(ctx, 1) call: the whole hot path (SCC-DFTB of every cell, the
dipole derivatives, forward contraction, photon half-flows, field on every cell, kicks and drift,
energies, the autocorrelation sample). Each step is bracketed by CUDA events on the library's
stream; a 256 MB buffer (larger than the 129 MB L2) is rewritten between steps, outside the events.
The headline arm is also timed as CUDA-graph replay (cavmd_step(chunk), one event pair per chunk,
no flush: the state a step reads is larger than L2) and end to end through the C ABI.

The judge (drift, heating and band error of each arm's dipole derivative and coupling against
explicit central-difference Born charges) runs on a resonant single-box cavity of 33 waters for
10^4 steps, four replicas (paper_2512_03277_gb300/judge.py).

Multi-GPU (torchrun): every rank propagates its own independent replica (its own velocities),
no data-path collective; value = all ranks' molecule-steps / max-over-ranks time (weak scaling).

cpu_baseline: the FP64 oracle (oracle/) as it stands, on a bounded sample of the headline arm's
workload, on one core and on every core of the host (one process per core, cells split between
them); its network charge model runs a seeded network (the cost does not depend on the weights).
--impl reference times the same oracle the same way, one oracle time step per step.
"""
import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

FP64_FLOPS_PER_CLK_SM = 4.0      # 2 FP64 FMA per clock per SM (1.25 TFLOP/s nominal at 2.07 GHz)
SM_MAX_MHZ_NOMINAL = 2070.0
FLUSH_BYTES = 256 << 20
CHARGE = {"mulliken": 0, "born_fd": 1, "born_central": 2, "born_mlp": 3}
PREC = {"fp64": 0, "mixed": 2}
ORACLE_CHARGE = {"mulliken": "mulliken", "born_fd": "born_fd", "born_central": "born_central",
                 "born_mlp": "network"}


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


def _kgrid_points(k):
    """Irreducible points of a Gamma-centred k x k x k grid (k and -k once): each solved as the real
    form of its complex problem, twice the orbitals."""
    pts = [(i, j, l) for i in range(k) for j in range(k) for l in range(k)]
    return sum(1 for (i, j, l) in pts if ((-i) % k, (-j) % k, (-l) % k) >= (i, j, l))


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


# ------------------------------------------------------------------------------ the host oracle

def _cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_shard(workload, lo, hi, charge_model, mlp, warmup, steps, seconds, barrier, out):
    """One process: the oracle's time step on cells lo..hi-1 of the workload (all its modes);
    `warmup` untimed steps, the barrier, then `steps` timed steps (or as many as `seconds` allow
    when steps is None). Puts (molecules, steps, t0, t1) on `out` (system-wide monotonic clock)."""
    import cavmd_synth as cs
    from oracle import cavity as OC
    from oracle import periodic as PR
    w = cs.make_workload(workload)
    sy = w["system"]
    off = sy.cell_offset
    a0, a1 = off[lo], off[hi]
    sub = cs.System(species=sy.species[a0:a1], cell_offset=(off[lo:hi + 1] - a0).astype(np.int32),
                    r=sy.r[a0:a1], p=sy.p[a0:a1], R_ref=sy.R_ref[lo:hi])
    mo = w["modes"]
    if w.get("lattice") is not None:
        mat = PR.PeriodicDFTBMatter(w["params"], sub, w["lattice"])
    else:
        kw = {"mlp_params": mlp} if charge_model == "network" else {}
        mat = OC.DFTBMatter(w["params"], sub, charge_model=charge_model,
                            born_interval=3 if charge_model == "born_fd" else 1, **kw)
    md = OC.CavityMD(mat, sub.r, sub.p, mo.k, mo.omega, mo.lam, mo.phi, sub.R_ref, w["options"]["dt"])
    for _ in range(warmup):
        md.step()
    if barrier is not None:
        barrier.wait()
    t0 = time.monotonic()
    n = 0
    while True:
        md.step()
        n += 1
        if steps is not None and n >= steps:
            break
        if steps is None and time.monotonic() - t0 >= seconds:
            break
    t1 = time.monotonic()
    out.put(((a1 - a0) // 3, n, t0, t1))


def oracle_throughput(workload, charge_model, mlp, workers, cells_per_worker, warmup, steps=None, seconds=10.0):
    """molecule-steps/s of the oracle on `workers` processes (one thread each, started with spawn),
    each stepping its own `cells_per_worker` cells; the time is that of the whole group (first
    start to last finish). Returns (value, total molecule-steps, seconds, steps per worker)."""
    import multiprocessing as mp
    import cavmd_synth as cs
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        n_cells = cs.make_workload(workload)["system"].n_cells
        workers = max(1, min(workers, n_cells // max(1, cells_per_worker)))
        q = ctx.Queue()
        bar = ctx.Barrier(workers)
        procs = [ctx.Process(target=_oracle_shard,
                             args=(workload, i * cells_per_worker, (i + 1) * cells_per_worker, charge_model, mlp,
                                   warmup, steps, seconds, bar, q)) for i in range(workers)]
        for p in procs:
            p.start()
        res = []
        while len(res) < len(procs):   # collect, and fail loudly if a worker died
            try:
                res.append(q.get(timeout=5))
            except Exception:
                dead = [p.exitcode for p in procs if p.exitcode not in (None, 0)]
                if dead:
                    for p in procs:
                        if p.is_alive():
                            p.terminate()
                    raise RuntimeError(f"an oracle worker failed (exit codes {dead})")
        for p in procs:
            p.join(timeout=60)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    total = sum(m * n for m, n, _, _ in res)
    el = max(t1 for *_, t1 in res) - min(t0 for _, _, t0, _ in res)
    return total / el, total, el, min(n for _, n, _, _ in res), workers


def _sample_cells(workload, n_total):
    """Cells per oracle process: a bounded sample of the workload (about 10-20 s of oracle work)."""
    if workload == "p33":
        return 1
    return max(1, min(n_total, 256 if workload in ("c3", "c4", "c5") else 512))


def cpu_baseline(workload, charge_model, mlp, n_total):
    """The oracle as it stands on one core and on every core of the host."""
    cores = _host_cores()
    n = _sample_cells(workload, n_total)
    v1, tot1, el1, k1, _ = oracle_throughput(workload, ORACLE_CHARGE[charge_model], mlp, 1, n, warmup=1, seconds=8.0)
    vall, tot, el, k, used = oracle_throughput(workload, ORACLE_CHARGE[charge_model], mlp, cores, n, warmup=1,
                                               steps=max(2, k1))
    return {"value": vall, "unit": "molecule-steps/s", "cores": used, "kind": "oracle",
            "value_one_core": v1, "nproc": cores, "cpu_model": _cpu_model(),
            "sample": f"{used} processes (one per core, one thread each), each the oracle's full time step "
                      f"({ORACLE_CHARGE[charge_model]} dipole derivatives, FP64 coupling to all modes) on its own "
                      f"{n} cells of workload {workload}, {k} steps after one warm-up step, {el:.1f} s; one core: "
                      f"{n} cells, {k1} steps, {el1:.1f} s. Each process's coupling sum covers its own cells only "
                      f"(the same work per cell as the full sum)"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import cavmd_synth as cs
    from paper_2512_03277_gb300 import cavmd as B
    w = cs.make_workload(args.workload)
    charge_model = _arm_defaults(args)[0][1]
    mlp = _network(B, charge_model, seeded=True)
    cores = _host_cores()
    n = _sample_cells(args.workload, w["system"].n_cells)
    value, tot, el, k, used = oracle_throughput(args.workload, ORACLE_CHARGE[charge_model], mlp, cores, n,
                                                warmup=args.warmup, steps=args.steps)
    sample = (f"{used} processes (one per core, one thread each), each the oracle's full time step "
              f"({ORACLE_CHARGE[charge_model]} dipole derivatives, FP64 coupling to all {w['modes'].n_modes} modes) "
              f"on its own {n} of the {w['system'].n_cells} cells, {args.warmup} warm-up and {args.steps} timed steps")
    line = {
        "impl": "reference", "metric": "molecule-steps/s", "value": value, "unit": "molecule-steps/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(args.workload, w, charge_model, "fp64"),
        "cpu_baseline": {"value": value, "unit": "molecule-steps/s", "cores": used, "kind": "oracle",
                         "nproc": cores, "cpu_model": _cpu_model(), "sample": sample},
        "e2e": {"value": value, "unit": "molecule-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ the GPU arms

def _arm_defaults(args):
    """[(precision, charge_model)] of the arms: the headline first."""
    grid = args.workload in ("c3", "c4", "c5")
    prec = args.precision or ("mixed" if grid else "fp64")
    charge = args.charge_model or ("born_mlp" if args.workload in ("c4", "c5") else "mulliken")
    arms = [(prec, charge)]
    compare = args.compare if args.compare is not None else args.workload in ("c4", "c5")
    if compare and (prec, charge) != ("fp64", "born_fd"):
        arms.append(("fp64", "born_fd"))
    return arms


def _network(B, charge_model, seeded=False):
    """The shipped trained network, else (and always with `seeded`, for the oracle's timing runs,
    whose inputs never come from the GPU) a seeded one; None for other models."""
    if charge_model != "born_mlp":
        return None
    p = None if seeded else B.trained_born_mlp()
    if p is not None:
        return p
    rng = np.random.default_rng(4)
    sizes = [(128, 32), (128,), (128, 128), (128,), (9, 128), (9,)]
    return np.concatenate([rng.uniform(-1, 1, s_).ravel() / np.sqrt(s_[-1]) * (len(s_) == 2)
                           for s_ in sizes]).astype(np.float32)


def _config(workload, w, charge_model="mulliken", precision="fp64", mode_positions="fixed", kgrid=1):
    sy, mo = w["system"], w["modes"]
    nw = sy.n_atoms // 3
    cells = (f"{nw} water" if nw == sy.n_cells else
             f"{sy.n_cells} clusters (H2O)_n, n = 1..8 ({nw} water molecules, up to 48 orbitals)")
    if w.get("lattice") is not None:
        bz = "Gamma point" if kgrid <= 1 else f"{kgrid} x {kgrid} x {kgrid} k-grid"
        cells = (f"{sy.n_cells} periodic cells of {nw // sy.n_cells} water (10 Angstrom cubes, {bz}, "
                 f"{nw} water molecules, {2 * nw // sy.n_cells * 3} orbitals per cell)")
    cm = {"mulliken": "Mulliken", "born_fd": "forward-FD Born every 3 steps",
          "born_central": "central-FD Born every 3 steps", "born_mlp": "network Born charges"}[charge_model]
    cp = "FP64 coupling" if precision == "fp64" else "BF16x3 tensor-core coupling"
    mp = ", mode functions at the moving cell centres of mass" if mode_positions == "com" else ""
    return {"workload": f"{workload}: {cells} x {mo.n_modes} modes, FP64 SCC-DFTB, {cm}, {cp}{mp}, dt 0.5 fs",
            "n_cells": sy.n_cells, "n_molecules": nw, "n_atoms": sy.n_atoms, "n_modes": mo.n_modes, "precision": precision,
            "charge_model": charge_model, "l2": "256 MB buffer rewritten between timed steps (L2 flush)",
            "parallelism": "replicas"}


def _make_ctx(P, w, args, local, precision, charge_model, mlp, graph_chunk):
    opt = P.default_options()
    opt.device = local
    if args.mixing is not None:
        opt.mixing = args.mixing
    opt.charge_model = CHARGE[charge_model]
    opt.precision = PREC[precision]
    if args.scc_history is not None:
        opt.scc_history = args.scc_history
    opt.autotune = 0 if args.no_autotune else 1
    opt.mode_positions = 1 if args.mode_positions == "com" else 0
    opt.acf_lags = args.acf_lags
    if args.kgrid > 1:
        opt.kgrid[:] = (args.kgrid,) * 3
    opt.graph_chunk = graph_chunk
    ctx = P.Context(w["system"], w["params"], w["modes"], opt, lattice=w.get("lattice"))
    if mlp is not None:
        ctx.cavmd_load_born_mlp(mlp)
    return ctx


def _time_steps(torch, ctx, args, ws, local, flush):
    """K per-step timed cavmd_step(1) calls (events on the library stream, L2 flush between
    steps), bracketed by barrier + synchronize; returns (total ms, max over ranks, wall s, clocks)."""
    import torch.distributed as dist
    stream = ctx.stream
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
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
    total_ms = float(sum(s.elapsed_time(e) for s, e in zip(starts, ends)))
    return total_ms, _reduce_max(total_ms, ws, f"cuda:{local}"), t_wall, clk


def _measure_arm(torch, P, w, args, ws, local, precision, charge_model, mlp, flush, headline):
    """Everything one arm reports. The headline arm adds the CUDA-graph and end-to-end figures."""
    import ctypes as C
    from paper_2512_03277_gb300 import cavmd as B
    sy = w["system"]
    N = sy.n_cells
    n_mol = sy.n_atoms // 3
    graph_chunk = max(1, min(50, args.steps))
    ctx = _make_ctx(P, w, args, local, precision, charge_model, mlp, graph_chunk)
    for _ in range(args.warmup):
        ctx.cavmd_step(1)
    ctx.cavmd_observables(want_arrays=False)
    ctx.cavmd_phase_times({"dftb": 2, "all": 1, "off": 0}[args.phase_events], reset=True)
    total_ms, max_ms, t_wall, clk = _time_steps(torch, ctx, args, ws, local, flush)
    timed_ms, timed_cnt = ctx.cavmd_phase_times(0, reset=True)
    # phase shares and launch counts from a second pass of the same steps, every launch timed
    ctx.cavmd_phase_times(1, reset=True)
    with torch.cuda.stream(ctx.stream):
        for _ in range(args.steps):
            flush.zero_()
            ctx.cavmd_step(1)
    torch.cuda.synchronize()
    phase_ms, phase_cnt = ctx.cavmd_phase_times(0, reset=True)
    value = _whole_job_value(n_mol, args.steps, ws, max_ms)
    ev = ctx.cavmd_get_eval()
    # roofline of the dominant kernel: the SCC-DFTB evaluation (FP64-ALU bound)
    dftb_ms = (phase_ms[0] / max(phase_cnt[0], 1)) if args.phase_events == "off" else \
        timed_ms[0] / max(timed_cnt[0], 1)
    periodic = w.get("lattice") is not None
    if periodic:
        n_orb = 2 * np.diff(sy.cell_offset)          # 6 per water: 2 per atom
        if args.kgrid > 1:   # the same count for each k-point's real form (2n orbitals, 2 n_occ occupied)
            nk = _kgrid_points(args.kgrid)
            flops = float(sum(nk * _periodic_flops_per_cell(i, 2 * n, 2 * (n * 2 // 3))
                              for i, n in zip(ev["scc_iters"], n_orb)))
        else:
            flops = float(sum(_periodic_flops_per_cell(i, n, n * 2 // 3) for i, n in zip(ev["scc_iters"], n_orb)))
    else:
        flops = float(_dftb_flops_per_cell(ev["scc_iters"], *_cell_shapes(sy)).sum())
    generic = not np.all(np.diff(sy.cell_offset) == 3)
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    peak = n_sm * FP64_FLOPS_PER_CLK_SM * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    achieved = flops / (dftb_ms * 1e-3) / 1e12
    names = ["dftb", "photon_forward", "field_kick_drift", "dipole_derivative"]
    shares = {nm: float(phase_ms[i] / max(phase_ms.sum(), 1e-30)) for i, nm in enumerate(names)}
    mixed = precision == "mixed"
    fd = charge_model in ("born_fd", "born_central")
    # phase scopes count calls; some calls launch more than one kernel: the forward product and its
    # reduction, the moving-position back product (one launch per half-flow), the network's three
    # kernels, the finite-difference copies after the Born refresh
    launches = int(phase_cnt.sum()) + (int(phase_cnt[3]) if fd else 0) + \
        2 * (int(phase_cnt[3]) if charge_model == "born_mlp" else 0) + (int(phase_cnt[0]) if mixed else 0) + \
        (int(phase_cnt[0]) if mixed and args.mode_positions == "com" else 0)
    arm = {
        "value": value, "unit": "molecule-steps/s", "ms_per_step": max_ms / args.steps,
        "precision": precision, "charge_model": charge_model,
        "config": _config(args.workload, w, charge_model, precision, args.mode_positions, args.kgrid),
        "roofline": {"bound": "alu",
                     "kernel": "k_dftb_periodic" if periodic else ("k_dftb_generic" if generic else "dftb_kernel<3,6>"),
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None, "flops_per_launch": flops, "avg_launch_ms": dftb_ms,
                     "mean_scc_iters": float(np.mean(ev["scc_iters"])),
                     "peak_note": f"FP64 ALU: {n_sm} SMs x 4 FP64 flop/clk x {SM_MAX_MHZ_NOMINAL:.0f} MHz (derived; "
                                  f"no FP64 figure in the measured peaks)",
                     "launch_time_source": "CUDA events in a second pass of the same steps"
                     if args.phase_events == "off" else "CUDA events around each SCC-DFTB launch in the timed region"},
        "phase_share": shares, "gpu_launches": launches, "clocks": clk, "tuning": ctx.cavmd_tuning(),
        "wall_s_timed_region": t_wall,
    }
    if fd:
        arm["born_interval"] = 3
    if headline:
        # CUDA-graph replay: cavmd_step(chunk) replays one captured graph of `chunk` steps; one
        # event pair per chunk, no flush inside a chunk (the state each step reads exceeds L2)
        chunks = max(1, args.steps // graph_chunk)
        ctx.cavmd_step(graph_chunk)           # capture (untimed)
        torch.cuda.synchronize()
        gs = [torch.cuda.Event(enable_timing=True) for _ in range(chunks)]
        ge = [torch.cuda.Event(enable_timing=True) for _ in range(chunks)]
        with torch.cuda.stream(ctx.stream):
            for i in range(chunks):
                flush.zero_()
                gs[i].record(ctx.stream)
                ctx.cavmd_step(graph_chunk)
                ge[i].record(ctx.stream)
        torch.cuda.synchronize()
        g_ms = float(sum(a.elapsed_time(b) for a, b in zip(gs, ge)))
        g_ms = _reduce_max(g_ms, ws, f"cuda:{local}")
        arm["graph"] = {"value": _whole_job_value(n_mol, chunks * graph_chunk, ws, g_ms), "unit": "molecule-steps/s",
                        "steps": chunks * graph_chunk, "chunk": graph_chunk,
                        "ms_per_step": g_ms / (chunks * graph_chunk),
                        "note": "cavmd_step(chunk) replaying one captured CUDA graph per chunk; events per chunk; "
                                "L2 flushed between chunks only"}
        # end to end through the C ABI: step + observables into pinned host buffers, wall clock
        pin = {k: torch.empty(n, dtype=torch.float64, pin_memory=True)
               for k, n in (("M", N), ("q", ctx.n_modes), ("p", ctx.n_modes), ("D", ctx.n_modes))}
        o = B.cavmd_obs()
        for k, t in pin.items():
            setattr(o, k, C.cast(t.data_ptr(), C.POINTER(C.c_double)))
        ctx.cavmd_step(1)
        ctx.cavmd_observables_into(o)
        # double-buffered read-out: step s's observables are queued into slot s % 2 behind the step
        # and collected after step s + 1 has been queued, so the host reads step s while s + 1 runs
        ne = args.e2e_steps
        t0 = time.perf_counter()
        for s in range(ne):
            ctx.cavmd_step(1)
            ctx.cavmd_observables_async(s % 2)
            if s > 0:
                ctx.cavmd_observables_wait_into((s - 1) % 2, o)
        ctx.cavmd_observables_wait_into((ne - 1) % 2, o)
        e2e_s = time.perf_counter() - t0
        e2e_s = _reduce_max(e2e_s * 1e3, ws, f"cuda:{local}") * 1e-3
        d2h = 8 * (16 + N + 3 * ctx.n_modes)   # one packed copy: energies, SCC iterations, status, M, q, p, D
        arm["e2e"] = {"value": n_mol * ne * ws / e2e_s, "unit": "molecule-steps/s", "h2d_bytes_per_step": 0,
                      "d2h_bytes_per_step": d2h, "steps": ne,
                      "note": "cavmd_step(1) + cavmd_observables_async / _wait (energies, per-cell dipoles, photon "
                              "q/p/D) every step, double-buffered so the host reads step s while step s + 1 runs; "
                              "the MD state stays on the device between steps, so no host input is copied per step"}
    obs = ctx.cavmd_observables(want_arrays=False)
    arm["energy_total"] = obs["e_total"]
    arm["temperature_K"] = obs["temperature"]
    ctx.cavmd_destroy()
    return arm


def _judge(P, params, arms, mlp, steps, replicas):
    """Drift, heating and band error of every arm's (dipole derivative, coupling) on the resonant
    box, against explicit central-difference Born charges with the FP64 coupling."""
    from paper_2512_03277_gb300 import judge as J
    cases = [("born_central", 0)] + [(cm, PREC[pr]) for pr, cm in arms]
    if ("mulliken", 0) not in cases:
        cases.append(("mulliken", 0))
    t0 = time.perf_counter()
    res = J.compare(P, params, cases, mlp=mlp, steps=steps, replicas=replicas)
    out = {}
    for (cm, pr), v in res.items():
        key = f"{cm}/{'fp64' if pr == 0 else 'mixed'}"
        out[key] = {"drift_ha_per_atom": v["drift"], "heating_K": v["heating"], "bend_ev": v["bend"],
                    "stretch_ev": v["stretch"], "band_error_mev": v["band_error_mev"]}
    out["setup"] = (f"33 waters (one per cell), resonant 2 x 2 mode grid (k = 0 at the bend, lambda 0.1), "
                    f"{steps} steps of 0.5 fs, {replicas} velocity seeds; reference: central-FD Born every step, "
                    f"FP64 coupling; drift = largest |slope x run| per atom over the seeds; heating = mean T "
                    f"over the last tenth minus the second tenth; {time.perf_counter() - t0:.0f} s")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c5")
    ap.add_argument("--e2e-steps", type=int, default=None, help="end-to-end steps (default: --steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mixing", type=float, default=None, help="charge mixing (default: the library's)")
    ap.add_argument("--charge-model", default=None, choices=list(CHARGE),
                    help="the headline arm's dipole derivative (default: network Born charges on c4/c5, else "
                         "Mulliken)")
    ap.add_argument("--precision", default=None, choices=list(PREC),
                    help="the headline arm's coupling: FP64, or BF16x3 on the tensor cores (grid modes; default on "
                         "c3-c5)")
    ap.add_argument("--compare", dest="compare", action="store_true", default=None,
                    help="also time the plain FP64 arm (forward-FD Born every 3 steps, FP64 coupling); default on "
                         "c4 and c5")
    ap.add_argument("--no-compare", dest="compare", action="store_false")
    ap.add_argument("--judge-steps", type=int, default=10000)
    ap.add_argument("--judge-replicas", type=int, default=4)
    ap.add_argument("--no-judge", action="store_true")
    ap.add_argument("--n-cells", type=int, default=None, help="trim the workload to this many cells")
    ap.add_argument("--phase-events", default="dftb", choices=["dftb", "all", "off"],
                    help="CUDA events inside the timed region: around the SCC-DFTB launches only (default; "
                         "the roofline's kernel time), around every launch, or none (kernel times from a "
                         "second pass); phase shares always come from a second pass with every launch timed")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes instead of timing candidates at init")
    ap.add_argument("--scc-history", type=int, default=None,
                    help="Anderson history of the cluster kernel (default: the library's)")
    ap.add_argument("--kgrid", type=int, default=1,
                    help="periodic workloads: sample the Brillouin zone on a Gamma-centred k x k x k grid "
                         "(the paper's cells: 3)")
    ap.add_argument("--mode-positions", default="fixed", choices=["fixed", "com"],
                    help="mode functions at the reference cell positions, or at the moving cell centres of mass")
    ap.add_argument("--acf-lags", type=int, default=None,
                    help="on-device autocorrelation lags (default: 1024 for c5, whose configuration asks for "
                         "it, else off)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.e2e_steps is None:
        args.e2e_steps = max(args.steps, 20)
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
    if args.acf_lags is None:
        args.acf_lags = 1024 if args.workload == "c5" else 0
    arms = _arm_defaults(args)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{local}")
    results = []
    for i, (prec, cm) in enumerate(arms):
        mlp = _network(B, cm)
        results.append(_measure_arm(torch, P, w, args, ws, local, prec, cm, mlp, flush, headline=(i == 0)))
        torch.cuda.empty_cache()
    head = results[0]
    trained = B.trained_born_mlp() is not None
    line = {
        "metric": "molecule-steps/s", "value": head["value"], "unit": "molecule-steps/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": head["config"], "roofline": head["roofline"],
        "phase_share": head["phase_share"], "e2e": head["e2e"], "graph": head["graph"],
        "gpu_launches": head["gpu_launches"], "acf_lags": args.acf_lags, "mode_positions": args.mode_positions,
        "clocks": head["clocks"], "tuning": head["tuning"], "wall_s_timed_region": head["wall_s_timed_region"],
        "energy_total": head["energy_total"], "temperature_K": head["temperature_K"],
        "network": ("trained (paper_2512_03277_gb300/data/born_mlp_water.f32)" if trained else
                    "seeded untrained weights (timing only)") if head["charge_model"] == "born_mlp" else None,
    }
    if len(results) > 1:
        plain = results[1]
        line["arms"] = {"surrogate_mixed": {k: v for k, v in head.items() if k not in ("e2e", "graph")},
                        "plain_fp64": plain}
        line["surrogate_over_plain"] = head["value"] / plain["value"]
    if rank == 0 and not args.no_judge and args.workload != "p33":
        mlp = _network(B, "born_mlp") if trained else None
        jarms = [(p, c) for p, c in arms if c != "born_mlp" or trained]
        line["judge"] = _judge(P, w["params"], jarms, mlp, args.judge_steps, args.judge_replicas)
        if not trained and any(c == "born_mlp" for _, c in arms):
            line["judge"]["note"] = "network arm not judged: no trained weights shipped"
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, head["charge_model"],
                                            _network(B, head["charge_model"], seeded=True), w["system"].n_cells)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
