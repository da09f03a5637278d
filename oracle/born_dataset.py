"""Training data of the Born-charge network: water geometries from 300 K trajectories, labelled with
the oracle's finite-difference Born tensors.

TEST INFRASTRUCTURE (a committed generator of stored values): it calls only the oracle and the
shared input generators, and writes an .npz file; nothing on the GPU path runs here.

Recipe (the configuration of the learned Born charges: geometries sampled from config-1-style
300 K trajectories, labelled with oracle finite-difference Born charges):
  * every worker runs one oracle trajectory of `cells` waters in the config-1 cavity (waters
    centred uniformly on a 2000 bohr line, 16 standing modes, g = 0.002 a.u., Mulliken charges,
    dt = 0.5 fs, the oracle's default exact-photon splitting), started from the textbook geometry
    with 0.02 bohr noise, a random rotation and 300 K Maxwell-Boltzmann momenta (seed 10 + worker);
  * equilibration: the waters start near their minimum, so equipartition would settle them near
    150 K; the momenta of all cells are rescaled by one common factor to a kinetic temperature of
    300 K over the six internal degrees of freedom of each water (the centre-of-mass motion is
    removed), every 25 steps for the first `equil` steps;
  * sampling: every `stride` steps for `samples` samples of every cell (no rescaling);
  * labels: full central-difference Born tensors Z_j[alpha][beta] = d mu_alpha / d r_j,beta with
    h = 1e-3 bohr (oracle.mlp.born_fd_tensors), and the Mulliken net charges Q_j.
Cells of trajectory workers >= n_workers - n_test_workers are the held-out set (disjoint
trajectories).

Usage: python -m oracle.born_dataset OUT.npz [--workers 16] [--cells 125] [--samples 100]
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

KB = 3.166811563e-6
WATER = [0, 1, 1]


def _internal_temperature(p, mass, n_cells):
    """Kinetic temperature over the 6 internal degrees of freedom of each 3-atom cell."""
    ek = 0.5 * np.sum(p * p / mass[:, None])
    return 2.0 * ek / (6.0 * n_cells * KB)


def trajectory_samples(worker: int, cells: int, equil: int, stride: int, samples: int):
    """Geometries (samples * cells, 3, 3) of one oracle trajectory, in sampling order."""
    import cavmd_synth as cs
    from oracle import cavity as OC
    w = cs.make_workload("c1", n_cells=cells)
    sy, mo, pa = w["system"], w["modes"], w["params"]
    rng = np.random.default_rng(10 + worker)
    centres = np.zeros((cells, 3))
    centres[:, 0] = rng.uniform(0.0, 2000.0, cells)
    pos = cs.water_batch(rng, centres)
    sy = cs.systems._water_system(pos, centres)
    sy.p = cs.mb_momenta(rng, sy, 300.0)
    mat = OC.DFTBMatter(pa, sy)
    md = OC.CavityMD(mat, sy.r, sy.p, mo.k, mo.omega, mo.lam, mo.phi, sy.R_ref, w["options"]["dt"])
    mass = mat.mass
    for s in range(equil):
        md.step()
        if (s + 1) % 25 == 0:
            md.p *= np.sqrt(300.0 / _internal_temperature(md.p, mass, cells))
    out = np.empty((samples, cells, 3, 3))
    for k in range(samples):
        for _ in range(stride):
            md.step()
        out[k] = md.r.reshape(cells, 3, 3)
    return out.reshape(-1, 3, 3)


def _worker(args):
    worker, cells, equil, stride, samples = args
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    import cavmd_synth as cs
    from oracle import mlp as NN
    t0 = time.time()
    pos = trajectory_samples(worker, cells, equil, stride, samples)
    params = cs.load_water_params()
    Z = np.empty((len(pos), 3, 3, 3))
    Q = np.empty((len(pos), 3))
    for a in range(0, len(pos), 2000):
        Z[a:a + 2000], Q[a:a + 2000] = NN.born_fd_tensors(params, WATER, pos[a:a + 2000], h=1e-3)
    return worker, pos, Z, Q, time.time() - t0


def generate(out_path: str, workers: int = 16, cells: int = 125, samples: int = 100, equil: int = 400,
             stride: int = 10, test_workers: int = 2, processes: int | None = None):
    import multiprocessing as mp
    processes = processes or min(workers, os.cpu_count() or 1)
    jobs = [(i, cells, equil, stride, samples) for i in range(workers)]
    with mp.get_context("spawn").Pool(processes) as pool:
        res = sorted(pool.map(_worker, jobs), key=lambda t: t[0])
    pos = np.concatenate([r[1] for r in res])
    Z = np.concatenate([r[2] for r in res])
    Q = np.concatenate([r[3] for r in res])
    traj = np.concatenate([np.full(len(r[1]), r[0], np.int32) for r in res])
    test = traj >= workers - test_workers
    np.savez_compressed(out_path, pos=pos, Z=Z, Q=Q, trajectory=traj, test=test,
                        recipe=np.array(f"{workers} trajectories x {cells} waters, {equil} equilibration steps "
                                        f"(rescaled to 300 K), {samples} samples every {stride} steps; central-FD "
                                        f"Born tensors h = 1e-3 bohr; trajectories >= {workers - test_workers} "
                                        f"held out"))
    return len(pos), int(test.sum()), max(r[4] for r in res)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("out")
    ap.add_argument("--workers", type=int, default=16)
    ap.add_argument("--cells", type=int, default=125)
    ap.add_argument("--samples", type=int, default=100)
    ap.add_argument("--equil", type=int, default=400)
    ap.add_argument("--stride", type=int, default=10)
    ap.add_argument("--test-workers", type=int, default=2)
    ap.add_argument("--processes", type=int, default=None)
    a = ap.parse_args()
    n, nt, tmax = generate(a.out, a.workers, a.cells, a.samples, a.equil, a.stride, a.test_workers, a.processes)
    print(f"{a.out}: {n} geometries ({nt} held out), slowest worker {tmax:.0f} s", file=sys.stderr)


if __name__ == "__main__":
    main()
