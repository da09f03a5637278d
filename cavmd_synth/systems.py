"""Seeded molecules, clusters, velocities and cavity-mode lists.

Recipes (all lengths in bohr, seeds: geometry 1, velocities 2, clusters 3):

* water: the textbook water geometry (r_OH = 1.809 bohr, 104.52 deg),
  centre of mass at the cell centre, a uniform random rotation, then
  N(0, 0.02 bohr) noise on every coordinate;
* clusters (H2O)_n: n waters placed one by one, each a rotated, noisy water
  as above whose centre of mass is uniform in a sphere of radius
  (3n / (4 pi rho))^(1/3) at liquid density rho, kept only when its centre is
  at least 4.8 bohr from every placed centre and each of its atoms at least
  3.0 bohr from every atom of the other waters (liquid water's closest
  intermolecular contact, the O...H hydrogen bond, is about 3.4 bohr); after
  200 rejected candidates for one water the cluster restarts in a sphere 5%
  larger (candidates are drawn 16 at a time). The synthetic overlap integrals are not a Gram matrix at any
  distance: closer contacts (about 1.4 bohr H...H) make S indefinite;
* momenta: Maxwell-Boltzmann at 300 K, centre-of-mass velocity removed per
  cell;
* modes: real cavity modes u_a(R) = cos(k_a . R + phi_a) with frequency
  omega_a from the dispersion omega(k) = c sqrt((pi/L)^2 + |k|^2) of the
  mirror gap L (a standing wave along the cavity line uses omega = c k), and
  amplitude lambda_a (sqrt(2) g for a single real standing or k = 0 mode,
  2 g for each of the cos / sin pair of a travelling +-k pair).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from .params import ELEM_H, ELEM_O, MASS_AMU, water_reference_geometry, load_water_params
from .units import AMU, C_LIGHT, DT_HALF_FS, KB, WATER_DENSITY

SEED_GEOMETRY = 1
SEED_VELOCITY = 2
SEED_CLUSTER = 3


@dataclass
class System:
    species: np.ndarray        # [n_atoms] int32 element ids
    cell_offset: np.ndarray    # [n_cells + 1] int32 first atom of each cell
    r: np.ndarray              # [n_atoms, 3] positions, bohr
    p: np.ndarray              # [n_atoms, 3] momenta, atomic units
    R_ref: np.ndarray          # [n_cells, 3] fixed reference centres of the mode functions

    @property
    def n_cells(self) -> int:
        return len(self.cell_offset) - 1

    @property
    def n_atoms(self) -> int:
        return len(self.species)


@dataclass
class Modes:
    k: np.ndarray              # [M, 3] wave vectors, 1/bohr
    omega: np.ndarray          # [M] Hartree
    lam: np.ndarray            # [M] coupling amplitudes lambda_a
    phi: np.ndarray            # [M] phase offsets (0: cos mode, -pi/2: sin mode)
    pol: np.ndarray = field(default_factory=lambda: np.array([1.0, 0.0, 0.0]))
    grid: Optional[dict] = None   # uniform in-plane grid description, when there is one

    @property
    def n_modes(self) -> int:
        return len(self.omega)


def random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotation matrices from normalised Gaussian quaternions."""
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1),
    ], 1)


def _centred_water(ref=None) -> np.ndarray:
    g = water_reference_geometry() if ref is None else np.asarray(ref, float)
    m = np.array([MASS_AMU[ELEM_O], MASS_AMU[ELEM_H], MASS_AMU[ELEM_H]])
    return g - (m[:, None] * g).sum(0) / m.sum()


def water_batch(rng: np.random.Generator, centres: np.ndarray, noise: float = 0.02, ref=None):
    """Positions [n, 3 atoms, 3] of n waters centred at ``centres``."""
    centres = np.asarray(centres, float)
    n = len(centres)
    g = _centred_water(ref)
    rot = random_rotations(rng, n)
    pos = np.einsum("nij,aj->nai", rot, g)
    pos += rng.normal(0.0, noise, size=pos.shape)
    return pos + centres[:, None, :]


def _water_system(pos: np.ndarray, centres: np.ndarray) -> System:
    n = pos.shape[0]
    species = np.tile(np.array([ELEM_O, ELEM_H, ELEM_H], np.int32), n)
    off = (3 * np.arange(n + 1)).astype(np.int32)
    return System(species=species, cell_offset=off, r=pos.reshape(-1, 3).copy(),
                  p=np.zeros((3 * n, 3)), R_ref=np.asarray(centres, float).copy())


def cluster_batch(rng: np.random.Generator, sizes, centres, noise: float = 0.02,
                  density: float = WATER_DENSITY, d_min: float = 4.8, d_atom: float = 3.0,
                  ref=None) -> System:
    """(H2O)_n clusters; cluster i holds sizes[i] waters around centres[i]. Candidates for each
    water are drawn 16 at a time and the first acceptable one is kept."""
    sizes = np.asarray(sizes, int)
    centres = np.asarray(centres, float)
    g = _centred_water(ref)
    species, pos, off = [], [], [0]
    for n, c in zip(sizes, centres):
        radius = (3.0 * n / (4.0 * np.pi * density)) ** (1.0 / 3.0)
        while True:
            coms, waters = [], []
            for _ in range(n):
                found = None
                for _batch in range(13):                     # about 200 candidates
                    x = rng.uniform(-radius, radius, (16, 3))
                    rot = random_rotations(rng, 16)
                    wat = np.einsum("kij,aj->kai", rot, g) + rng.normal(0.0, noise, (16, 3, 3)) + x[:, None, :]
                    good = (x * x).sum(1) <= radius * radius
                    if coms:
                        cm = np.array(coms)
                        good &= np.linalg.norm(x[:, None, :] - cm[None], axis=2).min(1) >= d_min
                        placed = np.concatenate(waters)
                        da = np.linalg.norm(wat[:, :, None, :] - placed[None, None], axis=3).min(axis=(1, 2))
                        good &= da >= d_atom
                    k = np.flatnonzero(good)
                    if len(k):
                        found = k[0]
                        break
                if found is None:
                    break
                coms.append(x[found])
                waters.append(wat[found])
            if len(coms) == n:
                break
            radius *= 1.05
        w = np.stack(waters) + c
        pos.append(w.reshape(-1, 3))
        species.append(np.tile(np.array([ELEM_O, ELEM_H, ELEM_H], np.int32), n))
        off.append(off[-1] + 3 * n)
    return System(species=np.concatenate(species), cell_offset=np.array(off, np.int32),
                  r=np.concatenate(pos), p=np.zeros((off[-1], 3)), R_ref=centres.copy())


def periodic_water_cells(rng: np.random.Generator, centres, n_waters: int = 33,
                         side: float = 10.0 * 1.8897261, noise: float = 0.02, d_min: float = 4.8,
                         d_atom: float = 3.0, ref=None):
    """Cubic periodic cells of n_waters waters each (33 per 10 Angstrom cube is liquid density).
    Each water is a rotated, noisy water as in water_batch whose centre of mass is uniform in the
    cube; it is kept when, under the minimum-image convention, its centre is at least d_min from
    every placed centre and each of its atoms at least d_atom from every atom of the other waters.
    After 400 rejected candidates for one water the cell restarts. Positions are unwrapped (each
    water whole) and the cube of cell i is centred on centres[i]. Returns (System, lattice) with
    lattice = side * I."""
    centres = np.asarray(centres, float)
    g = _centred_water(ref)
    lat = side * np.eye(3)
    species, pos, off = [], [], [0]

    def min_image(x):
        return x - side * np.round(x / side)

    for c in centres:
        while True:
            coms, waters = [], []
            for _ in range(n_waters):
                found = None
                for _batch in range(25):                     # 400 candidates
                    x = rng.uniform(0.0, side, (16, 3))
                    rot = random_rotations(rng, 16)
                    wat = np.einsum("kij,aj->kai", rot, g) + rng.normal(0.0, noise, (16, 3, 3)) + x[:, None, :]
                    good = np.ones(16, bool)
                    if coms:
                        dc = min_image(x[:, None, :] - np.array(coms)[None])
                        good &= np.sqrt((dc * dc).sum(2)).min(1) >= d_min
                        placed = np.concatenate(waters)
                        da = min_image(wat[:, :, None, :] - placed[None, None])
                        good &= np.sqrt((da * da).sum(3)).min(axis=(1, 2)) >= d_atom
                    k = np.flatnonzero(good)
                    if len(k):
                        found = k[0]
                        break
                if found is None:
                    break
                coms.append(x[found])
                waters.append(wat[found])
            if len(coms) == n_waters:
                break
        w = np.stack(waters) + (c - 0.5 * side)
        pos.append(w.reshape(-1, 3))
        species.append(np.tile(np.array([ELEM_O, ELEM_H, ELEM_H], np.int32), n_waters))
        off.append(off[-1] + 3 * n_waters)
    system = System(species=np.concatenate(species), cell_offset=np.array(off, np.int32),
                    r=np.concatenate(pos), p=np.zeros((off[-1], 3)), R_ref=centres.copy())
    return system, lat


def mb_momenta(rng: np.random.Generator, system: System, temperature: float = 300.0) -> np.ndarray:
    """Maxwell-Boltzmann momenta, centre-of-mass velocity removed in every cell."""
    m = np.array(MASS_AMU)[system.species] * AMU
    v = rng.normal(size=(system.n_atoms, 3)) * np.sqrt(KB * temperature / m)[:, None]
    off = system.cell_offset
    for c in range(system.n_cells):
        a, b = off[c], off[c + 1]
        vcm = (m[a:b, None] * v[a:b]).sum(0) / m[a:b].sum()
        v[a:b] -= vcm
    return m[:, None] * v


def random_centres(rng: np.random.Generator, n: int, box, d_min: float = 0.0) -> np.ndarray:
    """n points uniform in [0, box); with d_min > 0, by random sequential addition."""
    box = np.asarray(box, float)
    if d_min <= 0.0:
        return rng.uniform(0.0, 1.0, size=(n, 3)) * box
    pts = np.empty((n, 3))
    k = 0
    while k < n:
        x = rng.uniform(0.0, 1.0, 3) * box
        if k == 0 or np.min(np.sum((pts[:k] - x) ** 2, axis=1)) >= d_min * d_min:
            pts[k] = x
            k += 1
    return pts


def standing_modes(n_modes: int, L: float, g: float, n_r: float = 1.0) -> Modes:
    """Standing waves along the cavity line: k_n = n pi / L, u = sin(k_n x), omega = c k_n."""
    n = np.arange(1, n_modes + 1, dtype=float)
    kx = n * np.pi / L
    k = np.zeros((n_modes, 3))
    k[:, 0] = kx
    return Modes(k=k, omega=(C_LIGHT / n_r) * kx, lam=np.full(n_modes, np.sqrt(2.0) * g),
                 phi=np.full(n_modes, -np.pi / 2.0))


def line_modes(n_modes: int, L: float, g: float, k_max: float, n_r: float = 1.0) -> Modes:
    """Real modes on a uniform line of in-plane wave vectors k_x = j dk, j = 0..J (J = n_modes/2):
    cos at j = 0, a cos/sin pair for 0 < j < J and cos at j = J."""
    J = n_modes // 2
    dk = k_max / J
    ks, ph, lam = [], [], []
    for j in range(J + 1):
        for s in ((0,) if j in (0, J) else (0, 1)):
            ks.append(j * dk)
            ph.append(0.0 if s == 0 else -np.pi / 2.0)
            lam.append(np.sqrt(2.0) * g if j == 0 else 2.0 * g)
    kx = np.array(ks)
    k = np.zeros((len(kx), 3))
    k[:, 0] = kx
    omega = (C_LIGHT / n_r) * np.sqrt((np.pi / L) ** 2 + kx ** 2)
    return Modes(k=k, omega=omega, lam=np.array(lam), phi=np.array(ph),
                 grid={"kind": "line", "J": J, "dk": dk})


def grid_modes(Kx: int, Ky: int, dkx: float, dky: float, L: float, g: float, n_r: float = 1.0) -> Modes:
    """Real modes on a uniform in-plane grid: k = (jx dkx, jy dky, 0) with jx < Kx, jy < Ky/2, each
    with a cos and a sin mode (Kx * Ky modes). Mode index a = s + 2 (jy + (Ky/2) jx), s = 0 cos, 1 sin.
    The sin mode of k = 0 vanishes identically and gets lambda = 0."""
    Ky2 = Ky // 2
    jx, jy, s = np.meshgrid(np.arange(Kx), np.arange(Ky2), np.arange(2), indexing="ij")
    jx, jy, s = jx.ravel(), jy.ravel(), s.ravel()
    k = np.stack([jx * dkx, jy * dky, np.zeros_like(jx, dtype=float)], -1).astype(float)
    zero = (jx == 0) & (jy == 0)
    lam = np.where(zero, np.where(s == 0, np.sqrt(2.0) * g, 0.0), 2.0 * g)
    omega = (C_LIGHT / n_r) * np.sqrt((np.pi / L) ** 2 + k[:, 0] ** 2 + k[:, 1] ** 2)
    phi = np.where(s == 0, 0.0, -np.pi / 2.0)
    return Modes(k=k, omega=omega, lam=lam, phi=phi,
                 grid={"kind": "grid", "Kx": Kx, "Ky": Ky, "dkx": dkx, "dky": dky})


# ---------------------------------------------------------------------------------------------
# The workloads (c1..c5, and p33, periodic cells). ``n_cells`` trims a workload to fewer cells with the same recipe (the box
# shrinks so the density stays the same); ``n_modes`` does the same for the mode count.

WORKLOADS = ("c1", "c2", "c3", "c4", "c5", "p33")


def _slab_box(n_waters: float, thickness: float = 30.0):
    area = n_waters / WATER_DENSITY / thickness
    side = np.sqrt(area)
    return np.array([side, side, thickness])


def make_workload(name: str, n_cells: Optional[int] = None, n_modes: Optional[int] = None,
                  params=None):
    """Build one of the workloads. Returns a dict with system, modes, params and run options."""
    params = load_water_params() if params is None else params
    rg = np.random.default_rng(SEED_GEOMETRY)
    rv = np.random.default_rng(SEED_VELOCITY)
    opts = {"dt": DT_HALF_FS, "charge_model": "mulliken", "temperature": 300.0}
    if name == "c1":
        n = 8 if n_cells is None else n_cells
        centres = np.zeros((n, 3))
        centres[:, 0] = rg.uniform(0.0, 2000.0, n)
        system = _water_system(water_batch(rg, centres), centres)
        modes = standing_modes(16 if n_modes is None else n_modes, 2000.0, 0.002)
        opts.update(steps=1000, g=0.002)
    elif name == "c2":
        n = 4096 if n_cells is None else n_cells
        L = n / WATER_DENSITY / 900.0                     # slab L x 30 x 30 at liquid density
        centres = random_centres(rg, n, (L, 30.0, 30.0), d_min=5.0 if n > 1 else 0.0)
        system = _water_system(water_batch(rg, centres), centres)
        L0 = 4096 / WATER_DENSITY / 900.0                 # mode list of the full-size slab
        modes = line_modes(512 if n_modes is None else n_modes, L0, 0.001, k_max=10.0 * np.pi / L0)
        opts.update(steps=10000, g=0.001)
    elif name == "c3":
        n = 65536 if n_cells is None else n_cells
        rc = np.random.default_rng(SEED_CLUSTER)
        sizes = rc.integers(1, 9, size=n)
        box = _slab_box(float(sizes.sum()))
        centres = random_centres(rg, n, box)
        system = cluster_batch(rc, sizes, centres)
        box0 = _slab_box(65536 * 4.5)
        Kx, Ky = (64, 64) if n_modes is None else (int(np.sqrt(n_modes)), n_modes // int(np.sqrt(n_modes)))
        modes = grid_modes(Kx, Ky, 2 * np.pi / box0[0], 2 * np.pi / box0[1], 2000.0, 0.001)
        opts.update(steps=2000, g=0.001, precision="mixed")
    elif name in ("c4", "c5"):
        full = 16384 if name == "c4" else 262144
        n = full if n_cells is None else n_cells
        box = _slab_box(float(n))
        centres = random_centres(rg, n, box)
        system = _water_system(water_batch(rg, centres), centres)
        box0 = _slab_box(float(full))
        if n_modes is None:
            Kx, Ky = (32, 32) if name == "c4" else (64, 128)
        else:
            Kx = int(np.sqrt(n_modes))
            Ky = n_modes // Kx
        modes = grid_modes(Kx, Ky, 2 * np.pi / box0[0], 2 * np.pi / box0[1], 2000.0, 0.001)
        opts.update(steps=10000 if name == "c4" else 20000, g=0.001, charge_model="born_mlp",
                    precision="mixed")
    elif name == "p33":
        # the paper's cell: 33 waters in a periodic 10 Angstrom cube; the cubes sit side by side
        # along the cavity line (x), 304 of them (10,032 waters), 512 line modes as in c2
        n = 304 if n_cells is None else n_cells
        side = 10.0 * 1.8897261
        centres = np.zeros((n, 3))
        centres[:, 0] = (np.arange(n) + 0.5) * side
        system, lattice = periodic_water_cells(rg, centres, side=side)
        L0 = 304 * side
        modes = line_modes(512 if n_modes is None else n_modes, L0, 0.001, k_max=10.0 * np.pi / L0)
        opts.update(steps=2000, g=0.001, lattice=lattice)
    else:
        raise ValueError(f"unknown workload {name!r}")
    system.p = mb_momenta(rv, system, opts["temperature"])
    return {"name": name, "system": system, "modes": modes, "params": params, "options": opts,
            "lattice": opts.get("lattice")}
