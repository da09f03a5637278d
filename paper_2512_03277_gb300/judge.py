"""The judge of the surrogate forms: energy drift, heating and spectral bands of a charge model and
a coupling precision, from trajectories run through the library.

The paper (Results) tells Born from Mulliken dipole derivatives by the spurious heating the
Mulliken charges cause and by the positions of the IR bands. Here the same measures judge the
network Born charges and the BF16x3 tensor-core coupling against explicit finite-difference Born
charges (central differences every step, the conservative reference) with the FP64 coupling:
  drift     least-squares slope of E_total(t) times the run length, per atom (Ha/atom);
  heating   mean temperature over the last tenth of the run minus the mean over its second tenth
            (the first tenth is the equipartition transient from the initial state);
  bands     intensity-weighted mean frequency of the dipole spectrum in a window around each
            vibrational band; the band error of a run is its largest shift against the reference.
The spectrum is that of the paper (w^2 times the cosine transform of the windowed dipole
autocorrelation), from the correlation function the library accumulates on the device.

Resonant single-box cavity (the setting of Eq. hlm4): a line of independent waters, each its own
cell, and the smallest in-plane mode grid the tensor-core coupling accepts (2 x 2: k = 0 and one
k_x, each with a cos and a sin mode), the k = 0 mode tuned to the bend of the synthetic water and
the k_x pair detuned to 2.5 times the bend, away from both bands.
"""
from __future__ import annotations

import numpy as np

import cavmd_synth as cs

from . import spectra as S

KB = 3.166811563e-6                       # Hartree per kelvin
CHARGE = {"mulliken": 0, "born_fd": 1, "born_central": 2, "born_mlp": 3}
WATER = [0, 1, 1]


def resonant_box(params, n_waters: int = 33, seed: int = 0, lam: float = 0.1, spacing: float = 20.0):
    """(system, modes, w_bend): n_waters waters on a line (20 bohr apart, geometry seed 1) with
    300 K Maxwell-Boltzmann momenta from seed 100 + seed, and the resonant 2 x 2 mode grid."""
    wb = params.meta["harmonic_freq_hartree"][0]
    c = cs.units.C_LIGHT
    L = c * np.pi / wb                                   # k = 0 mode at the bend
    dkx = (wb / c) * np.sqrt(2.5 ** 2 - 1.0)             # k_x pair at 2.5 x the bend
    modes = cs.grid_modes(2, 2, dkx, 1.0, L, lam / np.sqrt(2.0))
    centres = np.zeros((n_waters, 3))
    centres[:, 0] = np.arange(n_waters) * spacing
    pos = cs.water_batch(np.random.default_rng(1), centres)
    sy = cs.systems._water_system(pos, centres)
    sy.p = cs.mb_momenta(np.random.default_rng(100 + seed), sy, 300.0)
    return sy, modes, wb


def resonant_workload(params, name: str = "c4", coupling: float = 0.1 * np.sqrt(33.0), top: float = 1.3):
    """(system, modes, w_bend): the cells of a grid workload (c4: 16,384 waters) and a mode grid of its
    size (c4: 32 x 32, 1024 modes) in a resonant cavity: the k = 0 mode at the bend and the in-plane
    wave vectors spaced so that the largest reaches `top` times the bend (the lower polariton band
    of the paper's angle-resolved setting; omega dt stays near 0.2, where the workload's own grid,
    spaced by 2 pi over the slab, puts its modes hundreds of times above the bands). The amplitudes
    make N sum_a lambda_a^2 over the cos modes, which all see nearly the same phase across the slab,
    equal the resonant box's collective coupling 0.1^2 x 33."""
    w = cs.make_workload(name, params=params)
    g = w["modes"].grid
    Kx, Ky2 = g["Kx"], g["Ky"] // 2
    wb = params.meta["harmonic_freq_hartree"][0]
    kz = wb / cs.units.C_LIGHT
    dk = kz * np.sqrt(top ** 2 - 1.0) / np.hypot(Kx - 1, Ky2 - 1)
    g0 = coupling / (2.0 * np.sqrt(w["system"].n_cells * Kx * Ky2))
    modes = cs.grid_modes(Kx, g["Ky"], dk, dk, np.pi / kz, g0)
    return w["system"], modes, wb


def temperature_curve(T, points: int = 11):
    """The temperature at `points` evenly spaced steps of a run (K)."""
    idx = np.linspace(0, len(T) - 1, points).astype(int)
    return [(int(i), float(T[i])) for i in idx]


def run(P, params, system, modes, model: str, precision: int, steps: int, mlp=None,
        born_interval: int | None = None, lags: int | None = None, lattice=None):
    """One trajectory of `steps` steps. model: 'mulliken', 'born_fd' (forward differences, every
    born_interval steps, 3 by default as in the paper), 'born_central' (every step unless
    born_interval is given) or 'born_mlp' (the network `mlp`). Returns the energy record, drift,
    temperature series and the total-dipole autocorrelation."""
    o = P.default_options()
    o.energy_history = steps + 1
    o.charge_model = CHARGE[model]
    if born_interval is None:
        born_interval = 3 if model == "born_fd" else 1
    o.born_interval = born_interval
    o.precision = precision
    o.acf_lags = (steps + 1) // 2 if lags is None else lags
    ctx = P.Context(system, params, modes, o, lattice=lattice)
    try:
        if model == "born_mlp":
            if mlp is None:
                raise ValueError("the network model needs its parameters")
            ctx.cavmd_load_born_mlp(mlp)
        ctx.cavmd_step(steps)
        h = ctx.cavmd_energy_history(steps + 1)
        acf, n = ctx.cavmd_autocorrelation()
    finally:
        ctx.cavmd_destroy()
    na = system.n_atoms
    e = h[:, 6] - h[0, 6]
    drift = float(np.polyfit(np.arange(len(e)), e, 1)[0] * len(e) / na)
    T = 2.0 * h[:, 0] / (3.0 * na * KB)
    return {"drift": drift, "T": T, "acf_dipole": acf[-1], "n_samples": n, "energy": h}


def heating(T) -> float:
    """Mean temperature over the last tenth of a run minus the mean over its second tenth (K)."""
    n = len(T)
    k = max(1, n // 10)
    return float(np.mean(T[-k:]) - np.mean(T[k:2 * k]))


def centroid(om, I, lo, hi) -> float:
    """Intensity-weighted mean frequency of I(om) over lo < om < hi."""
    m = (om > lo) & (om < hi)
    w = np.clip(I[m], 0.0, None)
    return float((om[m] * w).sum() / w.sum())


def bands(acf, dt, w_bend):
    """(bend, stretch) band centroids in eV of the spectrum of an averaged dipole correlation."""
    om, I = S.spectrum_from_acf(acf, dt)
    return (centroid(om, I, 0.8 * w_bend, 1.3 * w_bend) / S.EV,
            centroid(om, I, 1.35 * w_bend, 1.7 * w_bend) / S.EV)


def compare(P, params, cases, mlp=None, steps: int = 10000, replicas: int = 4, n_waters: int = 33,
            lam: float = 0.1):
    """Runs every (model, precision) of `cases` on the resonant box for `replicas` velocity seeds.
    The first case is the reference of the band errors. Returns {(model, precision): dict(drift =
    the largest |drift| over the replicas, heating = their mean, bend, stretch, band_error_mev)}."""
    out = {}
    dt = None
    wb = None
    for model, prec in cases:
        drifts, heats, acfs = [], [], []
        for seed in range(replicas):
            sy, modes, wb = resonant_box(params, n_waters, seed, lam)
            r = run(P, params, sy, modes, model, prec, steps, mlp=mlp)
            drifts.append(r["drift"])
            heats.append(heating(r["T"]))
            acfs.append(r["acf_dipole"])
        dt = P.default_options().dt
        bend, stretch = bands(np.mean(acfs, 0), dt, wb)
        out[(model, prec)] = {"drift": float(np.max(np.abs(drifts))), "heating": float(np.mean(heats)),
                              "bend": bend, "stretch": stretch}
    ref = out[cases[0]]
    for v in out.values():
        v["band_error_mev"] = 1e3 * max(abs(v["bend"] - ref["bend"]), abs(v["stretch"] - ref["stretch"]))
    return out
