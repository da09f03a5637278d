"""Energy drift and spectral bands of the charge models and of both coupling precisions on a
resonant cavity (GPU, 10^4 steps).

System: 33 synthetic waters, each its own cell, 300 K Maxwell-Boltzmann momenta, four replicas.
Cavity: the smallest in-plane mode grid the tensor-core coupling accepts (2 x 2: k = 0 and one k_x,
each with a cos and a sin mode), the k = 0 mode tuned to the bend of the synthetic water with
lambda = 0.1 (the single-box setting of Eq. hlm4), the k_x pair detuned to 2.5 times the bend.
Dipole derivatives:
  exact      central finite differences every step (conservative up to the FD error),
  network    the Born-charge network trained on the oracle's finite-difference tensors,
  mulliken   Mulliken charges (the paper's cheap replacement),
  paper      forward finite differences refreshed every 3 steps (the paper's scheme).
The exact and network runs are made with the FP64 coupling and with the BF16x3 tensor-core
coupling. The spectrum is the dipole autocorrelation (Hann window, w^2 weighting); the bend and
stretch bands are compared by their intensity-weighted mean frequencies, which are stable where
the polariton splitting makes the highest peak jump between branches.
Checked: the exact runs meet the 1e-6 Ha/atom drift target; the network drifts less than the
Mulliken model and moves the bands less; the tensor-core coupling changes neither the drift nor
the bands beyond the replica noise. The run is deterministic (fixed seeds, fixed-order sums)."""
import numpy as np
import pytest

import cavmd_synth as cs
from oracle import mlp as NN

pytestmark = pytest.mark.gpu
WATER = [0, 1, 1]
STEPS = 10000
REPLICAS = 4


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2512_03277_gb300 import build
    build.build()
    import paper_2512_03277_gb300 as P
    P.load_library()
    return P


def _modes(w_bend):
    c = cs.units.C_LIGHT
    L = c * np.pi / w_bend                                   # k = 0 mode at the bend
    dkx = (w_bend / c) * np.sqrt(2.5 ** 2 - 1.0)             # k_x pair at 2.5 x the bend
    return cs.grid_modes(2, 2, dkx, 1.0, L, 0.1 / np.sqrt(2.0))


def _system(seed):
    centres = np.zeros((33, 3))
    centres[:, 0] = np.arange(33) * 20.0
    pos = cs.water_batch(np.random.default_rng(1), centres)
    sy = cs.systems._water_system(pos, centres)
    sy.p = cs.mb_momenta(np.random.default_rng(100 + seed), sy, 300.0)
    return sy


def _run(P, params, modes, model, precision, mlp, seed):
    from paper_2512_03277_gb300 import spectra as S
    sy = _system(seed)
    o = P.default_options()
    o.energy_history = STEPS + 1
    o.charge_model = {"exact": 2, "network": 3, "mulliken": 0, "paper": 1}[model]
    o.born_interval = 3 if model == "paper" else 1
    o.precision = precision
    ctx = P.Context(sy, params, modes, o)
    if model == "network":
        ctx.cavmd_load_born_mlp(mlp)
    D = np.empty(STEPS + 1)
    D[0] = ctx.cavmd_observables()["D"][0]      # k = 0 cos mode: proportional to sum_n M_n
    for s in range(STEPS):
        ctx.cavmd_step(1)
        D[s + 1] = ctx.cavmd_observables()["D"][0]
    h = ctx.cavmd_energy_history(STEPS + 1)
    e = h[:, 6] - h[0, 6]
    drift = np.polyfit(np.arange(len(e)), e, 1)[0] * len(e) / sy.n_atoms
    om, I = S.spectrum(D, o.dt)
    ctx.cavmd_destroy()
    return drift, om, I


def _centroid(om, I, lo, hi):
    m = (om > lo) & (om < hi)
    w = np.clip(I[m], 0.0, None)
    return float((om[m] * w).sum() / w.sum())


def test_drift_and_bands_of_charge_models_and_coupling_precisions(P, capsys):
    from paper_2512_03277_gb300 import spectra as S
    from paper_2512_03277_gb300.cavmd import BornMLP
    params = cs.load_water_params()
    wb = params.meta["harmonic_freq_hartree"][0]
    modes = _modes(wb)
    pos = cs.water_batch(np.random.default_rng(21), np.zeros((1536, 3)), noise=0.06)
    Z, Q = NN.born_fd_tensors(params, WATER, pos)
    net = BornMLP(NN.init_params(np.random.default_rng(4)).astype(np.float32))
    net.cavmd_mlp_set_data(np.tile(WATER, len(pos)), pos.reshape(-1, 3), Q.ravel(), Z.reshape(-1, 3, 3))
    net.cavmd_mlp_train(epochs=120, batch_cells=64, lr=2e-3, seed=5)
    mlp = net.cavmd_mlp_get_params()
    out = {}
    for model, prec in (("exact", 0), ("exact", 2), ("network", 0), ("network", 2), ("mulliken", 0), ("paper", 0)):
        drifts, spec = [], []
        for seed in range(REPLICAS):
            d, om, I = _run(P, params, modes, model, prec, mlp, seed)
            drifts.append(d)
            spec.append(I)
        I = np.mean(spec, 0)
        out[(model, prec)] = (float(np.max(np.abs(drifts))), _centroid(om, I, 0.8 * wb, 1.3 * wb) / S.EV,
                              _centroid(om, I, 1.35 * wb, 1.7 * wb) / S.EV)
    ref = out[("exact", 0)]
    err = {k: max(abs(v[1] - ref[1]), abs(v[2] - ref[2])) for k, v in out.items()}
    with capsys.disabled():
        for (m, p), v in out.items():
            print(f"\n{m:9s} {'BF16x3' if p else 'FP64  '} max |drift| {v[0]:.2e} Ha/atom  bend {v[1]:.4f} eV  "
                  f"stretch {v[2]:.4f} eV  band error {1e3 * err[(m, p)]:.2f} meV", end="")
    assert out[("exact", 0)][0] < 1e-6 and out[("exact", 2)][0] < 1e-6
    for p in (0, 2):
        assert out[("network", p)][0] < out[("mulliken", 0)][0]
        assert err[("network", p)] < err[("mulliken", 0)]
    for m in ("exact", "network"):   # the tensor-core coupling against the FP64 coupling
        a, b = out[(m, 0)], out[(m, 2)]
        assert abs(a[1] - b[1]) < 1e-3 and abs(a[2] - b[2]) < 1e-3
        assert b[0] < 2.0 * a[0] + 1e-8
