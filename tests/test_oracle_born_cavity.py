"""Pins of the oracle's dipole derivatives, coupling contraction and time step: finite-difference
convergence orders, exact sum rules, the discrete Fourier transform, exact harmonic solutions,
the paper's own real-space Steps 1-4, energy conservation and the harmonic Rabi closed form."""
import json
import os

import numpy as np
import pytest

import cavmd_synth as cs
from cavmd_synth.params import ELEM_H, ELEM_O
from oracle import cavity as C
from oracle import dftb as D
from oracle import harmonic as HM
from oracle import paper_scheme as PS

WATER = [ELEM_O, ELEM_H, ELEM_H]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def params():
    return cs.load_water_params()


def _waters(n=2, seed=21):
    return cs.water_batch(np.random.default_rng(seed), np.zeros((n, 3)), noise=0.08)


# ------------------------------------------------------------------------ Born charges

def test_born_fd_convergence_orders(params):
    """Forward differences (the paper's choice) converge at O(h), central ones at O(h^2)."""
    pos = _waters(1)
    pol = np.array([1.0, 0.0, 0.0])
    c1 = D.born_fd(params, WATER, pos, pol, h=2e-3, scheme="central")
    c2 = D.born_fd(params, WATER, pos, pol, h=1e-3, scheme="central")
    ref = (4 * c2 - c1) / 3.0                                   # Richardson
    ef = [np.abs(D.born_fd(params, WATER, pos, pol, h=h, scheme="forward") - ref).max() for h in (2e-3, 1e-3)]
    ec = [np.abs(c - ref).max() for c in (c1, c2)]
    assert 1.7 < ef[0] / ef[1] < 2.3
    assert 3.3 < ec[0] / ec[1] < 4.7
    assert ec[1] < 1e-6


def _born_richardson(params, pos, pol):
    """Central differences at h and h/2 combined to O(h^4)."""
    c1 = D.born_fd(params, WATER, pos, pol, h=2e-3, scheme="central")
    c2 = D.born_fd(params, WATER, pos, pol, h=1e-3, scheme="central")
    return (4 * c2 - c1) / 3.0


def test_born_translation_sum_rule(params):
    """sum_j dM/dr_j = Q_cell pol (translating a neutral cell leaves its dipole unchanged)."""
    pos = _waters(2)
    b = _born_richardson(params, pos, np.array([1.0, 0.0, 0.0]))
    np.testing.assert_allclose(b.sum(1), 0.0, atol=1e-9)


def test_born_rotation_sum_rule(params):
    """sum_j Z_j (w x r_j) = w x mu for the full Born tensors Z_j = dmu/dr_j."""
    pos = _waters(1)
    mu = D.dftb(params, WATER, pos, forces=False)["mu"][0]
    Z = np.stack([_born_richardson(params, pos, e)[0] for e in np.eye(3)])   # Z[alpha, j, beta]
    for w in np.eye(3):
        lhs = np.einsum("ajb,jb->a", Z, np.cross(w, pos[0]))
        np.testing.assert_allclose(lhs, np.cross(w, mu), atol=1e-9)


def test_mulliken_charges_sum_to_zero(params):
    out = D.dftb(params, WATER, _waters(3))
    np.testing.assert_allclose(out["Q"].sum(-1), 0.0, atol=1e-12)


# ------------------------------------------------------------------------ coupling contraction

def test_forward_contraction_equals_fft():
    """Cells on a lattice and modes on the DFT grid: D_a is the real/imag part of an FFT."""
    N, a = 64, 7.0
    rng = np.random.default_rng(3)
    M = rng.normal(size=N)
    R = np.stack([np.arange(N) * a, np.zeros(N), np.zeros(N)], 1)
    J = np.arange(N // 2 + 1)
    k = np.zeros((2 * len(J), 3))
    k[:, 0] = np.repeat(2 * np.pi * J / (N * a), 2)
    phi = np.tile([0.0, -np.pi / 2], len(J))
    lam = np.full(len(k), 0.3)
    Dv = C.forward(C.mode_functions(k, phi, R), lam, M)
    F = np.fft.fft(M)                                            # sum_n M_n e^{-2 pi i j n / N}
    np.testing.assert_allclose(Dv[0::2], 0.3 * F.real[J], atol=1e-12)
    np.testing.assert_allclose(Dv[1::2], -0.3 * F.imag[J], atol=1e-12)


def test_field_on_cells_is_the_adjoint():
    rng = np.random.default_rng(4)
    U = rng.normal(size=(9, 13))
    lam, om, q = rng.uniform(0.1, 1, 9), rng.uniform(0.1, 1, 9), rng.normal(size=9)
    Dv = rng.normal(size=9)
    M = rng.normal(size=13)
    # <E, M> = sum_a lambda_a (omega q - D)_a (U M)_a
    E = C.field_on_cells(U, lam, om, q, Dv)
    np.testing.assert_allclose(E @ M, np.sum(lam * (om * q - Dv) * (U @ M)), rtol=1e-13)


# ------------------------------------------------------------------------ photon dynamics

def _harmonic_setup(N=4, mass=1500.0, wv=0.01, d=0.4, seed=0, spread=0.2):
    rng = np.random.default_rng(seed)
    R = np.stack([np.arange(N) * 13.0, np.zeros(N), np.zeros(N)], 1)
    hm = C.HarmonicMatter(R, mass, wv, d)
    r = R + rng.normal(0, spread, (N, 3))
    p = rng.normal(0, 0.5, (N, 3))
    return hm, R, r, p


@pytest.mark.parametrize("split", ["photon_exact", "strang", "paper"])
def test_free_photons_are_exact(split):
    """Zero coupling: every mode is a free oscillator, reproduced exactly at any omega dt."""
    hm, R, r, p = _harmonic_setup()
    k = np.zeros((3, 3))
    om = np.array([0.3, 1.7, 4.1])
    md = C.CavityMD(hm, r, p, k, om, np.zeros(3), np.zeros(3), R, 20.0, splitting=split,
                    photon_init="zero")
    md.q = np.array([0.2, -0.1, 0.05])
    md.pq = np.array([0.0, 0.3, -0.2])
    q0, p0 = md.q.copy(), md.pq.copy()
    for _ in range(50):
        md.step()
    t = 50 * 20.0
    np.testing.assert_allclose(md.q, q0 * np.cos(om * t) + p0 / om * np.sin(om * t), atol=1e-12)
    np.testing.assert_allclose(md.pq, p0 * np.cos(om * t) - om * q0 * np.sin(om * t), atol=1e-12)


def test_frozen_matter_displaced_oscillator():
    """Nuclei that do not move (huge mass): each mode oscillates exactly about D_a / omega_a."""
    hm, R, r, p = _harmonic_setup(mass=1e30, wv=0.0)
    k = np.zeros((2, 3))
    k[1, 0] = 0.05
    om = np.array([0.02, 0.9])
    lam = np.array([0.01, 0.02])
    md = C.CavityMD(hm, r, np.zeros_like(p), k, om, lam, np.zeros(2), R, 15.0, photon_init="zero")
    c = md.D / om
    for _ in range(40):
        md.step()
    t = 40 * 15.0
    np.testing.assert_allclose(md.q, c - c * np.cos(om * t), atol=1e-12)
    np.testing.assert_allclose(md.pq, om * c * np.sin(om * t), atol=1e-12)


def test_zero_coupling_reproduces_bare_dftb_bitwise(params):
    """lambda = 0 gives the bare velocity-Verlet DFTB trajectory bit for bit."""
    w = cs.make_workload("c1", n_cells=2)
    sy, mo = w["system"], w["modes"]
    dt = w["options"]["dt"]
    md = C.CavityMD(C.DFTBMatter(params, sy), sy.r, sy.p, mo.k, mo.omega, 0.0 * mo.lam, mo.phi,
                    sy.R_ref, dt)
    bare = C.DFTBMatter(params, sy)
    r, p = sy.r.copy(), sy.p.copy()
    F = bare(r)["F"]
    m = bare.mass[:, None]
    for _ in range(5):
        md.step()
        p = p + (0.5 * dt * F + 0.0)
        r = r + dt * p / m
        F = bare(r)["F"]
        p = p + (0.5 * dt * F + 0.0)
    assert np.array_equal(md.r, r) and np.array_equal(md.p, p)


@pytest.mark.parametrize("matter", ["harmonic", "dftb"])
def test_kspace_step_equals_paper_realspace_steps(params, matter):
    """Flat dispersion, cells on a lattice, modes on the DFT grid: the k-space form with the paper's
    step order reproduces the paper's real-space / reciprocal-space Steps 1-4 exactly."""
    N, a, w0, g0, dt = 8, 12.0, 0.012, 0.002, 10.0
    R = np.arange(N) * a
    Rv = np.stack([R, np.zeros(N), np.zeros(N)], 1)
    if matter == "harmonic":
        hm, _, r, p = _harmonic_setup(N=N, mass=1200.0, wv=0.011, d=0.6)
        hm.r0 = Rv.copy()
        r = Rv + np.random.default_rng(1).normal(0, 0.2, (N, 3))
        m1 = m2 = hm
        steps = 200
    else:
        cent = Rv
        pos = cs.water_batch(np.random.default_rng(2), cent)
        sy = cs.systems._water_system(pos, cent)
        sy.p = cs.mb_momenta(np.random.default_rng(3), sy)
        m1, m2 = C.DFTBMatter(params, sy), C.DFTBMatter(params, sy)
        r, p = sy.r, sy.p
        steps = 6
    kv = 2 * np.pi * np.arange(N) / (N * a)
    ps = PS.PaperRealSpaceMD(m1, r, p, R, kv, np.full(N, w0), g0, w0, dt)
    ks, ph, lam = [], [], []
    for j in range(N // 2 + 1):
        for s in ((0,) if j in (0, N // 2) else (0, 1)):
            ks.append(2 * np.pi * j / (N * a))
            ph.append(0.0 if s == 0 else -np.pi / 2)
            lam.append(np.sqrt(2) * g0 if j in (0, N // 2) else 2 * g0)
    K = np.zeros((N, 3))
    K[:, 0] = ks
    md = C.CavityMD(m2, r, p, K, np.full(N, w0), np.array(lam), np.array(ph), Rv, dt, splitting="paper")
    for _ in range(steps):
        ps.step()
        md.step()
    np.testing.assert_allclose(md.r, ps.r, atol=1e-11)
    np.testing.assert_allclose(md.p, ps.p, atol=1e-11)
    np.testing.assert_allclose(md.energies()["total"], ps.energies()["total"], rtol=1e-11)


def test_time_reversibility():
    hm, R, r, p = _harmonic_setup()
    k = np.zeros((2, 3))
    k[1, 0] = 0.07
    md = C.CavityMD(hm, r, p, k, np.array([0.02, 2.5]), np.array([0.01, 0.03]), np.zeros(2), R, 12.0)
    s0 = (md.r.copy(), md.p.copy(), md.q.copy(), md.pq.copy())
    for _ in range(100):
        md.step()
    md.p, md.pq = -md.p, -md.pq
    for _ in range(100):
        md.step()
    np.testing.assert_allclose(md.r, s0[0], atol=1e-10)
    np.testing.assert_allclose(-md.p, s0[1], atol=1e-10)
    np.testing.assert_allclose(md.q, s0[2], atol=1e-10)
    np.testing.assert_allclose(-md.pq, s0[3], atol=1e-10)


def _energy_error(params, dt, steps, charge_model="born_central"):
    w = cs.make_workload("c1", n_cells=2)
    sy, mo = w["system"], w["modes"]
    md = C.CavityMD(C.DFTBMatter(params, sy, charge_model=charge_model), sy.r, sy.p, mo.k, mo.omega,
                    mo.lam, mo.phi, sy.R_ref, dt)
    E0 = md.energies()["total"]
    e = []
    for _ in range(steps):
        md.step()
        e.append(md.energies()["total"] - E0)
    return np.array(e), sy.n_atoms


def test_energy_conservation_exact_born(params):
    """Exact dipole derivatives (central FD every step): the coupled system conserves energy at the
    level of the bare Verlet error, which falls as dt^2; no secular drift."""
    dt = cs.units.DT_HALF_FS
    e1, nat = _energy_error(params, dt, 300)
    e2, _ = _energy_error(params, dt / 2, 120)
    ratio = np.abs(e1[:60]).max() / np.abs(e2).max()
    assert 3.0 < ratio < 5.0
    assert np.abs(e1).max() / nat < 2e-5                     # bounded Verlet error
    drift = np.polyfit(np.arange(len(e1)), e1, 1)[0] * len(e1) / nat
    assert abs(drift) < 2e-7                                 # least-squares drift over the run


# ------------------------------------------------------------------------ Rabi splitting

def _spectrum_peaks(x, dt, n_peaks=2):
    n = len(x)
    win = np.hanning(n)
    pad = 16 * n
    spec = np.abs(np.fft.rfft((x - x.mean()) * win, pad))
    freqs = 2 * np.pi * np.fft.rfftfreq(pad, dt)
    idx = [i for i in range(1, len(spec) - 1) if spec[i] > spec[i - 1] and spec[i] >= spec[i + 1]]
    idx = sorted(idx, key=lambda i: -spec[i])[:n_peaks]
    return np.sort(freqs[idx])


@pytest.mark.parametrize("n_osc", [1, 4])
def test_rabi_splitting_from_md_matches_closed_form(n_osc):
    """N oscillators resonant with one k = 0 mode: the MD spectrum shows the two polariton peaks of
    the bright-mode closed form, and their splitting grows as sqrt(N)."""
    wv, mass, d, lam, dt = 0.01, 1.0, 1.0, 0.0015, 5.0
    R = np.zeros((n_osc, 3))
    hm = C.HarmonicMatter(R, mass, wv, d)
    rng = np.random.default_rng(9)
    r = R + rng.normal(0, 1.0, (n_osc, 3))
    md = C.CavityMD(hm, r, np.zeros((n_osc, 3)), np.zeros((1, 3)), np.array([wv]), np.array([lam]),
                    np.zeros(1), R, dt)
    xs = []
    for _ in range(24000):
        md.step()
        xs.append(md.q[0])
    peaks = _spectrum_peaks(np.array(xs), dt)
    expect = HM.polariton_frequencies(wv, wv, lam, d, n_osc, mass)
    resolution = 2 * np.pi / (len(xs) * dt)
    np.testing.assert_allclose(peaks, expect, atol=resolution)


def test_rabi_splitting_scaling_matches_paper_ratios():
    """The paper reports Rabi splittings of 0.012, 0.024, 0.036 eV at eta0, 2 eta0, 3 eta0 (linear
    in the coupling). The harmonic closed form reproduces those ratios in the same regime."""
    with open(os.path.join(GOLDEN, "paper_rabi_splitting.json")) as f:
        gold = json.load(f)
    mult = np.array(gold["eta_multiple"], float)
    split = np.array(gold["splitting_ev"], float)
    wv = 0.19 * cs.EV
    s = []
    for m in mult:
        w = HM.polariton_frequencies(wv, wv, 1e-4 * m, 1.0, 1, 1.0)
        s.append(w[1] - w[0])
    s = np.array(s)
    np.testing.assert_allclose(s / s[0], split / split[0], rtol=2e-3)
    # sqrt(N) scaling of the collective splitting at weak coupling
    s1 = np.diff(HM.polariton_frequencies(wv, wv, 1e-5, 1.0, 1))[0]
    s16 = np.diff(HM.polariton_frequencies(wv, wv, 1e-5, 1.0, 16))[0]
    np.testing.assert_allclose(s16 / s1, 4.0, rtol=1e-3)
