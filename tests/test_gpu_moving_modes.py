"""Moving mode positions (mode functions at the cells' instantaneous centres of mass) against the
FP64 oracle on the same seeded inputs.

Optical wave vectors (about 1e-4 / bohr) change a cell's mode phase by ~1e-4 rad over a whole
run, too little to tell the moving from the fixed form at test tolerances. These tests use
wave vectors of 0.1 to 0.3 / bohr and photons started at q = 0 (away from their minimum). Then
the position term is a visible part of the force, and every test checks that the fixed-position
oracle misses the GPU result by far more than the tolerance.

Tolerances are those of the fixed-position parity tests: trajectories 1e-9 (times the step
number) of the largest displacement, momentum and photon coordinate; forces 1e-9 of the
largest force."""
import numpy as np
import pytest

import cavmd_synth as cs
from oracle import cavity as OC

pytestmark = pytest.mark.gpu
F_REL = 1e-9


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


def _workload(name="c2", n_cells=12, M=24, seed=7, kmin=0.1, kmax=0.3):
    w = cs.make_workload(name, n_cells=n_cells, n_modes=M)
    rng = np.random.default_rng(seed)
    mo = w["modes"]
    k = rng.normal(0.0, 1.0, (mo.n_modes, 3))
    k *= rng.uniform(kmin, kmax, (mo.n_modes, 1)) / np.linalg.norm(k, axis=1, keepdims=True)
    w = dict(w, modes=cs.Modes(k=k, omega=mo.omega, lam=4.0 * mo.lam, phi=rng.uniform(-np.pi, np.pi, mo.n_modes)))
    return w


def _ctx(P, w, **opt):
    o = P.default_options()
    o.mode_positions = 1
    o.photon_init = 1
    for k, v in opt.items():
        setattr(o, k, v)
    return P.Context(w["system"], w["params"], w["modes"], o)


def _oracle(w, mode_positions="com"):
    sy, mo, pa = w["system"], w["modes"], w["params"]
    mat = OC.DFTBMatter(pa, sy)
    md = OC.CavityMD(mat, sy.r, sy.p, mo.k, mo.omega, mo.lam, mo.phi, sy.R_ref, w["options"]["dt"],
                     photon_init="zero", mode_positions=mode_positions)
    return mat, md


@pytest.mark.parametrize("name,n", [("c2", 12), ("c3", 10)])
def test_initial_forces_include_the_position_term(P, name, n):
    w = _workload(name, n)
    ctx = _ctx(P, w)
    _, md = _oracle(w)
    _, fixed = _oracle(w, "fixed")
    ev = ctx.cavmd_get_eval()
    fs = np.abs(md.F).max()
    np.testing.assert_allclose(ev["F_total"], md.F, rtol=0, atol=F_REL * fs)
    assert np.abs(fixed.F - md.F).max() > 1e4 * F_REL * fs


@pytest.mark.parametrize("name,n,steps", [("c2", 12, 6), ("c3", 10, 3)])
def test_trajectory_matches_oracle(P, name, n, steps):
    """Water cells (lane-group kernel) and clusters (persistent kernel); graph_chunk = 0 steps one
    call at a time, so every step opens with the stored field and position term."""
    w = _workload(name, n)
    ctx = _ctx(P, w, graph_chunk=0)
    _, md = _oracle(w)
    _, fixed = _oracle(w, "fixed")
    x0 = w["system"].r.copy()
    for s in range(steps):
        ctx.cavmd_step(1)
        md.step()
        fixed.step()
        st = ctx.cavmd_get_state()
        tol = 1e-9 * (1 + s)
        dr = md.r - x0
        np.testing.assert_allclose(st["r"] - x0, dr, rtol=0, atol=tol * np.abs(dr).max())
        np.testing.assert_allclose(st["p"], md.p, rtol=0, atol=tol * np.abs(md.p).max())
        np.testing.assert_allclose(st["q"], md.q, rtol=0, atol=tol * np.abs(md.q).max())
        np.testing.assert_allclose(st["pq"], md.pq, rtol=0, atol=tol * np.abs(md.pq).max() + 1e-15)
        np.testing.assert_allclose(ctx.cavmd_observables()["e_total"], md.energies()["total"], rtol=1e-11)
    assert np.abs(fixed.p - md.p).max() > 100 * tol * np.abs(md.p).max()   # 250x when written


def test_small_phase_changes_take_the_series_path(P):
    """Wave vectors of 0.01 to 0.03 / bohr: k.(R_n - R0_n) stays below 4e-3, so the mode functions
    come from the Taylor series of the phase change (the optical case) rather than sincos."""
    w = _workload(kmin=0.01, kmax=0.03)
    ctx = _ctx(P, w, graph_chunk=0)
    _, md = _oracle(w)
    sy = w["system"]
    x0 = sy.r.copy()
    for s in range(6):
        ctx.cavmd_step(1)
        md.step()
    R = OC.cell_centres(md.r, md.matter.mass, md.off)
    assert np.abs((R - sy.R_ref) @ w["modes"].k.T).max() < 4e-3
    st = ctx.cavmd_get_state()
    tol = 6e-9
    dr = md.r - x0
    np.testing.assert_allclose(st["r"] - x0, dr, rtol=0, atol=tol * np.abs(dr).max())
    np.testing.assert_allclose(st["p"], md.p, rtol=0, atol=tol * np.abs(md.p).max())
    np.testing.assert_allclose(st["q"], md.q, rtol=0, atol=tol * np.abs(md.q).max())
    np.testing.assert_allclose(ctx.cavmd_get_eval()["F_total"], md.F, rtol=0, atol=F_REL * np.abs(md.F).max())


def test_graph_replay_is_bitwise_identical(P):
    w = _workload()
    a = _ctx(P, w, graph_chunk=0)
    b = _ctx(P, w, graph_chunk=4)
    a.cavmd_step(9)
    b.cavmd_step(9)
    sa, sb = a.cavmd_get_state(), b.cavmd_get_state()
    for k in ("r", "p", "q", "pq"):
        assert np.array_equal(sa[k], sb[k]), k


def test_energy_history_matches_oracle(P):
    """100 steps: the GPU's total-energy record follows the oracle's step by step. Over 400 steps
    both errors peak at 2.1939e-4 Hartree (measured when this test was written). The position
    term's own conservation is pinned on the oracle (second-order energy error with exact dipole
    derivatives)."""
    steps = 100
    w = _workload()
    ctx = _ctx(P, w, energy_history=steps + 1, graph_chunk=25)
    _, md = _oracle(w)
    e_ref = [md.energies()["total"]]
    for _ in range(steps):
        md.step()
        e_ref.append(md.energies()["total"])
    e_ref = np.array(e_ref)
    ctx.cavmd_step(steps)
    h = ctx.cavmd_energy_history(steps + 1)
    scale = np.abs(e_ref - e_ref[0]).max()
    np.testing.assert_allclose(h[:, 6] - e_ref[0], e_ref - e_ref[0], rtol=0, atol=1e-4 * scale)
