"""Periodic cells at the Gamma point (cavmd_system.lattice) against the FP64 oracle
(oracle/periodic.py) on the same seeded inputs.

Cases: two-water cubes of 8.5 bohr, where every term (Slater-Koster blocks, repulsion, the gamma
remainder and the Ewald sums) has images, in a cubic and a sheared lattice; the paper's cell,
33 waters in a 10 Angstrom cube; a short trajectory with the cavity coupling; graph replay.
Tolerances are those of the isolated-cell parity tests: forces 1e-9 of the largest force,
populations 1e-10, cell energies 1e-10 Hartree; the dipole within what the population tolerance
implies for the cell's extent, and against the GPU's own charges to rounding; trajectories 1e-9
(times the step number) of the largest displacement, momentum and photon coordinate."""
import numpy as np
import pytest

import cavmd_synth as cs
from oracle import cavity as OC
from oracle import periodic as PR

pytestmark = pytest.mark.gpu
SIDE = 8.5
SHEARED = np.array([[8.5, 0.0, 0.0], [2.0, 8.5, 0.0], [-1.5, 1.0, 8.5]])


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


def _cells(n_cells, n_waters=2, side=SIDE, seed=21):
    rng = np.random.default_rng(seed)
    centres = np.zeros((n_cells, 3))
    centres[:, 0] = rng.uniform(0.0, 2000.0, n_cells)
    kw = dict(d_min=4.0, d_atom=2.8) if n_waters < 33 else {}
    sy, lat = cs.periodic_water_cells(rng, centres, n_waters=n_waters, side=side, **kw)
    sy.p = cs.mb_momenta(np.random.default_rng(seed + 1), sy, 300.0)
    return sy, lat


def _ctx(P, sy, lat, modes=None, **opt):
    params = cs.load_water_params()
    modes = cs.make_workload("c1", n_cells=2)["modes"] if modes is None else modes
    o = P.default_options()
    for k, v in opt.items():
        setattr(o, k, v)
    return P.Context(sy, params, modes, o, lattice=lat)


def _check_eval(ev, sy, lat, params):
    for c in range(sy.n_cells):
        s = slice(sy.cell_offset[c], sy.cell_offset[c + 1])
        ref = PR.dftb_periodic(params, sy.species[s], sy.r[s], lat)
        fs = np.abs(ref["F"]).max()
        np.testing.assert_allclose(ev["F_dftb"][s], ref["F"], rtol=0, atol=1e-9 * fs)
        np.testing.assert_allclose(ev["q_pop"][s], ref["q"], rtol=0, atol=1e-10)
        np.testing.assert_allclose(ev["E_cell"][c], ref["E"], rtol=0, atol=1e-10)
        # the dipole: from the GPU's own charges to rounding, and against the oracle within what
        # the population tolerance implies, 1e-10 sum_a |x_a - mean x| (neutral cell)
        x = sy.r[s, 0]
        Q = params.zval[sy.species[s]] - ev["q_pop"][s]
        np.testing.assert_allclose(ev["M"][c], Q @ (x - x[0]), rtol=0, atol=1e-13 * np.abs(Q).sum() * np.abs(x - x[0]).max())
        np.testing.assert_allclose(ev["M"][c], ref["mu"][0], rtol=0, atol=1e-10 * np.abs(x - x.mean()).sum())


@pytest.mark.parametrize("sheared", [False, True])
def test_small_cells_match_oracle(P, sheared):
    sy, lat = _cells(3)
    if sheared:
        lat = SHEARED
    params = cs.load_water_params()
    for c in range(sy.n_cells):   # the overlap stays positive definite in both lattices
        s = slice(sy.cell_offset[c], sy.cell_offset[c + 1])
        H0, S = PR.build_h0_s_periodic(params, PR.D.Layout(params, sy.species[s]), sy.r[s], lat)
        assert np.linalg.eigvalsh(S).min() > 0.05
    ctx = _ctx(P, sy, lat)
    _check_eval(ctx.cavmd_get_eval(), sy, lat, params)


def test_liquid_cells_of_33_waters_match_oracle(P):
    """The paper's cell (198 orbitals): two cells, cold start (Jacobi sweeps) at init."""
    sy, lat = _cells(2, n_waters=33, side=10.0 * cs.ANGSTROM, seed=5)
    ctx = _ctx(P, sy, lat)
    ev = ctx.cavmd_get_eval()
    assert ev["scc_iters"].max() < 200
    _check_eval(ev, sy, lat, cs.load_water_params())


def test_trajectory_matches_oracle(P):
    """Six steps of two periodic two-water cells coupled to 16 cavity modes; graph_chunk = 0 so
    every step is one call (warm starts: re-orthonormalised basis, Cayley updates)."""
    sy, lat = _cells(2)
    params = cs.load_water_params()
    w = cs.make_workload("c1", n_cells=2)
    mo = w["modes"]
    mo = cs.Modes(k=mo.k, omega=mo.omega, lam=20.0 * mo.lam, phi=mo.phi)
    ctx = _ctx(P, sy, lat, modes=mo, graph_chunk=0)
    mat = PR.PeriodicDFTBMatter(params, sy, lat)
    md = OC.CavityMD(mat, sy.r, sy.p, mo.k, mo.omega, mo.lam, mo.phi, sy.R_ref, w["options"]["dt"])
    x0 = sy.r.copy()
    for s in range(6):
        ctx.cavmd_step(1)
        md.step()
        st = ctx.cavmd_get_state()
        tol = 1e-9 * (1 + s)
        dr = md.r - x0
        np.testing.assert_allclose(st["r"] - x0, dr, rtol=0, atol=tol * np.abs(dr).max())
        np.testing.assert_allclose(st["p"], md.p, rtol=0, atol=tol * np.abs(md.p).max())
        np.testing.assert_allclose(st["q"], md.q, rtol=0, atol=tol * np.abs(md.q).max())
        # photon momenta start at 0 and grow by impulses dt lambda (omega q - D) that nearly cancel:
        # their scale is the impulse dt max|lambda| sum_n |M_n|, not their current size
        imp = w["options"]["dt"] * np.abs(mo.lam).max() * np.abs(md.out["M"]).sum()
        np.testing.assert_allclose(st["pq"], md.pq, rtol=0, atol=tol * (np.abs(md.pq).max() + imp))
        np.testing.assert_allclose(ctx.cavmd_observables()["e_total"], md.energies()["total"], rtol=1e-11)


def test_liquid_cell_warm_steps(P):
    """The paper's cell through warm steps: three steps against the oracle (the within-block
    Jacobi sweep and the Cayley updates at 198 orbitals), then 30 more in which the SCC iteration
    count stays flat (without the sweep it grew step by step until the SCC failed)."""
    sy, lat = _cells(1, n_waters=33, side=10.0 * cs.ANGSTROM, seed=5)
    params = cs.load_water_params()
    mo = cs.make_workload("c1", n_cells=2)["modes"]
    ctx = _ctx(P, sy, lat, modes=mo, graph_chunk=0)
    md = OC.CavityMD(PR.PeriodicDFTBMatter(params, sy, lat), sy.r, sy.p, mo.k, mo.omega, mo.lam, mo.phi,
                     sy.R_ref, cs.make_workload("c1", n_cells=2)["options"]["dt"])
    x0 = sy.r.copy()
    for s in range(3):
        ctx.cavmd_step(1)
        md.step()
        st = ctx.cavmd_get_state()
        tol = 1e-9 * (1 + s)
        dr = md.r - x0
        np.testing.assert_allclose(st["r"] - x0, dr, rtol=0, atol=tol * np.abs(dr).max())
        np.testing.assert_allclose(st["p"], md.p, rtol=0, atol=tol * np.abs(md.p).max())
        np.testing.assert_allclose(ctx.cavmd_get_eval()["q_pop"], md.matter.q, rtol=0, atol=1e-10)
    its = []
    for s in range(30):
        ctx.cavmd_step(1)
        its.append(ctx.cavmd_observables(want_arrays=False)["scc_iter_max"])
    assert max(its) <= 16, its


def test_graph_replay_is_bitwise_identical(P):
    sy, lat = _cells(3)
    a = _ctx(P, sy, lat, graph_chunk=0)
    b = _ctx(P, sy, lat, graph_chunk=4)
    a.cavmd_step(9)
    b.cavmd_step(9)
    sa, sb = a.cavmd_get_state(), b.cavmd_get_state()
    for k in ("r", "p", "q", "pq"):
        assert np.array_equal(sa[k], sb[k]), k


def test_full_size_p33_sampled(P):
    """The p33 workload at the size bench.py times (304 cells of 33 waters, 10,032 waters, 512
    modes): three sampled cells against the oracle, every cell's population sum (264 electrons),
    and one step."""
    w = cs.make_workload("p33")
    sy, lat = w["system"], w["lattice"]
    ctx = P.Context(sy, w["params"], w["modes"], P.default_options(), lattice=lat)
    ev = ctx.cavmd_get_eval()
    np.testing.assert_allclose(ev["q_pop"].reshape(sy.n_cells, -1).sum(1), 264.0, rtol=0, atol=1e-9)
    pick = [0, 151, 303]
    idx = np.concatenate([np.arange(sy.cell_offset[c], sy.cell_offset[c + 1]) for c in pick])
    sub = cs.System(species=sy.species[idx], cell_offset=np.arange(len(pick) + 1, dtype=np.int32) * 99,
                    r=sy.r[idx], p=sy.p[idx], R_ref=sy.R_ref[pick])
    sev = {k: (ev[k][idx] if k in ("F_dftb", "q_pop") else ev[k][pick]) for k in ("F_dftb", "q_pop", "E_cell", "M")}
    _check_eval(sev, sub, lat, w["params"])
    ctx.cavmd_step(1)
    st = ctx.cavmd_get_state()
    assert st["step"] == 1 and np.all(np.isfinite(st["p"])) and np.all(np.isfinite(st["q"]))


@pytest.mark.parametrize("model,code", [("born_fd", 1), ("born_central", 2)])
def test_born_charges_of_periodic_cells(P, model, code):
    """Finite-difference Born charges of periodic cells (forward as in the paper, and central) as
    displaced copies of every cell in the periodic kernel, against the oracle's born_fd_periodic;
    then three coupled steps with the charges refreshed every step, against the oracle's trajectory.
    Tolerance of b: 5e-8, the water kernels' (each side's fixed point within about 2e-12 of the
    exact one, times the lever arm, over h = 1e-3)."""
    sy, lat = _cells(3)
    params = cs.load_water_params()
    ctx = _ctx(P, sy, lat, charge_model=code, born_interval=1, graph_chunk=0)
    ev = ctx.cavmd_get_eval()
    mat = PR.PeriodicDFTBMatter(params, sy, lat, charge_model=model, born_interval=1)
    mo = cs.make_workload("c1", n_cells=2)["modes"]
    md = OC.CavityMD(mat, sy.r, sy.p, mo.k, mo.omega, mo.lam, mo.phi, sy.R_ref, 0.5 * 41.341373335)
    np.testing.assert_allclose(ev["b"], md.out["b"], rtol=0, atol=5e-8)
    assert np.abs(md.out["b"] - md.out["Q"][:, None] * np.array([1.0, 0.0, 0.0])).max() > 1e-3   # not Mulliken
    x0 = sy.r.copy()
    for s in range(3):
        ctx.cavmd_step(1)
        md.step()
        st = ctx.cavmd_get_state()
        tol = 1e-9 * (1 + s)
        np.testing.assert_allclose(st["r"] - x0, md.r - x0, rtol=0, atol=tol * np.abs(md.r - x0).max())
        np.testing.assert_allclose(st["p"], md.p, rtol=0, atol=tol * np.abs(md.p).max())
    np.testing.assert_allclose(ctx.cavmd_get_eval()["b"], md.out["b"], rtol=0, atol=5e-8)
