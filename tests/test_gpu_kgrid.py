"""Periodic cells on a k-grid (cavmd_options.kgrid; the paper's "Gamma point of a 3 x 3 x 3 folded
supercell") against the oracle's dftb_periodic_k on the same seeded inputs.

The oracle's k-grid is pinned against the explicit 27-copy supercell at the Gamma point (energy,
populations, forces, spectrum, and the finite-difference Born charges), so these tests reach the
paper's sampling through it. Cases: two-water cubes of 8.5 bohr, where the grid changes the
answer by far more than the tolerances, on the 3 x 3 x 3 grid (Gamma and 13 complex points) and
on 2 x 1 x 1 (two self-conjugate points); a sheared lattice; a coupled trajectory (warm starts of
every k-point's basis); finite-difference Born charges; the paper's 33-water cell. Tolerances are
those of the Gamma-point tests: forces 1e-9 of the largest force, populations 1e-10, cell
energies 1e-10 Hartree, trajectories 1e-9 (times the step number)."""
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


def _ctx(P, sy, lat, kgrid, modes=None, **opt):
    params = cs.load_water_params()
    modes = cs.make_workload("c1", n_cells=2)["modes"] if modes is None else modes
    o = P.default_options()
    o.kgrid[:] = kgrid
    for k, v in opt.items():
        setattr(o, k, v)
    return P.Context(sy, params, modes, o, lattice=lat)


def _check_eval(ev, sy, lat, params, kgrid):
    for c in range(sy.n_cells):
        s = slice(sy.cell_offset[c], sy.cell_offset[c + 1])
        ref = PR.dftb_periodic_k(params, sy.species[s], sy.r[s], lat, kgrid)
        fs = np.abs(ref["F"]).max()
        np.testing.assert_allclose(ev["F_dftb"][s], ref["F"], rtol=0, atol=1e-9 * fs)
        np.testing.assert_allclose(ev["q_pop"][s], ref["q"], rtol=0, atol=1e-10)
        np.testing.assert_allclose(ev["E_cell"][c], ref["E"], rtol=0, atol=1e-10)
        x = sy.r[s, 0]
        np.testing.assert_allclose(ev["M"][c], ref["mu"][0], rtol=0, atol=1e-10 * np.abs(x - x.mean()).sum())
        # the grid matters here: the Gamma point alone is another answer
        g = PR.dftb_periodic(params, sy.species[s], sy.r[s], lat, forces=False)
        assert abs(g["E"] - ref["E"]) > 1e3 * 1e-10


@pytest.mark.parametrize("kgrid,sheared", [((3, 3, 3), False), ((2, 1, 1), False), ((3, 3, 3), True)])
def test_small_cells_match_oracle(P, kgrid, sheared):
    sy, lat = _cells(3)
    if sheared:
        lat = SHEARED
    ctx = _ctx(P, sy, lat, kgrid)
    _check_eval(ctx.cavmd_get_eval(), sy, lat, cs.load_water_params(), kgrid)


def test_grid_111_is_the_gamma_kernel(P):
    """{1, 1, 1} and {0, 0, 0} run the Gamma-point kernel: bitwise the default context."""
    sy, lat = _cells(2)
    ref = _ctx(P, sy, lat, (1, 1, 1)).cavmd_get_eval()
    zero = _ctx(P, sy, lat, (0, 0, 0)).cavmd_get_eval()
    for k in ("F_dftb", "q_pop", "E_cell"):
        assert np.array_equal(ref[k], zero[k]), k


def test_trajectory_matches_oracle(P):
    """Four steps of two two-water cells on the 3 x 3 x 3 grid coupled to 16 cavity modes, one
    call per step (every k-point's basis warm started, re-orthonormalised and rotated)."""
    kgrid = (3, 3, 3)
    sy, lat = _cells(2)
    params = cs.load_water_params()
    w = cs.make_workload("c1", n_cells=2)
    mo = w["modes"]
    mo = cs.Modes(k=mo.k, omega=mo.omega, lam=20.0 * mo.lam, phi=mo.phi)
    ctx = _ctx(P, sy, lat, kgrid, modes=mo, graph_chunk=0)
    mat = PR.PeriodicDFTBMatter(params, sy, lat, kgrid=kgrid)
    md = OC.CavityMD(mat, sy.r, sy.p, mo.k, mo.omega, mo.lam, mo.phi, sy.R_ref, w["options"]["dt"])
    x0 = sy.r.copy()
    for s in range(4):
        ctx.cavmd_step(1)
        md.step()
        st = ctx.cavmd_get_state()
        tol = 1e-9 * (1 + s)
        dr = md.r - x0
        np.testing.assert_allclose(st["r"] - x0, dr, rtol=0, atol=tol * np.abs(dr).max())
        np.testing.assert_allclose(st["p"], md.p, rtol=0, atol=tol * np.abs(md.p).max())
        np.testing.assert_allclose(st["q"], md.q, rtol=0, atol=tol * np.abs(md.q).max())
        np.testing.assert_allclose(ctx.cavmd_observables()["e_total"], md.energies()["total"], rtol=1e-11)


def test_born_charges_on_the_grid(P):
    """Forward finite-difference Born charges (the paper's) of two cells on the 3 x 3 x 3 grid,
    displaced copies in the k-grid kernel, against the oracle's born_fd_periodic with the same grid
    (tolerance 5e-8, as for the Gamma point)."""
    kgrid = (3, 3, 3)
    sy, lat = _cells(2)
    params = cs.load_water_params()
    ctx = _ctx(P, sy, lat, kgrid, charge_model=1, born_interval=1)
    ev = ctx.cavmd_get_eval()
    mat = PR.PeriodicDFTBMatter(params, sy, lat, charge_model="born_fd", born_interval=1, kgrid=kgrid)
    out = mat(sy.r)
    np.testing.assert_allclose(ev["b"], out["b"], rtol=0, atol=5e-8)
    g = PR.PeriodicDFTBMatter(params, sy, lat, charge_model="born_fd", born_interval=1)(sy.r)
    assert np.abs(g["b"] - out["b"]).max() > 1e-3            # the grid changes the charges


def test_liquid_cell_of_33_waters(P):
    """The paper's cell (198 orbitals, real forms of 396) on the paper's 3 x 3 x 3 grid: one cell,
    cold start."""
    kgrid = (3, 3, 3)
    sy, lat = _cells(1, n_waters=33, side=10.0 * cs.ANGSTROM, seed=5)
    ctx = _ctx(P, sy, lat, kgrid)
    ev = ctx.cavmd_get_eval()
    params = cs.load_water_params()
    ref = PR.dftb_periodic_k(params, sy.species, sy.r, lat, kgrid)
    fs = np.abs(ref["F"]).max()
    np.testing.assert_allclose(ev["F_dftb"], ref["F"], rtol=0, atol=1e-9 * fs)
    np.testing.assert_allclose(ev["q_pop"], ref["q"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(ev["E_cell"][0], ref["E"], rtol=0, atol=1e-10)
    print(f"\n33-water cell on the 3 x 3 x 3 grid: {ev['scc_iters'].max()} SCC iterations, "
          f"E(k) - E(Gamma) = {ref['E'] - PR.dftb_periodic(params, sy.species, sy.r, lat, forces=False)['E']:.3e} Ha")


def test_p33_on_the_grid_sampled(P):
    """p33 on the 3 x 3 x 3 grid at the size bench.py times it (152 cells of 33 waters, one per SM):
    the last cell against the oracle's k-grid (its plain NumPy solve takes about 1.5 minutes), every
    cell's population sum (264 electrons)."""
    kgrid = (3, 3, 3)
    w = cs.make_workload("p33", n_cells=152)
    sy, lat, params = w["system"], w["lattice"], w["params"]
    o = P.default_options()
    o.kgrid[:] = kgrid
    ctx = P.Context(sy, params, w["modes"], o, lattice=lat)
    ev = ctx.cavmd_get_eval()
    np.testing.assert_allclose(ev["q_pop"].reshape(sy.n_cells, -1).sum(1), 264.0, rtol=0, atol=1e-9)
    for c in (151,):
        s = slice(sy.cell_offset[c], sy.cell_offset[c + 1])
        ref = PR.dftb_periodic_k(params, sy.species[s], sy.r[s], lat, kgrid)
        fs = np.abs(ref["F"]).max()
        np.testing.assert_allclose(ev["F_dftb"][s], ref["F"], rtol=0, atol=1e-9 * fs)
        np.testing.assert_allclose(ev["q_pop"][s], ref["q"], rtol=0, atol=1e-10)
        np.testing.assert_allclose(ev["E_cell"][c], ref["E"], rtol=0, atol=1e-10)


def test_graph_replay_is_bitwise_identical(P):
    """Two-water cells on the 3 x 3 x 3 grid: graph replay of four-step chunks against one call per
    step, bitwise."""
    sy, lat = _cells(2)
    a = _ctx(P, sy, lat, (3, 3, 3), graph_chunk=0)
    b = _ctx(P, sy, lat, (3, 3, 3), graph_chunk=4)
    a.cavmd_step(6)
    b.cavmd_step(6)
    sa, sb = a.cavmd_get_state(), b.cavmd_get_state()
    for k in ("r", "p", "q", "pq"):
        assert np.array_equal(sa[k], sb[k]), k


def test_periodic_cells_with_the_tensor_core_coupling(P):
    """Periodic cells (Gamma point and the 3 x 3 x 3 grid) coupled to config 4's 32 x 32 grid of modes
    through the BF16x3 tensor-core coupling: D and the total force within the bounds of
    tests/bf16x3.py against the plain contractions of the GPU's own dipoles. The cells all sit at
    y = 0, so the sin(jy thy) factors are exactly zero: the GPU's factorised phases give D = 0 for
    the jx = 0 sin modes, while the reference's cos(k.R - pi/2) carries the FP64 rounding of pi/2
    (about 6e-17); the D check adds 4 * 2^-52 lambda_a sum_n |M_n| for that."""
    from bf16x3 import bounds, direct_forward_and_field
    sy, lat = _cells(40)
    mo = cs.make_workload("c4", n_cells=40)["modes"]
    for kgrid in ((1, 1, 1), (3, 3, 3)):
        ctx = _ctx(P, sy, lat, kgrid, modes=mo, precision=2, photon_init=1)
        ev = ctx.cavmd_get_eval()
        obs = ctx.cavmd_observables()
        W = mo.lam * (mo.omega * obs["q"] - obs["D"])
        D_ref, E_ref = direct_forward_and_field(mo, sy.R_ref, ev["M"], W)
        bD, bE = bounds(mo, sy.R_ref, ev["M"], W)
        ref_round = 4.0 * 2.0 ** -52 * np.abs(mo.lam) * np.abs(ev["M"]).sum()
        assert np.all(np.abs(obs["D"] - D_ref) <= bD + ref_round)
        cell = np.repeat(np.arange(sy.n_cells), np.diff(sy.cell_offset))
        F_ref = ev["F_dftb"] + E_ref[cell][:, None] * ev["b"]
        assert np.all(np.abs(ev["F_total"] - F_ref) <= bE[cell][:, None] * np.abs(ev["b"]) + 1e-12)


@pytest.mark.parametrize("kgrid", [(1, 1, 1), (2, 1, 1)])
def test_largest_cell(P, kgrid):
    """The largest periodic cell the kernels take: 42 waters (126 atoms, 252 orbitals; the limits are
    128 atoms and 256 orbitals), at liquid density, at the Gamma point and on a 2 x 1 x 1 grid (real
    forms of 504, the widest problem the k-grid staging holds), against the oracle."""
    rng = np.random.default_rng(5)
    side = 10.0 * cs.ANGSTROM * (42.0 / 33.0) ** (1.0 / 3.0)
    sy, lat = cs.periodic_water_cells(rng, np.zeros((1, 3)), n_waters=42, side=side)
    params = cs.load_water_params()
    ctx = _ctx(P, sy, lat, kgrid)
    ev = ctx.cavmd_get_eval()
    ref = (PR.dftb_periodic(params, sy.species, sy.r, lat) if kgrid == (1, 1, 1)
           else PR.dftb_periodic_k(params, sy.species, sy.r, lat, kgrid))
    fs = np.abs(ref["F"]).max()
    np.testing.assert_allclose(ev["F_dftb"], ref["F"], rtol=0, atol=1e-9 * fs)
    np.testing.assert_allclose(ev["q_pop"], ref["q"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(ev["E_cell"][0], ref["E"], rtol=0, atol=1e-10)
