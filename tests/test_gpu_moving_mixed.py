"""Moving mode positions on the tensor-core (BF16x3) coupling against the FP64 oracle.

Every step rebuilds the factorised phase panels at the cells' centres of mass, and the back
product forms the field E_n and its gradient G_n = sum_a W_a grad u_a(R_n) (the position term of
the force, (m_j / m_n) M_n G_n). The bounds are derived in tests/bf16x3.py: D_a within EPS_D of
lambda_a sum_n mag(a, n) |M_n|, E_n within EPS_E of sum_a mag(a, n) |W_a| and each gradient
component within EPS_G of sum_a |k_a| mag'(a, n) |W_a|, all at the centres of mass.

The grid's wave vectors are scaled up twentyfold (to ~0.05-1.6 / bohr), the couplings fourfold and
the photons start at q = 0, so that the position term is a visible part of the force: every test
checks that dropping it misses the GPU result by far more than the bound."""
import numpy as np
import pytest

import cavmd_synth as cs
from oracle import cavity as OC

from bf16x3 import bounds, direct_forward_and_field, direct_gradient, grad_bounds

pytestmark = pytest.mark.gpu


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


def _workload(name="c4", n=300, scale=20.0):
    w = cs.make_workload(name, n_cells=n)
    mo = w["modes"]
    g = dict(mo.grid, dkx=mo.grid["dkx"] * scale, dky=mo.grid["dky"] * scale)
    return dict(w, modes=cs.Modes(k=mo.k * scale, omega=mo.omega, lam=4.0 * mo.lam, phi=mo.phi, pol=mo.pol, grid=g))


def _ctx(P, w, **opt):
    o = P.default_options()
    o.mode_positions = 1
    o.photon_init = 1
    for k, v in opt.items():
        setattr(o, k, v)
    return P.Context(w["system"], w["params"], w["modes"], o)


def _centres(w, r):
    sy = w["system"]
    mat = OC.DFTBMatter(w["params"], sy)
    off = np.asarray(sy.cell_offset)
    return OC.cell_centres(r, mat.mass, off), mat.mass, off


def _check_eval(ctx, w, r, label, margin=100.0):
    """D, and F_total = F_dftb + E_n b_j + (m_j / m_n) M_n G_n, against the plain contractions of the
    GPU's own dipoles at the centres of mass of positions r, within the bounds; the position term
    itself exceeds `margin` times the largest force bound."""
    mo = w["modes"]
    R, mass, off = _centres(w, r)
    ev = ctx.cavmd_get_eval()
    obs = ctx.cavmd_observables()
    M = ev["M"]
    W = mo.lam * (mo.omega * obs["q"] - obs["D"])
    D_ref, E_ref = direct_forward_and_field(mo, R, M, W)
    G_ref = direct_gradient(mo, R, W)
    bD, bE = bounds(mo, R, M, W)
    bGx, bGy = grad_bounds(mo, R, W)
    assert np.all(np.abs(obs["D"] - D_ref) <= bD + 1e-300)
    cell = np.repeat(np.arange(len(off) - 1), np.diff(off))
    mt = np.add.reduceat(mass, off[:-1])
    wm = (mass / mt[cell] * M[cell])[:, None]
    pos = wm * G_ref[cell]
    F_ref = ev["F_dftb"] + E_ref[cell][:, None] * ev["b"] + pos
    bG = np.stack([bGx, bGy, np.zeros_like(bGx)], 1)
    bF = bE[cell][:, None] * np.abs(ev["b"]) + np.abs(wm) * bG[cell] + 1e-12
    err = np.abs(ev["F_total"] - F_ref)
    assert np.all(err <= bF)
    assert np.abs(pos).max() > margin * bF.max()       # the position term is far above the bound
    live = bD > 0
    print(f"\n{label}: max |dD| / bound {np.max(np.abs(obs['D'] - D_ref)[live] / bD[live]):.3f}, "
          f"max |dF| / bound {np.max(err / bF):.3f}, position term / bound {np.abs(pos).max() / bF.max():.0f}")
    return bF


def test_initial_evaluation_within_bound(P):
    w = _workload()
    ctx = _ctx(P, w, precision=2)
    _check_eval(ctx, w, w["system"].r, "moving c4 300 cells, initial")


def _energy_tol(w, obs, M, r):
    """How far the total energy can move when every D_a moves within its bound: the photon sector
    depends on D_a through (omega_a q_a - D_a)^2 / 2, so by at most
    sum_a |omega_a q_a - D_a| bD_a + bD_a^2 / 2."""
    mo = w["modes"]
    R, _, _ = _centres(w, r)
    W = mo.lam * (mo.omega * obs["q"] - obs["D"])
    bD, _ = bounds(mo, R, M, W)
    return float(np.sum(np.abs(mo.omega * obs["q"] - obs["D"]) * bD + 0.5 * bD ** 2))


def test_steps_within_bound_and_track_fp64(P):
    """Ten steps against the FP64 moving-position path (which matches the oracle to 1e-9): momenta
    within twice the accumulated force bound (steps x dt x the largest force bound), the total
    energy within five times what the D bound allows at the start and at the end; after the steps
    D, E and G are within their bounds at the new centres of mass."""
    steps = 10
    w = _workload()
    a = _ctx(P, w)
    b = _ctx(P, w, precision=2)
    bF = _check_eval(b, w, w["system"].r, "moving c4 300 cells, step 0")
    tol_e = _energy_tol(w, b.cavmd_observables(), b.cavmd_get_eval()["M"], w["system"].r)
    a.cavmd_step(steps)
    b.cavmd_step(steps)
    sa, sb = a.cavmd_get_state(), b.cavmd_get_state()
    dt = w["options"]["dt"]
    tol_p = 2.0 * steps * dt * bF.max() + 1e-12 * np.abs(sa["p"]).max()
    np.testing.assert_allclose(sb["p"], sa["p"], rtol=0, atol=tol_p)
    ob = b.cavmd_observables()
    tol_e += _energy_tol(w, ob, b.cavmd_get_eval()["M"], sb["r"])
    assert abs(ob["e_total"] - a.cavmd_observables()["e_total"]) <= 5.0 * tol_e
    print(f"\nmoving c4 300 cells, {steps} steps: max |dp| / tol {np.abs(sb['p'] - sa['p']).max() / tol_p:.3f}, "
          f"|de| / tol {abs(ob['e_total'] - a.cavmd_observables()['e_total']) / (5 * tol_e):.3f}")
    _check_eval(b, w, sb["r"], f"moving c4 300 cells, step {steps}")


def test_graph_replay_is_bitwise_identical(P):
    w = _workload(n=200)
    a = _ctx(P, w, precision=2, graph_chunk=0)
    b = _ctx(P, w, precision=2, graph_chunk=4)
    a.cavmd_step(9)
    b.cavmd_step(9)
    sa, sb = a.cavmd_get_state(), b.cavmd_get_state()
    for k in ("r", "p", "q", "pq"):
        assert np.array_equal(sa[k], sb[k]), k


def test_full_size_c5_moving(P):
    """262,144 waters x 8192 modes (the largest configuration) with moving mode positions and the
    optical grid as generated: two steps, then every D_a, every cell's field and gradient against
    the plain FP64 contractions at the new centres of mass, within the bounds."""
    w = cs.make_workload("c5")
    ctx = _ctx(P, w, precision=2, photon_init=0)
    ctx.cavmd_step(2)
    st = ctx.cavmd_get_state()
    mo = w["modes"]
    R, mass, off = _centres(w, st["r"])
    ev = ctx.cavmd_get_eval()
    obs = ctx.cavmd_observables()
    M = ev["M"]
    W = mo.lam * (mo.omega * obs["q"] - obs["D"])
    D_ref, E_ref = direct_forward_and_field(mo, R, M, W)
    G_ref = direct_gradient(mo, R, W)
    bD, bE = bounds(mo, R, M, W)
    bGx, bGy = grad_bounds(mo, R, W)
    assert np.all(np.abs(obs["D"] - D_ref) <= bD + 1e-300)
    cell = np.repeat(np.arange(len(off) - 1), np.diff(off))
    mt = np.add.reduceat(mass, off[:-1])
    wm = (mass / mt[cell] * M[cell])[:, None]
    F_ref = ev["F_dftb"] + E_ref[cell][:, None] * ev["b"] + wm * G_ref[cell]
    bG = np.stack([bGx, bGy, np.zeros_like(bGx)], 1)
    bF = bE[cell][:, None] * np.abs(ev["b"]) + np.abs(wm) * bG[cell] + 1e-12
    assert np.all(np.abs(ev["F_total"] - F_ref) <= bF)
    live = bD > 0
    print(f"\nc5 moving full size: max |dD| / bound {np.max(np.abs(obs['D'] - D_ref)[live] / bD[live]):.3f} over "
          f"{mo.n_modes} modes, max |dF| / bound {np.max(np.abs(ev['F_total'] - F_ref) / bF):.3f}")


def test_clusters_within_bound(P):
    """Clusters of one to eight waters (the persistent cluster kernel, config 3's composition) with
    moving mode positions on the tensor cores: the initial evaluation and three steps later, with
    the grid's wave vectors scaled twofold (the position term is over 1000x the bound at the start;
    after three steps the photons have moved and it is checked at 10x)."""
    w = _workload("c3", n=40, scale=2.0)
    ctx = _ctx(P, w, precision=2, graph_chunk=0)
    _check_eval(ctx, w, w["system"].r, "moving c3 40 clusters, initial")
    ctx.cavmd_step(3)
    _check_eval(ctx, w, ctx.cavmd_get_state()["r"], "moving c3 40 clusters, step 3", margin=10.0)
