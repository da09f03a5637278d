"""Limits and degenerate cases of the GPU path.

  * Zero coupling (lambda = 0): the photons never move and the nuclei follow the bare
    velocity-Verlet SCC-DFTB trajectory (the oracle's bare integrator), one of the invariants the
    method fixes.
  * cavmd_step(0) changes nothing.
  * Config 5 at full size (262,144 waters, 8192 grid modes, BF16x3 coupling): sampled cells
    against the oracle, the charge sum of every cell, and every mode's D_a and every cell's field
    against the plain FP64 contraction within the derived BF16x3 bound (tests/bf16x3.py).
Tolerances: those of the other parity tests (trajectories 1e-9 times the step number of the
largest value; populations 1e-10; forces 1e-9 of the largest force)."""
import numpy as np
import pytest

import cavmd_synth as cs
from oracle import cavity as OC

from bf16x3 import bounds, direct_forward_and_field

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


def _ctx(P, w, **opt):
    o = P.default_options()
    for k, v in opt.items():
        setattr(o, k, v)
    return P.Context(w["system"], w["params"], w["modes"], o)


def test_zero_coupling_gives_bare_dftb_dynamics(P):
    w = cs.make_workload("c2", n_cells=23, n_modes=32)
    mo = w["modes"]
    w = dict(w, modes=cs.Modes(k=mo.k, omega=mo.omega, lam=np.zeros_like(mo.lam), phi=mo.phi))
    sy, pa = w["system"], w["params"]
    dt = w["options"]["dt"]
    ctx = _ctx(P, w, graph_chunk=0)
    bare = OC.DFTBMatter(pa, sy)
    r, p = sy.r.copy(), sy.p.copy()
    F = bare(r)["F"]
    m = bare.mass[:, None]
    x0 = r.copy()
    for s in range(5):
        ctx.cavmd_step(1)
        p = p + 0.5 * dt * F
        r = r + dt * p / m
        F = bare(r)["F"]
        p = p + 0.5 * dt * F
        st = ctx.cavmd_get_state()
        tol = 1e-9 * (1 + s)
        np.testing.assert_allclose(st["r"] - x0, r - x0, rtol=0, atol=tol * np.abs(r - x0).max())
        np.testing.assert_allclose(st["p"], p, rtol=0, atol=tol * np.abs(p).max())
        assert np.all(st["q"] == 0.0) and np.all(st["pq"] == 0.0)
    obs = ctx.cavmd_observables()
    assert obs["e_photon"] == 0.0 and obs["e_coupling"] == 0.0 and obs["e_dse"] == 0.0


def test_zero_steps_change_nothing(P):
    w = cs.make_workload("c2", n_cells=11, n_modes=16)
    ctx = _ctx(P, w)
    ctx.cavmd_step(3)
    a = ctx.cavmd_get_state()
    ctx.cavmd_step(0)
    b = ctx.cavmd_get_state()
    for k in ("r", "p", "q", "pq"):
        assert np.array_equal(a[k], b[k]), k
    assert a["step"] == b["step"] == 3


def test_full_size_c5_sampled(P):
    """262,144 waters x 8192 modes with the tensor-core coupling (the largest configuration):
    40 sampled cells against the oracle, the charge sum of every cell, all 8192 D_a and all
    262,144 fields against the plain contraction of the GPU's own dipoles within the BF16x3 bound,
    and one step."""
    w = cs.make_workload("c5")
    sy, mo, pa = w["system"], w["modes"], w["params"]
    ctx = _ctx(P, w, precision=2)
    ev = ctx.cavmd_get_eval()
    np.testing.assert_allclose(ev["q_pop"].reshape(-1, 3).sum(1), 8.0, rtol=0, atol=1e-11)
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(sy.n_cells, 40, replace=False))
    idx = (3 * pick[:, None] + np.arange(3)[None, :]).ravel()
    sub = cs.System(species=sy.species[idx], cell_offset=np.arange(len(pick) + 1, dtype=np.int32) * 3,
                    r=sy.r[idx], p=sy.p[idx], R_ref=sy.R_ref[pick])
    mat = OC.DFTBMatter(pa, sub)
    out = mat(sub.r)
    np.testing.assert_allclose(ev["F_dftb"][idx], out["F"], rtol=0, atol=1e-9 * np.abs(out["F"]).max())
    np.testing.assert_allclose(ev["q_pop"][idx], mat.q, rtol=0, atol=1e-10)
    np.testing.assert_allclose(ev["M"][pick], out["M"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(ev["E_cell"][pick], out["E"], rtol=0, atol=1e-10)
    # every D_a and every cell's field E_n against the plain FP64 contraction of the GPU's own dipoles,
    # within the BF16x3 bound (tests/bf16x3.py); E_n is seen through F_total = F_dftb + E_n b_j
    obs = ctx.cavmd_observables()
    W = mo.lam * (mo.omega * obs["q"] - obs["D"])
    D_ref, E_ref = direct_forward_and_field(mo, sy.R_ref, ev["M"], W)
    bD, bE = bounds(mo, sy.R_ref, ev["M"], W)
    assert np.all(np.abs(obs["D"] - D_ref) <= bD + 1e-300)
    cell = np.repeat(np.arange(sy.n_cells), 3)
    F_ref = ev["F_dftb"] + E_ref[cell][:, None] * ev["b"]
    assert np.all(np.abs(ev["F_total"] - F_ref) <= bE[cell][:, None] * np.abs(ev["b"]) + 1e-12)
    live = bD > 0                                   # the k = 0 sin mode has lambda = 0
    print(f"\nc5 full size: max |dD| / bound {np.max(np.abs(obs['D'] - D_ref)[live] / bD[live]):.3f} over "
          f"{mo.n_modes} modes")
    ctx.cavmd_step(1)
    st = ctx.cavmd_get_state()
    assert st["step"] == 1 and np.all(np.isfinite(st["p"])) and np.all(np.isfinite(st["q"]))
