"""Water clusters (H2O)_n, n = 1..8 (6 to 48 orbitals), through the persistent cluster kernel,
against the FP64 oracle on the same seeded inputs.

Tolerances: those of the water parity tests (forces 1e-9 relative to the largest force, Mulliken
populations, dipoles and cell energies 1e-10 absolute), which still hold for 48 x 48 problems:
both sides converge the charges to a residual below 1e-12 and the FP64 rounding of the 48-orbital
linear algebra stays near 1e-13 (condition numbers of S below 1e2 for these clusters).
"""
import numpy as np
import pytest

import cavmd_synth as cs
from oracle import cavity as OC

from bf16x3 import bounds, direct_forward_and_field

pytestmark = pytest.mark.gpu

F_REL, Q_ABS, E_ABS = 1e-9, 1e-10, 1e-10
B_ABS = 5e-8


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


def _oracle(w, **kw):
    sy, mo, pa = w["system"], w["modes"], w["params"]
    mat = OC.DFTBMatter(pa, sy, **kw)
    md = OC.CavityMD(mat, sy.r, sy.p, mo.k, mo.omega, mo.lam, mo.phi, sy.R_ref, w["options"]["dt"])
    return mat, md


def _sizes(w):
    return np.diff(w["system"].cell_offset) // 3


def _check_eval(ev, mat, md):
    ref = md.out
    fs = np.abs(ref["F"]).max()
    np.testing.assert_allclose(ev["F_dftb"], ref["F"], rtol=0, atol=F_REL * fs)
    np.testing.assert_allclose(ev["q_pop"], mat.q, rtol=0, atol=Q_ABS)
    np.testing.assert_allclose(ev["M"], ref["M"], rtol=0, atol=Q_ABS)
    np.testing.assert_allclose(ev["b"], ref["b"], rtol=0, atol=Q_ABS)
    np.testing.assert_allclose(ev["E_cell"], ref["E"], rtol=0, atol=E_ABS)


def test_cluster_batch_initial_evaluation(P):
    """40 clusters: 15 of more than 32 orbitals (a block each) and 25 smaller ones (a warp each,
    the last block with one idle warp)."""
    w = cs.make_workload("c3", n_cells=40, n_modes=64)
    sz = _sizes(w)
    assert (6 * sz > 32).sum() == 15 and (6 * sz <= 32).sum() % 2 == 1 and sz.max() == 8 and sz.min() == 1
    ctx = _ctx(P, w)
    mat, md = _oracle(w)
    ev = ctx.cavmd_get_eval()
    _check_eval(ev, mat, md)
    fs = np.abs(md.F).max()
    np.testing.assert_allclose(ev["F_total"], md.F, rtol=0, atol=F_REL * fs)
    # neutral cells: populations sum to the valence electrons of each cluster
    cell = np.repeat(np.arange(len(sz)), 3 * sz)
    np.testing.assert_allclose(np.bincount(cell, ev["q_pop"]), 8.0 * sz, rtol=0, atol=1e-11)
    obs = ctx.cavmd_observables()
    e = md.energies()
    for k, key in (("kinetic", "e_kin"), ("dftb", "e_dftb"), ("photon", "e_photon"),
                   ("coupling", "e_coupling"), ("dse", "e_dse")):
        np.testing.assert_allclose(obs[key], e[k], rtol=1e-11, atol=1e-12)


def test_cluster_trajectory(P):
    w = cs.make_workload("c3", n_cells=24, n_modes=36)
    ctx = _ctx(P, w, graph_chunk=0)
    mat, md = _oracle(w)
    x0 = w["system"].r.copy()
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
    _check_eval(ctx.cavmd_get_eval(), mat, md)


def test_cluster_born_central(P):
    """Central finite-difference dipole derivatives of clusters: 6 displaced copies per atom, each
    a queue item of its own size class."""
    w = cs.make_workload("c3", n_cells=10, n_modes=16)
    ctx = _ctx(P, w, charge_model=2, born_interval=1, fd_step=1e-3)
    mat, md = _oracle(w, charge_model="born_central", born_interval=1, fd_step=1e-3)
    ev = ctx.cavmd_get_eval()
    # the lever of a cluster dipole is up to about 8 bohr: 4x the water bound
    np.testing.assert_allclose(ev["b"], md.out["b"], rtol=0, atol=4 * B_ABS)
    fs = np.abs(md.out["F"]).max()
    np.testing.assert_allclose(ev["F_dftb"], md.out["F"], rtol=0, atol=F_REL * fs)


def test_cluster_graph_replay_and_determinism(P):
    """The work queue hands items to blocks in a run-dependent order, but every item is computed
    by a fixed sequence of operations: results are bitwise reproducible and graph replay equals
    direct launches."""
    w = cs.make_workload("c3", n_cells=60, n_modes=64)
    a = _ctx(P, w, graph_chunk=0)
    b = _ctx(P, w, graph_chunk=3)
    c = _ctx(P, w, graph_chunk=0)
    for x in (a, b, c):
        x.cavmd_step(7)
    sa, sb, sc = a.cavmd_get_state(), b.cavmd_get_state(), c.cavmd_get_state()
    for k in ("r", "p", "q", "pq"):
        assert np.array_equal(sa[k], sb[k]), k
        assert np.array_equal(sa[k], sc[k]), k


def test_cluster_mixed_precision_coupling(P):
    """The workload as specified: clusters with the tensor-core coupling on the 2D mode grid; the
    SCC part stays FP64 and matches the oracle, the coupling meets the BF16x3 bound."""
    w = cs.make_workload("c3", n_cells=48, n_modes=256)
    ctx = _ctx(P, w, precision=2)
    mat, md = _oracle(w)
    ev = ctx.cavmd_get_eval()
    fs = np.abs(md.out["F"]).max()
    np.testing.assert_allclose(ev["F_dftb"], md.out["F"], rtol=0, atol=F_REL * fs)
    np.testing.assert_allclose(ev["M"], md.out["M"], rtol=0, atol=Q_ABS)
    obs = ctx.cavmd_observables()
    mo = w["modes"]
    own = OC.forward(md.U, mo.lam, ev["M"])
    assert np.all(np.abs(obs["D"] - own) <= bounds(mo, w["system"].R_ref, ev["M"], np.zeros(mo.n_modes))[0] + 1e-300)


def test_mixed_waters_and_clusters_in_one_batch(P):
    """Monomers and clusters together (monomers then take the cluster kernel too): a water cell's
    result does not depend on the kernel that evaluated it beyond FP64 rounding."""
    w1 = cs.make_workload("c3", n_cells=30, n_modes=16)
    ctx = _ctx(P, w1)
    ev = ctx.cavmd_get_eval()
    sz = _sizes(w1)
    mono = np.where(sz == 1)[0]
    assert len(mono) >= 2
    off = w1["system"].cell_offset
    idx = np.concatenate([np.arange(off[c], off[c + 1]) for c in mono])
    sub = cs.System(species=w1["system"].species[idx], cell_offset=np.arange(len(mono) + 1, dtype=np.int32) * 3,
                    r=w1["system"].r[idx], p=w1["system"].p[idx], R_ref=w1["system"].R_ref[mono])
    w2 = dict(w1, system=sub)
    ev2 = _ctx(P, w2).cavmd_get_eval()          # all cells are waters: the lane-group kernel
    np.testing.assert_allclose(ev["F_dftb"][idx], ev2["F_dftb"], rtol=0, atol=1e-11 * np.abs(ev2["F_dftb"]).max())
    np.testing.assert_allclose(ev["q_pop"][idx], ev2["q_pop"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(ev["E_cell"][mono], ev2["E_cell"], rtol=0, atol=1e-12)


def test_full_size_c3_sampled(P):
    """65,536 clusters x 4096 modes with the tensor-core coupling, the benchmark configuration:
    sampled clusters of every size against the oracle, charge sums of all clusters, all 4096 D_a
    and every cluster's field against the plain contraction of the GPU's own dipoles within the
    BF16x3 bound (tests/bf16x3.py), one step."""
    w = cs.make_workload("c3")
    sy = w["system"]
    ctx = _ctx(P, w, precision=2)
    ev = ctx.cavmd_get_eval()
    sz = _sizes(w)
    off = sy.cell_offset
    cell = np.repeat(np.arange(len(sz)), 3 * sz)
    np.testing.assert_allclose(np.bincount(cell, ev["q_pop"]), 8.0 * sz, rtol=0, atol=1e-10)
    rng = np.random.default_rng(0)
    pick = np.concatenate([rng.choice(np.where(sz == n)[0], 2, replace=False) for n in range(1, 9)])
    idx = np.concatenate([np.arange(off[c], off[c + 1]) for c in pick])
    sub = cs.System(species=sy.species[idx], cell_offset=np.concatenate([[0], np.cumsum(3 * sz[pick])]).astype(np.int32),
                    r=sy.r[idx], p=sy.p[idx], R_ref=sy.R_ref[pick])
    out = OC.DFTBMatter(w["params"], sub)(sub.r)
    fs = np.abs(out["F"]).max()
    np.testing.assert_allclose(ev["F_dftb"][idx], out["F"], rtol=0, atol=F_REL * fs)
    np.testing.assert_allclose(ev["M"][pick], out["M"], rtol=0, atol=Q_ABS)
    np.testing.assert_allclose(ev["E_cell"][pick], out["E"], rtol=0, atol=E_ABS)
    mo = w["modes"]
    obs = ctx.cavmd_observables()
    W = mo.lam * (mo.omega * obs["q"] - obs["D"])
    D_ref, E_ref = direct_forward_and_field(mo, sy.R_ref, ev["M"], W)
    bD, bE = bounds(mo, sy.R_ref, ev["M"], W)
    assert np.all(np.abs(obs["D"] - D_ref) <= bD + 1e-300)
    F_ref = ev["F_dftb"] + E_ref[cell][:, None] * ev["b"]
    assert np.all(np.abs(ev["F_total"] - F_ref) <= bE[cell][:, None] * np.abs(ev["b"]) + 1e-12)
    ctx.cavmd_step(2)
    st = ctx.cavmd_get_state()
    assert np.all(np.isfinite(st["p"])) and st["step"] == 2
    it = ctx.cavmd_get_eval()["scc_iters"]
    assert it.max() < 40
