"""The paper's step order (splitting = CAVMD_SPLIT_PAPER): half-kicks with the instantaneous
coupling force (Eq. pj1), drift, evaluation, half-kick, then the free rotation of every mode by
omega dt (Eq. qknk, Step 3), against the FP64 oracle on the same seeded inputs.

Two references:
  * the oracle's k-space integrator with the same order (oracle/cavity.py, splitting="paper"),
    for general modes;
  * the oracle's real-space / reciprocal-space Steps 1-4 (oracle/paper_scheme.py): real-space
    photon coordinates q_n per box, the local coupling eta q_n mu_n + eta^2 mu_n^2 / (2 omega_0^2),
    a DFT to k-space, the rotation, and the DFT back. With cells on a line lattice, modes on its
    DFT grid and a flat dispersion the two are the same dynamics, so the GPU must reproduce the
    paper's own scheme.
Tolerances are those of the other trajectory tests: 1e-9 (times the step number) of the largest
displacement, momentum and photon coordinate."""
import numpy as np
import pytest

import cavmd_synth as cs
from oracle import cavity as OC
from oracle import paper_scheme as PS

pytestmark = pytest.mark.gpu
PAPER = 2


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
    o.splitting = PAPER
    for k, v in opt.items():
        setattr(o, k, v)
    return P.Context(w["system"], w["params"], w["modes"], o)


def _check(st, md, x0, s):
    tol = 1e-9 * (1 + s)
    dr = md.r - x0
    np.testing.assert_allclose(st["r"] - x0, dr, rtol=0, atol=tol * np.abs(dr).max())
    np.testing.assert_allclose(st["p"], md.p, rtol=0, atol=tol * np.abs(md.p).max())
    np.testing.assert_allclose(st["q"], md.q, rtol=0, atol=tol * np.abs(md.q).max())
    np.testing.assert_allclose(st["pq"], md.pq, rtol=0, atol=tol * np.abs(md.pq).max() + 1e-15)


@pytest.mark.parametrize("name,n,steps", [("c1", None, 20), ("c2", 37, 6)])
def test_trajectory_matches_oracle_paper_order(P, name, n, steps):
    w = cs.make_workload(name, n_cells=n)
    sy, mo, pa = w["system"], w["modes"], w["params"]
    ctx = _ctx(P, w, graph_chunk=0)
    md = OC.CavityMD(OC.DFTBMatter(pa, sy), sy.r, sy.p, mo.k, mo.omega, mo.lam, mo.phi, sy.R_ref,
                     w["options"]["dt"], splitting="paper")
    x0 = sy.r.copy()
    for s in range(steps):
        ctx.cavmd_step(1)
        md.step()
        _check(ctx.cavmd_get_state(), md, x0, s)
        np.testing.assert_allclose(ctx.cavmd_observables()["e_total"], md.energies()["total"], rtol=1e-11)
    # the order matters: the exact half-flows give another trajectory
    ex = OC.CavityMD(OC.DFTBMatter(pa, sy), sy.r, sy.p, mo.k, mo.omega, mo.lam, mo.phi, sy.R_ref, w["options"]["dt"])
    for _ in range(steps):
        ex.step()
    assert np.abs(ex.q - md.q).max() > 1e3 * 1e-9 * steps * np.abs(md.q).max()


def test_reproduces_the_papers_real_space_steps(P):
    """8 waters on a line lattice (a = 12 bohr), the 8 modes of its DFT grid with a flat
    dispersion: the GPU's k-space steps against the oracle's real-space Steps 1-4."""
    params = cs.load_water_params()
    N, a, w0, g0 = 8, 12.0, 0.012, 0.002
    cent = np.stack([np.arange(N) * a, np.zeros(N), np.zeros(N)], 1)
    pos = cs.water_batch(np.random.default_rng(2), cent)
    sy = cs.systems._water_system(pos, cent)
    sy.p = cs.mb_momenta(np.random.default_rng(3), sy, 300.0)
    ks, ph, lam = [], [], []
    for j in range(N // 2 + 1):
        for s in ((0,) if j in (0, N // 2) else (0, 1)):
            ks.append(2 * np.pi * j / (N * a))
            ph.append(0.0 if s == 0 else -np.pi / 2)
            lam.append(np.sqrt(2) * g0 if j in (0, N // 2) else 2 * g0)
    K = np.zeros((N, 3))
    K[:, 0] = ks
    modes = cs.Modes(k=K, omega=np.full(N, w0), lam=np.array(lam), phi=np.array(ph))
    dt = 0.5 * 41.341373335
    w = {"system": sy, "modes": modes, "params": params}
    ctx = _ctx(P, w, dt=dt, graph_chunk=0)
    ps = PS.PaperRealSpaceMD(OC.DFTBMatter(params, sy), sy.r, sy.p, cent[:, 0],
                             2 * np.pi * np.arange(N) / (N * a), np.full(N, w0), g0, w0, dt)
    x0 = sy.r.copy()
    for s in range(6):
        ctx.cavmd_step(1)
        ps.step()
        st = ctx.cavmd_get_state()
        tol = 1e-9 * (1 + s)
        dr = ps.r - x0
        np.testing.assert_allclose(st["r"] - x0, dr, rtol=0, atol=tol * np.abs(dr).max())
        np.testing.assert_allclose(st["p"], ps.p, rtol=0, atol=tol * np.abs(ps.p).max())
        np.testing.assert_allclose(ctx.cavmd_observables()["e_total"], ps.energies()["total"], rtol=1e-11)


def test_graph_replay_is_bitwise_identical(P):
    w = cs.make_workload("c2", n_cells=24, n_modes=32)
    a = _ctx(P, w, graph_chunk=0)
    b = _ctx(P, w, graph_chunk=4)
    a.cavmd_step(9)
    b.cavmd_step(9)
    sa, sb = a.cavmd_get_state(), b.cavmd_get_state()
    for k in ("r", "p", "q", "pq"):
        assert np.array_equal(sa[k], sb[k]), k


def test_mixed_coupling_tracks_fp64(P):
    """The BF16x3 tensor-core coupling in the paper's order: ten steps stay within the bounds of
    the exact-half-flow mixed test (1e-6 of the largest momentum, 1e-4 of the largest photon
    coordinate, 1e-9 relative in the total energy). The kick-then-rotate order is stable only for
    omega dt below about 1, so the modes are an 8 x 8 grid near the cavity fundamental
    (omega ~ 0.01 Hartree, omega dt ~ 0.2), not config 4's grid (omega dt up to 1830)."""
    w = cs.make_workload("c4", n_cells=256)
    L = np.pi * cs.units.C_LIGHT / 0.01
    w = dict(w, modes=cs.grid_modes(8, 8, 5e-6, 5e-6, L, 0.002))
    assert w["modes"].omega.max() * w["options"]["dt"] < 0.3
    a = _ctx(P, w, precision=0)
    b = _ctx(P, w, precision=2)
    a.cavmd_step(10)
    b.cavmd_step(10)
    sa, sb = a.cavmd_get_state(), b.cavmd_get_state()
    np.testing.assert_allclose(sb["p"], sa["p"], rtol=0, atol=1e-6 * np.abs(sa["p"]).max())
    np.testing.assert_allclose(sb["q"], sa["q"], rtol=0, atol=1e-4 * np.abs(sa["q"]).max())
    np.testing.assert_allclose(b.cavmd_observables()["e_total"], a.cavmd_observables()["e_total"], rtol=1e-9)


@pytest.mark.parametrize("name,n,steps,prec", [("c1", None, 20, 0), ("c2", 37, 6, 0), ("c4", 64, 6, 0)])
def test_strang_splitting_matches_oracle(P, name, n, steps, prec):
    """splitting = CAVMD_SPLIT_STRANG: kick(dt/2), drift and free rotation of every mode over dt,
    evaluation, kick(dt/2), against the oracle's splitting="strang" (both the fixed order and the
    energy record); the rotation inside the step makes it another trajectory than the paper's order."""
    w = cs.make_workload(name, n_cells=n)
    sy, mo, pa = w["system"], w["modes"], w["params"]
    ctx = _ctx(P, w, graph_chunk=0, splitting=1, precision=prec)
    md = OC.CavityMD(OC.DFTBMatter(pa, sy), sy.r, sy.p, mo.k, mo.omega, mo.lam, mo.phi, sy.R_ref,
                     w["options"]["dt"], splitting="strang")
    x0 = sy.r.copy()
    for s in range(steps):
        ctx.cavmd_step(1)
        md.step()
        _check(ctx.cavmd_get_state(), md, x0, s)
        np.testing.assert_allclose(ctx.cavmd_observables()["e_total"], md.energies()["total"], rtol=1e-11)
    po = OC.CavityMD(OC.DFTBMatter(pa, sy), sy.r, sy.p, mo.k, mo.omega, mo.lam, mo.phi, sy.R_ref,
                     w["options"]["dt"], splitting="paper")
    for _ in range(steps):
        po.step()
    assert np.abs(po.q - md.q).max() > 1e3 * 1e-9 * steps * np.abs(md.q).max()


def test_strang_graph_replay_is_bitwise_direct(P):
    w = cs.make_workload("c2", n_cells=21, n_modes=32)
    a = _ctx(P, w, graph_chunk=0, splitting=1)
    b = _ctx(P, w, graph_chunk=5, splitting=1)
    a.cavmd_step(12)
    b.cavmd_step(12)
    sa, sb = a.cavmd_get_state(), b.cavmd_get_state()
    for k in ("r", "p", "q", "pq"):
        assert np.array_equal(sa[k], sb[k]), k


def _lattice_case(N=8, a=12.0, w0=0.012, g0=0.002, disp=False):
    """N waters on a line lattice (spacing a) and the real modes of its wave-vector grid; with
    `disp` the dispersion omega_k = omega_0 sqrt(1 + 3 (k / k_max)^2) rises to twice omega_0."""
    params = cs.load_water_params()
    cent = np.stack([np.arange(N) * a, np.zeros(N), np.zeros(N)], 1)
    pos = cs.water_batch(np.random.default_rng(2), cent)
    sy = cs.systems._water_system(pos, cent)
    sy.p = cs.mb_momenta(np.random.default_rng(3), sy, 300.0)
    kmax = np.pi / a

    def om(k):
        return w0 * np.sqrt(1.0 + 3.0 * (k / kmax) ** 2) if disp else w0 + 0.0 * k

    ks, ph, lam = [], [], []
    for j in range(N // 2 + 1):
        for s in ((0,) if j in (0, N // 2) else (0, 1)):
            ks.append(2 * np.pi * j / (N * a))
            ph.append(0.0 if s == 0 else -np.pi / 2)
            lam.append(np.sqrt(2) * g0 if j in (0, N // 2) else 2 * g0)
    K = np.zeros((N, 3))
    K[:, 0] = ks
    modes = cs.Modes(k=K, omega=om(np.array(ks)), lam=np.array(lam), phi=np.array(ph))
    kc = 2 * np.pi * np.arange(N) / (N * a)
    kc_fold = np.minimum(kc, 2 * np.pi / a - kc)           # k_j and k_{N-j} share omega
    return params, cent, sy, modes, kc, om(kc_fold)


@pytest.mark.parametrize("disp", [False, True])
def test_real_space_scheme_matches_the_papers_steps(P, disp):
    """splitting = CAVMD_SPLIT_REAL_SPACE, the paper's scheme as printed (Eq. hlm3 with Steps 1-4):
    real-space photon coordinates per cell, the local coupling, the transforms and the rotation of
    every mode with its own frequency, against oracle/paper_scheme.py; with a flat dispersion and
    with one that rises to twice omega_0 (where the scheme is the paper's approximation, not the
    exact k-space dynamics)."""
    N, a, w0, g0 = 8, 12.0, 0.012, 0.002
    params, cent, sy, modes, kc, wk = _lattice_case(N, a, w0, g0, disp)
    dt = 0.5 * 41.341373335
    w = {"system": sy, "modes": modes, "params": params}
    ctx = _ctx(P, w, dt=dt, graph_chunk=0, splitting=3, real_space_g0=g0, real_space_omega0=w0)
    ps = PS.PaperRealSpaceMD(OC.DFTBMatter(params, sy), sy.r, sy.p, cent[:, 0], kc, wk, g0, w0, dt)
    st = ctx.cavmd_get_state()
    np.testing.assert_allclose(st["q"], ps.qn, rtol=0, atol=1e-12 * np.abs(ps.qn).max())   # Step 0
    x0 = sy.r.copy()
    for s in range(6):
        ctx.cavmd_step(1)
        ps.step()
        st = ctx.cavmd_get_state()
        tol = 1e-9 * (1 + s)
        dr = ps.r - x0
        np.testing.assert_allclose(st["r"] - x0, dr, rtol=0, atol=tol * np.abs(dr).max())
        np.testing.assert_allclose(st["p"], ps.p, rtol=0, atol=tol * np.abs(ps.p).max())
        np.testing.assert_allclose(st["q"], ps.qn, rtol=0, atol=tol * np.abs(ps.qn).max())
        np.testing.assert_allclose(st["pq"], ps.pn, rtol=0, atol=tol * np.abs(ps.pn).max())
        if not disp:   # the oracle's local photon energy is the free energy of a flat dispersion
            np.testing.assert_allclose(ctx.cavmd_observables()["e_total"], ps.energies()["total"], rtol=1e-11)
    if disp:   # the dispersion changes the photon trajectory
        flat = PS.PaperRealSpaceMD(OC.DFTBMatter(params, sy), sy.r, sy.p, cent[:, 0], kc, np.full(N, w0), g0, w0, dt)
        for _ in range(6):
            flat.step()
        assert np.abs(flat.qn - ps.qn).max() > 1e3 * 6e-9 * np.abs(ps.qn).max()


def test_real_space_scheme_graph_and_resume(P):
    N, a, w0, g0 = 8, 12.0, 0.012, 0.002
    params, cent, sy, modes, kc, wk = _lattice_case(N, a, w0, g0, True)
    w = {"system": sy, "modes": modes, "params": params}
    kw = dict(splitting=3, real_space_g0=g0, real_space_omega0=w0)
    x = _ctx(P, w, graph_chunk=0, **kw)
    y = _ctx(P, w, graph_chunk=4, **kw)
    x.cavmd_step(9)
    y.cavmd_step(9)
    sx, sy_ = x.cavmd_get_state(), y.cavmd_get_state()
    for k in ("r", "p", "q", "pq"):
        assert np.array_equal(sx[k], sy_[k]), k
    # a run resumed from a saved state follows the original one (the re-evaluation at the saved
    # positions converges the charges from a cold start, so to the trajectory tolerance)
    z = _ctx(P, w, graph_chunk=0, **kw)
    z.cavmd_set_state(sx)
    assert z.cavmd_get_state()["step"] == 9
    x.cavmd_step(3)
    z.cavmd_step(3)
    a_, b_ = x.cavmd_get_state(), z.cavmd_get_state()
    for k in ("r", "p", "q", "pq"):
        np.testing.assert_allclose(b_[k], a_[k], rtol=0, atol=1e-9 * np.abs(a_[k]).max() + 1e-15)
