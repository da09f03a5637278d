"""Pins of the SCC-DFTB oracle against things other than itself: closed forms (Gaussian-orbital
overlaps, the H2 two-level problem), a library generalised eigensolver, exact invariances,
finite differences of the energy, and the fixed-point property of the charges."""
import numpy as np
import pytest
import scipy.linalg

import cavmd_synth as cs
from cavmd_synth.params import ELEM_H, ELEM_O, draw_sk_params
from oracle import dftb as D

WATER = [ELEM_O, ELEM_H, ELEM_H]


@pytest.fixture(scope="module")
def params():
    return cs.load_water_params()


def _rand_unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


# ------------------------------------------------------------------------ Slater-Koster rotation

def _gto_ss(a, b, R):
    """<g_a(r)|g_b(r - R)> for unnormalised s Gaussians exp(-a r^2) (Gaussian product theorem)."""
    p = a + b
    return (np.pi / p) ** 1.5 * np.exp(-a * b / p * np.dot(R, R))


def _gto_block(a, b, A, B):
    """Exact overlaps between {s, x, y, z} Gaussians on A (exponent a) and on B (exponent b):
    with P = (a A + b B)/(a + b): <s|s> = S0, <s_A|p_B,i> = (P - B)_i S0,
    <p_A,i|s_B> = (P - A)_i S0, <p_A,i|p_B,j> = [(P - A)_i (P - B)_j + delta_ij / 2(a+b)] S0."""
    S0 = _gto_ss(a, b, B - A)
    P = (a * A + b * B) / (a + b)
    PA, PB = P - A, P - B
    blk = np.zeros((4, 4))
    blk[0, 0] = S0
    blk[0, 1:] = PB * S0
    blk[1:, 0] = PA * S0
    blk[1:, 1:] = (np.outer(PA, PB) + np.eye(3) / (2 * (a + b))) * S0
    return blk


def test_sk_rotation_reproduces_gaussian_overlaps():
    """Radial integrals taken along z, rotated by the oracle's SK rules, must equal the exact
    overlap of Gaussian s/p orbitals for any bond direction: pins signs, indices, transposes."""
    rng = np.random.default_rng(5)
    a, b = 0.7, 0.45
    for r in (0.8, 1.9, 3.1):
        z = np.array([0.0, 0.0, r])
        ref = _gto_block(a, b, np.zeros(3), z)
        ref_ba = _gto_block(b, a, np.zeros(3), z)      # B's orbitals first, bond along +z
        vals = {"ss": np.array(ref[0, 0]), "sp": np.array(ref[0, 3]),
                # table entry with B first: s on B, p on A along the B -> A... taken with B first
                "ps": np.array(ref_ba[0, 3]),
                "pps": np.array(ref[3, 3]), "ppp": np.array(ref[1, 1])}
        for e in _rand_unit(rng, 6):
            blk = D.sk_block(vals, e[None], 4, 4)[0]
            direct = _gto_block(a, b, np.zeros(3), r * e)
            np.testing.assert_allclose(blk, direct, atol=1e-14, rtol=1e-12)


def test_sk_block_gradient_matches_finite_differences(params):
    rng = np.random.default_rng(6)
    h = 1e-6
    for ea, eb in ((ELEM_O, ELEM_O), (ELEM_O, ELEM_H), (ELEM_H, ELEM_O), (ELEM_H, ELEM_H)):
        na, nb = params.norb[ea], params.norb[eb]
        for dist in (1.7, 4.0, 11.4):                   # 11.4 lies inside the cutoff taper
            d = dist * _rand_unit(rng, 1)[0]
            for table in (params.h0, params.s):
                def blk(dv):
                    r = np.linalg.norm(dv)
                    v, _ = D._pair_integrals(table, params, ea, eb, np.array([r]))
                    return D.sk_block(v, (dv / r)[None], na, nb)[0]
                r = np.linalg.norm(d)
                v, dv = D._pair_integrals(table, params, ea, eb, np.array([r]))
                g = D.sk_block_grad(v, dv, (d / r)[None], np.array([r]), na, nb)[0]
                for k in range(3):
                    e = np.zeros(3)
                    e[k] = h
                    fd = (blk(d + e) - blk(d - e)) / (2 * h)
                    np.testing.assert_allclose(g[k], fd, atol=1e-9)


def test_radial_and_cutoff_values():
    par = (2.0, 1.5, 0.3, 0.1)
    r = np.array([1.0, 10.9, 11.5, 12.0, 12.5])
    v, dv = D.radial(par, r, 12.0, 1.0)
    plain = 2.0 * np.exp(-1.5 * r) * (1 + 0.3 * r + 0.1 * r * r)
    taper = np.array([1.0, 1.0, 0.5, 0.0, 0.0])        # cos taper: 1 below 11, 1/2 at 11.5, 0 past 12
    np.testing.assert_allclose(v, plain * taper, rtol=1e-14, atol=1e-300)
    h = 1e-6
    fd = (D.radial(par, r + h, 12.0, 1.0)[0] - D.radial(par, r - h, 12.0, 1.0)[0]) / (2 * h)
    np.testing.assert_allclose(dv[:4], fd[:4], rtol=1e-7, atol=1e-12)


# ------------------------------------------------------------------------ eigenproblem

def test_h2_closed_form(params):
    """H2 with s orbitals only: eps = (alpha +- beta)/(1 +- s) and dq = 0 by symmetry."""
    pos = np.array([[[0.0, 0.0, 0.0], [0.3, -0.4, 1.3]]])
    lay = D.Layout(params, [ELEM_H, ELEM_H])
    H0, S = D.build_h0_s(params, lay, pos)
    alpha, beta, s = H0[0, 0, 0], H0[0, 0, 1], S[0, 0, 1]
    eps, C = D.gen_eigh(H0, S)
    expect = np.sort([(alpha + beta) / (1 + s), (alpha - beta) / (1 - s)])
    np.testing.assert_allclose(eps[0], expect, rtol=1e-14)
    out = D.dftb(params, [ELEM_H, ELEM_H], pos)
    np.testing.assert_allclose(out["q"], 1.0, atol=1e-13)
    # closed-form energy: 2 * bonding level (dq = 0, no second-order term) + repulsion
    erep, _ = D.e_rep(params, lay, pos)
    np.testing.assert_allclose(out["E"], 2 * expect[0] + erep, rtol=1e-13)


def test_generalised_eigensolver_against_scipy():
    rng = np.random.default_rng(7)
    for n in (6, 12, 48):
        A = rng.normal(size=(3, n, n))
        H = A + np.swapaxes(A, -1, -2)
        Bm = rng.normal(size=(3, n, n)) * 0.3
        S = np.eye(n) + Bm @ np.swapaxes(Bm, -1, -2) / n
        e, C = D.gen_eigh(H, S)
        for b in range(3):
            ref = scipy.linalg.eigh(H[b], S[b], eigvals_only=True)
            np.testing.assert_allclose(e[b], ref, rtol=1e-11, atol=1e-11)
            np.testing.assert_allclose(H[b] @ C[b] - S[b] @ C[b] * e[b], 0.0, atol=1e-11)
            np.testing.assert_allclose(C[b].T @ S[b] @ C[b], np.eye(n), atol=1e-12)


# ------------------------------------------------------------------------ SCC

def _waters(n=6, seed=11):
    rng = np.random.default_rng(seed)
    return cs.water_batch(rng, np.zeros((n, 3)), noise=0.08)


def test_mulliken_population_sum(params):
    out = D.dftb(params, WATER, _waters())
    np.testing.assert_allclose(out["q"].sum(-1), 8.0, atol=1e-12)


def test_scc_fixed_point(params):
    """The converged populations reproduce themselves through one more SCC map evaluation."""
    pos = _waters()
    lay = D.Layout(params, WATER)
    out = D.dftb(params, WATER, pos)
    H0, S = D.build_h0_s(params, lay, pos)
    gam = D.gamma_matrix(params, lay, pos)
    dq = out["q"] - lay.zval
    shift = np.einsum("bij,bj->bi", gam, dq)[:, lay.atom_of_orb]
    H = H0 + 0.5 * S * (shift[:, :, None] + shift[:, None, :])
    _, C = D.gen_eigh(H, S)
    Co = C[:, :, :4]
    q_map = D.mulliken(lay, 2 * Co @ np.swapaxes(Co, -1, -2), S)
    np.testing.assert_allclose(q_map, out["q"], atol=1e-12)


def test_klopman_ohno_limits(params):
    lay = D.Layout(params, WATER)
    pos = _waters(1)
    g = D.gamma_matrix(params, lay, pos)[0]
    np.testing.assert_allclose(np.diag(g), params.hubbard[lay.species], rtol=1e-15)
    far = pos.copy()
    far[0, 1] += np.array([1e6, 0, 0])
    gf = D.gamma_matrix(params, lay, far)[0]
    np.testing.assert_allclose(gf[0, 1] * np.linalg.norm(far[0, 1] - far[0, 0]), 1.0, rtol=1e-9)


def test_small_u_reduces_to_non_scc():
    """gamma -> 0 as U -> 0: the SCC result equals the plain (non-SCC) tight-binding solution."""
    p = cs.load_water_params()
    p.hubbard = np.array([1e-9, 1e-9])
    pos = _waters(3)
    out = D.dftb(p, WATER, pos)
    lay = D.Layout(p, WATER)
    H0, S = D.build_h0_s(p, lay, pos)
    for b in range(3):
        e, C = scipy.linalg.eigh(H0[b], S[b])
        P = 2 * C[:, :4] @ C[:, :4].T
        q = D.mulliken(lay, P[None], S[b][None])[0]
        np.testing.assert_allclose(out["q"][b], q, atol=1e-10)


def test_mixing_parameter_does_not_change_converged_result(params):
    pos = _waters(3)
    a = D.dftb(params, WATER, pos, beta=0.2)
    b = D.dftb(params, WATER, pos, beta=0.7)
    np.testing.assert_allclose(a["q"], b["q"], atol=1e-11)
    np.testing.assert_allclose(a["F"], b["F"], atol=1e-11)


# ------------------------------------------------------------------------ energy, forces, invariance

def _rigid(rng, pos):
    Rm = cs.systems.random_rotations(rng, 1)[0]
    return pos @ Rm.T + rng.normal(size=3) * 3.0, Rm


@pytest.mark.parametrize("nmol", [1, 3])
def test_rigid_motion_invariance(params, nmol):
    rng = np.random.default_rng(12)
    sys_ = cs.cluster_batch(rng, [nmol], np.zeros((1, 3)))
    pos = sys_.r[None]
    out = D.dftb(params, sys_.species, pos)
    moved, Rm = _rigid(rng, pos[0])
    out2 = D.dftb(params, sys_.species, moved[None])
    np.testing.assert_allclose(out2["E"], out["E"], rtol=1e-12)
    np.testing.assert_allclose(out2["eps"], out["eps"], atol=1e-12)
    np.testing.assert_allclose(out2["q"], out["q"], atol=1e-11)
    np.testing.assert_allclose(out2["F"][0], out["F"][0] @ Rm.T, atol=1e-11)


@pytest.mark.parametrize("nmol", [1, 2])
def test_forces_match_energy_finite_differences(params, nmol):
    rng = np.random.default_rng(13)
    sys_ = cs.cluster_batch(rng, [nmol], np.zeros((1, 3)), noise=0.1)
    pos = sys_.r[None]
    out = D.dftb(params, sys_.species, pos)
    h = 1e-4
    nat = pos.shape[1]
    disp = []
    for j in range(nat):
        for k in range(3):
            for sgn in (1, -1):
                d = pos[0].copy()
                d[j, k] += sgn * h
                disp.append(d)
    E = D.dftb(params, sys_.species, np.array(disp), q0=np.tile(out["q"], (len(disp), 1)))["E"]
    fd = -(E[0::2] - E[1::2]).reshape(nat, 3) / (2 * h)
    scale = np.abs(out["F"]).max()
    np.testing.assert_allclose(out["F"][0], fd, atol=1e-7 * scale + 1e-10)


def test_net_force_and_torque_vanish(params):
    pos = _waters(4)
    out = D.dftb(params, WATER, pos)
    F = out["F"]
    np.testing.assert_allclose(F.sum(1), 0.0, atol=1e-13)
    torque = np.cross(pos, F).sum(1)
    np.testing.assert_allclose(torque, 0.0, atol=1e-12)


def test_stored_water_is_a_minimum(params):
    """The stored set's textbook geometry is stationary (the repulsion fit)."""
    geo = cs.water_reference_geometry()[None]
    out = D.dftb(params, WATER, geo)
    np.testing.assert_allclose(out["F"], 0.0, atol=1e-12)


def test_overlap_assembly_matches_gaussian_basis(params, monkeypatch):
    """With Gaussian-orbital radial integrals swapped in, the assembled overlap of a water must
    equal the overlap matrix of that Gaussian basis built orbital by orbital (pins where each
    block and its transpose land)."""
    expo = {ELEM_O: 0.55, ELEM_H: 0.35}

    def gto_integrals(table, prm, ea, eb, r):
        vals = {k: np.zeros_like(r) for k in ("ss", "sp", "ps", "pps", "ppp")}
        for i, rr in enumerate(r):
            z = np.array([0.0, 0.0, rr])
            ab = _gto_block(expo[ea], expo[eb], np.zeros(3), z)
            ba = _gto_block(expo[eb], expo[ea], np.zeros(3), z)
            vals["ss"][i], vals["sp"][i], vals["ps"][i] = ab[0, 0], ab[0, 3], ba[0, 3]
            vals["pps"][i], vals["ppp"][i] = ab[3, 3], ab[1, 1]
        return vals, {k: np.zeros_like(r) for k in vals}

    monkeypatch.setattr(D, "_pair_integrals", gto_integrals)
    pos = _waters(1, seed=3)
    lay = D.Layout(params, WATER)
    _, S = D.build_h0_s(params, lay, pos)
    n = lay.norb
    direct = np.eye(n)
    for a in range(3):
        for b in range(3):
            if a == b:
                continue
            blk = _gto_block(expo[lay.species[a]], expo[lay.species[b]], pos[0, a], pos[0, b])
            na, nb = lay.norb_atom[a], lay.norb_atom[b]
            direct[lay.off[a]:lay.off[a + 1], lay.off[b]:lay.off[b + 1]] = blk[:na, :nb]
    np.testing.assert_allclose(S[0], direct, atol=1e-14)
