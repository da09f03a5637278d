"""Pins of the periodic (Gamma-point) oracle against what the mathematics fixes.

* Ewald lattice sums: the Madelung constants of rock salt (conventional cubic cell and the
  primitive fcc cell, a non-orthogonal lattice) and caesium chloride; every entry of the
  potential matrix independent of the splitting parameter alpha (this pins the self and
  neutralising-background terms, which move with alpha).
* Image bookkeeping: H0, S, the repulsion and the short-range gamma remainder against sums over
  an explicit block of 5 x 5 x 5 copies of the cell, built from the cluster oracle's pinned
  two-centre routines with no cutoff logic of their own.
* The isolated-molecule limit: one water in a large cube differs from the cluster oracle by the
  tin-foil dipole term -2 pi mu^2 / (3 V) (de Leeuw, Perram and Smith 1980), to leading order in
  1/V; charges and forces converge to the cluster values.
* Analytic forces against central finite differences of the energy, in a cube small enough that
  every term has images.
* Lattice translations of one molecule and rigid shifts of the whole cell change nothing; the
  populations sum to the valence electron count.
* k-point sampling: the Gamma-centred 3 x 3 x 3 grid of a cell equals the Gamma point of the
  explicit 3 x 3 x 3 supercell (energy per cell, populations, forces and the whole band spectrum,
  by Bloch's theorem); a 1 x 1 x 1 grid is the Gamma point; forces on a 2 x 2 x 1 grid against
  central finite differences.
"""
import math

import numpy as np
import pytest

import cavmd_synth as cs
from oracle import dftb as D
from oracle import periodic as PR

M_NACL = 1.747564594633182      # rock salt, per ion pair, nearest-neighbour distance
M_CSCL = 1.762674773070999      # caesium chloride, per ion pair, nearest-neighbour distance


@pytest.fixture(scope="module")
def params():
    return cs.load_water_params()


def _rock_salt_conventional(a):
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]]) * a
    pos = np.concatenate([fcc, fcc + np.array([.5, 0, 0]) * a])
    Q = np.concatenate([np.ones(4), -np.ones(4)])
    return a * np.eye(3), pos, Q


def test_madelung_rock_salt_conventional():
    a = 5.3
    lat, pos, Q = _rock_salt_conventional(a)
    E = PR.coulomb_energy(lat, pos, Q)
    np.testing.assert_allclose(E, -4.0 * M_NACL / (a / 2.0), rtol=1e-12)


def test_madelung_rock_salt_primitive_fcc():
    a = 5.3
    lat = np.array([[0, .5, .5], [.5, 0, .5], [.5, .5, 0]]) * a
    pos = np.array([[0.0, 0.0, 0.0], [a / 2.0, 0.0, 0.0]])
    E = PR.coulomb_energy(lat, pos, np.array([1.0, -1.0]))
    np.testing.assert_allclose(E, -M_NACL / (a / 2.0), rtol=1e-12)


def test_madelung_caesium_chloride():
    a = 4.1
    pos = np.array([[0.0, 0.0, 0.0], [a / 2, a / 2, a / 2]])
    E = PR.coulomb_energy(a * np.eye(3), pos, np.array([1.0, -1.0]))
    np.testing.assert_allclose(E, -M_CSCL / (math.sqrt(3.0) * a / 2.0), rtol=1e-12)


SHEARED = np.array([[8.5, 0.0, 0.0], [5.0, 8.0, 0.0], [-4.0, 3.5, 8.5]])


@pytest.mark.parametrize("lat", [np.array([[9.0, 0.4, 0.0], [0.0, 8.0, -0.7], [0.5, 0.0, 10.0]]), SHEARED])
def test_ewald_entries_do_not_depend_on_alpha(lat):
    rng = np.random.default_rng(4)
    pos = rng.uniform(-3.0, 12.0, (5, 3))
    a0 = PR.default_alpha(lat)
    ref, dref = PR.ewald_matrix(lat, pos, a0, with_grad=True)
    for s in (0.6, 1.7):
        phi, dphi = PR.ewald_matrix(lat, pos, a0 * s, with_grad=True)
        np.testing.assert_allclose(phi, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
        np.testing.assert_allclose(dphi, dref, rtol=0, atol=1e-13 * np.abs(dref).max())


@pytest.mark.parametrize("lat", [SHEARED, np.array([[6.0, 0.0, 0.0], [11.0, 3.0, 0.0], [-7.0, 9.0, 5.0]]),
                                 np.array([[3.0, 0.5, 0.0], [0.0, 20.0, 0.0], [0.0, 19.0, 2.5]])])
def test_image_lists_are_complete(lat):
    """Every image within r_max, against brute force over n in [-30, 30]^3."""
    rng = np.random.default_rng(9)
    m = np.stack(np.meshgrid(*[np.arange(-30, 31)] * 3, indexing="ij"), -1).reshape(-1, 3)
    for _ in range(20):
        d = rng.uniform(-3.0, 3.0, 3) + (rng.integers(-2, 3, 3) @ lat if lat[0, 0] > 5.0 else 0.0)
        brute = d + m @ lat
        r = np.linalg.norm(brute, axis=1)
        brute = brute[(r < 12.0) & (r > 0.0)]
        got = PR.pair_images(lat, d, 12.0)
        assert len(got) == len(brute)
        key = lambda x: np.lexsort(np.round(x, 9).T)
        np.testing.assert_allclose(got[key(got)], brute[key(brute)], rtol=0, atol=1e-9)


def _two_waters(side=8.5, seed=11):
    rng = np.random.default_rng(seed)
    sy, lat = cs.periodic_water_cells(rng, np.array([[3.0, -2.0, 1.0]]), n_waters=2, side=side,
                                      d_min=4.0, d_atom=2.8)
    return sy, lat


def _copies(lat, n=3):
    m = np.stack(np.meshgrid(*[np.arange(-n, n + 1)] * 3, indexing="ij"), -1).reshape(-1, 3)
    return m @ lat


@pytest.mark.parametrize("sheared", [False, True])
def test_images_against_an_explicit_block_of_copies(params, sheared):
    sy, lat = _two_waters()
    if sheared:
        lat = SHEARED
    lay = D.Layout(params, sy.species)
    pos = sy.r
    H0, S = PR.build_h0_s_periodic(params, lay, pos, lat)
    T = _copies(lat)
    assert np.linalg.norm(T, axis=1)[np.linalg.norm(T, axis=1) > 0].min() < params.r_cut
    Hb = np.zeros_like(H0)
    Sb = np.zeros_like(S)
    for a in range(lay.nat):
        sa = slice(lay.off[a], lay.off[a + 1])
        Hb[sa, sa] += np.diag(np.where(np.arange(lay.norb_atom[a]) == 0, params.onsite[lay.species[a], 0],
                                       params.onsite[lay.species[a], 1]))
        Sb[sa, sa] += np.eye(lay.norb_atom[a])
        for b in range(lay.nat):
            sb = slice(lay.off[b], lay.off[b + 1])
            x = pos[b] + T - pos[a]
            r = np.linalg.norm(x, axis=1)
            x, r = x[r > 0], r[r > 0]
            for M, table in ((Hb, params.h0), (Sb, params.s)):
                vals, _ = D._pair_integrals(table, params, lay.species[a], lay.species[b], r)
                M[sa, sb] += D.sk_block(vals, x / r[:, None], lay.norb_atom[a], lay.norb_atom[b]).sum(0)
    np.testing.assert_allclose(H0, Hb, rtol=0, atol=1e-14)
    np.testing.assert_allclose(S, Sb, rtol=0, atol=1e-14)


def test_repulsion_and_gamma_remainder_against_copies(params):
    sy, lat = _two_waters()
    lay = D.Layout(params, sy.species)
    pos = sy.r
    T = _copies(lat)
    erep, _ = PR.e_rep_periodic(params, lay, pos, lat)
    # the explicit block: the central cell against every copy, each pair counted from both ends
    big = (pos[None, :, :] + T[:, None, :]).reshape(-1, 3)
    spec_big = np.tile(lay.species, len(T))
    e = 0.0
    for a in range(lay.nat):
        x = big - pos[a]
        r = np.linalg.norm(x, axis=1)
        keep = r > 0
        rr = r[keep]
        ab = params.rep[lay.species[a], spec_big[keep]]
        f, _ = D.cutoff(rr, params.r_cut, params.taper)
        e += 0.5 * np.sum(ab[:, 0] * np.exp(-ab[:, 1] * rr) * f)
    np.testing.assert_allclose(erep, e, rtol=1e-14)
    # gamma minus its Ewald part: U_A on the diagonal plus the tapered Klopman-Ohno remainder,
    # taken from the cluster oracle's gamma on the explicit copies
    gam = PR.gamma_periodic(params, lay, pos, lat)
    phi = PR.ewald_matrix(lat, pos)
    both = np.concatenate([pos, big])
    sp = np.concatenate([lay.species, spec_big])
    gko = D.gamma_matrix(params, D.Layout(params, sp), both[None])[0][:lay.nat, lay.nat:]
    d = np.linalg.norm(big[None, :, :] - pos[:, None, :], axis=2)
    f, _ = D.cutoff(d, params.r_cut, params.taper)
    with np.errstate(divide="ignore"):
        rem = np.where(d > 0, (gko - 1.0 / d) * f, 0.0)
    ref = rem.reshape(lay.nat, len(T), lay.nat).sum(1) + np.diag(params.hubbard[lay.species])
    np.testing.assert_allclose(gam - phi, ref, rtol=0, atol=1e-14)


def _one_water(params, side):
    rng = np.random.default_rng(3)
    cent = np.array([[0.3, -0.2, 0.1]])
    pos = cs.water_batch(rng, cent)[0]
    return pos, side * np.eye(3)


def test_isolated_limit_tin_foil_dipole_term(params):
    pos, _ = _one_water(params, 1.0)
    spec = np.array([cs.ELEM_O, cs.ELEM_H, cs.ELEM_H])
    iso = D.dftb(params, spec, pos[None])
    mu = iso["mu"][0]
    for side, tol in ((40.0, 2e-2), (70.0, 4e-3)):
        lat = side * np.eye(3)
        per = PR.dftb_periodic(params, spec, pos, lat)
        V = side ** 3
        lead = -2.0 * math.pi * (mu @ mu) / (3.0 * V)
        np.testing.assert_allclose((per["E"] - iso["E"][0]) / lead, 1.0, rtol=0, atol=tol)
        assert np.abs(per["q"] - iso["q"][0]).max() < 50.0 / V
        assert np.abs(per["F"] - iso["F"][0]).max() < 50.0 / V
    np.testing.assert_allclose(per["mu"], mu, rtol=0, atol=1e-3)


def test_forces_against_finite_differences(params):
    sy, lat = _two_waters()
    pos = sy.r.copy()
    out = PR.dftb_periodic(params, sy.species, pos, lat, tol=1e-13)
    h = 1e-4
    fd = np.zeros_like(pos)
    for j in range(len(pos)):
        for k in range(3):
            e = []
            for s in (1.0, -1.0):
                p = pos.copy()
                p[j, k] += s * h
                e.append(PR.dftb_periodic(params, sy.species, p, lat, q0=out["q"], tol=1e-13,
                                          forces=False)["E"])
            fd[j, k] = -(e[0] - e[1]) / (2.0 * h)
    np.testing.assert_allclose(out["F"], fd, rtol=0, atol=1e-7 * np.abs(out["F"]).max())


def test_translations_change_nothing(params):
    sy, lat = _two_waters()
    pos = sy.r.copy()
    ref = PR.dftb_periodic(params, sy.species, pos, lat)
    np.testing.assert_allclose(ref["q"].sum(), 16.0, rtol=0, atol=1e-10)
    moved = pos.copy()
    moved[3:6] += lat[0] - 2.0 * lat[2]           # the second water one image over
    out = PR.dftb_periodic(params, sy.species, moved, lat)
    np.testing.assert_allclose(out["E"], ref["E"], rtol=1e-13)
    np.testing.assert_allclose(out["F"], ref["F"], rtol=0, atol=1e-10 * np.abs(ref["F"]).max())
    np.testing.assert_allclose(out["q"], ref["q"], rtol=0, atol=1e-11)
    out = PR.dftb_periodic(params, sy.species, pos + np.array([0.37, -1.3, 2.9]), lat)
    np.testing.assert_allclose(out["E"], ref["E"], rtol=1e-13)
    np.testing.assert_allclose(out["q"], ref["q"], rtol=0, atol=1e-11)


def test_liquid_cell_of_33_waters(params):
    """The paper's cell: 33 waters in a 10 Angstrom cube. Populations sum to 264 electrons,
    the overlap is positive definite, the gap is open, and the sum of forces vanishes (no
    external field acts on an isolated periodic cell)."""
    sy, lat = cs.periodic_water_cells(np.random.default_rng(5), np.zeros((1, 3)))
    out = PR.dftb_periodic(params, sy.species, sy.r, lat)
    np.testing.assert_allclose(out["q"].sum(), 264.0, rtol=0, atol=1e-9)
    assert np.linalg.eigvalsh(out["S"]).min() > 0.1 and out["gap"] > 0.3
    np.testing.assert_allclose(out["F"].sum(0), 0.0, rtol=0, atol=1e-10 * np.abs(out["F"]).max())


def _supercell(pos, species, lat, m=3):
    cells = np.stack(np.meshgrid(*[np.arange(m)] * 3, indexing="ij"), -1).reshape(-1, 3)
    return (pos[None, :, :] + (cells @ lat)[:, None, :]).reshape(-1, 3), np.tile(species, len(cells)), m * lat


def test_kgrid_equals_gamma_point_of_the_supercell(params):
    sy, lat = _two_waters()
    k3 = PR.dftb_periodic_k(params, sy.species, sy.r, lat, (3, 3, 3))
    pos_s, spec_s, lat_s = _supercell(sy.r, sy.species, lat)
    sc = PR.dftb_periodic(params, spec_s, pos_s, lat_s)
    nat = len(sy.species)
    np.testing.assert_allclose(sc["E"] / 27.0, k3["E"], rtol=0, atol=1e-12)
    for c in range(27):   # every copy carries the cell's populations and forces
        np.testing.assert_allclose(sc["q"][c * nat:(c + 1) * nat], k3["q"], rtol=0, atol=1e-12)
        np.testing.assert_allclose(sc["F"][c * nat:(c + 1) * nat], k3["F"], rtol=0, atol=1e-11 * np.abs(k3["F"]).max())
    np.testing.assert_allclose(np.sort(sc["eps"]), np.sort(k3["eps"].ravel()), rtol=0, atol=1e-11)
    # the grid matters in this small cube: the Gamma point alone is another answer
    g = PR.dftb_periodic(params, sy.species, sy.r, lat)
    assert abs(g["E"] - k3["E"]) > 1e-3


def test_kgrid_111_is_the_gamma_point(params):
    sy, lat = _two_waters()
    g = PR.dftb_periodic(params, sy.species, sy.r, lat)
    k1 = PR.dftb_periodic_k(params, sy.species, sy.r, lat, (1, 1, 1))
    np.testing.assert_allclose(k1["E"], g["E"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(k1["q"], g["q"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(k1["F"], g["F"], rtol=0, atol=1e-12)


def test_kgrid_forces_against_finite_differences(params):
    sy, lat = _two_waters()
    pos = sy.r.copy()
    out = PR.dftb_periodic_k(params, sy.species, pos, lat, (2, 2, 1), tol=1e-13)
    h = 1e-4
    fd = np.zeros_like(pos)
    for j in range(len(pos)):
        for k in range(3):
            e = []
            for sg in (1.0, -1.0):
                p = pos.copy()
                p[j, k] += sg * h
                e.append(PR.dftb_periodic_k(params, sy.species, p, lat, (2, 2, 1), q0=out["q"], tol=1e-13,
                                            forces=False)["E"])
            fd[j, k] = -(e[0] - e[1]) / (2.0 * h)
    np.testing.assert_allclose(out["F"], fd, rtol=0, atol=1e-7 * np.abs(out["F"]).max())


def test_born_charges_of_a_periodic_cell(params):
    """Finite-difference Born charges of a periodic cell (born_fd_periodic): central differences obey
    the translation sum rule sum_j b_j = Q_cell pol = 0 (to O(h^2)); forward and central differences
    differ at O(h) (halving h halves the gap); and one water in a large cube approaches the isolated
    molecule's charges as the cube grows (the images' field falls off as 1 / V)."""
    from oracle import dftb as D
    sy, lat = _two_waters()
    pos, spec = sy.r, sy.species
    pol = np.array([1.0, 0.0, 0.0])
    bc = PR.born_fd_periodic(params, spec, pos, lat, pol, h=1e-3, scheme="central")
    assert np.abs(bc.sum(0)).max() < 1e-6
    g1 = np.abs(PR.born_fd_periodic(params, spec, pos, lat, pol, h=1e-3) - bc).max()
    g2 = np.abs(PR.born_fd_periodic(params, spec, pos, lat, pol, h=5e-4) - bc).max()
    assert 0.35 < g2 / g1 < 0.65
    w, _ = _one_water(params, 1.0)
    iso = D.born_fd(params, [0, 1, 1], w[None], pol, h=1e-3, scheme="central")[0]
    gaps = []
    for side in (40.0, 80.0):
        bp = PR.born_fd_periodic(params, [0, 1, 1], w, side * np.eye(3), pol, h=1e-3, scheme="central")
        gaps.append(np.abs(bp - iso).max())
    assert gaps[1] < 0.25 * gaps[0] and gaps[1] < 2e-3 * np.abs(iso).max()


def test_kgrid_born_charges_equal_the_supercells(params):
    """Born charges on the 3 x 3 x 3 k-grid (born_fd_periodic with kgrid) against the explicit
    supercell at the Gamma point: moving atom j of the cell moves it in every copy, so the cell's
    dipole change is the supercell's divided by 27 (Bloch's theorem, exact up to rounding). Two
    entries, forward differences from the same reference charges."""
    sy, lat = _two_waters()
    pol = np.array([1.0, 0.0, 0.0])
    h = 1e-3
    ref = PR.dftb_periodic_k(params, sy.species, sy.r, lat, (3, 3, 3), forces=False)
    bk = PR.born_fd_periodic(params, sy.species, sy.r, lat, pol, h=h, q_ref=ref["q"], mu_ref=ref["mu"],
                             kgrid=(3, 3, 3))
    pos_s, spec_s, lat_s = _supercell(sy.r, sy.species, lat)
    nat = len(sy.species)
    q0 = np.tile(ref["q"], 27)
    m0 = PR.dftb_periodic(params, spec_s, pos_s, lat_s, q0=q0, forces=False)["mu"] @ pol
    for j, k in ((0, 0), (4, 2)):
        p = pos_s.copy()
        p[j::nat, k] += h
        m1 = PR.dftb_periodic(params, spec_s, p, lat_s, q0=q0, forces=False)["mu"] @ pol
        np.testing.assert_allclose(bk[j, k], (m1 - m0) / (27.0 * h), rtol=0, atol=1e-7)
    # and the grid matters: the Gamma point's Born charges differ
    bg = PR.born_fd_periodic(params, sy.species, sy.r, lat, pol, h=h)
    assert np.abs(bg - bk).max() > 1e-3
