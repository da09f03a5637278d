"""Plain FP64 CPU oracle: Gamma-point SCC-DFTB of periodic cells.

TEST INFRASTRUCTURE ONLY. This module exists to check the CUDA path. Only the
test suite, the smoke check and the CPU-baseline leg of the benchmark may
import it; the library itself never does.

The paper's per-molecule systems are periodic (section "Computational details":
a cubic 10 Angstrom cell of 33 waters, periodic in all three directions, with
Gamma-point Brillouin-zone sampling). The paper prints none of the equations;
the textbook Gamma-point forms, written out, are:

* lattice translations T = n1 a1 + n2 a2 + n3 a3 (a_i the rows of ``lattice``);
  positions are unwrapped, so molecules stay whole;
* H0 and S at Gamma: the (A, B) block is the sum over every image T of the
  two-centre Slater-Koster block at d = r_B + T - r_A with |d| < r_cut; for
  A = B the T = 0 term is the on-site block;
* gamma at Gamma: the Klopman-Ohno function is split as 1/r + s(r). The 1/r part
  is the Ewald lattice sum (tin-foil boundary, neutralising background). The
  remainder s(r) = 1/sqrt(r^2 + c^2) - 1/r falls off only as r^-3, so its image
  sum is cut with the Slater-Koster cosine taper at r_cut. The on-site value of
  the Klopman-Ohno function is U_A;
* repulsion: one half of the pair sum over all images, cut at r_cut;
* the SCC loop, energy and analytic forces of oracle.dftb with these matrices,
  every derivative term summed over the same images.

Pins live in tests/test_oracle_periodic.py (Madelung constants, the Ewald
splitting parameter, the isolated-molecule limit with its tin-foil dipole term,
explicit supercell sums, finite-difference forces, lattice-translation
invariance).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

from . import dftb as D


# ---------------------------------------------------------------------------- lattice images

def image_shifts(lattice, r_max):
    """Integer translations n (K, 3) covering every image d + n @ lattice with |.| < r_max of a
    separation d whose fractional coordinates lie in [-1/2, 1/2]. The height of the cell
    across face i is h_i = 1 / |column i of lattice^-1|; |d + T| >= h_i (|n_i| - 1/2)."""
    inv = np.linalg.inv(lattice)
    h = 1.0 / np.linalg.norm(inv, axis=0)
    N = np.ceil(r_max / h + 0.5).astype(int)
    axes = [np.arange(-n, n + 1) for n in N]
    return np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)


def wrap(lattice, d):
    """d minus the lattice vector that brings its fractional coordinates into [-1/2, 1/2]."""
    inv = np.linalg.inv(lattice)
    f = d @ inv
    return d - np.round(f) @ lattice


def pair_images(lattice, d, r_max, shifts=None):
    """Every image d + T (K', 3) of the separation d with 0 < |d + T| < r_max."""
    if shifts is None:
        shifts = image_shifts(lattice, r_max)
    x = wrap(lattice, d)[None, :] + shifts @ lattice
    r = np.linalg.norm(x, axis=1)
    return x[(r < r_max) & (r > 0.0)]


# ---------------------------------------------------------------------------- H0 and S at Gamma

def build_h0_s_periodic(params, lay, pos, lattice, with_grad=False):
    """H0 and S (n, n) at Gamma for one cell; with_grad adds, per pair A < B, the image vectors
    and the derivative blocks d/dR_B of each image's two-centre block."""
    n = lay.norb
    H0 = np.zeros((n, n))
    S = np.zeros((n, n))
    shifts = image_shifts(lattice, params.r_cut)
    for a in range(lay.nat):
        e = lay.species[a]
        o = lay.off[a]
        H0[o, o] = params.onsite[e, 0]
        S[o, o] = 1.0
        if lay.norb_atom[a] == 4:
            for i in range(1, 4):
                H0[o + i, o + i] = params.onsite[e, 1]
                S[o + i, o + i] = 1.0
    grads = {}
    for a in range(lay.nat):
        for b in range(a, lay.nat):
            x = pair_images(lattice, pos[b] - pos[a], params.r_cut, shifts)
            if len(x) == 0:
                continue
            r = np.linalg.norm(x, axis=1)
            e = x / r[:, None]
            ea, eb = lay.species[a], lay.species[b]
            na, nb = lay.norb_atom[a], lay.norb_atom[b]
            sa, sb = slice(lay.off[a], lay.off[a + 1]), slice(lay.off[b], lay.off[b + 1])
            for M, table, key in ((H0, params.h0, "h"), (S, params.s, "s")):
                vals, dvals = D._pair_integrals(table, params, ea, eb, r)
                blk = D.sk_block(vals, e, na, nb).sum(0)
                if a == b:
                    # images of the atom itself: T and -T both appear, the sum is symmetric
                    M[sa, sa] += blk
                else:
                    M[sa, sb] += blk
                    M[sb, sa] += blk.T
                    if with_grad:
                        grads[(a, b, key)] = D.sk_block_grad(vals, dvals, e, r, na, nb)
            if with_grad and a != b:
                grads[(a, b, "x")] = x
    return (H0, S, grads) if with_grad else (H0, S)


# ---------------------------------------------------------------------------- Ewald 1/r lattice sum

def default_alpha(lattice):
    """Ewald splitting parameter sqrt(pi) / V^(1/3): real and reciprocal sums of similar size."""
    V = abs(np.linalg.det(lattice))
    return math.sqrt(math.pi) / V ** (1.0 / 3.0)


EWALD_X = 6.5     # erfc(6.5) ~ 4e-20 and exp(-6.5^2) ~ 5e-19: both sums cut where terms < 1e-18


def reciprocal_vectors(lattice, alpha):
    """Nonzero reciprocal vectors G = m @ (2 pi lattice^-T) with |G| < 2 alpha EWALD_X."""
    B = 2.0 * np.pi * np.linalg.inv(lattice).T
    g_max = 2.0 * alpha * EWALD_X
    m = image_shifts(B, g_max)
    G = m @ B
    g = np.linalg.norm(G, axis=1)
    return G[(g > 0.0) & (g < g_max)]


def ewald_matrix(lattice, pos, alpha=None, with_grad=False):
    """phi (nat, nat): the potential at r_A of a unit point charge at r_B and all its images,
    with a neutralising background and tin-foil boundary (Ewald 1921):

        phi(d) = sum_T erfc(alpha |d+T|) / |d+T|
               + (4 pi / V) sum_{G != 0} exp(-G^2 / 4 alpha^2) / G^2 cos(G . d)
               - pi / (alpha^2 V),

    and on the diagonal the same sum without the T = 0 term, minus 2 alpha / sqrt(pi).
    with_grad adds dphi (nat, nat, 3) = grad_d phi at d = r_B - r_A (zero on the diagonal)."""
    if alpha is None:
        alpha = default_alpha(lattice)
    V = abs(np.linalg.det(lattice))
    nat = len(pos)
    r_real = EWALD_X / alpha
    shifts = image_shifts(lattice, r_real)
    G = reciprocal_vectors(lattice, alpha)
    g2 = np.sum(G * G, axis=1)
    wG = 4.0 * np.pi / V * np.exp(-g2 / (4.0 * alpha * alpha)) / g2
    phi = np.zeros((nat, nat))
    dphi = np.zeros((nat, nat, 3))
    for a in range(nat):
        for b in range(nat):
            d = pos[b] - pos[a]
            x = wrap(lattice, d)[None, :] + shifts @ lattice
            r = np.linalg.norm(x, axis=1)
            keep = (r < r_real) & (r > 0.0)
            x, r = x[keep], r[keep]
            real = np.sum(erfc(alpha * r) / r)
            phase = G @ d
            rec = np.sum(wG * np.cos(phase))
            phi[a, b] = real + rec - np.pi / (alpha * alpha * V)
            if a == b:
                phi[a, b] -= 2.0 * alpha / math.sqrt(math.pi)
            elif with_grad:
                dr = -(erfc(alpha * r) / r ** 2
                       + 2.0 * alpha / math.sqrt(math.pi) * np.exp(-(alpha * r) ** 2) / r)
                dphi[a, b] = np.sum((dr / r)[:, None] * x, axis=0) - np.sum((wG * np.sin(phase))[:, None] * G, axis=0)
    return (phi, dphi) if with_grad else phi


def coulomb_energy(lattice, pos, Q, alpha=None):
    """Electrostatic energy per cell of point charges Q (neutral or with background),
    E = 1/2 sum_AB Q_A Q_B phi_AB."""
    phi = ewald_matrix(lattice, pos, alpha)
    return 0.5 * Q @ phi @ Q


# ---------------------------------------------------------------------------- gamma and repulsion at Gamma

def gamma_periodic(params, lay, pos, lattice, alpha=None, with_grad=False):
    """gamma at Gamma (nat, nat) = Ewald phi + tapered Klopman-Ohno remainder over images, with
    U_A added on the diagonal; with_grad adds dgam[A, B] = d gamma_AB / d r_B (A != B)."""
    out = ewald_matrix(lattice, pos, alpha, with_grad)
    phi, dphi = out if with_grad else (out, None)
    U = params.hubbard[lay.species]
    gam = phi.copy()
    dgam = dphi.copy() if with_grad else None
    shifts = image_shifts(lattice, params.r_cut)
    for a in range(lay.nat):
        gam[a, a] += U[a]
        for b in range(lay.nat):
            c = 2.0 / (U[a] + U[b])
            x = pair_images(lattice, pos[b] - pos[a], params.r_cut, shifts)
            if len(x) == 0:
                continue
            r = np.linalg.norm(x, axis=1)
            f, df = D.cutoff(r, params.r_cut, params.taper)
            s = 1.0 / np.sqrt(r * r + c * c) - 1.0 / r
            ds = -r / (r * r + c * c) ** 1.5 + 1.0 / (r * r)
            gam[a, b] += np.sum(s * f)
            if with_grad and a != b:
                dgam[a, b] += np.sum(((ds * f + s * df) / r)[:, None] * x, axis=0)
    return (gam, dgam) if with_grad else gam


def e_rep_periodic(params, lay, pos, lattice):
    """Repulsion energy per cell, 1/2 sum_A sum_B sum_T' V_rep(|r_B + T - r_A|) f_cut, and its
    gradient (nat, 3)."""
    E = 0.0
    G = np.zeros((lay.nat, 3))
    shifts = image_shifts(lattice, params.r_cut)
    for a in range(lay.nat):
        for b in range(lay.nat):
            arep, brep = params.rep[lay.species[a], lay.species[b]]
            x = pair_images(lattice, pos[b] - pos[a], params.r_cut, shifts)
            if len(x) == 0:
                continue
            r = np.linalg.norm(x, axis=1)
            f, df = D.cutoff(r, params.r_cut, params.taper)
            v = arep * np.exp(-brep * r)
            E += 0.5 * np.sum(v * f)
            if a != b:
                # d/dr_B of the (a, b) terms; the (b, a) terms give the same, so the halves add up
                G[b] += np.sum(((-brep * v * f + v * df) / r)[:, None] * x, axis=0)
    return E, G


# ---------------------------------------------------------------------------- one evaluation

def dftb_periodic(params, species, pos, lattice, q0=None, alpha=None, beta=0.5, tol=1e-12,
                  max_iter=400, forces=True):
    """One Gamma-point SCC-DFTB evaluation of one periodic cell.

    pos (nat, 3) unwrapped positions; lattice (3, 3) with the lattice vectors as rows.
    Returns E, F (nat, 3), q, Q = Z - q, mu = sum_A Q_A r_A (unwrapped positions), iters,
    eps, P, gap."""
    pos = np.asarray(pos, float)
    lattice = np.asarray(lattice, float)
    lay = D.Layout(params, species)
    if forces:
        H0, S, grads = build_h0_s_periodic(params, lay, pos, lattice, with_grad=True)
        gam, dgam = gamma_periodic(params, lay, pos, lattice, alpha, with_grad=True)
    else:
        H0, S = build_h0_s_periodic(params, lay, pos, lattice)
        gam = gamma_periodic(params, lay, pos, lattice, alpha)
    res = D.scc(params, lay, H0[None], S[None], gam[None], q0=None if q0 is None else q0[None],
                beta=beta, tol=tol, max_iter=max_iter)
    q = res["q"][0]
    Q = lay.zval - q
    out = {"q": q, "Q": Q, "mu": Q @ pos, "iters": res["iters"], "eps": res["eps"][0],
           "P": res["P"][0], "gap": res["gap"][0], "H0": H0, "S": S, "gamma": gam}
    P, W, shift = res["P"][0], res["W"][0], res["shift"][0]
    dq = q - lay.zval
    erep, G = e_rep_periodic(params, lay, pos, lattice)
    out["E"] = np.sum(P * H0) + 0.5 * dq @ gam @ dq + erep
    if not forces:
        return out
    for a in range(lay.nat):
        for b in range(a + 1, lay.nat):
            if (a, b, "x") not in grads:
                continue
            sa, sb = slice(lay.off[a], lay.off[a + 1]), slice(lay.off[b], lay.off[b + 1])
            Pab = P[sa, sb]
            Xab = Pab * 0.5 * (shift[a] + shift[b]) - W[sa, sb]
            # factor 2: the (B, A) block is the transpose and contributes equally
            g = 2.0 * (np.einsum("ij,tkij->k", Pab, grads[(a, b, "h")])
                       + np.einsum("ij,tkij->k", Xab, grads[(a, b, "s")]))
            G[b] += g
            G[a] -= g
    # second-order term with the charges held: dE2/dr_C = dq_C sum_A dq_A dgamma_AC / dr_C
    G += dq[:, None] * np.einsum("a,abk->bk", dq, dgam)
    out["F"] = -G
    return out


# ---------------------------------------------------------------------------- k-point sampling
#
# The paper samples the Brillouin zone at the Gamma point of a 3 x 3 x 3 folded supercell, i.e. on
# the Gamma-centred 3 x 3 x 3 grid of the cell itself. At each k the Bloch sums
#     H0(k)_{mu nu} = sum_T exp(i k.T) h_{mu nu}(r_B + T - r_A),  S(k) likewise,
# give a Hermitian generalised eigenproblem; the lowest n_occ bands are occupied at every k (an
# insulator); populations, band energy and forces are the k averages, and the force weights of an
# image T are the real-space densities rho_{mu nu}(T) = sum_k w_k Re[P(k)_{nu mu} exp(i k.T)].

def kgrid_points(kgrid):
    """Gamma-centred grid: fractional k = (i/n1, j/n2, l/n3) in units of the reciprocal lattice
    vectors (k.T = 2 pi f.n for T = n @ lattice), equal weights."""
    n1, n2, n3 = kgrid
    f = np.array([(i / n1, j / n2, l / n3) for i in range(n1) for j in range(n2) for l in range(n3)])
    return f, np.full(len(f), 1.0 / len(f))


def pair_images_n(lattice, d, r_max, shifts=None):
    """pair_images, with the integer translation n (T = n @ lattice, taken from r_B - r_A) of each."""
    if shifts is None:
        shifts = image_shifts(lattice, r_max)
    n0 = np.round(d @ np.linalg.inv(lattice))
    x = (d - n0 @ lattice)[None, :] + shifts @ lattice
    n = shifts - n0[None, :]
    r = np.linalg.norm(x, axis=1)
    keep = (r < r_max) & (r > 0.0)
    return x[keep], n[keep]


def build_hk_sk(params, lay, pos, lattice, fk):
    """H0(k), S(k) (K, n, n) complex for the fractional k-points fk (K, 3); and, per pair A < B,
    the image vectors, their integer translations and the derivative blocks of each image."""
    n = lay.norb
    K = len(fk)
    H0 = np.zeros((K, n, n), complex)
    S = np.zeros((K, n, n), complex)
    shifts = image_shifts(lattice, params.r_cut)
    for a in range(lay.nat):
        e = lay.species[a]
        o = lay.off[a]
        H0[:, o, o] = params.onsite[e, 0]
        S[:, o, o] = 1.0
        if lay.norb_atom[a] == 4:
            for i in range(1, 4):
                H0[:, o + i, o + i] = params.onsite[e, 1]
                S[:, o + i, o + i] = 1.0
    grads = {}
    for a in range(lay.nat):
        for b in range(a, lay.nat):
            x, nT = pair_images_n(lattice, pos[b] - pos[a], params.r_cut, shifts)
            if len(x) == 0:
                continue
            r = np.linalg.norm(x, axis=1)
            e = x / r[:, None]
            ph = np.exp(2j * np.pi * (fk @ nT.T))           # (K, images)
            ea, eb = lay.species[a], lay.species[b]
            na, nb = lay.norb_atom[a], lay.norb_atom[b]
            sa, sb = slice(lay.off[a], lay.off[a + 1]), slice(lay.off[b], lay.off[b + 1])
            for M, table, key in ((H0, params.h0, "h"), (S, params.s, "s")):
                vals, dvals = D._pair_integrals(table, params, ea, eb, r)
                blk = np.einsum("kt,tij->kij", ph, D.sk_block(vals, e, na, nb))
                if a == b:
                    M[:, sa, sa] += blk                      # images of the atom itself: Hermitian
                else:
                    M[:, sa, sb] += blk
                    M[:, sb, sa] += np.conj(np.swapaxes(blk, -1, -2))
                    grads[(a, b, key)] = D.sk_block_grad(vals, dvals, e, r, na, nb)
            if a != b:
                grads[(a, b, "x")] = x
                grads[(a, b, "n")] = nT
    return H0, S, grads


def dftb_periodic_k(params, species, pos, lattice, kgrid=(3, 3, 3), q0=None, alpha=None, beta=0.5,
                    tol=1e-12, max_iter=400, forces=True):
    """SCC-DFTB of one periodic cell sampled on the Gamma-centred k-grid ``kgrid``.

    Returns E (per cell), F, q, Q, mu = sum_A Q_A r_A, iters, eps (K, n) and gap (the smallest
    LUMO - HOMO over the grid)."""
    pos = np.asarray(pos, float)
    lattice = np.asarray(lattice, float)
    lay = D.Layout(params, species)
    fk, wk = kgrid_points(kgrid)
    H0, S, grads = build_hk_sk(params, lay, pos, lattice, fk)
    gam, dgam = gamma_periodic(params, lay, pos, lattice, alpha, with_grad=True)
    Z = lay.zval
    nocc = lay.n_occ
    q = Z.copy() if q0 is None else np.array(q0, float, copy=True)
    for it in range(1, max_iter + 1):
        shift = gam @ (q - Z)
        so = shift[lay.atom_of_orb]
        qorb = np.zeros(lay.norb)
        for k in range(len(fk)):
            Hk = H0[k] + 0.5 * S[k] * (so[:, None] + so[None, :])
            eps, C = scipy_eigh(Hk, S[k])
            Co = C[:, :nocc]
            Pk = 2.0 * Co @ Co.conj().T
            qorb += wk[k] * np.sum(Pk * S[k].conj(), axis=1).real      # (P(k) S(k))_mu mu
        q_out = np.array([qorb[lay.off[a]:lay.off[a + 1]].sum() for a in range(lay.nat)])
        if np.max(np.abs(q_out - q)) < tol:
            q = q_out
            break
        q = q + beta * (q_out - q)
    else:
        raise D.SCCError(f"SCC did not converge in {max_iter} iterations")
    dq = q - Z
    shift = gam @ dq
    so = shift[lay.atom_of_orb]
    n = lay.norb
    P = np.zeros((len(fk), n, n), complex)
    W = np.zeros((len(fk), n, n), complex)
    eps_all = np.zeros((len(fk), n))
    for k in range(len(fk)):
        Hk = H0[k] + 0.5 * S[k] * (so[:, None] + so[None, :])
        eps, C = scipy_eigh(Hk, S[k])
        Co = C[:, :nocc]
        P[k] = 2.0 * Co @ Co.conj().T
        W[k] = 2.0 * (Co * eps[None, :nocc]) @ Co.conj().T
        eps_all[k] = eps
    erep, G = e_rep_periodic(params, lay, pos, lattice)
    E = float(np.sum(wk[:, None, None] * P * H0.conj()).real) + 0.5 * dq @ gam @ dq + erep
    Q = Z - q
    out = {"E": E, "q": q, "Q": Q, "mu": Q @ pos, "iters": it, "eps": eps_all,
           "gap": (eps_all[:, nocc].min() - eps_all[:, nocc - 1].max()) if nocc < n else np.inf}
    if not forces:
        return out
    for a in range(lay.nat):
        for b in range(a + 1, lay.nat):
            if (a, b, "x") not in grads:
                continue
            sa, sb = slice(lay.off[a], lay.off[a + 1]), slice(lay.off[b], lay.off[b + 1])
            ph = np.exp(2j * np.pi * (fk @ grads[(a, b, "n")].T))   # (K, images)
            # rho(T)_{mu nu} = sum_k w_k Re[P(k)_{nu mu} exp(i k.T)], mu of A, nu of B
            rho = np.einsum("k,kt,kji->tij", wk, ph, P[:, sb, sa]).real
            om = np.einsum("k,kt,kji->tij", wk, ph, W[:, sb, sa]).real
            X = rho * 0.5 * (shift[a] + shift[b]) - om
            g = 2.0 * (np.einsum("tij,tkij->k", rho, grads[(a, b, "h")])
                       + np.einsum("tij,tkij->k", X, grads[(a, b, "s")]))
            G[b] += g
            G[a] -= g
    G += dq[:, None] * np.einsum("a,abk->bk", dq, dgam)
    out["F"] = -G
    return out


def scipy_eigh(H, S):
    """Generalised Hermitian eigenproblem H c = e S c, eigenvalues ascending (library routine)."""
    from scipy.linalg import eigh
    return eigh(H, S)


# ---------------------------------------------------------------------------- cells for the cavity step

def _cell_solver(kgrid):
    """dftb_periodic (the Gamma point) or dftb_periodic_k on the given Gamma-centred grid."""
    if kgrid is None or tuple(kgrid) == (1, 1, 1):
        return dftb_periodic
    return lambda *a, **k: dftb_periodic_k(*a, kgrid=tuple(kgrid), **k)


def born_fd_periodic(params, species, pos, lattice, pol, h=1e-3, scheme="forward", q_ref=None, mu_ref=None,
                     alpha=None, beta=0.5, tol=1e-12, max_iter=400, kgrid=None):
    """Finite-difference dipole derivative b_j = d(pol . mu)/dr_j of one periodic cell, shape (nat, 3):
    the Born charges of the paper's periodic cells (Results: forward differences, refreshed every
    3 steps). 'forward' is [M(r + h e) - M(r)] / h, 'central' [M(r + h e) - M(r - h e)] / 2h, with mu
    the unwrapped cell dipole of dftb_periodic (or of dftb_periodic_k on the grid kgrid); every
    displaced solve starts from the reference populations."""
    pos = np.asarray(pos, float)
    pol = np.asarray(pol, float)
    solve = _cell_solver(kgrid)
    if q_ref is None or mu_ref is None:
        ref = solve(params, species, pos, lattice, alpha=alpha, beta=beta, tol=tol, max_iter=max_iter,
                    forces=False)
        q_ref, mu_ref = ref["q"], ref["mu"]
    kw = dict(q0=q_ref, alpha=alpha, beta=beta, tol=tol, max_iter=max_iter, forces=False)
    M0 = mu_ref @ pol
    b = np.zeros((len(pos), 3))
    for j in range(len(pos)):
        for k in range(3):
            dp = pos.copy()
            dp[j, k] += h
            Mp = solve(params, species, dp, lattice, **kw)["mu"] @ pol
            if scheme == "forward":
                b[j, k] = (Mp - M0) / h
            else:
                dm = pos.copy()
                dm[j, k] -= h
                Mm = solve(params, species, dm, lattice, **kw)["mu"] @ pol
                b[j, k] = (Mp - Mm) / (2.0 * h)
    return b


class PeriodicDFTBMatter:
    """Periodic cells evaluated with dftb_periodic (or, with kgrid, dftb_periodic_k on that
    Gamma-centred grid), with the interface of oracle.cavity's DFTBMatter: Mulliken charges
    (b_j = Q_j pol) or finite-difference Born charges ('born_fd', forward, or 'born_central';
    refreshed every born_interval evaluations). lattice: (3, 3) shared by all cells or
    (n_cells, 3, 3)."""

    def __init__(self, params, system, lattice, pol=(1.0, 0.0, 0.0), alpha=None, beta=0.5,
                 tol=1e-12, max_iter=400, charge_model="mulliken", born_interval=1, fd_step=1e-3, kgrid=None):
        self.params = params
        self.species = np.asarray(system.species)
        self.off = np.asarray(system.cell_offset)
        self.n_cells = len(self.off) - 1
        lat = np.asarray(lattice, float)
        self.lattice = np.broadcast_to(lat, (self.n_cells, 3, 3)) if lat.ndim == 2 else lat
        self.pol = np.asarray(pol, float)
        self.mass = params.mass[self.species]
        self.cell_of_atom = np.repeat(np.arange(self.n_cells), np.diff(self.off))
        self.charge_model = charge_model
        self.born_interval = born_interval
        self.fd_step = fd_step
        self.alpha = alpha
        self.kw = dict(beta=beta, tol=tol, max_iter=max_iter)
        self.kgrid = kgrid
        self.q = None
        self.b = None
        self.n_eval = 0
        self.iters = []

    def __call__(self, r):
        n_at = len(self.species)
        F = np.zeros((n_at, 3))
        E = np.zeros(self.n_cells)
        Mn = np.zeros(self.n_cells)
        Q = np.zeros(n_at)
        q_all = np.zeros(n_at)
        iters = []
        refresh = self.charge_model != "mulliken" and ((self.n_eval % self.born_interval == 0) or self.b is None)
        b = Q[:, None] * self.pol if self.charge_model == "mulliken" else (
            np.zeros((n_at, 3)) if refresh else self.b.copy())
        for c in range(self.n_cells):
            s = slice(self.off[c], self.off[c + 1])
            q0 = None if self.q is None else self.q[s]
            out = _cell_solver(self.kgrid)(self.params, self.species[s], r[s], self.lattice[c], q0=q0,
                                           alpha=self.alpha, **self.kw)
            iters.append(out["iters"])
            F[s] = out["F"]
            E[c] = out["E"]
            Q[s] = out["Q"]
            q_all[s] = out["q"]
            Mn[c] = out["mu"] @ self.pol
            if refresh:
                scheme = "forward" if self.charge_model == "born_fd" else "central"
                b[s] = born_fd_periodic(self.params, self.species[s], r[s], self.lattice[c], self.pol,
                                        h=self.fd_step, scheme=scheme, q_ref=out["q"], mu_ref=out["mu"],
                                        alpha=self.alpha, kgrid=self.kgrid, **self.kw)
        self.q = q_all
        if self.charge_model == "mulliken":
            b = Q[:, None] * self.pol
        self.b = b
        self.n_eval += 1
        self.iters.append(max(iters) if iters else 0)
        return {"F": F, "E": E, "M": Mn, "b": self.b.copy(), "Q": Q}
