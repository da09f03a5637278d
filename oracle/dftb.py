"""Plain FP64 CPU oracle: second-order SCC-DFTB of isolated molecules and clusters.

TEST INFRASTRUCTURE ONLY. This module exists to check the CUDA path. Only the
test suite, the smoke check and the CPU-baseline leg of the benchmark may
import it; the library itself never does.

The paper names the electronic-structure method (second-order SCC-DFTB, as run
by DFTB+, section "Computational details") but prints none of its equations.
What follows is the textbook method written out step by step:

* two-centre Hamiltonian H0 and overlap S from Slater-Koster tables
  (Slater & Koster 1954 direction-cosine rules) with synthetic radial
  functions (cavmd_synth.params);
* Klopman-Ohno gamma_AB(r) = 1 / sqrt(r^2 + (2 / (U_A + U_B))^2);
* the self-consistent-charge loop
      eps_A = sum_B gamma_AB dq_B,  H = H0 + 1/2 S o (eps_A + eps_B),
      H c = e S c,  P = sum_i f_i c_i c_i^T,  q_A = sum_{mu in A} (P S)_mu,mu,
  with linear mixing q <- q + beta (q_out - q) (beta = 0.5; converged results do not depend on it);
* E = sum P H0 + 1/2 sum gamma dq dq + E_rep and its analytic gradient
      dE/dR = sum P dH0 + sum (P 1/2 (eps_A + eps_B) - W) dS
              + 1/2 sum dq_A dq_B dgamma + dE_rep,   W = sum_i f_i e_i c_i c_i^T.

Every routine is vectorised over a batch of B molecules that share one species
list (one water, or one cluster size); no other blocking or reordering.
Parity pins for each routine live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import numpy as np

SS, SP, PPS, PPP = 0, 1, 2, 3


# ---------------------------------------------------------------------------- radial functions

def cutoff(r, r_cut, taper):
    """Smooth cutoff: 1 below r_cut - taper, cosine taper to 0 at r_cut. Returns (f, df/dr)."""
    r = np.asarray(r, float)
    x = (r - (r_cut - taper)) / taper
    inside = (x > 0.0) & (x < 1.0)
    f = np.where(x <= 0.0, 1.0, np.where(inside, 0.5 * (1.0 + np.cos(np.pi * x)), 0.0))
    df = np.where(inside, -0.5 * np.pi / taper * np.sin(np.pi * x), 0.0)
    return f, df


def radial(par, r, r_cut, taper):
    """V(r) = a exp(-b r) (1 + c1 r + c2 r^2) f_cut(r) and dV/dr."""
    a, b, c1, c2 = par
    e = a * np.exp(-b * r)
    poly = 1.0 + c1 * r + c2 * r * r
    dpoly = c1 + 2.0 * c2 * r
    f, df = cutoff(r, r_cut, taper)
    v = e * poly * f
    dv = e * (-b * poly * f + dpoly * f + poly * df)
    return v, dv


# ---------------------------------------------------------------------------- Slater-Koster blocks

def sk_block(vals, e, na, nb):
    """Two-centre block <mu_A | nu_B> from radial integrals and the unit vector e (A -> B).

    vals: dict with 'ss', 'sp' (s on A, p on B), 'ps' (s on B, p on A; the table entry taken with
    B as the first atom) and 'pps', 'ppp', each of shape (...). Orbital order s, px, py, pz.
    Rules (Slater & Koster 1954, Table I):
        <s|s> = ss;  <s_A|p_B,i> = e_i sp;  <p_A,i|s_B> = -e_i ps;
        <p_A,i|p_B,j> = e_i e_j pps + (delta_ij - e_i e_j) ppp.
    """
    shape = e.shape[:-1]
    blk = np.zeros(shape + (na, nb))
    blk[..., 0, 0] = vals["ss"]
    if nb == 4:
        blk[..., 0, 1:] = e * vals["sp"][..., None]
    if na == 4:
        blk[..., 1:, 0] = -e * vals["ps"][..., None]
    if na == 4 and nb == 4:
        ee = e[..., :, None] * e[..., None, :]
        eye = np.eye(3)
        blk[..., 1:, 1:] = ee * vals["pps"][..., None, None] + (eye - ee) * vals["ppp"][..., None, None]
    return blk


def sk_block_grad(vals, dvals, e, r, na, nb):
    """d<mu_A|nu_B>/dR_B (= -d/dR_A), shape (..., 3, na, nb), by the chain rule on sk_block with
    dr/dR_B,k = e_k and de_i/dR_B,k = (delta_ik - e_i e_k) / r."""
    shape = e.shape[:-1]
    eye = np.eye(3)
    de = (eye - e[..., :, None] * e[..., None, :]) / r[..., None, None]     # [.., i, k] = de_i/dR_k
    g = np.zeros(shape + (3, na, nb))
    g[..., :, 0, 0] = dvals["ss"][..., None] * e
    if nb == 4:
        # d(e_i sp)/dR_k = de_i/dR_k sp + e_i sp' e_k
        g[..., :, 0, 1:] = (np.swapaxes(de, -1, -2) * vals["sp"][..., None, None]
                            + e[..., :, None] * e[..., None, :] * dvals["sp"][..., None, None])
    if na == 4:
        g[..., :, 1:, 0] = -(np.swapaxes(de, -1, -2) * vals["ps"][..., None, None]
                             + e[..., :, None] * e[..., None, :] * dvals["ps"][..., None, None])
    if na == 4 and nb == 4:
        dsp = vals["pps"] - vals["ppp"]
        ddsp = dvals["pps"] - dvals["ppp"]
        # d(e_i e_j)/dR_k = de_i/dR_k e_j + e_i de_j/dR_k   -> index order [k, i, j]
        dee = (np.einsum("...ik,...j->...kij", de, e) + np.einsum("...i,...jk->...kij", e, de))
        eee = np.einsum("...k,...i,...j->...kij", e, e, e)
        g[..., :, 1:, 1:] = (dee * dsp[..., None, None, None] + eee * ddsp[..., None, None, None]
                             + eye[None, :, :] * (dvals["ppp"][..., None] * e)[..., :, None, None])
    return g


def _pair_integrals(table, params, ea, eb, r):
    """Radial values and derivatives of all integrals between elements ea (A) and eb (B)."""
    vals, dvals = {}, {}
    zero = np.zeros_like(r)
    for key, (x, y, kind) in {"ss": (ea, eb, SS), "sp": (ea, eb, SP), "ps": (eb, ea, SP),
                              "pps": (ea, eb, PPS), "ppp": (ea, eb, PPP)}.items():
        par = table[x, y, kind]
        if np.all(par == 0.0):
            vals[key], dvals[key] = zero, zero
        else:
            vals[key], dvals[key] = radial(par, r, params.r_cut, params.taper)
    return vals, dvals


# ---------------------------------------------------------------------------- molecule layout

class Layout:
    """Orbital bookkeeping for one species list (e.g. O, H, H)."""

    def __init__(self, params, species):
        self.species = np.asarray(species, int)
        self.nat = len(self.species)
        self.norb_atom = params.norb[self.species].astype(int)
        self.off = np.concatenate([[0], np.cumsum(self.norb_atom)])
        self.norb = int(self.off[-1])
        self.atom_of_orb = np.repeat(np.arange(self.nat), self.norb_atom)
        self.zval = params.zval[self.species]
        self.n_el = float(self.zval.sum())
        self.n_occ = int(round(self.n_el)) // 2
        self.pairs = [(a, b) for a in range(self.nat) for b in range(a + 1, self.nat)]


def build_h0_s(params, lay, pos, with_grad=False):
    """H0 and S (B, n, n) for positions pos (B, nat, 3); optionally the per-pair derivative
    blocks d/dR_B of the (A, B) off-diagonal blocks, keyed by the pair (A, B)."""
    B = pos.shape[0]
    n = lay.norb
    H0 = np.zeros((B, n, n))
    S = np.zeros((B, n, n))
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
    for (a, b) in lay.pairs:
        d = pos[:, b] - pos[:, a]
        r = np.linalg.norm(d, axis=-1)
        e = d / r[:, None]
        ea, eb = lay.species[a], lay.species[b]
        na, nb = lay.norb_atom[a], lay.norb_atom[b]
        sa, sb = slice(lay.off[a], lay.off[a + 1]), slice(lay.off[b], lay.off[b + 1])
        for M, table, key in ((H0, params.h0, "h"), (S, params.s, "s")):
            vals, dvals = _pair_integrals(table, params, ea, eb, r)
            blk = sk_block(vals, e, na, nb)
            M[:, sa, sb] = blk
            M[:, sb, sa] = np.swapaxes(blk, -1, -2)
            if with_grad:
                grads[(a, b, key)] = sk_block_grad(vals, dvals, e, r, na, nb)
    return (H0, S, grads) if with_grad else (H0, S)


def gamma_matrix(params, lay, pos, with_grad=False):
    """Klopman-Ohno gamma (B, nat, nat); with_grad adds dgamma/dr for every pair."""
    U = params.hubbard[lay.species]
    d = pos[:, None, :, :] - pos[:, :, None, :]
    r2 = np.sum(d * d, axis=-1)
    c = 2.0 / (U[:, None] + U[None, :])
    g = 1.0 / np.sqrt(r2 + c * c)
    if not with_grad:
        return g
    dg_dr = -np.sqrt(r2) * g ** 3           # d gamma / d r
    return g, dg_dr


def e_rep(params, lay, pos):
    """Pair repulsion energy (B,) and its gradient dE/dR (B, nat, 3)."""
    B = pos.shape[0]
    E = np.zeros(B)
    G = np.zeros((B, lay.nat, 3))
    for (a, b) in lay.pairs:
        arep, brep = params.rep[lay.species[a], lay.species[b]]
        d = pos[:, b] - pos[:, a]
        r = np.linalg.norm(d, axis=-1)
        f, df = cutoff(r, params.r_cut, params.taper)
        v = arep * np.exp(-brep * r)
        E += v * f
        dv = (-brep * v * f + v * df)[:, None] * d / r[:, None]
        G[:, b] += dv
        G[:, a] -= dv
    return E, G


# ---------------------------------------------------------------------------- eigen / SCC

def gen_eigh(H, S):
    """Generalised symmetric eigenproblem H c = e S c (batched) via S = L L^T:
    L^-1 H L^-T v = e v, c = L^-T v. Library routines: Cholesky, inverse, eigh."""
    L = np.linalg.cholesky(S)
    Li = np.linalg.inv(L)
    Hp = Li @ H @ np.swapaxes(Li, -1, -2)
    Hp = 0.5 * (Hp + np.swapaxes(Hp, -1, -2))
    e, V = np.linalg.eigh(Hp)
    C = np.swapaxes(Li, -1, -2) @ V
    return e, C


class SCCError(RuntimeError):
    pass


def mulliken(lay, P, S):
    """Atomic Mulliken populations q_A = sum_{mu in A} (P S)_mu,mu, shape (B, nat)."""
    qorb = np.sum(P * S, axis=-1)          # (P S)_mu,mu for symmetric S
    q = np.zeros(P.shape[:-2] + (lay.nat,))
    for a in range(lay.nat):
        q[..., a] = qorb[..., lay.off[a]:lay.off[a + 1]].sum(-1)
    return q


def scc(params, lay, H0, S, gam, q0=None, beta=0.5, tol=1e-12, max_iter=400, min_gap=1e-3):
    """Self-consistent-charge loop (batched). Returns a dict with the converged populations q,
    density P, energy-weighted density W, eigenvalues, atomic shifts and iteration count."""
    B = H0.shape[0]
    Z = lay.zval
    q = np.tile(Z, (B, 1)) if q0 is None else np.array(q0, float, copy=True)
    nocc = lay.n_occ
    it = 0
    for it in range(1, max_iter + 1):
        dq = q - Z
        shift = np.einsum("bij,bj->bi", gam, dq)
        so = shift[:, lay.atom_of_orb]
        H = H0 + 0.5 * S * (so[:, :, None] + so[:, None, :])
        eps, C = gen_eigh(H, S)
        Co = C[:, :, :nocc]
        P = 2.0 * Co @ np.swapaxes(Co, -1, -2)
        q_out = mulliken(lay, P, S)
        res = np.max(np.abs(q_out - q), axis=-1)
        if np.all(res < tol):
            q = q_out
            break
        q = q + beta * (q_out - q)
    else:
        raise SCCError(f"SCC did not converge in {max_iter} iterations (max residual {res.max():.3e})")
    gap = eps[:, nocc] - eps[:, nocc - 1] if nocc < lay.norb else np.full(B, np.inf)
    if np.any(gap < min_gap):
        raise SCCError("degenerate or vanishing HOMO-LUMO gap")
    W = 2.0 * (Co * eps[:, None, :nocc]) @ np.swapaxes(Co, -1, -2)
    dq = q - Z
    shift = np.einsum("bij,bj->bi", gam, dq)
    return {"q": q, "P": P, "W": W, "eps": eps, "C": C, "shift": shift, "iters": it, "gap": gap}


def energy_and_gradient(params, lay, pos, H0, S, grads, gam, dgam, res):
    """E_DFTB (B,) and dE/dR (B, nat, 3) at SCC convergence."""
    P, W, q, shift = res["P"], res["W"], res["q"], res["shift"]
    dq = q - lay.zval
    erep, grep = e_rep(params, lay, pos)
    E = np.sum(P * H0, axis=(-1, -2)) + 0.5 * np.einsum("bi,bij,bj->b", dq, gam, dq) + erep
    G = grep.copy()
    for (a, b) in lay.pairs:
        sa, sb = slice(lay.off[a], lay.off[a + 1]), slice(lay.off[b], lay.off[b + 1])
        Pab = P[:, sa, sb]
        Xab = Pab * (0.5 * (shift[:, a] + shift[:, b]))[:, None, None] - W[:, sa, sb]
        # factor 2: the (B, A) block is the transpose and contributes equally
        g = 2.0 * (np.einsum("bij,bkij->bk", Pab, grads[(a, b, "h")])
                   + np.einsum("bij,bkij->bk", Xab, grads[(a, b, "s")]))
        d = pos[:, b] - pos[:, a]
        r = np.linalg.norm(d, axis=-1)
        g += (dq[:, a] * dq[:, b] * dgam[:, a, b])[:, None] * d / r[:, None]
        G[:, b] += g
        G[:, a] -= g
    return E, G


def dftb(params, species, pos, q0=None, beta=0.5, tol=1e-12, max_iter=400, forces=True):
    """One SCC-DFTB evaluation of a batch of molecules sharing ``species``.

    pos: (B, nat, 3). Returns dict with E (B,), F (B, nat, 3) = -dE/dR, q (B, nat) Mulliken
    populations, Q = Z - q net atomic charges, mu (B, 3) dipole sum_A Q_A R_A, iters."""
    pos = np.asarray(pos, float)
    lay = Layout(params, species)
    if forces:
        H0, S, grads = build_h0_s(params, lay, pos, with_grad=True)
        gam, dgam = gamma_matrix(params, lay, pos, with_grad=True)
    else:
        H0, S = build_h0_s(params, lay, pos)
        gam = gamma_matrix(params, lay, pos)
    res = scc(params, lay, H0, S, gam, q0=q0, beta=beta, tol=tol, max_iter=max_iter)
    Q = lay.zval - res["q"]
    out = {"q": res["q"], "Q": Q, "mu": np.einsum("ba,bak->bk", Q, pos), "iters": res["iters"],
           "eps": res["eps"], "P": res["P"], "gap": res["gap"]}
    if forces:
        E, G = energy_and_gradient(params, lay, pos, H0, S, grads, gam, dgam, res)
        out["E"] = E
        out["F"] = -G
    return out


def born_fd(params, species, pos, pol, h=1e-3, scheme="forward", q_ref=None, mu_ref=None,
            beta=0.5, tol=1e-12, max_iter=400):
    """Finite-difference dipole derivative b_j = d(pol . mu)/dr_j, shape (B, nat, 3).

    'forward' is the paper's [M(r + h) - M(r)] / h (Results, first paragraph); 'central' uses
    [M(r + h) - M(r - h)] / 2h. Displaced solves start from the reference populations."""
    pos = np.asarray(pos, float)
    B, nat, _ = pos.shape
    pol = np.asarray(pol, float)
    if q_ref is None or mu_ref is None:
        ref = dftb(params, species, pos, beta=beta, tol=tol, max_iter=max_iter, forces=False)
        q_ref, mu_ref = ref["q"], ref["mu"]
    M0 = mu_ref @ pol
    b = np.zeros((B, nat, 3))
    for j in range(nat):
        for k in range(3):
            dp = pos.copy()
            dp[:, j, k] += h
            Mp = dftb(params, species, dp, q0=q_ref, beta=beta, tol=tol, max_iter=max_iter,
                      forces=False)["mu"] @ pol
            if scheme == "forward":
                b[:, j, k] = (Mp - M0) / h
            else:
                dm = pos.copy()
                dm[:, j, k] -= h
                Mm = dftb(params, species, dm, q0=q_ref, beta=beta, tol=tol, max_iter=max_iter,
                          forces=False)["mu"] @ pol
                b[:, j, k] = (Mp - Mm) / (2.0 * h)
    return b
