"""Synthetic Slater-Koster parameter sets drawn from a seed.

The paper runs DFTB+ with a real water parameter set that is not available
here, so both implementations read a synthetic set with the same functional
form. Every two-centre integral tau (ss-sigma, sp-sigma, pp-sigma, pp-pi) of
the Hamiltonian H0 and of the overlap S uses the radial form

    V_tau(r) = a * exp(-b r) * (1 + c1 r + c2 r^2) * f_cut(r)

with b ~ U[1, 2] per bohr and c1, c2 ~ U[0, 0.5]. The amplitude a is drawn so
that |V_tau(r0)| (taper aside) is a uniform draw from a per-integral range at
the reference distance r0 = 2 bohr, with a fixed sign per integral. The
cutoff f_cut is 1 below r_cut - taper and a cosine taper to 0 at r_cut.

On-site energies, Hubbard parameters U and valence charges are fixed per
element. The pair repulsion a_rep * exp(-b_rep r) * f_cut(r) has a fixed
b_rep; the two amplitudes a_rep(O-H) and a_rep(H-H) of the water set are
fitted so that the textbook water geometry is the minimum of the synthetic
surface. That fit needs the energy surface itself, so it is not done here:
it is stored in ``data/water_sk.json`` by a script that lives with the
oracle.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field

import numpy as np

from .units import AMU

ELEM_O = 0
ELEM_H = 1
N_ELEM = 2
N_ORB = (4, 1)                 # O: s, px, py, pz;  H: s
ZVAL = (6.0, 1.0)              # valence electrons (neutral atom populations)
MASS_AMU = (15.9994, 1.00794)
HUBBARD = (0.50, 0.42)         # Hartree; Klopman-Ohno gamma reaches U at r = 0
ONSITE = ((-0.88, -0.33), (-0.24, 0.0))   # (eps_s, eps_p) in Hartree

SS, SP, PPS, PPP = 0, 1, 2, 3  # integral kinds; SP means s on the first atom, p on the second

R0 = 2.0          # bohr, reference distance of the amplitude draw
R_CUT = 12.0      # bohr
TAPER = 1.0       # bohr, width of the cosine taper below R_CUT

# (sign, low, high) of V_tau(R0) per integral kind, overlap and Hamiltonian
_S_SPEC = {SS: (+1, 0.30, 0.45), SP: (-1, 0.25, 0.40), PPS: (-1, 0.15, 0.30), PPP: (+1, 0.08, 0.18)}
_H_SPEC = {SS: (-1, 0.30, 0.45), SP: (+1, 0.30, 0.45), PPS: (+1, 0.20, 0.35), PPP: (-1, 0.08, 0.18)}

# fixed decay constants of the pair repulsion (per bohr)
B_REP = {(ELEM_O, ELEM_O): 1.5, (ELEM_O, ELEM_H): 2.0, (ELEM_H, ELEM_H): 1.5}


@dataclass
class SKParams:
    """A complete synthetic parameter set (arrays indexed by element ids)."""
    onsite: np.ndarray            # [N_ELEM, 2]  eps_s, eps_p
    hubbard: np.ndarray           # [N_ELEM]
    zval: np.ndarray              # [N_ELEM]
    mass: np.ndarray              # [N_ELEM] in electron masses
    norb: np.ndarray              # [N_ELEM] 1 or 4
    h0: np.ndarray                # [N_ELEM, N_ELEM, 4 kinds, 4 = (a, b, c1, c2)]
    s: np.ndarray                 # same layout for the overlap
    rep: np.ndarray               # [N_ELEM, N_ELEM, 2 = (a_rep, b_rep)]
    r_cut: float = R_CUT
    taper: float = TAPER
    seed: int = -1
    meta: dict = field(default_factory=dict)

    def to_json(self) -> dict:
        return {
            "seed": self.seed, "r_cut": self.r_cut, "taper": self.taper,
            "onsite": self.onsite.tolist(), "hubbard": self.hubbard.tolist(),
            "zval": self.zval.tolist(), "mass": self.mass.tolist(), "norb": self.norb.tolist(),
            "h0": self.h0.tolist(), "s": self.s.tolist(), "rep": self.rep.tolist(),
            "meta": self.meta,
        }

    @staticmethod
    def from_json(d: dict) -> "SKParams":
        return SKParams(
            onsite=np.array(d["onsite"], float), hubbard=np.array(d["hubbard"], float),
            zval=np.array(d["zval"], float), mass=np.array(d["mass"], float),
            norb=np.array(d["norb"], np.int32), h0=np.array(d["h0"], float),
            s=np.array(d["s"], float), rep=np.array(d["rep"], float),
            r_cut=float(d["r_cut"]), taper=float(d["taper"]), seed=int(d["seed"]),
            meta=dict(d.get("meta", {})))


def _valid_kinds(ea: int, eb: int):
    """Integral kinds that exist between element ea (first) and eb (second)."""
    kinds = [SS]
    if N_ORB[eb] == 4:
        kinds.append(SP)           # s on ea, p on eb
    if N_ORB[ea] == 4 and N_ORB[eb] == 4:
        kinds += [PPS, PPP]
    return kinds


def draw_sk_params(seed: int, a_rep=None) -> SKParams:
    """Draw a synthetic parameter set from ``seed``.

    ``a_rep`` optionally gives the repulsion amplitudes as a dict
    {(ea, eb): a}; missing pairs default to 1.0 Hartree.
    """
    rng = np.random.default_rng(seed)
    h0 = np.zeros((N_ELEM, N_ELEM, 4, 4))
    s = np.zeros((N_ELEM, N_ELEM, 4, 4))
    for table, spec in ((s, _S_SPEC), (h0, _H_SPEC)):
        for ea in range(N_ELEM):
            for eb in range(N_ELEM):
                for kind in _valid_kinds(ea, eb):
                    symmetric = kind != SP
                    if symmetric and eb < ea:
                        continue            # drawn once for the unordered pair
                    b = rng.uniform(1.0, 2.0)
                    c1 = rng.uniform(0.0, 0.5)
                    c2 = rng.uniform(0.0, 0.5)
                    sign, lo, hi = spec[kind]
                    mag = rng.uniform(lo, hi)
                    a = sign * mag * np.exp(b * R0) / (1.0 + c1 * R0 + c2 * R0 * R0)
                    table[ea, eb, kind] = (a, b, c1, c2)
                    if symmetric:
                        table[eb, ea, kind] = (a, b, c1, c2)
    rep = np.zeros((N_ELEM, N_ELEM, 2))
    for (ea, eb), brep in B_REP.items():
        a = 1.0 if a_rep is None else float(a_rep.get((ea, eb), a_rep.get((eb, ea), 1.0)))
        rep[ea, eb] = rep[eb, ea] = (a, brep)
    return SKParams(
        onsite=np.array(ONSITE, float), hubbard=np.array(HUBBARD, float),
        zval=np.array(ZVAL, float), mass=np.array(MASS_AMU, float) * AMU,
        norb=np.array(N_ORB, np.int32), h0=h0, s=s, rep=rep, seed=seed)


_DATA = os.path.join(os.path.dirname(__file__), "data")


def load_water_params(name: str = "water_sk.json") -> SKParams:
    """The stored water parameter set (seed draw plus fitted repulsion)."""
    with open(os.path.join(_DATA, name)) as f:
        return SKParams.from_json(json.load(f))


def water_reference_geometry(r_oh: float = 1.809, angle_deg: float = 104.52) -> np.ndarray:
    """Textbook water (O, H, H) in bohr, O at the origin, molecule in the xy plane."""
    h = np.deg2rad(angle_deg) / 2.0
    return np.array([[0.0, 0.0, 0.0],
                     [r_oh * np.sin(h), r_oh * np.cos(h), 0.0],
                     [-r_oh * np.sin(h), r_oh * np.cos(h), 0.0]])
