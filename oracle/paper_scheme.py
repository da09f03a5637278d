"""Plain FP64 CPU oracle: the paper's real-space / reciprocal-space propagation (Steps 1-4).

TEST INFRASTRUCTURE ONLY (see oracle/dftb.py).

Cells sit on a line lattice R_n = n a (n = 0..N-1) with N in-plane modes k_j = 2 pi j / (N a).
With the approximation sqrt(omega_k) ~ sqrt(omega_0) the coupling becomes local (Eq. hlm3):
eta q_n mu_n + eta^2 / (2 omega_0^2) mu_n^2 with eta = sqrt(2N) g0 omega_0. One step:

  Step 1 (Eq. pj1): half-kick the local photon momenta with -eta mu_n and the nuclei with
      F^m = -grad V - eta q_n dmu/dr - eta^2 mu_n / omega_0^2 dmu/dr (Eq. dpj), drift the
      nuclei, re-evaluate the matter at the new positions, half-kick both again with q fixed;
  Step 2 (Eqs. qkink_ak, qk_nk): a_k = sum_n sqrt(omega_0 / 2N) (q_n + i p_n / omega_0) e^{-ikR_n},
      q_k = (a_k + a_k*) / sqrt(2 omega_k),  p_k = i sqrt(omega_k / 2) (a_k* - a_k);
  Step 3 (Eq. qknk): rotate every (q_k, p_k) analytically over dt at omega_k;
  Step 4 (Eqs. qkink_an, nk_qk): a_n = sum_k sqrt(omega_k / 2N) (q_k + i p_k / omega_k) e^{ikR_n},
      q_n = (a_n + a_n*) / sqrt(2 omega_0),  p_n = i sqrt(omega_0 / 2) (a_n* - a_n).

With a flat dispersion (omega_k = omega_0 for all k) this is an exact rewriting of the k-space
Hamiltonian, which is what the parity test uses it for.
"""
from __future__ import annotations

import numpy as np


class PaperRealSpaceMD:
    def __init__(self, matter, r, p, R, kvals, omega_k, g0, omega0, dt):
        self.matter = matter
        self.r = np.array(r, float)
        self.p = np.array(p, float)
        self.R = np.asarray(R, float)             # lattice positions along x, (N,)
        self.k = np.asarray(kvals, float)         # (N,)
        self.wk = np.asarray(omega_k, float)
        self.N = len(self.R)
        self.w0 = float(omega0)
        self.eta = np.sqrt(2.0 * self.N) * g0 * self.w0
        self.dt = float(dt)
        self.cell = matter.cell_of_atom
        self.out = matter(self.r)
        # Step 0 with frozen nuclei ends at the photon minimum: q_n = -eta mu_n / omega_0^2, p_n = 0
        self.qn = -self.eta * self.out["M"] / self.w0 ** 2
        self.pn = np.zeros(self.N)

    def _forces(self):
        Mn, b = self.out["M"], self.out["b"]
        coef = self.eta * self.qn + self.eta ** 2 * Mn / self.w0 ** 2
        Fm = self.out["F"] - coef[self.cell][:, None] * b
        Fc = -self.eta * Mn
        return Fm, Fc

    def step(self):
        h = 0.5 * self.dt
        m = self.matter.mass[:, None]
        Fm, Fc = self._forces()
        self.pn = self.pn + h * Fc
        self.p = self.p + h * Fm
        self.r = self.r + self.dt * self.p / m
        self.out = self.matter(self.r)
        Fm, Fc = self._forces()
        self.p = self.p + h * Fm
        self.pn = self.pn + h * Fc
        # Step 2
        ph = np.exp(-1j * np.outer(self.k, self.R))                         # e^{-ikR_n}, (k, n)
        ak = ph @ (np.sqrt(self.w0 / (2 * self.N)) * (self.qn + 1j * self.pn / self.w0))
        qk = ((ak + ak.conj()) / np.sqrt(2.0 * self.wk)).real
        pk = (1j * np.sqrt(self.wk / 2.0) * (ak.conj() - ak)).real
        # Step 3
        c, s = np.cos(self.wk * self.dt), np.sin(self.wk * self.dt)
        qk, pk = qk * c + pk * s / self.wk, pk * c - self.wk * qk * s
        # Step 4
        an = ph.conj().T @ (np.sqrt(self.wk / (2 * self.N)) * (qk + 1j * pk / self.wk))
        self.qn = ((an + an.conj()) / np.sqrt(2.0 * self.w0)).real
        self.pn = (1j * np.sqrt(self.w0 / 2.0) * (an.conj() - an)).real

    def energies(self):
        """Valid for a flat dispersion, where the free photon energy is local."""
        m = self.matter.mass
        kin = float(np.sum(self.p ** 2 / (2.0 * m[:, None])))
        Mn = self.out["M"]
        photon = float(np.sum(0.5 * self.pn ** 2 + 0.5 * self.w0 ** 2 * self.qn ** 2
                              + self.eta * self.qn * Mn + self.eta ** 2 / (2 * self.w0 ** 2) * Mn ** 2))
        return {"kinetic": kin, "dftb": float(np.sum(self.out["E"])), "photon": photon,
                "total": kin + float(np.sum(self.out["E"])) + photon}
