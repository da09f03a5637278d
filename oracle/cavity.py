"""Plain FP64 CPU oracle: multimode light-matter coupling and the time step.

TEST INFRASTRUCTURE ONLY (see oracle/dftb.py).

Classical k-space form of the dipole-gauge Hamiltonian beyond the long-wavelength
approximation (Eq. hlm_bigin, expanded in Eq. hlm2). A travelling mode pair +-k with
mode function f_k(R) = g0 / sqrt(omega_k) e^{ikR} is written as two real modes with
u_a(R) = cos(k.R) and sin(k.R) and amplitude lambda_a = 2 g0 (sqrt(2) g0 for a single
real mode such as k = 0). With classical (q_a, p_a) the photon part becomes

    H_ph = sum_a 1/2 p_a^2 + 1/2 (omega_a q_a - D_a)^2,   D_a = lambda_a sum_n u_a(R_n) M_n,

whose 1/2 D^2 term is the dipole self-energy of Eq. hlm2. M_n = pol . mu_n is the
projected cell dipole (Eq. hm and the text after it). The forces (k-space form of
Eq. dpj) are

    on a nucleus j of cell n:  F_j = -dV_n/dr_j + E_n b_j,
        E_n = sum_a lambda_a u_a(R_n) (omega_a q_a - D_a),  b_j = dM_n/dr_j;
    on photon mode a:          -omega_a^2 q_a + omega_a D_a.

Three splittings of one velocity-Verlet-like step (all symmetric, one matter evaluation):
  * "photon_exact" (default): H = T_nuc + H_2 with H_2 = V(r) + H_ph(q, p; r). At frozen
    nuclei H_2 is exactly solvable: each mode rotates about its displaced centre D_a / omega_a
    (the analytic rotation of Eq. qknk, shifted), and the nuclear momenta take the time
    integral of -dH_2/dr in closed form,
        dp_j = tau F_j^V + [sum_a lambda_a u_a(R_n) Y_a] b_j,
        Y_a = y_a sin(omega_a tau) + p_a (1 - cos(omega_a tau)) / omega_a,  y_a = q_a - D_a/omega_a,
    which reduces to the kick tau E_n b_j of Eq. dpj when omega_a tau -> 0. Step:
    H_2(dt/2), drift(dt), H_2(dt/2). It stays stable when omega_a dt >> 1;
  * "strang": H = A + B with A = sum p^2/2m + sum 1/2 (p_a^2 + omega_a^2 q_a^2) (drift and
    the rotation of Eq. qknk) and B = V(r) - sum omega_a q_a D_a + 1/2 sum D_a^2 (kicks):
    kick_B(dt/2), flow_A(dt), kick_B(dt/2);
  * "paper": kick_B(dt/2), drift(dt), kick_B(dt/2), rotate(dt): the paper's Step 1
    (Eq. pj1) followed by the reciprocal-space rotation of Step 3 (Eq. qknk).
"""
from __future__ import annotations

import numpy as np

from . import dftb as D

KB = 3.166811563e-6


# ---------------------------------------------------------------------------- coupling

def mode_functions(k, phi, R):
    """u[a, n] = cos(k_a . R_n + phi_a), shape (M, N)."""
    return np.cos(np.asarray(k) @ np.asarray(R).T + np.asarray(phi)[:, None])


def mode_function_sines(k, phi, R):
    """s[a, n] = sin(k_a . R_n + phi_a): grad u_a(R) = -k_a s_a(R)."""
    return np.sin(np.asarray(k) @ np.asarray(R).T + np.asarray(phi)[:, None])


def cell_centres(r, mass, off):
    """Centre of mass of every cell, shape (N, 3)."""
    r = np.asarray(r, float)
    out = np.zeros((len(off) - 1, 3))
    for n in range(len(off) - 1):
        m = mass[off[n]:off[n + 1]]
        out[n] = (m[:, None] * r[off[n]:off[n + 1]]).sum(0) / m.sum()
    return out


def field_gradient_on_cells(S, lam, k, w):
    """G_n = sum_a lambda_a w_a grad u_a(R_n) = -sum_a lambda_a w_a k_a s_a(R_n), shape (N, 3)."""
    return -S.T @ ((lam * w)[:, None] * np.asarray(k))


def forward(U, lam, M):
    """D_a = lambda_a sum_n u_a(R_n) M_n."""
    return lam * (U @ M)


def field_on_cells(U, lam, omega, q, Dv):
    """E_n = sum_a lambda_a u_a(R_n) (omega_a q_a - D_a)."""
    return U.T @ (lam * (omega * q - Dv))


def rotate(q, p, omega, t):
    """Exact free-oscillator flow over time t (Eq. qknk)."""
    c, s = np.cos(omega * t), np.sin(omega * t)
    return q * c + p * s / omega, p * c - omega * q * s


# ---------------------------------------------------------------------------- matter models

class DFTBMatter:
    """Cells evaluated with oracle.dftb; dipole derivative by Mulliken charges, FD Born or the
    Born-charge network.

    charge_model: 'mulliken' (b_j = Q_j pol, the paper's cheap replacement), 'born_fd' (forward
    differences, the paper's choice), 'born_central' (central differences, for tests) or 'network'
    (b_j = pol^T Z_j with Z_j the Born tensor of the per-atom network of oracle/mlp.py with
    parameters mlp_params, evaluated in FP64 on every evaluation).
    born_interval: refresh the finite-difference b every this many evaluations (the paper uses 3);
    stale otherwise."""

    def __init__(self, params, system, pol=(1.0, 0.0, 0.0), charge_model="mulliken",
                 born_interval=1, fd_step=1e-3, beta=0.5, tol=1e-12, max_iter=400, mlp_params=None):
        self.params = params
        self.species = np.asarray(system.species)
        self.off = np.asarray(system.cell_offset)
        self.n_cells = len(self.off) - 1
        self.pol = np.asarray(pol, float)
        self.mass = params.mass[self.species]
        self.cell_of_atom = np.repeat(np.arange(self.n_cells), np.diff(self.off))
        self.charge_model = charge_model
        if charge_model == "network" and mlp_params is None:
            raise ValueError("charge_model 'network' needs mlp_params")
        self.mlp_params = None if mlp_params is None else np.asarray(mlp_params, float)
        self.born_interval = born_interval
        self.fd_step = fd_step
        self.kw = dict(beta=beta, tol=tol, max_iter=max_iter)
        groups = {}
        for c in range(self.n_cells):
            key = tuple(self.species[self.off[c]:self.off[c + 1]])
            groups.setdefault(key, []).append(c)
        self.groups = [(list(k), np.array(v)) for k, v in groups.items()]
        self.q = None               # warm-start populations per atom
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
        refresh = (self.n_eval % self.born_interval == 0) or self.b is None
        b = np.zeros((n_at, 3)) if refresh else self.b.copy()
        iters = []
        for spec, cells in self.groups:
            nat = len(spec)
            idx = (self.off[cells][:, None] + np.arange(nat)[None, :])
            pos = r[idx]
            q0 = None if self.q is None else self.q[idx]
            out = D.dftb(self.params, spec, pos, q0=q0, **self.kw)
            iters.append(out["iters"])
            F[idx] = out["F"]
            E[cells] = out["E"]
            Q[idx] = out["Q"]
            q_all[idx] = out["q"]
            Mn[cells] = out["mu"] @ self.pol
            if self.charge_model == "mulliken":
                b[idx] = out["Q"][..., None] * self.pol
            elif self.charge_model == "network":
                from . import mlp as NN
                nc = len(cells)
                Z = NN.predict(self.mlp_params, np.tile(spec, nc), pos.reshape(-1, 3),
                               np.arange(nc + 1) * nat, out["Q"].ravel())
                b[idx] = np.einsum("a,jab->jb", self.pol, Z).reshape(nc, nat, 3)
            elif refresh:
                scheme = "forward" if self.charge_model == "born_fd" else "central"
                b[idx] = D.born_fd(self.params, spec, pos, self.pol, h=self.fd_step, scheme=scheme,
                                   q_ref=out["q"], mu_ref=out["mu"], **self.kw)
        self.q = q_all
        self.b = b
        self.n_eval += 1
        self.iters.append(max(iters))
        return {"E": E, "F": F, "M": Mn, "b": b, "Q": Q}


class HarmonicMatter:
    """N identical isotropic oscillators, one 'atom' per cell: V = 1/2 m w^2 |r - r0|^2 and a
    linear dipole M_n = d pol . (r_n - r0_n). A test model for the coupling and the integrator."""

    def __init__(self, r0, mass, omega_v, d, pol=(1.0, 0.0, 0.0)):
        self.r0 = np.asarray(r0, float)
        self.n_cells = len(self.r0)
        self.mass = np.full(self.n_cells, float(mass))
        self.w = float(omega_v)
        self.d = float(d)
        self.pol = np.asarray(pol, float)
        self.cell_of_atom = np.arange(self.n_cells)

    def __call__(self, r):
        x = r - self.r0
        E = 0.5 * self.mass * self.w ** 2 * np.sum(x * x, axis=1)
        F = -(self.mass * self.w ** 2)[:, None] * x
        M = self.d * (x @ self.pol)
        b = np.tile(self.d * self.pol, (self.n_cells, 1))
        return {"E": E, "F": F, "M": M, "b": b}


# ---------------------------------------------------------------------------- dynamics

class CavityMD:
    """State and time step of the coupled nuclei + photon system.

    mode_positions: "fixed" evaluates u_a at the reference cell positions R_ref (the paper's
    boxes sit at fixed positions R_n); "com" evaluates it at every cell's instantaneous centre
    of mass R_n(r) = sum_j m_j r_j / m_n, regenerated after every drift. Then D_a depends on the
    nuclear positions through u_a(R_n) as well, and -dH_ph/dr_j gains
        (m_j / m_n) M_n sum_a lambda_a (omega_a q_a - D_a) grad u_a(R_n),  grad u_a = -k_a sin(k_a.R + phi_a).
    R_n is frozen during the exact H_2 flow, so that flow stays exact and its time-integrated
    force gains the same term with Y_a in place of (omega_a q_a - D_a). Only the photon_exact
    splitting supports it."""

    def __init__(self, matter, r, p, modes_k, omega, lam, phi, R_ref, dt, splitting="photon_exact",
                 photon_init="relaxed", U=None, mode_positions="fixed"):
        self.matter = matter
        self.r = np.array(r, float)
        self.p = np.array(p, float)
        self.omega = np.asarray(omega, float)
        self.lam = np.asarray(lam, float)
        self.k = np.asarray(modes_k, float)
        self.phi = np.asarray(phi, float)
        if mode_positions not in ("fixed", "com"):
            raise ValueError(mode_positions)
        if mode_positions == "com" and (splitting != "photon_exact" or U is not None):
            raise ValueError("moving mode positions need the photon_exact splitting and no given U")
        self.moving = mode_positions == "com"
        self.off = np.concatenate([[0], np.cumsum(np.bincount(matter.cell_of_atom))]).astype(int)
        self.w_atom = None
        if self.moving:
            m = matter.mass
            mc = np.bincount(matter.cell_of_atom, m)
            self.w_atom = m / mc[matter.cell_of_atom]          # m_j / m_n
            self._mode_functions()
        else:
            self.U = mode_functions(modes_k, phi, R_ref) if U is None else np.asarray(U, float)
        self.dt = float(dt)
        self.splitting = splitting
        self.cell = matter.cell_of_atom
        self.step_count = 0
        self._evaluate_matter()
        self.D = forward(self.U, self.lam, self.out["M"])
        if photon_init == "relaxed":         # p_a = 0, q_a = D_a / omega_a: minimum of H_ph
            self.q = self.D / self.omega
        else:
            self.q = np.zeros_like(self.omega)
        self.pq = np.zeros_like(self.omega)
        self._coupling_force()

    def _evaluate_matter(self):
        self.out = self.matter(self.r)

    def _mode_functions(self):
        """u_a and sin(k_a.R + phi_a) at the current cell centres of mass (moving positions)."""
        self.R = cell_centres(self.r, self.matter.mass, self.off)
        self.U = mode_functions(self.k, self.phi, self.R)
        self.S = mode_function_sines(self.k, self.phi, self.R)

    def _position_term(self, w):
        """Force (or time-integrated force) on every nucleus through u_a(R_n): with weights
        w_a = omega_a q_a - D_a (or Y_a), (m_j / m_n) M_n sum_a lambda_a w_a grad u_a(R_n)."""
        G = field_gradient_on_cells(self.S, self.lam, self.k, w)
        return (self.w_atom * self.out["M"][self.cell])[:, None] * G[self.cell]

    def _coupling_force(self):
        self.E_field = field_on_cells(self.U, self.lam, self.omega, self.q, self.D)
        self.F = self.out["F"] + self.E_field[self.cell][:, None] * self.out["b"]
        if self.moving:
            self.F = self.F + self._position_term(self.omega * self.q - self.D)

    def _kick(self, h):
        self.p += h * self.F
        self.pq += h * self.omega * self.D

    def _h2_flow(self, tau):
        """Exact flow of H_2 = V + H_ph over time tau at frozen nuclei."""
        w = self.omega
        c = self.D / w
        y = self.q - c
        p0 = self.pq
        sn, cs = np.sin(w * tau), np.cos(w * tau)
        Y = y * sn + p0 * (1.0 - cs) / w
        self.E_field = field_on_cells(self.U, self.lam, np.ones_like(w), Y, np.zeros_like(w))
        self.p += tau * self.out["F"] + self.E_field[self.cell][:, None] * self.out["b"]
        if self.moving:
            self.p += self._position_term(Y)
        self.q = c + y * cs + p0 * sn / w
        self.pq = p0 * cs - w * y * sn

    def step(self):
        h = 0.5 * self.dt
        m = self.matter.mass[:, None]
        if self.splitting == "photon_exact":
            self._h2_flow(h)
            self.r += self.dt * self.p / m
            if self.moving:
                self._mode_functions()
            self._evaluate_matter()
            self.D = forward(self.U, self.lam, self.out["M"])
            self._h2_flow(h)
            self._coupling_force()
        elif self.splitting == "strang":
            self._kick(h)
            self.r += self.dt * self.p / m
            self.q, self.pq = rotate(self.q, self.pq, self.omega, self.dt)
            self._evaluate_matter()
            self.D = forward(self.U, self.lam, self.out["M"])
            self._coupling_force()
            self._kick(h)
        elif self.splitting == "paper":
            self._kick(h)
            self.r += self.dt * self.p / m
            self._evaluate_matter()
            self.D = forward(self.U, self.lam, self.out["M"])
            self._coupling_force()
            self._kick(h)
            self.q, self.pq = rotate(self.q, self.pq, self.omega, self.dt)
            self._coupling_force()               # forces at the rotated photon coordinates
        else:
            raise ValueError(self.splitting)
        self.step_count += 1

    def energies(self):
        m = self.matter.mass
        kin = float(np.sum(self.p ** 2 / (2.0 * m[:, None])))
        e_matter = float(np.sum(self.out["E"]))
        photon = float(np.sum(0.5 * self.pq ** 2 + 0.5 * (self.omega * self.q - self.D) ** 2))
        return {
            "kinetic": kin, "dftb": e_matter, "photon": photon,
            "coupling": float(-np.sum(self.omega * self.q * self.D)),
            "dse": float(0.5 * np.sum(self.D ** 2)),
            "photon_free": float(np.sum(0.5 * (self.pq ** 2 + (self.omega * self.q) ** 2))),
            "total": kin + e_matter + photon,
            "temperature": 2.0 * kin / (3.0 * len(m) * KB),
        }
