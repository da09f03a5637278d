"""Plain FP64 CPU oracle of the per-atom Born-charge network.

TEST INFRASTRUCTURE ONLY (see oracle/dftb.py).

The paper obtains dmu/dr (Born charges) by forward finite differences, "the computational
bottleneck", or replaces them with Mulliken charges, which is cheap but makes the coupling
force non-conservative and heats the system (Results). A small per-atom network stands in:

  features x_j (32): radial symmetry functions per neighbour element (11 Gaussians x 2 elements),
      8 angular terms (zeta in {1, 2, 4, 8}, lambda in {+1, -1}) and the element one-hot of j,
      over the other atoms of j's cell within the cutoff r_c = 8 bohr;
  local frame R_j (rows e1, e2, e3): e1 towards the nearest neighbour, e2 the part of the vector to
      the second-nearest neighbour orthogonal to e1, e3 = e1 x e2;
  network: y = W3 s(W2 s(W1 x + b1) + b2) + b3, s(z) = z sigmoid(z) (SiLU), 32 -> 128 -> 128 -> 9,
      weights rounded to bfloat16 (round to nearest even);
  tensor: T_j = y reshaped 3 x 3 in the local frame, Z_lab_j = R_j^T T_j R_j;
  Born tensor: Z_j = Q_j I + Z_lab_j - mean_{k in cell} Z_lab_k  (Q_j the Mulliken net charge), so
      sum_j Z_j = Q_cell I holds exactly and a zero network gives the Mulliken charges;
  dipole derivative for polarisation pol: b_j[beta] = sum_alpha pol[alpha] Z_j[alpha][beta].

Loss: L = sum_j |Z_j - Z_j^ref|^2 / (9 n_atoms). Its gradient is written out by hand below and
pinned against finite differences in the tests.
"""
from __future__ import annotations

import numpy as np

NFEAT, HID, NOUT = 32, 128, 9
RC = 8.0
ETA_R = 2.0
MU_R = 0.8 + 0.7 * np.arange(11)
ETA_A = 0.05
ZETAS = (1.0, 2.0, 4.0, 8.0)
N_ELEM = 2
SHAPES = [("W1", (HID, NFEAT)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (NOUT, HID)), ("b3", (NOUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n], float).reshape(shp)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], float).ravel() for name, _ in SHAPES])


def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _fc(r):
    return np.where(r < RC, 0.5 * (np.cos(np.pi * r / RC) + 1.0), 0.0)


def features_and_frames(species, pos, cell_offset):
    """Per-atom features (n_atoms, 32) and local frames (n_atoms, 3, 3), intra-cell neighbours."""
    species = np.asarray(species)
    pos = np.asarray(pos, float)
    nat = len(species)
    X = np.zeros((nat, NFEAT))
    R = np.zeros((nat, 3, 3))
    for c in range(len(cell_offset) - 1):
        a0, a1 = cell_offset[c], cell_offset[c + 1]
        for j in range(a0, a1):
            nb = [k for k in range(a0, a1) if k != j and np.linalg.norm(pos[k] - pos[j]) < RC]
            d = {k: pos[k] - pos[j] for k in nb}
            r = {k: np.linalg.norm(d[k]) for k in nb}
            for k in nb:
                e = species[k]
                X[j, 11 * e:11 * e + 11] += np.exp(-ETA_R * (r[k] - MU_R) ** 2) * _fc(r[k])
            for a, k in enumerate(nb):
                for l in nb[a + 1:]:
                    cos = d[k] @ d[l] / (r[k] * r[l])
                    rad = np.exp(-ETA_A * (r[k] ** 2 + r[l] ** 2)) * _fc(r[k]) * _fc(r[l])
                    for zi, z in enumerate(ZETAS):
                        for li, lam in enumerate((1.0, -1.0)):
                            X[j, 22 + 2 * zi + li] += 2.0 ** (1.0 - z) * (1.0 + lam * cos) ** z * rad
            X[j, 30 + species[j]] = 1.0
            order = sorted(nb, key=lambda k: (r[k], k))
            k1, k2 = order[0], order[1]
            e1 = d[k1] / r[k1]
            v = d[k2] - (d[k2] @ e1) * e1
            e2 = v / np.linalg.norm(v)
            R[j] = np.stack([e1, e2, np.cross(e1, e2)])
    return X, R


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params_bf16, X):
    """Network outputs y (n, 9) and the activations needed by the backward pass."""
    p = unpack(params_bf16)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = silu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = silu(z2)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (X, z1, h1, z2, h2)


def born_tensors(y, R, Q, cell_offset):
    """Z_j = Q_j I + R^T T R - cell mean, from network outputs y (n, 9)."""
    T = y.reshape(-1, 3, 3)
    Zl = np.einsum("nai,nab,nbj->nij", R, T, R)
    Z = Zl.copy()
    for c in range(len(cell_offset) - 1):
        a0, a1 = cell_offset[c], cell_offset[c + 1]
        Z[a0:a1] -= Zl[a0:a1].mean(0)
    Z += np.asarray(Q, float)[:, None, None] * np.eye(3)
    return Z


def predict(params, species, pos, cell_offset, Q, round_bf16=True):
    X, R = features_and_frames(species, pos, cell_offset)
    y, _ = forward(bf16_round(params) if round_bf16 else np.asarray(params, float), X)
    return born_tensors(y, R, Q, cell_offset)


def loss_and_grad(params, X, R, Q, cell_offset, Zref, round_bf16=True):
    """Loss and its gradient with respect to the (bf16-rounded) parameters."""
    pb = bf16_round(params) if round_bf16 else np.asarray(params, float)
    p = unpack(pb)
    y, (X_, z1, h1, z2, h2) = forward(pb, X)
    Z = born_tensors(y, R, Q, cell_offset)
    n = len(X)
    diff = Z - Zref
    L = np.sum(diff ** 2) / (9 * n)
    gZ = 2.0 * diff / (9 * n)
    # through the cell-mean subtraction (a projection) and the rotation
    gZl = gZ.copy()
    for c in range(len(cell_offset) - 1):
        a0, a1 = cell_offset[c], cell_offset[c + 1]
        gZl[a0:a1] -= gZ[a0:a1].mean(0)
    gT = np.einsum("nai,nij,nbj->nab", R, gZl, R)
    gy = gT.reshape(n, 9)
    g = {"W3": gy.T @ h2, "b3": gy.sum(0)}
    gz2 = (gy @ p["W3"]) * dsilu(z2)
    g["W2"] = gz2.T @ h1
    g["b2"] = gz2.sum(0)
    gz1 = (gz2 @ p["W2"]) * dsilu(z1)
    g["W1"] = gz1.T @ X
    g["b1"] = gz1.sum(0)
    return L, pack(g)


def init_params(rng):
    """Seeded initial weights: uniform +-1/sqrt(fan_in), last layer and biases zero (the network
    starts as the Mulliken model)."""
    d = {}
    d["W1"] = rng.uniform(-1, 1, (HID, NFEAT)) / np.sqrt(NFEAT)
    d["b1"] = np.zeros(HID)
    d["W2"] = rng.uniform(-1, 1, (HID, HID)) / np.sqrt(HID)
    d["b2"] = np.zeros(HID)
    d["W3"] = np.zeros((NOUT, HID))
    d["b3"] = np.zeros(NOUT)
    return pack(d)


def born_fd_tensors(params_sk, species, pos, h=1e-3, q_ref=None):
    """Full central finite-difference Born tensors Z_j[alpha][beta] = d mu_alpha / d r_j,beta of a
    batch of molecules sharing `species`, pos (B, nat, 3). Returns (Z (B, nat, 3, 3), Q (B, nat))."""
    from . import dftb as D
    pos = np.asarray(pos, float)
    B, nat, _ = pos.shape
    ref = D.dftb(params_sk, species, pos, forces=False)
    Z = np.zeros((B, nat, 3, 3))
    for j in range(nat):
        for k in range(3):
            dp = pos.copy()
            dp[:, j, k] += h
            dm = pos.copy()
            dm[:, j, k] -= h
            mp = D.dftb(params_sk, species, dp, q0=ref["q"], forces=False)["mu"]
            mm = D.dftb(params_sk, species, dm, q0=ref["q"], forces=False)["mu"]
            Z[:, j, :, k] = (mp - mm) / (2 * h)
    return Z, ref["Q"]
