"""Error bound of the BF16x3 tensor-core coupling, derived from what the kernels do, and the
per-result bound arrays the GPU tests compare against.

Modes on a uniform in-plane grid, a = (jx, jy, cos|sin), with thx_n = dkx X_n and thy_n = dky Y_n.
The kernels contract the factorised phases cos|sin(jx thx_n) and cos|sin(jy thy_n) (cos(a + b) =
cos a cos b - sin a sin b, sin(a + b) = sin a cos b + cos a sin b), so the magnitude each D_a and
E_n is bounded against is the factorised one,
    mag(a, n) = |cos(jx thx) cos(jy thy)| + |sin(jx thx) sin(jy thy)|   (cos modes)
                |sin(jx thx) cos(jy thy)| + |cos(jx thx) sin(jy thy)|   (sin modes),
which is at least |u_a(R_n)| and at most 1.

Per-term error of one product ab. Each FP32 operand x is split x = h + l + e with h = bf16(x),
l = bf16(x - h): |x - h| <= 2^-8 |x|, |l| <= 2^-8 (1 + 2^-8) |x| and |e| <= 2^-16 |x|. The
kernel forms h_a h_b + h_a l_b + l_a h_b (each exact in FP32), which misses
l_a l_b + (h_a + l_a) e_b + e_a (h_b + l_b) + e_a e_b: at most 3.01 * 2^-16 |ab| = 4.59e-5 |ab|.
Operands are rounded to FP32 once (phases, M_n and the phase-times-M product, the weights W):
at most 4 * 2^-24 = 2.4e-7 more.

Forward D_a = lambda_a (G[..] -+ G[..]), G = A B^T over cells. Each TMEM accumulator covers one
32-cell stage: 6 MMAs (2 K-steps of 16 cells, 3 products each). Allowing each MMA 2^-22 of the
running sum of magnitudes (rounding or truncation of the FP32 accumulator and of the 16-product
sum) gives 6 * 2^-22 = 1.4e-6. Stages are folded into compensated (two-sum) FP32 sums: 2^-23
more. CTA partials are summed in FP64. Total below 4.8e-5 of lambda_a sum_n mag(a, n) |M_n|,
whatever the number of cells: EPS_D = 5e-5.

Back E_n = sum_i A[i][n] T[n][i], T = Wt Y^T over the KY <= 128 y-phase columns in one fresh
accumulator: 8 K-steps x 3 MMAs = 24 MMAs, 24 * 2^-22 = 5.7e-6. The epilogue sums 32 rows at a
time in FP32 (32 * 2^-24 = 1.9e-6) and the chunks in FP64. Total below 5.4e-5 of
sum_a mag(a, n) |W_a| (W_a carries lambda_a): EPS_E = 6e-5.

Moving mode positions. The panels are rebuilt every step at the centres of mass with FP32 phases
from an exact fixed-point reduction of the angle: the remainder is truncated to FP32 (below 2^-23
relative) and sincospif adds at most 1 ulp (2^-23 relative), so each phase factor carries up to
2^-22 instead of 2^-24; with both factors of a term that adds 6 * 2^-24 = 3.6e-7 to either total.
The field's gradient G_n = sum_a W_a grad u_a(R_n) (k_a in plane, G_z = 0) comes from the same
products: G_x scales the x phase rows by -+ jx dkx in the FP32 epilogue, G_y uses weights scaled by
-+ jy dky in FP32 (each scale and product adds 2^-24 twice). The magnitude it is bounded against is
that of the derivative of the factorised phases,
    mag'(a, n) = |sin(jx thx) cos(jy thy)| + |cos(jx thx) sin(jy thy)|   (cos modes)
                 |cos(jx thx) cos(jy thy)| + |sin(jx thx) sin(jy thy)|   (sin modes),
times jx dkx (G_x) or jy dky (G_y): below 5.5e-5 of sum_a |k_a,x| mag'(a, n) |W_a|, EPS_G = 6e-5.
"""
import concurrent.futures as cf
import os

import numpy as np

EPS_D = 5e-5
EPS_E = 6e-5
EPS_G = 6e-5


def grid_indices(modes):
    """(jx, jy, s, dkx, dky) of modes on a uniform in-plane grid (s = 0 cos, 1 sin)."""
    kx, ky = modes.k[:, 0], modes.k[:, 1]
    dkx = kx[kx > 0].min() if np.any(kx > 0) else 1.0
    dky = ky[ky > 0].min() if np.any(ky > 0) else 1.0
    jx = np.rint(kx / dkx).astype(int)
    jy = np.rint(ky / dky).astype(int)
    s = (np.abs(modes.phi) > 1e-12).astype(int)
    return jx, jy, s, dkx, dky


def _tables(j, theta):
    """|cos(j theta_n)| and |sin(j theta_n)| for j = 0 .. max(j), shape (J, N)."""
    a = np.arange(j.max() + 1)[:, None] * theta[None, :]
    return np.abs(np.cos(a)), np.abs(np.sin(a))


def bounds(modes, R, M, W):
    """EPS_D lambda_a sum_n mag(a, n) |M_n| for every mode, and EPS_E sum_a mag(a, n) |W_a| for
    every cell (R: the cells' mode-function centres, M: their dipoles, W_a: the field weights)."""
    jx, jy, s, dkx, dky = grid_indices(modes)
    cx, sx = _tables(jx, dkx * R[:, 0])
    cy, sy = _tables(jy, dky * R[:, 1])
    aM = np.abs(M)
    Pcc = (cx * aM) @ cy.T
    Pss = (sx * aM) @ sy.T
    Psc = (sx * aM) @ cy.T
    Pcs = (cx * aM) @ sy.T
    magM = np.where(s == 0, Pcc[jx, jy] + Pss[jx, jy], Psc[jx, jy] + Pcs[jx, jy])
    bD = EPS_D * np.abs(modes.lam) * magM
    Wc = np.zeros((cx.shape[0], cy.shape[0]))
    Ws = np.zeros_like(Wc)
    np.add.at(Wc, (jx[s == 0], jy[s == 0]), np.abs(W[s == 0]))
    np.add.at(Ws, (jx[s == 1], jy[s == 1]), np.abs(W[s == 1]))
    magE = (np.sum(cx * (Wc @ cy), 0) + np.sum(sx * (Wc @ sy), 0) + np.sum(sx * (Ws @ cy), 0)
            + np.sum(cx * (Ws @ sy), 0))
    return bD, EPS_E * magE


def grad_bounds(modes, R, W):
    """EPS_G sum_a |k_a,x| mag'(a, n) |W_a| and the same with k_a,y for every cell: the bounds of the
    gradient components G_x, G_y of the field at the cells' centres R (G_z = 0 on the grid)."""
    jx, jy, s, dkx, dky = grid_indices(modes)
    cx, sx = _tables(jx, dkx * R[:, 0])
    cy, sy = _tables(jy, dky * R[:, 1])
    Wc = np.zeros((cx.shape[0], cy.shape[0]))
    Ws = np.zeros_like(Wc)
    np.add.at(Wc, (jx[s == 0], jy[s == 0]), np.abs(W[s == 0]))
    np.add.at(Ws, (jx[s == 1], jy[s == 1]), np.abs(W[s == 1]))
    out = []
    for ax, ay in ((dkx * np.arange(cx.shape[0]), np.ones(cy.shape[0])),
                   (np.ones(cx.shape[0]), dky * np.arange(cy.shape[0]))):
        Vc = Wc * ax[:, None] * ay[None, :]
        Vs = Ws * ax[:, None] * ay[None, :]
        # cos modes: |sx cy| + |cx sy|; sin modes: |cx cy| + |sx sy|
        mag = (np.sum(sx * (Vc @ cy), 0) + np.sum(cx * (Vc @ sy), 0) + np.sum(cx * (Vs @ cy), 0)
               + np.sum(sx * (Vs @ sy), 0))
        out.append(EPS_G * mag)
    return out[0], out[1]


def direct_gradient(modes, R, W, chunk=64):
    """The plain definition G_n = sum_a W_a grad u_a(R_n), grad u_a = -k_a sin(k_a . R + phi_a), over
    chunks of modes on the host's cores. Returns [N, 3]."""
    from oracle import cavity as OC
    nm = len(modes.lam)
    parts = [(a, min(nm, a + chunk)) for a in range(0, nm, chunk)]

    def one(ab):
        a, b = ab
        S = OC.mode_function_sines(modes.k[a:b], modes.phi[a:b], R)
        return -(S.T @ (W[a:b, None] * modes.k[a:b]))

    G = np.zeros((len(R), 3))
    with cf.ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        for g in ex.map(one, parts):
            G += g
    return G


def direct_forward_and_field(modes, R, M, W, chunk=64):
    """The plain definitions D_a = lambda_a sum_n u_a(R_n) M_n and E_n = sum_a u_a(R_n) W_a with
    u_a(R) = cos(k_a . R + phi_a) (the oracle's mode functions), over chunks of modes on the host's
    cores. Returns (D [M], E [N])."""
    from oracle import cavity as OC
    nm = len(modes.lam)
    parts = [(a, min(nm, a + chunk)) for a in range(0, nm, chunk)]

    def one(ab):
        a, b = ab
        U = OC.mode_functions(modes.k[a:b], modes.phi[a:b], R)
        return a, OC.forward(U, modes.lam[a:b], M), U.T @ W[a:b]

    D = np.empty(nm)
    E = np.zeros(len(M))
    with cf.ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        for a, d, e in ex.map(one, parts):
            D[a:a + len(d)] = d
            E += e
    return D, E
