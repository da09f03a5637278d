"""Closed forms of the harmonic test model (Rabi splitting).

TEST INFRASTRUCTURE ONLY (see oracle/dftb.py).

N identical oscillators of unit mass-weighted frequency omega_v with linear dipoles
M_n = d x_n couple to one k = 0 mode (u = 1, amplitude lambda, frequency omega_c):
    H = sum_n 1/2 (p_n^2 + omega_v^2 x_n^2) + 1/2 p^2 + 1/2 (omega_c q - lambda d sum_n x_n)^2.
Only the bright combination X = sum_n x_n / sqrt(N) couples, through lambda d sqrt(N). The two
polariton frequencies are the square roots of the eigenvalues of
    [[omega_v^2 + N lambda^2 d^2, -omega_c lambda d sqrt(N)], [-omega_c lambda d sqrt(N), omega_c^2]]
(the Jaynes-Cummings picture the paper appeals to in Results: splitting linear in the coupling).
For unit-mass-weighted coordinates with physical mass m, use d / sqrt(m) in place of d.
"""
import numpy as np


def polariton_frequencies(omega_v, omega_c, lam, d, n, mass=1.0):
    g = lam * (d / np.sqrt(mass)) * np.sqrt(n)
    K = np.array([[omega_v ** 2 + g * g, -omega_c * g], [-omega_c * g, omega_c ** 2]])
    w2 = np.linalg.eigvalsh(K)
    return np.sqrt(w2)
