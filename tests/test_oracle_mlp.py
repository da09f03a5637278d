"""Pins of the Born-charge network oracle: its hand-written gradient against finite differences
of the loss, rotation equivariance of the predicted tensors, the translation sum rule, the
Mulliken limit of a zero network, and the full finite-difference Born tensors against the
single-polarisation routine of the DFTB oracle."""
import numpy as np
import pytest

import cavmd_synth as cs
from cavmd_synth.params import ELEM_H, ELEM_O
from oracle import dftb as D
from oracle import mlp as NN

WATER = [ELEM_O, ELEM_H, ELEM_H]


def _cells(n, seed=0, noise=0.08):
    rng = np.random.default_rng(seed)
    pos = cs.water_batch(rng, np.zeros((n, 3)), noise=noise)
    species = np.tile(WATER, n)
    off = 3 * np.arange(n + 1)
    return species, pos.reshape(-1, 3), off, pos


def _random_params(seed=1, scale=0.3):
    rng = np.random.default_rng(seed)
    p = NN.init_params(rng)
    d = NN.unpack(p)
    d["W3"] = rng.normal(0, scale, d["W3"].shape)
    d["b1"] = rng.normal(0, 0.1, d["b1"].shape)
    d["b3"] = rng.normal(0, 0.1, d["b3"].shape)
    return NN.pack(d)


def test_gradient_matches_finite_differences():
    species, pos, off, _ = _cells(3)
    X, R = NN.features_and_frames(species, pos, off)
    rng = np.random.default_rng(2)
    Q = rng.normal(0, 0.3, len(species))
    Zref = rng.normal(0, 0.5, (len(species), 3, 3))
    p = _random_params()
    L, g = NN.loss_and_grad(p, X, R, Q, off, Zref, round_bf16=False)
    idx = rng.choice(NN.N_PARAMS, 60, replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (NN.loss_and_grad(pp, X, R, Q, off, Zref, round_bf16=False)[0]
              - NN.loss_and_grad(pm, X, R, Q, off, Zref, round_bf16=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g).max())


def test_rotation_equivariance_and_sum_rule():
    species, pos, off, _ = _cells(2, seed=3)
    rng = np.random.default_rng(4)
    Q = rng.normal(0, 0.3, len(species))
    for c in range(2):
        Q[3 * c:3 * c + 3] -= Q[3 * c:3 * c + 3].mean()
    p = _random_params()
    Z = NN.predict(p, species, pos, off, Q)
    Rm = cs.systems.random_rotations(rng, 1)[0]
    Z2 = NN.predict(p, species, pos @ Rm.T + 5.0, off, Q)
    np.testing.assert_allclose(Z2, np.einsum("ai,nij,bj->nab", Rm, Z, Rm), atol=1e-12)
    for c in range(2):
        np.testing.assert_allclose(Z[3 * c:3 * c + 3].sum(0), 0.0, atol=1e-12)


def test_zero_network_is_the_mulliken_model():
    species, pos, off, _ = _cells(2, seed=5)
    Q = np.array([-0.6, 0.3, 0.3, -0.5, 0.25, 0.25])
    p = NN.init_params(np.random.default_rng(0))
    Z = NN.predict(p, species, pos, off, Q)
    np.testing.assert_allclose(Z, Q[:, None, None] * np.eye(3), atol=1e-15)


def test_bf16_rounding_is_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -2.5 + 2 ** -10], np.float32)
    np.testing.assert_array_equal(NN.bf16_round(x), [1.0, 1.0, 1.0 + 2 ** -6, 1.0, -2.5])


def test_full_born_tensor_matches_single_polarisation_routine():
    params = cs.load_water_params()
    _, _, _, pos = _cells(2, seed=6)
    Z, Q = NN.born_fd_tensors(params, WATER, pos)
    for a, pol in enumerate(np.eye(3)):
        b = D.born_fd(params, WATER, pos, pol, h=1e-3, scheme="central")
        np.testing.assert_allclose(Z[:, :, a, :], b, atol=1e-12)
    np.testing.assert_allclose(Z.sum(1), 0.0, atol=1e-6)        # translation sum rule, O(h^2)


def test_network_charge_model_of_the_cavity_oracle():
    """The cavity oracle's 'network' dipole derivative: with a zero network it is the Mulliken
    model exactly (b_j = Q_j pol), and with any network it is pol^T Z_j of the network's Born
    tensors, a sum rule sum_j b_j = Q_cell pol = 0 holding for neutral cells."""
    from oracle import cavity as OC
    w = cs.make_workload("c1", n_cells=5)
    sy, pa = w["system"], w["params"]
    mul = OC.DFTBMatter(pa, sy)(sy.r)
    zero = OC.DFTBMatter(pa, sy, charge_model="network", mlp_params=np.zeros(NN.N_PARAMS))(sy.r)
    np.testing.assert_allclose(zero["b"], mul["b"], rtol=0, atol=1e-15)
    p = _random_params(seed=7)
    net = OC.DFTBMatter(pa, sy, charge_model="network", mlp_params=p)(sy.r)
    Z = NN.predict(p, sy.species, sy.r, sy.cell_offset, net["Q"])
    np.testing.assert_allclose(net["b"], Z[:, 0, :], rtol=0, atol=1e-14)     # pol = x
    np.testing.assert_allclose(net["b"].reshape(-1, 3, 3).sum(1), 0.0, atol=1e-12)
    assert np.abs(net["b"] - mul["b"]).max() > 1e-3
    with pytest.raises(ValueError):
        OC.DFTBMatter(pa, sy, charge_model="network")
