"""The Born-charge network on the GPU against the FP64 oracle of the same network, and what the
trained network gains over the Mulliken model it starts from. Forward, backward and weight
gradients run on the tcgen05 tensor cores (BF16 operands, FP32 accumulation).

Tolerances: the GPU evaluates the network in FP32 with the same bfloat16 weights the oracle uses
in FP64; a 128-term FP32 dot product with O(1) terms carries up to about 1e-5 absolute error, so
predicted tensors are compared at 2e-5 and gradients at 1e-4 of their largest entry."""
import numpy as np
import pytest

import cavmd_synth as cs
from cavmd_synth.params import ELEM_H, ELEM_O
from oracle import cavity as OC
from oracle import mlp as NN

pytestmark = pytest.mark.gpu
WATER = [ELEM_O, ELEM_H, ELEM_H]


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2512_03277_gb300 import build
    build.build()
    import paper_2512_03277_gb300 as P
    P.load_library()
    return P


def _labelled(n, seed, noise=0.06):
    """n thermal-like waters and their oracle central-FD Born tensors and Mulliken charges."""
    params = cs.load_water_params()
    pos = cs.water_batch(np.random.default_rng(seed), np.zeros((n, 3)), noise=noise)
    Z, Q = NN.born_fd_tensors(params, WATER, pos)
    return pos, Z.reshape(-1, 3, 3), Q.ravel()


def _random_params(seed):
    rng = np.random.default_rng(seed)
    d = NN.unpack(NN.init_params(rng))
    d["W3"] = rng.normal(0, 0.3, d["W3"].shape)
    d["b1"] = rng.normal(0, 0.1, d["b1"].shape)
    d["b3"] = rng.normal(0, 0.1, d["b3"].shape)
    return NN.pack(d).astype(np.float32)


def test_network_forward_and_gradient_match_oracle(P):
    from paper_2512_03277_gb300.cavmd import BornMLP
    pos, Z, Q = _labelled(40, seed=11)
    n = len(pos)
    species = np.tile(WATER, n)
    off = 3 * np.arange(n + 1)
    p = _random_params(3)
    net = BornMLP(p)
    net.cavmd_mlp_set_data(species, pos.reshape(-1, 3), Q, Z)
    X, R = NN.features_and_frames(species, pos.reshape(-1, 3), off)
    Zp = NN.born_tensors(NN.forward(NN.bf16_round(p), X)[0], R, Q, off)
    np.testing.assert_allclose(net.cavmd_mlp_predict(), Zp, rtol=0, atol=2e-5)
    L, g = NN.loss_and_grad(p, X, R, Q, off, Z)
    Lg, gg = net.cavmd_mlp_loss_grad()
    np.testing.assert_allclose(Lg, L, rtol=1e-5)
    np.testing.assert_allclose(gg, g, rtol=0, atol=1e-4 * np.abs(g).max())
    np.testing.assert_array_equal(net.cavmd_mlp_get_params(), NN.bf16_round(p).astype(np.float32))


def _trajectory_labelled(worker, cells, samples):
    """Geometries of one oracle 300 K trajectory (the recipe of oracle/born_dataset.py) and their
    oracle central-FD Born tensors and Mulliken charges."""
    from oracle import born_dataset as BD
    params = cs.load_water_params()
    pos = BD.trajectory_samples(worker, cells, equil=200, stride=10, samples=samples)
    Z, Q = NN.born_fd_tensors(params, WATER, pos)
    return pos, Z.reshape(-1, 3, 3), Q.ravel()


def test_trained_network_beats_mulliken_and_drives_the_dynamics(P):
    """Trained on the tensor cores on geometries of two 300 K oracle trajectories, tested on a third."""
    from paper_2512_03277_gb300.cavmd import BornMLP
    parts = [_trajectory_labelled(w, 120, 12) for w in (0, 1)]
    pos_tr = np.concatenate([p[0] for p in parts])
    Z_tr = np.concatenate([p[1] for p in parts])
    Q_tr = np.concatenate([p[2] for p in parts])
    pos_te, Z_te, Q_te = _trajectory_labelled(2, 120, 5)
    net = BornMLP(NN.init_params(np.random.default_rng(4)).astype(np.float32))
    net.cavmd_mlp_set_data(np.tile(WATER, len(pos_tr)), pos_tr.reshape(-1, 3), Q_tr, Z_tr)
    losses = net.cavmd_mlp_train(epochs=120, batch_cells=64, lr=2e-3, weight_decay=0.0, seed=5)
    assert losses[-1] < 0.2 * losses[0]
    params = net.cavmd_mlp_get_params()
    net.cavmd_mlp_set_data(np.tile(WATER, len(pos_te)), pos_te.reshape(-1, 3), Q_te, Z_te)
    Zp = net.cavmd_mlp_predict()
    mull = Q_te[:, None, None] * np.eye(3)
    err_net = np.sqrt(np.mean((Zp - Z_te) ** 2))
    err_mul = np.sqrt(np.mean((mull - Z_te) ** 2))
    assert err_net < 0.5 * err_mul, (err_net, err_mul)
    # the trained network drives a time step
    w = cs.make_workload("c1")
    sy, mo, pa = w["system"], w["modes"], w["params"]
    o = P.default_options()
    o.charge_model = 3
    ctx = P.Context(sy, pa, mo, o)
    ctx.cavmd_load_born_mlp(params)
    ctx.cavmd_step(20)
    obs = ctx.cavmd_observables()
    assert np.isfinite(obs["e_total"])


def test_network_inside_a_time_step_matches_oracle(P):
    """A seeded network (weights from a generator, not from training on the GPU) inside a time step:
    b equals the oracle network's b on the same cells, and the oracle's network charge model steps
    the same trajectory."""
    w = cs.make_workload("c1")
    sy, mo, pa = w["system"], w["modes"], w["params"]
    params = _random_params(8)
    o = P.default_options()
    o.charge_model = 3
    ctx = P.Context(sy, pa, mo, o)
    ctx.cavmd_load_born_mlp(params)
    ev = ctx.cavmd_get_eval()
    mat = OC.DFTBMatter(pa, sy, charge_model="network", mlp_params=params)
    md = OC.CavityMD(mat, sy.r, sy.p, mo.k, mo.omega, mo.lam, mo.phi, sy.R_ref, w["options"]["dt"])
    np.testing.assert_allclose(ev["b"], md.out["b"], rtol=0, atol=2e-5)    # pol = x
    for s in range(3):
        ctx.cavmd_step(1)
        md.step()
    st = ctx.cavmd_get_state()
    np.testing.assert_allclose(st["p"], md.p, rtol=0, atol=1e-5 * np.abs(md.p).max())


def test_shipped_network_on_fresh_trajectory_geometries(P):
    """The network shipped with the library (paper_2512_03277_gb300/data/born_mlp_water.f32, trained by
    train_born_mlp.py on the oracle's 300 K trajectory data) against the oracle's finite-difference
    Born tensors of geometries from a trajectory it never saw: its error is well below the Mulliken
    model's."""
    from paper_2512_03277_gb300 import cavmd as B
    params = B.trained_born_mlp()
    if params is None:
        pytest.skip("no trained network shipped")
    pos, Z, Q = _trajectory_labelled(101, 150, 4)
    net = B.BornMLP(params)
    net.cavmd_mlp_set_data(np.tile(WATER, len(pos)), pos.reshape(-1, 3), Q, None)
    Zp = net.cavmd_mlp_predict()
    err_net = np.sqrt(np.mean((Zp - Z) ** 2))
    err_mul = np.sqrt(np.mean((Q[:, None, None] * np.eye(3) - Z) ** 2))
    print(f"\nshipped network: held-out RMS {err_net:.4f} e, Mulliken {err_mul:.4f} e")
    assert err_net < 0.35 * err_mul, (err_net, err_mul)
