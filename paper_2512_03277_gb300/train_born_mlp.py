"""Train the Born-charge network on the GPU with the library's own kernels (cavmd_mlp_*).

Input: an .npz of water geometries and reference Born tensors, arrays
  pos (n, 3, 3)     bohr, atoms O, H, H of each water;
  Z   (n, 3, 3, 3)  Z[c, j, alpha, beta] = d mu_alpha / d r_{j, beta};
  Q   (n, 3)        Mulliken net charges of the geometry;
  test (n,)         True for the held-out geometries (disjoint trajectories).
Output: the trained parameters (CAVMD_MLP_NPARAMS little-endian float32 values, the bfloat16 weights
the time step loads with cavmd_load_born_mlp) and a JSON report with the held-out RMS error of the
network and of the Mulliken model (Z = Q I) it starts from.

Schedule: AdamW, batches of `batch` waters, the learning rate decayed by a cosine over the epochs
(one cavmd_mlp_train call per epoch, the optimiser state carried across calls).

Usage: python -m paper_2512_03277_gb300.train_born_mlp DATA.npz --out W.f32 [--report R.json]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

NF, NH, NO = 32, 128, 9


def initial_params(seed: int = 4) -> np.ndarray:
    """Seeded start: weights uniform in +-1/sqrt(fan_in), the output layer and every bias zero,
    so the untrained network is the Mulliken model."""
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, (NH, NF)) / np.sqrt(NF)
    W2 = rng.uniform(-1, 1, (NH, NH)) / np.sqrt(NH)
    parts = [W1, np.zeros(NH), W2, np.zeros(NH), np.zeros((NO, NH)), np.zeros(NO)]
    return np.concatenate([x.ravel() for x in parts]).astype(np.float32)


def rms_errors(net, pos, Q, Z):
    """(network RMS, Mulliken RMS) of the Born tensors of the given waters."""
    n = len(pos)
    net.cavmd_mlp_set_data(np.tile([0, 1, 1], n), pos.reshape(-1, 3), Q.ravel(), None)
    Zp = net.cavmd_mlp_predict().reshape(n, 3, 3, 3)
    mul = Q[:, :, None, None] * np.eye(3)
    return float(np.sqrt(np.mean((Zp - Z) ** 2))), float(np.sqrt(np.mean((mul - Z) ** 2)))


def train(data, epochs=60, batch=256, lr=2e-3, weight_decay=0.0, seed=5, device=0, log=None):
    from .cavmd import BornMLP
    test = data["test"].astype(bool)
    tr = ~test
    pos, Z, Q = data["pos"], data["Z"], data["Q"]
    net = BornMLP(initial_params(), device=device)
    n = int(tr.sum())
    net.cavmd_mlp_set_data(np.tile([0, 1, 1], n), pos[tr].reshape(-1, 3), Q[tr].ravel(),
                           Z[tr].reshape(-1, 3, 3))
    t0 = time.time()
    losses = []
    for ep in range(epochs):
        lr_ep = 0.5 * lr * (1.0 + np.cos(np.pi * ep / epochs))
        losses.append(float(net.cavmd_mlp_train(1, batch, float(lr_ep), weight_decay, seed + ep)[0]))
        if log:
            log(f"epoch {ep + 1}/{epochs}: lr {lr_ep:.2e}, mean batch loss {losses[-1]:.4e}")
    t_train = time.time() - t0
    params = net.cavmd_mlp_get_params()
    e_net, e_mul = rms_errors(net, pos[test], Q[test], Z[test])
    e_tr, _ = rms_errors(net, pos[tr][:20000], Q[tr][:20000], Z[tr][:20000])
    net.cavmd_mlp_destroy()
    report = {"train_waters": n, "test_waters": int(test.sum()), "epochs": epochs, "batch_waters": batch,
              "lr": lr, "train_seconds": t_train, "loss_first_epoch": losses[0], "loss_last_epoch": losses[-1],
              "test_rms_network": e_net, "test_rms_mulliken": e_mul, "train_rms_network_first_20000": e_tr,
              "ratio_network_over_mulliken": e_net / e_mul}
    return params, report


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("data")
    ap.add_argument("--out", required=True)
    ap.add_argument("--report", default=None)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--device", type=int, default=0)
    a = ap.parse_args()
    d = dict(np.load(a.data))
    params, rep = train(d, a.epochs, a.batch, a.lr, device=a.device, log=print)
    np.asarray(params, "<f4").tofile(a.out)
    rep["recipe"] = str(d.get("recipe", ""))
    txt = json.dumps(rep, indent=1)
    print(txt)
    if a.report:
        with open(a.report, "w") as f:
            f.write(txt + "\n")


if __name__ == "__main__":
    main()
