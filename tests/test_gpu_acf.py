"""Device-accumulated autocorrelation functions against their definition.

The reference is computed here from the synchronised states copied to the host after every step
(photon coordinates q_a and the cell dipoles M_n, summed on the host):
    C_c(l) = 1/(n - l) sum_{t=l}^{n-1} (x_t - xbar)(x_{t-l} - xbar).
The device folds every sample into lag products in FP64 and removes the mean exactly at the end,
so the two agree to rounding (relative 1e-10 of C(0) allows for the cancellation of the mean)."""
import numpy as np
import pytest

import cavmd_synth as cs

pytestmark = pytest.mark.gpu


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


def _ctx(P, w, **opt):
    o = P.default_options()
    for k, v in opt.items():
        setattr(o, k, v)
    return P.Context(w["system"], w["params"], w["modes"], o)


def _definition(x, L):
    n = len(x)
    xb = x.mean(0)
    out = np.zeros((L,) + x.shape[1:])
    for l in range(min(L, n)):
        out[l] = ((x[l:] - xb) * (x[:n - l] - xb)).sum(0) / (n - l)
    return out


def _record(ctx, steps):
    rows = []
    o = ctx.cavmd_observables()
    rows.append(np.concatenate([o["q"], [o["M"].sum()]]))
    for _ in range(steps):
        ctx.cavmd_step(1)
        o = ctx.cavmd_observables()
        rows.append(np.concatenate([o["q"], [o["M"].sum()]]))
    return np.array(rows)


@pytest.mark.parametrize("L,steps", [(64, 300), (256, 100)])
def test_acf_matches_definition(P, L, steps):
    """Lags beyond the samples (L = 256 > 101 samples) are zero; the ring wraps for L = 64."""
    w = cs.make_workload("c1")
    ctx = _ctx(P, w, acf_lags=L, graph_chunk=0)
    x = _record(ctx, steps)
    acf, n = ctx.cavmd_autocorrelation()
    assert n == steps + 1 and acf.shape == (w["modes"].n_modes + 1, L)
    ref = _definition(x, L).T
    scale = np.abs(ref[:, :1]) + 1e-300
    assert np.all(np.abs(acf - ref) <= 1e-10 * scale), np.max(np.abs(acf - ref) / scale)
    if L > n:
        assert np.all(acf[:, n:] == 0.0)


def test_acf_graph_replay_and_reset(P):
    w = cs.make_workload("c2", n_cells=24, n_modes=32)
    a = _ctx(P, w, acf_lags=16, graph_chunk=0)
    b = _ctx(P, w, acf_lags=16, graph_chunk=5)
    a.cavmd_step(23)
    b.cavmd_step(23)
    ca, na = a.cavmd_autocorrelation(reset=True)
    cb, nb = b.cavmd_autocorrelation()
    assert na == nb == 24 and np.array_equal(ca, cb)
    # after a reset the accumulation restarts with the next step's sample
    a.cavmd_step(10)
    _, n = a.cavmd_autocorrelation()
    assert n == 10
    # set_state starts a new segment whose first sample is the state set
    st = a.cavmd_get_state()
    a.cavmd_set_state(st)
    _, n = a.cavmd_autocorrelation()
    assert n == 1


def test_acf_requires_lags(P):
    import paper_2512_03277_gb300 as PP
    w = cs.make_workload("c1", n_cells=2)
    ctx = _ctx(P, w)
    with pytest.raises(PP.CavmdError) as ex:
        ctx.cavmd_autocorrelation()
    assert ex.value.code == -1
