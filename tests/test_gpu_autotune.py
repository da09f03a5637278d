"""The launch-shape tuner: it changes how work maps to threads and blocks, never the arithmetic,
so tuned and untuned contexts follow bitwise identical trajectories."""
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


@pytest.mark.parametrize("name,n,kernel,extra", [
    ("c3", 40, "k_dftb_generic", {}),
    ("c2", 200, "dftb_kernel<3,6>", {}),
    ("c3", 12, "k_dftb_generic", {"charge_model": 1, "born_interval": 2}),
])
def test_tuned_and_default_shapes_give_identical_trajectories(P, name, n, kernel, extra):
    w = cs.make_workload(name, n_cells=n, n_modes=64)
    a = _ctx(P, w, autotune=0, **extra)
    b = _ctx(P, w, autotune=1, **extra)
    rep = b.cavmd_tuning()
    assert rep.startswith(kernel) and "candidates" in rep
    assert "not tuned" in a.cavmd_tuning()
    a.cavmd_step(5)
    b.cavmd_step(5)
    sa, sb = a.cavmd_get_state(), b.cavmd_get_state()
    for k in ("r", "p", "q", "pq"):
        assert np.array_equal(sa[k], sb[k]), k
