"""The double-buffered read-out (cavmd_observables_async / cavmd_observables_wait).

Checked: an async read-out followed by its wait returns exactly what cavmd_observables returns
at the same point; in the pipelined loop (queue slot s % 2 after step s, collect slot (s - 1) % 2
after step s + 1 is queued) every collected energy equals the energy history's record of that
step, and the arrays equal a synchronous read-out taken then; misuse returns INVALID_ARG."""
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


def _ctx(P, **opt):
    w = cs.make_workload("c2", n_cells=40, n_modes=64)
    o = P.default_options()
    for k, v in opt.items():
        setattr(o, k, v)
    return P.Context(w["system"], w["params"], w["modes"], o)


def test_async_equals_synchronous(P):
    ctx = _ctx(P)
    ctx.cavmd_step(3)
    ctx.cavmd_observables_async(1)
    a = ctx.cavmd_observables_wait(1)
    b = ctx.cavmd_observables()
    for k in ("e_total", "e_kin", "e_photon", "step", "scc_iter_max"):
        assert a[k] == b[k], k
    for k in ("M", "q", "p", "D"):
        assert np.array_equal(a[k], b[k]), k


def test_pipelined_loop_reads_every_step(P):
    steps = 12
    ctx = _ctx(P, energy_history=64, graph_chunk=0)
    got = []
    for s in range(steps):
        ctx.cavmd_step(1)
        ctx.cavmd_observables_async(s % 2)
        if s > 0:
            got.append(ctx.cavmd_observables_wait((s - 1) % 2))
    got.append(ctx.cavmd_observables_wait((steps - 1) % 2))
    h = ctx.cavmd_energy_history(steps + 1)          # steps 0..steps
    assert [g["step"] for g in got] == list(range(1, steps + 1))
    for g in got:
        assert g["e_total"] == h[g["step"], 6] and g["e_kin"] == h[g["step"], 0]
    # the arrays of the last read-out are those of the final state
    last = ctx.cavmd_observables()
    for k in ("M", "q", "p", "D"):
        assert np.array_equal(got[-1][k], last[k]), k


def test_misuse_is_rejected(P):
    import paper_2512_03277_gb300 as PP
    ctx = _ctx(P)
    with pytest.raises(PP.CavmdError) as ex:
        ctx.cavmd_observables_wait(0)               # nothing queued
    assert ex.value.code == -1
    ctx.cavmd_observables_async(0, want_arrays=False)
    with pytest.raises(PP.CavmdError) as ex:
        ctx.cavmd_observables_wait(0, want_arrays=True)
    assert ex.value.code == -1
    with pytest.raises(PP.CavmdError) as ex:
        ctx.cavmd_observables_async(2)
    assert ex.value.code == -1
