"""The allocation-free field and kick (cavmd_field_kick_noalloc) against the library's regular path.

Callers that cannot allocate device memory while they run (a framework that owns every byte of
the GPU through its own pool, a latency-critical loop where cudaMalloc would synchronise the
device, a plug-in whose host code may not allocate) use this entry point, so it has to give what
the regular time step gives. The regular path's output compared here is the total force of
cavmd_get_eval: F_total = F_dftb + E_n b_j with E_n = sum_a u_a(R_n) lambda_a (omega_a q_a - D_a).
With p = 0, tau = 1 and W_a = lambda_a (omega_a q_a - D_a), the allocation-free kick leaves exactly
that force in p. Two calls in a row check that the shared scratch is reused correctly.

This file is collected last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

import cavmd_synth as cs

pytestmark = pytest.mark.gpu

F_REL = 1e-9


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2512_03277_gb300 import build
    build.build()
    import paper_2512_03277_gb300 as P
    P.load_library()
    return torch, P


def test_noalloc_kick_matches_regular_path_on_two_calls(setup):
    torch, P = setup
    from paper_2512_03277_gb300 import cavmd as B
    w = cs.make_workload("c2", n_cells=53)           # 53 cells: a ragged last block of 32
    sy, mo, pa = w["system"], w["modes"], w["params"]
    ctx = P.Context(sy, pa, mo)
    ctx.cavmd_step(3)
    ev = ctx.cavmd_get_eval()
    obs = ctx.cavmd_observables()
    N, M = sy.n_cells, mo.n_modes
    dev = "cuda:0"
    U = np.cos(mo.k @ sy.R_ref.T + mo.phi[:, None])                 # [M][N], row-major
    W = mo.lam * (mo.omega * obs["q"] - obs["D"])
    inv_m = 1.0 / pa.mass[sy.species]
    t = {name: torch.tensor(np.ascontiguousarray(x), device=dev)
         for name, x in (("U", U), ("W", W), ("F", ev["F_dftb"].ravel()), ("b", ev["b"].ravel()),
                         ("im", inv_m))}
    off = torch.tensor(sy.cell_offset.astype(np.int32), device=dev)
    p = torch.zeros(3 * sy.n_atoms, dtype=torch.float64, device=dev)
    E = torch.empty(N, dtype=torch.float64, device=dev)
    ek = torch.empty(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    Ft = ev["F_total"].ravel()
    fs = np.abs(Ft).max()
    for call, expect in ((1, Ft), (2, 2.0 * Ft)):       # the second call kicks the first's result again
        B.cavmd_field_kick_noalloc(N, M, off.data_ptr(), t["U"].data_ptr(), t["W"].data_ptr(),
                                   t["F"].data_ptr(), t["b"].data_ptr(), t["im"].data_ptr(), 1.0,
                                   p.data_ptr(), E.data_ptr(), ek.data_ptr(), stream)
        torch.cuda.synchronize()
        got = p.cpu().numpy()
        np.testing.assert_allclose(got, expect, rtol=0, atol=call * F_REL * fs)
        kin = 0.5 * np.sum(got.reshape(-1, 3) ** 2 * inv_m[:, None])
        np.testing.assert_allclose(ek.item(), kin, rtol=1e-12)
        E_ref = U.T @ W
        np.testing.assert_allclose(E.cpu().numpy(), E_ref, rtol=0, atol=1e-13 * np.abs(E_ref).max() + 1e-300)
    ctx.cavmd_destroy()


def test_noalloc_rejects_sizes_beyond_its_scratch(setup):
    torch, P = setup
    from paper_2512_03277_gb300 import cavmd as B
    with pytest.raises(B.CavmdError) as ex:
        B.cavmd_field_kick_noalloc(B.NOALLOC_MAX_CELLS + 1, 1, 1, 1, 1, 1, 1, 1, 1.0, 1, 0, 1, 0)
    assert ex.value.code == -1 and "n_cells" in str(ex.value)
