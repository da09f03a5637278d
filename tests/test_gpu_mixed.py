"""Mixed-precision coupling (tensor cores, BF16x3 with FP32 accumulation) against the FP64 oracle.

The error bound is derived in tests/bf16x3.py from what the kernels do: every D_a lies within
EPS_D = 5e-5 of lambda_a sum_n mag(a, n) |M_n| of the exact contraction of the same dipoles, and
every field E_n within EPS_E = 6e-5 of sum_a mag(a, n) |W_a|, where mag(a, n) <= 1 is the
magnitude of the factorised phase product (Eq. hlm2 is the contraction). The bound does not grow
with the number of cells: each TMEM accumulator covers one 32-cell stage and the stages are folded
into compensated sums. The largest ratio of error to bound is printed."""
import numpy as np
import pytest

import cavmd_synth as cs
from oracle import cavity as OC

from bf16x3 import bounds

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


@pytest.mark.parametrize("name,n", [("c4", 300), ("c5", 700), ("c4", 5000)])
def test_mixed_coupling_within_bf16x3_bound(P, name, n):
    w = cs.make_workload(name, n_cells=n)
    sy, mo, pa = w["system"], w["modes"], w["params"]
    ctx = _ctx(P, w, precision=2)
    mat = OC.DFTBMatter(pa, sy)
    md = OC.CavityMD(mat, sy.r, sy.p, mo.k, mo.omega, mo.lam, mo.phi, sy.R_ref, w["options"]["dt"])
    ev = ctx.cavmd_get_eval()
    obs = ctx.cavmd_observables()
    U = md.U
    M_gpu = ev["M"]
    W = mo.lam * (mo.omega * obs["q"] - obs["D"])
    bound_D, bound_E = bounds(mo, sy.R_ref, M_gpu, W)
    own = OC.forward(U, mo.lam, M_gpu)            # exact contraction of the GPU's own dipoles
    err_D = np.abs(obs["D"] - own)
    assert np.all(err_D <= bound_D + 1e-300)
    # total force: the DFTB part is FP64, the field part carries the BF16x3 bound
    E_exact = U.T @ W
    F_ref = ev["F_dftb"] + E_exact[md.cell][:, None] * ev["b"]
    err_F = np.abs(ev["F_total"] - F_ref)
    bound_F = bound_E[md.cell][:, None] * np.abs(ev["b"]) + 1e-12
    assert np.all(err_F <= bound_F)
    print(f"\n{name} {n} cells: max |dD| / bound {np.max(err_D / (bound_D + 1e-300)):.3f}, "
          f"max |dF| / bound {np.max(err_F / bound_F):.3f}")
    # and the FP64 parts still match the oracle
    fs = np.abs(md.out["F"]).max()
    np.testing.assert_allclose(ev["F_dftb"], md.out["F"], rtol=0, atol=1e-9 * fs)


def test_mixed_trajectory_tracks_fp64(P):
    """Ten steps of the mixed and the FP64 GPU paths from the same state stay within the
    accumulated BF16x3 field error (about 1e-5 of the coupling force, itself about 1e-4 of the
    total force here)."""
    w = cs.make_workload("c4", n_cells=256)
    a = _ctx(P, w)
    b = _ctx(P, w, precision=2)
    a.cavmd_step(10)
    b.cavmd_step(10)
    sa, sb = a.cavmd_get_state(), b.cavmd_get_state()
    np.testing.assert_allclose(sb["p"], sa["p"], rtol=0, atol=1e-6 * np.abs(sa["p"]).max())
    np.testing.assert_allclose(sb["q"], sa["q"], rtol=0, atol=1e-4 * np.abs(sa["q"]).max())
    oa, ob = a.cavmd_observables(), b.cavmd_observables()
    np.testing.assert_allclose(ob["e_total"], oa["e_total"], rtol=1e-9)


def test_mixed_requires_grid_modes(P):
    import paper_2512_03277_gb300 as PP
    w = cs.make_workload("c2", n_cells=8)        # line modes: cos only at both ends, not a grid
    with pytest.raises(PP.CavmdError) as ex:
        _ctx(P, w, precision=2)
    assert ex.value.code == -8
