"""Mixed-precision coupling (tensor cores, BF16x3 with FP32 accumulation) against the FP64 oracle.

Error bound used below: each operand x is split x = hi + lo with hi = bf16(x), lo = bf16(x - hi),
so |x - hi - lo| <= 2^-18 |x|; a product is formed as hi hi + hi lo + lo hi, dropping lo lo
(<= 2^-18 |ab|); with the FP32 inputs (2^-24) and FP32 accumulation over at most 64 cells per
CTA in these tests (64 * 2^-24), every D_a and E_n lies within 3e-5 of the sum of the absolute
values of its terms, lambda_a sum_n |u_a(R_n) M_n| and sum_a |u_a(R_n) W_a|."""
import numpy as np
import pytest

import cavmd_synth as cs
from oracle import cavity as OC

pytestmark = pytest.mark.gpu
REL = 3e-5


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


@pytest.mark.parametrize("name,n", [("c4", 300), ("c5", 700)])
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
    bound_D = REL * np.abs(mo.lam) * (np.abs(U) @ np.abs(M_gpu))
    own = OC.forward(U, mo.lam, M_gpu)            # exact contraction of the GPU's own dipoles
    assert np.all(np.abs(obs["D"] - own) <= bound_D + 1e-300)
    # total force: the DFTB part is FP64, the field part carries the BF16x3 bound
    W = mo.lam * (mo.omega * obs["q"] - obs["D"])
    E_exact = U.T @ W
    bound_E = REL * (np.abs(U).T @ np.abs(W))
    F_ref = ev["F_dftb"] + E_exact[md.cell][:, None] * ev["b"]
    bound_F = bound_E[md.cell][:, None] * np.abs(ev["b"]) + 1e-12
    assert np.all(np.abs(ev["F_total"] - F_ref) <= bound_F)
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
