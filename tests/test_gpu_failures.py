"""The error codes of the C ABI, each caused by inputs the host accepts and the kernels' own checks
turn into a status (no fault, trap or unbounded wait on the GPU; every device loop involved is
bounded):
  S_NOT_PD        a water bent to 30 degrees (H...H 0.94 bohr): the synthetic overlap matrix has an
                  eigenvalue of -0.39 (checked against the oracle's S below), so its Cholesky factor
                  does not exist;
  ZERO_GAP        a cell of one oxygen atom: s^2 p^4 leaves one of three degenerate p levels empty,
                  so HOMO and LUMO coincide;
  NONFINITE       a state whose momentum is finite but whose kinetic energy overflows (|p| = 1e160):
                  the energy record of the evaluation is not finite;
  DEVICE_TIMEOUT  a cold start allowed one Jacobi sweep (options.jacobi_max_sweeps = 1) on cells
                  that need several;
and the context stays usable after a status: a good state set afterwards steps normally."""
import numpy as np
import pytest

import cavmd_synth as cs
from oracle import dftb as D

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


def _opts(P, **kw):
    o = P.default_options()
    o.scc_max_iter = 40
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _bent_water(angle_deg, r_oh=1.81):
    a = np.radians(angle_deg) / 2
    return np.array([[0.0, 0.0, 0.0], [r_oh * np.sin(a), r_oh * np.cos(a), 0.0],
                     [-r_oh * np.sin(a), r_oh * np.cos(a), 0.0]])


def _with_first_cell(w, pos):
    """The workload with its first water replaced by `pos` (centred where the first water was)."""
    sy = w["system"]
    r = sy.r.copy()
    r[0:3] = pos - pos.mean(0) + sy.r[0:3].mean(0)
    return cs.System(species=sy.species, cell_offset=sy.cell_offset, r=r, p=sy.p, R_ref=sy.R_ref)


def test_overlap_not_positive_definite(P):
    params = cs.load_water_params()
    pos = _bent_water(30.0)
    _, S = D.build_h0_s(params, D.Layout(params, [0, 1, 1]), pos[None])
    assert np.linalg.eigvalsh(S[0]).min() < -0.3          # the input really is indefinite
    w = cs.make_workload("c1")
    with pytest.raises(P.CavmdError) as ex:
        P.Context(_with_first_cell(w, pos), w["params"], w["modes"], _opts(P))
    assert ex.value.code == -5, str(ex.value)


def test_degenerate_homo_lumo(P):
    w = cs.make_workload("c1", n_cells=2)
    sy = w["system"]
    # cell 0: a lone oxygen atom (4 orbitals, 6 electrons); cell 1: a water
    species = np.concatenate([[0], sy.species[3:6]]).astype(np.int32)
    r = np.concatenate([sy.r[0:1], sy.r[3:6]])
    p = np.zeros_like(r)
    lone = cs.System(species=species, cell_offset=np.array([0, 1, 4], np.int32), r=r, p=p, R_ref=sy.R_ref)
    with pytest.raises(P.CavmdError) as ex:
        P.Context(lone, w["params"], w["modes"], _opts(P))
    assert ex.value.code == -6, str(ex.value)


def test_nonfinite_energy_then_recovery(P):
    w = cs.make_workload("c1")
    ctx = P.Context(w["system"], w["params"], w["modes"], _opts(P))
    good = ctx.cavmd_get_state()
    bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in good.items()}
    bad["p"][4, 0] = 1e160                                 # finite; its square is not
    with pytest.raises(P.CavmdError) as ex:
        ctx.cavmd_set_state(bad)
    assert ex.value.code == -4, str(ex.value)
    ctx.cavmd_set_state(good)                              # the context is still usable
    ctx.cavmd_step(3)
    obs = ctx.cavmd_observables()
    assert np.isfinite(obs["e_total"]) and obs["step"] == good["step"] + 3


@pytest.mark.parametrize("name,n", [("c1", 8), ("c3", 12)])
def test_cold_start_sweep_bound(P, name, n):
    """Waters take the lane-group kernel, clusters the persistent cluster kernel: both report the
    bound of their cold-start sweeps; the same cells with the default bound evaluate normally."""
    w = cs.make_workload(name, n_cells=n, n_modes=16)
    with pytest.raises(P.CavmdError) as ex:
        P.Context(w["system"], w["params"], w["modes"], _opts(P, jacobi_max_sweeps=1))
    assert ex.value.code == -7, str(ex.value)
    ctx = P.Context(w["system"], w["params"], w["modes"], _opts(P))
    ctx.cavmd_step(2)
    assert np.isfinite(ctx.cavmd_observables()["e_total"])


def test_sweep_bound_option_is_validated(P):
    w = cs.make_workload("c1")
    with pytest.raises(P.CavmdError) as ex:
        P.Context(w["system"], w["params"], w["modes"], _opts(P, jacobi_max_sweeps=-1))
    assert ex.value.code == -1
