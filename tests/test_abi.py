"""The C ABI on a machine without a GPU: the library builds, loads, exports every function the
header declares, lays its structs out as the binding expects, and rejects invalid input on the
host before any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import cavmd_synth as cs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cavmd.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2512_03277_gb300 import build
    build.build()
    import paper_2512_03277_gb300 as P
    return P.load_library()


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(cavmd_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("cavmd_init", "cavmd_step", "cavmd_observables", "cavmd_get_state",
                     "cavmd_set_state", "cavmd_last_error", "cavmd_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), f"{name} declared in cavmd.h but not exported"


def test_struct_layouts_match_binding(lib):
    from paper_2512_03277_gb300 import cavmd as B
    for i, st in enumerate(B.STRUCTS):
        assert lib.cavmd_struct_size(i) == C.sizeof(st)


def test_default_options(lib):
    import paper_2512_03277_gb300 as P
    o = P.default_options()
    assert abs(o.dt - 0.5 * cs.FS) < 1e-12
    assert o.scc_tol == 1e-12 and o.precision == 0 and o.charge_model == 0 and o.splitting == 0


def _init_rc(lib, system, params, modes, opt=None, lattice=None):
    """Call cavmd_init through the C ABI and return (rc, message). Invalid inputs are rejected
    by host-side validation before any CUDA call, so this runs without a GPU."""
    from paper_2512_03277_gb300 import cavmd as B
    opt = B.default_options() if opt is None else opt
    sysc = B.cavmd_system()
    off = np.ascontiguousarray(system.cell_offset, np.int32)
    spec = np.ascontiguousarray(system.species, np.int32)
    r = np.ascontiguousarray(system.r, np.float64).ravel()
    p = np.ascontiguousarray(system.p, np.float64).ravel()
    sysc.n_cells, sysc.n_atoms = len(off) - 1, len(spec)
    sysc.cell_offset, sysc.species = B._ptr(off, C.c_int32), B._ptr(spec, C.c_int32)
    sysc.r, sysc.p = B._ptr(r), B._ptr(p)
    if lattice is not None:
        lat = np.ascontiguousarray(lattice, np.float64).reshape(9)
        sysc.lattice = B._ptr(lat)
    md = B.cavmd_modes()
    k = np.ascontiguousarray(modes.k, np.float64).ravel()
    w, lam, phi = (np.ascontiguousarray(x, np.float64) for x in (modes.omega, modes.lam, modes.phi))
    md.n_modes = len(w)
    md.k, md.omega, md.lambda_, md.phi = B._ptr(k), B._ptr(w), B._ptr(lam), B._ptr(phi)
    md.pol[:] = [1.0, 0.0, 0.0]
    sk = B.sk_tables(params)
    h = C.c_void_p()
    rc = lib.cavmd_init(C.byref(h), C.byref(sysc), C.byref(sk), C.byref(md), C.byref(opt))
    assert not h.value
    return rc, lib.cavmd_last_error(None).decode()


@pytest.fixture(scope="module")
def small():
    return cs.make_workload("c1", n_cells=2)


def test_rejects_negative_frequency(lib, small):
    m = small["modes"]
    m2 = cs.Modes(k=m.k, omega=-m.omega, lam=m.lam, phi=m.phi)
    rc, msg = _init_rc(lib, small["system"], small["params"], m2)
    assert rc == -1 and "frequenc" in msg


def test_rejects_bad_cell_offsets(lib, small):
    s = small["system"]
    bad = cs.System(species=s.species, cell_offset=np.array([0, 3, 5], np.int32), r=s.r, p=s.p, R_ref=s.R_ref)
    rc, msg = _init_rc(lib, bad, small["params"], small["modes"])
    assert rc == -1


def test_rejects_nonfinite_positions(lib, small):
    s = small["system"]
    r = s.r.copy()
    r[1, 2] = np.nan
    bad = cs.System(species=s.species, cell_offset=s.cell_offset, r=r, p=s.p, R_ref=s.R_ref)
    rc, _ = _init_rc(lib, bad, small["params"], small["modes"])
    assert rc == -1


def test_rejects_unsupported_composition(lib, small):
    """Clusters up to 64 orbitals are evaluated; (H2O)_11 has 66 and is refused before any device
    work, as is a cell with an odd orbital count (here an s-only element carrying two electrons)."""
    rng = np.random.default_rng(0)
    cl = cs.cluster_batch(rng, [11], np.zeros((1, 3)))
    cl.p = np.zeros_like(cl.r)
    rc, msg = _init_rc(lib, cl, small["params"], small["modes"])
    assert rc == -8 and "64" in msg
    pa = small["params"]
    odd = cs.System(species=np.array([1], np.int32), cell_offset=np.array([0, 1], np.int32),
                    r=np.zeros((1, 3)), p=np.zeros((1, 3)), R_ref=np.zeros((1, 3)))
    zval = pa.zval.copy()
    zval[1] = 2.0
    from dataclasses import replace
    rc, msg = _init_rc(lib, odd, replace(pa, zval=zval), small["modes"])
    assert rc == -8


def test_rejects_bad_options(lib, small):
    import paper_2512_03277_gb300 as P
    o = P.default_options()
    o.dt = 0.0
    assert _init_rc(lib, small["system"], small["params"], small["modes"], o)[0] == -1
    o = P.default_options()
    o.mixing = 1.5
    assert _init_rc(lib, small["system"], small["params"], small["modes"], o)[0] == -1
    o = P.default_options()
    o.mode_positions = 2
    assert _init_rc(lib, small["system"], small["params"], small["modes"], o)[0] == -1
    o = P.default_options()
    o.mode_positions = 1
    o.splitting = 2      # moving mode positions take the photon-exact splitting
    assert _init_rc(lib, small["system"], small["params"], small["modes"], o)[0] == -8
    o = P.default_options()
    o.jacobi_max_sweeps = 1001
    assert _init_rc(lib, small["system"], small["params"], small["modes"], o)[0] == -1
    o = P.default_options()
    o.splitting = 3
    assert _init_rc(lib, small["system"], small["params"], small["modes"], o)[0] == -1
    assert list(P.default_options().kgrid) == [1, 1, 1]
    for kg in ((3, 3, 3), (0, 1, 1), (9, 1, 1)):   # a grid on isolated cells; a partly zero or too fine grid
        o = P.default_options()
        o.kgrid[:] = kg
        assert _init_rc(lib, small["system"], small["params"], small["modes"], o)[0] == -1, kg


def test_rejects_empty_inputs(lib, small):
    """No cells, or no modes: refused on the host before any device work."""
    s = small["system"]
    empty = cs.System(species=np.zeros(0, np.int32), cell_offset=np.zeros(1, np.int32),
                      r=np.zeros((0, 3)), p=np.zeros((0, 3)), R_ref=np.zeros((0, 3)))
    assert _init_rc(lib, empty, small["params"], small["modes"])[0] == -1
    mo = small["modes"]
    none = cs.Modes(k=np.zeros((0, 3)), omega=np.zeros(0), lam=np.zeros(0), phi=np.zeros(0))
    assert _init_rc(lib, s, small["params"], none)[0] == -1


def test_periodic_cells_validation(lib, small):
    """Periodic cells: linearly dependent lattice vectors are invalid; the network charge model is
    refused as unsupported (Mulliken and finite-difference Born charges are built); both before any
    device work."""
    sy, lat = cs.periodic_water_cells(np.random.default_rng(5), np.zeros((1, 3)), n_waters=2, side=8.5,
                                      d_min=4.0, d_atom=2.8)
    flat = lat.copy()
    flat[2] = flat[0] + flat[1]
    rc, msg = _init_rc(lib, sy, small["params"], small["modes"], lattice=flat)
    assert rc == -1 and "lattice" in msg
    import paper_2512_03277_gb300 as P
    o = P.default_options()
    o.charge_model = 3
    rc, msg = _init_rc(lib, sy, small["params"], small["modes"], opt=o, lattice=lat)
    assert rc == -8 and "Mulliken" in msg
