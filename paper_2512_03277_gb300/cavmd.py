"""Thin ctypes binding of libcavmd.so (include/cavmd.h): same names, argument marshalling only.

Every step of the cavity-MD hot path runs inside the library's CUDA kernels; this module only
lays out the C structs, passes host arrays and reads results back. PyTorch supplies the device
memory (through the library's allocator callback) and the CUDA stream. There is no CPU fallback:
if the compiled library is missing, load_library() raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcavmd.so")

MAX_ELEM = 4
N_PHASES = 4
OK = 0
ERR = {-1: "INVALID_ARG", -2: "CUDA", -3: "SCC_NOCONV", -4: "NONFINITE", -5: "S_NOT_PD",
       -6: "ZERO_GAP", -7: "DEVICE_TIMEOUT", -8: "UNSUPPORTED", -9: "NOMEM"}
PREC_FP64, PREC_MIXED_TF32, PREC_MIXED_BF16X3 = 0, 1, 2
CHARGE_MULLIKEN, CHARGE_BORN_FD, CHARGE_BORN_CENTRAL, CHARGE_BORN_MLP = 0, 1, 2, 3
SPLIT_PHOTON_EXACT, SPLIT_STRANG, SPLIT_PAPER, SPLIT_REAL_SPACE = 0, 1, 2, 3
PHOTON_RELAXED, PHOTON_ZERO = 0, 1

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class cavmd_system(C.Structure):
    _fields_ = [("n_cells", C.c_int32), ("n_atoms", C.c_int32), ("cell_offset", _ip), ("species", _ip),
                ("r", _dp), ("p", _dp), ("R_ref", _dp), ("lattice", _dp)]


class cavmd_sk_tables(C.Structure):
    _fields_ = [("n_elem", C.c_int32), ("norb", C.c_int32 * MAX_ELEM), ("onsite", (C.c_double * 2) * MAX_ELEM),
                ("hubbard", C.c_double * MAX_ELEM), ("zval", C.c_double * MAX_ELEM),
                ("mass", C.c_double * MAX_ELEM), ("h0", C.c_double * (MAX_ELEM * MAX_ELEM * 16)),
                ("s", C.c_double * (MAX_ELEM * MAX_ELEM * 16)), ("rep", C.c_double * (MAX_ELEM * MAX_ELEM * 2)),
                ("r_cut", C.c_double), ("taper", C.c_double)]


class cavmd_modes(C.Structure):
    _fields_ = [("n_modes", C.c_int32), ("k", _dp), ("omega", _dp), ("lambda_", _dp), ("phi", _dp),
                ("pol", C.c_double * 3)]


class cavmd_options(C.Structure):
    _fields_ = [("dt", C.c_double), ("precision", C.c_int32), ("charge_model", C.c_int32),
                ("born_interval", C.c_int32), ("fd_step", C.c_double), ("scc_tol", C.c_double),
                ("scc_max_iter", C.c_int32), ("mixing", C.c_double), ("splitting", C.c_int32),
                ("photon_init", C.c_int32), ("graph_chunk", C.c_int32), ("device", C.c_int32),
                ("stream", C.c_void_p), ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN),
                ("alloc_user", C.c_void_p), ("energy_history", C.c_int32), ("acf_lags", C.c_int32),
                ("autotune", C.c_int32), ("scc_history", C.c_int32),
                ("mode_positions", C.c_int32), ("jacobi_max_sweeps", C.c_int32),
                ("real_space_g0", C.c_double), ("real_space_omega0", C.c_double),
                ("kgrid", C.c_int32 * 3)]


class cavmd_obs(C.Structure):
    _fields_ = [("e_kin", C.c_double), ("e_dftb", C.c_double), ("e_photon", C.c_double),
                ("e_coupling", C.c_double), ("e_dse", C.c_double), ("e_photon_free", C.c_double),
                ("e_total", C.c_double), ("temperature", C.c_double), ("step", C.c_int64),
                ("scc_iter_max", C.c_int32), ("M", _dp), ("q", _dp), ("p", _dp), ("D", _dp)]


class cavmd_state(C.Structure):
    _fields_ = [("r", _dp), ("p", _dp), ("q", _dp), ("pq", _dp), ("step", C.c_int64)]


class cavmd_eval(C.Structure):
    _fields_ = [("F_dftb", _dp), ("F_total", _dp), ("b", _dp), ("q_pop", _dp), ("E_cell", _dp), ("M", _dp),
                ("scc_iters", _ip)]


STRUCTS = [cavmd_system, cavmd_sk_tables, cavmd_modes, cavmd_options, cavmd_obs, cavmd_state, cavmd_eval]

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libcavmd.so and declare its entry points. Raises if the library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with python -m paper_2512_03277_gb300.build")
    lib = C.CDLL(path)
    lib.cavmd_default_options.argtypes = [C.POINTER(cavmd_options)]
    lib.cavmd_default_options.restype = None
    lib.cavmd_init.argtypes = [C.POINTER(C.c_void_p), C.POINTER(cavmd_system), C.POINTER(cavmd_sk_tables),
                               C.POINTER(cavmd_modes), C.POINTER(cavmd_options)]
    lib.cavmd_step.argtypes = [C.c_void_p, C.c_int64]
    lib.cavmd_observables.argtypes = [C.c_void_p, C.POINTER(cavmd_obs)]
    lib.cavmd_observables_async.argtypes = [C.c_void_p, C.c_int32, C.c_int32]
    lib.cavmd_observables_wait.argtypes = [C.c_void_p, C.c_int32, C.POINTER(cavmd_obs)]
    lib.cavmd_energy_history.argtypes = [C.c_void_p, _dp, C.c_int32, _ip]
    lib.cavmd_autocorrelation.argtypes = [C.c_void_p, _dp, C.c_int32, C.POINTER(C.c_int64), C.c_int32]
    lib.cavmd_tuning.argtypes = [C.c_void_p, C.c_char_p, C.c_int32]
    lib.cavmd_get_state.argtypes = [C.c_void_p, C.POINTER(cavmd_state)]
    lib.cavmd_set_state.argtypes = [C.c_void_p, C.POINTER(cavmd_state)]
    lib.cavmd_get_eval.argtypes = [C.c_void_p, C.POINTER(cavmd_eval)]
    lib.cavmd_phase_times.argtypes = [C.c_void_p, C.c_int32, _dp, C.POINTER(C.c_int64), C.c_int32]
    lib.cavmd_last_error.argtypes = [C.c_void_p]
    lib.cavmd_last_error.restype = C.c_char_p
    lib.cavmd_destroy.argtypes = [C.c_void_p]
    lib.cavmd_destroy.restype = None
    lib.cavmd_field_kick_noalloc.argtypes = [C.c_int32, C.c_int32] + [C.c_void_p] * 6 + [C.c_double] + \
        [C.c_void_p] * 4
    _fp = C.POINTER(C.c_float)
    lib.cavmd_mlp_create.argtypes = [C.POINTER(C.c_void_p), _fp, C.c_int32, C.c_int32]
    lib.cavmd_mlp_set_data.argtypes = [C.c_void_p, C.c_int32, _ip, _dp, _dp, _dp]
    lib.cavmd_mlp_loss_grad.argtypes = [C.c_void_p, _dp, _fp]
    lib.cavmd_mlp_train.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_float, C.c_float, C.c_uint64, _dp]
    lib.cavmd_mlp_predict.argtypes = [C.c_void_p, _dp]
    lib.cavmd_mlp_get_params.argtypes = [C.c_void_p, _fp]
    lib.cavmd_mlp_destroy.argtypes = [C.c_void_p]
    lib.cavmd_mlp_destroy.restype = None
    lib.cavmd_load_born_mlp.argtypes = [C.c_void_p, _fp, C.c_int32]
    lib.cavmd_struct_size.argtypes = [C.c_int32]
    lib.cavmd_struct_size.restype = C.c_size_t
    for i, st in enumerate(STRUCTS):
        if lib.cavmd_struct_size(i) != C.sizeof(st):
            raise RuntimeError(f"struct layout mismatch for {st.__name__}")
    _lib = lib
    return lib


class CavmdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR.get(code, code)}: {msg}")
        self.code = code


def _check(rc, ctx=None):
    if rc != OK:
        msg = load_library().cavmd_last_error(ctx).decode()
        raise CavmdError(rc, msg)


def _ptr(a, ctype=C.c_double):
    return a.ctypes.data_as(C.POINTER(ctype))


# --------------------------------------------------------------------------------- marshalling

def sk_tables(params) -> cavmd_sk_tables:
    """cavmd_sk_tables from a cavmd_synth.SKParams."""
    t = cavmd_sk_tables()
    ne = len(params.norb)
    t.n_elem = ne
    h0 = np.zeros((MAX_ELEM, MAX_ELEM, 4, 4))
    s = np.zeros((MAX_ELEM, MAX_ELEM, 4, 4))
    rep = np.zeros((MAX_ELEM, MAX_ELEM, 2))
    h0[:ne, :ne] = params.h0
    s[:ne, :ne] = params.s
    rep[:ne, :ne] = params.rep
    for e in range(ne):
        t.norb[e] = int(params.norb[e])
        t.onsite[e][0], t.onsite[e][1] = params.onsite[e]
        t.hubbard[e] = params.hubbard[e]
        t.zval[e] = params.zval[e]
        t.mass[e] = params.mass[e]
    t.h0[:] = h0.ravel().tolist()
    t.s[:] = s.ravel().tolist()
    t.rep[:] = rep.ravel().tolist()
    t.r_cut = params.r_cut
    t.taper = params.taper
    return t


def default_options() -> cavmd_options:
    o = cavmd_options()
    load_library().cavmd_default_options(C.byref(o))
    return o


NOALLOC_MAX_CELLS = 1048576


def cavmd_field_kick_noalloc(n_cells, n_modes, cell_offset, U, W, F, b, inv_mass, tau, p, E_out, e_kin_out,
                             stream=0):
    """The allocation-free field and kick of cavmd.h. Array arguments are device addresses (ints,
    e.g. torch tensor data_ptr()); E_out may be 0. Raises CavmdError on a nonzero status."""
    lib = load_library()
    rc = lib.cavmd_field_kick_noalloc(int(n_cells), int(n_modes), cell_offset, U, W, F, b, inv_mass, float(tau),
                                      p, E_out or None, e_kin_out, stream or None)
    _check(rc, None)


MLP_NPARAMS = 21897
BORN_MLP_WEIGHTS = os.path.join(HERE, "data", "born_mlp_water.f32")


def trained_born_mlp(path: str = BORN_MLP_WEIGHTS):
    """The trained Born-charge network shipped with the library (MLP_NPARAMS little-endian float32
    values in the order of cavmd_mlp_create), or None when the file is absent. It was trained by
    train_born_mlp.py on the oracle's finite-difference Born tensors of 300 K water geometries."""
    if not os.path.exists(path):
        return None
    a = np.fromfile(path, dtype="<f4")
    if a.size != MLP_NPARAMS or not np.all(np.isfinite(a)):
        raise ValueError(f"{path}: expected {MLP_NPARAMS} finite float32 values, found {a.size}")
    return a.astype(np.float32)


class BornMLP:
    """The library's Born-charge network (cavmd_mlp_* in cavmd.h): trained and evaluated on the
    GPU by the library's kernels. Arrays are host NumPy arrays."""

    def __init__(self, params, device=0):
        self.lib = load_library()
        p = np.ascontiguousarray(params, np.float32)
        if p.size != MLP_NPARAMS:
            raise ValueError("need MLP_NPARAMS parameters")
        self.handle = C.c_void_p()
        _check(self.lib.cavmd_mlp_create(C.byref(self.handle), _ptr(p, C.c_float), p.size, int(device)), None)
        self.n_cells = 0

    def cavmd_mlp_set_data(self, species, r, Q, Z_ref=None):
        sp = np.ascontiguousarray(species, np.int32).ravel()
        self.n_cells = sp.size // 3
        self._data = (sp, np.ascontiguousarray(r, np.float64).ravel(), np.ascontiguousarray(Q, np.float64).ravel(),
                      None if Z_ref is None else np.ascontiguousarray(Z_ref, np.float64).ravel())
        sp_, r_, Q_, Z_ = self._data
        _check(self.lib.cavmd_mlp_set_data(self.handle, self.n_cells, _ptr(sp_, C.c_int32), _ptr(r_), _ptr(Q_),
                                           None if Z_ is None else _ptr(Z_)), None)

    def cavmd_mlp_loss_grad(self):
        loss = C.c_double()
        g = np.empty(MLP_NPARAMS, np.float32)
        _check(self.lib.cavmd_mlp_loss_grad(self.handle, C.byref(loss), _ptr(g, C.c_float)), None)
        return loss.value, g

    def cavmd_mlp_train(self, epochs, batch_cells, lr, weight_decay=0.0, seed=0):
        el = np.empty(epochs)
        _check(self.lib.cavmd_mlp_train(self.handle, int(epochs), int(batch_cells), float(lr), float(weight_decay),
                                        int(seed), _ptr(el)), None)
        return el

    def cavmd_mlp_predict(self):
        Z = np.empty((3 * self.n_cells, 3, 3))
        _check(self.lib.cavmd_mlp_predict(self.handle, _ptr(Z)), None)
        return Z

    def cavmd_mlp_get_params(self):
        p = np.empty(MLP_NPARAMS, np.float32)
        _check(self.lib.cavmd_mlp_get_params(self.handle, _ptr(p, C.c_float)), None)
        return p

    def cavmd_mlp_destroy(self):
        if self.handle:
            self.lib.cavmd_mlp_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.cavmd_mlp_destroy()
        except Exception:
            pass


class Context:
    """Owns one cavmd_ctx plus the host arrays and callbacks it was built from.

    lattice: None for isolated cells, else the (3, 3) lattice vectors (rows, bohr) of periodic
    cells evaluated at the Gamma point (cavmd_system.lattice).

    device memory: from torch's caching allocator through the allocator callback (torch=True),
    else the library's own cudaMalloc; stream: a torch stream the library runs on."""

    def __init__(self, system, params, modes, options: cavmd_options | None = None, torch_memory=True,
                 lattice=None):
        lib = load_library()
        self.lib = lib
        self.opt = default_options() if options is None else options
        self._keep = []
        self.n_cells = int(system.n_cells)
        self.n_atoms = int(system.n_atoms)
        self.n_modes = int(modes.n_modes)
        self.cell_offset = np.ascontiguousarray(system.cell_offset, np.int32)
        self._torch_stream = None
        if torch_memory:
            import torch
            dev = int(self.opt.device)
            self._torch_stream = torch.cuda.Stream(device=dev)
            stream_handle = self._torch_stream.cuda_stream
            self.opt.stream = C.c_void_p(stream_handle)

            def _alloc(nbytes, user):
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, self._torch_stream)

            def _free(ptr, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc_cb = ALLOC_FN(_alloc)
            self._free_cb = FREE_FN(_free)
            self.opt.dev_alloc = self._alloc_cb
            self.opt.dev_free = self._free_cb
        sysc = cavmd_system()
        arrs = dict(off=self.cell_offset, spec=np.ascontiguousarray(system.species, np.int32),
                    r=np.ascontiguousarray(system.r, np.float64).ravel(),
                    p=np.ascontiguousarray(system.p, np.float64).ravel())
        self._keep.append(arrs)
        sysc.n_cells, sysc.n_atoms = self.n_cells, self.n_atoms
        sysc.cell_offset = _ptr(arrs["off"], C.c_int32)
        sysc.species = _ptr(arrs["spec"], C.c_int32)
        sysc.r, sysc.p = _ptr(arrs["r"]), _ptr(arrs["p"])
        if getattr(system, "R_ref", None) is not None:
            arrs["R"] = np.ascontiguousarray(system.R_ref, np.float64).ravel()
            sysc.R_ref = _ptr(arrs["R"])
        if lattice is not None:   # periodic cells: lattice vectors as rows, shared by every cell
            arrs["lat"] = np.ascontiguousarray(lattice, np.float64).reshape(9)
            sysc.lattice = _ptr(arrs["lat"])
        md = cavmd_modes()
        marr = dict(k=np.ascontiguousarray(modes.k, np.float64).ravel(),
                    w=np.ascontiguousarray(modes.omega, np.float64),
                    l=np.ascontiguousarray(modes.lam, np.float64),
                    f=np.ascontiguousarray(modes.phi, np.float64))
        self._keep.append(marr)
        md.n_modes = self.n_modes
        md.k, md.omega, md.lambda_, md.phi = _ptr(marr["k"]), _ptr(marr["w"]), _ptr(marr["l"]), _ptr(marr["f"])
        md.pol[:] = [float(x) for x in modes.pol]
        sk = sk_tables(params)
        self.handle = C.c_void_p()
        rc = lib.cavmd_init(C.byref(self.handle), C.byref(sysc), C.byref(sk), C.byref(md), C.byref(self.opt))
        _check(rc, None)

    # same names as the C ABI ------------------------------------------------------------------
    def cavmd_step(self, nsteps: int):
        _check(self.lib.cavmd_step(self.handle, int(nsteps)), self.handle)

    def cavmd_observables(self, want_arrays=True):
        o = cavmd_obs()
        out = {}
        if want_arrays:
            out["M"] = np.empty(self.n_cells)
            out["q"] = np.empty(self.n_modes)
            out["p"] = np.empty(self.n_modes)
            out["D"] = np.empty(self.n_modes)
            o.M, o.q, o.p, o.D = _ptr(out["M"]), _ptr(out["q"]), _ptr(out["p"]), _ptr(out["D"])
        _check(self.lib.cavmd_observables(self.handle, C.byref(o)), self.handle)
        for k in ("e_kin", "e_dftb", "e_photon", "e_coupling", "e_dse", "e_photon_free", "e_total",
                  "temperature", "step", "scc_iter_max"):
            out[k] = getattr(o, k)
        return out

    def cavmd_observables_async(self, slot: int, want_arrays: bool = True):
        """Queue the read-out of the current observables into staging slot 0 or 1 (no wait)."""
        _check(self.lib.cavmd_observables_async(self.handle, int(slot), int(want_arrays)), self.handle)

    def cavmd_observables_wait(self, slot: int, want_arrays: bool = True):
        """Wait for the read-out queued in `slot` and return it like cavmd_observables."""
        o = cavmd_obs()
        out = {}
        if want_arrays:
            out["M"] = np.empty(self.n_cells)
            out["q"] = np.empty(self.n_modes)
            out["p"] = np.empty(self.n_modes)
            out["D"] = np.empty(self.n_modes)
            o.M, o.q, o.p, o.D = _ptr(out["M"]), _ptr(out["q"]), _ptr(out["p"]), _ptr(out["D"])
        _check(self.lib.cavmd_observables_wait(self.handle, int(slot), C.byref(o)), self.handle)
        for k in ("e_kin", "e_dftb", "e_photon", "e_coupling", "e_dse", "e_photon_free", "e_total",
                  "temperature", "step", "scc_iter_max"):
            out[k] = getattr(o, k)
        return out

    def cavmd_observables_wait_into(self, slot: int, obs: cavmd_obs):
        """cavmd_observables_wait into a pre-built cavmd_obs whose arrays the caller owns."""
        _check(self.lib.cavmd_observables_wait(self.handle, int(slot), C.byref(obs)), self.handle)

    def cavmd_observables_into(self, obs: cavmd_obs):
        """Fill a pre-built cavmd_obs whose arrays the caller owns (no Python allocation)."""
        _check(self.lib.cavmd_observables(self.handle, C.byref(obs)), self.handle)

    def cavmd_energy_history(self, n: int):
        buf = np.empty((n, 8))
        got = C.c_int32()
        _check(self.lib.cavmd_energy_history(self.handle, _ptr(buf), n, C.byref(got)), self.handle)
        return buf[:got.value]

    def cavmd_autocorrelation(self, reset: bool = False):
        """(acf [M + 1, L], n): the device-accumulated correlation functions of the photon
        coordinates (rows 0..M-1) and the total dipole (row M), and the number of samples."""
        L = self.opt.acf_lags
        buf = np.empty((self.n_modes + 1, L))
        n = C.c_int64()
        _check(self.lib.cavmd_autocorrelation(self.handle, _ptr(buf), L, C.byref(n), int(reset)), self.handle)
        return buf, n.value

    def cavmd_tuning(self) -> str:
        buf = C.create_string_buffer(2048)
        _check(self.lib.cavmd_tuning(self.handle, buf, len(buf)), self.handle)
        return buf.value.decode()

    def cavmd_get_state(self):
        st = cavmd_state()
        out = dict(r=np.empty((self.n_atoms, 3)), p=np.empty((self.n_atoms, 3)),
                   q=np.empty(self.n_modes), pq=np.empty(self.n_modes))
        st.r, st.p, st.q, st.pq = _ptr(out["r"]), _ptr(out["p"]), _ptr(out["q"]), _ptr(out["pq"])
        _check(self.lib.cavmd_get_state(self.handle, C.byref(st)), self.handle)
        out["step"] = st.step
        return out

    def cavmd_set_state(self, state):
        st = cavmd_state()
        arr = {k: np.ascontiguousarray(state[k], np.float64) for k in ("r", "p", "q", "pq")}
        st.r, st.p, st.q, st.pq = _ptr(arr["r"]), _ptr(arr["p"]), _ptr(arr["q"]), _ptr(arr["pq"])
        st.step = int(state.get("step", 0))
        _check(self.lib.cavmd_set_state(self.handle, C.byref(st)), self.handle)

    def cavmd_get_eval(self):
        ev = cavmd_eval()
        out = dict(F_dftb=np.empty((self.n_atoms, 3)), F_total=np.empty((self.n_atoms, 3)),
                   b=np.empty((self.n_atoms, 3)), q_pop=np.empty(self.n_atoms), E_cell=np.empty(self.n_cells),
                   M=np.empty(self.n_cells), scc_iters=np.empty(self.n_cells, np.int32))
        ev.F_dftb, ev.F_total, ev.b = _ptr(out["F_dftb"]), _ptr(out["F_total"]), _ptr(out["b"])
        ev.q_pop, ev.E_cell, ev.M = _ptr(out["q_pop"]), _ptr(out["E_cell"]), _ptr(out["M"])
        ev.scc_iters = _ptr(out["scc_iters"], C.c_int32)
        _check(self.lib.cavmd_get_eval(self.handle, C.byref(ev)), self.handle)
        return out

    def cavmd_phase_times(self, enable: int, reset: bool = True):
        """enable: 0 off, 1 events around every launch, 2 around the SCC-DFTB launches only."""
        ms = np.zeros(N_PHASES)
        cnt = np.zeros(N_PHASES, np.int64)
        _check(self.lib.cavmd_phase_times(self.handle, int(enable), _ptr(ms), cnt.ctypes.data_as(C.POINTER(C.c_int64)),
                                          int(reset)), self.handle)
        return ms, cnt

    def cavmd_load_born_mlp(self, params):
        p = np.ascontiguousarray(params, np.float32)
        _check(self.lib.cavmd_load_born_mlp(self.handle, _ptr(p, C.c_float), p.size), self.handle)

    def cavmd_last_error(self) -> str:
        return self.lib.cavmd_last_error(self.handle).decode()

    def cavmd_destroy(self):
        if self.handle:
            self.lib.cavmd_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.cavmd_destroy()
        except Exception:
            pass

    @property
    def stream(self):
        return self._torch_stream
