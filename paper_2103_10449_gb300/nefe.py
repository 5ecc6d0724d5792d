"""ctypes binding of libnefe.so (include/nefe.h): same names, argument marshalling only.

Every step of the computation runs in the library's CUDA kernels.  Device buffers passed
to the stateless calls are torch CUDA tensors (their data pointers are handed over);
PyTorch only provides device memory and streams.  Importing this module does not need a
GPU; calling into the library does, and a missing library raises instead of falling back.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

NEFE_OK, NEFE_EINVAL, NEFE_ENOMEM, NEFE_ECUDA, NEFE_EOVERFLOW = 0, -1, -2, -3, -4
NEFE_ENAN, NEFE_EDEGEN, NEFE_ETIMEOUT, NEFE_ESTATE = -6, -7, -8, -9
NEFE_ERR_NBR_OVERFLOW, NEFE_ERR_SHELL_OVERFLOW, NEFE_ERR_NAN, NEFE_ERR_DEGEN, NEFE_ERR_BOX = 1, 2, 4, 8, 16
NEFE_ERR_CELL, NEFE_ERR_TIMEOUT = 32, 64
NEFE_FP32, NEFE_FP64 = 0, 1
NEFE_POT_SW, NEFE_POT_EINSTEIN, NEFE_POT_UF = 0, 1, 2
NEFE_REF_EINSTEIN, NEFE_REF_UF = 0, 1
NEFE_UF_CAP = 256
NEFE_BARO_NONE, NEFE_BARO_ISO, NEFE_BARO_ANISO = 0, 1, 2
NEFE_SCHED_NONE, NEFE_SCHED_FL, NEFE_SCHED_RS, NEFE_SCHED_AS = 0, 1, 2, 3
NEFE_DCCI_TEMP, NEFE_DCCI_PRESS = 0, 1
CODE_SHIFT = 27
INDEX_MASK = (1 << CODE_SHIFT) - 1


class NefeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libnefe error {code}: {msg}")
        self.code = code


class nefe_sw_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("eps", "sigma", "A", "B", "p", "q", "a", "lambda3",
                                               "gamma", "cos0")]


class nefe_uf_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("p", "sigma", "T", "rc")]


class nefe_system_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("x", ctypes.POINTER(ctypes.c_double)),
                ("v", ctypes.POINTER(ctypes.c_double)), ("r0", ctypes.POINTER(ctypes.c_double)),
                ("box", ctypes.c_double * 3), ("mass", ctypes.c_double), ("pot", ctypes.c_int),
                ("k_int", ctypes.c_double)]


class nefe_schedule(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("direction", ctypes.c_int), ("nsteps", ctypes.c_long),
                ("k_E", ctypes.c_double), ("lambda_f", ctypes.c_double), ("P_GPa", ctypes.c_double),
                ("P0_GPa", ctypes.c_double), ("P1_GPa", ctypes.c_double), ("lambda0", ctypes.c_double),
                ("ref", ctypes.c_int)]


class nefe_adjoint_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("x", ctypes.POINTER(ctypes.c_double)),
                ("v", ctypes.POINTER(ctypes.c_double)), ("r0", ctypes.POINTER(ctypes.c_double)),
                ("box", ctypes.c_double * 3), ("mass", ctypes.c_double), ("dt", ctypes.c_double),
                ("T", ctypes.c_double), ("tdamp", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("sys_id", ctypes.c_uint64), ("kind", ctypes.c_int), ("direction", ctypes.c_int),
                ("nsched", ctypes.c_long), ("k_E", ctypes.c_double), ("lambda_f", ctypes.c_double),
                ("P_GPa", ctypes.c_double), ("skin", ctypes.c_double), ("nbr_cap", ctypes.c_int),
                ("checkpoint_every", ctypes.c_int)]


class nefe_results(ctypes.Structure):
    _fields_ = [("W", ctypes.c_double), ("lambda_", ctypes.c_double), ("step", ctypes.c_long),
                ("U", ctypes.c_double), ("U_E", ctypes.c_double), ("K", ctypes.c_double),
                ("T", ctypes.c_double), ("P", ctypes.c_double * 6), ("V", ctypes.c_double),
                ("box", ctypes.c_double * 3), ("dHdl", ctypes.c_double), ("H", ctypes.c_double),
                ("mean_H", ctypes.c_double), ("mean_dHdl", ctypes.c_double),
                ("mean_P", ctypes.c_double), ("mean_V", ctypes.c_double),
                ("P_target", ctypes.c_double), ("error", ctypes.c_uint)]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            if isinstance(v, ctypes.Array):
                v = np.array(v[:])
            d[name.rstrip("_")] = v
        return d


_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_dbl_p = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p

# name -> (argtypes); every function returns int except nefe_last_error
SIGNATURES = {
    "nefe_sw_params_silicon": [ctypes.POINTER(nefe_sw_params)],
    "nefe_cell_bin": [_vp, ctypes.c_int, _c_dbl_p, ctypes.c_double, _c_int_p, _vp, _vp, _vp, ctypes.c_int, _vp],
    "nefe_cell_bin_noalloc": [_vp, ctypes.c_int, _c_dbl_p, ctypes.c_double, _c_int_p, _vp, _vp, _vp, ctypes.c_int, _vp],
    "nefe_neighbor_build": [_vp, ctypes.c_int, _c_dbl_p, ctypes.c_double, ctypes.c_int, _vp, _vp, _c_int_p, _vp],
    "nefe_sw_forces": [_vp, ctypes.c_int, _c_dbl_p, ctypes.c_double, _vp, _vp, ctypes.c_int,
                       ctypes.POINTER(nefe_sw_params), ctypes.c_int, _vp, _vp, _vp, _c_int_p, _vp],
    "nefe_uf_forces": [_vp, ctypes.c_int, _c_dbl_p, ctypes.c_double, ctypes.c_double,
                       ctypes.POINTER(nefe_uf_params), ctypes.c_int, _vp, _vp, _vp, _vp],
    "nefe_set_uf_params": [_vp, ctypes.c_int, ctypes.POINTER(nefe_uf_params)],
    "nefe_sw_energy_grad": [_vp, ctypes.c_int, _c_dbl_p, ctypes.c_double, _vp, _vp, ctypes.c_int,
                            ctypes.POINTER(nefe_sw_params), ctypes.c_int, _vp, _vp, _vp],
    "nefe_sw_dual": [_vp, _vp, ctypes.c_int, _c_dbl_p, ctypes.c_double, _vp, _vp, ctypes.c_int,
                     ctypes.POINTER(nefe_sw_params), _c_dbl_p, _vp, _vp, _vp, _vp],
    "nefe_adjoint_create": [ctypes.POINTER(_vp), ctypes.c_int, _vp, ctypes.POINTER(nefe_adjoint_desc),
                            ctypes.POINTER(nefe_sw_params)],
    "nefe_adjoint_destroy": [_vp],
    "nefe_adjoint_set_params": [_vp, ctypes.POINTER(nefe_sw_params)],
    "nefe_adjoint_forward": [_vp, ctypes.c_long, _c_dbl_p],
    "nefe_adjoint_backward": [_vp, _c_dbl_p, _c_dbl_p, _c_dbl_p],
    "nefe_adjoint_tangent": [_vp, ctypes.c_long, _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_dbl_p],
    "nefe_adjoint_state": [_vp, _c_dbl_p, _c_dbl_p],
    "nefe_langevin_noise": [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, _vp, _vp],
    "nefe_create": [ctypes.POINTER(_vp), ctypes.c_int, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int],
    "nefe_destroy": [_vp],
    "nefe_add_system": [_vp, ctypes.POINTER(nefe_system_desc), _c_int_p],
    "nefe_set_sw_params": [_vp, ctypes.c_int, ctypes.POINTER(nefe_sw_params)],
    "nefe_set_thermostat": [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_uint64],
    "nefe_set_barostat": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double],
    "nefe_set_schedule": [_vp, ctypes.c_int, ctypes.POINTER(nefe_schedule)],
    "nefe_pair_dcci": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                       ctypes.c_double, ctypes.c_double, ctypes.c_long, _c_int_p],
    "nefe_set_trace": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_long],
    "nefe_setup": [_vp],
    "nefe_run": [_vp, ctypes.c_long],
    "nefe_sync": [_vp],
    "nefe_get_results": [_vp, ctypes.c_int, ctypes.POINTER(nefe_results)],
    "nefe_get_pair": [_vp, ctypes.c_int, _c_dbl_p, _c_dbl_p, _c_dbl_p, ctypes.POINTER(ctypes.c_uint)],
    "nefe_get_state": [_vp, ctypes.c_int, _c_dbl_p, _c_dbl_p, _c_dbl_p],
    "nefe_set_state": [_vp, ctypes.c_int, _c_dbl_p, _c_dbl_p],
    "nefe_get_trace": [_vp, ctypes.c_int, _c_dbl_p, ctypes.c_long, ctypes.POINTER(ctypes.c_long)],
    "nefe_save": [_vp, ctypes.c_char_p],
    "nefe_load": [_vp, ctypes.c_char_p],
    "nefe_autotune": [_vp],
    "nefe_get_tuning": [_vp, _c_int_p, _c_dbl_p],
    "nefe_set_tuning": [_vp, ctypes.c_int],
    "nefe_set_gather_tuning": [_vp, ctypes.c_int],
    "nefe_get_lanes": [_vp, _c_int_p],
    "nefe_set_list_tuning": [_vp, ctypes.c_int],
    "nefe_set_rebuild_policy": [_vp, ctypes.c_int],
    "nefe_check_barrier_timeout": [ctypes.c_int, ctypes.c_double],
    "nefe_set_cooperative_rebuild": [_vp, ctypes.c_int],
    "nefe_get_rebuild_policy": [_vp, _c_int_p],
    "nefe_launch_count": [_vp, ctypes.POINTER(ctypes.c_long)],
    "nefe_set_state_all": [_vp, _c_dbl_p, _c_dbl_p],
    "nefe_get_state_all": [_vp, _c_dbl_p, _c_dbl_p],
    "nefe_get_results_all": [_vp, ctypes.POINTER(nefe_results), ctypes.c_int],
    "nefe_get_list_stats": [_vp, ctypes.c_int, _c_dbl_p, _c_int_p, ctypes.POINTER(ctypes.c_long)],
    "nefe_get_shell_stats": [_vp, _c_dbl_p, _c_int_p],
    "nefe_set_profiling": [_vp, ctypes.c_int],
    "nefe_get_profile": [_vp, _c_dbl_p, ctypes.POINTER(ctypes.c_long)],
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libnefe.so (building it with nvcc first when missing or stale).  With the
    environment variable NEFE_DEBUG_BOUNDS=1 the process loads libnefe_debug.so instead, the
    same sources built with index checks on every atom index read from device data."""
    global _lib
    if _lib is not None:
        return _lib
    debug = os.environ.get("NEFE_DEBUG_BOUNDS", "0") == "1"
    path = _build.LIB_DEBUG if debug else _build.LIB
    if build_if_missing and _build.needs_build(debug):
        _build.build(debug=debug)
    if not os.path.exists(path):
        raise NefeError(NEFE_ECUDA, f"{path} is missing: run paper_2103_10449_gb300.build")
    L = ctypes.CDLL(path)
    for name, argtypes in SIGNATURES.items():
        fn = getattr(L, name)
        fn.argtypes = argtypes
        fn.restype = ctypes.c_int
    L.nefe_last_error.argtypes = []
    L.nefe_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(rc):
    if rc != NEFE_OK:
        raise NefeError(rc, load().nefe_last_error().decode())
    return rc


def _ptr(t):
    """Device pointer of a torch tensor (or None)."""
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    """cudaStream_t of a torch stream, a raw handle (int) or the current torch stream (None)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _box(box):
    return (ctypes.c_double * 3)(*[float(b) for b in box])


def nefe_sw_params_silicon() -> nefe_sw_params:
    p = nefe_sw_params()
    _check(load().nefe_sw_params_silicon(ctypes.byref(p)))
    return p


def params_from(seq) -> nefe_sw_params:
    return nefe_sw_params(*[float(v) for v in seq])


# ---------------------------------------------------------------------- stateless calls
def nefe_cell_bin(x, n, box, rcs, cell_of, cell_start, perm, ncell_cap, stream=None):
    nc3 = (ctypes.c_int * 3)()
    _check(load().nefe_cell_bin(_ptr(x), int(n), _box(box), float(rcs), nc3, _ptr(cell_of),
                                _ptr(cell_start), _ptr(perm), int(ncell_cap), _stream(stream)))
    return tuple(nc3)


NOALLOC_MAX_ATOMS = 65536
NOALLOC_MAX_CELLS = 65536


def nefe_cell_bin_noalloc(x, n, box, rcs, cell_of, cell_start, perm, ncell_cap, stream=None):
    """Same as nefe_cell_bin without any device allocation (fixed in-library scratch)."""
    nc3 = (ctypes.c_int * 3)()
    _check(load().nefe_cell_bin_noalloc(_ptr(x), int(n), _box(box), float(rcs), nc3, _ptr(cell_of),
                                        _ptr(cell_start), _ptr(perm), int(ncell_cap), _stream(stream)))
    return tuple(nc3)


def nefe_neighbor_build(x, n, box, rcs, cap, nbr, cnt, stream=None, check=True):
    ovf = ctypes.c_int(0)
    rc = load().nefe_neighbor_build(_ptr(x), int(n), _box(box), float(rcs), int(cap), _ptr(nbr), _ptr(cnt),
                                    ctypes.byref(ovf), _stream(stream))
    if check or rc not in (NEFE_OK, NEFE_EOVERFLOW):
        _check(rc)
    return ovf.value


def nefe_sw_forces(x, n, box, rcs, nbr, cnt, cap, prm, precision, f, e_atom=None, energy_virial=None,
                   stream=None):
    ovf = ctypes.c_int(0)
    _check(load().nefe_sw_forces(_ptr(x), int(n), _box(box), float(rcs), _ptr(nbr), _ptr(cnt), int(cap),
                                 ctypes.byref(prm), int(precision), _ptr(f), _ptr(e_atom),
                                 _ptr(energy_virial), ctypes.byref(ovf), _stream(stream)))
    return ovf.value


def uf_params(p=25.0, sigma=2.0, T=2200.0, rc=8.0) -> nefe_uf_params:
    return nefe_uf_params(float(p), float(sigma), float(T), float(rc))


def nefe_uf_forces(x, n, box, rcs, skin, uf, precision, f, e_atom=None, energy_virial=None, stream=None):
    _check(load().nefe_uf_forces(_ptr(x), int(n), _box(box), float(rcs), float(skin), ctypes.byref(uf),
                                 int(precision), _ptr(f), _ptr(e_atom), _ptr(energy_virial), _stream(stream)))


def nefe_sw_energy_grad(x, n, box, rcs, nbr, cnt, cap, prm, precision, f, energy_grad, stream=None):
    _check(load().nefe_sw_energy_grad(_ptr(x), int(n), _box(box), float(rcs), _ptr(nbr), _ptr(cnt), int(cap),
                                      ctypes.byref(prm), int(precision), _ptr(f), _ptr(energy_grad),
                                      _stream(stream)))


def nefe_sw_dual(x, w, n, box, rcs, nbr, cnt, cap, prm, dtheta, f, fd, out16, stream=None):
    dth = None if dtheta is None else (ctypes.c_double * 7)(*[float(v) for v in dtheta])
    _check(load().nefe_sw_dual(_ptr(x), _ptr(w), int(n), _box(box), float(rcs), _ptr(nbr), _ptr(cnt), int(cap),
                               ctypes.byref(prm), dth, _ptr(f), _ptr(fd), _ptr(out16), _stream(stream)))


def nefe_langevin_noise(seed, sys_id, step, n, precision, xi, stream=None):
    _check(load().nefe_langevin_noise(int(seed), int(sys_id), int(step), int(n), int(precision), _ptr(xi),
                                      _stream(stream)))


def nefe_check_barrier_timeout(device=0, limit_ms=50.0):
    """Return code of the grid barrier's time-limit check: NEFE_ETIMEOUT when the barrier that can
    never complete gave up by its limit (the expected outcome), NEFE_OK otherwise."""
    return load().nefe_check_barrier_timeout(int(device), float(limit_ms))


# ---------------------------------------------------------------------- context API
def _dp(a):
    return None if a is None else a.ctypes.data_as(_c_dbl_p)


class Context:
    """Owns one nefe_ctx; methods are the nefe_* context calls with numpy arguments."""

    def __init__(self, device=0, precision=NEFE_FP32, dt=0.001, skin=0.5, nbr_cap=48, stream=None):
        self._L = load()
        h = ctypes.c_void_p()
        s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        _check(self._L.nefe_create(ctypes.byref(h), int(device), s, int(precision), float(dt), float(skin),
                                   int(nbr_cap)))
        self.h = h
        self.n = []
        self._keep = []

    def close(self):
        if self.h is not None and self.h.value:
            self._L.nefe_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_system(self, x, box, v=None, r0=None, mass=28.0855, pot=NEFE_POT_SW, k_int=0.0):
        x = np.ascontiguousarray(x, dtype=np.float64)
        v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
        r0 = None if r0 is None else np.ascontiguousarray(r0, dtype=np.float64)
        d = nefe_system_desc(n=x.shape[0], x=_dp(x), v=_dp(v), r0=_dp(r0),
                             box=(ctypes.c_double * 3)(*[float(b) for b in box]), mass=float(mass),
                             pot=int(pot), k_int=float(k_int))
        sid = ctypes.c_int(-1)
        _check(self._L.nefe_add_system(self.h, ctypes.byref(d), ctypes.byref(sid)))
        self.n.append(x.shape[0])
        return sid.value

    def set_sw_params(self, sys, prm):
        _check(self._L.nefe_set_sw_params(self.h, int(sys), ctypes.byref(prm)))

    def set_uf_params(self, sys, uf):
        _check(self._L.nefe_set_uf_params(self.h, int(sys), ctypes.byref(uf)))

    def set_thermostat(self, sys, T, damp, seed):
        _check(self._L.nefe_set_thermostat(self.h, int(sys), float(T), float(damp), int(seed)))

    def set_barostat(self, sys, mode, P_GPa, pdamp):
        _check(self._L.nefe_set_barostat(self.h, int(sys), int(mode), float(P_GPa), float(pdamp)))

    def set_schedule(self, sys, kind, direction=1, nsteps=1, k_E=0.0, lambda_f=1.0, P_GPa=0.0, P0_GPa=0.0,
                     P1_GPa=0.0, lambda0=1.0, ref=NEFE_REF_EINSTEIN):
        s = nefe_schedule(kind=kind, direction=direction, nsteps=nsteps, k_E=k_E, lambda_f=lambda_f, P_GPa=P_GPa,
                          P0_GPa=P0_GPa, P1_GPa=P1_GPa, lambda0=lambda0, ref=ref)
        _check(self._L.nefe_set_schedule(self.h, int(sys), ctypes.byref(s)))

    def pair_dcci(self, a, b, T0, P0_GPa, mode, frm, to, nsteps):
        pid = ctypes.c_int(-1)
        _check(self._L.nefe_pair_dcci(self.h, int(a), int(b), float(T0), float(P0_GPa), int(mode), float(frm),
                                      float(to), int(nsteps), ctypes.byref(pid)))
        return pid.value

    def set_trace(self, sys, every, cap):
        _check(self._L.nefe_set_trace(self.h, int(sys), int(every), int(cap)))

    def setup(self):
        _check(self._L.nefe_setup(self.h))

    def run(self, nsteps):
        _check(self._L.nefe_run(self.h, int(nsteps)))

    def sync(self):
        _check(self._L.nefe_sync(self.h))

    def results(self, sys):
        r = nefe_results()
        _check(self._L.nefe_get_results(self.h, int(sys), ctypes.byref(r)))
        return r.as_dict()

    def pair(self, p):
        T, P, lam, err = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_uint()
        _check(self._L.nefe_get_pair(self.h, int(p), ctypes.byref(T), ctypes.byref(P), ctypes.byref(lam),
                                     ctypes.byref(err)))
        return T.value, P.value, lam.value, err.value

    def get_state(self, sys):
        n = self.n[sys]
        x = np.zeros((n, 3)); v = np.zeros((n, 3)); box = np.zeros(3)
        _check(self._L.nefe_get_state(self.h, int(sys), _dp(x), _dp(v), _dp(box)))
        return x, v, box

    def set_state(self, sys, x=None, v=None):
        x = None if x is None else np.ascontiguousarray(x, dtype=np.float64)
        v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
        _check(self._L.nefe_set_state(self.h, int(sys), _dp(x), _dp(v)))

    def trace(self, sys, cap=1 << 20):
        buf = np.zeros((cap, 9))
        n = ctypes.c_long(0)
        _check(self._L.nefe_get_trace(self.h, int(sys), _dp(buf), int(cap), ctypes.byref(n)))
        return buf[: n.value].copy()

    def save(self, path):
        _check(self._L.nefe_save(self.h, str(path).encode()))

    def load(self, path):
        _check(self._L.nefe_load(self.h, str(path).encode()))

    def autotune(self):
        _check(self._L.nefe_autotune(self.h))
        return self.tuning()

    def tuning(self):
        lanes, us = ctypes.c_int(), ctypes.c_double()
        _check(self._L.nefe_get_tuning(self.h, ctypes.byref(lanes), ctypes.byref(us)))
        return lanes.value, us.value

    def lanes(self):
        """(pass A, pass B, list build) lanes per atom in use."""
        out = (ctypes.c_int * 3)()
        _check(self._L.nefe_get_lanes(self.h, out))
        return tuple(out[:])

    def set_tuning(self, lanes, gather_lanes=None, list_lanes=None):
        _check(self._L.nefe_set_tuning(self.h, int(lanes)))
        if gather_lanes is not None:
            _check(self._L.nefe_set_gather_tuning(self.h, int(gather_lanes)))
        if list_lanes is not None:
            _check(self._L.nefe_set_list_tuning(self.h, int(list_lanes)))

    def set_rebuild_policy(self, all_systems):
        """1: every system rebuilds its list on a step where any system needs it; 0: each on its own."""
        _check(self._L.nefe_set_rebuild_policy(self.h, int(all_systems)))

    def set_cooperative_rebuild(self, on):
        """1: the list rebuild as one cooperative launch with grid barriers; 0: the kernel sequence."""
        _check(self._L.nefe_set_cooperative_rebuild(self.h, int(on)))

    def rebuild_policy(self):
        out = ctypes.c_int()
        _check(self._L.nefe_get_rebuild_policy(self.h, ctypes.byref(out)))
        return out.value

    def set_state_all(self, x=None, v=None):
        """x, v: host (Ntot, 3) float64 arrays (pinned memory makes the copy faster)."""
        _check(self._L.nefe_set_state_all(self.h, _dp(x), _dp(v)))

    def get_state_all(self, x=None, v=None):
        _check(self._L.nefe_get_state_all(self.h, _dp(x), _dp(v)))

    def results_all(self, count=None):
        count = len(self.n) if count is None else count
        arr = (nefe_results * max(1, count))()
        _check(self._L.nefe_get_results_all(self.h, arr, int(count)))
        return [arr[i].as_dict() for i in range(count)]

    def list_stats(self, sys=-1):
        m, mx, nb = ctypes.c_double(), ctypes.c_int(), ctypes.c_long()
        _check(self._L.nefe_get_list_stats(self.h, int(sys), ctypes.byref(m), ctypes.byref(mx), ctypes.byref(nb)))
        return m.value, mx.value, nb.value

    def shell_stats(self):
        mean = ctypes.c_double(0.0)
        mx = ctypes.c_int(0)
        _check(self._L.nefe_get_shell_stats(self.h, ctypes.byref(mean), ctypes.byref(mx)))
        return mean.value, mx.value

    def set_profiling(self, enable=True):
        _check(self._L.nefe_set_profiling(self.h, int(bool(enable))))

    def profile(self):
        """Mean durations (us) of force pass A and pass B over the last graph replay."""
        us, n = (ctypes.c_double * 2)(), ctypes.c_long()
        _check(self._L.nefe_get_profile(self.h, us, ctypes.byref(n)))
        return us[0], us[1], n.value

    def launch_count(self):
        c = ctypes.c_long(0)
        _check(self._L.nefe_launch_count(self.h, ctypes.byref(c)))
        return c.value


def _host_aos(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(n, 3)
    return a


class Adjoint:
    """Switching work W(theta) of one FP64 NVT switching run and its derivatives (adjoint sweep
    over checkpointed segments, or a tangent-linear run) through the C ABI."""

    def __init__(self, x, v, box, prm=None, kind=NEFE_SCHED_FL, r0=None, direction=1, nsched=1000,
                 k_E=5.0, lambda_f=1.0, P_GPa=0.0, T=400.0, tdamp=0.1, seed=1, sys_id=0, mass=28.0855,
                 dt=0.001, skin=0.5, nbr_cap=48, checkpoint_every=45, device=0, stream=None):
        self.n = len(x)
        self._x = _host_aos(x, self.n)
        self._v = _host_aos(v, self.n)
        self._r0 = None if r0 is None else _host_aos(r0, self.n)
        d = nefe_adjoint_desc()
        d.n = self.n
        d.x = self._x.ctypes.data_as(_c_dbl_p)
        d.v = self._v.ctypes.data_as(_c_dbl_p)
        d.r0 = None if self._r0 is None else self._r0.ctypes.data_as(_c_dbl_p)
        d.box[:] = [float(b) for b in box]
        d.mass, d.dt, d.T, d.tdamp = float(mass), float(dt), float(T), float(tdamp)
        d.seed, d.sys_id, d.kind, d.direction, d.nsched = int(seed), int(sys_id), int(kind), int(direction), int(nsched)
        d.k_E, d.lambda_f, d.P_GPa, d.skin = float(k_E), float(lambda_f), float(P_GPa), float(skin)
        d.nbr_cap, d.checkpoint_every = int(nbr_cap), int(checkpoint_every)
        self.prm = nefe_sw_params_silicon() if prm is None else (prm if isinstance(prm, nefe_sw_params) else params_from(prm))
        self._h = _vp()
        _check(load().nefe_adjoint_create(ctypes.byref(self._h), int(device), _stream(stream), ctypes.byref(d),
                                          ctypes.byref(self.prm)))

    def close(self):
        if self._h:
            load().nefe_adjoint_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, prm):
        self.prm = prm if isinstance(prm, nefe_sw_params) else params_from(prm)
        _check(load().nefe_adjoint_set_params(self._h, ctypes.byref(self.prm)))

    def forward(self, nsteps):
        W = ctypes.c_double(0.0)
        _check(load().nefe_adjoint_forward(self._h, int(nsteps), ctypes.byref(W)))
        return W.value

    def backward(self, initial_state=False):
        g = (ctypes.c_double * 7)()
        if initial_state:
            gx = np.zeros((self.n, 3))
            gv = np.zeros((self.n, 3))
            _check(load().nefe_adjoint_backward(self._h, g, gx.ctypes.data_as(_c_dbl_p), gv.ctypes.data_as(_c_dbl_p)))
            return np.array(g[:]), gx, gv
        _check(load().nefe_adjoint_backward(self._h, g, None, None))
        return np.array(g[:])

    def tangent(self, nsteps, dtheta, dx0=None, dv0=None):
        dth = (ctypes.c_double * 7)(*[float(v) for v in dtheta])
        ax = None if dx0 is None else _host_aos(dx0, self.n)
        av = None if dv0 is None else _host_aos(dv0, self.n)
        W = ctypes.c_double(0.0)
        dW = ctypes.c_double(0.0)
        _check(load().nefe_adjoint_tangent(self._h, int(nsteps), dth,
                                           None if ax is None else ax.ctypes.data_as(_c_dbl_p),
                                           None if av is None else av.ctypes.data_as(_c_dbl_p),
                                           ctypes.byref(W), ctypes.byref(dW)))
        return W.value, dW.value

    def state(self):
        x = np.zeros((self.n, 3))
        v = np.zeros((self.n, 3))
        _check(load().nefe_adjoint_state(self._h, x.ctypes.data_as(_c_dbl_p), v.ctypes.data_as(_c_dbl_p)))
        return x, v
