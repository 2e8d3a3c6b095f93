"""ctypes binding of the C ABI in include/rsv.h (argument marshalling only).

Every computation happens in librsv.so; this module converts numpy arrays and
torch tensors to pointers and rsv_* status codes to exceptions. There is no
fallback: if the library is missing, importing anything that needs it raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librsv.so")

RSV_C128 = 0
RSV_C64 = 1
PRECISIONS = {"c128": RSV_C128, "complex128": RSV_C128, "c64": RSV_C64, "complex64": RSV_C64}

ERRORS = {
    -1: "RSV_ERR_INVALID_ARG", -2: "RSV_ERR_OUT_OF_MEMORY", -3: "RSV_ERR_NOT_CONVERGED",
    -4: "RSV_ERR_TIMEOUT", -5: "RSV_ERR_CUDA", -6: "RSV_ERR_COINCIDENT_ATOMS", -7: "RSV_ERR_NOT_FOUND",
}


class RsvError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Problem_(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("dim", C.c_int32), ("positions_um", C.POINTER(C.c_double)),
                ("c6", C.c_double), ("t_ns", C.c_int32), ("omega_rows", C.c_int32), ("delta_rows", C.c_int32),
                ("phi_rows", C.c_int32), ("omega", C.POINTER(C.c_double)), ("delta", C.POINTER(C.c_double)),
                ("phi", C.POINTER(C.c_double)), ("initial_state", C.c_void_p)]


class Config_(C.Structure):
    _fields_ = [("dt_ns", C.c_int32), ("precision", C.c_int32), ("krylov_tol", C.c_double),
                ("m_max", C.c_int32), ("max_substeps", C.c_int32), ("obs_stride", C.c_int32),
                ("flags", C.c_int32)]


class Stats_(C.Structure):
    _fields_ = [("steps", C.c_int64), ("krylov_iterations", C.c_int64), ("substeps", C.c_int64),
                ("max_error_estimate", C.c_double), ("seconds", C.c_double), ("kernel_launches", C.c_int64),
                ("tile_passes", C.c_int32), ("segment_bits", C.c_int32), ("l2_partner_bits", C.c_int32),
                ("tile_order_bits", C.c_int32), ("krylov_dim_max", C.c_int32), ("strided_tile_bits", C.c_int32),
                ("phase_gauge_steps", C.c_int64)]


KERNEL_KINDS = ("pass_first", "pass_second", "control", "combine", "setup")


class ServerConfig_(C.Structure):
    _fields_ = [("slots", C.c_int32), ("batch_atoms", C.c_int32), ("memory_bytes", C.c_size_t),
                ("max_bypass_s", C.c_double)]


class KernelTimes_(C.Structure):
    _fields_ = [("ms", C.c_double * 5), ("launches", C.c_int64 * 5), ("bytes", C.c_double * 5),
                ("control_step_ms", C.c_double), ("control_steps", C.c_int64),
                ("control_check_ms", C.c_double), ("control_checks", C.c_int64)]


_lib = None


def lib():
    """The loaded librsv.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2510_09813_b300.build`")
        L = C.CDLL(LIB_PATH)
        P, I32, I64, U64, D, SZ = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double, C.c_size_t
        PD = C.POINTER(C.c_double)
        sig = {
            "rsv_create": (I32, [C.POINTER(P), I32, SZ, P]),
            "rsv_destroy": (None, [P]),
            "rsv_last_error": (C.c_char_p, []),
            "rsv_version": (C.c_char_p, []),
            "rsv_footprint_bytes": (SZ, [I32, I32, I32]),
            "rsv_pair_energies": (I32, [I32, I32, PD, D, PD]),
            "rsv_num_steps": (I32, [I32, I32]),
            "rsv_midpoint_parameters": (I32, [C.POINTER(Problem_), I32, PD, PD, PD, PD]),
            "rsv_apply_hamiltonian": (I32, [P, I32, I32, PD, PD, PD, PD, P, P]),
            "rsv_observe": (I32, [P, I32, I32, P, PD, PD]),
            "rsv_hamiltonian_create": (I32, [P, I32, I32, PD, PD, PD, PD, C.POINTER(P)]),
            "rsv_hamiltonian_apply": (I32, [P, P, P]),
            "rsv_hamiltonian_sync": (I32, [P]),
            "rsv_hamiltonian_destroy": (None, [P]),
            "rsv_hamiltonian_expectation": (I32, [P, P, PD]),
            "rsv_correlations": (I32, [P, I32, I32, P, PD]),
            "rsv_run_shots": (I32, [P, C.POINTER(Problem_), C.POINTER(Config_), I32, PD, PD, PD, PD, I32,
                                    C.POINTER(I32)]),
            "rsv_sample": (I32, [P, I32, I32, P, I64, U64, C.POINTER(C.c_uint64)]),
            "rsv_overlap": (I32, [P, I32, I32, P, P, PD]),
            "rsv_fidelity": (I32, [P, I32, I32, P, P, PD]),
            "rsv_request_bytes": (I32, [C.POINTER(Problem_), C.POINTER(Config_), C.POINTER(SZ)]),
            "rsv_check_bounded_wait": (I32, [P]),
            "rsv_run_batch": (I32, [P, C.POINTER(Problem_), I32, C.POINTER(Config_), C.POINTER(P)]),
            "rsv_lindblad_run": (I32, [P, C.POINTER(Problem_), C.POINTER(Config_), PD, PD, P, P, PD, I32,
                                       C.POINTER(I32), C.POINTER(Stats_)]),
            "rsv_gradient": (I32, [P, C.POINTER(Problem_), C.POINTER(Config_), PD, I32, PD, PD, PD, PD,
                                   C.POINTER(I64), C.POINTER(Stats_)]),
            "rsv_observe_static": (I32, [I32, I32, P, P, P]),
            "rsv_solver_create": (I32, [P, C.POINTER(Problem_), C.POINTER(Config_), C.POINTER(P)]),
            "rsv_solver_destroy": (None, [P]),
            "rsv_solver_step": (I32, [P, I32]),
            "rsv_solver_progress": (I32, [P, C.POINTER(I32), C.POINTER(I32)]),
            "rsv_solver_rewind": (I32, [P]),
            "rsv_solver_state_device": (I32, [P, C.POINTER(P), C.POINTER(SZ)]),
            "rsv_solver_get_state": (I32, [P, P, SZ]),
            "rsv_solver_set_state": (I32, [P, P, SZ]),
            "rsv_solver_set_state_device": (I32, [P, P, SZ]),
            "rsv_solver_occupations": (I32, [P, PD, I32, C.POINTER(I32)]),
            "rsv_solver_stats": (I32, [P, C.POINTER(Stats_)]),
            "rsv_solver_set_profiling": (I32, [P, I32]),
            "rsv_solver_kernel_times": (I32, [P, C.POINTER(KernelTimes_)]),
            "rsv_run": (I32, [P, C.POINTER(Problem_), C.POINTER(Config_), C.POINTER(P)]),
            "rsv_result_state": (I32, [P, P, SZ]),
            "rsv_result_state_device": (I32, [P, C.POINTER(P), C.POINTER(SZ)]),
            "rsv_result_occupations": (I32, [P, PD, I32, C.POINTER(I32)]),
            "rsv_result_sample": (I32, [P, I64, U64, C.POINTER(C.c_uint64)]),
            "rsv_result_stats": (I32, [P, C.POINTER(Stats_)]),
            "rsv_result_free": (None, [P]),
            "rsv_batch_create": (I32, [P, C.POINTER(Problem_), I32, C.POINTER(Config_), C.POINTER(P)]),
            "rsv_batch_run": (I32, [P]),
            "rsv_batch_state": (I32, [P, I32, P, SZ]),
            "rsv_batch_state_device": (I32, [P, I32, C.POINTER(P), C.POINTER(SZ)]),
            "rsv_batch_occupations": (I32, [P, I32, PD, I32, C.POINTER(I32)]),
            "rsv_batch_stats": (I32, [P, I32, C.POINTER(Stats_)]),
            "rsv_batch_destroy": (None, [P]),
            "rsv_result_times": (I32, [P, PD, PD]),
            "rsv_server_create": (I32, [P, C.POINTER(ServerConfig_), C.POINTER(P)]),
            "rsv_submit": (I32, [P, C.POINTER(Problem_), C.POINTER(Config_), C.POINTER(U64)]),
            "rsv_poll": (I32, [P, U64, I32, C.POINTER(P)]),
            "rsv_server_load": (I32, [P, C.POINTER(I32), C.POINTER(I32), C.POINTER(SZ)]),
            "rsv_server_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(code: int):
    if code != 0:
        raise RsvError(code, lib().rsv_last_error().decode())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def precision_code(p) -> int:
    if isinstance(p, int):
        return p
    return PRECISIONS[p]


def amp_dtype(precision) -> np.dtype:
    return np.dtype(np.complex64) if precision_code(precision) == RSV_C64 else np.dtype(np.complex128)


class ProblemArgs:
    """Keeps the numpy buffers of an rsv_problem alive while the struct is in use."""

    def __init__(self, positions, c6, t_ns, omega, delta, phi=None, initial_state=None):
        pos = _f64(positions)
        if pos.ndim != 2 or pos.shape[1] not in (2, 3):
            raise ValueError("positions must be [n][2] or [n][3]")
        n = pos.shape[0]

        def rows(a):
            a = _f64(a)
            if a.ndim == 1:
                a = a[None, :]
            if a.shape[1] != t_ns:
                raise ValueError("pulse length must equal t_ns")
            return np.ascontiguousarray(a)

        self.pos, self.om, self.de = pos, rows(omega), rows(delta)
        self.ph = rows(phi) if phi is not None else None
        self.init = None if initial_state is None else np.ascontiguousarray(initial_state)
        s = Problem_()
        s.n_atoms = n
        s.dim = pos.shape[1]
        s.positions_um = _dptr(self.pos)
        s.c6 = float(c6)
        s.t_ns = int(t_ns)
        s.omega_rows = self.om.shape[0]
        s.delta_rows = self.de.shape[0]
        s.phi_rows = 0 if self.ph is None else self.ph.shape[0]
        s.omega = _dptr(self.om)
        s.delta = _dptr(self.de)
        s.phi = _dptr(self.ph) if self.ph is not None else C.POINTER(C.c_double)()
        s.initial_state = None if self.init is None else self.init.ctypes.data
        self.struct = s
        self.n = n

    @classmethod
    def from_problem(cls, p, initial_state=None):
        return cls(p.positions, p.c6, p.t_ns, p.omega, p.delta, p.phi, initial_state)


FLAG_CONTROL_LAUNCH = 1


def make_config(dt_ns, precision="c128", krylov_tol=0.0, m_max=0, max_substeps=0, obs_stride=1,
                control_launch=False) -> Config_:
    c = Config_()
    c.dt_ns = int(dt_ns)
    c.precision = precision_code(precision)
    c.krylov_tol = float(krylov_tol)
    c.m_max = int(m_max)
    c.max_substeps = int(max_substeps)
    c.obs_stride = int(obs_stride)
    c.flags = FLAG_CONTROL_LAUNCH if control_launch else 0
    return c
