"""Python front end of the rsv C ABI (same names as include/rsv.h, marshalling only).

PyTorch is used for device memory and streams: device buffers are torch CUDA
tensors (complex64 / complex128) and a Context runs on torch's current CUDA
stream unless given another one.
"""
from __future__ import annotations

import ctypes as C
import weakref

import numpy as np

from . import _lib as L
from ._lib import RSV_C64, RSV_C128, RsvError, amp_dtype, check, precision_code  # noqa: F401


CUDA_STREAM_LEGACY = 0x1  # cudaStreamLegacy handle value


def _torch():
    import torch
    return torch


class Context:
    """rsv_ctx: a device, a stream and a device-memory arena."""

    def __init__(self, device: int = 0, arena_bytes: int = 0, stream=None):
        torch = _torch()
        if stream is None:
            torch.cuda.set_device(device)
            stream = torch.cuda.current_stream(device).cuda_stream
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        if not stream:
            # torch's default stream is the legacy NULL stream; name it explicitly
            # (cudaStreamLegacy) so the library orders its work with torch's.
            stream = CUDA_STREAM_LEGACY
        self.device = device
        self._h = C.c_void_p()
        self._children = weakref.WeakSet()  # solvers/results to close before the context
        check(L.lib().rsv_create(C.byref(self._h), int(device), int(arena_bytes), C.c_void_p(stream)))

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("context is closed")
        return self._h

    def _adopt(self, child):
        self._children.add(child)

    def close(self):
        if self._h:
            for ch in list(self._children):
                ch.close()
            L.lib().rsv_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def version() -> str:
    return L.lib().rsv_version().decode()


def footprint_bytes(n_atoms: int, precision="c64", m_max: int = 30) -> int:
    return int(L.lib().rsv_footprint_bytes(int(n_atoms), precision_code(precision), int(m_max)))


def pair_energies(positions, c6: float) -> np.ndarray:
    pos = np.ascontiguousarray(np.asarray(positions, dtype=np.float64))
    n, dim = pos.shape
    out = np.empty((n, n))
    check(L.lib().rsv_pair_energies(n, dim, L._dptr(pos), float(c6), L._dptr(out)))
    return out


def num_steps(t_ns: int, dt_ns: int) -> int:
    return int(L.lib().rsv_num_steps(int(t_ns), int(dt_ns)))


def midpoint_parameters(problem, dt_ns: int):
    """(omega[K][n], delta[K][n], phi[K][n], tau_us[K]) by the midpoint rule."""
    pa = L.ProblemArgs.from_problem(problem)
    K = num_steps(problem.t_ns, dt_ns)
    om, de, ph, tau = np.empty((K, pa.n)), np.empty((K, pa.n)), np.empty((K, pa.n)), np.empty(K)
    check(L.lib().rsv_midpoint_parameters(C.byref(pa.struct), int(dt_ns), L._dptr(om), L._dptr(de),
                                          L._dptr(ph), L._dptr(tau)))
    return om, de, ph, tau


def _check_state(t, n, precision):
    torch = _torch()
    want = torch.complex64 if precision_code(precision) == RSV_C64 else torch.complex128
    if not (t.is_cuda and t.dtype == want and t.is_contiguous() and t.numel() == 2 ** n):
        raise ValueError(f"expected a contiguous CUDA {want} tensor of 2**{n} amplitudes")
    return C.c_void_p(t.data_ptr())


def apply_hamiltonian(ctx: Context, n_atoms: int, precision, v_pairs, omega, delta, phi, x, y):
    """y = H x (Eq. (3)) on CUDA tensors x, y."""
    V = np.ascontiguousarray(np.asarray(v_pairs, dtype=np.float64))
    om = np.ascontiguousarray(np.asarray(omega, dtype=np.float64))
    de = np.ascontiguousarray(np.asarray(delta, dtype=np.float64))
    ph = None if phi is None else np.ascontiguousarray(np.asarray(phi, dtype=np.float64))
    check(L.lib().rsv_apply_hamiltonian(
        ctx.handle, int(n_atoms), precision_code(precision), L._dptr(V), L._dptr(om), L._dptr(de),
        L._dptr(ph) if ph is not None else C.POINTER(C.c_double)(),
        _check_state(x, n_atoms, precision), _check_state(y, n_atoms, precision)))


class Hamiltonian:
    """rsv_hamiltonian: H of Eq. (3) prepared once for repeated y = H x."""

    def __init__(self, ctx: Context, n_atoms: int, precision, v_pairs, omega, delta, phi=None):
        self.ctx, self.n, self.precision = ctx, int(n_atoms), precision_code(precision)
        V = np.ascontiguousarray(np.asarray(v_pairs, dtype=np.float64))
        om = np.ascontiguousarray(np.asarray(omega, dtype=np.float64))
        de = np.ascontiguousarray(np.asarray(delta, dtype=np.float64))
        ph = None if phi is None else np.ascontiguousarray(np.asarray(phi, dtype=np.float64))
        self._h = C.c_void_p()
        check(L.lib().rsv_hamiltonian_create(ctx.handle, self.n, self.precision, L._dptr(V), L._dptr(om), L._dptr(de),
                                             L._dptr(ph) if ph is not None else C.POINTER(C.c_double)(),
                                             C.byref(self._h)))
        ctx._adopt(self)

    def apply(self, x, y):
        """Enqueue y = H x on the context stream (no synchronisation)."""
        check(L.lib().rsv_hamiltonian_apply(self._h, _check_state(x, self.n, self.precision),
                                            _check_state(y, self.n, self.precision)))

    def sync(self):
        check(L.lib().rsv_hamiltonian_sync(self._h))

    def expectation(self, psi) -> tuple[complex, float]:
        """(<psi|H|psi>, <psi|H^2|psi>) of a CUDA state tensor (unnormalised)."""
        out = np.empty(3)
        check(L.lib().rsv_hamiltonian_expectation(self._h, _check_state(psi, self.n, self.precision), L._dptr(out)))
        return complex(out[0], out[1]), float(out[2])

    def close(self):
        if self._h:
            L.lib().rsv_hamiltonian_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def observe(ctx: Context, n_atoms: int, precision, psi):
    """(|psi|^2, <n_i>[n]) of a CUDA state tensor."""
    norm2 = C.c_double()
    occ = np.empty(n_atoms)
    check(L.lib().rsv_observe(ctx.handle, int(n_atoms), precision_code(precision),
                              _check_state(psi, n_atoms, precision), C.byref(norm2), L._dptr(occ)))
    return norm2.value, occ


def correlations(ctx: Context, n_atoms: int, precision, psi) -> np.ndarray:
    """C[i][j] = sum_b |psi_b|^2 b_i b_j (atom order) of a CUDA state tensor."""
    out = np.empty((n_atoms, n_atoms))
    check(L.lib().rsv_correlations(ctx.handle, int(n_atoms), precision_code(precision),
                                   _check_state(psi, n_atoms, precision), L._dptr(out)))
    return out


def observe_static(n_atoms: int, precision, psi, out, stream=None):
    """rsv_observe_static: out[0] = |psi|^2, out[1 + i] = <n_i>, written on the
    device into the caller's float64 CUDA tensor `out` (n_atoms + 1 entries)
    without a context or any allocation; enqueued on `stream` (default: the
    current torch stream), returns without waiting."""
    torch = _torch()
    if not (out.is_cuda and out.dtype == torch.float64 and out.is_contiguous() and out.numel() >= n_atoms + 1):
        raise ValueError(f"out must be a contiguous CUDA float64 tensor of at least {n_atoms + 1} entries")
    s = torch.cuda.current_stream(psi.device) if stream is None else stream
    with torch.cuda.device(psi.device):
        check(L.lib().rsv_observe_static(int(n_atoms), precision_code(precision), _check_state(psi, n_atoms, precision),
                                         C.c_void_p(out.data_ptr()), C.c_void_p(s.cuda_stream or CUDA_STREAM_LEGACY)))


def sample(ctx: Context, n_atoms: int, precision, psi, shots: int, seed: int) -> np.ndarray:
    out = np.empty(int(shots), dtype=np.uint64)
    check(L.lib().rsv_sample(ctx.handle, int(n_atoms), precision_code(precision),
                             _check_state(psi, n_atoms, precision), int(shots), int(seed),
                             out.ctypes.data_as(C.POINTER(C.c_uint64))))
    return out


class Solver:
    """rsv_solver: one problem resident on the device, advanced step by step."""

    def __init__(self, ctx: Context, problem, dt_ns: int, precision="c128", krylov_tol=0.0, m_max=0,
                 max_substeps=0, obs_stride=1, initial_state=None, control_launch=False):
        self.ctx = ctx
        self.precision = precision_code(precision)
        init = None
        if initial_state is not None:
            init = np.ascontiguousarray(np.asarray(initial_state, dtype=amp_dtype(precision)))
        self._pa = L.ProblemArgs.from_problem(problem, init)
        self.n = self._pa.n
        self._cfg = L.make_config(dt_ns, precision, krylov_tol, m_max, max_substeps, obs_stride, control_launch)
        self._h = C.c_void_p()
        check(L.lib().rsv_solver_create(ctx.handle, C.byref(self._pa.struct), C.byref(self._cfg),
                                        C.byref(self._h)))
        ctx._adopt(self)

    def step(self, n_steps: int):
        check(L.lib().rsv_solver_step(self._h, int(n_steps)))

    def progress(self):
        d, t = C.c_int32(), C.c_int32()
        check(L.lib().rsv_solver_progress(self._h, C.byref(d), C.byref(t)))
        return d.value, t.value

    def rewind(self):
        """Back to t = 0 and the initial state."""
        check(L.lib().rsv_solver_rewind(self._h))

    def run_to_end(self):
        d, t = self.progress()
        self.step(t - d)

    def state(self) -> np.ndarray:
        out = np.empty(2 ** self.n, dtype=amp_dtype(self.precision))
        check(L.lib().rsv_solver_get_state(self._h, C.c_void_p(out.ctypes.data), out.nbytes))
        return out

    def set_state(self, psi):
        a = np.ascontiguousarray(np.asarray(psi, dtype=amp_dtype(self.precision)))
        check(L.lib().rsv_solver_set_state(self._h, C.c_void_p(a.ctypes.data), a.nbytes))

    def set_state_device(self, psi_tensor):
        """Copy a CUDA tensor (contiguous, the solver's dtype) into the state."""
        ptr = _check_state(psi_tensor, self.n, self.precision)
        nbytes = psi_tensor.numel() * psi_tensor.element_size()
        check(L.lib().rsv_solver_set_state_device(self._h, ptr, nbytes))

    def state_device_ptr(self):
        p, b = C.c_void_p(), C.c_size_t()
        check(L.lib().rsv_solver_state_device(self._h, C.byref(p), C.byref(b)))
        return p.value, b.value

    def occupations(self) -> np.ndarray:
        rows = C.c_int32()
        check(L.lib().rsv_solver_occupations(self._h, C.POINTER(C.c_double)(), 0, C.byref(rows)))
        out = np.empty((rows.value, self.n))
        check(L.lib().rsv_solver_occupations(self._h, L._dptr(out), rows.value, C.byref(rows)))
        return out

    def stats(self) -> dict:
        s = L.Stats_()
        check(L.lib().rsv_solver_stats(self._h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in L.Stats_._fields_}

    def set_profiling(self, on: bool):
        check(L.lib().rsv_solver_set_profiling(self._h, 1 if on else 0))

    def kernel_times(self) -> dict:
        """{kind: {"ms", "launches", "bytes"}} accumulated while profiling was on,
        and "control_step": the Krylov control step's device time wherever it
        ran ({"ms", "steps", "check_ms", "checks"})."""
        t = L.KernelTimes_()
        check(L.lib().rsv_solver_kernel_times(self._h, C.byref(t)))
        out = {k: {"ms": t.ms[i], "launches": t.launches[i], "bytes": t.bytes[i]}
               for i, k in enumerate(L.KERNEL_KINDS)}
        out["control_step"] = {"ms": t.control_step_ms, "steps": t.control_steps, "check_ms": t.control_check_ms,
                               "checks": t.control_checks}
        return out

    def close(self):
        if self._h:
            L.lib().rsv_solver_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Result:
    """rsv_result of a whole solve."""

    def __init__(self, ctx, h, n, precision):
        self.ctx = ctx
        self._h, self.n, self.precision = h, n, precision
        ctx._adopt(self)

    def state(self) -> np.ndarray:
        out = np.empty(2 ** self.n, dtype=amp_dtype(self.precision))
        check(L.lib().rsv_result_state(self._h, C.c_void_p(out.ctypes.data), out.nbytes))
        return out

    def occupations(self) -> np.ndarray:
        rows = C.c_int32()
        check(L.lib().rsv_result_occupations(self._h, C.POINTER(C.c_double)(), 0, C.byref(rows)))
        out = np.empty((rows.value, self.n))
        check(L.lib().rsv_result_occupations(self._h, L._dptr(out), rows.value, C.byref(rows)))
        return out

    def sample(self, shots: int, seed: int) -> np.ndarray:
        out = np.empty(int(shots), dtype=np.uint64)
        check(L.lib().rsv_result_sample(self._h, int(shots), int(seed), out.ctypes.data_as(C.POINTER(C.c_uint64))))
        return out

    def stats(self) -> dict:
        s = L.Stats_()
        check(L.lib().rsv_result_stats(self._h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in L.Stats_._fields_}

    def times(self) -> tuple[float, float]:
        """(wait_s, service_s): queueing and solve time of a served request."""
        w, v = C.c_double(), C.c_double()
        check(L.lib().rsv_result_times(self._h, C.byref(w), C.byref(v)))
        return w.value, v.value

    def close(self):
        if self._h:
            L.lib().rsv_result_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """rsv_batch: many independent registers (<= 20 atoms each) evolved over
    their whole pulse sequences by one persistent launch (graph replay)."""

    def __init__(self, ctx: Context, problems, dt_ns: int, precision="c64", krylov_tol=0.0, m_max=0,
                 max_substeps=0, obs_stride=1, initial_states=None):
        self.ctx = ctx
        self.precision = precision_code(precision)
        inits = initial_states if initial_states is not None else [None] * len(problems)
        self._pas = []
        for p, init in zip(problems, inits):
            a = None if init is None else np.ascontiguousarray(np.asarray(init, dtype=amp_dtype(precision)))
            self._pas.append(L.ProblemArgs.from_problem(p, a))
        self.n = [pa.n for pa in self._pas]
        arr = (L.Problem_ * len(self._pas))(*[pa.struct for pa in self._pas])
        self._cfg = L.make_config(dt_ns, precision, krylov_tol, m_max, max_substeps, obs_stride)
        self._h = C.c_void_p()
        check(L.lib().rsv_batch_create(ctx.handle, arr, len(self._pas), C.byref(self._cfg), C.byref(self._h)))
        ctx._adopt(self)

    def __len__(self):
        return len(self.n)

    def run(self):
        check(L.lib().rsv_batch_run(self._h))

    def state(self, i: int) -> np.ndarray:
        out = np.empty(2 ** self.n[i], dtype=amp_dtype(self.precision))
        check(L.lib().rsv_batch_state(self._h, int(i), C.c_void_p(out.ctypes.data), out.nbytes))
        return out

    def state_device_ptr(self, i: int):
        p, b = C.c_void_p(), C.c_size_t()
        check(L.lib().rsv_batch_state_device(self._h, int(i), C.byref(p), C.byref(b)))
        return p.value, b.value

    def occupations(self, i: int) -> np.ndarray:
        rows = C.c_int32()
        check(L.lib().rsv_batch_occupations(self._h, int(i), C.POINTER(C.c_double)(), 0, C.byref(rows)))
        out = np.empty((rows.value, self.n[i]))
        check(L.lib().rsv_batch_occupations(self._h, int(i), L._dptr(out), rows.value, C.byref(rows)))
        return out

    def stats(self, i: int = -1) -> dict:
        s = L.Stats_()
        check(L.lib().rsv_batch_stats(self._h, int(i), C.byref(s)))
        return {k: getattr(s, k) for k, _ in L.Stats_._fields_}

    def close(self):
        if self._h:
            L.lib().rsv_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """rsv_server: solves submitted at any time, admitted by device footprint,
    run concurrently on their own streams (continuous batching)."""

    def __init__(self, ctx: Context, slots: int = 4, memory_bytes: int = 0, max_bypass_s: float = 0.0,
                 batch_atoms: int = 0):
        self.ctx = ctx
        cfg = L.ServerConfig_()
        cfg.slots, cfg.batch_atoms = int(slots), int(batch_atoms)
        cfg.memory_bytes, cfg.max_bypass_s = int(memory_bytes), float(max_bypass_s)
        self._h = C.c_void_p()
        check(L.lib().rsv_server_create(ctx.handle, C.byref(cfg), C.byref(self._h)))
        self._precision = {}
        ctx._adopt(self)

    def submit(self, problem, dt_ns: int, precision="c64", krylov_tol=0.0, m_max=0, max_substeps=0, obs_stride=1,
               initial_state=None) -> int:
        init = None
        if initial_state is not None:
            init = np.ascontiguousarray(np.asarray(initial_state, dtype=amp_dtype(precision)))
        pa = L.ProblemArgs.from_problem(problem, init)
        cfg = L.make_config(dt_ns, precision, krylov_tol, m_max, max_substeps, obs_stride)
        t = C.c_uint64()
        check(L.lib().rsv_submit(self._h, C.byref(pa.struct), C.byref(cfg), C.byref(t)))
        self._precision[t.value] = (pa.n, precision_code(precision))
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1):
        """The Result of `ticket`, or None if it is still pending after timeout_ms."""
        h = C.c_void_p()
        code = L.lib().rsv_poll(self._h, C.c_uint64(ticket), int(timeout_ms), C.byref(h))
        if code == -4:
            return None
        n, prec = self._precision.pop(ticket, (0, 0))
        check(code)
        return Result(self.ctx, h, n, prec)

    def load(self) -> tuple[int, int, int]:
        q, r, b = C.c_int32(), C.c_int32(), C.c_size_t()
        check(L.lib().rsv_server_load(self._h, C.byref(q), C.byref(r), C.byref(b)))
        return q.value, r.value, b.value

    def close(self):
        if self._h:
            L.lib().rsv_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_shots(ctx: Context, problem, dt_ns: int, omega_scale, delta_shift, pos_shift_um=None, precision="c64",
              krylov_tol=0.0, m_max=0, max_substeps=0, obs_stride=1) -> np.ndarray:
    """rsv_run_shots: mean occupation rows over perturbed copies of `problem`
    (copy s: Omega * omega_scale[s], delta + delta_shift[s], positions +
    pos_shift_um[s]); the draws are the caller's."""
    pa = L.ProblemArgs.from_problem(problem)
    cfg = L.make_config(dt_ns, precision, krylov_tol, m_max, max_substeps, obs_stride)
    sc = np.ascontiguousarray(np.asarray(omega_scale, dtype=np.float64))
    sh = np.ascontiguousarray(np.asarray(delta_shift, dtype=np.float64))
    if sc.shape != sh.shape or sc.ndim != 1:
        raise ValueError("omega_scale and delta_shift must be 1-D of the same length")
    ps = None
    if pos_shift_um is not None:
        ps = np.ascontiguousarray(np.asarray(pos_shift_um, dtype=np.float64))
        if ps.shape != (sc.size,) + pa.pos.shape:
            raise ValueError("pos_shift_um must be [shots][n_atoms][dim]")
    rows = C.c_int32()
    args = (ctx.handle, C.byref(pa.struct), C.byref(cfg), int(sc.size), L._dptr(sc), L._dptr(sh),
            L._dptr(ps) if ps is not None else C.POINTER(C.c_double)())
    check(L.lib().rsv_run_shots(*args, C.POINTER(C.c_double)(), 0, C.byref(rows)))
    out = np.empty((rows.value, pa.n))
    check(L.lib().rsv_run_shots(*args, L._dptr(out), rows.value, C.byref(rows)))
    return out


def overlap(ctx: Context, n_atoms: int, precision, a, b) -> tuple[complex, float, float]:
    """(<a|b>, |a|^2, |b|^2) of two CUDA state tensors (rsv_overlap)."""
    out = np.empty(4)
    check(L.lib().rsv_overlap(ctx.handle, int(n_atoms), precision_code(precision), _check_state(a, n_atoms, precision),
                              _check_state(b, n_atoms, precision), L._dptr(out)))
    return complex(out[0], out[1]), float(out[2]), float(out[3])


def fidelity(ctx: Context, n_atoms: int, precision, target, psi) -> float:
    """|<target|psi>|^2 / (|target|^2 |psi|^2) of two CUDA state tensors (rsv_fidelity)."""
    out = C.c_double()
    check(L.lib().rsv_fidelity(ctx.handle, int(n_atoms), precision_code(precision),
                               _check_state(target, n_atoms, precision), _check_state(psi, n_atoms, precision),
                               C.byref(out)))
    return out.value


def request_bytes(problem, dt_ns: int, precision="c64", krylov_tol=0.0, m_max=0, max_substeps=0,
                  obs_stride=1) -> int:
    """rsv_request_bytes: the device footprint a server charges for this request."""
    pa = L.ProblemArgs.from_problem(problem)
    cfg = L.make_config(dt_ns, precision, krylov_tol, m_max, max_substeps, obs_stride)
    out = C.c_size_t()
    check(L.lib().rsv_request_bytes(C.byref(pa.struct), C.byref(cfg), C.byref(out)))
    return out.value


class Gradient:
    """Result of rsv_gradient: value = <sum_i w_i n_i>(T) and its derivatives
    with respect to the pulse samples, shaped like the problem's arrays."""

    def __init__(self, value, d_omega, d_delta, d_phi, nodes, stats):
        self.value, self.d_omega, self.d_delta, self.d_phi = value, d_omega, d_delta, d_phi
        self.nodes, self.stats = nodes, stats


def gradient(ctx: Context, problem, dt_ns: int, weights, precision="c128", panels=0, krylov_tol=0.0, m_max=0,
             max_substeps=0, initial_state=None) -> Gradient:
    """rsv_gradient: d<O>(T)/d(pulse samples) for O = sum_i weights[i] n_i."""
    init = None
    if initial_state is not None:
        init = np.ascontiguousarray(np.asarray(initial_state, dtype=amp_dtype(precision)))
    pa = L.ProblemArgs.from_problem(problem, init)
    cfg = L.make_config(dt_ns, precision, krylov_tol, m_max, max_substeps, 0)
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    if w.shape != (pa.n,):
        raise ValueError("weights must have one entry per atom")
    d_om, d_de = np.empty_like(pa.om), np.empty_like(pa.de)
    d_ph = None if pa.ph is None else np.empty_like(pa.ph)
    value = C.c_double()
    nodes = C.c_int64()
    st = L.Stats_()
    check(L.lib().rsv_gradient(ctx.handle, C.byref(pa.struct), C.byref(cfg), L._dptr(w), int(panels),
                               C.byref(value), L._dptr(d_om), L._dptr(d_de),
                               L._dptr(d_ph) if d_ph is not None else C.POINTER(C.c_double)(),
                               C.byref(nodes), C.byref(st)))
    return Gradient(value.value, d_om, d_de, d_ph, nodes.value, {k: getattr(st, k) for k, _ in L.Stats_._fields_})


class LindbladResult:
    """Result of rsv_lindblad_run: the final density matrix, the occupation
    rows tr(rho n_i) and the run's statistics."""

    def __init__(self, rho, occupations, stats):
        self.rho, self.occupations, self.stats = rho, occupations, stats


def lindblad_run(ctx: Context, problem, dt_ns: int, g_dephasing=None, g_relaxation=None, rho0=None,
                 krylov_tol=0.0, m_max=0, max_substeps=0, obs_stride=1, precision="c128") -> LindbladResult:
    """rsv_lindblad_run: the Lindblad master equation with per-atom Rydberg
    dephasing and spontaneous decay rates (1/us)."""
    pa = L.ProblemArgs.from_problem(problem)
    n = pa.n
    cfg = L.make_config(dt_ns, precision, krylov_tol, m_max, max_substeps, obs_stride)
    cdt = amp_dtype(precision)

    def rates(g):
        if g is None:
            return None
        g = np.ascontiguousarray(np.asarray(g, dtype=np.float64))
        if g.shape != (n,):
            raise ValueError("rates must have one entry per atom")
        return g

    gd, gr = rates(g_dephasing), rates(g_relaxation)
    r0 = None
    if rho0 is not None:
        r0 = np.ascontiguousarray(np.asarray(rho0, dtype=cdt))
        if r0.shape != (2 ** n, 2 ** n):
            raise ValueError("rho0 must be [2^n][2^n]")
    nulld = C.POINTER(C.c_double)()
    rows = C.c_int32()
    args = (ctx.handle, C.byref(pa.struct), C.byref(cfg), L._dptr(gd) if gd is not None else nulld,
            L._dptr(gr) if gr is not None else nulld, None if r0 is None else r0.ctypes.data)
    check(L.lib().rsv_lindblad_run(*args, None, nulld, 0, C.byref(rows), None))
    rho = np.empty((2 ** n, 2 ** n), dtype=cdt)
    occ = np.empty((rows.value, n))
    st = L.Stats_()
    check(L.lib().rsv_lindblad_run(*args, rho.ctypes.data, L._dptr(occ), rows.value, C.byref(rows), C.byref(st)))
    return LindbladResult(rho, occ[:rows.value], {k: getattr(st, k) for k, _ in L.Stats_._fields_})


def run_batch(ctx: Context, problems, dt_ns: int, precision="c64", krylov_tol=0.0, m_max=0, max_substeps=0,
              obs_stride=1) -> list:
    """rsv_run_batch: one Result per problem; registers of at most 20 atoms
    share one batched launch, larger ones run on the streaming solver."""
    args = [L.ProblemArgs.from_problem(p) for p in problems]
    arr = (L.Problem_ * len(args))(*[a.struct for a in args])
    cfg = L.make_config(dt_ns, precision, krylov_tol, m_max, max_substeps, obs_stride)
    outs = (C.c_void_p * len(args))()
    check(L.lib().rsv_run_batch(ctx.handle, arr, len(args), C.byref(cfg), outs))
    return [Result(ctx, C.c_void_p(outs[i]), args[i].n, precision_code(precision)) for i in range(len(args))]


def run(ctx: Context, problem, dt_ns: int, precision="c128", krylov_tol=0.0, m_max=0, max_substeps=0,
        obs_stride=1, initial_state=None) -> Result:
    """rsv_run: the whole sequence, host inputs in, a Result out."""
    init = None
    if initial_state is not None:
        init = np.ascontiguousarray(np.asarray(initial_state, dtype=amp_dtype(precision)))
    pa = L.ProblemArgs.from_problem(problem, init)
    cfg = L.make_config(dt_ns, precision, krylov_tol, m_max, max_substeps, obs_stride)
    h = C.c_void_p()
    check(L.lib().rsv_run(ctx.handle, C.byref(pa.struct), C.byref(cfg), C.byref(h)))
    return Result(ctx, h, pa.n, precision_code(precision))
