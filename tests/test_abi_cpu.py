"""C ABI checks that need no GPU: the library loads and exports every symbol
include/rsv.h declares, host-side preparation agrees with the oracle, and
device calls fail with a status code (not a crash) when CUDA has no device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import rydberg as O
from paper_2510_09813_b300 import _lib as L
from paper_2510_09813_b300 import api
from paper_2510_09813_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "rsv.h")).read()
    return re.findall(r"^RSV_API\s+[\w\s\*]+?\b(rsv_\w+)\s*\(", txt, flags=re.M)


def test_library_exports_every_declared_symbol():
    names = header_symbols()
    assert len(names) >= 27
    lib = L.lib()
    for n in names:
        assert hasattr(lib, n), n
    # and the binding declares a signature for each
    for n in names:
        assert getattr(lib, n).argtypes is not None, n


def test_version():
    assert "sm_103a" in api.version()


def test_pair_energies_match_oracle():
    rng = np.random.Generator(np.random.PCG64(1))
    pos = W.random_register(rng, 9, 25.0)
    assert np.allclose(api.pair_energies(pos, W.C6_DEFAULT), O.pair_interactions(pos, W.C6_DEFAULT),
                       rtol=1e-15, atol=0)
    pos3 = np.hstack([pos, rng.uniform(0, 5, (9, 1))])
    V3 = api.pair_energies(pos3, 3.0)
    assert np.allclose(V3, O.pair_interactions(pos3, 3.0), rtol=1e-15, atol=0)


def test_coincident_atoms_rejected():
    with pytest.raises(L.RsvError) as e:
        api.pair_energies([[0.0, 0.0], [1.0, 1.0], [0.0, 0.0]], 1.0)
    assert e.value.code == -6


@pytest.mark.parametrize("t_ns,dt", [(1000, 10), (2000, 5), (203, 7), (25, 10), (9, 1), (5, 8)])
def test_midpoint_parameters_match_oracle(t_ns, dt):
    rng = np.random.Generator(np.random.PCG64(t_ns + dt))
    n = 4
    prob = W.Problem(W.chain(n, 6.0), W.C6_DEFAULT, t_ns, rng.normal(size=(n, t_ns)),
                     rng.normal(size=(1, t_ns)), rng.normal(size=(n, t_ns)))
    om, de, ph, tau = api.midpoint_parameters(prob, dt)
    ref = O.step_parameters(n, t_ns, dt, prob.omega, prob.delta, prob.phi)
    assert len(ref) == api.num_steps(t_ns, dt) == len(tau)
    for k, (tk, o, d, p) in enumerate(ref):
        assert tau[k] == tk
        assert np.array_equal(om[k], o) and np.array_equal(de[k], d) and np.array_equal(ph[k], p)


def test_footprint_matches_paper_accounting():
    # Sec. III.A.1: complex128 vectors of 16 * 2^N bytes; at N = 26 state + diagonal
    # + 15 Krylov vectors stay below 20 GB. Our footprint (state, m_max basis vectors,
    # two work vectors, no stored diagonal) obeys the same bound.
    with open(os.path.join(ROOT, "tests", "golden", "paper_memory.txt")) as f:
        n, bpa, gb, kv, max_gb = [float(x) for x in next(l for l in f if not l.startswith("#")).split()]
    fp = api.footprint_bytes(int(n), "c128", int(kv))
    assert fp >= (kv + 1) * bpa * 2 ** int(n)
    assert fp / 1e9 < max_gb
    # complex64 halves the vectors
    assert api.footprint_bytes(26, "c64", 15) < fp / 1.9
    assert api.footprint_bytes(0, "c64", 15) == 0


def test_invalid_arguments_return_status():
    lib = L.lib()
    assert lib.rsv_pair_energies(0, 2, None, 1.0, None) == -1
    assert lib.rsv_num_steps(0, 10) == 0
    pa = L.ProblemArgs(W.chain(3, 6.0), 1.0, 10, np.ones(10), np.zeros(10))
    pa.struct.omega_rows = 2  # neither 1 nor n_atoms
    out = np.empty(3 * 1)
    assert lib.rsv_midpoint_parameters(C.byref(pa.struct), 10, L._dptr(out), L._dptr(out), L._dptr(out),
                                       L._dptr(out)) == -1
    assert b"omega rows" in lib.rsv_last_error()


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    st = L.lib().rsv_create(C.byref(h), 0, 0, None)
    assert st in (-5, -1) and not h.value


def test_new_entries_reject_bad_arguments_without_a_gpu():
    """Argument checks of the later entries run before any device work."""
    lib = L.lib()
    assert lib.rsv_correlations(None, 4, L.RSV_C64, None, None) == -1
    assert lib.rsv_hamiltonian_expectation(None, None, None) == -1
    assert lib.rsv_run_shots(None, None, None, 1, None, None, None, None, 0, None) == -1
    assert lib.rsv_batch_run(None) == -1
    assert lib.rsv_poll(None, 1, 0, None) == -1
    assert lib.rsv_observe_static(4, L.RSV_C64, None, None, None) == -1
    assert lib.rsv_observe_static(32, L.RSV_C64, C.c_void_p(16), C.c_void_p(16), None) == -1
    assert b"limit of 31 atoms" in lib.rsv_last_error()


def test_overlap_and_gradient_reject_bad_arguments_without_a_gpu():
    lib = L.lib()
    out = np.zeros(4)
    assert lib.rsv_overlap(None, 4, L.RSV_C64, None, None, L._dptr(out)) == -1
    pa = L.ProblemArgs([[0.0, 0.0], [6.0, 0.0]], 5420158.53, 20, np.ones(20), np.zeros(20))
    cfg = L.make_config(10, "c128", 0.0, 0, 0, 0)
    w = np.ones(2)
    v = C.c_double()
    d_om, d_de = np.zeros((1, 20)), np.zeros((1, 20))
    assert lib.rsv_gradient(None, C.byref(pa.struct), C.byref(cfg), L._dptr(w), 0, C.byref(v), L._dptr(d_om),
                            L._dptr(d_de), None, None, None) == -1
    assert b"NULL" in lib.rsv_last_error()
    assert lib.rsv_run_batch(None, C.byref(pa.struct), 1, C.byref(cfg), None) == -1
    assert lib.rsv_check_bounded_wait(None) == -1
    rows = C.c_int32()
    assert lib.rsv_lindblad_run(None, C.byref(pa.struct), C.byref(cfg), None, None, None, None, None, 0,
                                C.byref(rows), None) == -1


def test_request_bytes_is_footprint_plus_sequence():
    """The server's charge for a request: rsv_footprint_bytes plus the per-step
    parameters and occupation rows, each rounded to 256 bytes (host-only)."""
    rng = np.random.Generator(np.random.PCG64(3))
    p = W.random_knot_problem(rng, 12, 100)
    base = api.footprint_bytes(12, "c64", 30)
    b1 = api.request_bytes(p, 10, "c64", obs_stride=0)
    b2 = api.request_bytes(p, 10, "c64", obs_stride=1)
    b3 = api.request_bytes(p, 5, "c64", obs_stride=0)
    assert base < b1 < b2 and b1 < b3
    assert (b1 - base) % 256 == 0 and (b2 - base) % 256 == 0
    # 10 steps of 10 ns (obs_stride 1: 12 rows of 12 doubles)
    assert b2 - b1 == ((8 * 12 * 12 + 255) // 256 - (8 * 12 * 2 + 255) // 256) * 256
    with pytest.raises(api.RsvError):
        api.request_bytes(p, 0, "c64")
