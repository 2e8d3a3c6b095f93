"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (complex128 path / complex64 path):
  * matvec: max |y_gpu - y_ref| <= tol * (|E|_max + sum_i |Omega_i|/2) * max|x|
    with tol = 1e-13 / 2e-6 (FP64 vs FP32 rounding of a sum of N+1 terms);
  * time evolution: infidelity <= 1e-10 / 1e-5 against the oracle, plus a raw
    norm difference <= 1e-9 for complex128 (no global phase is dropped);
  * occupations: max |d<n_i>| <= 1e-10 / 1e-5.
"""
import math
import os

import numpy as np
import pytest

from oracle import rydberg as O
from paper_2510_09813_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MATVEC_TOL = {"c128": 1e-13, "c64": 2e-6}
INFID_TOL = {"c128": 1e-10, "c64": 1e-5}
OCC_TOL = {"c128": 1e-10, "c64": 1e-5}
TDT = {"c128": torch.complex128, "c64": torch.complex64}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2510_09813_b300 import api
    c = api.Context(0)
    yield c
    c.close()


def api():
    from paper_2510_09813_b300 import api as A
    return A


def rand_state_gpu(n, prec, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    dt = torch.float32 if prec == "c64" else torch.float64
    re = torch.randn(2 ** n, generator=g, device="cuda", dtype=dt)
    im = torch.randn(2 ** n, generator=g, device="cuda", dtype=dt)
    v = torch.complex(re, im)
    return v / torch.linalg.vector_norm(v)


def scale_of(V, om, de):
    n = V.shape[0]
    return float(np.sum(np.abs(V)) / 2 + np.sum(np.abs(de)) + np.sum(np.abs(om)) / 2 + 1.0)


# ---------------------------------------------------------------------------
# Matvec y = H x
# ---------------------------------------------------------------------------

MATVEC_CASES = [(n, p) for p in ("c128", "c64") for n in (1, 2, 3, 5, 8, 9, 11, 12, 13, 14, 15, 16, 18, 20, 22)]
MATVEC_CASES += [(24, "c64"), (23, "c128")]


@pytest.mark.parametrize("n,prec", MATVEC_CASES)
@pytest.mark.parametrize("with_phi", [False, True])
def test_matvec_matches_oracle(ctx, n, prec, with_phi):
    if n >= 20 and with_phi:
        pytest.skip("phase variant covered at smaller sizes")
    rng = np.random.Generator(np.random.PCG64(1000 + n))
    side = 5.0 * math.ceil(math.sqrt(n)) + 5.0
    pos = W.random_register(rng, n, side)
    V = O.pair_interactions(pos, W.C6_DEFAULT)
    om = rng.uniform(2.0, 9.0, n)
    de = rng.normal(0.0, 3.0, n)
    ph = rng.uniform(-math.pi, math.pi, n) if with_phi else np.zeros(n)
    x = rand_state_gpu(n, prec, seed=n)
    y = torch.empty_like(x)
    api().apply_hamiltonian(ctx, n, prec, V, om, de, ph if with_phi else None, x, y)
    torch.cuda.synchronize()
    xh = x.cpu().numpy().astype(np.complex128)
    ref = O.apply_hamiltonian(xh, V, om, de, ph)
    err = np.max(np.abs(y.cpu().numpy().astype(np.complex128) - ref))
    assert err <= MATVEC_TOL[prec] * scale_of(V, om, de) * np.max(np.abs(xh)), err


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_matvec_full_size_sampled_rows(ctx, prec):
    """N = 28 random box (c64) / N = 26 (c128): rows of H x checked one by one."""
    n = 28 if prec == "c64" else 26
    prob = W.random_box(seed=3, n=n)
    V = O.pair_interactions(prob.positions, prob.c6)
    om, de = prob.omega[:, 0], prob.delta[:, 0]
    x = rand_state_gpu(n, prec, seed=99)
    y = torch.empty_like(x)
    api().apply_hamiltonian(ctx, n, prec, V, om, de, None, x, y)
    torch.cuda.synchronize()
    rng = np.random.Generator(np.random.PCG64(5))
    D = 2 ** n
    idx = [0, 1, D - 1, D - 2, 2 ** 13 - 1, 2 ** 13, 2 ** 22, 2 ** 22 - 1] + list(rng.integers(0, D, 120))
    need = sorted({int(b) for b in idx} | {int(b) ^ (1 << q) for b in idx for q in range(n)})
    xs = x[torch.tensor(need, device="cuda")].cpu().numpy().astype(np.complex128)
    lookup = dict(zip(need, xs))
    ref = O.hamiltonian_rows(idx, lookup, V, om, de, np.zeros(n))
    got = y[torch.tensor(idx, device="cuda")].cpu().numpy().astype(np.complex128)
    err = np.max(np.abs(got - ref))
    assert err <= MATVEC_TOL[prec] * scale_of(V, om, de) * np.max(np.abs(xs)), err


# ---------------------------------------------------------------------------
# Time evolution against the oracle
# ---------------------------------------------------------------------------

def gpu_evolve(ctx, prob, dt, prec, **kw):
    s = api().Solver(ctx, prob, dt, prec, **kw)
    s.run_to_end()
    return s.state().astype(np.complex128), s.occupations(), s.stats()


def oracle_evolve(prob, dt, psi0=None):
    # The oracle's Chebyshev path: the same product of step exponentials as its
    # Lanczos path (the two, and dense expm, agree to 1e-13 in the oracle pins),
    # 10-100x faster than the fully re-orthogonalised Lanczos.
    return O.evolve(prob.positions, prob.c6, prob.t_ns, dt, prob.omega, prob.delta, prob.phi, psi0=psi0,
                    method="cheb")


@pytest.fixture(scope="module")
def rabi_chain_ref():
    prob = W.rabi_chain()  # 8 atoms, 6 um, Omega = 2 pi, T = 1 us
    psi, occ = oracle_evolve(prob, 10)
    return prob, psi, occ


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_rabi_chain_n8(ctx, rabi_chain_ref, prec):
    prob, ref, occ_ref = rabi_chain_ref
    psi, occ, st = gpu_evolve(ctx, prob, 10, prec)
    assert st["steps"] == 100
    assert occ.shape == occ_ref.shape
    assert O.infidelity(psi, ref) <= INFID_TOL[prec]
    if prec == "c128":
        assert O.norm_difference(psi, ref) <= 1e-9
    assert np.max(np.abs(occ - occ_ref)) <= OCC_TOL[prec]


@pytest.fixture(scope="module")
def sweep_3x4_ref():
    # the oracle's full 400-step evolution, written by tests/golden/make_sweep_3x4.py
    # (about ten minutes of CPU); test_oracle_pins checks its first steps afresh
    prob = W.adiabatic_sweep_lattice(3, 4)
    with np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sweep_3x4_dt10.npz")) as g:
        return prob, g["psi"], g["occ"]


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_adiabatic_sweep_3x4_full_length(ctx, sweep_3x4_ref, prec):
    prob, ref, occ_ref = sweep_3x4_ref
    psi, occ, st = gpu_evolve(ctx, prob, 10, prec)
    assert st["steps"] == 400
    assert O.infidelity(psi, ref) <= INFID_TOL[prec]
    if prec == "c128":
        assert O.norm_difference(psi, ref) <= 1e-9
    assert np.max(np.abs(occ - occ_ref)) <= OCC_TOL[prec]


@pytest.fixture(scope="module")
def sweep_4x5_window_ref():
    full = W.adiabatic_sweep_lattice(4, 5)
    lo, hi = 2000, 2020
    prob = W.Problem(full.positions, full.c6, hi - lo, full.omega[:, lo:hi], full.delta[:, lo:hi], None)
    psi0 = W.random_state(20, 20)
    ref, occ_ref = oracle_evolve(prob, 10, psi0=psi0)
    return prob, psi0, ref, occ_ref


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_adiabatic_sweep_4x5_window(ctx, sweep_4x5_window_ref, prec):
    """The 20-atom 4x5 lattice, two steps from t = 2 us of the sweep (peak drive,
    delta crossing zero), from a random state: full-size geometry of both passes."""
    prob, psi0, ref, occ_ref = sweep_4x5_window_ref
    psi, occ, _ = gpu_evolve(ctx, prob, 10, prec, initial_state=psi0)
    assert O.infidelity(psi, ref) <= INFID_TOL[prec]
    if prec == "c128":
        assert O.norm_difference(psi, ref) <= 1e-9
    assert np.max(np.abs(occ - occ_ref)) <= OCC_TOL[prec]


@pytest.fixture(scope="module")
def sweep_4x5_ref():
    # the oracle's full 400-step evolution of the 20-atom 4x5 sweep (Chebyshev
    # path, complex128), written by tests/golden/make_sweep_4x5.py (about two
    # hours of one host core)
    prob = W.adiabatic_sweep_lattice(4, 5)
    with np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sweep_4x5_dt10.npz")) as g:
        return prob, g["psi"], g["occ"]


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_adiabatic_sweep_4x5_full_length(ctx, sweep_4x5_ref, prec):
    """The 20-atom 4x5 adiabatic sweep over all 400 steps (Sec. III.A.1's
    accuracy study on an adiabatic sequence, by its norm-difference metric and
    by infidelity), element by element on every occupation row."""
    prob, ref, occ_ref = sweep_4x5_ref
    psi, occ, st = gpu_evolve(ctx, prob, 10, prec)
    assert st["steps"] == 400
    assert occ.shape == occ_ref.shape
    assert O.infidelity(psi, ref) <= INFID_TOL[prec]
    if prec == "c128":
        assert O.norm_difference(psi, ref) <= 1e-9
    assert np.max(np.abs(occ - occ_ref)) <= OCC_TOL[prec]


N_BIG = 24


@pytest.fixture(scope="module")
def random_box_n24_ref():
    """One 5-ns step of the 24-atom random box (the benchmark register's first
    24 atoms and drives) from a random state, by the oracle's Chebyshev path:
    the largest evolution the host compares directly (about 35 matvecs of
    2^24 amplitudes)."""
    base = W.random_box(seed=3, n=28, t_ns=5)
    prob = W.Problem(base.positions[:N_BIG], base.c6, 5, base.omega[:N_BIG], base.delta[:N_BIG], None)
    psi0 = W.random_state(24, N_BIG)
    ref, occ_ref = oracle_evolve(prob, 5, psi0=psi0)
    return prob, psi0, ref, occ_ref


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_random_box_n24_one_step(ctx, random_box_n24_ref, prec):
    prob, psi0, ref, occ_ref = random_box_n24_ref
    psi, occ, st = gpu_evolve(ctx, prob, 5, prec, initial_state=psi0, m_max=40)
    assert st["tile_passes"] == 2
    assert O.infidelity(psi, ref) <= INFID_TOL[prec]
    if prec == "c128":
        assert O.norm_difference(psi, ref) <= 1e-9
    assert np.max(np.abs(occ - occ_ref)) <= OCC_TOL[prec]


# every strided-pass shape the autotuner times: (segment bits c, tile-order
# bits, x-only 64 KiB tiles)
SHAPES = [(seg, f1, 0) for seg in (4, 5) for f1 in (0, 2, 4)]
SHAPES += [(seg, f1, 1) for seg in (2, 3, 4, 5) for f1 in sorted({0, max(0, 5 - seg), max(0, 5 - seg) + 1})]


def force_shape(monkeypatch, seg, f1, x_only):
    monkeypatch.setenv("RSV_SEGMENT_BITS", str(seg))
    monkeypatch.setenv("RSV_TILE_ORDER_BITS", str(f1))
    monkeypatch.setenv("RSV_STRIDED_X_ONLY", str(x_only))


@pytest.mark.parametrize("seg,f1,x_only", SHAPES)
def test_strided_shape_candidates(random_box_n24_ref, monkeypatch, seg, f1, x_only):
    """Every strided-pass shape the autotuner may pick (segment bits c x tile
    order bits x tile kind), forced by the plan override instead of the tuner:
    one Lanczos step at N = 24 in both precisions against the oracle, and
    sampled rows of the 28-atom matvec through the prepared operator against
    hamiltonian_rows."""
    force_shape(monkeypatch, seg, f1, x_only)
    c = api().Context(0)
    prob, psi0, ref, occ_ref = random_box_n24_ref
    for prec in ("c64", "c128"):
        psi, occ, st = gpu_evolve(c, prob, 5, prec, initial_state=psi0, m_max=40)
        assert st["segment_bits"] == seg and st["tile_order_bits"] == f1
        tile = (13 if prec == "c64" else 12) if x_only else (12 if prec == "c64" else 11)
        assert st["strided_tile_bits"] == tile
        assert O.infidelity(psi, ref) <= INFID_TOL[prec]
        assert np.max(np.abs(occ - occ_ref)) <= OCC_TOL[prec]
    n = 28
    box = W.random_box(seed=3, n=n)
    V = O.pair_interactions(box.positions, box.c6)
    om, de = box.omega[:, 0], box.delta[:, 0]
    x = rand_state_gpu(n, "c64", seed=500 + seg * 8 + f1)
    y = torch.empty_like(x)
    h = api().Hamiltonian(c, n, "c64", V, om, de, None)
    h.apply(x, y)
    h.sync()
    h.close()
    rng = np.random.Generator(np.random.PCG64(seg * 8 + f1))
    D = 2 ** n
    idx = [0, D - 1, 2 ** 12 - 1, 2 ** 12, 2 ** 20 - 1, 2 ** 20] + list(rng.integers(0, D, 60))
    need = sorted({int(b) for b in idx} | {int(b) ^ (1 << q) for b in idx for q in range(n)})
    xs = x[torch.tensor(need, device="cuda")].cpu().numpy().astype(np.complex128)
    want = O.hamiltonian_rows(idx, dict(zip(need, xs)), V, om, de, np.zeros(n))
    got = y[torch.tensor(idx, device="cuda")].cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(got - want)) <= MATVEC_TOL["c64"] * scale_of(V, om, de) * np.max(np.abs(xs))
    del x, y
    c.close()


X_ONLY_MATVEC = [(n, prec, seg) for prec in ("c64", "c128") for n in (20, 21, 22) for seg in (2, 3, 4, 5)
                 if n - (12 if prec == "c64" else 11) >= (13 if prec == "c64" else 12) - seg]


@pytest.mark.parametrize("n,prec,seg", X_ONLY_MATVEC)
@pytest.mark.parametrize("with_phi", [False, True])
def test_x_only_strided_matvec(monkeypatch, n, prec, seg, with_phi):
    """The x-only strided pass element by element against the oracle, at the
    sizes where its 64 KiB tile just fits (no partner bit left for L2) and a
    few bits beyond, through the prepared operator with the shape forced."""
    force_shape(monkeypatch, seg, max(0, 5 - seg), 1)
    c = api().Context(0)
    rng = np.random.Generator(np.random.PCG64(2000 + n * 8 + seg))
    side = 5.0 * math.ceil(math.sqrt(n)) + 5.0
    pos = W.random_register(rng, n, side)
    V = O.pair_interactions(pos, W.C6_DEFAULT)
    om = rng.uniform(2.0, 9.0, n)
    de = rng.normal(0.0, 3.0, n)
    ph = rng.uniform(-math.pi, math.pi, n) if with_phi else np.zeros(n)
    x = rand_state_gpu(n, prec, seed=7000 + n)
    y = torch.empty_like(x)
    h = api().Hamiltonian(c, n, prec, V, om, de, ph if with_phi else None)
    h.apply(x, y)
    h.sync()
    h.close()
    xh = x.cpu().numpy().astype(np.complex128)
    ref = O.apply_hamiltonian(xh, V, om, de, ph)
    err = np.max(np.abs(y.cpu().numpy().astype(np.complex128) - ref))
    assert err <= MATVEC_TOL[prec] * scale_of(V, om, de) * np.max(np.abs(xh)), err
    c.close()


@pytest.mark.parametrize("n,prec", [(1, "c128"), (1, "c64"), (2, "c64"), (6, "c128"), (10, "c64"), (14, "c128"),
                                    (15, "c64"), (16, "c64"), (17, "c128")])
def test_random_problems_with_phase(ctx, n, prec):
    """Time-dependent global pulses with a phase, odd dt and a ragged last step."""
    rng = np.random.Generator(np.random.PCG64(300 + n))
    prob = W.random_knot_problem(rng, n, 47, with_phi=True)
    psi0 = W.random_state(n, n)
    ref, occ_ref = oracle_evolve(prob, 7, psi0=psi0)
    psi, occ, _ = gpu_evolve(ctx, prob, 7, prec, initial_state=psi0)
    assert O.infidelity(psi, ref) <= INFID_TOL[prec]
    assert np.max(np.abs(occ - occ_ref)) <= OCC_TOL[prec]


@pytest.fixture(scope="module")
def phase_gauge_ref():
    n = 21
    rng = np.random.Generator(np.random.PCG64(700 + n))
    base = W.random_knot_problem(rng, n, 47, with_phi=True)
    t = np.arange(47)
    phi = np.stack([base.phi[0] + rng.uniform(-np.pi, np.pi) + 0.02 * (q + 1) * t for q in range(n)])
    prob = W.Problem(base.positions, base.c6, 47, base.omega, base.delta, phi)
    psi0 = W.random_state(700 + n, n)
    ref, occ_ref = oracle_evolve(prob, 7, psi0=psi0)
    return prob, psi0, ref, occ_ref


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_phase_gauge_on_two_pass_plans(ctx, phase_gauge_ref, prec):
    """A laser phase on the two-pass plans runs in the gauge frame (psi <- U^dagger
    psi, real-coefficient passes, psi <- U psi, U = exp(-i sum phi_i n_i)): 21
    atoms, per-atom phases that change every step, a random start state and a
    ragged last step, against the oracle, with every step counted as gauged."""
    prob, psi0, ref, occ_ref = phase_gauge_ref
    psi, occ, st = gpu_evolve(ctx, prob, 7, prec, initial_state=psi0)
    assert st["tile_passes"] == 2 and st["phase_gauge_steps"] == st["steps"] == 7
    assert O.infidelity(psi, ref) <= INFID_TOL[prec]
    if prec == "c128":
        assert O.norm_difference(psi, ref) <= 1e-9
    assert np.max(np.abs(occ - occ_ref)) <= OCC_TOL[prec]


def test_per_atom_pulses(ctx):
    rng = np.random.Generator(np.random.PCG64(17))
    n, t_ns = 9, 60
    pos = W.random_register(rng, n, 20.0)
    prob = W.Problem(pos, W.C6_DEFAULT, t_ns, rng.uniform(2, 12, (n, t_ns)), rng.normal(0, 4, (n, t_ns)),
                     rng.uniform(-1, 1, (n, t_ns)))
    ref, occ_ref = oracle_evolve(prob, 5)
    for prec in ("c128", "c64"):
        psi, occ, _ = gpu_evolve(ctx, prob, 5, prec)
        assert O.infidelity(psi, ref) <= INFID_TOL[prec]
        assert np.max(np.abs(occ - occ_ref)) <= OCC_TOL[prec]


def test_krylov_restarts_match(ctx):
    """m_max small forces restarts inside a step; the result must not change."""
    prob = W.rabi_chain(8, 8.0, omega=2 * math.pi, t_ns=100)
    ref, _ = oracle_evolve(prob, 20)
    psi, _, st = gpu_evolve(ctx, prob, 20, "c128", m_max=12, max_substeps=400)
    assert st["substeps"] > 0
    assert O.infidelity(psi, ref) <= 1e-10
    assert O.norm_difference(psi, ref) <= 1e-9


@pytest.mark.parametrize("n,prec,shape", [(10, "c64", None), (19, "c128", None), (22, "c64", (5, 0, 1)),
                                           (22, "c128", (4, 2, 0)), (22, "c128", (3, 2, 1))])
def test_fused_control_matches_control_launch(monkeypatch, n, prec, shape):
    """The Krylov control step run by the last CTA of each iteration's last
    pass (the default) against the same step as a launch of its own
    (RSV_FLAG_CONTROL_LAUNCH): identical arithmetic, so identical states and
    Krylov statistics, bit for bit, on the single-pass kernel and both
    second-pass kernels; no control launches when fused. Then the state
    against the oracle."""
    A = api()
    if shape:
        force_shape(monkeypatch, *shape)
    c = A.Context(0)
    prob = W.random_box(seed=11, n=n, side_um=5.0 * math.ceil(math.sqrt(n)), t_ns=40)
    out = {}
    for launch in (False, True):
        s = A.Solver(c, prob, 10, prec, control_launch=launch)
        s.set_profiling(True)
        s.run_to_end()
        kt = s.kernel_times()
        out[launch] = (s.state(), s.stats(), kt["control"]["launches"], kt["pass_first"]["launches"])
        s.close()
    (psi_f, st_f, ctl_f, nf), (psi_l, st_l, ctl_l, nl) = out[False], out[True]
    assert np.array_equal(psi_f.view(np.uint8), psi_l.view(np.uint8))
    for k in ("krylov_iterations", "substeps", "max_error_estimate"):
        assert st_f[k] == st_l[k], k
    assert ctl_f == 0 and ctl_l == nl == nf >= st_f["krylov_iterations"] > 0  # setup launches are apart
    if shape:
        assert st_f["segment_bits"] == shape[0] and st_f["tile_order_bits"] == shape[1]
    ref, _ = oracle_evolve(prob, 10)
    assert O.infidelity(psi_f.astype(np.complex128), ref) <= INFID_TOL[prec]
    bad = A.L.make_config(10, prec)
    bad.flags = 2
    pa = A.L.ProblemArgs.from_problem(prob, None)
    h = A.C.c_void_p()
    assert A.L.lib().rsv_solver_create(c.handle, A.C.byref(pa.struct), A.C.byref(bad), A.C.byref(h)) == -1
    c.close()


def test_zero_drive_diagonal(ctx):
    """Omega = 0 from a superposition: H is diagonal but the Krylov space still grows."""
    n, t_ns = 10, 50
    rng = np.random.Generator(np.random.PCG64(4))
    prob = W.Problem(W.random_register(rng, n, 20.0), W.C6_DEFAULT, t_ns, np.zeros(t_ns),
                     rng.normal(0, 3, t_ns), None)
    psi0 = W.random_state(8, n)
    ref, _ = oracle_evolve(prob, 10, psi0=psi0)
    psi, _, st = gpu_evolve(ctx, prob, 10, "c128", initial_state=psi0)
    assert O.infidelity(psi, ref) <= 1e-10
    assert O.norm_difference(psi, ref) <= 1e-9


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_zero_drive_breakdown(ctx, prec):
    """Omega = 0 from |0...0>: H psi = 0, the Krylov space breaks down at m = 1
    and the state must stay exactly |0...0>."""
    n, t_ns = 12, 30
    prob = W.Problem(W.chain(n, 5.0), W.C6_DEFAULT, t_ns, np.zeros(t_ns), np.full(t_ns, 2.0), None)
    psi, occ, st = gpu_evolve(ctx, prob, 10, prec)
    assert st["krylov_iterations"] == 3
    assert psi[0] == 1.0 and np.all(psi[1:] == 0)


# ---------------------------------------------------------------------------
# Full-size (N = 28, complex64) closed forms
# ---------------------------------------------------------------------------

def test_n28_noninteracting_product_state(ctx):
    """C6 = 0 on the 28-atom random box: each atom is an independent Rabi problem."""
    base = W.random_box(seed=3, n=28, t_ns=40)
    prob = W.Problem(base.positions, 0.0, base.t_ns, base.omega, base.delta, None)
    s = api().Solver(ctx, prob, 5, "c64", obs_stride=8)
    s.run_to_end()
    occ = s.occupations()
    t = base.t_ns / 1000.0
    singles = []
    for i in range(28):
        om, de = base.omega[i, 0], base.delta[i, 0]
        w = 0.5 * math.hypot(om, de)
        c0 = np.exp(1j * de * t / 2) * (math.cos(w * t) - 1j * de / 2 * math.sin(w * t) / w)
        c1 = np.exp(1j * de * t / 2) * (-1j * om / 2 * math.sin(w * t) / w)
        singles.append((c0, c1))
    assert np.max(np.abs(occ[-1] - [abs(c[1]) ** 2 for c in singles])) <= 1e-5
    ptr, nbytes = s.state_device_ptr()
    rng = np.random.Generator(np.random.PCG64(1))
    idx = [0, 2 ** 28 - 1] + list(rng.integers(0, 2 ** 28, 64))
    psi = s.state()
    for b in idx:
        amp = 1.0 + 0j
        for i in range(28):
            amp *= singles[i][(int(b) >> (27 - i)) & 1]
        assert abs(complex(psi[int(b)]) - amp) <= 1e-5 * max(1.0, abs(amp)) + 1e-6


def test_n28_zero_drive_phases(ctx):
    """Omega = 0 on the 28-atom random box from a random product state:
    psi_b(T) = exp(-i T E(b)) psi_b(0) with E from explicit pair sums."""
    base = W.random_box(seed=3, n=28, t_ns=10)
    n = 28
    prob = W.Problem(base.positions, base.c6, base.t_ns, np.zeros((1, base.t_ns)), base.delta, None)
    singles = W.random_product_state(5, n)
    # build the product state on the GPU (input construction)
    psi0 = torch.ones(1, dtype=torch.complex64, device="cuda")
    for i in range(n):
        psi0 = torch.kron(psi0, torch.tensor(singles[i], dtype=torch.complex64, device="cuda"))
    s = api().Solver(ctx, prob, 2, "c64", obs_stride=0, m_max=40)
    s.set_state_device(psi0)
    s.run_to_end()
    psi = s.state()
    V = O.pair_interactions(base.positions, base.c6)
    de = base.delta[:, 0]
    T = base.t_ns / 1000.0
    # Basis states drawn from the product state's own distribution |a0(b)|^2
    # (bit i set with probability |s_i[1]|^2): the Krylov tolerance bounds the
    # psi-weighted error, so amplitudes of negligible weight may carry large
    # relative errors without affecting any result; these draws weigh each
    # relative error the way the tolerance does.
    rng = np.random.Generator(np.random.PCG64(2))
    p1 = np.array([abs(singles[i][1]) ** 2 for i in range(n)])
    draws = [sum(1 << (n - 1 - i) for i in range(n) if rng.random() < p1[i]) for _ in range(50)]
    worst = 0.0
    for b in draws:
        b = int(b)
        occ = [(b >> (n - 1 - i)) & 1 for i in range(n)]
        e = -sum(de[i] for i in range(n) if occ[i])
        e += sum(V[i, j] for i in range(n) for j in range(i + 1, n) if occ[i] and occ[j])
        a0 = 1.0 + 0j
        for i in range(n):
            a0 *= singles[i][occ[i]]
        ref = np.exp(-1j * e * T) * a0
        worst = max(worst, (abs(complex(psi[b]) - ref) - 1e-12) / abs(a0))
    # The complex64 diagonal E(b) is three FP32 terms, each rounded once from
    # FP64, summed in FP32, and multiplied into FP32 amplitudes: about 6 unit
    # roundoffs (2^-24) of |E| <= sum_{i<j} V_ij + sum_i |delta_i|, i.e. a phase
    # error of 6 * 2^-24 * |E|max * T (8 is used). The five Krylov steps add
    # their tolerance (1e-7 per step, relative) and FP32 rounding of their
    # iterations, covered by 1e-5.
    e_max = float(np.sum(np.triu(V, 1)) + np.sum(np.abs(de)))
    bound = 8 * 2.0 ** -24 * e_max * T + 1e-5
    assert worst <= bound, (worst, bound)


def test_n28_norm_conservation_random_box(ctx):
    prob = W.random_box(seed=3, n=28, t_ns=20)
    s = api().Solver(ctx, prob, 5, "c64", m_max=20, obs_stride=1)
    s.run_to_end()
    ptr, _ = s.state_device_ptr()
    n2, occ = api().observe(ctx, 28, "c64", torch.from_numpy(s.state()).cuda())
    assert abs(n2 - 1.0) <= 1e-5
    assert np.all(occ >= -1e-7) and np.all(occ <= 1 + 1e-6)


def test_n28_full_sequence_conserves_norm_and_energy(ctx):
    """The whole 2 us random box (400 steps of a constant Hamiltonian, complex64,
    m_max 20): |psi| stays 1 and <H> stays at its initial value 0 (|0...0> has
    E = 0 and no drive expectation). Every step's Krylov error is at most
    tol = 1e-7 relative, so |Delta <H>| <= 2 * 400 * tol * |H|; FP32 rounding of
    the 2^28-term inner product adds ~1e-6 |H|. The bound used, 1e-4 |H|, is
    above both."""
    prob = W.random_box(seed=3, n=28)
    s = api().Solver(ctx, prob, 5, "c64", m_max=20, obs_stride=0)
    s.run_to_end()
    assert s.progress() == (400, 400)
    psi = torch.from_numpy(s.state()).cuda()
    s.close()
    V = O.pair_interactions(prob.positions, prob.c6)
    om, de = prob.omega[:, 0], prob.delta[:, 0]
    h = api().Hamiltonian(ctx, 28, "c64", V, om, de, None)
    y = torch.empty_like(psi)
    h.apply(psi, y)
    h.sync()
    h.close()
    n2 = float(torch.sum(torch.abs(psi.to(torch.complex128)) ** 2))
    energy = complex(torch.vdot(psi.to(torch.complex128), y.to(torch.complex128)))
    assert abs(n2 - 1.0) <= 1e-5
    assert abs(energy.imag) <= 1e-4 * scale_of(V, om, de)
    assert abs(energy.real) <= 1e-4 * scale_of(V, om, de)


# ---------------------------------------------------------------------------
# Observables and sampling
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,prec", [(1, "c64"), (7, "c128"), (13, "c64"), (16, "c128"), (21, "c64")])
def test_observe_matches_oracle(ctx, n, prec):
    x = rand_state_gpu(n, prec, seed=7 * n)
    n2, occ = api().observe(ctx, n, prec, x)
    xh = x.cpu().numpy()
    ref = O.occupations(xh)
    p = xh.real.astype(np.float64) ** 2 + xh.imag.astype(np.float64) ** 2
    assert abs(n2 - p.sum()) <= 1e-12
    assert np.max(np.abs(occ - ref)) <= 1e-12


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_sampling_matches_oracle_inverse_cdf(ctx, prec):
    n = 10
    x = rand_state_gpu(n, prec, seed=3)
    shots, seed = 5000, 2024
    got = api().sample(ctx, n, prec, x, shots, seed)
    xh = x.cpu().numpy()
    ref = O.sample_bitstrings(xh, shots, seed)
    mism = np.nonzero(got != ref)[0]
    # only shots whose uniform sits within rounding of a cdf boundary may differ
    p = xh.real.astype(np.float64) ** 2 + xh.imag.astype(np.float64) ** 2
    cdf = np.cumsum(p)
    for s in mism:
        u = O.shot_uniform(seed, int(s)) * cdf[-1]
        assert np.min(np.abs(cdf - u)) <= 1e-12
    assert len(mism) <= 2


def test_sampling_distribution_large(ctx):
    n = 20
    x = rand_state_gpu(n, "c64", seed=11)
    p = (x.abs() ** 2).double().cpu().numpy()
    coarse = p.reshape(64, -1).sum(axis=1)
    got = api().sample(ctx, n, "c64", x, 200000, 9)
    counts = np.bincount((got >> np.uint64(n - 6)).astype(np.int64), minlength=64) / 200000
    assert 0.5 * np.sum(np.abs(counts - coarse / coarse.sum())) < 0.01


# ---------------------------------------------------------------------------
# Errors and the whole-solve entry point
# ---------------------------------------------------------------------------

def test_run_entry_and_errors(ctx):
    A = api()
    prob = W.rabi_chain(6, 6.0, t_ns=200)
    r = A.run(ctx, prob, 10, "c128", obs_stride=5)
    ref, occ_ref = oracle_evolve(prob, 10)
    assert O.infidelity(r.state(), ref) <= 1e-10
    occ = r.occupations()
    assert occ.shape == (1 + 20 // 5, 6)
    assert np.max(np.abs(occ[-1] - occ_ref[-1])) <= 1e-10
    samples = r.sample(1000, 5)
    assert samples.max() < 64
    st = r.stats()
    assert st["steps"] == 20 and st["krylov_iterations"] >= 20
    r.close()
    bad = W.Problem(np.array([[0.0, 0.0], [0.0, 0.0]]), 1.0, 10, np.ones(10), np.zeros(10))
    with pytest.raises(A.RsvError) as e:
        A.run(ctx, bad, 10, "c64")
    assert e.value.code == -6
    with pytest.raises(A.RsvError):
        A.run(ctx, prob, 0, "c64")
    zero = np.zeros(64, dtype=np.complex128)
    with pytest.raises(A.RsvError):
        A.run(ctx, prob, 10, "c128", initial_state=zero)


def test_arena_admission(ctx):
    A = api()
    small = A.Context(0, arena_bytes=64 << 20)
    prob = W.rabi_chain(8, 6.0, t_ns=50)
    r = A.run(small, prob, 10, "c64")
    r.close()
    big = W.random_box(seed=3, n=22, t_ns=10)
    with pytest.raises(A.RsvError) as e:
        A.Solver(small, big, 5, "c128", m_max=30)
    assert e.value.code == -2
    small.close()
