"""Pins for the CPU oracle against facts that do not come from the oracle itself:
closed forms, brute force, invariants, symmetries and published test vectors.

Each pin is chosen so that a plausible slip in the oracle (a dropped drive term,
a wrong sign of delta, a transposed <0|h|1>/<1|h|0>, a reversed bit order, an
off-by-one midpoint index) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import rydberg as O
from paper_2510_09813_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Independent closed forms (written here from the physics, not from the oracle)
# ---------------------------------------------------------------------------

def two_level_propagator(omega, delta, phi, t):
    """exp(-i h t) for h = [[0, W e^{i phi}], [W e^{-i phi}, -delta]], W = omega/2.

    h = -delta/2 + M with M^2 = w^2 I, w = sqrt(omega^2 + delta^2)/2, so
    exp(-i h t) = e^{i delta t/2} (cos(w t) I - i sin(w t)/w M).
    """
    w = 0.5 * math.hypot(omega, delta)
    M = np.array([[delta / 2, omega / 2 * np.exp(1j * phi)],
                  [omega / 2 * np.exp(-1j * phi), -delta / 2]])
    s = math.sin(w * t) / w if w > 0 else t
    return np.exp(1j * delta * t / 2) * (math.cos(w * t) * np.eye(2) - 1j * s * M)


def kron_all(vs):
    out = np.array([1.0 + 0j])
    for v in vs:
        out = np.kron(out, v)
    return out


# ---------------------------------------------------------------------------
# Published vectors
# ---------------------------------------------------------------------------

def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    assert len(rows) == 3
    for r in rows:
        assert O.philox4x32_10(r[0:4], r[4:6]) == r[6:10]


def test_shot_uniform_range_and_mean():
    u = np.array([O.shot_uniform(1234, s) for s in range(4000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.02
    # counters differ -> values differ
    assert len(np.unique(u)) == u.size


# ---------------------------------------------------------------------------
# Register and Hamiltonian structure
# ---------------------------------------------------------------------------

def test_pair_interaction_value_and_coincident():
    V = O.pair_interactions([[0.0, 0.0], [6.0, 0.0], [0.0, 5.0]], 5420158.53)
    assert V[0, 1] == pytest.approx(5420158.53 / 6.0 ** 6, rel=1e-15)
    assert V[0, 2] == pytest.approx(5420158.53 / 5.0 ** 6, rel=1e-15)
    assert V[1, 2] == pytest.approx(5420158.53 / 61.0 ** 3, rel=1e-15)
    assert np.all(np.diag(V) == 0) and np.allclose(V, V.T)
    with pytest.raises(ValueError):
        O.pair_interactions([[1.0, 2.0], [1.0, 2.0]], 1.0)


def test_two_atom_diagonal_and_bit_order():
    # atom 0 is the most significant bit: b = 1 means atom 1 excited.
    V = O.pair_interactions([[0.0, 0.0], [6.0, 0.0]], 5420158.53)
    d = np.array([1.5, -0.25])
    H = O.dense_hamiltonian(V, np.zeros(2), d, np.zeros(2))
    v01 = 5420158.53 / 46656.0
    assert np.allclose(np.diag(H).real, [0.0, -d[1], -d[0], v01 - d[0] - d[1]], rtol=0, atol=1e-12)
    # drive on atom 0 only couples b and b ^ 2
    H = O.dense_hamiltonian(V, np.array([2.0, 0.0]), np.zeros(2), np.array([0.3, 0.0]))
    assert H[2, 0] == pytest.approx(1.0 * np.exp(-0.3j))  # <1|h|0> for atom 0
    assert H[0, 2] == pytest.approx(1.0 * np.exp(0.3j))
    assert H[1, 0] == 0 and H[3, 1] == pytest.approx(np.exp(-0.3j))


def test_dense_is_hermitian_and_matches_matrix_free():
    rng = np.random.Generator(np.random.PCG64(7))
    n = 6
    pos = W.random_register(rng, n, 20.0)
    V = O.pair_interactions(pos, W.C6_DEFAULT)
    om, de, ph = rng.uniform(0, 7, n), rng.normal(0, 3, n), rng.uniform(-3, 3, n)
    H = O.dense_hamiltonian(V, om, de, ph)
    assert np.allclose(H, H.conj().T, atol=1e-12)
    x = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
    y = O.apply_hamiltonian(x, V, om, de, ph)
    assert np.allclose(y, H @ x, atol=1e-9)
    a = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
    assert np.vdot(a, O.apply_hamiltonian(x, V, om, de, ph)) == pytest.approx(
        np.conj(np.vdot(x, O.apply_hamiltonian(a, V, om, de, ph))), rel=1e-12)


def test_diagonal_energies_brute_force():
    rng = np.random.Generator(np.random.PCG64(8))
    n = 7
    V = O.pair_interactions(W.random_register(rng, n, 25.0), W.C6_DEFAULT)
    de = rng.normal(0, 2, n)
    E = O.diagonal_energies(V, de)
    for b in [0, 1, 5, 64, 77, 127]:
        occ = [(b >> (n - 1 - i)) & 1 for i in range(n)]
        e = sum(V[i, j] for i in range(n) for j in range(n) if i < j and occ[i] and occ[j])
        e -= sum(de[i] for i in range(n) if occ[i])
        assert E[b] == pytest.approx(e, rel=1e-13, abs=1e-12)


# ---------------------------------------------------------------------------
# Midpoint rule (Sec. III)
# ---------------------------------------------------------------------------

def test_step_schedule_and_midpoints():
    assert O.step_schedule(1000, 10)[:2] == [(0, 10), (10, 10)]
    assert len(O.step_schedule(1000, 10)) == 100
    assert O.step_schedule(25, 10) == [(0, 10), (10, 10), (20, 5)]
    s = np.arange(100, dtype=float) * 3.0 + 1.0  # linear: midpoint value = s(m)
    # even dt: m integer
    assert O.midpoint_value(s, 20, 10) == 1.0 + 3.0 * 25
    # odd dt: m = start + 2.5 -> average of floor and ceil
    assert O.midpoint_value(s, 10, 5) == 1.0 + 3.0 * 12.5
    # the last step: indices clamp to the final sample
    assert O.midpoint_value(s, 99, 1) == 0.5 * (s[99] + s[99])
    st = O.step_parameters(2, 30, 10, np.vstack([s[:30], 2 * s[:30]]), s[None, :30])
    assert len(st) == 3 and st[1][0] == pytest.approx(0.01)
    assert np.allclose(st[1][1], [1 + 3 * 15, 2 * (1 + 3 * 15)])


# ---------------------------------------------------------------------------
# Closed forms of the dynamics
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("method", ["dense", "krylov"])
def test_single_atom_closed_form_constant_pulse(method):
    om, de, ph, t_ns = 2 * math.pi * 1.1, 3.7, 0.6, 700
    psi, occ = O.evolve([[0.0, 0.0]], W.C6_DEFAULT, t_ns, 10, np.full(t_ns, om), np.full(t_ns, de),
                        np.full(t_ns, ph), method=method)
    ref = two_level_propagator(om, de, ph, t_ns / 1000.0) @ np.array([1.0, 0.0])
    assert np.allclose(psi, ref, atol=1e-11)
    assert occ[-1, 0] == pytest.approx(abs(ref[1]) ** 2, abs=1e-11)


def test_full_rabi_cycle():
    # Omega = 2 pi rad/us, delta = 0: P1(0.5 us) = 1, P1(1 us) = 0.
    psi, occ = O.evolve([[0.0, 0.0]], 1.0, 1000, 10, np.full(1000, 2 * math.pi), np.zeros(1000))
    assert occ[50, 0] == pytest.approx(1.0, abs=1e-12)
    assert occ[100, 0] == pytest.approx(0.0, abs=1e-12)


def test_single_atom_piecewise_linear_midpoint():
    # Linear ramps sampled at 1 ns: the midpoint value of each step is the ramp at
    # its centre, so the result is a product of exact 2x2 propagators.
    t_ns, dt = 203, 7  # odd dt and a ragged last step
    t = np.arange(t_ns) / 1000.0
    om = 5.0 + 20.0 * t
    de = -4.0 + 30.0 * t
    ph = 0.2 + 3.0 * t
    psi, _ = O.evolve([[0.0, 0.0]], 1.0, t_ns, dt, om, de, ph)
    ref = np.array([1.0 + 0j, 0.0])
    start = 0
    while start < t_ns:
        length = min(dt, t_ns - start)
        mid_us = (start + length / 2) / 1000.0
        mid_us = min(mid_us, (t_ns - 1) / 1000.0)
        U = two_level_propagator(5.0 + 20.0 * mid_us, -4.0 + 30.0 * mid_us, 0.2 + 3.0 * mid_us,
                                 length / 1000.0)
        ref = U @ ref
        start += length
    assert np.allclose(psi, ref, atol=1e-11)


def test_noninteracting_product_state():
    # C6 = 0: each atom evolves alone; amplitude b = prod_i c^{(i)}_{b_i} with atom 0 = MSB.
    n, t_ns = 5, 300
    om = np.array([1.0, 2.5, 4.0, 5.5, 7.0]) * math.pi
    de = np.array([-3.0, 0.0, 1.5, 4.0, -6.0])
    ph = np.array([0.0, 0.4, -1.0, 2.0, 3.0])
    psi, occ = O.evolve(W.chain(n, 5.0), 0.0, t_ns, 10, np.repeat(om[:, None], t_ns, 1),
                        np.repeat(de[:, None], t_ns, 1), np.repeat(ph[:, None], t_ns, 1))
    singles = [two_level_propagator(om[i], de[i], ph[i], t_ns / 1000.0) @ np.array([1.0, 0.0])
               for i in range(n)]
    assert np.allclose(psi, kron_all(singles), atol=1e-11)
    assert np.allclose(occ[-1], [abs(s[1]) ** 2 for s in singles], atol=1e-11)


def test_zero_drive_pure_phases():
    # Omega = 0: psi_b(T) = exp(-i sum_k E_k(b) tau_k) psi_b(0), E from explicit pair loops.
    rng = np.random.Generator(np.random.PCG64(11))
    n, t_ns, dt = 6, 95, 10
    pos = W.random_register(rng, n, 20.0)
    de_samples = rng.normal(0, 2, (n, t_ns))
    psi0 = kron_all([v for v in W.random_product_state(12, n)])
    psi, _ = O.evolve(pos, W.C6_DEFAULT, t_ns, dt, np.zeros((1, t_ns)), de_samples, psi0=psi0)
    c6 = W.C6_DEFAULT
    phase = np.zeros(2 ** n)
    for start, length in O.step_schedule(t_ns, dt):
        lo = min((2 * start + length) // 2, t_ns - 1)
        hi = min((2 * start + length + 1) // 2, t_ns - 1)
        d = 0.5 * (de_samples[:, lo] + de_samples[:, hi])
        for b in range(2 ** n):
            occ = [(b >> (n - 1 - i)) & 1 for i in range(n)]
            e = -sum(d[i] for i in range(n) if occ[i])
            for i in range(n):
                for j in range(i + 1, n):
                    if occ[i] and occ[j]:
                        e += c6 / np.sum((pos[i] - pos[j]) ** 2) ** 3
            phase[b] += e * length / 1000.0
    assert np.allclose(psi, np.exp(-1j * phase) * psi0, atol=1e-10)


def test_two_atom_symmetric_subspace():
    # Equal drive on both atoms: dynamics stays in {|00>, |W>, |11>} with the exact
    # 3x3 Hamiltonian [[0, O/sqrt2, 0], [O/sqrt2, -d, O/sqrt2], [0, O/sqrt2, V - 2d]].
    r, om, de, t_ns = 7.0, 2 * math.pi * 1.3, 2.0, 800
    Vv = W.C6_DEFAULT / r ** 6
    psi, _ = O.evolve([[0.0, 0.0], [r, 0.0]], W.C6_DEFAULT, t_ns, 10, np.full(t_ns, om), np.full(t_ns, de))
    h3 = np.array([[0, om / math.sqrt(2), 0], [om / math.sqrt(2), -de, om / math.sqrt(2)],
                   [0, om / math.sqrt(2), Vv - 2 * de]])
    ev, U = np.linalg.eigh(h3)
    c = U @ (np.exp(-1j * ev * t_ns / 1000.0) * (U.T @ np.array([1.0, 0, 0])))
    assert psi[0] == pytest.approx(c[0], abs=1e-11)
    assert psi[1] == pytest.approx(c[1] / math.sqrt(2), abs=1e-11)
    assert psi[2] == pytest.approx(c[1] / math.sqrt(2), abs=1e-11)
    assert psi[3] == pytest.approx(c[2], abs=1e-11)


def test_blockade_limit():
    # V >> Omega: |11> is blocked, the pair oscillates at sqrt(2) Omega.
    om, t_ns = 2 * math.pi, 400
    psi, _ = O.evolve([[0.0, 0.0], [3.0, 0.0]], W.C6_DEFAULT, t_ns, 5, np.full(t_ns, om), np.zeros(t_ns))
    t = t_ns / 1000.0
    p_w = abs(psi[1]) ** 2 + abs(psi[2]) ** 2
    assert p_w == pytest.approx(math.sin(math.sqrt(2) * om * t / 2) ** 2, abs=2e-3)
    assert abs(psi[3]) ** 2 < 1e-4


# ---------------------------------------------------------------------------
# Brute force agreement and invariants
# ---------------------------------------------------------------------------

def test_dense_vs_krylov_time_dependent():
    rng = np.random.Generator(np.random.PCG64(21))
    prob = W.random_knot_problem(rng, 7, 120, with_phi=True)
    a, occ_a = O.evolve(prob.positions, prob.c6, prob.t_ns, 10, prob.omega, prob.delta, prob.phi,
                        method="dense")
    b, occ_b = O.evolve(prob.positions, prob.c6, prob.t_ns, 10, prob.omega, prob.delta, prob.phi,
                        method="krylov")
    assert O.norm_difference(a, b) < 1e-11
    assert np.max(np.abs(occ_a - occ_b)) < 1e-11


def test_krylov_substepping_matches_dense():
    rng = np.random.Generator(np.random.PCG64(22))
    prob = W.random_knot_problem(rng, 6, 60)
    V = O.pair_interactions(prob.positions, prob.c6)
    tau, om, de, ph = O.step_parameters(6, 60, 60, prob.omega, prob.delta)[0]
    H = O.dense_hamiltonian(V, om, de, ph)
    psi0 = W.random_state(3, 6)
    ref = scipy.linalg.expm(-1j * tau * H) @ psi0
    E = O.diagonal_energies(V, de)
    out, stats = O.lanczos_expm(lambda x: O.apply_hamiltonian(x, V, om, de, ph, E), psi0, tau,
                                tol=1e-13, m_max=5)
    assert len(stats) > 1  # forced to restart
    assert O.norm_difference(out, ref) < 1e-11


def test_norm_and_energy_conservation_constant_pulse():
    prob = W.rabi_chain(6, 6.0, t_ns=300)
    V = O.pair_interactions(prob.positions, prob.c6)
    n = 6
    om, de, ph = np.full(n, prob.omega[0, 0]), np.zeros(n), np.zeros(n)
    psi, _ = O.evolve(prob.positions, prob.c6, prob.t_ns, 10, prob.omega, prob.delta)
    H = O.dense_hamiltonian(V, om, de, ph)
    psi0 = O.zero_state(n)
    assert np.linalg.norm(psi) == pytest.approx(1.0, abs=1e-12)
    assert np.vdot(psi, H @ psi).real == pytest.approx(np.vdot(psi0, H @ psi0).real, abs=1e-10)


def test_time_reversal():
    # H real (phi = 0): exp(+iH t) = conj(exp(-iH t) conj(.)), so evolving conj(psi_T)
    # forward and conjugating returns psi_0.
    rng = np.random.Generator(np.random.PCG64(31))
    n, t_ns = 6, 200
    pos = W.random_register(rng, n, 18.0)
    om, de = np.full(t_ns, 9.0), np.full(t_ns, -2.0)
    psi0 = W.random_state(5, n)
    psi_t, _ = O.evolve(pos, W.C6_DEFAULT, t_ns, 10, om, de, psi0=psi0)
    back, _ = O.evolve(pos, W.C6_DEFAULT, t_ns, 10, om, de, psi0=np.conj(psi_t))
    assert O.norm_difference(np.conj(back), psi0) < 1e-10


def test_mirror_symmetry_rabi_chain():
    prob = W.rabi_chain(8, 6.0, t_ns=200)
    _, occ = O.evolve(prob.positions, prob.c6, prob.t_ns, 10, prob.omega, prob.delta)
    assert np.allclose(occ, occ[:, ::-1], atol=1e-12)


def test_uniform_phase_gauge_identity():
    # H(phi) = U H(0) U^dagger with U = exp(-i phi sum_i n_i): from |0..0>,
    # amplitude b picks up exp(-i phi popcount(b)).
    rng = np.random.Generator(np.random.PCG64(41))
    n, t_ns, phi = 6, 150, 0.9
    pos = W.random_register(rng, n, 16.0)
    om, de = np.full(t_ns, 11.0), np.full(t_ns, 1.5)
    a, _ = O.evolve(pos, W.C6_DEFAULT, t_ns, 10, om, de)
    b, _ = O.evolve(pos, W.C6_DEFAULT, t_ns, 10, om, de, np.full(t_ns, phi))
    pop = np.array([bin(k).count("1") for k in range(2 ** n)])
    assert np.allclose(b, np.exp(-1j * phi * pop) * a, atol=1e-11)


def test_atom_permutation_permutes_bits():
    rng = np.random.Generator(np.random.PCG64(42))
    n, t_ns = 5, 120
    pos = W.random_register(rng, n, 15.0)
    om = rng.uniform(3, 9, n)
    perm = np.array([3, 0, 4, 1, 2])
    a, occ_a = O.evolve(pos, W.C6_DEFAULT, t_ns, 10, np.repeat(om[:, None], t_ns, 1), np.zeros((1, t_ns)))
    b, occ_b = O.evolve(pos[perm], W.C6_DEFAULT, t_ns, 10, np.repeat(om[perm][:, None], t_ns, 1),
                        np.zeros((1, t_ns)))
    assert np.allclose(occ_b[-1], occ_a[-1][perm], atol=1e-12)
    at = a.reshape((2,) * n)
    assert np.allclose(b.reshape((2,) * n), np.transpose(at, perm), atol=1e-11)


# ---------------------------------------------------------------------------
# Observables, metrics and sampling
# ---------------------------------------------------------------------------

def test_occupations_and_metrics():
    singles = W.random_product_state(3, 4)
    psi = kron_all(singles)
    assert np.allclose(O.occupations(psi), [abs(s[1]) ** 2 for s in singles], atol=1e-14)
    assert O.infidelity(psi, 1j * psi) == pytest.approx(0.0, abs=1e-14)
    x = W.random_state(1, 4)
    assert O.infidelity(psi, x) == pytest.approx(1 - abs(np.vdot(psi, x)) ** 2, abs=1e-13)
    assert O.norm_difference(psi, -psi) == pytest.approx(2.0)


def test_sampling_distribution():
    prob = W.rabi_chain(8, 6.0, t_ns=400)
    psi, _ = O.evolve(prob.positions, prob.c6, prob.t_ns, 10, prob.omega, prob.delta)
    shots = 20000
    s = O.sample_bitstrings(psi, shots, seed=99)
    p = np.abs(psi) ** 2
    counts = np.bincount(s.astype(np.int64), minlength=256)
    tv = 0.5 * np.sum(np.abs(counts / shots - p))
    assert tv < 0.03
    # inverse CDF by brute force with the same uniforms
    cdf = np.cumsum(p)
    for k in range(50):
        u = O.shot_uniform(99, k) * cdf[-1]
        b = next(i for i in range(256) if cdf[i] > u)
        assert s[k] == b


def test_paper_memory_figures():
    # Sec. III.A.1: 16 * 2^N bytes per complex128 vector, ~1 GB at N = 26;
    # state + diagonal + 15 Krylov vectors below 20 GB.
    with open(os.path.join(GOLDEN, "paper_memory.txt")) as f:
        row = [float(x) for x in next(l for l in f if not l.startswith("#")).split()]
    n, bpa, gb, kv, max_gb = row
    state = bpa * 2 ** int(n)
    assert state / 1e9 == pytest.approx(gb, rel=0.1)
    assert (state * (kv + 1) + 8 * 2 ** int(n)) / 1e9 < max_gb


def test_hamiltonian_rows_match_dense():
    rng = np.random.Generator(np.random.PCG64(77))
    n = 6
    V = O.pair_interactions(W.random_register(rng, n, 18.0), W.C6_DEFAULT)
    om, de, ph = rng.uniform(0, 7, n), rng.normal(0, 3, n), rng.uniform(-3, 3, n)
    H = O.dense_hamiltonian(V, om, de, ph)
    x = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
    idx = [0, 1, 17, 40, 63]
    assert np.allclose(O.hamiltonian_rows(idx, x, V, om, de, ph), (H @ x)[idx], atol=1e-10)


def test_sweep_3x4_golden_matches_the_oracle():
    """The stored 400-step evolution of the 3x4 sweep (GPU parity reference) is
    the oracle's: its first 12 occupation rows are recomputed here, and its
    final state is normalised."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sweep_3x4_dt10.npz")
    with np.load(path) as g:
        psi, occ = g["psi"], g["occ"]
    assert psi.shape == (2 ** 12,) and occ.shape == (401, 12)
    assert abs(np.linalg.norm(psi) - 1.0) < 1e-12
    prob = W.adiabatic_sweep_lattice(3, 4)
    t_ns = 110
    _, occ_head = O.evolve(prob.positions, prob.c6, t_ns, 10, prob.omega[:, :t_ns], prob.delta[:, :t_ns], None,
                           method="krylov", tol=1e-14)
    assert np.max(np.abs(np.asarray(occ_head) - occ[:12])) <= 1e-12


def test_sweep_4x5_golden_matches_the_oracle():
    """The stored 400-step evolution of the 20-atom 4x5 sweep (written with the
    oracle's Chebyshev path) agrees with the oracle's Lanczos path, an
    independent algorithm, on its first occupation rows; its final state is
    normalised and has the lattice's mirror symmetry in the occupations."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sweep_4x5_dt10.npz")
    with np.load(path) as g:
        psi, occ = g["psi"], g["occ"]
    assert psi.shape == (2 ** 20,) and occ.shape == (401, 20)
    assert abs(np.linalg.norm(psi) - 1.0) < 1e-12
    # the 4x5 lattice is symmetric under the 180-degree rotation i -> 19 - i
    assert np.max(np.abs(occ - occ[:, ::-1])) < 1e-10
    prob = W.adiabatic_sweep_lattice(4, 5)
    t_ns = 30
    _, occ_head = O.evolve(prob.positions, prob.c6, t_ns, 10, prob.omega[:, :t_ns], prob.delta[:, :t_ns], None,
                           method="krylov", tol=1e-14)
    assert np.max(np.abs(np.asarray(occ_head) - occ[:4])) <= 1e-12


def test_correlations_and_energy_moments():
    """Product states: <n_i n_j> = <n_i><n_j> for i != j and <n_i n_i> = <n_i>.
    A basis state at Omega = 0 is an eigenstate: <H> = E(b), variance 0. A
    single atom from |0> with Omega, delta: <H> = 0 and <H^2> = Omega^2 / 4."""
    rng = np.random.Generator(np.random.PCG64(41))
    n = 6
    ab = W.random_product_state(5, n)
    psi = ab[0]
    for i in range(1, n):
        psi = np.kron(psi, ab[i])
    C = O.correlations(psi)
    occ = O.occupations(psi)
    assert np.allclose(np.diag(C), occ, atol=1e-14)
    off = C - np.outer(occ, occ)
    np.fill_diagonal(off, 0.0)
    assert np.max(np.abs(off)) < 1e-14
    # basis state b at Omega = 0
    pos = W.random_register(rng, n, 20.0)
    V = O.pair_interactions(pos, W.C6_DEFAULT)
    de = rng.normal(0, 3, n)
    b = 0b101101
    e = np.zeros(2 ** n, dtype=np.complex128)
    e[b] = 1.0
    E1, E2 = O.energy_moments(e, V, np.zeros(n), de)
    Eb = O.diagonal_energies(V, de)[b]
    assert abs(E1 - Eb) < 1e-9 * max(1.0, abs(Eb)) and abs(E2 - Eb ** 2) < 1e-9 * max(1.0, Eb ** 2)
    # one atom from |0>: H|0> = Omega/2 |1>
    E1, E2 = O.energy_moments(np.array([1.0, 0.0]), np.zeros((1, 1)), np.array([3.0]), np.array([1.5]))
    assert abs(E1) < 1e-15 and abs(E2 - 9.0 / 4.0) < 1e-14


# ---------------------------------------------------------------------------
# Overlap and gradients (Sec. III results; Sec. V: differentiability)
# ---------------------------------------------------------------------------

def test_overlap_of_product_states():
    """<a|b> of two product states is the product of the single-atom overlaps."""
    rng = np.random.default_rng(41)
    n = 6
    a1 = rng.normal(size=(n, 2)) + 1j * rng.normal(size=(n, 2))
    b1 = rng.normal(size=(n, 2)) + 1j * rng.normal(size=(n, 2))
    a, b = np.ones(1, complex), np.ones(1, complex)
    for i in range(n):
        a, b = np.kron(a, a1[i]), np.kron(b, b1[i])
    ov, aa, bb = O.overlap(a, b)
    want = np.prod([np.conj(a1[i]) @ b1[i] for i in range(n)])
    assert abs(ov - want) <= 1e-12 * abs(want)
    assert abs(aa - np.prod([np.sum(np.abs(a1[i]) ** 2) for i in range(n)])) <= 1e-12 * aa
    assert abs(bb - np.prod([np.sum(np.abs(b1[i]) ** 2) for i in range(n)])) <= 1e-12 * bb


def _gradient_case(seed, n, t_ns, dt, phi_rows):
    rng = np.random.default_rng(seed)
    pos = np.array([[0.0, 0.0], [6.0, 0.0], [3.0, 5.5], [9.0, 5.0]])[:n]
    om = rng.uniform(2, 10, (n, t_ns))
    de = rng.normal(0, 5, (1, t_ns))
    ph = None if phi_rows == 0 else rng.uniform(-1, 1, (phi_rows, t_ns))
    w = rng.normal(size=n)
    return pos, om, de, ph, w


@pytest.mark.parametrize("seed,n,t_ns,dt,phi_rows", [(5, 3, 47, 10, 3), (6, 4, 36, 7, 1), (7, 2, 30, 10, 0)])
def test_gradient_matches_finite_differences(seed, n, t_ns, dt, phi_rows):
    """Central differences of the dense forward evolution, on every sample the
    midpoint rule reads (the others have zero gradient on both sides)."""
    pos, om, de, ph, w = _gradient_case(seed, n, t_ns, dt, phi_rows)
    c6 = W.C6_DEFAULT
    B = O.occupation_bits(n)

    def value(om_, de_, ph_):
        psi, _ = O.evolve(pos, c6, t_ns, dt, om_, de_, ph_, method="dense", record_occupations=False)
        return float(np.real(np.vdot(psi, (B @ w) * psi)))

    v, d_om, d_de, d_ph = O.occupation_gradient(pos, c6, t_ns, dt, om, de, ph, w)
    assert abs(v - value(om, de, ph)) <= 1e-13
    used = sorted({x for s in O.step_schedule(t_ns, dt) for x in O.midpoint_samples(t_ns, *s)})
    unused = [x for x in range(t_ns) if x not in used]
    h = 1e-5
    for name, arr, grad in (("om", om, d_om), ("de", de, d_de), ("ph", ph, d_ph)):
        if arr is None:
            assert grad is None
            continue
        assert np.all(grad[:, unused] == 0.0)
        for r in range(arr.shape[0]):
            for s in used[r % 2::2]:
                a, b = arr.copy(), arr.copy()
                a[r, s] += h
                b[r, s] -= h
                pick = lambda x: (x if name == "om" else om, x if name == "de" else de, x if name == "ph" else ph)
                fd = (value(*pick(a)) - value(*pick(b))) / (2 * h)
                assert abs(grad[r, s] - fd) <= 2e-9 * max(1.0, abs(fd)), (name, r, s, grad[r, s], fd)


def test_gradient_single_atom_resonant_closed_form():
    """One atom on resonance (delta = phi = 0) from |0>: the drive is a rotation
    about x by theta = sum_k Omega_bar_k tau_k, so P1 = sin^2(theta / 2),
    dP1/dOmega_bar_k = tau_k sin(theta) / 2, and every delta-derivative is zero
    (the first-order change of the amplitude <1|U|0> is real while the
    amplitude itself is imaginary)."""
    rng = np.random.default_rng(1)
    t_ns, dt = 53, 10
    om = rng.uniform(1, 8, (1, t_ns))
    de = np.zeros((1, t_ns))
    v, d_om, d_de, _ = O.occupation_gradient([[0.0, 0.0]], 1.0, t_ns, dt, om, de)
    sched = O.step_schedule(t_ns, dt)
    bars = [0.5 * (om[0, lo] + om[0, hi]) for lo, hi in (O.midpoint_samples(t_ns, *s) for s in sched)]
    theta = sum(b * s[1] / 1000.0 for b, s in zip(bars, sched))
    assert abs(v - math.sin(theta / 2) ** 2) <= 1e-14
    want = np.zeros_like(om)
    for s in sched:
        lo, hi = O.midpoint_samples(t_ns, *s)
        g = (s[1] / 1000.0) * math.sin(theta) / 2
        want[0, lo] += 0.5 * g
        want[0, hi] += 0.5 * g
    assert np.max(np.abs(d_om - want)) <= 1e-14
    assert np.max(np.abs(d_de)) <= 1e-15


def test_gradient_uniform_phase_sum_rule():
    """A phase shared by all atoms and constant in time is a gauge from |0...0>:
    the observable does not depend on it, so its sample derivatives sum to 0
    (while individual samples need not vanish)."""
    pos, om, de, _, w = _gradient_case(9, 3, 40, 10, 0)
    ph = np.full((1, 40), 0.7)
    _, _, _, d_ph = O.occupation_gradient(pos, W.C6_DEFAULT, 40, 10, om, de, ph, w)
    assert np.max(np.abs(d_ph)) > 1e-5
    assert abs(d_ph.sum()) <= 1e-14


# ---------------------------------------------------------------------------
# Lindblad master equation (Sec. III.A: open-system dynamics)
# ---------------------------------------------------------------------------

def test_lindblad_without_noise_is_the_pure_state():
    """Zero rates: rho(T) = psi(T) psi(T)^dag of the (pinned) pure-state evolution."""
    rng = np.random.default_rng(2)
    n, t = 3, 60
    pos = np.array([[0.0, 0.0], [6.0, 0.0], [3.0, 5.5]])
    om, de, ph = rng.uniform(2, 10, (n, t)), rng.normal(0, 5, (1, t)), rng.uniform(-1, 1, (n, t))
    rho, occ = O.lindblad_evolve(pos, W.C6_DEFAULT, t, 10, om, de, ph)
    psi, occ2 = O.evolve(pos, W.C6_DEFAULT, t, 10, om, de, ph, method="dense")
    assert np.max(np.abs(rho - np.outer(psi, psi.conj()))) <= 1e-13
    assert np.max(np.abs(occ - occ2)) <= 1e-13


def test_lindblad_single_atom_closed_forms():
    """Undriven atom: the excited population decays as e^{-g_r t}; the
    coherence rho_01 turns at the detuning (E_1 = -delta) and decays at
    (g_deph + g_relax) / 2."""
    g = 0.7
    rho, occ = O.lindblad_evolve([[0.0, 0.0]], 1.0, 2000, 50, np.zeros((1, 2000)), np.full((1, 2000), 3.0),
                                 None, [0.0], [g], rho0=np.array([[0, 0], [0, 1]], complex))
    assert abs(occ[-1, 0] - math.exp(-g * 2.0)) <= 1e-13
    assert abs(occ[20, 0] - math.exp(-g * 1.0)) <= 1e-13
    gd, gr, de, T = 0.4, 0.3, 2.0, 1500
    rho, _ = O.lindblad_evolve([[0.0, 0.0]], 1.0, T, 30, np.zeros((1, T)), np.full((1, T), de), None, [gd], [gr],
                               rho0=np.full((2, 2), 0.5, complex))
    t = T / 1000
    assert abs(rho[0, 1] - 0.5 * np.exp(-1j * de * t) * np.exp(-(gd + gr) * t / 2)) <= 1e-13
    assert abs(rho[1, 1] - 0.5 * math.exp(-gr * t)) <= 1e-13


def test_lindblad_driven_damped_steady_state():
    """Resonance fluorescence: a driven atom with decay g settles at
    rho_11 = (Omega^2 / 4) / (delta^2 + Omega^2 / 2 + g^2 / 4)."""
    Om, dl, g, T = 3.0, 1.5, 2.0, 20000
    _, occ = O.lindblad_evolve([[0.0, 0.0]], 1.0, T, 100, np.full((1, T), Om), np.full((1, T), dl), None,
                               [0.0], [g])
    assert abs(occ[-1, 0] - (Om ** 2 / 4) / (dl ** 2 + Om ** 2 / 2 + g ** 2 / 4)) <= 1e-9


def test_lindblad_state_stays_a_density_matrix():
    """Trace 1, Hermitian and positive semidefinite at every step, with both
    channels on three interacting atoms."""
    rng = np.random.default_rng(8)
    n, t = 3, 40
    pos = np.array([[0.0, 0.0], [6.0, 0.0], [3.0, 5.5]])
    om, de = rng.uniform(2, 10, (1, t)), rng.normal(0, 5, (n, t))
    V = O.pair_interactions(pos, W.C6_DEFAULT)
    jumps = O.jump_operators(n, [0.5, 0.0, 1.0], [0.3, 0.8, 0.0])
    rho = np.zeros((8, 8), complex)
    rho[0, 0] = 1.0
    for tau, o, d, p in O.step_parameters(n, t, 10, om, de, None):
        rho = (scipy.linalg.expm(tau * O.liouvillian(O.dense_hamiltonian(V, o, d, p), jumps)) @ rho.reshape(-1)
               ).reshape(8, 8)
        assert abs(np.trace(rho) - 1.0) <= 1e-13
        assert np.max(np.abs(rho - rho.conj().T)) <= 1e-14
        assert np.min(np.linalg.eigvalsh(0.5 * (rho + rho.conj().T))) >= -1e-13


def test_dense_krylov_and_chebyshev_agree():
    """Three independent evaluations of the same product of step exponentials
    (scaling-and-squaring expm of the dense H, Lanczos, and the Chebyshev
    expansion over the Gershgorin interval) agree, with phases and
    time-dependent pulses; at 12 atoms without the dense path."""
    rng = np.random.default_rng(3)
    prob = W.random_knot_problem(rng, 6, 100, with_phi=True)
    args = (prob.positions, prob.c6, prob.t_ns, 10, prob.omega, prob.delta, prob.phi)
    a, _ = O.evolve(*args, method="dense")
    b, _ = O.evolve(*args, method="cheb")
    c, _ = O.evolve(*args, method="krylov", tol=1e-14)
    assert O.norm_difference(a, b) <= 1e-13
    assert O.norm_difference(a, c) <= 1e-13
    prob = W.random_knot_problem(rng, 12, 20, with_phi=True)
    args = (prob.positions, prob.c6, prob.t_ns, 10, prob.omega, prob.delta, prob.phi)
    b, _ = O.evolve(*args, method="cheb")
    c, _ = O.evolve(*args, method="krylov", tol=1e-14)
    assert O.norm_difference(b, c) <= 1e-13


def test_chebyshev_single_atom_closed_form():
    """The Chebyshev path alone against the two-level closed form."""
    om, de, ph, t = 5.0, 2.0, 0.4, 0.37
    U = two_level_propagator(om, de, ph, t)
    V = np.zeros((1, 1))
    H = O.dense_hamiltonian(V, [om], [de], [ph])
    lo, hi = O.spectral_bounds(V, np.array([om]), np.array([de]))
    psi0 = np.array([0.6, 0.8j])
    got = O.chebyshev_expm(lambda x: H @ x, psi0, t, lo, hi)
    assert np.max(np.abs(got - U @ psi0)) <= 1e-14


def test_phase_minimised_norm_difference():
    """Against brute force over a fine grid of global phases, and zero for a
    pure phase."""
    rng = np.random.default_rng(12)
    a = rng.normal(size=16) + 1j * rng.normal(size=16)
    b = a + 0.05 * (rng.normal(size=16) + 1j * rng.normal(size=16))
    b = b * np.exp(0.7j)
    got = O.phase_min_norm_difference(a, b)
    grid = min(np.linalg.norm(a - np.exp(1j * t) * b) for t in np.linspace(0, 2 * math.pi, 200001))
    assert got <= grid + 1e-12
    assert grid - got <= 1e-6
    assert O.phase_min_norm_difference(a, np.exp(-1.3j) * a) <= 1e-13
    assert O.norm_difference(a, np.exp(-1.3j) * a) > 1.0
