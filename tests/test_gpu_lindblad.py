"""GPU parity of the Lindblad master equation (rsv_lindblad_run) against the
oracle's dense superoperator exponentials, and its invariants at sizes the
dense oracle does not reach.

Tolerance (complex128): each Krylov piece is accepted at an a-posteriori
error of p = 1e-12 relative to |rho|_F <= 1, and the pieces add up over the
steps, so rho and the occupation rows must match to 1e-10 for the sequences
used here (at most 20 steps). complex64: p = 1e-7 per piece plus FP32
rounding of the diagonal differences E(r) - E(c) (about 2^-24 of up to 1e3
rad/us, i.e. a phase error near 6e-7 per 10-ns step), so 20 steps stay below
5e-5.
"""
import numpy as np
import pytest

from oracle import rydberg as O
from paper_2510_09813_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10
TOL_C64 = 5e-5
POS = np.array([[0.0, 0.0], [6.0, 0.0], [3.0, 5.5], [9.0, 5.0], [12.0, 0.0], [6.0, 10.0], [0.0, 11.0]])


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


@pytest.mark.parametrize("n,t_ns,dt,orow,drow,prow", [
    (1, 200, 10, 1, 1, 1),
    (2, 100, 10, 2, 1, 0),
    (3, 60, 10, 1, 3, 3),
    (4, 40, 7, 4, 4, 1),
    (5, 20, 10, 1, 1, 0),
])
def test_lindblad_matches_oracle(ctx, n, t_ns, dt, orow, drow, prow):
    rng = np.random.default_rng(500 + n)
    om = rng.uniform(2, 10, (orow, t_ns))
    de = rng.normal(0, 5, (drow, t_ns))
    ph = None if prow == 0 else rng.uniform(-1, 1, (prow, t_ns))
    gd = rng.uniform(0, 2, n) * (rng.random(n) < 0.7)
    gr = rng.uniform(0, 2, n) * (rng.random(n) < 0.7)
    prob = W.Problem(positions=POS[:n].copy(), c6=W.C6_DEFAULT, t_ns=t_ns, omega=om, delta=de, phi=ph)
    got = api().lindblad_run(ctx, prob, dt, gd, gr, obs_stride=1)
    rho, occ = O.lindblad_evolve(prob.positions, prob.c6, t_ns, dt, om, de, ph, gd, gr)
    assert got.occupations.shape == occ.shape
    assert np.max(np.abs(got.rho - rho)) <= TOL
    assert np.max(np.abs(got.occupations - occ)) <= TOL
    assert got.stats["steps"] == len(O.step_schedule(t_ns, dt))


@pytest.mark.parametrize("n,t_ns,dt,orow,drow,prow", [(1, 200, 10, 1, 1, 1), (3, 60, 10, 1, 3, 3),
                                                      (5, 20, 10, 1, 1, 0)])
def test_lindblad_complex64_matches_oracle(ctx, n, t_ns, dt, orow, drow, prow):
    rng = np.random.default_rng(600 + n)
    om = rng.uniform(2, 10, (orow, t_ns))
    de = rng.normal(0, 5, (drow, t_ns))
    ph = None if prow == 0 else rng.uniform(-1, 1, (prow, t_ns))
    gd, gr = rng.uniform(0, 2, n), rng.uniform(0, 2, n)
    prob = W.Problem(positions=POS[:n].copy(), c6=W.C6_DEFAULT, t_ns=t_ns, omega=om, delta=de, phi=ph)
    got = api().lindblad_run(ctx, prob, dt, gd, gr, obs_stride=1, precision="c64")
    rho, occ = O.lindblad_evolve(prob.positions, prob.c6, t_ns, dt, om, de, ph, gd, gr)
    assert got.rho.dtype == np.complex64
    assert np.max(np.abs(got.rho.astype(np.complex128) - rho)) <= TOL_C64
    assert np.max(np.abs(got.occupations - occ)) <= TOL_C64


def test_lindblad_from_a_given_mixed_state(ctx):
    rng = np.random.default_rng(77)
    n, t_ns = 3, 50
    A = rng.normal(size=(8, 8)) + 1j * rng.normal(size=(8, 8))
    rho0 = A @ A.conj().T
    rho0 /= np.trace(rho0).real
    prob = W.Problem(positions=POS[:n].copy(), c6=W.C6_DEFAULT, t_ns=t_ns, omega=rng.uniform(2, 8, (1, t_ns)),
                     delta=rng.normal(0, 3, (1, t_ns)), phi=None)
    gd, gr = np.array([0.3, 0.0, 0.7]), np.array([0.0, 1.1, 0.4])
    got = api().lindblad_run(ctx, prob, 10, gd, gr, rho0=rho0, obs_stride=0)
    rho, occ = O.lindblad_evolve(prob.positions, prob.c6, t_ns, 10, prob.omega, prob.delta, None, gd, gr, rho0=rho0)
    assert np.max(np.abs(got.rho - rho)) <= TOL
    assert np.max(np.abs(got.occupations - occ[[0, -1]])) <= TOL


def test_lindblad_without_noise_is_the_pure_solve(ctx):
    """Zero rates at N = 7: rho(T) = psi psi^dag of the library's own pure-state solve."""
    rng = np.random.default_rng(7)
    n, t_ns = 7, 80
    prob = W.Problem(positions=POS.copy(), c6=W.C6_DEFAULT, t_ns=t_ns, omega=rng.uniform(2, 8, (n, t_ns)),
                     delta=rng.normal(0, 3, (1, t_ns)), phi=rng.uniform(-1, 1, (1, t_ns)))
    got = api().lindblad_run(ctx, prob, 10, obs_stride=0)
    r = api().run(ctx, prob, 10, "c128", obs_stride=0)
    psi = r.state()
    occ = r.occupations()
    r.close()
    assert np.max(np.abs(got.rho - np.outer(psi, psi.conj()))) <= TOL
    assert np.max(np.abs(got.occupations - occ)) <= TOL


def test_lindblad_steady_state_of_a_driven_damped_atom(ctx):
    """rho_11 -> (Omega^2 / 4) / (delta^2 + Omega^2 / 2 + g^2 / 4) (20 us)."""
    Om, dl, g, T = 3.0, 1.5, 2.0, 20000
    prob = W.Problem(positions=np.zeros((1, 2)), c6=1.0, t_ns=T, omega=np.full((1, T), Om),
                     delta=np.full((1, T), dl), phi=None)
    got = api().lindblad_run(ctx, prob, 100, None, [g], obs_stride=0)
    assert abs(got.occupations[-1, 0] - (Om ** 2 / 4) / (dl ** 2 + Om ** 2 / 2 + g ** 2 / 4)) <= 1e-8


def test_lindblad_stays_a_density_matrix_at_n9(ctx):
    """N = 9 (4^9 amplitudes): trace 1, Hermitian, positive semidefinite."""
    rng = np.random.default_rng(9)
    n, t_ns = 9, 30
    pos = W.random_register(rng, n, 20.0, 5.0)
    prob = W.Problem(positions=pos, c6=W.C6_DEFAULT, t_ns=t_ns, omega=rng.uniform(2, 8, (1, t_ns)),
                     delta=rng.normal(0, 3, (1, t_ns)), phi=None)
    got = api().lindblad_run(ctx, prob, 10, rng.uniform(0, 1, n), rng.uniform(0, 1, n), obs_stride=0)
    rho = got.rho
    assert abs(np.trace(rho) - 1.0) <= 1e-10
    assert np.max(np.abs(rho - rho.conj().T)) <= 1e-12
    assert np.min(np.linalg.eigvalsh(0.5 * (rho + rho.conj().T))) >= -1e-10
    assert np.allclose(got.occupations[-1], np.real(np.diag(rho)) @ O.occupation_bits(n), rtol=0, atol=1e-12)
    g32 = api().lindblad_run(ctx, prob, 10, rng.uniform(0, 1, n), rng.uniform(0, 1, n), obs_stride=0,
                             precision="c64")
    r32 = g32.rho.astype(np.complex128)
    assert abs(np.trace(r32) - 1.0) <= 2e-5
    assert np.max(np.abs(r32 - r32.conj().T)) <= 1e-5


def test_lindblad_rejects_bad_arguments(ctx):
    from paper_2510_09813_b300 import _lib as L
    prob = W.Problem(positions=np.array([[0.0, 0.0], [6.0, 0.0]]), c6=W.C6_DEFAULT, t_ns=20, omega=np.ones((1, 20)),
                     delta=np.zeros((1, 20)), phi=None)
    with pytest.raises(Exception):
        api().lindblad_run(ctx, prob, 10, [-1.0, 0.0], None)
    big = W.Problem(positions=np.arange(30.0).reshape(15, 2) * 10, c6=W.C6_DEFAULT, t_ns=20,
                    omega=np.ones((1, 20)), delta=np.zeros((1, 20)), phi=None)
    with pytest.raises(Exception, match="<= 14"):
        api().lindblad_run(ctx, big, 10)
    with pytest.raises(ValueError):
        api().lindblad_run(ctx, prob, 10, rho0=np.eye(3))
    assert L.RSV_C128 != L.RSV_C64
