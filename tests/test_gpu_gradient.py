"""GPU parity of the pulse gradient (rsv_gradient) and of the overlap with a
target state (rsv_overlap).

Gradients are compared with the oracle's exact adjoint (Frechet derivatives of
the dense step exponentials) on every sample. Tolerances, from the error
sources: the quadrature is below 1e-13 relative, so what remains is the
Krylov tolerance p (1e-12 for complex128, 1e-7 for complex64) of each of the
backward evolutions plus complex64's FP32 rounding. Each derivative is a time
integral over one step of a sum bounded by |G| |lambda| |psi| <=
max(1, Omega_max) * sum_i |w_i|, so the bound used is tol * S with
S = sum_i |w_i| * max(1, max Omega) and tol = 1e-9 (c128) / 3e-5 (c64).

At the two-pass size (N = 14, complex128) no dense oracle fits; there the
gradient is checked against central differences of the library's own forward
solve on sampled entries (a property at any size).
"""
import numpy as np
import pytest

from oracle import rydberg as O
from paper_2510_09813_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRAD_TOL = {"c128": 1e-9, "c64": 3e-5}
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


POS = np.array([[0.0, 0.0], [6.0, 0.0], [3.0, 5.5], [9.0, 5.0], [12.0, 0.0], [6.0, 10.0], [0.0, 11.0]])


def make_case(seed, n, t_ns, orow, drow, prow):
    rng = np.random.default_rng(seed)
    om = rng.uniform(2, 10, (orow, t_ns))
    de = rng.normal(0, 5, (drow, t_ns))
    ph = None if prow == 0 else rng.uniform(-1, 1, (prow, t_ns))
    prob = W.Problem(positions=POS[:n].copy(), c6=W.C6_DEFAULT, t_ns=t_ns, omega=om, delta=de, phi=ph)
    return prob, rng.normal(size=n)


@pytest.mark.parametrize("n,prec,t_ns,dt,orow,drow,prow", [
    (1, "c128", 53, 10, 1, 1, 0),
    (3, "c128", 47, 10, 3, 1, 3),
    (4, "c64", 36, 7, 1, 4, 1),
    (5, "c128", 40, 10, 5, 5, 1),
    (6, "c64", 30, 10, 1, 1, 6),
    (7, "c128", 25, 10, 7, 1, 0),
])
def test_gradient_matches_oracle(ctx, n, prec, t_ns, dt, orow, drow, prow):
    prob, w = make_case(300 + n, n, t_ns, orow, drow, prow)
    got = api().gradient(ctx, prob, dt, w, precision=prec)
    v, d_om, d_de, d_ph = O.occupation_gradient(prob.positions, prob.c6, t_ns, dt, prob.omega, prob.delta,
                                                prob.phi, w)
    S = np.sum(np.abs(w)) * max(1.0, float(np.max(prob.omega)))
    tol = GRAD_TOL[prec] * S
    assert abs(got.value - v) <= tol
    assert got.d_omega.shape == d_om.shape and got.d_delta.shape == d_de.shape
    assert np.max(np.abs(got.d_omega - d_om)) <= tol
    assert np.max(np.abs(got.d_delta - d_de)) <= tol
    if prow:
        assert np.max(np.abs(got.d_phi - d_ph)) <= tol
    else:
        assert got.d_phi is None
    assert got.nodes >= 8 * O.step_schedule(t_ns, dt).__len__()
    assert got.stats["kernel_launches"] > 0


def test_zero_observable_has_zero_gradient(ctx):
    prob, _ = make_case(11, 3, 30, 1, 1, 1)
    got = api().gradient(ctx, prob, 10, np.zeros(3), precision="c128")
    assert got.value == 0.0
    assert not np.any(got.d_omega) and not np.any(got.d_delta) and not np.any(got.d_phi)


def test_fixed_panels_agree_with_automatic(ctx):
    """A weakly interacting register: one panel per step already meets the
    bound, and twelve panels give the same derivatives."""
    rng = np.random.default_rng(5)
    pos = np.array([[0.0, 0.0], [14.0, 0.0], [0.0, 14.0]])
    prob = W.Problem(positions=pos, c6=W.C6_DEFAULT, t_ns=40, omega=rng.uniform(2, 6, (1, 40)),
                     delta=rng.normal(0, 2, (1, 40)), phi=None)
    w = np.array([1.0, 0.5, -1.0])
    a = api().gradient(ctx, prob, 10, w, precision="c128", panels=1)
    b = api().gradient(ctx, prob, 10, w, precision="c128", panels=12)
    assert a.nodes == 4 * 8 and b.nodes == 4 * 96
    assert np.max(np.abs(a.d_omega - b.d_omega)) <= 1e-10
    assert np.max(np.abs(a.d_delta - b.d_delta)) <= 1e-10


def test_two_pass_size_against_finite_differences(ctx):
    """N = 14 complex128 (two streaming passes per matvec): sampled entries of
    the gradient against central differences of the forward solve."""
    n, t_ns, dt = 14, 20, 10
    rng = np.random.default_rng(14)
    pos = W.random_register(rng, n, 30.0, 7.0)
    om = rng.uniform(2, 6, (1, t_ns))
    de = rng.normal(0, 2, (1, t_ns))
    prob = W.Problem(positions=pos, c6=W.C6_DEFAULT, t_ns=t_ns, omega=om, delta=de, phi=None)
    w = rng.normal(size=n)
    g = api().gradient(ctx, prob, dt, w, precision="c128")

    def value(om_, de_):
        p = W.Problem(positions=pos, c6=W.C6_DEFAULT, t_ns=t_ns, omega=om_, delta=de_, phi=None)
        r = api().run(ctx, p, dt, "c128", krylov_tol=1e-14, obs_stride=0)
        occ = r.occupations()[-1]
        r.close()
        return float(occ @ w)

    assert abs(g.value - value(om, de)) <= 1e-10 * np.sum(np.abs(w))
    h = 1e-4
    for arr, grad, is_om in ((om, g.d_omega, True), (de, g.d_delta, False)):
        s = 5  # the first step's midpoint sample
        a, b = arr.copy(), arr.copy()
        a[0, s] += h
        b[0, s] -= h
        fd = (value(a, de) - value(b, de)) / (2 * h) if is_om else (value(om, a) - value(om, b)) / (2 * h)
        assert abs(grad[0, s] - fd) <= 1e-6 * max(1.0, abs(fd)), (is_om, grad[0, s], fd)


@pytest.mark.parametrize("n,prec", [(1, "c64"), (3, "c128"), (11, "c64"), (16, "c128"), (20, "c64")])
def test_overlap_matches_oracle(ctx, n, prec):
    g = torch.Generator(device="cuda").manual_seed(40 + n)
    a = torch.randn(2 ** n, dtype=TDT[prec], device="cuda", generator=g)
    b = torch.randn(2 ** n, dtype=TDT[prec], device="cuda", generator=g)
    ov, aa, bb = api().overlap(ctx, n, prec, a, b)
    r_ov, r_aa, r_bb = O.overlap(a.cpu().numpy(), b.cpu().numpy())
    scale = np.sqrt(r_aa * r_bb)
    assert abs(ov - r_ov) <= 1e-12 * scale
    assert abs(aa - r_aa) <= 1e-12 * r_aa and abs(bb - r_bb) <= 1e-12 * r_bb
    assert abs(api().fidelity(ctx, n, prec, a, a) - 1.0) <= 1e-12


def test_fidelity_at_chosen_times(ctx):
    """A solver stepped to chosen times: the fidelity of its state with the
    oracle's state at those times is 1 within the solve tolerance."""
    prob, _ = make_case(21, 5, 60, 1, 1, 1)
    s = api().Solver(ctx, prob, 10, precision="c128")
    psi = O.zero_state(5)
    V = O.pair_interactions(prob.positions, prob.c6)
    steps = O.step_parameters(5, 60, 10, prob.omega, prob.delta, prob.phi)
    import scipy.linalg
    for k, (tau, o, d, p) in enumerate(steps):
        psi = scipy.linalg.expm(-1j * tau * O.dense_hamiltonian(V, o, d, p)) @ psi
        s.step(1)
        if k in (1, 4):
            target = torch.tensor(psi, dtype=torch.complex128, device="cuda")
            cur = torch.tensor(s.state(), dtype=torch.complex128, device="cuda")
            assert 1.0 - api().fidelity(ctx, 5, "c128", target, cur) <= 1e-10
    s.close()
