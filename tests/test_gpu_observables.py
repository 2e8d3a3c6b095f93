"""GPU parity of the extra observables: pair correlations <n_i n_j>
(rsv_correlations) and energy moments <H>, <H^2> (rsv_hamiltonian_expectation),
against the oracle and against closed forms at the full 28-atom size.

Tolerances: the correlations are FP64-class sums of exact products of the
state's own amplitudes, so they match the oracle's sums of the same values to
1e-12 relative. The energy moments inherit the matvec's rounding (FP64 /
FP32 sums of N + 1 terms per row): |d<H>| <= 10 * tol * scale * |psi|^2 and
|d<H^2>| <= 20 * tol * <H^2>, with tol = 1e-13 / 2e-6.
"""
import math

import numpy as np
import pytest

from oracle import rydberg as O
from paper_2510_09813_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MATVEC_TOL = {"c128": 1e-13, "c64": 2e-6}
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


def scale_of(V, om, de):
    return float(np.sum(np.abs(V)) / 2 + np.sum(np.abs(de)) + np.sum(np.abs(om)) / 2 + 1.0)


def setup(n, prec, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = W.random_register(rng, n, 5.0 * math.ceil(math.sqrt(n)) + 5.0, 5.0)
    V = O.pair_interactions(pos, W.C6_DEFAULT)
    om, de, ph = rng.uniform(1, 12, n), rng.normal(0, 5, n), rng.uniform(-math.pi, math.pi, n)
    g = torch.Generator(device="cuda").manual_seed(seed)
    psi = torch.randn(2 ** n, dtype=TDT[prec], device="cuda", generator=g) * 0.3
    return V, om, de, ph, psi


@pytest.mark.parametrize("n,prec", [(1, "c64"), (2, "c128"), (5, "c64"), (12, "c128"), (16, "c64"), (17, "c128"),
                                    (20, "c64")])
def test_correlations_match_oracle(ctx, n, prec):
    _, _, _, _, psi = setup(n, prec, 700 + n)
    got = api().correlations(ctx, n, prec, psi)
    ref = O.correlations(psi.cpu().numpy().astype(np.complex128))
    norm2 = float(np.sum(np.abs(psi.cpu().numpy().astype(np.complex128)) ** 2))
    assert got.shape == (n, n)
    assert np.max(np.abs(got - ref)) <= 1e-12 * norm2
    assert np.allclose(got, got.T, rtol=0, atol=1e-12 * norm2)


@pytest.mark.parametrize("n,prec", [(1, "c128"), (6, "c64"), (13, "c128"), (15, "c64"), (18, "c128"), (21, "c64")])
def test_energy_moments_match_oracle(ctx, n, prec):
    V, om, de, ph, psi = setup(n, prec, 800 + n)
    h = api().Hamiltonian(ctx, n, prec, V, om, de, ph)
    e1, e2 = h.expectation(psi)
    h.close()
    x = psi.cpu().numpy().astype(np.complex128)
    r1, r2 = O.energy_moments(x, V, om, de, ph)
    norm2 = float(np.vdot(x, x).real)
    assert abs(e1 - r1) <= 10 * MATVEC_TOL[prec] * scale_of(V, om, de) * norm2
    assert abs(e2 - r2) <= 20 * MATVEC_TOL[prec] * r2


def test_n28_closed_forms(ctx):
    """28 atoms, complex64, 2^28 amplitudes.
    |0...0>: <H> = 0 and <H^2> = |H|0>|^2 = sum_i Omega_i^2 / 4 (H|0> is the sum
    of the single excitations with amplitude Omega_i / 2).
    A product state prod_i (a_i|0> + b_i|1>): <n_i n_j> = |b_i|^2 |b_j|^2 for
    i != j and <n_i n_i> = |b_i|^2."""
    n = 28
    prob = W.random_box(seed=3, n=n)
    V = O.pair_interactions(prob.positions, prob.c6)
    om, de = prob.omega[:, 0], prob.delta[:, 0]
    zero = torch.zeros(2 ** n, dtype=torch.complex64, device="cuda")
    zero[0] = 1.0
    h = api().Hamiltonian(ctx, n, "c64", V, om, de, None)
    e1, e2 = h.expectation(zero)
    h.close()
    want = float(np.sum(om ** 2) / 4)
    assert abs(e1) <= 1e-6 * want
    assert abs(e2 - want) <= 1e-6 * want
    del zero
    ab = W.random_product_state(9, n)
    psi = torch.ones(1, dtype=torch.complex64, device="cuda")
    for i in range(n):  # atom 0 is the most significant bit
        psi = torch.kron(psi, torch.tensor(ab[i], dtype=torch.complex64, device="cuda"))
    C = api().correlations(ctx, n, "c64", psi)
    pb = np.abs(ab[:, 1]) ** 2
    ref = np.outer(pb, pb)
    np.fill_diagonal(ref, pb)
    assert np.max(np.abs(C - ref)) <= 1e-5
