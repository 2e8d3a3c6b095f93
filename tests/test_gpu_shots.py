"""GPU parity of shot-to-shot noise averaging (rsv_run_shots): the mean
occupation rows over perturbed copies of one problem against the oracle's
evolution of the same copies (same draws), averaged. Tolerances as for single
solves: 1e-10 (complex128) / 1e-5 (complex64) per occupation.
"""
import numpy as np
import pytest

from oracle import rydberg as O
from paper_2510_09813_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OCC_TOL = {"c128": 1e-10, "c64": 1e-5}


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


def oracle_mean(prob, dt, scale, shift, pos_shift):
    rows = []
    for k in range(len(scale)):
        pos = prob.positions + (pos_shift[k] if pos_shift is not None else 0.0)
        _, occ = O.evolve(pos, prob.c6, prob.t_ns, dt, prob.omega * scale[k], prob.delta + shift[k], prob.phi,
                          method="cheb")  # the oracle's Chebyshev path (pinned to its Lanczos path)
        rows.append(np.asarray(occ))
    return np.mean(rows, axis=0)


@pytest.mark.parametrize("n,prec,t_ns,with_pos", [(8, "c128", 300, True), (10, "c64", 200, False),
                                                   (13, "c128", 100, True), (21, "c64", 20, False)])
def test_shot_average_matches_oracle(ctx, n, prec, t_ns, with_pos):
    rng = np.random.Generator(np.random.PCG64(900 + n))
    prob = W.random_knot_problem(rng, n, t_ns)
    shots = 6 if n <= 20 else 2
    scale = rng.normal(1.0, 0.05, shots)
    shift = rng.normal(0.0, 0.5, shots)
    pos_shift = rng.normal(0.0, 0.1, (shots, n, 2)) if with_pos else None
    got = api().run_shots(ctx, prob, 10, scale, shift, pos_shift, precision=prec, obs_stride=1)
    ref = oracle_mean(prob, 10, scale, shift, pos_shift)
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) <= OCC_TOL[prec]


def test_unperturbed_shots_equal_one_solve(ctx):
    rng = np.random.Generator(np.random.PCG64(77))
    prob = W.random_knot_problem(rng, 9, 150)
    got = api().run_shots(ctx, prob, 10, np.ones(4), np.zeros(4), precision="c128", obs_stride=5)
    one = api().run(ctx, prob, 10, "c128", obs_stride=5)
    assert got.shape == one.occupations().shape
    assert np.max(np.abs(got - one.occupations())) <= 1e-10
    one.close()
