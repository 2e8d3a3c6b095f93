"""GPU parity of the batched persistent path (rsv_batch_*) against the CPU
oracle and against the one-problem-at-a-time solver.

Tolerances as in test_gpu_parity: infidelity <= 1e-10 (complex128) / 1e-5
(complex64) against the oracle, occupations within 1e-10 / 1e-5. The batch
runs every register of a mixed-size list in one launch, so each register's
result must equal its own solve regardless of which CTA ran it or what ran
beside it.
"""
import math

import numpy as np
import pytest

from oracle import rydberg as O
from paper_2510_09813_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

INFID_TOL = {"c128": 1e-10, "c64": 1e-5}
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


def oracle_evolve(prob, dt, psi0=None):
    # the oracle's Chebyshev path (pinned to its Lanczos and dense paths)
    return O.evolve(prob.positions, prob.c6, prob.t_ns, dt, prob.omega, prob.delta, prob.phi, psi0=psi0,
                    method="cheb")


def mixed_problems(seed, sizes, t_ns, with_phi=False):
    out = []
    for k, n in enumerate(sizes):
        rng = np.random.Generator(np.random.PCG64([seed, k]))
        out.append(W.random_knot_problem(rng, n, t_ns, with_phi=with_phi))
    return out


# sizes span: below one warp of amplitudes, below the CTA width, one shared-
# memory chunk exactly, and several chunks (partner chunks read from memory)
SIZES = {"c64": [1, 3, 5, 8, 10, 12, 13, 14], "c128": [2, 4, 7, 9, 11, 12, 13]}


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("with_phi", [False, True])
def test_batch_matches_oracle(ctx, prec, with_phi):
    probs = mixed_problems(11 if with_phi else 10, SIZES[prec], 120, with_phi=with_phi)
    b = api().Batch(ctx, probs, 10, prec, obs_stride=1)
    b.run()
    for i, p in enumerate(probs):
        ref, occ_ref = oracle_evolve(p, 10)
        psi = b.state(i).astype(np.complex128)
        occ = b.occupations(i)
        assert occ.shape == occ_ref.shape
        assert O.infidelity(psi, ref) <= INFID_TOL[prec], (i, p.positions.shape[0])
        if prec == "c128":
            assert O.norm_difference(psi, ref) <= 1e-9
        assert np.max(np.abs(occ - occ_ref)) <= OCC_TOL[prec]
    st = b.stats()
    assert st["steps"] == 12 * len(probs)
    b.close()


def test_batch_full_sequence_and_initial_states(ctx):
    """8-knot pulses over 301 ns with dt = 7 (43 steps, a ragged last step),
    random initial states, occupation rows every 10 steps and at the end."""
    sizes = [6, 9, 11, 13]
    probs = mixed_problems(12, sizes, 301)
    inits = [W.random_state(50 + k, n) for k, n in enumerate(sizes)]
    b = api().Batch(ctx, probs, 7, "c128", obs_stride=10, initial_states=inits)
    b.run()
    for i, p in enumerate(probs):
        ref, occ_ref = oracle_evolve(p, 7, psi0=inits[i])
        psi = b.state(i)
        assert O.infidelity(psi, ref) <= 1e-10
        occ = b.occupations(i)
        rows = [0] + [k for k in range(1, len(occ_ref)) if k % 10 == 0 or k == len(occ_ref) - 1]
        assert np.max(np.abs(occ - occ_ref[rows])) <= 1e-10
    b.close()


def test_batch_matches_solver_up_to_18_atoms(ctx):
    """Registers of 15-18 atoms (several chunks) against the streaming solver in
    complex128, itself oracle-checked at these sizes."""
    sizes = [18, 15, 17, 16, 10]
    probs = mixed_problems(13, sizes, 60)
    b = api().Batch(ctx, probs, 10, "c64", obs_stride=1)
    b.run()
    for i, p in enumerate(probs):
        s = api().Solver(ctx, p, 10, "c128", obs_stride=1)
        s.run_to_end()
        ref, occ_ref = s.state(), s.occupations()
        s.close()
        assert O.infidelity(b.state(i).astype(np.complex128), ref) <= 1e-5
        assert np.max(np.abs(b.occupations(i) - occ_ref)) <= 1e-5
    b.close()


@pytest.mark.parametrize("prec,sizes", [("c128", [15, 16, 11]), ("c64", [17, 15, 12, 9])])
def test_batch_cooperative_registers_match_oracle(ctx, prec, sizes):
    """Registers of 15 atoms and more are solved by a whole thread-block cluster
    (chunks split across its CTAs, sums and Krylov decisions through
    distributed shared memory); smaller ones in the same launch by one CTA."""
    probs = mixed_problems(16, sizes, 50, with_phi=True)
    b = api().Batch(ctx, probs, 10, prec, obs_stride=1)
    b.run()
    for i, p in enumerate(probs):
        ref, occ_ref = oracle_evolve(p, 10)
        assert O.infidelity(b.state(i).astype(np.complex128), ref) <= INFID_TOL[prec]
        assert np.max(np.abs(b.occupations(i) - occ_ref)) <= OCC_TOL[prec]
    b.close()


def test_batch_rerun_is_identical_and_restarts(ctx):
    """A second run (graph replay) repeats the first bit for bit; a small m_max
    forces substeps that must not change the result beyond tolerance."""
    probs = mixed_problems(14, [12, 7, 14, 9, 13, 11], 80)
    b = api().Batch(ctx, probs, 20, "c128", m_max=8, max_substeps=200)
    b.run()
    first = [b.state(i).copy() for i in range(len(probs))]
    st = b.stats()
    assert st["substeps"] > 0
    b.run()
    for i, p in enumerate(probs):
        assert np.array_equal(b.state(i), first[i])
        ref, _ = oracle_evolve(p, 20)
        assert O.infidelity(first[i], ref) <= 1e-10
    b.close()


def test_batch_alone_equals_in_mix(ctx):
    """Each register's result is the same alone and inside a larger batch."""
    probs = mixed_problems(15, [11, 13, 9, 14, 12, 10, 13, 8], 50)
    mix = api().Batch(ctx, probs, 10, "c64")
    mix.run()
    for i in (0, 3, 6):
        alone = api().Batch(ctx, [probs[i]], 10, "c64")
        alone.run()
        assert np.array_equal(alone.state(0), mix.state(i))
        alone.close()
    mix.close()


def test_run_batch_mixes_batched_and_streaming(ctx):
    """rsv_run_batch: the registers of at most 20 atoms share one batched
    launch and match their complex128 streaming solves; the 21-atom problem
    runs on the streaming solver and equals rsv_run exactly."""
    probs = mixed_problems(31, [9, 21, 6, 12], 50)
    res = api().run_batch(ctx, probs, 10, "c64", obs_stride=1)
    assert len(res) == len(probs)
    for r, p in zip(res, probs):
        n = p.positions.shape[0]
        if n <= 20:
            s = api().Solver(ctx, p, 10, "c128", obs_stride=1)
            s.run_to_end()
            ref, occ_ref = s.state(), s.occupations()
            s.close()
            assert O.infidelity(r.state().astype(np.complex128), ref) <= 1e-5
            assert np.max(np.abs(r.occupations() - occ_ref)) <= 1e-5
        else:
            one = api().run(ctx, p, 10, "c64", obs_stride=1)
            assert np.array_equal(r.state(), one.state())
            assert np.array_equal(r.occupations(), one.occupations())
            one.close()
        assert r.stats()["steps"] == 5
    for r in res:
        r.close()


def test_batch_rejects_large_registers(ctx):
    rng = np.random.Generator(np.random.PCG64(3))
    big = W.random_knot_problem(rng, 21, 20)
    with pytest.raises(api().RsvError, match="batched limit"):
        api().Batch(ctx, [big], 10, "c64")


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_batch_autotuned_depth(ctx, prec):
    """m_max < 0: the batch times its Krylov-depth candidates on a sample of
    the registers and keeps one of them; the registers then match the oracle."""
    sizes = [10, 16, 12, 14, 11, 15, 13, 10, 16, 12, 14, 11]
    probs = mixed_problems(51, sizes, 120)
    b = api().Batch(ctx, probs, 10, prec, m_max=-1, obs_stride=1)
    b.run()
    st = b.stats()
    assert st["krylov_dim_max"] in (12, 16, 20, 24, 32, 40)
    for i in (0, 1, 5, 11):
        ref, occ_ref = oracle_evolve(probs[i], 10)
        psi = b.state(i).astype(np.complex128)
        assert O.infidelity(psi, ref) <= INFID_TOL[prec], i
        assert np.max(np.abs(b.occupations(i) - occ_ref)) <= OCC_TOL[prec]
    b.close()
