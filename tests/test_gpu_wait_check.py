"""Failure detection without a GPU fault: a device wait that nothing completes
gives up after its time limit, the kernel sets an error word and returns, the
host reports RSV_ERR_TIMEOUT, and the context keeps working."""
import numpy as np
import pytest

from oracle import rydberg as O
from paper_2510_09813_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2510_09813_b300 import api
    c = api.Context(0)
    yield c
    c.close()


def test_bounded_wait_reports_timeout_and_context_survives(ctx):
    from paper_2510_09813_b300 import _lib as L
    from paper_2510_09813_b300 import api
    assert L.lib().rsv_check_bounded_wait(ctx.handle) == -4  # RSV_ERR_TIMEOUT
    assert b"timed out" in L.lib().rsv_last_error()
    prob = W.rabi_chain(t_ns=100)
    r = api.run(ctx, prob, 10, "c128", obs_stride=0)
    psi = r.state()
    r.close()
    ref, _ = O.evolve(prob.positions, prob.c6, prob.t_ns, 10, prob.omega, prob.delta, prob.phi, method="dense")
    assert O.infidelity(psi, ref) <= 1e-10
    assert np.isclose(np.vdot(psi, psi).real, 1.0, rtol=0, atol=1e-12)
