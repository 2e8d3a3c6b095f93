"""GPU parity of the prepared Hamiltonian operator (rsv_hamiltonian_*).

The operator runs the same streaming passes as rsv_apply_hamiltonian with
tables built once, so its products equal the one-shot call's exactly; against
the oracle the matvec tolerance of test_gpu_parity applies (FP64 / FP32
rounding of a sum of N + 1 terms).
"""
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


def setup(n, prec, seed, with_phi):
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = W.random_register(rng, n, 5.0 * np.ceil(np.sqrt(n)) + 5.0, 5.0)
    V = O.pair_interactions(pos, W.C6_DEFAULT)
    om = rng.uniform(1.0, 12.0, n)
    de = rng.normal(0.0, 5.0, n)
    ph = rng.uniform(-np.pi, np.pi, n) if with_phi else None
    g = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.randn(2 ** n, dtype=TDT[prec], device="cuda", generator=g)
    return V, om, de, ph, x


@pytest.mark.parametrize("n,prec", [(3, "c64"), (12, "c64"), (13, "c128"), (15, "c64"), (17, "c128"), (20, "c64"),
                                    (22, "c64"), (21, "c128")])
@pytest.mark.parametrize("with_phi", [False, True])
def test_operator_equals_one_shot(ctx, n, prec, with_phi):
    V, om, de, ph, x = setup(n, prec, 400 + n, with_phi)
    y0 = torch.empty_like(x)
    api().apply_hamiltonian(ctx, n, prec, V, om, de, ph, x, y0)
    h = api().Hamiltonian(ctx, n, prec, V, om, de, ph)
    y1 = torch.full_like(x, float("nan"))
    y2 = torch.full_like(x, float("nan"))
    h.apply(x, y1)
    h.apply(x, y2)  # twice in a row, same operands
    h.sync()
    assert torch.equal(y1, y0) and torch.equal(y2, y0)
    h.close()


@pytest.mark.parametrize("n,prec", [(11, "c128"), (16, "c64"), (19, "c128")])
def test_operator_matches_oracle(ctx, n, prec):
    V, om, de, ph, x = setup(n, prec, 500 + n, True)
    h = api().Hamiltonian(ctx, n, prec, V, om, de, ph)
    y = torch.empty_like(x)
    h.apply(x, y)
    h.sync()
    xr = x.cpu().numpy().astype(np.complex128)
    ref = O.apply_hamiltonian(xr, V, om, de, ph)
    scale = float(np.sum(np.abs(V)) / 2 + np.sum(np.abs(de)) + np.sum(np.abs(om)) / 2 + 1.0)
    err = np.max(np.abs(y.cpu().numpy() - ref))
    assert err <= MATVEC_TOL[prec] * scale * np.max(np.abs(xr))
    h.close()


def test_operator_alternating_operands(ctx):
    """The cached tensor maps follow the operands: ping-pong between buffers."""
    n, prec = 18, "c64"
    V, om, de, ph, x = setup(n, prec, 77, False)
    h = api().Hamiltonian(ctx, n, prec, V, om, de, ph)
    a, b = x.clone(), torch.empty_like(x)
    for _ in range(3):
        h.apply(a, b)
        h.apply(b, a)
    h.sync()
    ref = x.clone()
    tmp = torch.empty_like(x)
    for _ in range(3):
        api().apply_hamiltonian(ctx, n, prec, V, om, de, ph, ref, tmp)
        api().apply_hamiltonian(ctx, n, prec, V, om, de, ph, tmp, ref)
    assert torch.equal(a, ref)
    h.close()
