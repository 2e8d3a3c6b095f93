"""rsv_observe_static (the context-free, allocation-free observation entry)
against rsv_observe on the same seeded device states.

Both entries run the same FP64 reductions (exact products, compensated sums),
so |psi|^2 agrees to a relative 1e-13 and every <n_i> to 1e-13 * |psi|^2.
Each case calls the static entry twice in a row into outputs pre-filled with
NaN, and checks that those calls change neither the device's free memory nor
torch's allocator. Named to be collected after the other test files.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-13
TDT = {"c128": torch.complex128, "c64": torch.complex64}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2510_09813_b300 import api
    c = api.Context(0)
    yield c
    c.close()


def _state(n, precision, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    psi = torch.randn(2 ** n, dtype=TDT[precision], device="cuda", generator=g)
    # a few exact zeros and a non-unit norm, as a mid-run state can have
    psi[:: 7] = 0
    return psi * 0.37


@pytest.mark.parametrize("n,precision", [(1, "c128"), (3, "c64"), (12, "c64"), (17, "c128"), (20, "c64"),
                                         (22, "c128"), (26, "c64")])
def test_static_matches_observe_twice(ctx, n, precision):
    from paper_2510_09813_b300 import api
    psi = _state(n, precision, seed=1000 + n)
    norm2_ref, occ_ref = api.observe(ctx, n, precision, psi)
    # first call on the device does the set-up; then two calls in a row
    warm = torch.full((n + 1,), float("nan"), dtype=torch.float64, device="cuda")
    api.observe_static(n, precision, psi, warm)
    torch.cuda.synchronize()
    outs = [torch.full((n + 1,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    free0 = torch.cuda.mem_get_info()[0]
    alloc0 = torch.cuda.memory_allocated()
    for out in outs:
        api.observe_static(n, precision, psi, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    for out in [warm] + outs:
        o = out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert abs(o[0] - norm2_ref) <= TOL * norm2_ref
        np.testing.assert_allclose(o[1:], occ_ref, rtol=0, atol=TOL * norm2_ref)


def test_static_on_side_stream(ctx):
    from paper_2510_09813_b300 import api
    n = 21
    psi = _state(n, "c64", seed=7)
    norm2_ref, occ_ref = api.observe(ctx, n, "c64", psi)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    out = torch.full((n + 1,), float("nan"), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(s):
        api.observe_static(n, "c64", psi, out, stream=s)
        api.observe_static(n, "c64", psi, out, stream=s)
    s.synchronize()
    o = out.cpu().numpy()
    assert abs(o[0] - norm2_ref) <= TOL * norm2_ref
    np.testing.assert_allclose(o[1:], occ_ref, rtol=0, atol=TOL * norm2_ref)


def test_static_rejects_beyond_limit(ctx):
    """Host-side checks: nothing is launched for these calls."""
    from paper_2510_09813_b300 import _lib as L
    psi = _state(4, "c64", seed=3)
    out = torch.zeros(40, dtype=torch.float64, device="cuda")
    lib = L.lib()
    p, o = C.c_void_p(psi.data_ptr()), C.c_void_p(out.data_ptr())
    assert lib.rsv_observe_static(32, L.RSV_C64, p, o, None) == -1
    assert "limit of 31 atoms" in lib.rsv_last_error().decode()
    assert lib.rsv_observe_static(0, L.RSV_C64, p, o, None) == -1
    assert lib.rsv_observe_static(4, 7, p, o, None) == -1
    assert lib.rsv_observe_static(4, L.RSV_C64, None, o, None) == -1
    assert lib.rsv_observe_static(4, L.RSV_C64, p, C.c_void_p(out.data_ptr() + 4), None) == -1
    assert lib.rsv_observe_static(4, L.RSV_C64, C.c_void_p(psi.data_ptr() + 8), o, None) == -1
    # host memory in place of a device buffer is refused before any launch
    host = np.zeros(40)
    h = C.c_void_p(host.ctypes.data)
    assert lib.rsv_observe_static(4, L.RSV_C64, p, h, None) == -1
    assert "device memory of the current device" in lib.rsv_last_error().decode()
    hpsi = np.zeros(2 ** 4, dtype=np.complex64)
    assert lib.rsv_observe_static(4, L.RSV_C64, C.c_void_p(hpsi.ctypes.data), o, None) == -1
