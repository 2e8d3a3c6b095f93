"""GPU tests of the request server (rsv_server_*, rsv_submit, rsv_poll).

Requests of mixed size and precision are submitted while others run; each
result must be the same as the same request solved alone (rsv_run on the
same context) within the parity tolerances (infidelity 1e-10 for
complex128, 1e-5 for complex64; occupations 1e-10 / 1e-5), and admission must
keep the bytes held by running solves within the server's memory.
"""
import threading
import time

import numpy as np
import pytest

from oracle import rydberg as O
from paper_2510_09813_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

INFID_TOL = {"c128": 1e-10, "c64": 1e-5}
OCC_TOL = {"c128": 1e-10, "c64": 1e-5}


def api():
    from paper_2510_09813_b300 import api as A
    return A


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    c = api().Context(0, arena_bytes=24 << 30)
    yield c
    c.close()


def requests(seed, sizes, t_lo=60, t_hi=200):
    out = []
    for k, n in enumerate(sizes):
        rng = np.random.Generator(np.random.PCG64([seed, k]))
        t_ns = int(rng.integers(t_lo, t_hi + 1))
        prec = "c64" if k % 2 == 0 else "c128"
        out.append((W.random_knot_problem(rng, n, t_ns), prec))
    return out


def test_results_alone_equal_in_mix(ctx):
    """Each request's result is the same served alone and served in a mix of
    requests that run concurrently on their own streams."""
    reqs = requests(21, [14, 9, 20, 12, 17, 11, 22, 15, 8, 19, 13, 16, 12, 12, 9, 9])
    srv = api().Server(ctx, slots=4)
    t_sub, tickets = [], []
    for p, prec in reqs:
        t_sub.append(time.perf_counter())
        tickets.append(srv.submit(p, 10, prec, obs_stride=1))
    results = [srv.poll(t, timeout_ms=-1) for t in tickets]
    srv.close()
    # the mix really ran concurrently: service intervals [admission, completion]
    # (host submission time + the server's wait and service times) overlap
    spans = []
    for ts, r in zip(t_sub, results):
        w, sv = r.times()
        spans.append((ts + w, ts + w + sv))
    overlaps = sum(1 for i in range(len(spans)) for j in range(i + 1, len(spans))
                   if min(spans[i][1], spans[j][1]) - max(spans[i][0], spans[j][0]) > 1e-3)
    assert overlaps >= 3, spans
    for (p, prec), r in zip(reqs, results):
        one = api().Server(ctx, slots=1)
        alone = one.poll(one.submit(p, 10, prec, obs_stride=1))
        a, b = alone.state(), r.state()
        # same kernels, same fixed reduction trees: the mix changes nothing at all
        assert np.array_equal(a, b)
        assert np.array_equal(alone.occupations(), r.occupations())
        # and against the streaming solver run directly, within the tolerance
        ref = api().run(ctx, p, 10, prec, obs_stride=1)
        assert O.infidelity(b.astype(np.complex128), ref.state().astype(np.complex128)) <= INFID_TOL[prec]
        assert np.max(np.abs(r.occupations() - ref.occupations())) <= OCC_TOL[prec]
        w, sv = r.times()
        assert w >= 0.0 and sv > 0.0
        for x in (alone, ref, r):
            x.close()
        one.close()


@pytest.mark.parametrize("sizes,t_ns", [([10] * 8, [100] * 8),
                                         ([10, 13, 16, 11, 18, 12, 15, 14], [100, 60, 140, 80, 100, 120, 60, 90])])
def test_batched_lane_groups_requests(ctx, sizes, t_ns):
    """With batch_atoms set, requests of at most that many atoms and the same
    config queued together are solved by one batched launch (they share
    admission and completion times), whatever their sizes and durations. Each
    result is bit for bit the request's own batched solve (a batch of one: a
    register's computation does not depend on its batch neighbours), and
    within the tolerance of the streaming solver; a request served alone
    with nothing to group with runs on the streaming solver."""
    probs = [W.random_knot_problem(np.random.Generator(np.random.PCG64([31, k])), n, t)
             for k, (n, t) in enumerate(zip(sizes, t_ns))]
    srv = api().Server(ctx, slots=1, batch_atoms=20)
    tickets = [srv.submit(p, 10, "c64", obs_stride=1) for p in probs]
    results = [srv.poll(t) for t in tickets]
    srv.close()
    service = [r.times()[1] for r in results]
    # the first request may have started alone before the others were queued
    assert max(service.count(v) for v in service) >= 2
    for p, r in zip(probs, results):
        ref = api().run(ctx, p, 10, "c64", obs_stride=1)
        assert O.infidelity(r.state().astype(np.complex128), ref.state().astype(np.complex128)) <= INFID_TOL["c64"]
        assert np.max(np.abs(r.occupations() - ref.occupations())) <= OCC_TOL["c64"]
        if service.count(r.times()[1]) >= 2:
            (own,) = api().run_batch(ctx, [p], 10, "c64", obs_stride=1)
            assert np.array_equal(own.state(), r.state())
            own.close()
        else:
            assert np.array_equal(ref.state(), r.state())
        for x in (ref, r):
            x.close()
    one = api().Server(ctx, slots=1, batch_atoms=20)
    alone = one.poll(one.submit(probs[0], 10, "c64", obs_stride=1))
    ref = api().run(ctx, probs[0], 10, "c64", obs_stride=1)
    assert np.array_equal(alone.state(), ref.state())
    for x in (alone, ref):
        x.close()
    one.close()


def test_served_result_matches_oracle(ctx):
    rng = np.random.Generator(np.random.PCG64(77))
    p = W.random_knot_problem(rng, 10, 150, with_phi=True)
    srv = api().Server(ctx, slots=2)
    t = srv.submit(p, 10, "c128", obs_stride=1)
    r = srv.poll(t)
    ref, occ_ref = O.evolve(p.positions, p.c6, p.t_ns, 10, p.omega, p.delta, p.phi, method="cheb")
    assert O.infidelity(r.state(), ref) <= 1e-10
    assert np.max(np.abs(r.occupations() - occ_ref)) <= 1e-10
    r.close()
    srv.close()


def test_admission_respects_memory(ctx):
    """A server whose memory holds about two of these solves never runs more
    than fits; every request still completes, also the ones that waited."""
    reqs = requests(22, [21, 21, 21, 21, 21, 21], t_lo=40, t_hi=60)
    reqs = [(p, "c128") for p, _ in reqs]
    one = api().footprint_bytes(21, "c128", 30)
    srv = api().Server(ctx, slots=6, memory_bytes=int(2.5 * one), max_bypass_s=-1)
    peak = {"bytes": 0, "running": 0}
    stop = threading.Event()

    def sample():
        while not stop.is_set():
            q, r, b = srv.load()
            peak["bytes"] = max(peak["bytes"], b)
            peak["running"] = max(peak["running"], r)
            time.sleep(0.001)

    th = threading.Thread(target=sample)
    th.start()
    tickets = [srv.submit(p, 10, prec) for p, prec in reqs]
    results = [srv.poll(t) for t in tickets]
    stop.set()
    th.join()
    assert peak["bytes"] <= int(2.5 * one)
    assert 1 <= peak["running"] <= 2
    waits = [r.times()[0] for r in results]
    assert max(waits) > 0.0
    for r in results:
        r.close()
    srv.close()


def test_errors(ctx):
    A = api()
    srv = A.Server(ctx, slots=1, memory_bytes=64 << 20)
    rng = np.random.Generator(np.random.PCG64(5))
    big = W.random_knot_problem(rng, 22, 20)
    with pytest.raises(A.RsvError) as e:
        srv.submit(big, 10, "c128")
    assert e.value.code == -2
    with pytest.raises(A.RsvError) as e:
        srv.poll(12345, 0)
    assert e.value.code == -7
    # 2000 one-ns steps cannot finish within the first poll
    small = W.random_knot_problem(rng, 10, 2000)
    t = srv.submit(small, 1, "c128")
    assert srv.poll(t, 0) is None
    r = srv.poll(t, -1)
    assert r is not None
    with pytest.raises(A.RsvError) as e:
        srv.poll(t, 0)  # retired once claimed
    assert e.value.code == -7
    r.close()
    srv.close()


def test_running_count_shows_concurrency(ctx):
    """While a burst is served by 4 slots, the server reports more than one
    solve running at the same time."""
    reqs = requests(23, [20, 20, 20, 20, 20, 20], t_lo=150, t_hi=200)
    srv = api().Server(ctx, slots=4)
    peak = {"running": 0}
    stop = threading.Event()

    def sample():
        while not stop.is_set():
            peak["running"] = max(peak["running"], srv.load()[1])
            time.sleep(0.0005)

    th = threading.Thread(target=sample)
    th.start()
    tickets = [srv.submit(p, 10, prec, obs_stride=0) for p, prec in reqs]
    results = [srv.poll(t) for t in tickets]
    stop.set()
    th.join()
    assert peak["running"] >= 2
    for r in results:
        r.close()
    srv.close()


def test_unfreed_results_delay_admission(ctx):
    """A finished result keeps its state charged to the server's memory until
    it is freed: with room for one solve plus half a state, the next request
    waits (it does not fail) while the first result is held, and runs once
    that result is freed. The charge of a held result is its state alone."""
    A = api()
    rng = np.random.Generator(np.random.PCG64(41))
    p1 = W.random_knot_problem(rng, 16, 60)
    p2 = W.random_knot_problem(rng, 16, 60)
    need = A.request_bytes(p1, 10, "c128", m_max=12, obs_stride=0)
    assert need == A.request_bytes(p2, 10, "c128", m_max=12, obs_stride=0)
    state = (2 ** 16) * 16
    srv = A.Server(ctx, slots=2, memory_bytes=need + state // 2, max_bypass_s=-1)
    r1 = srv.poll(srv.submit(p1, 10, "c128", m_max=12, obs_stride=0))
    q, running, held = srv.load()
    assert running == 0 and held == state
    t2 = srv.submit(p2, 10, "c128", m_max=12, obs_stride=0)
    assert srv.poll(t2, 300) is None  # waits behind the held state
    q, running, held = srv.load()
    assert q == 1 and running == 0
    ref1 = A.run(ctx, p1, 10, "c128", m_max=12, obs_stride=0)
    assert np.array_equal(r1.state(), ref1.state())  # the held state is intact
    r1.close()
    r2 = srv.poll(t2, -1)
    assert r2 is not None
    ref2 = A.run(ctx, p2, 10, "c128", m_max=12, obs_stride=0)
    assert np.array_equal(r2.state(), ref2.state())
    r2.close()
    assert srv.load()[2] == 0
    for x in (ref1, ref2):
        x.close()
    srv.close()
