"""The request server (cg_server_* in include/cellgraph.h).

Serving must never change a result: every request's cells and edges are
compared bit for bit with the oracle, and with the same request served alone,
in a mix of concurrently running requests, and under an HBM budget so small
that admission has to hold requests back. Failures are made on the host only
(an injected allocation failure, a request larger than the whole budget, a
shutdown with requests still queued); no GPU fault is involved.
"""
import time

import numpy as np
import pytest

import oracle
from paper_1503_06029_gb300 import cellgraph, inputs

torch = pytest.importorskip("torch")


def _scenes(n_scenes, n_hi, seed):
    spec = inputs.scene_batch_spec(n_scenes=n_scenes, seed=seed, n_hi=n_hi)
    return [inputs.batch_scene(spec, s) for s in range(n_scenes)]


def _degenerate(seed=3):
    """Thirty-two constraints through the origin with repeated normals: far more
    points land exactly on constraints than in general position, so the
    vectors outnumber the first table-size guess and the request is re-run."""
    rng = np.random.default_rng(seed)
    base = rng.integers(-50, 51, size=(8, 2)).astype(np.int32)
    a = np.concatenate([base, -base, base, -base])
    return inputs.Scene(pts=rng.integers(-300, 301, size=(50_000, 2)).astype(np.int32), a=a,
                        b=np.zeros(32, np.int64))


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def wanted():
    cache = {}

    def get(key, sc):
        if key not in cache:
            cache[key] = oracle.build(sc.pts, sc.a, sc.b, 64)
        return cache[key]

    return get


def _check(srv, t, sc, want):
    r = srv.result(t)
    assert r["status"] == 0, r["error"]
    cells, edges = srv.fetch(t)
    want_c, want_e = want
    assert np.array_equal(cells.reshape(want_c.shape), want_c)
    assert np.array_equal(edges, want_e)
    return cells, edges


@pytest.mark.gpu
def test_each_result_is_the_same_alone_and_in_the_mix(dev, wanted):
    scenes = _scenes(24, 60_000, seed=21) + [inputs.planes_3d(n=0, ell=24, seed=1), _degenerate()]
    with cellgraph.Server(0, hbm_budget_bytes=4 << 30, max_inflight=8) as srv:
        alone = []
        for i, sc in enumerate(scenes):
            t = srv.submit(sc.pts, sc.a, sc.b)
            assert srv.wait(t, 60.0)
            assert srv.poll(t) == cellgraph.REQ_DONE
            alone.append(_check(srv, t, sc, wanted(i, sc)))
            srv.release(t)
        # All at once: requests overlap on the device.
        tickets = [srv.submit(sc.pts, sc.a, sc.b) for sc in scenes]
        for i, (t, sc) in enumerate(zip(tickets, scenes)):
            assert srv.wait(t, 120.0)
            c, e = _check(srv, t, sc, wanted(i, sc))
            assert np.array_equal(c, alone[i][0]) and np.array_equal(e, alone[i][1])
        st = srv.stats()
        assert st["max_running"] > 1, st
        assert st["failed"] == 0
        for t in tickets:
            srv.release(t)
        assert srv.stats()["bytes_in_use"] == 0


@pytest.mark.gpu
def test_requests_that_outgrow_their_first_capacity_are_rerun(dev, wanted, monkeypatch):
    # A first table guess of 1024 slots (512 vectors) is too small for most of
    # these scenes: they overflow, are re-queued with larger capacities, and
    # still give exactly the oracle's output.
    monkeypatch.setenv("CG_FIRST_TABLE_CAP", "1024")
    scenes = _scenes(10, 150_000, seed=27)
    with cellgraph.Server(0, hbm_budget_bytes=4 << 30, max_inflight=4) as srv:
        ts = [srv.submit(sc.pts, sc.a, sc.b) for sc in scenes]
        for i, (t, sc) in enumerate(zip(ts, scenes)):
            assert srv.wait(t, 120.0)
            _check(srv, t, sc, wanted(("r", i), sc))
        assert srv.stats()["retried"] >= 1
        assert sum(srv.result(t)["retries"] for t in ts) == srv.stats()["retried"]


@pytest.mark.gpu
def test_small_budget_holds_requests_back_without_changing_results(dev, wanted):
    scenes = _scenes(12, 80_000, seed=22)
    with cellgraph.Server(0, hbm_budget_bytes=64 << 30, max_inflight=4) as big:
        t = big.submit(scenes[0].pts, scenes[0].a, scenes[0].b)
        big.wait(t)
        one = big.stats()["peak_bytes"]
        big.release(t)
    budget = 2 * one + one // 2  # about two requests of the first one's size
    with cellgraph.Server(0, hbm_budget_bytes=budget, max_inflight=8) as srv:
        tickets = [(i, srv.submit(sc.pts, sc.a, sc.b)) for i, sc in enumerate(scenes)]
        for i, t in tickets:
            srv.wait(t, 120.0)
            r = srv.result(t)
            if r["status"] == cellgraph.ERR_CAPACITY:  # larger than the whole budget
                continue
            _check(srv, t, scenes[i], wanted(("b", i), scenes[i]))
            srv.release(t)  # frees its memory for the next admissions
        st = srv.stats()
        assert st["peak_bytes"] <= budget, st
        assert st["completed"] >= 1


@pytest.mark.gpu
def test_request_larger_than_the_budget_fails_alone(dev, wanted):
    small = _scenes(3, 5_000, seed=23)
    big = inputs.planes_3d(n=400_000, ell=64, seed=5)
    with cellgraph.Server(0, hbm_budget_bytes=4 << 20, max_inflight=4) as srv:
        t_big = srv.submit(big.pts, big.a, big.b)
        ts = [srv.submit(sc.pts, sc.a, sc.b) for sc in small]
        assert srv.wait(t_big, 60.0)
        r = srv.result(t_big)
        assert r["status"] == cellgraph.ERR_CAPACITY
        assert "budget" in r["error"]
        for i, (t, sc) in enumerate(zip(ts, small)):
            assert srv.wait(t, 60.0)
            _check(srv, t, sc, wanted(("s", i), sc))


@pytest.mark.gpu
def test_injected_allocation_failure_fails_one_request(dev, wanted):
    scenes = _scenes(6, 20_000, seed=24)
    with cellgraph.Server(0, hbm_budget_bytes=2 << 30, max_inflight=1) as srv:
        srv.inject_alloc_failures(1)
        ts = [srv.submit(sc.pts, sc.a, sc.b) for sc in scenes]
        statuses = []
        for t in ts:
            assert srv.wait(t, 60.0)
            statuses.append(srv.result(t)["status"])
        assert statuses[0] == cellgraph.ERR_OOM  # the first admitted request
        assert statuses[1:] == [0] * (len(scenes) - 1)
        for i in range(1, len(scenes)):
            _check(srv, ts[i], scenes[i], wanted(("i", i), scenes[i]))
        with pytest.raises(cellgraph.CellGraphError):
            srv.fetch(ts[0])
        # The server keeps serving: the same scene again succeeds.
        t = srv.submit(scenes[0].pts, scenes[0].a, scenes[0].b)
        assert srv.wait(t, 60.0)
        _check(srv, t, scenes[0], wanted(("i", 0), scenes[0]))
        assert srv.stats()["failed"] == 1


@pytest.mark.gpu
def test_device_inputs_and_latency_stamps(dev, wanted):
    scenes = _scenes(8, 40_000, seed=25)
    with cellgraph.Server(0, hbm_budget_bytes=2 << 30, max_inflight=4) as srv:
        dts = [tuple(torch.from_numpy(x).to(dev) for x in (s.pts, s.a, s.b)) for s in scenes]
        torch.cuda.synchronize()
        ts = [srv.submit(*d) for d in dts]
        for i, t in enumerate(ts):
            assert srv.wait(t, 60.0)
            _check(srv, t, scenes[i], wanted(("d", i), scenes[i]))
            r = srv.result(t)
            assert 0 <= r["submit_us"] <= r["admit_us"] <= r["done_us"]
        with pytest.raises(cellgraph.CellGraphError):
            srv.release(12345)


@pytest.mark.gpu
def test_shutdown_with_queued_requests(dev):
    scenes = _scenes(10, 200_000, seed=26)
    srv = cellgraph.Server(0, hbm_budget_bytes=2 << 30, max_inflight=1)
    ts = [srv.submit(sc.pts, sc.a, sc.b) for sc in scenes]
    t0 = time.time()
    srv.close()  # running requests finish, queued ones fail, memory is freed
    assert time.time() - t0 < 60.0


@pytest.mark.gpu
def test_invalid_submissions_are_rejected(dev):
    with cellgraph.Server(0, hbm_budget_bytes=1 << 30, max_inflight=2) as srv:
        sc = inputs.lines_2d(n=100)
        with pytest.raises(cellgraph.CellGraphError):
            srv.submit(sc.pts, sc.a[:0], sc.b[:0])  # l = 0
        with pytest.raises(cellgraph.CellGraphError):
            srv.submit(np.zeros((4, 5), np.int32), np.zeros((3, 5), np.int32),
                       np.zeros(3, np.int64))  # d = 5


def test_create_without_a_device_is_refused():
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    try:
        lib = cellgraph.load_library()
    except (OSError, cellgraph.CellGraphError):
        pytest.skip("library not built")
    import ctypes

    h = ctypes.c_void_p()
    assert lib.cg_server_create(0, 1 << 30, 4, ctypes.byref(h)) != 0
    assert lib.cg_server_create(0, 1 << 30, 0, ctypes.byref(h)) == cellgraph.ERR_INVALID_ARG
    assert lib.cg_server_destroy(None) == 0


@pytest.mark.gpu
def test_pinned_host_inputs(dev, wanted):
    """Requests whose host arrays are pinned (asynchronous copies into the
    work block) give the same results."""
    scenes = _scenes(8, 80_000, seed=28)
    pin = lambda x: torch.from_numpy(x).pin_memory().numpy()
    pinned = [(pin(s.pts), pin(s.a), pin(s.b)) for s in scenes]
    with cellgraph.Server(0, hbm_budget_bytes=2 << 30, max_inflight=4) as srv:
        ts = [srv.submit(*p) for p in pinned]
        for i, (t, sc) in enumerate(zip(ts, scenes)):
            assert srv.wait(t, 60.0)
            _check(srv, t, sc, wanted(("p", i), sc))


@pytest.mark.gpu
@pytest.mark.parametrize("where", ["host", "pinned", "device"])
def test_requests_started_together_match_the_oracle(dev, wanted, where):
    """Many l <= 64 scenes at once: the scheduler starts the requests it admits
    in one pass together through the segmented kernels (one sign + insert
    launch, one sort and one search for all of them). Every result is the
    oracle's, whether the inputs are pageable or pinned host arrays (copied
    into each request's block) or device arrays."""
    spec = inputs.scene_batch_spec(n_scenes=48, seed=31, ell_hi=64, n_hi=30_000)
    scenes = [inputs.batch_scene(spec, s) for s in range(48)]
    if where == "host":
        args = [(s.pts, s.a, s.b) for s in scenes]
    elif where == "pinned":
        pin = lambda x: torch.from_numpy(x).pin_memory().numpy()
        args = [(pin(s.pts), pin(s.a), pin(s.b)) for s in scenes]
    else:
        args = [tuple(torch.from_numpy(x).to(dev) for x in (s.pts, s.a, s.b)) for s in scenes]
        torch.cuda.synchronize()
    with cellgraph.Server(0, hbm_budget_bytes=4 << 30, max_inflight=64) as srv:
        for _ in range(2):
            ts = [srv.submit(*a) for a in args]
            for i, (t, sc) in enumerate(zip(ts, scenes)):
                assert srv.wait(t, 120.0)
                _check(srv, t, sc, wanted(("g", i), sc))
                srv.release(t)
        st = srv.stats()
        assert st["failed"] == 0
        assert st["grouped"] >= 4 and st["groups"] >= 1, st
        assert st["bytes_in_use"] == 0


@pytest.mark.gpu
def test_requests_started_together_are_retried_one_by_one(dev, wanted, monkeypatch):
    """Requests started together whose first table guess (1,024 slots) is too
    small overflow inside the group; each is settled on its own, re-queued
    with a larger table, and still gives the oracle's output."""
    monkeypatch.setenv("CG_FIRST_TABLE_CAP", "1024")
    spec = inputs.scene_batch_spec(n_scenes=32, seed=33, ell_lo=24, ell_hi=64, n_lo=2e4, n_hi=6e4)
    scenes = [inputs.batch_scene(spec, s) for s in range(32)]
    with cellgraph.Server(0, hbm_budget_bytes=4 << 30, max_inflight=64) as srv:
        ts = [srv.submit(s.pts, s.a, s.b) for s in scenes]
        for i, (t, sc) in enumerate(zip(ts, scenes)):
            assert srv.wait(t, 120.0)
            _check(srv, t, sc, wanted(("gr", i), sc))
            srv.release(t)
        st = srv.stats()
        assert st["failed"] == 0
        assert st["grouped"] >= 4, st
        assert st["retried"] >= 1, st
        assert st["bytes_in_use"] == 0
