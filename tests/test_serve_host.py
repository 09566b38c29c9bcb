"""Host logic of the continuous-batching server, on CPU: requests are routed
to one pool per class, a pool is created only while free device memory
covers its buffers plus the reserve (otherwise the request waits and an
idle pool is released to make room), the number of pools is capped, and
every request's future completes with its own result.  The pools here are
stand-ins that finish a request as soon as it is queued (the real pools,
which run Alg. 1 on the GPU, are covered by tests/test_gpu_serve.py)."""
import time

import numpy as np
import pytest

import workloads as W
from paper_2411_06225_gb300 import serve


class FakeQueue:
    """A pool's request queue whose put() completes the request at once."""

    def __init__(self, pool):
        self.pool = pool

    def put(self, req):
        self.pool.served.append(req.id)
        self.pool.server._completed(req, dict(id=req.id, key=serve.class_key(req.cfg),
                                              U=None, K=1, converged=True, latency=0.0))

    def empty(self):
        return True


class FakePool:
    def __init__(self, cfg, slots, precision, weight_seed, server):
        self.cfg, self.server = cfg, server
        self.queue = FakeQueue(self)
        self.iterations = 0
        self.idle_since = time.perf_counter()
        self.served = []
        self.closed = False
        server.created.append(self)

    def busy(self):
        return False

    def close(self):
        self.closed = True


@pytest.fixture
def server(monkeypatch):
    """A server with stand-in pools and a device whose free memory the test
    sets: `srv.free_fn(srv)` returns the free bytes."""
    import torch
    monkeypatch.setattr(serve, "Pool", FakePool)
    srv = serve.Server(precision="mixed", slots=4, reserve_bytes=1 << 30)
    srv.created = []
    srv.free_fn = lambda s: 1 << 50
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda *a: (srv.free_fn(srv), 1 << 50))
    srv.start()
    yield srv
    srv.stop()


def requests(n):
    return [(r["cfg"], W.initial_condition(r["cfg"])[0]) for r in W.serving_stream(n, rate=1.0)]


def test_class_key_separates_what_a_context_fixes():
    cfg = W.config("swe2d", nx=32, ny=32, N=8)
    assert serve.class_key(cfg) == serve.class_key(dict(cfg))
    assert serve.class_key(cfg) != serve.class_key(dict(cfg, N=16))
    assert serve.class_key(cfg) != serve.class_key(dict(cfg, tol=1e-7))
    b = np.zeros(32 * 32)
    assert serve.class_key(dict(cfg, bathymetry=b)) != serve.class_key(cfg)
    assert serve.class_key(dict(cfg, bathymetry=b)) == serve.class_key(dict(cfg, bathymetry=b.copy()))


def test_one_pool_per_class_and_every_future_completes(server):
    reqs = requests(12)
    futs = [server.submit(cfg, u0) for cfg, u0 in reqs]
    res = [f.result(timeout=10) for f in futs]
    assert [r["id"] for r in res] == list(range(len(reqs)))
    keys = {serve.class_key(cfg) for cfg, _ in reqs}
    assert len(server.created) == len(keys)
    for r, (cfg, _) in zip(res, reqs):
        assert r["key"] == serve.class_key(cfg)
    assert server.completed == len(reqs)


def test_a_pool_waits_for_memory_and_an_idle_pool_makes_room(server):
    reqs = requests(12)
    cfg_a = reqs[0][0]
    other = [(c, u) for c, u in reqs if serve.class_key(c) != serve.class_key(cfg_a)]
    assert other
    cfg_b, u_b = other[0]
    need = max(serve.pool_bytes(c, server.slots, server.precision) for c in (cfg_a, cfg_b))
    # room for a pool only while no pool exists
    server.free_fn = lambda srv: srv.reserve + (2 * need if not srv.pools else need // 2)
    fa = server.submit(cfg_a, reqs[0][1])
    assert fa.result(timeout=10)["key"] == serve.class_key(cfg_a)
    fb = server.submit(cfg_b, u_b)
    # B waits until A's pool has been idle long enough to be released
    assert fb.result(timeout=10)["key"] == serve.class_key(cfg_b)
    assert len(server.created) == 2 and server.created[0].closed
    assert list(server.pools) == [serve.class_key(cfg_b)]


def test_the_number_of_pools_is_capped(server):
    server.max_pools = 1
    reqs = requests(12)
    keys = []
    for cfg, u0 in reqs:
        if serve.class_key(cfg) not in keys:
            keys.append(serve.class_key(cfg))
    futs = [server.submit(cfg, u0) for cfg, u0 in reqs]
    assert all(f.result(timeout=20)["converged"] for f in futs)
    # at most one pool at any time: every earlier pool was closed
    assert len(server.pools) == 1
    assert all(p.closed for p in server.created[:-1])
    assert len(server.created) >= len(keys)


def test_request_stream_is_seeded_poisson_over_the_stated_mix():
    """The C5 request stream: the same seed gives the same stream, arrivals
    increase with exponential gaps of mean 1 / rate, grid sides and slice
    counts come from the stated sets (each drawn), every request its own
    seeded bump of the shallow-water system."""
    a = W.serving_stream(2000, rate=4.0)
    b = W.serving_stream(2000, rate=4.0)
    assert [(r["arrival"], r["cfg"]["seed"]) for r in a] == [(r["arrival"], r["cfg"]["seed"]) for r in b]
    t = np.array([r["arrival"] for r in a])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    # mean of 2000 exponential gaps: 1/4 within 5 standard errors
    assert abs(gaps.mean() - 0.25) < 5 * 0.25 / np.sqrt(2000)
    # exponential: the coefficient of variation is 1
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1
    grids = {r["cfg"]["nx"] for r in a}
    slices = {r["cfg"]["N"] for r in a}
    assert grids == {64, 128, 256} and slices == {32, 64, 128}
    assert all(r["cfg"]["nx"] == r["cfg"]["ny"] and r["cfg"]["pde"] == "swe2d" for r in a)
    assert len({r["cfg"]["seed"] for r in a}) > 1990
    assert W.serving_stream(50, rate=4.0, seed=1)[0]["arrival"] != a[0]["arrival"]
