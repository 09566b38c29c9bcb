"""Continuous-batching RandNet-Parareal server.

Requests (an IVP of Eq. 1: a workload dict plus an initial state) arrive at
any time.  Requests of one *class* (same PDE, grid, slice count and solver
settings) share a pooled context whose B member slots they occupy; every
turn of the serving loop

  1. admits waiting requests into free slots (creating a pool for a new class
     only while free HBM covers its buffers plus a reserve): the request's
     k = 0 coarse sweep runs and its states and dataset stay on the device;
  2. advances every pool with active members by one iteration of Alg. 1
     (``rnp_iterate``): the fine steps of all its members share one launch,
     and pools run in their own threads and CUDA streams so that different
     classes overlap on the GPU;
  3. completes finished members (result copied to the host, slot freed).

A request that arrives while others are iterating joins its pool at the next
turn, without waiting for the others to finish.
"""
from __future__ import annotations

import ctypes as C
import queue
import threading
import time
from concurrent.futures import Future

import numpy as np

from . import (RNP_MEMBER_ACTIVE, RNP_MEMBER_CONVERGED, RNP_MEMBER_FREE, RNP_OK,
               RnpError, Solver, dim, lib, problem)

CLASS_KEYS = ("pde", "nx", "ny", "nz", "lx", "ly", "lz", "t0", "tN", "N", "nF", "nG",
              "M", "m", "lam", "tol", "max_iters", "corr", "gscheme", "fscheme", "bc")


def class_key(cfg: dict) -> tuple:
    """Requests with equal keys share a pooled context (a bottom profile is
    part of the class: it is fixed per context)."""
    b = cfg.get("bathymetry")
    bkey = None if b is None else np.ascontiguousarray(b, np.float64).tobytes()
    return tuple(cfg.get(k) for k in CLASS_KEYS) + (tuple(cfg["param"]), bkey)


def pool_bytes(cfg: dict, slots: int, precision: str) -> int:
    """Device bytes of a pooled context (the allocations of rnp_create)."""
    d = dim(problem(cfg))
    N, M = cfg["N"], cfg["M"]
    kmax = min(cfg.get("max_iters", N), N)
    cap = sum(N - k + 1 for k in range(1, kmax + 1))
    per = 8 * d * ((N + 1) + 3 * N + 2) + 8 * M * (N + 1)
    per += cap * d * (8 + (4 if precision == "mixed" else 8)) + cap * (8 * M + 8 + 8 * 32)
    shared = 8 * M * d + (4 * M * d if precision == "mixed" else 0)
    return slots * per + shared + (64 << 20)


class Request:
    def __init__(self, rid, cfg, u0, arrival):
        self.id, self.cfg, self.u0, self.arrival = rid, cfg, u0, arrival
        self.future: Future = Future()
        self.t_admit = self.t_done = None


class Pool:
    """One class of requests: a context with `slots` members, its stream and
    its own serving thread (admit -> iterate -> complete), so that pools of
    different classes advance independently and overlap on the GPU."""

    def __init__(self, cfg, slots, precision, weight_seed, server):
        import torch
        self.cfg = dict(cfg, batch=slots, seed=weight_seed)
        self.stream = torch.cuda.Stream()
        self.solver = Solver(problem(self.cfg, precision=precision, autotune=0),
                             stream=self.stream)
        self.slots = slots
        self.members = [None] * slots
        self.d = self.solver.d
        self.N = self.cfg["N"]
        self.queue: "queue.Queue[Request]" = queue.Queue()
        self.server = server
        self.iterations = 0
        self.idle_since = time.perf_counter()
        self._stop = threading.Event()
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    def free_slot(self):
        for i, r in enumerate(self.members):
            if r is None:
                return i
        return None

    def busy(self):
        return any(r is not None for r in self.members) or not self.queue.empty()

    def _start(self, slot, req):
        import torch
        with torch.cuda.stream(self.stream):
            u0 = torch.as_tensor(np.ascontiguousarray(req.u0, np.float64), device="cuda")
            st = lib().rnp_member_start(self.solver._ctx, slot, C.c_void_p(u0.data_ptr()))
        if st != RNP_OK:
            raise RnpError(st, lib().rnp_last_error(self.solver._ctx).decode())
        self.members[slot] = req
        req.t_admit = time.perf_counter()

    def _iterate(self):
        n = C.c_int(0)
        st = lib().rnp_iterate(self.solver._ctx, C.byref(n))
        if st != RNP_OK:
            raise RnpError(st, lib().rnp_last_error(self.solver._ctx).decode())
        self.iterations += 1
        return n.value

    def _collect(self):
        import torch
        for slot, req in enumerate(self.members):
            if req is None:
                continue
            state, K, L = C.c_int(), C.c_int(), C.c_int()
            lib().rnp_member_status(self.solver._ctx, slot, C.byref(state), C.byref(K),
                                    C.byref(L))
            if state.value in (RNP_MEMBER_ACTIVE, RNP_MEMBER_FREE):
                continue
            with torch.cuda.stream(self.stream):
                U = torch.empty((self.N + 1, self.d), dtype=torch.float64, device="cuda")
                lib().rnp_member_result(self.solver._ctx, slot, C.c_void_p(U.data_ptr()))
                Uh = U.cpu()
            self.members[slot] = None
            req.t_done = time.perf_counter()
            self.server._completed(req, dict(id=req.id, U=Uh.numpy(), K=K.value,
                                             converged=state.value == RNP_MEMBER_CONVERGED,
                                             latency=req.t_done - req.arrival))

    def _loop(self):
        try:
            while not self._stop.is_set():
                # admit queued requests into free slots (they join mid-flight)
                while True:
                    slot = self.free_slot()
                    if slot is None:
                        break
                    try:
                        req = self.queue.get_nowait()
                    except queue.Empty:
                        break
                    self._start(slot, req)
                if any(r is not None for r in self.members):
                    self._iterate()
                    self._collect()
                    self.idle_since = time.perf_counter()
                else:
                    try:
                        req = self.queue.get(timeout=0.002)
                        self.queue.put(req)
                    except queue.Empty:
                        pass
        except Exception as e:  # fail this pool's requests; the server goes on
            for r in self.members:
                if r is not None and not r.future.done():
                    r.future.set_exception(e)
            while not self.queue.empty():
                r = self.queue.get_nowait()
                if not r.future.done():
                    r.future.set_exception(e)

    def close(self):
        self._stop.set()
        self.thread.join()
        self.solver.close()


class Server:
    """Continuous-batching server; see the module docstring.  A dispatcher
    thread routes arrivals to their class's pool, creating a pool while free
    HBM covers it plus a reserve (otherwise the request waits, and idle pools
    are released to make room)."""

    def __init__(self, precision: str = "mixed", slots: int = 4,
                 reserve_bytes: int = 8 << 30, weight_seed: int = 2415, max_pools: int = 16):
        self.precision = precision
        self.slots = slots
        self.reserve = reserve_bytes
        self.weight_seed = weight_seed
        self.max_pools = max_pools
        self.pools: dict = {}
        self.waiting: list = []
        self.inbox: "queue.Queue[Request]" = queue.Queue()
        self._stop = threading.Event()
        self._thread = None
        self._lock = threading.Lock()
        self.completed = 0
        self.next_id = 0

    @property
    def turns(self):
        return sum(p.iterations for p in self.pools.values())

    def submit(self, cfg: dict, u0: np.ndarray, arrival: float | None = None) -> Future:
        with self._lock:
            rid = self.next_id
            self.next_id += 1
        req = Request(rid, cfg, u0, time.perf_counter() if arrival is None else arrival)
        self.inbox.put(req)
        return req.future

    def _completed(self, req, result):
        with self._lock:
            self.completed += 1
        req.future.set_result(result)

    def start(self):
        self._thread = threading.Thread(target=self._dispatch, daemon=True)
        self._thread.start()

    def stop(self):
        self._stop.set()
        if self._thread:
            self._thread.join()
        for p in self.pools.values():
            p.close()

    def _route(self):
        import torch
        still = []
        for req in self.waiting:
            key = class_key(req.cfg)
            pool = self.pools.get(key)
            if pool is None:
                need = pool_bytes(req.cfg, self.slots, self.precision)
                free, _ = torch.cuda.mem_get_info()
                if len(self.pools) >= self.max_pools or free - need < self.reserve:
                    idle = [k for k, p in self.pools.items()
                            if not p.busy() and time.perf_counter() - p.idle_since > 0.05]
                    if idle:
                        self.pools.pop(idle[0]).close()
                    still.append(req)
                    continue
                try:
                    pool = self.pools[key] = Pool(req.cfg, self.slots, self.precision,
                                                  self.weight_seed, self)
                except RnpError as e:
                    req.future.set_exception(e)
                    continue
            pool.queue.put(req)
        self.waiting = still

    def _dispatch(self):
        while not self._stop.is_set():
            try:
                self.waiting.append(self.inbox.get(timeout=0.002))
                while True:
                    self.waiting.append(self.inbox.get_nowait())
            except queue.Empty:
                pass
            if self.waiting:
                self._route()


def run_stream(reqs: list[dict], precision: str = "mixed", slots: int = 4,
               time_scale: float = 1.0) -> dict:
    """Replay a request stream (workloads.serving_stream) against a server:
    request r is submitted at its arrival time; returns latency percentiles
    and throughput."""
    import workloads as W
    srv = Server(precision=precision, slots=slots)
    srv.start()
    t0 = time.perf_counter()
    futs = []
    for r in reqs:
        target = t0 + r["arrival"] * time_scale
        while time.perf_counter() < target:
            time.sleep(min(0.001, max(0.0, target - time.perf_counter())))
        u0 = W.initial_condition(r["cfg"])[0]
        futs.append(srv.submit(r["cfg"], u0, arrival=target))
    res = [f.result() for f in futs]
    t_end = time.perf_counter()
    srv.stop()
    lat = np.array([x["latency"] for x in res]) * 1e3
    return dict(n=len(res), p50_ms=float(np.percentile(lat, 50)),
                p99_ms=float(np.percentile(lat, 99)), mean_ms=float(lat.mean()),
                solves_per_s=len(res) / (t_end - t0), converged=sum(x["converged"] for x in res),
                K_mean=float(np.mean([x["K"] for x in res])), wall_s=t_end - t0,
                pools=len(srv.pools), iterations=srv.turns)


def main():
    import argparse
    import json

    import workloads as W
    ap = argparse.ArgumentParser(description="serve a Poisson stream of shallow-water solves")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--rate", type=float, default=0.0,
                    help="arrivals per second (0: 0.7 x measured closed-loop throughput)")
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--precision", default="mixed")
    ap.add_argument("--max-iters", type=int, default=12)
    args = ap.parse_args()
    base = W.serving_stream(args.requests, rate=1.0)
    for r in base:
        r["cfg"]["max_iters"] = min(args.max_iters, r["cfg"]["N"])
    rate = args.rate
    if rate <= 0:
        closed = run_stream([dict(r, arrival=0.0) for r in base[: max(8, args.requests // 4)]],
                            args.precision, args.slots)
        rate = 0.7 * closed["solves_per_s"]
    out = {}
    for frac in (0.3, 0.7, 0.9):
        reqs = W.serving_stream(args.requests, rate=rate * frac / 0.7)
        for r in reqs:
            r["cfg"]["max_iters"] = min(args.max_iters, r["cfg"]["N"])
        out[f"{frac:.1f}x"] = run_stream(reqs, args.precision, args.slots)
    print(json.dumps(dict(metric="serving latency", closed_loop_rate=rate / 0.7, **out)))


if __name__ == "__main__":
    main()
