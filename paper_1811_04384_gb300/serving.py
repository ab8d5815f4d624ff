"""Serving: continuous batching of Ising simulation jobs (include/ising.h,
ising_server_*), plus the Poisson request stream of the serving
configuration.  Argument marshalling only: admission, batching and the sweeps
run in the library's worker thread and kernels."""
from __future__ import annotations

import ctypes
import math
import threading
import time

import numpy as np

from . import ISING_EBUSY, ISING_OK, ISING_ETIMEOUT, IsingError, load, _check
from ._abi import IsingJob, IsingResult

STATES = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "cancelled"}


class Request:
    """One job and its caller-owned result arrays (kept alive until done)."""

    def __init__(self, L, beta, seed, sweeps, every=1, hot=True, want_spins=False, rng=0):
        self.L, self.beta, self.seed = int(L), float(beta), int(seed)
        self.rng = int(rng)
        self.sweeps, self.every, self.hot = int(sweeps), int(every), bool(hot)
        self.E = np.zeros(self.sweeps // self.every, dtype=np.int64)
        self.M = np.zeros(self.sweeps // self.every, dtype=np.int64)
        self.spins = np.empty((self.L, self.L), dtype=np.int8) if want_spins else None
        self.id = None
        self.result = None

    def job(self) -> IsingJob:
        return IsingJob(self.L, self.beta, self.seed, 1 if self.hot else 0, self.sweeps, self.every,
                        self.E.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                        self.M.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                        self.spins.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)) if self.spins is not None else None,
                        self.rng)


class Server:
    def __init__(self, hbm_budget_bytes: int, max_jobs: int | None = None, epoch_sweeps: int | None = None):
        """A server with an arena of hbm_budget_bytes.  With neither limit given
        this is ising_server_create (256 running jobs, 50-sweep epochs);
        otherwise ising_server_create_ex with the missing limit at its default."""
        lib = load()
        h = ctypes.c_void_p()
        if max_jobs is None and epoch_sweeps is None:
            _check(lib.ising_server_create(int(hbm_budget_bytes), ctypes.byref(h)), "ising_server_create")
        else:
            _check(lib.ising_server_create_ex(int(hbm_budget_bytes), int(max_jobs or 256), int(epoch_sweeps or 50),
                                              ctypes.byref(h)), "ising_server_create_ex")
        self._h = h
        self._live = {}

    def submit(self, req: Request) -> int:
        jid = ctypes.c_uint64()
        job = req.job()
        _check(load().ising_server_submit(self._h, ctypes.byref(job), ctypes.byref(jid)), "ising_server_submit")
        req.id = int(jid.value)
        self._live[req.id] = req
        return req.id

    def poll(self, jid: int) -> IsingResult:
        r = IsingResult()
        _check(load().ising_server_poll(self._h, int(jid), ctypes.byref(r)), "ising_server_poll")
        return r

    def wait(self, jid: int, timeout_ms: int = -1) -> IsingResult:
        r = IsingResult()
        rc = load().ising_server_wait(self._h, int(jid), int(timeout_ms), ctypes.byref(r))
        if rc not in (ISING_OK, ISING_ETIMEOUT):
            raise IsingError(rc, "ising_server_wait")
        return r

    def cancel(self, jid: int):
        _check(load().ising_server_cancel(self._h, int(jid)), "ising_server_cancel")

    def release(self, jid: int):
        _check(load().ising_server_release(self._h, int(jid)), "ising_server_release")
        self._live.pop(int(jid), None)

    def inject_fault(self, epochs: int = 0):
        """Test hook (ising_server_inject_fault): a host exception in the worker
        at the start of the epoch `epochs` epochs from now; -1 disarms it."""
        _check(load().ising_server_inject_fault(self._h, int(epochs)), "ising_server_inject_fault")

    def stats(self):
        jobs, eps = ctypes.c_int64(), ctypes.c_int64()
        upd, busy = ctypes.c_double(), ctypes.c_double()
        _check(load().ising_server_stats(self._h, ctypes.byref(jobs), ctypes.byref(upd), ctypes.byref(eps),
                                         ctypes.byref(busy)), "ising_server_stats")
        return {"jobs_done": jobs.value, "spin_updates": upd.value, "epochs": eps.value, "busy_s": busy.value}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value is not None:
            load().ising_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def poisson_stream(n: int, rate: float = 200.0, seed: int = 13):
    """The serving configuration's request stream: exponential inter-arrival
    times (mean 1/rate s), L uniform on {64..4096} (powers of two), T uniform
    on [1.5, 3.5], sweeps log-uniform on [100, 10000], hot starts with
    per-request seeds; all from numpy default_rng(seed)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    Ls = rng.choice([64, 128, 256, 512, 1024, 2048, 4096], size=n)
    Ts = rng.uniform(1.5, 3.5, size=n)
    sweeps = np.exp(rng.uniform(math.log(100), math.log(10000), size=n)).astype(np.int64)
    seeds = rng.integers(1, 2**63, size=n, dtype=np.uint64)
    return [(float(t[k]), int(Ls[k]), 1.0 / float(Ts[k]), int(seeds[k]), int(sweeps[k])) for k in range(n)]


def serve_stream(stream, hbm_budget_bytes: int, max_jobs: int = 256, epoch_sweeps: int = 50, every: int = 1):
    """Submit each request at its arrival time, wait for all, and return the
    requests (with their results) and the server's totals."""
    reqs = []
    with Server(hbm_budget_bytes, max_jobs, epoch_sweeps) as srv:
        t0 = time.perf_counter()
        for (ta, L, beta, seed, sweeps) in stream:
            delay = ta - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            r = Request(L, beta, seed, sweeps, every)
            srv.submit(r)
            reqs.append(r)
        for r in reqs:
            r.result = srv.wait(r.id)
        wall = time.perf_counter() - t0
        stats = srv.stats()
    stats["wall_s"] = wall
    return reqs, stats
