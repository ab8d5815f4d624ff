"""Oracle for the multi-spin Ising Metropolis chain: TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It wraps ``oracle.c`` (plain single-threaded C,
one int8 per spin, its own Philox4x32-10 and threshold table) through ctypes
and shares nothing with the CUDA library.

Every function cites the part of Hassani & Rafibakhsh (arXiv:1811.04384) it
follows: Eq. 1 (Hamiltonian), Sec. 2 (Metropolis rule), Eq. 3 and Table 1
(group value a and dE = 8 - 4a), Sec. 5.3 (energy as right + down bonds),
Eq. 2 (averages over iterations), Sec. 4-5 and Appendix A (the paper's own
chain of random memory-word updates in two column phases, rw_*).
"""
from __future__ import annotations

import ctypes
import multiprocessing as mp
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so with gcc (no -march flags,
    so the same source builds on x86_64 and aarch64)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i8p = ctypes.POINTER(ctypes.c_int8)
        sig = {
            "ora_philox4x32_10": (None, [u32p, u32p, u32p]),
            "ora_philox4x64_10": (None, [u64p, u64p, u64p]),
            "ora_philox4x32_r": (None, [u32p, u32p, ctypes.c_int, u32p]),
            "ora_set_sweep_rounds": (None, [ctypes.c_int]),
            "ora_half_sweep_rows": (None, [ctypes.c_int, i8p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                           u64p, ctypes.c_int, ctypes.c_int]),
            "ora_philox4x32_10_many": (None, [ctypes.c_int64, u32p, u32p, u32p]),
            "ora_site_draw_r": (ctypes.c_uint32, [ctypes.c_uint64, ctypes.c_uint64,
                                                  ctypes.c_int, ctypes.c_int, ctypes.c_int]),
            "ora_site_draw": (ctypes.c_uint32, [ctypes.c_uint64, ctypes.c_uint64,
                                                ctypes.c_int, ctypes.c_int]),
            "ora_thresholds": (None, [ctypes.c_double, u64p]),
            "ora_group_value": (ctypes.c_int, [ctypes.c_int, i8p, ctypes.c_int, ctypes.c_int]),
            "ora_delta_energy": (ctypes.c_int, [ctypes.c_int, i8p, ctypes.c_int, ctypes.c_int]),
            "ora_energy": (ctypes.c_int64, [ctypes.c_int, i8p]),
            "ora_magnetization": (ctypes.c_int64, [ctypes.c_int, i8p]),
            "ora_init_hot": (None, [ctypes.c_int, ctypes.c_uint64, i8p]),
            "ora_init_cold": (None, [ctypes.c_int, ctypes.c_int8, i8p]),
            "ora_half_sweep": (None, [ctypes.c_int, i8p, ctypes.c_uint64, ctypes.c_uint64,
                                      ctypes.c_int, u64p, i64p]),
            "ora_sweep": (None, [ctypes.c_int, i8p, ctypes.c_uint64, ctypes.c_uint64,
                                 ctypes.c_double, i64p]),
            "ora_run": (None, [ctypes.c_int, i8p, ctypes.c_uint64, ctypes.c_double,
                               ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, i64p, i64p]),
            "ora_rw_select": (None, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
            "ora_rw_step": (None, [ctypes.c_int, ctypes.c_int, i8p, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
                                   u64p, i64p]),
            "ora_rw_iteration": (None, [ctypes.c_int, ctypes.c_int, i8p, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.c_int, u64p, ctypes.c_int, i64p]),
            "ora_rw_run": (None, [ctypes.c_int, ctypes.c_int, i8p, ctypes.c_uint64, ctypes.c_double,
                                  ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, i64p, i64p,
                                  i64p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray, ctype):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctype))


# --- Philox (SC'11) -----------------------------------------------------------

def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().ora_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                              _ptr(out, ctypes.c_uint32))
    return out


def philox4x32_10_many(ctr, key) -> np.ndarray:
    """Philox4x32-10 blocks of n counters (n x 4 uint32)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros_like(c)
    _load().ora_philox4x32_10_many(c.shape[0], _ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                                   _ptr(out, ctypes.c_uint32))
    return out


def half_sweep_rows(s: np.ndarray, seed: int, t: int, c: int, beta: float, i0: int, i1: int) -> None:
    """Update colour c at sweep t in rows i0..i1-1 only (rows i0-1 and i1 are
    read as halos): one strip of a row-strip partition (Sec. 4)."""
    L = s.shape[0]
    _check(L, s)
    thr = np.array(thresholds(beta), dtype=np.uint64)
    _load().ora_half_sweep_rows(L, _ptr(s, ctypes.c_int8), seed, t, c, _ptr(thr, ctypes.c_uint64), i0, i1)


def philox4x32_r(ctr, key, rounds: int) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().ora_philox4x32_r(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), int(rounds),
                             _ptr(out, ctypes.c_uint32))
    return out


class sweep_rounds:
    """Context manager: the oracle's sweeps use `rounds` Philox rounds (10 is
    the default scheme, 7 the opt-in cheaper one); the hot start keeps 10."""

    def __init__(self, rounds: int):
        self.rounds = int(rounds)

    def __enter__(self):
        _load().ora_set_sweep_rounds(self.rounds)
        return self

    def __exit__(self, *exc):
        _load().ora_set_sweep_rounds(10)


def philox4x64_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    _load().ora_philox4x64_10(_ptr(c, ctypes.c_uint64), _ptr(k, ctypes.c_uint64),
                              _ptr(out, ctypes.c_uint64))
    return out


def site_draw(seed: int, t: int, i: int, j: int) -> int:
    """Philox draw of site (i, j) at sweep t (t = 0 is the hot start)."""
    return int(_load().ora_site_draw(seed, t, i, j))


# --- thresholds (Sec. 2 step 3, Table 1) -----------------------------------------

def thresholds(beta: float) -> tuple[int, int]:
    thr = np.zeros(2, dtype=np.uint64)
    _load().ora_thresholds(float(beta), _ptr(thr, ctypes.c_uint64))
    return int(thr[0]), int(thr[1])


# --- lattice -------------------------------------------------------------------

def _check(L: int, s: np.ndarray):
    assert s.dtype == np.int8 and s.shape == (L, L) and s.flags["C_CONTIGUOUS"]


def init_hot(L: int, seed: int) -> np.ndarray:
    s = np.zeros((L, L), dtype=np.int8)
    _load().ora_init_hot(L, seed, _ptr(s, ctypes.c_int8))
    return s


def init_cold(L: int, spin: int = 1) -> np.ndarray:
    s = np.zeros((L, L), dtype=np.int8)
    _load().ora_init_cold(L, spin, _ptr(s, ctypes.c_int8))
    return s


def group_value(s: np.ndarray, i: int, j: int) -> int:
    L = s.shape[0]
    _check(L, s)
    return int(_load().ora_group_value(L, _ptr(s, ctypes.c_int8), i, j))


def delta_energy(s: np.ndarray, i: int, j: int) -> int:
    L = s.shape[0]
    _check(L, s)
    return int(_load().ora_delta_energy(L, _ptr(s, ctypes.c_int8), i, j))


def energy(s: np.ndarray) -> int:
    L = s.shape[0]
    _check(L, s)
    return int(_load().ora_energy(L, _ptr(s, ctypes.c_int8)))


def magnetization(s: np.ndarray) -> int:
    L = s.shape[0]
    _check(L, s)
    return int(_load().ora_magnetization(L, _ptr(s, ctypes.c_int8)))


def half_sweep(s: np.ndarray, seed: int, t: int, c: int, beta: float,
               stats: np.ndarray | None = None) -> None:
    """In-place Metropolis update of colour c at sweep t.  stats, if given, is an
    int64[10]: [0..4] proposals by group value a, [5..9] accepted flips."""
    L = s.shape[0]
    _check(L, s)
    thr = np.array(thresholds(beta), dtype=np.uint64)
    sp = None
    if stats is not None:
        assert stats.dtype == np.int64 and stats.shape == (10,)
        sp = _ptr(stats, ctypes.c_int64)
    _load().ora_half_sweep(L, _ptr(s, ctypes.c_int8), seed, t, c,
                           _ptr(thr, ctypes.c_uint64), sp)


def half_sweep_thr(s: np.ndarray, seed: int, t: int, c: int, thr0: int, thr1: int) -> None:
    """half_sweep with the two integer thresholds given directly."""
    L = s.shape[0]
    _check(L, s)
    thr = np.array([thr0, thr1], dtype=np.uint64)
    _load().ora_half_sweep(L, _ptr(s, ctypes.c_int8), seed, t, c,
                           _ptr(thr, ctypes.c_uint64), None)


def sweep(s: np.ndarray, seed: int, t: int, beta: float,
          stats: np.ndarray | None = None) -> None:
    L = s.shape[0]
    _check(L, s)
    sp = None
    if stats is not None:
        assert stats.dtype == np.int64 and stats.shape == (10,)
        sp = _ptr(stats, ctypes.c_int64)
    _load().ora_sweep(L, _ptr(s, ctypes.c_int8), seed, t, float(beta), sp)


def run(s: np.ndarray, seed: int, beta: float, t0: int, n: int, every: int = 1):
    """Sweeps t0+1..t0+n in place; returns the int64 (E, M) series recorded after
    sweeps t0+every, t0+2*every, ... (n // every entries)."""
    L = s.shape[0]
    _check(L, s)
    k = n // every if every > 0 else 0
    E = np.zeros(max(k, 1), dtype=np.int64)
    M = np.zeros(max(k, 1), dtype=np.int64)
    _load().ora_run(L, _ptr(s, ctypes.c_int8), seed, float(beta), t0, n, every,
                    _ptr(E, ctypes.c_int64), _ptr(M, ctypes.c_int64))
    return E[:k], M[:k]


# --- the paper's own chain: random memory words (Sec. 4-5, Appendix A) ----------

def rw_check(L: int, F: int, nstrips: int):
    assert 1 <= F <= 22 and L % F == 0 and L // F >= (2 if F > 1 else 1), (L, F)
    assert nstrips >= 1 and L % nstrips == 0 and L // nstrips >= 2, (L, nstrips)


def rw_select(seed: int, t: int, phase: int, strip: int, step: int, N: int, col0: int, h: int):
    """(row, column) of the word that update `step` of strip `strip` in phase
    `phase` of iteration t picks from the half strip [col0, col0 + h)."""
    I, J = ctypes.c_int(), ctypes.c_int()
    _load().ora_rw_select(seed, t, phase, strip, step, N, col0, h, ctypes.byref(I), ctypes.byref(J))
    return I.value, J.value


def rw_step(s: np.ndarray, seed: int, t: int, phase: int, strip: int, step: int, col0: int, h: int,
            thr0: int, thr1: int, F: int = 21) -> None:
    """One word update of the random-word chain in place: update `step` of
    strip `strip` in phase `phase` of iteration t, on the half strip
    [col0, col0 + h), with the integer thresholds given directly."""
    L = s.shape[0]
    _check(L, s)
    thr = np.array([thr0, thr1], dtype=np.uint64)
    _load().ora_rw_step(L, F, _ptr(s, ctypes.c_int8), seed, t, phase, strip, step, col0, h,
                        _ptr(thr, ctypes.c_uint64), None)


def rw_iteration(s: np.ndarray, seed: int, t: int, beta: float, nstrips: int, F: int = 21,
                 reverse: bool = False, stats: np.ndarray | None = None) -> None:
    """One iteration t of the random-word chain in place (both phases, every
    strip); reverse runs the strips of each phase in the opposite order."""
    L = s.shape[0]
    _check(L, s)
    rw_check(L, F, nstrips)
    thr = np.array(thresholds(beta), dtype=np.uint64)
    sp = None
    if stats is not None:
        assert stats.dtype == np.int64 and stats.shape == (10,)
        sp = _ptr(stats, ctypes.c_int64)
    _load().ora_rw_iteration(L, F, _ptr(s, ctypes.c_int8), seed, t, nstrips, _ptr(thr, ctypes.c_uint64),
                             1 if reverse else 0, sp)


def rw_run(s: np.ndarray, seed: int, beta: float, t0: int, n: int, nstrips: int, every: int = 1, F: int = 21,
           stats: np.ndarray | None = None):
    """Iterations t0+1 .. t0+n of the random-word chain in place; returns the
    int64 (E, M) series recorded after iterations t0+every, t0+2*every, ..."""
    L = s.shape[0]
    _check(L, s)
    rw_check(L, F, nstrips)
    k = n // every if every > 0 else 0
    E = np.zeros(max(k, 1), dtype=np.int64)
    M = np.zeros(max(k, 1), dtype=np.int64)
    sp = None
    if stats is not None:
        assert stats.dtype == np.int64 and stats.shape == (10,)
        sp = _ptr(stats, ctypes.c_int64)
    _load().ora_rw_run(L, F, _ptr(s, ctypes.c_int8), seed, float(beta), t0, n, every, nstrips,
                       _ptr(E, ctypes.c_int64), _ptr(M, ctypes.c_int64), sp)
    return E[:k], M[:k]


def means(E: np.ndarray, M: np.ndarray, L: int) -> tuple[float, float]:
    """Eq. 2: per-spin averages over the recorded sweeps, from int64 sums and one
    FP64 division each (<E>/N_s, <|M|>/N_s)."""
    n = len(E)
    sE = int(np.sum(E.astype(object)))
    sM = int(np.sum(np.abs(M).astype(object)))
    return sE / (n * L * L), sM / (n * L * L)


# --- independent jobs on several host cores ---------------------------------------

def run_job(job):
    """One independent oracle run: job = (L, seed, beta, hot, sweeps, every).
    Hot start from `seed` (else all +1), sweeps 1..sweeps; returns the
    (E, M) series recorded every `every` sweeps and the final spins."""
    L, seed, beta, hot, sweeps, every = job
    s = init_hot(L, seed) if hot else init_cold(L, 1)
    E, M = run(s, seed, beta, 0, sweeps, every)
    return E, M, s


def run_jobs(jobs, processes: int | None = None):
    """run_job over a list of jobs, in a spawn-context process pool (a
    spawned worker inherits no CUDA state of the caller, so this may be
    called after GPU work).  Results come back in the order of `jobs`."""
    jobs = list(jobs)
    if not jobs:
        return []
    build()
    n = max(1, min(len(jobs), processes or os.cpu_count() or 1))
    if n == 1:
        return [run_job(j) for j in jobs]
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.map(run_job, jobs, chunksize=1)
