"""GB300-native multi-spin Ising Metropolis (Hassani & Rafibakhsh,
arXiv:1811.04384): a thin Python binding of the C ABI in include/ising.h.

Every step of the simulation runs in the CUDA kernels of libising.so; this
module only marshals arguments.  There is no CPU fallback: if the library has
not been built (``paper_1811_04384_gb300.build.build()``) or cannot be loaded,
``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._abi import declare, SYMBOLS  # noqa: F401

_PKG = os.path.dirname(os.path.abspath(__file__))
# ISING_LIBRARY selects another build of the library (the checked one,
# _build/libising_checked.so); the default is the normal build
LIB_PATH = os.environ.get("ISING_LIBRARY") or os.path.join(_PKG, "_build", "libising.so")

ISING_OK = 0
ISING_EINVAL = -1
ISING_ENOMEM = -2
ISING_ECUDA = -3
ISING_ETIMEOUT = -4
ISING_EBUSY = -5
ISING_ENOTFOUND = -6
ISING_EINTERNAL = -7
ISING_LAYOUT_ROW_PACKED = 0
ISING_LAYOUT_COLUMN_INTERLEAVED = 1
ISING_RNG_PHILOX4X32_10 = 0
ISING_RNG_PHILOX4X32_7 = 1
ISING_CHAIN_CHECKERBOARD = 0
ISING_CHAIN_RANDOM_WORDS = 1
ISING_PATH_AUTO = 0
ISING_PATH_LAUNCHES = 1
ISING_PATH_RESIDENT = 2
ISING_PATH_CLUSTER = 3
ISING_NOALLOC_MAX_RECORDS = 1024   # records one ising_sweep_record_noalloc call can hold

_lib = None


class IsingError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        detail = ""
        if _lib is not None and code == ISING_ECUDA:
            detail = " (" + _lib.ising_last_cuda_error().decode() + ")"
        msg = _lib.ising_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg}{detail}")


def load() -> ctypes.CDLL:
    """Load libising.so (built in-tree).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1811_04384_gb300.build.build() "
                          "(the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    declare(lib)
    _lib = lib
    return lib


def _check(rc: int, where: str):
    if rc != ISING_OK:
        raise IsingError(rc, where)


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        return ctypes.c_void_p(None)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)   # torch.cuda.Stream


def bytes_required(L: int) -> int:
    """Device bytes a lattice of side L needs (ising_bytes_required), for caller-owned buffers."""
    return int(load().ising_bytes_required(L))


class Lattice:
    """One L x L lattice resident in device memory (see include/ising.h)."""

    def __init__(self, L: int, seed: int, *, buffer=None, stream=None, layout: int = 0):
        lib = load()
        self.L = int(L)
        self.seed = int(seed)
        self._buffer = buffer      # keeps a caller-owned (torch) buffer alive
        h = ctypes.c_void_p()
        if layout != ISING_LAYOUT_ROW_PACKED:
            _check(lib.ising_create_layout(self.L, self.seed, int(layout), ctypes.byref(h)), "ising_create_layout")
            if stream is not None:
                _check(lib.ising_set_stream(h, _stream_ptr(stream)), "ising_set_stream")
        elif buffer is None:
            _check(lib.ising_create(self.L, self.seed, ctypes.byref(h)), "ising_create")
            if stream is not None:
                _check(lib.ising_set_stream(h, _stream_ptr(stream)), "ising_set_stream")
        else:
            ptr = buffer.data_ptr() if hasattr(buffer, "data_ptr") else int(buffer)
            nbytes = buffer.numel() * buffer.element_size() if hasattr(buffer, "numel") else bytes_required(L)
            _check(lib.ising_create_on(self.L, self.seed, ctypes.c_void_p(ptr), nbytes, _stream_ptr(stream),
                                       ctypes.byref(h)), "ising_create_on")
        self._h = h

    # -- lifetime ---------------------------------------------------------------
    def close(self):
        """Release the lattice (ising_destroy); also done by the context manager."""
        if getattr(self, "_h", None) is not None and self._h.value is not None:
            load().ising_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- state ------------------------------------------------------------------
    def init_hot(self):
        """Hot start (ising_init_hot): each spin from the site's Philox draw at t = 0; t = 0."""
        _check(load().ising_init_hot(self._h), "ising_init_hot")

    def init_cold(self, spin: int = 1):
        """Cold start (ising_init_cold): every spin = spin (+1 or -1); t = 0."""
        _check(load().ising_init_cold(self._h, int(spin)), "ising_init_cold")

    def set_beta(self, beta: float):
        """Inverse temperature (ising_set_beta); builds the integer thresholds."""
        _check(load().ising_set_beta(self._h, float(beta)), "ising_set_beta")

    def thresholds(self) -> tuple[int, int]:
        """The two integer thresholds in use (ising_get_thresholds): (thr[a=0], thr[a=1])."""
        thr = (ctypes.c_uint64 * 2)()
        _check(load().ising_get_thresholds(self._h, thr), "ising_get_thresholds")
        return int(thr[0]), int(thr[1])

    @property
    def t(self) -> int:
        """Sweep counter (ising_get_sweep / ising_set_sweep)."""
        v = ctypes.c_uint64()
        _check(load().ising_get_sweep(self._h, ctypes.byref(v)), "ising_get_sweep")
        return int(v.value)

    @t.setter
    def t(self, value: int):
        _check(load().ising_set_sweep(self._h, int(value)), "ising_set_sweep")

    def set_stream(self, stream):
        """CUDA stream for all further work (ising_set_stream): a torch.cuda.Stream, a handle or None."""
        _check(load().ising_set_stream(self._h, _stream_ptr(stream)), "ising_set_stream")

    def set_tiling(self, rows: int = 4, block_words: int = 0, block_groups: int = 128):
        """Launch shape of the half-sweep kernels (ising_set_tiling); results do not depend on it."""
        _check(load().ising_set_tiling(self._h, rows, block_words, block_groups), "ising_set_tiling")

    def run_states(self, states, sweeps: int, every: int = 1):
        """ising_run_states: for each int8 L x L array in `states` (pinned host
        memory overlaps its copy with the previous state's sweeps), set the
        spins and run `sweeps` sweeps with a record every `every`; returns int64
        E and M of shape (len(states), sweeps // every)."""
        arrs = [np.ascontiguousarray(a, dtype=np.int8) for a in states]
        for a in arrs:
            assert a.size == self.L * self.L
        n = len(arrs)
        R = max(int(sweeps), 0) // max(int(every), 1)
        E = np.zeros((n, R), dtype=np.int64)
        M = np.zeros((n, R), dtype=np.int64)
        ptrs = (ctypes.c_void_p * max(n, 1))(*[a.ctypes.data_as(ctypes.c_void_p).value for a in arrs])
        _check(load().ising_run_states(self._h, ptrs, n, int(sweeps), int(every),
                                       E.ctypes.data_as(ctypes.c_void_p), M.ctypes.data_as(ctypes.c_void_p)),
               "ising_run_states")
        return E, M

    def set_item_lanes(self, lanes: int = 0):
        """Lanes per thread item on the launch path: 1, 2, 4, 8 or 0 (auto)."""
        _check(load().ising_set_item_lanes(self._h, int(lanes)), "ising_set_item_lanes")

    def set_rng(self, scheme: int):
        """ISING_RNG_PHILOX4X32_10 (default) or the opt-in ISING_RNG_PHILOX4X32_7."""
        _check(load().ising_set_rng(self._h, int(scheme)), "ising_set_rng")

    def set_chain(self, chain: int, nstrips: int = 1):
        """ISING_CHAIN_CHECKERBOARD (default) or the paper's ISING_CHAIN_RANDOM_WORDS
        with `nstrips` column strips (column-interleaved lattices only)."""
        _check(load().ising_set_chain(self._h, int(chain), int(nstrips)), "ising_set_chain")

    def set_path(self, path: int):
        """ISING_PATH_AUTO, ISING_PATH_LAUNCHES, ISING_PATH_RESIDENT or ISING_PATH_CLUSTER."""
        _check(load().ising_set_path(self._h, int(path)), "ising_set_path")

    def set_clusters(self, clusters: int = 0):
        """Clusters of one cluster-path launch (ising_set_clusters): 0 = automatic."""
        _check(load().ising_set_clusters(self._h, int(clusters)), "ising_set_clusters")

    def inject_stall(self, launches: int = 1):
        """Test hook (ising_cluster_inject_stall): the next launches' waits between clusters give up."""
        _check(load().ising_cluster_inject_stall(self._h, int(launches)), "ising_cluster_inject_stall")

    def inject_absent(self, after: int = 0):
        """Test hook (ising_cluster_inject_absent): the launch with several
        clusters after `after` more of them counts on one block more than it
        has, so it writes nothing and the call finishes on the launch path; -1 clears."""
        _check(load().ising_cluster_inject_absent(self._h, int(after)), "ising_cluster_inject_absent")

    def get_path(self) -> int:
        """The path the next sweeps take (ising_get_path): ISING_PATH_RESIDENT,
        ISING_PATH_CLUSTER or ISING_PATH_LAUNCHES."""
        p = ctypes.c_int32(0)
        _check(load().ising_get_path(self._h, ctypes.byref(p)), "ising_get_path")
        return p.value

    def layout(self) -> tuple[int, int, int]:
        """(W, pitch, live fields of the last word) of the row-packed layout (ising_layout)."""
        W, P, r = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(load().ising_layout(self._h, ctypes.byref(W), ctypes.byref(P), ctypes.byref(r)), "ising_layout")
        return W.value, P.value, r.value

    # -- dynamics ---------------------------------------------------------------
    def sweep(self, n: int = 1):
        """Run n sweeps (ising_sweep); asynchronous on the lattice's stream."""
        _check(load().ising_sweep(self._h, int(n)), "ising_sweep")

    def sweep_record(self, n: int, every: int = 1):
        """Run n sweeps; returns int64 arrays E, M recorded every `every` sweeps (ising_sweep_record)."""
        k = n // every
        E = np.zeros(max(k, 1), dtype=np.int64)
        M = np.zeros(max(k, 1), dtype=np.int64)
        _check(load().ising_sweep_record(self._h, int(n), int(every), E.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                         M.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))), "ising_sweep_record")
        return E[:k], M[:k]

    def energy(self) -> int:
        """Current energy, exact int64 (ising_energy)."""
        v = ctypes.c_int64()
        _check(load().ising_energy(self._h, ctypes.byref(v)), "ising_energy")
        return int(v.value)

    def magnetization(self) -> int:
        """Current magnetisation, exact int64 (ising_magnetization)."""
        v = ctypes.c_int64()
        _check(load().ising_magnetization(self._h, ctypes.byref(v)), "ising_magnetization")
        return int(v.value)

    # -- spin I/O ---------------------------------------------------------------
    def get_spins(self, out: np.ndarray | None = None) -> np.ndarray:
        """The spins as an L x L int8 array of +1 / -1 (ising_get_spins)."""
        if out is None:
            out = np.empty((self.L, self.L), dtype=np.int8)
        assert out.dtype == np.int8 and out.size == self.L * self.L and out.flags["C_CONTIGUOUS"]
        _check(load().ising_get_spins(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), out.size),
               "ising_get_spins")
        return out

    def set_spins(self, s: np.ndarray):
        """Set the spins from an L x L int8 array, > 0 is up (ising_set_spins); pinned arrays are read in place."""
        s = np.ascontiguousarray(s, dtype=np.int8)
        assert s.size == self.L * self.L
        _check(load().ising_set_spins(self._h, s.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), s.size),
               "ising_set_spins")

    def get_words(self) -> np.ndarray:
        """The packed words of both colours, shape (2, L, pitch) (ising_get_words), for checkpoints."""
        _, P, _ = self.layout()
        out = np.empty(2 * self.L * P, dtype=np.uint64)
        _check(load().ising_get_words(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), out.size),
               "ising_get_words")
        return out.reshape(2, self.L, P)

    def set_words(self, words: np.ndarray):
        """Set the packed words of both colours (ising_set_words)."""
        w = np.ascontiguousarray(words, dtype=np.uint64).reshape(-1)
        _check(load().ising_set_words(self._h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), w.size),
               "ising_set_words")

    def device_words(self, c: int) -> int:
        """Device address of colour c's packed words (ising_device_words)."""
        p = ctypes.c_void_p()
        _check(load().ising_device_words(self._h, int(c), ctypes.byref(p)), "ising_device_words")
        return int(p.value)


def _ptr_array(arrays, ctype):
    """A C array of pointers to the given numpy arrays (None -> NULL)."""
    arr = (ctypes.c_void_p * len(arrays))()
    for k, a in enumerate(arrays):
        arr[k] = None if a is None else a.ctypes.data_as(ctypes.c_void_p).value
    return arr


class Batch:
    """Independent replicas of uneven L, each with its own beta, seed and
    start, swept together (see ising_batch_* in include/ising.h)."""

    def __init__(self, L, beta, seed, hot=None):
        lib = load()
        self.L = np.ascontiguousarray(L, dtype=np.int32)
        self.n = len(self.L)
        self.beta = np.ascontiguousarray(beta, dtype=np.float64)
        self.seed = np.ascontiguousarray(seed, dtype=np.uint64)
        hot_arr = None if hot is None else np.ascontiguousarray(hot, dtype=np.uint8)
        assert len(self.beta) == self.n and len(self.seed) == self.n
        h = ctypes.c_void_p()
        _check(lib.ising_batch_create(self.n, self.L.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      self.beta.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      self.seed.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                      None if hot_arr is None else hot_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                      ctypes.byref(h)), "ising_batch_create")
        self._h = h

    def close(self):
        """Release the batch (ising_batch_destroy); also done by the context manager."""
        if getattr(self, "_h", None) is not None and self._h.value is not None:
            load().ising_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_rng(self, scheme: int):
        """Random-number scheme of every replica (ising_batch_set_rng)."""
        _check(load().ising_batch_set_rng(self._h, int(scheme)), "ising_batch_set_rng")

    def set_tiling(self, threads_per_tile: int = 128, graph_chunk: int = 50):
        """Threads per tile and sweeps per captured graph (ising_batch_set_tiling); results do not depend on them."""
        _check(load().ising_batch_set_tiling(self._h, threads_per_tile, graph_chunk), "ising_batch_set_tiling")

    def set_lanes(self, lanes: int = 4):
        """Independent graph branches the replicas are split into (1..8)."""
        _check(load().ising_batch_set_lanes(self._h, int(lanes)), "ising_batch_set_lanes")

    def sweep(self, sweeps, every: int = 1, record: bool = True):
        """Replica r runs sweeps[r] sweeps; returns lists of int64 E and M arrays
        (sweeps[r] // every entries each), or None if record is False."""
        sw = np.ascontiguousarray(np.broadcast_to(np.asarray(sweeps, dtype=np.int64), (self.n,)))
        E = [np.zeros(max(int(s), 0) // max(every, 1), dtype=np.int64) for s in sw] if record else None
        M = [np.zeros(max(int(s), 0) // max(every, 1), dtype=np.int64) for s in sw] if record else None
        pe = _ptr_array(E, ctypes.c_int64) if record else None
        pm = _ptr_array(M, ctypes.c_int64) if record else None
        _check(load().ising_batch_sweep(self._h, sw.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), int(every),
                                        pe, pm), "ising_batch_sweep")
        return (E, M) if record else None

    def get_spins(self, r: int) -> np.ndarray:
        """Spins of replica r as an L x L int8 array (ising_batch_get_spins)."""
        L = int(self.L[r])
        out = np.empty((L, L), dtype=np.int8)
        _check(load().ising_batch_get_spins(self._h, int(r), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                                            out.size), "ising_batch_get_spins")
        return out

    def t(self, r: int) -> int:
        """Sweep counter of replica r (ising_batch_get_sweep)."""
        v = ctypes.c_uint64()
        _check(load().ising_batch_get_sweep(self._h, int(r), ctypes.byref(v)), "ising_batch_get_sweep")
        return int(v.value)


def batch_run(L, beta, seed, hot, sweeps, every: int = 1, final_spins: bool = False):
    """The one-call batch entry (ising_batch_run): returns (E, M, spins)."""
    lib = load()
    L = np.ascontiguousarray(L, dtype=np.int32)
    n = len(L)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    seed = np.ascontiguousarray(seed, dtype=np.uint64)
    hot = np.ascontiguousarray(hot, dtype=np.uint8)
    sw = np.ascontiguousarray(np.broadcast_to(np.asarray(sweeps, dtype=np.int64), (n,)))
    E = [np.zeros(int(s) // every, dtype=np.int64) for s in sw]
    M = [np.zeros(int(s) // every, dtype=np.int64) for s in sw]
    S = [np.empty((int(l), int(l)), dtype=np.int8) for l in L] if final_spins else None
    _check(lib.ising_batch_run(n, L.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               beta.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                               seed.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                               hot.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                               sw.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), int(every),
                               _ptr_array(E, ctypes.c_int64), _ptr_array(M, ctypes.c_int64),
                               _ptr_array(S, ctypes.c_int8) if S is not None else None), "ising_batch_run")
    return E, M, S


def philox_blocks(seed: int, ctr: np.ndarray) -> np.ndarray:
    """Philox4x32-10 blocks of the given counters (n x 4 uint32) on the device."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(c)
    _check(load().ising_philox_blocks(int(seed), c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), c.shape[0]),
           "ising_philox_blocks")
    return out


def check_status() -> tuple[bool, int]:
    """(checked build?, first out-of-range index record or 0) from
    ising_check_status; reading clears the record."""
    c, v = ctypes.c_int32(), ctypes.c_uint64()
    _check(load().ising_check_status(ctypes.byref(c), ctypes.byref(v)), "ising_check_status")
    return bool(c.value), int(v.value)


def probe_int_pipes() -> dict:
    """Integer instruction throughput of the current device (ising_probe_int_pipes):
    lane operations per SM per clock of 32x32->64 multiply-adds, 32-bit
    multiply-adds and three-input XORs, and the SM count."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    n = ctypes.c_int32()
    _check(load().ising_probe_int_pipes(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(n)),
           "ising_probe_int_pipes")
    return {"mulwide_per_sm_clk": a.value, "mad32_per_sm_clk": b.value, "lop3_per_sm_clk": c.value,
            "sm_count": n.value}


def means(E: np.ndarray, M: np.ndarray, L: int) -> tuple[float, float]:
    """Eq. 2 (ising_means): <E>/N and <|M|>/N over the recorded sweeps, from
    exact integer sums and one FP64 division each."""
    e = np.ascontiguousarray(E, dtype=np.int64)
    m = np.ascontiguousarray(M, dtype=np.int64)
    assert e.shape == m.shape and e.ndim == 1
    me, mm = ctypes.c_double(), ctypes.c_double()
    _check(load().ising_means(e.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                              m.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), e.size, int(L),
                              ctypes.byref(me), ctypes.byref(mm)), "ising_means")
    return me.value, mm.value
