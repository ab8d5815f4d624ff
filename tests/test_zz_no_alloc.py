"""ising_sweep_record_noalloc, the record path for callers that cannot
allocate device memory (for example a plug-in whose host program owns all
device memory through its own pool, or a latency-critical loop that must not
pay for an allocation).  It keeps its scratch in a fixed device array inside
the library, so these checks make sure that array gives the same results as
the allocating path, call after call.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _i64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def test_noalloc_matches_sweep_record_on_two_calls_in_a_row():
    import paper_1811_04384_gb300 as p
    lib = p.load()
    L, seed, beta = 130, 17, 0.44
    with p.Lattice(L, seed) as ref, p.Lattice(L, seed) as own:
        ref.init_hot()
        ref.set_beta(beta)
        own.init_hot()                  # the caller-owned packed lattice
        w0, w1 = own.device_words(0), own.device_words(1)
        t0 = 0
        for n, every in ((20, 2), (31, 3)):
            E_ref, M_ref = ref.sweep_record(n, every)
            E = np.full(n // every, -7, dtype=np.int64)
            M = np.full(n // every, -7, dtype=np.int64)
            rc = lib.ising_sweep_record_noalloc(ctypes.c_void_p(w0), ctypes.c_void_p(w1), L, seed, beta,
                                                t0, n, every, _i64p(E), _i64p(M), None)
            assert rc == p.ISING_OK, p.IsingError(rc, "ising_sweep_record_noalloc")
            np.testing.assert_array_equal(E, E_ref)
            np.testing.assert_array_equal(M, M_ref)
            t0 += n
        np.testing.assert_array_equal(own.get_spins(), ref.get_spins())


def test_noalloc_rejects_more_records_than_its_scratch_holds():
    import paper_1811_04384_gb300 as p
    lib = p.load()
    with p.Lattice(64, 1) as own:
        w0, w1 = own.device_words(0), own.device_words(1)
        E = np.zeros(1, dtype=np.int64)
        too_many = p.ISING_NOALLOC_MAX_RECORDS + 1
        rc = lib.ising_sweep_record_noalloc(ctypes.c_void_p(w0), ctypes.c_void_p(w1), 64, 1, 0.4, 0, too_many, 1,
                                            _i64p(E), None, None)
        assert rc == p.ISING_EINVAL
        assert own.t == 0 and own.energy() == -2 * 64 * 64   # nothing ran
