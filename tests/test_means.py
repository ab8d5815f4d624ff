"""Eq. 2 (per-spin averages over the recorded iterations): the oracle's
`means` pinned to hand-summed series and to two exact dynamical limits, and
the library's host entry point ising_means equal to it bit for bit.  No GPU:
ising_means is host arithmetic on caller arrays."""
import ctypes
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def golden_cases():
    cases = []
    for line in open(os.path.join(HERE, "golden", "means_cases.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        L, e, m, me, mm = [f.strip() for f in line.split("|")]
        cases.append((int(L), np.array(e.split(), dtype=np.int64), np.array(m.split(), dtype=np.int64),
                      float(me), float(mm)))
    return cases


@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: f"L{c[0]}n{len(c[1])}")
def test_oracle_means_hand_summed(case):
    L, E, M, me, mm = case
    assert oracle.means(E, M, L) == (me, mm)


def test_oracle_means_frozen_ground_state():
    """beta >= 32 ln2 / 4: from a cold start no uphill flip is ever accepted
    and every site has a = 0, so E_t = -2 L^2 and M_t = L^2 at every sweep:
    the means are exactly -2 and 1."""
    for L in (4, 8, 10):
        s = oracle.init_cold(L, 1)
        E, M = oracle.run(s, 5, 6.0, 0, 7, 1)
        assert oracle.means(E, M, L) == (-2.0, 1.0)
        s = oracle.init_cold(L, -1)
        E, M = oracle.run(s, 5, 6.0, 0, 7, 1)
        assert (M < 0).all()
        assert oracle.means(E, M, L) == (-2.0, 1.0)


def test_oracle_means_infinite_temperature():
    """beta = 0: every site flips every half-sweep, so E_t = E_0 and
    M_t = (-1)^t M_0: the means are E_0 / L^2 and |M_0| / L^2 whatever the
    number of records (M alternates in sign, so a mean of M would be 0 or
    M_0 / (n L^2))."""
    for L, seed in ((6, 3), (10, 8), (16, 2)):
        s = oracle.init_hot(L, seed)
        E0, M0 = oracle.energy(s), oracle.magnetization(s)
        assert M0 != 0
        E, M = oracle.run(s, seed, 0.0, 0, 6, 1)
        assert oracle.means(E, M, L) == (E0 / L**2, abs(M0) / L**2)


def test_oracle_means_record_interval():
    """A series recorded every 3rd sweep is the every-sweep series sampled at
    t = 3, 6, ...: Eq. 2 over those records only."""
    L, seed, beta = 12, 4, 0.44
    s1 = oracle.init_hot(L, seed)
    E1, M1 = oracle.run(s1, seed, beta, 0, 12, 1)
    s3 = oracle.init_hot(L, seed)
    E3, M3 = oracle.run(s3, seed, beta, 0, 12, 3)
    np.testing.assert_array_equal(E3, E1[2::3])
    e, m = oracle.means(E3, M3, L)
    assert e == int(E1[2::3].sum()) / (4 * L * L)
    assert m == int(np.abs(M1[2::3]).sum()) / (4 * L * L)


@pytest.fixture(scope="module")
def lib():
    from paper_1811_04384_gb300 import build
    build.build()
    import paper_1811_04384_gb300 as p
    return p.load()


def c_means(lib, E, M, L):
    E = np.ascontiguousarray(E, dtype=np.int64)
    M = np.ascontiguousarray(M, dtype=np.int64)
    me, mm = ctypes.c_double(), ctypes.c_double()
    rc = lib.ising_means(E.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                         M.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), E.size, L, ctypes.byref(me),
                         ctypes.byref(mm))
    assert rc == 0
    return me.value, mm.value


@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: f"L{c[0]}n{len(c[1])}")
def test_library_means_hand_summed(lib, case):
    L, E, M, me, mm = case
    assert c_means(lib, E, M, L) == (me, mm)


def test_library_means_equal_oracle_on_oracle_series(lib):
    import paper_1811_04384_gb300 as p
    for L, seed, beta, n in ((16, 1, 1 / 2.269, 300), (42, 9, 0.3, 120), (64, 1, 1 / 2.269, 60)):
        s = oracle.init_hot(L, seed)
        E, M = oracle.run(s, seed, beta, 0, n, 1)
        assert c_means(lib, E, M, L) == oracle.means(E, M, L)
        assert p.means(E, M, L) == oracle.means(E, M, L)


def test_library_means_large_sums(lib):
    """Records of the largest lattice: the 128-bit sums stay exact; the
    quotient is correctly rounded while the sum is below 2^53 and within
    1e-15 relative of the exact ratio beyond."""
    L = 32768
    n = 5_500_000
    rng = np.random.default_rng(5)
    E = -rng.integers(3 * L * L // 2, 2 * L * L, size=n, dtype=np.int64)
    M = rng.integers(-L * L, L * L, size=n, dtype=np.int64)
    assert -int(E.sum()) > 2**53
    e, m = c_means(lib, E, M, L)
    eo, mo = oracle.means(E, M, L)
    assert abs(e - eo) <= 1e-15 * abs(eo) and abs(m - mo) <= 1e-15 * abs(mo)
    small = slice(0, 100)
    assert c_means(lib, E[small], M[small], L) == oracle.means(E[small], M[small], L)


def test_library_means_rejects_bad_arguments(lib):
    import paper_1811_04384_gb300 as p
    E = np.zeros(3, dtype=np.int64)
    pe = E.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d = ctypes.c_double()
    assert lib.ising_means(pe, pe, 0, 64, ctypes.byref(d), ctypes.byref(d)) == p.ISING_EINVAL
    assert lib.ising_means(pe, pe, 3, 63, ctypes.byref(d), ctypes.byref(d)) == p.ISING_EINVAL
    assert lib.ising_means(None, pe, 3, 64, ctypes.byref(d), None) == p.ISING_EINVAL
    assert lib.ising_means(pe, pe, 3, 64, None, None) == p.ISING_EINVAL
    assert lib.ising_means(pe, None, 3, 64, ctypes.byref(d), None) == 0
