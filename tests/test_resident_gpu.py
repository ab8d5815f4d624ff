"""The on-chip (temporal-blocked) path: the whole lattice in one block's
shared memory for all requested sweeps.  Bit-exact with the launch path and
the oracle; covers the L classes that fit (up to 2 L pitch 8 B <= 220 KB)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ising():
    import paper_1811_04384_gb300 as p
    p.load()
    return p


def run(ising, L, seed, beta, n, every, path, hot=True):
    with ising.Lattice(L, seed) as lat:
        lat.set_path(path)
        if hot:
            lat.init_hot()
        lat.set_beta(beta)
        E, M = lat.sweep_record(n, every)
        lat.sweep(3)
        return E, M, lat.get_spins(), lat.t, lat.energy()


# The on-chip forms by thread items (ceil(L/4) * W): masks drawn beforehand
# with one row a thread up to 256 items (L <= 204), two rows a thread up to
# 512 (L = 206 .. 292), the draws inside the on-chip kernel (one thread per
# item) above (L >= 294).  W = 1 up to L = 42, so both wraps fall in one word.
@pytest.mark.parametrize("L", [4, 6, 10, 42, 44, 46, 64, 66, 84, 86, 100, 126, 128, 130, 168, 170, 200,
                               204, 206, 256, 292, 294, 300, 512, 700])
def test_resident_equals_launches(ising, L):
    beta = 0.3 + (L % 7) * 0.05
    a = run(ising, L, 40 + L, beta, 25, 3, ising.ISING_PATH_RESIDENT)
    b = run(ising, L, 40 + L, beta, 25, 3, ising.ISING_PATH_LAUNCHES)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    assert a[3] == 28


@pytest.mark.parametrize("L", [32, 64, 66, 130, 256])
def test_resident_seven_round_scheme_equals_launches(ising, L):
    def go(path):
        with ising.Lattice(L, 9) as lat:
            lat.set_rng(ising.ISING_RNG_PHILOX4X32_7)
            lat.set_path(path)
            lat.init_hot()
            lat.set_beta(0.42)
            E, M = lat.sweep_record(12, 1)
            return E, M, lat.get_spins()
    for x, y in zip(go(ising.ISING_PATH_RESIDENT), go(ising.ISING_PATH_LAUNCHES)):
        np.testing.assert_array_equal(x, y)


def test_resident_matches_oracle_plain_config(ising):
    E, M, S, _, _ = run(ising, 64, 1, 1.0 / 2.269, 1000, 1, ising.ISING_PATH_RESIDENT)
    s = oracle.init_hot(64, 1)
    Eo, Mo = oracle.run(s, 1, 1.0 / 2.269, 0, 1000, 1)
    oracle.run(s, 1, 1.0 / 2.269, 1000, 3, 3)
    np.testing.assert_array_equal(E, Eo)
    np.testing.assert_array_equal(M, Mo)
    np.testing.assert_array_equal(S, s)


def test_resident_many_records_and_chunks(ising):
    # more records than one device chunk holds (1024), and a remainder
    a = run(ising, 32, 5, 0.44, 2600, 2, ising.ISING_PATH_RESIDENT)
    b = run(ising, 32, 5, 0.44, 2600, 2, ising.ISING_PATH_LAUNCHES)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_resident_masks_drawn_in_pieces(ising):
    # L = 292 (511 items): the 16 MB mask buffer holds 255 sweeps, so 600
    # sweeps are drawn and applied in three pieces; records every 7 sweeps
    # straddle the piece boundaries
    a = run(ising, 292, 8, 0.43, 600, 7, ising.ISING_PATH_RESIDENT)
    b = run(ising, 292, 8, 0.43, 600, 7, ising.ISING_PATH_LAUNCHES)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    assert a[3] == 603


def test_resident_plain_sweeps_in_pieces(ising):
    # 600 sweeps without records in three mask pieces, then the energy: the
    # same state as the launch path's graph replays and leftovers
    def go(path):
        with ising.Lattice(292, 4) as lat:
            lat.set_path(path)
            lat.init_hot()
            lat.set_beta(0.41)
            lat.sweep(600)
            return lat.get_spins(), lat.energy(), lat.magnetization(), lat.t
    a, b = go(ising.ISING_PATH_RESIDENT), go(ising.ISING_PATH_LAUNCHES)
    np.testing.assert_array_equal(a[0], b[0])
    assert a[1:] == b[1:] and a[3] == 600


def test_resident_rejects_lattices_that_do_not_fit(ising):
    with ising.Lattice(1024, 1) as lat:
        with pytest.raises(ising.IsingError):
            lat.set_path(ising.ISING_PATH_RESIDENT)
        lat.set_path(ising.ISING_PATH_AUTO)     # auto falls back to launches
        lat.sweep(1)
    with ising.Lattice(64, 1) as lat:
        with pytest.raises(ising.IsingError):
            lat.set_path(7)
