"""The paper's column-interleaved word layout (Sec. 3): N x L words, word
S(I, J) holding s(I + kN, J), one-field rotation across the top and bottom
word rows, Eq. 3 in arithmetic form.  Same chain as the row-packed layout, so
spins and E/M are bit-exact with the oracle and with the default layout."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ising():
    import paper_1811_04384_gb300 as p
    p.load()
    return p


def interleaved(ising, L, seed):
    return ising.Lattice(L, seed, layout=ising.ISING_LAYOUT_COLUMN_INTERLEAVED)


@pytest.mark.parametrize("path", ["auto", "launches"])
@pytest.mark.parametrize("L", [84, 168, 252])
def test_interleaved_matches_oracle(ising, L, path):
    """Automatic path (the cluster path at these sizes) and the graph replays."""
    beta = 0.41
    with interleaved(ising, L, 5 + L) as lat:
        if path == "launches":
            lat.set_path(ising.ISING_PATH_LAUNCHES)
        lat.init_hot()
        np.testing.assert_array_equal(lat.get_spins(), oracle.init_hot(L, 5 + L))
        lat.set_beta(beta)
        E, M = lat.sweep_record(12, 2)
        spins = lat.get_spins()
        e_now, m_now = lat.energy(), lat.magnetization()
    s = oracle.init_hot(L, 5 + L)
    Eo, Mo = oracle.run(s, 5 + L, beta, 0, 12, 2)
    np.testing.assert_array_equal(E, Eo)
    np.testing.assert_array_equal(M, Mo)
    np.testing.assert_array_equal(spins, s)
    assert e_now == oracle.energy(s) and m_now == oracle.magnetization(s)


@pytest.mark.parametrize("path", ["auto", "launches"])
@pytest.mark.parametrize("L", [1008, 2016])
def test_paper_sizes_equal_row_packed(ising, L, path):
    """The paper's lattice sizes (N = 48 and 96 word rows), the interleaved
    lattice on the automatic path (the cluster path at L = 1008) and on the
    graph replays, the row-packed one on its automatic path."""
    with interleaved(ising, L, 11) as a, ising.Lattice(L, 11) as b:
        if path == "launches":
            a.set_path(ising.ISING_PATH_LAUNCHES)
        for lat in (a, b):
            lat.init_hot()
            lat.set_beta(1.0 / 2.269)
        Ea, Ma = a.sweep_record(20, 1)
        Eb, Mb = b.sweep_record(20, 1)
        np.testing.assert_array_equal(Ea, Eb)
        np.testing.assert_array_equal(Ma, Mb)
        np.testing.assert_array_equal(a.get_spins(), b.get_spins())
        # long enough for the replayed graphs of both layouts (32-sweep chunks)
        for lat in (a, b):
            lat.sweep(40)
        Ea2, Ma2 = a.sweep_record(70, 1)
        Eb2, Mb2 = b.sweep_record(70, 1)
        np.testing.assert_array_equal(Ea2, Eb2)
        np.testing.assert_array_equal(Ma2, Mb2)
        np.testing.assert_array_equal(a.get_spins(), b.get_spins())
    if L == 1008:
        s = oracle.init_hot(L, 11)
        Eo, _ = oracle.run(s, 11, 1.0 / 2.269, 0, 20, 1)
        np.testing.assert_array_equal(Ea, Eo)


def test_interleaved_spin_io_cold_start_and_seven_rounds(ising):
    L = 168
    rng = np.random.default_rng(2)
    s = np.where(rng.random((L, L)) < 0.3, 1, -1).astype(np.int8)
    with interleaved(ising, L, 3) as lat:
        assert lat.energy() == -2 * L * L and lat.magnetization() == L * L   # created cold +1
        lat.set_spins(s)
        np.testing.assert_array_equal(lat.get_spins(), s)
        assert lat.energy() == oracle.energy(s)
        lat.init_cold(-1)
        assert lat.magnetization() == -L * L
        lat.init_hot()
        lat.set_rng(ising.ISING_RNG_PHILOX4X32_7)
        lat.set_beta(0.5)
        E, M = lat.sweep_record(6, 3)
        got = lat.get_spins()
    with oracle.sweep_rounds(7):
        so = oracle.init_hot(L, 3)
        Eo, Mo = oracle.run(so, 3, 0.5, 0, 6, 3)
    np.testing.assert_array_equal(E, Eo)
    np.testing.assert_array_equal(got, so)


def test_interleaved_rejects_sizes_and_row_packed_calls(ising):
    for bad in (42, 126, 170, 0):
        with pytest.raises(ising.IsingError):
            interleaved(ising, bad, 1)
    with interleaved(ising, 84, 1) as lat:
        with pytest.raises(ising.IsingError):
            lat.get_words()
        with pytest.raises(ising.IsingError):
            lat.layout()
        with pytest.raises(ising.IsingError):
            lat.set_path(ising.ISING_PATH_RESIDENT)
        with pytest.raises(ising.IsingError):
            lat.set_tiling(4, 32, 4)
        with pytest.raises(ising.IsingError):
            lat.set_item_lanes(4)


def test_interleaved_run_states_equals_calls_in_turn(ising):
    """ising_run_states on the paper's layout runs the calls in turn."""
    L = 168
    rng = np.random.default_rng(3)
    states = [np.where(rng.random((L, L)) < 0.5, 1, -1).astype(np.int8) for _ in range(3)]
    with interleaved(ising, L, 2) as a, interleaved(ising, L, 2) as b:
        for lat in (a, b):
            lat.set_beta(0.44)
        E1, M1 = a.run_states(states, 6, 2)
        for k, st in enumerate(states):
            b.set_spins(st)
            E, M = b.sweep_record(6, 2)
            np.testing.assert_array_equal(E1[k], E)
            np.testing.assert_array_equal(M1[k], M)
        np.testing.assert_array_equal(a.get_spins(), b.get_spins())
