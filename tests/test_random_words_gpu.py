"""The paper's own chain on the GPU (random memory-word updates in two column
phases per iteration, the strips of a phase in parallel, each strip's
updates in sequence order): spins and the E/M series equal the oracle's
sequential chain word for word, at L = 84 .. 252 (N = 4 .. 12 word rows),
for one strip (the paper's one-process program) up to two columns per strip,
odd and even strip widths, and the temperature limits."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

BETA_TC = 1.0 / 2.269


@pytest.fixture(scope="module")
def ising():
    import paper_1811_04384_gb300 as p
    p.load()
    return p


def gpu_rw(ising, L, seed, beta, n, nstrips, every=1, hot=True, t0=0):
    with ising.Lattice(L, seed, layout=ising.ISING_LAYOUT_COLUMN_INTERLEAVED) as lat:
        if hot:
            lat.init_hot()
        lat.set_chain(ising.ISING_CHAIN_RANDOM_WORDS, nstrips)
        lat.set_beta(beta)
        if t0:
            lat.t = t0
        E, M = lat.sweep_record(n, every)
        return E, M, lat.get_spins(), lat.t


def oracle_rw(L, seed, beta, n, nstrips, every=1, hot=True, t0=0):
    s = oracle.init_hot(L, seed) if hot else oracle.init_cold(L, 1)
    E, M = oracle.rw_run(s, seed, beta, t0, n, nstrips, every)
    return E, M, s


CASES = [
    (84, 1, BETA_TC, 3, 1), (84, 2, 0.3, 3, 1), (84, 3, BETA_TC, 2, 2), (84, 42, BETA_TC, 4, 1),
    (84, 6, 0.0, 3, 1), (168, 4, BETA_TC, 3, 1), (168, 12, 0.6, 2, 1), (168, 84, BETA_TC, 2, 1),
    (252, 1, BETA_TC, 2, 1), (252, 12, BETA_TC, 3, 3), (252, 7, 0.44, 2, 1), (252, 126, 0.3, 2, 2),
]


@pytest.mark.parametrize("L,nstrips,beta,n,every", CASES)
def test_random_words_match_oracle(ising, L, nstrips, beta, n, every):
    seed = 1000 + L + nstrips
    E, M, S, t = gpu_rw(ising, L, seed, beta, n, nstrips, every)
    Eo, Mo, so = oracle_rw(L, seed, beta, n, nstrips, every)
    np.testing.assert_array_equal(E, Eo)
    np.testing.assert_array_equal(M, Mo)
    np.testing.assert_array_equal(S, so)
    assert t == n


@pytest.mark.parametrize("L,nstrips,path", [(1008, 1, None), (168, 6, "launches"), (1008, 1, "launches")])
def test_random_words_every_form(ising, L, nstrips, path):
    """The forms of the kernel: a half strip too wide for shared memory
    (L = 1008 in one strip: 48 x 506 words) works in global memory; with the
    launch path each strip draws its own updates instead of reading draws
    made first on all SMs.  All equal the oracle."""
    seed = 77 + L
    with ising.Lattice(L, seed, layout=ising.ISING_LAYOUT_COLUMN_INTERLEAVED) as lat:
        if path == "launches":
            lat.set_path(ising.ISING_PATH_LAUNCHES)
        lat.init_hot()
        lat.set_chain(ising.ISING_CHAIN_RANDOM_WORDS, nstrips)
        lat.set_beta(BETA_TC)
        E, M = lat.sweep_record(1, 1)
        S = lat.get_spins()
    Eo, Mo, so = oracle_rw(L, seed, BETA_TC, 1, nstrips)
    np.testing.assert_array_equal(E, Eo)
    np.testing.assert_array_equal(M, Mo)
    np.testing.assert_array_equal(S, so)


def test_random_words_cold_and_frozen(ising):
    """Cold start: at beta = 6 the ground state stays frozen; at T_c the chain
    leaves it exactly as the oracle does."""
    E, M, S, _ = gpu_rw(ising, 168, 5, 6.0, 3, 4, hot=False)
    assert (E == -2 * 168 * 168).all() and (M == 168 * 168).all()
    E, M, S, _ = gpu_rw(ising, 168, 5, BETA_TC, 3, 4, hot=False)
    Eo, Mo, so = oracle_rw(168, 5, BETA_TC, 3, 4, hot=False)
    np.testing.assert_array_equal(E, Eo)
    np.testing.assert_array_equal(S, so)


def test_random_words_resume_at_t(ising):
    """Iterations are keyed by t: starting at t0 = 2^32 + 5 (the high word of
    the counter) equals the oracle from the same t0."""
    t0 = (1 << 32) + 5
    E, M, S, t = gpu_rw(ising, 84, 9, BETA_TC, 2, 6, t0=t0)
    Eo, Mo, so = oracle_rw(84, 9, BETA_TC, 2, 6, t0=t0)
    np.testing.assert_array_equal(E, Eo)
    np.testing.assert_array_equal(S, so)
    assert t == t0 + 2


def test_switching_chains(ising):
    """Checkerboard sweeps, then random-word iterations, then checkerboard
    again on one lattice: each part follows its own chain from the state the
    previous one left."""
    L, seed = 168, 77
    with ising.Lattice(L, seed, layout=ising.ISING_LAYOUT_COLUMN_INTERLEAVED) as lat:
        lat.init_hot()
        lat.set_beta(BETA_TC)
        lat.sweep(3)
        lat.set_chain(ising.ISING_CHAIN_RANDOM_WORDS, 12)
        lat.sweep(2)
        lat.set_chain(ising.ISING_CHAIN_CHECKERBOARD)
        E, M = lat.sweep_record(2, 1)
        S = lat.get_spins()
    s = oracle.init_hot(L, seed)
    oracle.run(s, seed, BETA_TC, 0, 3, 3)
    oracle.rw_run(s, seed, BETA_TC, 3, 2, 12)
    Eo, Mo = oracle.run(s, seed, BETA_TC, 5, 2, 1)
    np.testing.assert_array_equal(E, Eo)
    np.testing.assert_array_equal(M, Mo)
    np.testing.assert_array_equal(S, s)


def test_random_words_bad_arguments(ising):
    with ising.Lattice(84, 1) as lat:                      # row-packed: no random-word chain
        with pytest.raises(ising.IsingError):
            lat.set_chain(ising.ISING_CHAIN_RANDOM_WORDS, 1)
    with ising.Lattice(84, 1, layout=ising.ISING_LAYOUT_COLUMN_INTERLEAVED) as lat:
        for bad in (0, 5, 43, 84):                          # 84 strips: one column each
            with pytest.raises(ising.IsingError):
                lat.set_chain(ising.ISING_CHAIN_RANDOM_WORDS, bad)
        with pytest.raises(ising.IsingError):
            lat.set_chain(7, 1)
