"""The cluster path (one thread-block cluster keeping the lattice in its
blocks' shared memory, halos exchanged through distributed shared memory),
in the row-packed layout and in the paper's column-interleaved layout,
against the oracle, bit-exact: int64 E/M series and final spins.

Cases span two rows per block (L = 32, two half-sweeps per phase), the
automatic range with one cluster (L = 296 just above the on-chip path, with
two mask pieces) and with several (their halos between clusters through
global memory), L % 4 == 2, records out of step with the phases and pieces,
odd numbers of half-sweeps per call, cold starts, beta = 0 (every flip
accepted) and a frozen
lattice, runs continued across calls and paths, and ising_run_states.
"""
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


# (L, sweeps, every, beta, forced): forced sets ISING_PATH_CLUSTER, else the
# automatic choice must be the cluster path
CASES = [
    (32, 9, 1, 0.44, True),        # two rows per block: phases of two half-sweeps
    (64, 13, 2, 0.3, True),        # four rows per block, phases of 4
    (296, 37, 1, BETA_TC, False),  # 74 half-sweeps: phases of 12 and a short last one
    (296, 300, 7, 0.41, False),    # two mask pieces (256 + 44 sweeps), records across them
    (514, 20, 3, 0.3, False),      # L % 4 == 2; 6 records, out of step with the phases
    (1008, 24, 4, 0.44, False),    # the paper's L = 1008
    (1080, 60, 5, BETA_TC, False), # four clusters
    (1176, 8, 2, 0.44, False),     # six clusters
    (1500, 6, 1, 0.44, True),      # five clusters
    (1600, 3, 1, BETA_TC, True),   # five clusters
]


def test_cluster_path_matches_oracle(ising):
    got = []
    for L, n, every, beta, forced in CASES:
        with ising.Lattice(L, L + 7) as lat:
            if forced:
                lat.set_path(ising.ISING_PATH_CLUSTER)
            assert lat.get_path() == ising.ISING_PATH_CLUSTER, L
            lat.init_hot()
            lat.set_beta(beta)
            E, M = lat.sweep_record(n, every)
            assert lat.t == n
            got.append((E, M, lat.get_spins()))
    ora = oracle.run_jobs([(L, L + 7, beta, True, n, every) for L, n, every, beta, _ in CASES])
    for (E, M, S), (Eo, Mo, So), case in zip(got, ora, CASES):
        np.testing.assert_array_equal(E, Eo, err_msg=str(case))
        np.testing.assert_array_equal(M, Mo, err_msg=str(case))
        np.testing.assert_array_equal(S, So, err_msg=str(case))


# the paper's column-interleaved layout (L % 84 == 0): (L, sweeps, every,
# beta, forced)
CI_CASES = [
    (84, 9, 1, 0.44, False),       # N = 4 word rows, 16 blocks of 4 or 8 columns, phases of 4
    (252, 26, 3, BETA_TC, False),  # phases of 12, records out of step with them
    (504, 300, 7, 0.41, False),    # two mask pieces (256 + 44 sweeps)
    (840, 20, 4, 0.44, False),     # two pairs per thread
    (1008, 24, 5, BETA_TC, False), # the paper's L = 1008 (N = 48), four clusters
    (1092, 6, 1, 0.44, False),     # four clusters
    (1260, 4, 1, 0.41, True),      # four pairs per thread
    (1512, 3, 1, BETA_TC, True),   # two mask slabs, four pairs per thread
]


def test_interleaved_cluster_path_matches_oracle(ising):
    got = []
    for L, n, every, beta, forced in CI_CASES:
        with ising.Lattice(L, L + 3, layout=ising.ISING_LAYOUT_COLUMN_INTERLEAVED) as lat:
            if forced:
                lat.set_path(ising.ISING_PATH_CLUSTER)
            assert lat.get_path() == ising.ISING_PATH_CLUSTER, L
            lat.init_hot()
            lat.set_beta(beta)
            E, M = lat.sweep_record(n, every)
            assert lat.t == n
            got.append((E, M, lat.get_spins()))
    ora = oracle.run_jobs([(L, L + 3, beta, True, n, every) for L, n, every, beta, _ in CI_CASES])
    for (E, M, S), (Eo, Mo, So), case in zip(got, ora, CI_CASES):
        np.testing.assert_array_equal(E, Eo, err_msg=str(case))
        np.testing.assert_array_equal(M, Mo, err_msg=str(case))
        np.testing.assert_array_equal(S, So, err_msg=str(case))


def test_interleaved_cluster_extremes_and_continuation(ising):
    """beta = 0 and a frozen cold lattice in the interleaved layout, then a
    run continued across the cluster path and the graph replays."""
    L = 336
    for beta, cold in ((0.0, False), (5.0, True)):
        with ising.Lattice(L, 8, layout=ising.ISING_LAYOUT_COLUMN_INTERLEAVED) as lat:
            lat.init_cold(1) if cold else lat.init_hot()
            lat.set_beta(beta)
            E, M = lat.sweep_record(4, 1)
            S = lat.get_spins()
        s = oracle.init_cold(L, 1) if cold else oracle.init_hot(L, 8)
        Eo, Mo = oracle.run(s, 8, beta, 0, 4, 1)
        np.testing.assert_array_equal(E, Eo)
        np.testing.assert_array_equal(M, Mo)
        np.testing.assert_array_equal(S, s)
    with ising.Lattice(L, 9, layout=ising.ISING_LAYOUT_COLUMN_INTERLEAVED) as lat:
        lat.init_hot()
        lat.set_beta(0.43)
        lat.sweep(5)
        lat.set_path(ising.ISING_PATH_LAUNCHES)
        E1, M1 = lat.sweep_record(6, 2)
        lat.set_path(ising.ISING_PATH_AUTO)
        E2, M2 = lat.sweep_record(9, 3)
        S = lat.get_spins()
    s = oracle.init_hot(L, 9)
    oracle.run(s, 9, 0.43, 0, 5, 5)
    Eo1, Mo1 = oracle.run(s, 9, 0.43, 5, 6, 2)
    Eo2, Mo2 = oracle.run(s, 9, 0.43, 11, 9, 3)
    for got, want in ((E1, Eo1), (M1, Mo1), (E2, Eo2), (M2, Mo2), (S, s)):
        np.testing.assert_array_equal(got, want)


# several clusters per launch, halos between clusters through global memory:
# (L, clusters, sweeps, every)
MULTI_CASES = [
    (600, 2, 26, 3),     # 32 blocks of 18-19 rows
    (600, 2, 300, 10),   # two pieces (256 + 44 sweeps): the flags carry on across launches
    (1000, 3, 14, 2),    # 48 blocks
    (1600, 2, 8, 4),     # 50 rows per block
    (2016, 3, 6, 1),     # the paper's L = 2016
    (3000, 5, 3, 1),     # 80 blocks
]


def test_multi_cluster_matches_oracle(ising):
    got = []
    for L, G, n, every in MULTI_CASES:
        with ising.Lattice(L, L + 11) as lat:
            lat.set_clusters(G)
            assert lat.get_path() == ising.ISING_PATH_CLUSTER, (L, G)
            lat.init_hot()
            lat.set_beta(0.42)
            E, M = lat.sweep_record(n, every)
            got.append((E, M, lat.get_spins()))
    ora = oracle.run_jobs([(L, L + 11, 0.42, True, n, every) for L, G, n, every in MULTI_CASES])
    for (E, M, S), (Eo, Mo, So), case in zip(got, ora, MULTI_CASES):
        np.testing.assert_array_equal(E, Eo, err_msg=str(case))
        np.testing.assert_array_equal(M, Mo, err_msg=str(case))
        np.testing.assert_array_equal(S, So, err_msg=str(case))


# the column-interleaved layout on several clusters: (L, clusters, sweeps, every)
CI_MULTI_CASES = [
    (504, 2, 20, 3),
    (1008, 3, 12, 2),
    (2016, 4, 4, 1),     # the paper's cases 1-2 size
    (3024, 5, 2, 1),
]


def test_interleaved_multi_cluster_matches_oracle(ising):
    got = []
    for L, G, n, every in CI_MULTI_CASES:
        with ising.Lattice(L, L + 13, layout=ising.ISING_LAYOUT_COLUMN_INTERLEAVED) as lat:
            lat.set_clusters(G)
            assert lat.get_path() == ising.ISING_PATH_CLUSTER, (L, G)
            lat.init_hot()
            lat.set_beta(0.44)
            E, M = lat.sweep_record(n, every)
            got.append((E, M, lat.get_spins()))
    ora = oracle.run_jobs([(L, L + 13, 0.44, True, n, every) for L, G, n, every in CI_MULTI_CASES])
    for (E, M, S), (Eo, Mo, So), case in zip(got, ora, CI_MULTI_CASES):
        np.testing.assert_array_equal(E, Eo, err_msg=str(case))
        np.testing.assert_array_equal(M, Mo, err_msg=str(case))
        np.testing.assert_array_equal(S, So, err_msg=str(case))


def test_multi_cluster_continued_and_rejected(ising):
    """Calls continued with 2, then 3 clusters, then 1 (the exchange flags
    only ever rise across launches), and the counts a lattice rejects."""
    L, seed, beta = 900, 17, 0.44
    with ising.Lattice(L, seed) as lat:
        lat.init_hot()
        lat.set_beta(beta)
        lat.set_clusters(2)
        lat.sweep(5)
        E1, M1 = lat.sweep_record(7, 1)
        lat.set_clusters(3)
        E2, M2 = lat.sweep_record(8, 2)
        lat.set_clusters(1)
        E3, M3 = lat.sweep_record(3, 3)
        S = lat.get_spins()
        for bad in (-1, 17, 16):
            with pytest.raises(ising.IsingError):
                lat.set_clusters(bad)
    s = oracle.init_hot(L, seed)
    oracle.run(s, seed, beta, 0, 5, 5)
    for (E, M), (t0, n, every) in zip([(E1, M1), (E2, M2), (E3, M3)], [(5, 7, 1), (12, 8, 2), (20, 3, 3)]):
        Eo, Mo = oracle.run(s, seed, beta, t0, n, every)
        np.testing.assert_array_equal(E, Eo)
        np.testing.assert_array_equal(M, Mo)
    np.testing.assert_array_equal(S, s)
    with ising.Lattice(84, 1, layout=ising.ISING_LAYOUT_COLUMN_INTERLEAVED) as lat:
        with pytest.raises(ising.IsingError):
            lat.set_clusters(2)      # 21 column groups of 4 for 32 blocks


def test_multi_cluster_wait_gives_up_and_recovers(ising):
    """A launch whose waits between clusters can never be satisfied (the test
    hook): each wait gives up after a second of the GPU's clock, the call
    returns ISING_ETIMEOUT, the context stays usable, and after restoring a
    checkpoint the run continues bit-exactly."""
    L, seed, beta = 600, 23, 0.43
    with ising.Lattice(L, seed) as lat:
        lat.set_clusters(2)
        lat.init_hot()
        lat.set_beta(beta)
        lat.sweep(3)
        words, t = lat.get_words(), lat.t
        lat.inject_stall(1)
        with pytest.raises(ising.IsingError) as err:
            lat.sweep(2)
        assert err.value.code == ising.ISING_ETIMEOUT
        lat.set_words(words)
        lat.t = t
        E, M = lat.sweep_record(6, 2)
        S = lat.get_spins()
    s = oracle.init_hot(L, seed)
    oracle.run(s, seed, beta, 0, 3, 3)
    Eo, Mo = oracle.run(s, seed, beta, 3, 6, 2)
    np.testing.assert_array_equal(E, Eo)
    np.testing.assert_array_equal(M, Mo)
    np.testing.assert_array_equal(S, s)


def test_interleaved_multi_cluster_wait_gives_up_and_recovers(ising):
    """The same give-up in the column-interleaved cluster kernel (its halo
    columns between clusters wait on the same flags), with the checkpoint
    taken as spins."""
    L, seed, beta = 504, 29, 0.43
    with ising.Lattice(L, seed, layout=ising.ISING_LAYOUT_COLUMN_INTERLEAVED) as lat:
        lat.set_clusters(2)
        lat.init_hot()
        lat.set_beta(beta)
        lat.sweep(3)
        spins, t = lat.get_spins(), lat.t
        lat.inject_stall(1)
        with pytest.raises(ising.IsingError) as err:
            lat.sweep(2)
        assert err.value.code == ising.ISING_ETIMEOUT
        lat.set_spins(spins)
        lat.t = t
        E, M = lat.sweep_record(6, 2)
        S = lat.get_spins()
    s = oracle.init_hot(L, seed)
    oracle.run(s, seed, beta, 0, 3, 3)
    Eo, Mo = oracle.run(s, seed, beta, 3, 6, 2)
    np.testing.assert_array_equal(E, Eo)
    np.testing.assert_array_equal(M, Mo)
    np.testing.assert_array_equal(S, s)


# (L, layout, after, sweeps, every): the launch with several clusters after
# `after` more of them counts on one block more than it has
ABSENT_CASES = [
    (1008, "row", 1, 400, 7),      # piece 0 (256 sweeps) on four clusters, piece 1 (144) on the launch path
    (1008, "ci", 1, 400, 5),       # the same in the column-interleaved layout
    (2016, "row", 0, 20, 3),       # the first launch already: the whole call on the launch path
]


def test_launch_without_all_blocks_resident_writes_nothing(ising):
    """A launch with several clusters whose blocks were not all resident at
    once (the test hook) writes nothing: the pieces before it stand, the rest
    of the call runs on the launch path, and every result equals the
    oracle's.  The automatic choice then keeps to one cluster (none fits
    L = 2016: the launch path) until ising_set_path."""
    got, jobs = [], []
    for L, layout, after, n, every in ABSENT_CASES:
        lay = ising.ISING_LAYOUT_ROW_PACKED if layout == "row" else ising.ISING_LAYOUT_COLUMN_INTERLEAVED
        with ising.Lattice(L, L + 3, layout=lay) as lat:
            lat.init_hot()
            lat.set_beta(0.43)
            assert lat.get_path() == ising.ISING_PATH_CLUSTER
            lat.inject_absent(after)
            E, M = lat.sweep_record(n, every)
            path_after = lat.get_path()
            lat.set_path(ising.ISING_PATH_AUTO)
            assert lat.get_path() == ising.ISING_PATH_CLUSTER
            E2, M2 = lat.sweep_record(6, 2)
            got.append((E, M, E2, M2, lat.get_spins(), path_after))
        jobs.append((L, L + 3, 0.43, True, n, every))
    ora = oracle.run_jobs(jobs)
    for (E, M, E2, M2, S, path_after), (Eo, Mo, So), case in zip(got, ora, ABSENT_CASES):
        L, layout, after, n, every = case
        np.testing.assert_array_equal(E, Eo, err_msg=str(case))
        np.testing.assert_array_equal(M, Mo, err_msg=str(case))
        s = So.copy()
        Eo2, Mo2 = oracle.run(s, L + 3, 0.43, n, 6, 2)
        np.testing.assert_array_equal(E2, Eo2, err_msg=str(case))
        np.testing.assert_array_equal(M2, Mo2, err_msg=str(case))
        np.testing.assert_array_equal(S, s, err_msg=str(case))
        assert path_after == (ising.ISING_PATH_LAUNCHES if L == 2016 else ising.ISING_PATH_CLUSTER), case


def test_launch_without_all_blocks_resident_inside_run_states(ising):
    """The same inside ising_run_states: the second state's first launch
    gives up, and its sweeps and records on the launch path land in that
    state's count slots."""
    L, seed, beta, sweeps, every = 1008, 31, 0.42, 180, 9     # one piece per state
    rng = np.random.default_rng(8)
    states = [np.where(rng.random((L, L)) < 0.3 + 0.3 * k, 1, -1).astype(np.int8) for k in range(2)]
    with ising.Lattice(L, seed) as lat:
        lat.set_beta(beta)
        assert lat.get_path() == ising.ISING_PATH_CLUSTER
        lat.inject_absent(1)                                  # the second state's launch
        E, M = lat.run_states(states, sweeps, every)
        S = lat.get_spins()
    for k, st in enumerate(states):
        s = st.copy()
        Eo, Mo = oracle.run(s, seed, beta, k * sweeps, sweeps, every)
        np.testing.assert_array_equal(E[k], Eo)
        np.testing.assert_array_equal(M[k], Mo)
    np.testing.assert_array_equal(S, s)


def test_cluster_continued_across_calls_and_paths(ising):
    """Plain sweeps, recorded sweeps, a switch to the graph replays and back:
    the sweep counter carries the draws across the calls and paths."""
    L, seed, beta = 400, 31, 0.42
    with ising.Lattice(L, seed) as lat:
        lat.init_hot()
        lat.set_beta(beta)
        assert lat.get_path() == ising.ISING_PATH_CLUSTER
        lat.sweep(5)
        E1, M1 = lat.sweep_record(7, 1)
        lat.set_path(ising.ISING_PATH_LAUNCHES)
        assert lat.get_path() == ising.ISING_PATH_LAUNCHES
        E2, M2 = lat.sweep_record(3, 1)
        lat.set_path(ising.ISING_PATH_AUTO)
        E3, M3 = lat.sweep_record(11, 2)
        S = lat.get_spins()
        assert lat.t == 26
    s = oracle.init_hot(L, seed)
    oracle.run(s, seed, beta, 0, 5, 5)
    for (E, M), (t0, n, every) in zip([(E1, M1), (E2, M2), (E3, M3)], [(5, 7, 1), (12, 3, 1), (15, 11, 2)]):
        Eo, Mo = oracle.run(s, seed, beta, t0, n, every)
        np.testing.assert_array_equal(E, Eo)
        np.testing.assert_array_equal(M, Mo)
    np.testing.assert_array_equal(S, s)


@pytest.mark.parametrize("beta,cold", [(0.0, False), (5.0, True), (0.6, True)])
def test_cluster_extremes(ising, beta, cold):
    """beta = 0 (every flip accepted: the always-accept masks), a frozen
    lattice (beta = 5 from all +1: nothing flips) and a cold start."""
    L, seed, n = 600, 5, 4
    with ising.Lattice(L, seed) as lat:
        if cold:
            lat.init_cold(1)
        else:
            lat.init_hot()
        lat.set_beta(beta)
        E, M = lat.sweep_record(n, 1)
        S = lat.get_spins()
    s = oracle.init_cold(L, 1) if cold else oracle.init_hot(L, seed)
    Eo, Mo = oracle.run(s, seed, beta, 0, n, 1)
    np.testing.assert_array_equal(E, Eo)
    np.testing.assert_array_equal(M, Mo)
    np.testing.assert_array_equal(S, s)
    if beta == 5.0:
        assert (S == 1).all() and (M == L * L).all()


def test_cluster_run_states(ising):
    """ising_run_states on the cluster path: each state continues the sweep
    counter, its records land in its own count slots."""
    L, seed, beta, sweeps, every = 340, 9, 0.41, 6, 2
    rng = np.random.default_rng(4)
    states = [np.where(rng.random((L, L)) < 0.2 + 0.2 * k, 1, -1).astype(np.int8) for k in range(3)]
    with ising.Lattice(L, seed) as lat:
        lat.set_beta(beta)
        assert lat.get_path() == ising.ISING_PATH_CLUSTER
        E, M = lat.run_states(states, sweeps, every)
        S = lat.get_spins()
    for k, st in enumerate(states):
        s = st.copy()
        Eo, Mo = oracle.run(s, seed, beta, k * sweeps, sweeps, every)
        np.testing.assert_array_equal(E[k], Eo)
        np.testing.assert_array_equal(M[k], Mo)
    np.testing.assert_array_equal(S, s)


def test_cluster_path_choice(ising):
    """Automatic choice by size; the forced path where no plan exists is
    rejected (too few rows per block; above the automatic range a share of
    rows too large for one cluster's shared memory) and leaves the path
    unchanged."""
    expect = {128: ising.ISING_PATH_RESIDENT, 130: ising.ISING_PATH_CLUSTER, 292: ising.ISING_PATH_CLUSTER,
              1176: ising.ISING_PATH_CLUSTER, 2016: ising.ISING_PATH_CLUSTER, 3000: ising.ISING_PATH_CLUSTER,
              3002: ising.ISING_PATH_LAUNCHES}
    for L, path in expect.items():
        with ising.Lattice(L, 1) as lat:
            assert lat.get_path() == path, L
    for L in (4, 8192):
        with ising.Lattice(L, 1) as lat:
            with pytest.raises(ising.IsingError):
                lat.set_path(ising.ISING_PATH_CLUSTER)
            assert lat.get_path() != ising.ISING_PATH_CLUSTER
    with ising.Lattice(8400, 1, layout=ising.ISING_LAYOUT_COLUMN_INTERLEAVED) as lat:
        with pytest.raises(ising.IsingError):
            lat.set_path(ising.ISING_PATH_CLUSTER)
        assert lat.get_path() == ising.ISING_PATH_LAUNCHES
    for L, path in ((1008, ising.ISING_PATH_CLUSTER), (2604, ising.ISING_PATH_CLUSTER),
                    (2688, ising.ISING_PATH_LAUNCHES)):
        with ising.Lattice(L, 1, layout=ising.ISING_LAYOUT_COLUMN_INTERLEAVED) as lat:
            assert lat.get_path() == path, L
    with ising.Lattice(1008, 1, layout=ising.ISING_LAYOUT_COLUMN_INTERLEAVED) as lat:
        lat.set_path(ising.ISING_PATH_LAUNCHES)
        assert lat.get_path() == ising.ISING_PATH_LAUNCHES
