"""Batched replicas (uneven L, own beta/seed/start, own sweep counts) against
the single-lattice path and the oracle: every replica bit-exact."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ising():
    import paper_1811_04384_gb300 as p
    p.load()
    return p


def plain_run(ising, L, beta, seed, hot, n, every):
    with ising.Lattice(L, seed) as lat:
        if hot:
            lat.init_hot()
        lat.set_beta(beta)
        E, M = lat.sweep_record(n, every)
        return E, M, lat.get_spins()


def test_batch_matches_plain_and_oracle(ising):
    Ls = [4, 6, 10, 32, 42, 44, 64, 86, 128, 130, 256, 260]
    rng = np.random.default_rng(5)
    betas = rng.uniform(1 / 3.5, 1 / 1.5, len(Ls))
    seeds = rng.integers(0, 2**63, len(Ls), dtype=np.uint64)
    hot = [1, 0] * (len(Ls) // 2)
    sweeps = [7, 12, 3, 12, 9, 12, 12, 5, 12, 11, 12, 8]
    with ising.Batch(Ls, betas, seeds, hot) as b:
        E, M = b.sweep(sweeps, every=1)
        for r, L in enumerate(Ls):
            Ep, Mp, Sp = plain_run(ising, L, betas[r], int(seeds[r]), hot[r], sweeps[r], 1)
            np.testing.assert_array_equal(E[r], Ep)
            np.testing.assert_array_equal(M[r], Mp)
            np.testing.assert_array_equal(b.get_spins(r), Sp)
            assert b.t(r) == sweeps[r]
            if L <= 130:
                s = oracle.init_hot(L, int(seeds[r])) if hot[r] else oracle.init_cold(L, 1)
                Eo, Mo = oracle.run(s, int(seeds[r]), float(betas[r]), 0, sweeps[r], 1)
                np.testing.assert_array_equal(E[r], Eo)
                np.testing.assert_array_equal(b.get_spins(r), s)


@pytest.mark.parametrize("threads,chunk", [(64, 1), (128, 7), (256, 50), (128, 1024)])
def test_batch_tiling_and_chunk_do_not_change_results(ising, threads, chunk):
    Ls = [8, 64, 100, 258]
    betas = [0.3, 0.44, 0.5, 0.6]
    seeds = [1, 2, 3, 4]
    with ising.Batch(Ls, betas, seeds, [1, 1, 1, 1]) as ref, ising.Batch(Ls, betas, seeds, [1, 1, 1, 1]) as b:
        b.set_tiling(threads, chunk)
        E0, M0 = ref.sweep(23, every=2)
        E1, M1 = b.sweep(23, every=2)
        for r in range(4):
            np.testing.assert_array_equal(E0[r], E1[r])
            np.testing.assert_array_equal(M0[r], M1[r])
            np.testing.assert_array_equal(ref.get_spins(r), b.get_spins(r))


@pytest.mark.parametrize("lanes,threads", [(1, 128), (3, 64), (4, 256), (8, 128)])
def test_batch_lanes_do_not_change_results(ising, lanes, threads):
    """Splitting the replicas into independent graph branches (8 lanes for 5
    replicas leaves lanes empty) gives the same series and spins as one lane."""
    Ls = [8, 64, 100, 258, 46]
    betas = [0.3, 0.44, 0.5, 0.6, 0.2]
    seeds = [1, 2, 3, 4, 5]
    with ising.Batch(Ls, betas, seeds, [1] * 5) as ref, ising.Batch(Ls, betas, seeds, [1] * 5) as b:
        ref.set_lanes(1)
        b.set_tiling(threads, 7)
        b.set_lanes(lanes)
        E0, M0 = ref.sweep([23, 23, 17, 23, 5], every=1)
        E1, M1 = b.sweep([23, 23, 17, 23, 5], every=1)
        b.set_lanes(2)                       # re-split between calls: the chain continues
        E2, M2 = b.sweep([4, 4, 4, 4, 4], every=2)
        E3, M3 = ref.sweep([4, 4, 4, 4, 4], every=2)
        for r in range(5):
            np.testing.assert_array_equal(E0[r], E1[r])
            np.testing.assert_array_equal(M0[r], M1[r])
            np.testing.assert_array_equal(E2[r], E3[r])
            np.testing.assert_array_equal(M2[r], M3[r])
            np.testing.assert_array_equal(ref.get_spins(r), b.get_spins(r))


def test_batch_continues_across_calls(ising):
    Ls = [32, 64]
    with ising.Batch(Ls, [0.4, 0.45], [9, 10], [1, 1]) as b, ising.Batch(Ls, [0.4, 0.45], [9, 10], [1, 1]) as c:
        Ea, Ma = b.sweep([20, 20], every=4)
        Eb1, Mb1 = c.sweep([8, 12], every=4)
        Eb2, Mb2 = c.sweep([12, 8], every=4)
        for r in range(2):
            np.testing.assert_array_equal(Ea[r], np.concatenate([Eb1[r], Eb2[r]]))
            np.testing.assert_array_equal(b.get_spins(r), c.get_spins(r))


def test_batch_run_one_call(ising):
    Ls = [16, 48]
    E, M, S = ising.batch_run(Ls, [0.3, 0.5], [5, 6], [1, 0], [10, 6], every=2, final_spins=True)
    for r, L in enumerate(Ls):
        Ep, Mp, Sp = plain_run(ising, L, [0.3, 0.5][r], [5, 6][r], [1, 0][r], [10, 6][r], 2)
        np.testing.assert_array_equal(E[r], Ep)
        np.testing.assert_array_equal(M[r], Mp)
        np.testing.assert_array_equal(S[r], Sp)


def test_batch_rejects_bad_arguments(ising):
    with pytest.raises(ising.IsingError):
        ising.Batch([63], [0.4], [1])
    with pytest.raises(ising.IsingError):
        ising.Batch([64], [-0.1], [1])
    with ising.Batch([64], [0.4], [1]) as b:
        with pytest.raises(ising.IsingError):
            b.set_tiling(96, 10)
        for bad in (0, 9, -1):
            with pytest.raises(ising.IsingError):
                b.set_lanes(bad)
        with pytest.raises(ising.IsingError):
            b.sweep([-1])


def test_batched_configuration_at_full_size(ising):
    """All 512 replicas of the batched configuration (L on {32..2048}, T on
    [1.5, 3.5], seed 11), 8 sweeps with E/M every sweep: every replica equals
    its single-lattice run; replicas up to L = 128 also equal the oracle."""
    import bench
    Ls, betas, seeds = bench.batched_replicas()
    n = len(Ls)
    sweeps = 8
    with ising.Batch(Ls, betas, seeds, np.ones(n, dtype=np.uint8)) as b:
        E, M = b.sweep(sweeps, every=1)
        checked_oracle = 0
        for r in range(n):
            Ep, Mp, Sp = plain_run(ising, int(Ls[r]), float(betas[r]), int(seeds[r]), 1, sweeps, 1)
            np.testing.assert_array_equal(E[r], Ep)
            np.testing.assert_array_equal(M[r], Mp)
            if r % 16 == 0:
                np.testing.assert_array_equal(b.get_spins(r), Sp)
            if Ls[r] <= 128 and checked_oracle < 12:
                s = oracle.init_hot(int(Ls[r]), int(seeds[r]))
                Eo, Mo = oracle.run(s, int(seeds[r]), float(betas[r]), 0, sweeps, 1)
                np.testing.assert_array_equal(E[r], Eo)
                np.testing.assert_array_equal(M[r], Mo)
                checked_oracle += 1
        assert checked_oracle == 12
