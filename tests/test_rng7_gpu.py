"""The opt-in 7-round Philox scheme: bit-exact with the oracle run with the
same scheme, on the launch and on-chip paths; it differs from the default."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ising():
    import paper_1811_04384_gb300 as p
    p.load()
    return p


@pytest.mark.parametrize("L", [6, 44, 64, 130, 258])
@pytest.mark.parametrize("path", [1, 2])
def test_seven_rounds_match_oracle(ising, L, path):
    beta = 0.42
    with ising.Lattice(L, 99) as lat:
        lat.set_rng(ising.ISING_RNG_PHILOX4X32_7)
        if path == 2 and L > 700:
            pytest.skip("does not fit on chip")
        lat.set_path(path)
        lat.init_hot()
        lat.set_beta(beta)
        E, M = lat.sweep_record(9, 3)
        spins = lat.get_spins()
    with oracle.sweep_rounds(7):
        s = oracle.init_hot(L, 99)
        Eo, Mo = oracle.run(s, 99, beta, 0, 9, 3)
    np.testing.assert_array_equal(E, Eo)
    np.testing.assert_array_equal(M, Mo)
    np.testing.assert_array_equal(spins, s)
    s10 = oracle.init_hot(L, 99)
    oracle.run(s10, 99, beta, 0, 9, 3)
    assert not np.array_equal(spins, s10)


@pytest.mark.parametrize("L", [64, 258])
def test_seven_rounds_through_graph_replays(ising, L):
    """Long enough for the launch path's replayed graphs (record chunks and
    32-sweep chunks) with the 7-round kernels and item lanes."""
    beta = 0.45
    with ising.Lattice(L, 7) as lat:
        lat.set_rng(ising.ISING_RNG_PHILOX4X32_7)
        lat.set_path(ising.ISING_PATH_LAUNCHES)
        lat.init_hot()
        lat.set_beta(beta)
        E, M = lat.sweep_record(66, 3)
        lat.sweep(40)
        spins = lat.get_spins()
    with oracle.sweep_rounds(7):
        s = oracle.init_hot(L, 7)
        Eo, Mo = oracle.run(s, 7, beta, 0, 66, 3)
        oracle.run(s, 7, beta, 66, 40, 40)
    np.testing.assert_array_equal(E, Eo)
    np.testing.assert_array_equal(M, Mo)
    np.testing.assert_array_equal(spins, s)


def test_rng_scheme_rejects_unknown(ising):
    with ising.Lattice(64, 1) as lat:
        with pytest.raises(ising.IsingError):
            lat.set_rng(5)


def test_seven_rounds_in_batches_and_served_jobs(ising):
    from paper_1811_04384_gb300 import serving
    Ls, betas, seeds = [32, 64, 130], [0.3, 0.44, 0.6], [4, 5, 6]
    with ising.Batch(Ls, betas, seeds, [1, 1, 1]) as b:
        b.set_rng(ising.ISING_RNG_PHILOX4X32_7)
        E, M = b.sweep(11, every=1)
        spins = [b.get_spins(r) for r in range(3)]
    reqs = [serving.Request(L, be, s, 11, 1, rng=ising.ISING_RNG_PHILOX4X32_7, want_spins=True)
            for L, be, s in zip(Ls, betas, seeds)]
    with serving.Server(64 << 20, max_jobs=4, epoch_sweeps=4) as srv:
        for r in reqs:
            srv.submit(r)
        for r in reqs:
            assert srv.wait(r.id).status == 0
    for r, (L, be, s) in enumerate(zip(Ls, betas, seeds)):
        with oracle.sweep_rounds(7):
            so = oracle.init_hot(L, s)
            Eo, Mo = oracle.run(so, s, be, 0, 11, 1)
        np.testing.assert_array_equal(E[r], Eo)
        np.testing.assert_array_equal(spins[r], so)
        np.testing.assert_array_equal(reqs[r].E, Eo)
        np.testing.assert_array_equal(reqs[r].spins, so)
