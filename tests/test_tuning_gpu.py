"""Autotuner: every candidate must give bit-identical results (checked inside
the library); the chosen shape is valid and, applied, changes nothing."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ising():
    import paper_1811_04384_gb300 as p
    p.load()
    return p


@pytest.mark.parametrize("L", [64, 258, 1024])
def test_autotune_lattice_choice_is_valid_and_neutral(ising, L):
    from paper_1811_04384_gb300 import tuning
    best = tuning.tune_lattice(L, sweeps=4)
    assert best["path"] in (ising.ISING_PATH_LAUNCHES, ising.ISING_PATH_RESIDENT)
    assert best["ns_per_update"] > 0
    assert best["item_lanes"] in (0, 1, 2, 4, 8)
    if L > 740:
        assert best["path"] == ising.ISING_PATH_LAUNCHES
    table = {"device": tuning._device_name(), "lattice": {str(L): best}}
    with ising.Lattice(L, 17) as lat:
        assert tuning.apply(lat, table)
        lat.init_hot()
        lat.set_beta(0.44)
        E, M = lat.sweep_record(6, 2)
        spins = lat.get_spins()
    if L <= 258:
        s = oracle.init_hot(L, 17)
        Eo, Mo = oracle.run(s, 17, 0.44, 0, 6, 2)
        np.testing.assert_array_equal(E, Eo)
        np.testing.assert_array_equal(spins, s)


def test_autotune_batch_choice_is_valid(ising):
    from paper_1811_04384_gb300 import tuning
    best = tuning.tune_batch([32, 64, 256], [0.3, 0.44, 0.6], [1, 2, 3], [1, 1, 1], sweeps=5)
    assert best["threads_per_tile"] in (64, 128, 256)
    assert best["graph_chunk"] in (10, 50, 200)
    assert best["lanes"] in (1, 2, 4)
    assert best["ns_per_update"] > 0
