"""GPU path vs oracle, element by element and bit-exact: spins (int8 per
site), int64 energy and magnetisation series, thresholds and Philox blocks.
Every case goes through the C ABI (libising.so) and the oracle (oracle.c)
on the same seeded inputs.

L classes covered (21 spins per word, L/2 sites per colour-row):
  4, 6        one word, 2-3 live fields (both wraps in one word)
  42          one full word
  44, 46      a partial last word of 1-2 fields
  10, 12, 34  rows not a multiple of 8, and L % 4 == 2 (a partial row group)
  64 .. 260   several words per row, several blocks, ragged tails
"""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

BETA_TC = 1.0 / 2.269
L_CLASSES = [4, 6, 8, 10, 12, 34, 42, 44, 46, 64, 84, 86, 126, 130, 258, 260]


@pytest.fixture(scope="module")
def ising():
    import paper_1811_04384_gb300 as p
    p.load()
    return p


def gpu_run(ising, L, seed, beta, n, every=1, hot=True, cold_spin=1, tiling=None):
    with ising.Lattice(L, seed) as lat:
        if tiling:
            lat.set_tiling(*tiling)
        if hot:
            lat.init_hot()
        else:
            lat.init_cold(cold_spin)
        lat.set_beta(beta)
        E, M = lat.sweep_record(n, every)
        return lat.get_spins(), E, M, lat.t


def oracle_run(L, seed, beta, n, every=1, hot=True, cold_spin=1):
    s = oracle.init_hot(L, seed) if hot else oracle.init_cold(L, cold_spin)
    E, M = oracle.run(s, seed, beta, 0, n, every)
    return s, E, M


# ----------------------------------------------------------------------------- primitives

def test_philox_blocks_match_oracle(ising):
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2**32, size=(4000, 4), dtype=np.uint64).astype(np.uint32)
    for seed in (0, 1, 0xDEADBEEFCAFEF00D):
        got = ising.philox_blocks(seed, ctr)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for k in range(0, len(ctr), 7):
            np.testing.assert_array_equal(got[k], oracle.philox4x32_10(ctr[k], key))


def test_philox_million_counters(ising):
    """10^6 counters with all four words varying, including the carry edges."""
    rng = np.random.default_rng(11)
    ctr = rng.integers(0, 2**32, size=(1_000_000, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0xFFFFFFFF] * 4, [0, 0, 0, 0], [0xFFFFFFFF, 0, 0xFFFFFFFF, 0], [1, 1, 1, 1]]
    for seed in (3, 0xFFFFFFFFFFFFFFFF):
        got = ising.philox_blocks(seed, ctr)
        ref = oracle.philox4x32_10_many(ctr, [seed & 0xFFFFFFFF, seed >> 32])
        np.testing.assert_array_equal(got, ref)


def test_thresholds_match_oracle(ising):
    betas = [0.0, 1e-300, 1e-17, 1e-16, 0.1, 0.25, BETA_TC, 0.5, 1.0, 2.0,
             32 * math.log(2) / 8 * (1 - 1e-12), 32 * math.log(2) / 8 * (1 + 1e-12),
             32 * math.log(2) / 4, 10.0, math.inf]
    betas += list(np.random.default_rng(2).uniform(0, 3, 200))
    with ising.Lattice(8, 1) as lat:
        for b in betas:
            lat.set_beta(b)
            assert lat.thresholds() == oracle.thresholds(b), b
        for bad in (-1.0, -1e-300, math.nan):
            with pytest.raises(ising.IsingError):
                lat.set_beta(bad)


@pytest.mark.parametrize("L", L_CLASSES + [1000, 1024, 1026])
def test_hot_start_matches_oracle(ising, L):
    with ising.Lattice(L, 1 + L) as lat:
        lat.init_hot()
        np.testing.assert_array_equal(lat.get_spins(), oracle.init_hot(L, 1 + L))
        s = oracle.init_hot(L, 1 + L)
        assert lat.energy() == oracle.energy(s)
        assert lat.magnetization() == oracle.magnetization(s)


@pytest.mark.parametrize("L", L_CLASSES)
def test_set_get_spins_and_observables(ising, L):
    rng = np.random.default_rng(L)
    s = np.where(rng.random((L, L)) < 0.4, 1, -1).astype(np.int8)
    with ising.Lattice(L, 3) as lat:
        lat.set_spins(s)
        np.testing.assert_array_equal(lat.get_spins(), s)
        assert lat.energy() == oracle.energy(s)
        assert lat.magnetization() == oracle.magnetization(s)
        # packed words round-trip and keep the dead fields and bit 63 zero
        w = lat.get_words()
        W, P, r = lat.layout()
        assert W == math.ceil(L / 2 / 21) and P == W + (W & 1) and r == L // 2 - 21 * (W - 1)
        live_last = sum(1 << (3 * k) for k in range(r))
        assert ((w[:, :, W - 1] & ~np.uint64(live_last)) == 0).all()
        assert ((w[:, :, W:] == 0)).all()
        assert ((w >> np.uint64(63)) == 0).all()
        lat.init_cold(-1)
        lat.set_words(w)
        np.testing.assert_array_equal(lat.get_spins(), s)


def test_cold_start(ising):
    for L in (4, 46, 64):
        with ising.Lattice(L, 0) as lat:
            assert lat.energy() == -2 * L * L and lat.magnetization() == L * L   # created cold +1
            lat.init_cold(-1)
            assert (lat.get_spins() == -1).all()
            assert lat.energy() == -2 * L * L and lat.magnetization() == -L * L


# ----------------------------------------------------------------------------- sweeps

@pytest.mark.parametrize("L", L_CLASSES)
def test_sweeps_match_oracle_every_l_class(ising, L):
    beta = [0.2, BETA_TC, 0.6, 1.0][L % 4]
    n = 12
    s_g, E_g, M_g, t = gpu_run(ising, L, 100 + L, beta, n)
    s_o, E_o, M_o = oracle_run(L, 100 + L, beta, n)
    np.testing.assert_array_equal(s_g, s_o)
    np.testing.assert_array_equal(E_g, E_o)
    np.testing.assert_array_equal(M_g, M_o)
    assert t == n


@pytest.mark.parametrize("beta", [0.0, 1e-18, 0.05, 0.3, BETA_TC, 0.7, 2.0, 3.0, 6.0, math.inf])
def test_sweeps_match_oracle_across_temperatures(ising, beta):
    L = 86
    s_g, E_g, M_g, _ = gpu_run(ising, L, 9, beta, 10)
    s_o, E_o, M_o = oracle_run(L, 9, beta, 10)
    np.testing.assert_array_equal(s_g, s_o)
    np.testing.assert_array_equal(E_g, E_o)
    np.testing.assert_array_equal(M_g, M_o)


def test_half_sweep_boundary_cases(ising):
    """One half-sweep at a time (via sweeps of a single colour pair) from the
    antiferromagnetic state: every colour-0 site has a = 4 and flips."""
    for L in (4, 6, 44, 130):
        ii, jj = np.indices((L, L))
        afm = np.where((ii + jj) % 2 == 0, 1, -1).astype(np.int8)
        with ising.Lattice(L, 5) as lat:
            lat.set_spins(afm)
            lat.set_beta(0.8)
            E, M = lat.sweep_record(1, 1)
            s = afm.copy()
            Eo, Mo = oracle.run(s, 5, 0.8, 0, 1, 1)
            np.testing.assert_array_equal(lat.get_spins(), s)
            assert E[0] == Eo[0] and M[0] == Mo[0]


@pytest.mark.parametrize("tiling", [(4, 16, 2), (4, 32, 1), (4, 64, 4), (4, 32, 8), (4, 16, 16), (4, 64, 1),
                                    (4, 0, 64), (4, 0, 128), (4, 0, 192), (4, 0, 256)])
def test_tiling_does_not_change_results(ising, tiling):
    """2-D block shapes and 1-D item grids (L = 260: 65 row groups x 7 words,
    455 items, so every 1-D block size leaves a ragged last block)."""
    L = 260
    ref = gpu_run(ising, L, 77, BETA_TC, 6, tiling=(4, 32, 4))
    got = gpu_run(ising, L, 77, BETA_TC, 6, tiling=tiling)
    for a, b in zip(ref[:3], got[:3]):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("L", [4, 44, 46, 130, 258, 1026])
@pytest.mark.parametrize("lanes", [2, 4, 8])
def test_item_lanes_do_not_change_results(ising, L, lanes):
    """Launch path with 2, 4 or 8 lanes per thread item (fields split over the
    lanes, accept bits merged by shuffles) against one thread per item, with
    records every sweep and a ragged last word / row group."""
    def go(F):
        with ising.Lattice(L, 21) as lat:
            lat.set_path(ising.ISING_PATH_LAUNCHES)
            lat.set_item_lanes(F)
            lat.init_hot()
            lat.set_beta(BETA_TC)
            E, M = lat.sweep_record(7, 1)
            return E, M, lat.get_spins()
    for a, b in zip(go(1), go(lanes)):
        np.testing.assert_array_equal(a, b)


def test_item_lanes_match_oracle(ising):
    L = 46
    with ising.Lattice(L, 8) as lat:
        lat.set_path(ising.ISING_PATH_LAUNCHES)
        lat.set_item_lanes(4)
        lat.init_hot()
        lat.set_beta(0.41)
        E, M = lat.sweep_record(9, 3)
        S = lat.get_spins()
    s = oracle.init_hot(L, 8)
    Eo, Mo = oracle.run(s, 8, 0.41, 0, 9, 3)
    np.testing.assert_array_equal(E, Eo)
    np.testing.assert_array_equal(M, Mo)
    np.testing.assert_array_equal(S, s)


def test_item_lanes_rejects_bad_values(ising):
    with ising.Lattice(64, 1) as lat:
        for bad in (3, 16, -1):
            with pytest.raises(ising.IsingError):
                lat.set_item_lanes(bad)


@pytest.mark.parametrize("L", [4, 46, 64, 1024, 1026])
def test_set_spins_from_pinned_host_memory(ising, L):
    """ising_set_spins reads pinned host memory directly in its pack kernel
    and copies pageable memory through a device buffer: both give the same
    words, the round trip returns the spins, and a chain continued from them
    equals the oracle (small L)."""
    import torch
    rng = np.random.default_rng(L)
    spins = np.where(rng.random((L, L)) < 0.4, 1, -1).astype(np.int8)
    pinned = torch.empty((L, L), dtype=torch.int8, pin_memory=True)
    pinned.numpy()[:] = spins
    with ising.Lattice(L, 5) as a, ising.Lattice(L, 5) as b:
        a.set_spins(spins)                   # pageable
        b.set_spins(pinned.numpy())          # pinned, read in place
        np.testing.assert_array_equal(a.get_words(), b.get_words())
        np.testing.assert_array_equal(b.get_spins(), spins)
        b.set_beta(0.45)
        E, M = b.sweep_record(3, 1)
    if L <= 64:
        s = spins.copy()
        Eo, Mo = oracle.run(s, 5, 0.45, 0, 3, 1)
        np.testing.assert_array_equal(E, Eo)
        np.testing.assert_array_equal(M, Mo)


@pytest.mark.parametrize("L,sweeps,every", [(46, 7, 2), (260, 6, 3), (1026, 4, 2), (260, 3, 5)])
def test_run_states_equals_calls_in_turn(ising, L, sweeps, every):
    """ising_run_states (copies of the next state overlapping the sweeps) gives
    the E/M series and final lattice of set_spins + sweep_record in turn, with
    pinned and pageable inputs; L = 46 takes the on-chip path, 260 and 1026
    the launch path; sweeps < every records nothing."""
    import torch
    rng = np.random.default_rng(L + sweeps)
    states = []
    for k in range(5):
        a = np.where(rng.random((L, L)) < 0.3 + 0.1 * k, 1, -1).astype(np.int8)
        if k % 2:
            p = torch.empty((L, L), dtype=torch.int8, pin_memory=True)
            p.numpy()[:] = a
            a = p.numpy()
        states.append(a)
    R = sweeps // every
    with ising.Lattice(L, 13) as ref:
        ref.set_beta(0.43)
        E0, M0 = [], []
        for a in states:
            ref.set_spins(a)
            E, M = ref.sweep_record(sweeps, every)
            E0.append(E)
            M0.append(M)
        S0, t0 = ref.get_spins(), ref.t
    with ising.Lattice(L, 13) as lat:
        lat.set_beta(0.43)
        E1, M1 = lat.run_states(states, sweeps, every)
        S1, t1 = lat.get_spins(), lat.t
    assert E1.shape == (5, R)
    for k in range(5):
        np.testing.assert_array_equal(E1[k], E0[k])
        np.testing.assert_array_equal(M1[k], M0[k])
    np.testing.assert_array_equal(S1, S0)
    assert t1 == t0 == 5 * sweeps


@pytest.mark.parametrize("L", [260, 516, 700])
def test_graph_replays_equal_on_chip_path(ising, L):
    """The launch path replays captured graphs for these sizes (32-sweep
    chunks; record chunks for every <= 64, with the record slot picked on the
    device): it equals the on-chip path, which launches no graphs, across
    record intervals on both sides of the graph limit, a re-capture after
    set_beta, and remainders."""
    def go(path):
        with ising.Lattice(L, 31) as lat:
            lat.set_path(path)
            lat.init_hot()
            lat.set_beta(0.42)
            out = [lat.sweep_record(70, 1), lat.sweep_record(70, 7), lat.sweep_record(130, 65)]
            lat.sweep(100)
            lat.set_beta(0.47)
            out.append(lat.sweep_record(66, 64))
            lat.sweep(33)
            return out, lat.get_spins(), lat.t
    a, sa, ta = go(ising.ISING_PATH_LAUNCHES)
    b, sb, tb = go(ising.ISING_PATH_RESIDENT)
    for (Ea, Ma), (Eb, Mb) in zip(a, b):
        np.testing.assert_array_equal(Ea, Eb)
        np.testing.assert_array_equal(Ma, Mb)
    np.testing.assert_array_equal(sa, sb)
    assert ta == tb == 70 + 70 + 130 + 100 + 66 + 33


@pytest.mark.parametrize("layout", ["row_packed", "column_interleaved"])
@pytest.mark.parametrize("beta", [0.0, 1e-18, BETA_TC, 6.0, math.inf])
def test_graphs_drawing_masks_first_at_threshold_limits(ising, beta, layout):
    """Graph replays, which draw the masks of 8 sweeps at a time one piece
    ahead and then apply them, at the threshold limits: 2^32 (beta = 0: every
    site flips), just below 2^32, 0 (beta >= 5.55: only dE <= 0 flips), in
    both word layouts.  70 sweeps span two 32-sweep graphs, the draw pieces
    and a plain remainder."""
    L, seed = (300, 12) if layout == "row_packed" else (336, 12)
    code = ising.ISING_LAYOUT_ROW_PACKED if layout == "row_packed" else ising.ISING_LAYOUT_COLUMN_INTERLEAVED
    with ising.Lattice(L, seed, layout=code) as lat:
        lat.set_path(ising.ISING_PATH_LAUNCHES)
        lat.init_hot()
        lat.set_beta(beta)
        E, M = lat.sweep_record(70, 1)
        lat.sweep(70)
        S = lat.get_spins()
    s = oracle.init_hot(L, seed)
    Eo, Mo = oracle.run(s, seed, beta, 0, 70, 1)
    oracle.run(s, seed, beta, 70, 70, 70)
    np.testing.assert_array_equal(E, Eo)
    np.testing.assert_array_equal(M, Mo)
    np.testing.assert_array_equal(S, s)


@pytest.mark.parametrize("L", [300, 1026])
def test_graphs_drawing_masks_first_keep_dead_fields_zero(ising, L):
    """Canary for the apply-only half-sweeps of the graphs: after graph
    replays at beta = 0 and at T_c the dead fields, bit 63 and the pitch
    padding of both colour arrays are still zero, and at beta = 0 every
    sweep negates every spin."""
    with ising.Lattice(L, 3) as lat:
        lat.set_path(ising.ISING_PATH_LAUNCHES)
        lat.init_hot()
        W, P, r = lat.layout()
        live_last = sum(1 << (3 * k) for k in range(r))
        s0 = lat.get_spins()
        lat.set_beta(0.0)
        E, M = lat.sweep_record(64, 1)
        assert (E == E[0]).all()
        assert (M[::2] == -M[1::2]).all() and M[1] == int(s0.sum())
        np.testing.assert_array_equal(lat.get_spins(), s0)
        for beta in (0.0, BETA_TC):
            lat.set_beta(beta)
            lat.sweep(64)
            w = lat.get_words()
            assert ((w[:, :, W - 1] & ~np.uint64(live_last)) == 0).all()
            assert ((w[:, :, :W - 1] & ~np.uint64(0x1249249249249249)) == 0).all()
            assert (w[:, :, W:] == 0).all()


@pytest.mark.parametrize("L", [2600, 4096])
def test_graphs_with_short_pieces_equal_fused_launches(ising, L):
    """Above 32,768 thread items a graph draws fewer sweeps per piece (6 at
    L = 2600, 2 at L = 4096, so that the mask buffers stay within 32 MB):
    64 recorded sweeps through graph replays equal the same sweeps run one
    call at a time, which use the fused half-sweeps (no graph)."""
    def go(graphs):
        with ising.Lattice(L, 17) as lat:
            lat.set_path(ising.ISING_PATH_LAUNCHES)
            lat.init_hot()
            lat.set_beta(0.43)
            if graphs:
                E, M = lat.sweep_record(64, 1)
            else:
                parts = [lat.sweep_record(1, 1) for _ in range(64)]
                E = np.concatenate([p[0] for p in parts])
                M = np.concatenate([p[1] for p in parts])
            return E, M, lat.get_spins(), lat.t
    a, b = go(True), go(False)
    for x, y in zip(a[:3], b[:3]):
        np.testing.assert_array_equal(x, y)
    assert a[3] == b[3] == 64


def test_graphs_with_short_pieces_match_oracle(ising):
    """The graph replays with short drawn pieces against the oracle:
    L = 2600 (6 sweeps per piece) with a record after each of 32 sweeps (one
    replay of the record graph, six pieces), L = 3000 (4 sweeps per piece)
    with a record every 2nd sweep (one replay of 16 records), and L = 2600
    through the no-record graph (32 sweeps) followed by 2 recorded sweeps:
    E/M at every record and the final spins."""
    seed, beta = 23, 0.43
    cases = [(2600, 32, 1, False), (3000, 32, 2, False), (2600, 34, 1, True)]
    got = []
    for L, n, every, plain_graph in cases:
        with ising.Lattice(L, seed) as lat:
            lat.set_path(ising.ISING_PATH_LAUNCHES)
            lat.init_hot()
            lat.set_beta(beta)
            if plain_graph:
                lat.sweep(32)
                E, M = lat.sweep_record(n - 32, every)
            else:
                E, M = lat.sweep_record(n, every)
            got.append((E, M, lat.get_spins()))
    ora = oracle.run_jobs([(L, seed, beta, True, n, every) for (L, n, every, _) in cases])
    for (E, M, S), (Eo, Mo, so), (L, n, every, plain_graph) in zip(got, ora, cases):
        if plain_graph:
            Eo, Mo = Eo[-len(E):], Mo[-len(M):]
        np.testing.assert_array_equal(E, Eo)
        np.testing.assert_array_equal(M, Mo)
        np.testing.assert_array_equal(S, so)


def test_graph_replays_match_oracle(ising):
    L, seed, beta = 1026, 6, 0.44
    with ising.Lattice(L, seed) as lat:
        lat.set_path(ising.ISING_PATH_LAUNCHES)
        lat.init_hot()
        lat.set_beta(beta)
        E, M = lat.sweep_record(40, 4)
        S = lat.get_spins()
    s = oracle.init_hot(L, seed)
    Eo, Mo = oracle.run(s, seed, beta, 0, 40, 4)
    np.testing.assert_array_equal(E, Eo)
    np.testing.assert_array_equal(M, Mo)
    np.testing.assert_array_equal(S, s)


def test_run_states_edge_cases(ising):
    """No states: nothing runs; NULL outputs; more records per state than one
    device chunk (the calls then run in turn); bad arguments rejected."""
    import ctypes
    L = 260
    st = np.where(np.random.default_rng(1).random((L, L)) < 0.5, 1, -1).astype(np.int8)
    with ising.Lattice(L, 4) as lat, ising.Lattice(L, 4) as ref:
        lat.set_beta(0.4)
        ref.set_beta(0.4)
        E, M = lat.run_states([], 10, 2)
        assert E.shape == (0, 5) and lat.t == 0
        lib = ising.load()
        ptrs = (ctypes.c_void_p * 2)(st.ctypes.data, st.ctypes.data)
        assert lib.ising_run_states(lat._h, ptrs, 2, 5, 1, None, None) == 0
        ref.set_spins(st)
        ref.sweep_record(5, 1)
        ref.set_spins(st)
        ref.sweep_record(5, 1)
        np.testing.assert_array_equal(lat.get_spins(), ref.get_spins())
        E1, M1 = lat.run_states([st], 1100, 1)            # 1100 records > 1024 per chunk
        ref.set_spins(st)
        E2, M2 = ref.sweep_record(1100, 1)
        np.testing.assert_array_equal(E1[0], E2)
        np.testing.assert_array_equal(M1[0], M2)
        null_states = (ctypes.c_void_p * 1)(None)
        assert lib.ising_run_states(lat._h, null_states, 1, 5, 1, None, None) == ising.ISING_EINVAL
        assert lib.ising_run_states(lat._h, ptrs, 1, 5, 0, None, None) == ising.ISING_EINVAL
        assert lib.ising_run_states(lat._h, ptrs, 1, -1, 1, None, None) == ising.ISING_EINVAL


def test_rejected_tilings(ising):
    with ising.Lattice(64, 1) as lat:
        for bad in [(8, 32, 4), (4, 48, 4), (4, 64, 8), (4, 16, 1), (4, 32, 3), (4, 0, 32), (4, 0, 96),
                    (4, 0, 512), (4, -16, 8)]:
            with pytest.raises(ising.IsingError):
                lat.set_tiling(*bad)


def test_recording_interval_and_remainder(ising):
    L = 64
    s1, E1, M1, t1 = gpu_run(ising, L, 4, 0.4, 23, every=1)
    s5, E5, M5, t5 = gpu_run(ising, L, 4, 0.4, 23, every=5)
    np.testing.assert_array_equal(E5, E1[4::5][:4])
    np.testing.assert_array_equal(M5, M1[4::5][:4])
    np.testing.assert_array_equal(s1, s5)
    assert t1 == t5 == 23


def test_resume_equals_uninterrupted(ising):
    L = 84
    with ising.Lattice(L, 12) as a, ising.Lattice(L, 12) as b:
        for lat in (a, b):
            lat.init_hot()
            lat.set_beta(0.41)
        Ea, Ma = a.sweep_record(30, 1)
        Eb1, Mb1 = b.sweep_record(10, 1)
        saved = b.get_words()
        t = b.t
        b.init_cold(1)
        b.set_words(saved)
        b.t = t
        Eb2, Mb2 = b.sweep_record(20, 1)
        np.testing.assert_array_equal(Ea, np.concatenate([Eb1, Eb2]))
        np.testing.assert_array_equal(Ma, np.concatenate([Mb1, Mb2]))
        np.testing.assert_array_equal(a.get_spins(), b.get_spins())


def test_high_word_of_sweep_counter(ising):
    L = 46
    t0 = (1 << 32) - 3
    with ising.Lattice(L, 21) as lat:
        lat.init_hot()
        lat.set_beta(0.35)
        lat.t = t0
        E, M = lat.sweep_record(6, 1)
        s = oracle.init_hot(L, 21)
        Eo, Mo = oracle.run(s, 21, 0.35, t0, 6, 1)
        np.testing.assert_array_equal(lat.get_spins(), s)
        np.testing.assert_array_equal(E, Eo)
        np.testing.assert_array_equal(M, Mo)


def test_plain_sweep_without_record_then_energy(ising):
    L = 130
    with ising.Lattice(L, 8) as lat:
        lat.init_hot()
        lat.set_beta(0.5)
        lat.sweep(7)
        s = oracle.init_hot(L, 8)
        oracle.run(s, 8, 0.5, 0, 7, 7)
        np.testing.assert_array_equal(lat.get_spins(), s)
        assert lat.energy() == oracle.energy(s)
        assert lat.magnetization() == oracle.magnetization(s)


def test_torch_owned_memory_and_stream(ising):
    torch = pytest.importorskip("torch")
    L = 64
    nbytes = ising.bytes_required(L)
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    with ising.Lattice(L, 31, buffer=buf, stream=stream) as lat:
        lat.init_hot()
        lat.set_beta(BETA_TC)
        E, M = lat.sweep_record(8, 2)
        s = oracle.init_hot(L, 31)
        Eo, Mo = oracle.run(s, 31, BETA_TC, 0, 8, 2)
        np.testing.assert_array_equal(E, Eo)
        np.testing.assert_array_equal(M, Mo)
        np.testing.assert_array_equal(lat.get_spins(), s)


# ----------------------------------------------------------------------------- configs

def test_config_plain_L64_1000_sweeps(ising):
    """L=64, T=2.269, hot start seed 1, 1000 sweeps, E and M every sweep."""
    s_g, E_g, M_g, _ = gpu_run(ising, 64, 1, BETA_TC, 1000)
    s_o, E_o, M_o = oracle_run(64, 1, BETA_TC, 1000)
    np.testing.assert_array_equal(E_g, E_o)
    np.testing.assert_array_equal(M_g, M_o)
    np.testing.assert_array_equal(s_g, s_o)
    assert ising.means(E_g, M_g, 64) == oracle.means(E_o, M_o, 64)


@pytest.mark.parametrize("T", [1.0, 2.3, 3.5])
def test_config_scan_L1024_sampled(ising, T):
    """L=1024 cold start seed 7: the first 20 sweeps at three of the scan's
    temperatures, full lattice and every-sweep series."""
    beta = 1.0 / T
    s_g, E_g, M_g, _ = gpu_run(ising, 1024, 7, beta, 20, hot=False)
    s_o, E_o, M_o = oracle_run(1024, 7, beta, 20, hot=False)
    np.testing.assert_array_equal(E_g, E_o)
    np.testing.assert_array_equal(M_g, M_o)
    np.testing.assert_array_equal(s_g, s_o)


def test_config_large_L16384_first_sweeps(ising):
    """L=16384 (the roofline configuration), hot start seed 3: the full lattice
    and E/M after the hot start and after each of two sweeps, at the bench's
    launch shape."""
    L = 16384
    with ising.Lattice(L, 3) as lat:
        lat.init_hot()
        lat.set_beta(BETA_TC)
        s = oracle.init_hot(L, 3)
        np.testing.assert_array_equal(lat.get_spins(), s)
        assert lat.energy() == oracle.energy(s)
        E, M = lat.sweep_record(2, 1)
        Eo, Mo = oracle.run(s, 3, BETA_TC, 0, 2, 1)
        np.testing.assert_array_equal(E, Eo)
        np.testing.assert_array_equal(M, Mo)
        np.testing.assert_array_equal(lat.get_spins(), s)


def test_config_large_L16384_run_states(ising):
    """The bench's end-to-end form at full size: ising_run_states with pinned
    int8 states of L = 16384 (the copy of state k+1 overlapping the sweeps of
    state k) equals set_spins + sweep_record in turn; the first state's first
    record also equals the oracle's."""
    import torch
    L = 16384
    with ising.Lattice(L, 3) as lat, ising.Lattice(L, 3) as ref:
        lat.init_hot()
        base = lat.get_spins()
        states = []
        for k in range(3):
            p = torch.empty((L, L), dtype=torch.int8, pin_memory=True)
            a = p.numpy()
            a[:] = base
            a[k::7, :] *= -1                      # a different state each time
            states.append(a)
        for x in (lat, ref):
            x.set_beta(BETA_TC)
        E1, M1 = lat.run_states(states, 4, 2)
        for k in range(3):
            ref.set_spins(states[k])
            E, M = ref.sweep_record(4, 2)
            np.testing.assert_array_equal(E1[k], E)
            np.testing.assert_array_equal(M1[k], M)
        np.testing.assert_array_equal(lat.get_spins(), ref.get_spins())
    s = states[0].copy()
    Eo, Mo = oracle.run(s, 3, BETA_TC, 0, 2, 2)
    assert E1[0][0] == Eo[0] and M1[0][0] == Mo[0]


def test_max_size_lattice(ising):
    """L = 32768 (the largest allowed): properties that hold at any size."""
    L = 32768
    with ising.Lattice(L, 2) as lat:
        assert lat.energy() == -2 * L * L and lat.magnetization() == L * L
        lat.set_beta(6.0)               # frozen: both thresholds are 0
        E, M = lat.sweep_record(2, 1)
        assert (E == -2 * L * L).all() and (M == L * L).all()
        lat.set_beta(0.0)               # every spin flips every sweep
        E, M = lat.sweep_record(3, 1)
        assert (E == -2 * L * L).all()
        assert list(M) == [-L * L, L * L, -L * L]


@pytest.mark.parametrize("L", [4, 44, 46, 86, 130, 258])
def test_sweeps_keep_dead_fields_and_padding_zero(ising, L):
    """Canary check: after many sweeps at beta = 0 (every live spin flips every
    sweep) and at T_c, the dead fields of the last word, bit 63 and the pitch
    padding are still zero in both colour arrays."""
    with ising.Lattice(L, 8) as lat:
        lat.init_hot()
        W, P, r = lat.layout()
        live_last = sum(1 << (3 * k) for k in range(r))
        for beta in (0.0, BETA_TC):
            lat.set_beta(beta)
            lat.sweep(25)
            w = lat.get_words()
            assert ((w[:, :, W - 1] & ~np.uint64(live_last)) == 0).all()
            assert ((w[:, :, :W - 1] & ~np.uint64(0x1249249249249249)) == 0).all()
            assert (w[:, :, W:] == 0).all()
