"""Pins of the oracle's random-word chain (the paper's own update scheme,
Sec. 4-5 and the Appendix A program): memory word (I, J) holds the spins
(I + kN, J); each phase updates 10 x (words of the half) randomly chosen
words of one half of every strip; each chosen word gets the Metropolis rule
on all its spins at once.  Pinned against exact enumeration (4 x 4 torus,
words of 1 and 2 spins), Kaufman's finite torus (L = 42, the paper's 21-spin
words), the acceptance rule, the two temperature limits, the word selection
re-derived here from the Philox blocks, and the order independence of the
strips of one phase."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import exact

BETA_TC = 1.0 / 2.269
HERE = os.path.dirname(os.path.abspath(__file__))


def load_exact():
    vals = {}
    for line in open(os.path.join(HERE, "golden", "exact_values.txt")):
        if line.startswith("#") or not line.strip():
            continue
        kind, L, beta, value = line.split()
        vals[(kind, L, float(beta))] = float(value)
    return vals


def visit_counts(L, F, nstrips, seed, t):
    """How often each word (I, J) is chosen in iteration t, re-derived from
    the Philox4x32-10 blocks and the selection rule: update s of strip q in
    phase p uses block 0 of counter (s, 8q, lo32(t), 2^31 | hi32(t) << 1 | p);
    row = floor(w0 N / 2^32), column = half-strip start + floor(w1 h / 2^32),
    10 N h updates per half strip."""
    N, NC = L // F, L // nstrips
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    count = np.zeros((N, L), dtype=np.int64)
    for p in (0, 1):
        h = NC // 2 if p == 0 else NC - NC // 2
        for q in range(nstrips):
            col0 = q * NC + (0 if p == 0 else NC // 2)
            n = 10 * N * h
            ctr = np.zeros((n, 4), dtype=np.uint32)
            ctr[:, 0] = np.arange(n)
            ctr[:, 1] = 8 * q
            ctr[:, 2] = t & 0xFFFFFFFF
            ctr[:, 3] = 0x80000000 | ((t >> 32) << 1) | p
            w = oracle.philox4x32_10_many(ctr, key).astype(np.uint64)
            I = (w[:, 0] * np.uint64(N)) >> np.uint64(32)
            J = col0 + ((w[:, 1] * np.uint64(h)) >> np.uint64(32))
            np.add.at(count, (I.astype(np.int64), J.astype(np.int64)), 1)
    return count


@pytest.mark.parametrize("L,F,nstrips", [(42, 21, 1), (42, 21, 3), (42, 21, 14), (84, 21, 6), (12, 2, 2)])
def test_infinite_temperature_negates_each_visited_word(L, F, nstrips):
    """beta = 0: every spin of a chosen word flips, so after one iteration a
    spin is negated iff its word was chosen an odd number of times."""
    N = L // F
    seed, t = 0x1234_5678_9ABC, 7
    s0 = oracle.init_hot(L, 5)
    s = s0.copy()
    oracle.rw_iteration(s, seed, t, 0.0, nstrips, F=F)
    count = visit_counts(L, F, nstrips, seed, t)
    assert count.sum() == 10 * L * N
    sign = np.where(count % 2 == 1, -1, 1)
    expected = s0 * np.tile(sign, (F, 1)).astype(np.int8)   # site (I + kN, J) belongs to word (I, J)
    np.testing.assert_array_equal(s, expected)


def test_select_matches_rederived_rule():
    L, F, nstrips, seed, t = 84, 21, 6, 99, 3
    N, NC = L // F, L // nstrips
    for p in (0, 1):
        h = NC // 2 if p == 0 else NC - NC // 2
        for q in (0, 5):
            col0 = q * NC + (0 if p == 0 else NC // 2)
            for step in (0, 1, 17, 10 * N * h - 1):
                w = oracle.philox4x32_10([step, 8 * q, t, 0x80000000 | p], [seed, 0])
                assert oracle.rw_select(seed, t, p, q, step, N, col0, h) == (
                    int(w[0]) * N >> 32, col0 + (int(w[1]) * h >> 32))


def test_frozen_ground_state():
    """beta >= 32 ln2 / 4: no uphill flip is accepted, and in a ground state
    every spin has a = 0."""
    for spin in (1, -1):
        s = oracle.init_cold(42, spin)
        E, M = oracle.rw_run(s, 3, 6.0, 0, 4, nstrips=3)
        assert (E == -2 * 42 * 42).all() and (M == spin * 42 * 42).all()


def test_proposals_per_iteration_and_acceptance():
    """Each iteration proposes 10 flips per spin on average (Table 2): 10 L^2
    proposals, including strips with an odd column count (L = 42 in 14
    strips of 3 columns: 1 + 2 per phase pair).  A proposal with a >= 2
    always flips; one with a in {0, 1} flips with frequency thr[a] / 2^32."""
    L, beta = 42, 0.3
    stats = np.zeros(10, dtype=np.int64)
    s = oracle.init_hot(L, 8)
    oracle.rw_run(s, 8, beta, 0, 1, nstrips=14, stats=stats)
    assert stats[:5].sum() == 10 * L * L
    for nstrips in (1, 2, 3):
        oracle.rw_run(s, 8, beta, 1, 60, nstrips=nstrips, stats=stats)
    assert stats[:5].sum() == 181 * 10 * L * L
    t0, t1 = oracle.thresholds(beta)
    for a, thr in ((0, t0), (1, t1)):
        n, k = stats[a], stats[5 + a]
        p = thr / 2**32
        assert n > 10000
        assert abs(k / n - p) < 5 * math.sqrt(p * (1 - p) / n)
    for a in (2, 3, 4):
        assert stats[5 + a] == stats[a]


def test_strip_order_does_not_change_the_result():
    """The strips of one phase update non-neighbouring words: running them in
    reverse order gives the same lattice (the paper's processes run
    concurrently)."""
    for L, nstrips in ((84, 6), (84, 42), (168, 4)):
        a = oracle.init_hot(L, 21)
        b = a.copy()
        for t in (1, 2, 3):
            oracle.rw_iteration(a, 77, t, 0.44, nstrips)
            oracle.rw_iteration(b, 77, t, 0.44, nstrips, reverse=True)
        np.testing.assert_array_equal(a, b)
        assert not np.array_equal(a, oracle.init_hot(L, 21))


@pytest.mark.parametrize("F,nstrips,beta", [(1, 2, BETA_TC), (2, 1, BETA_TC), (2, 2, 0.7), (1, 1, 0.2)])
def test_4x4_random_word_chain_matches_exact_enumeration(F, nstrips, beta):
    """The chain's law on the 4 x 4 torus, with words of 1 spin (N = 4) and of
    2 spins (N = 2): the Boltzmann means of the exact enumeration."""
    vals = load_exact()
    e_ex = vals[("enum_e_per_spin", "4", beta)]
    m_ex = vals[("enum_absm_per_spin", "4", beta)]
    s = oracle.init_hot(4, 31)
    oracle.rw_run(s, 31, beta, 0, 200, nstrips, F=F)
    E, M = oracle.rw_run(s, 31, beta, 200, 40000, nstrips, F=F)
    e, de = exact.binned_error(E / 16.0, 50)
    m, dm = exact.binned_error(np.abs(M) / 16.0, 50)
    assert abs(e - e_ex) < 4.5 * de, (e, e_ex, de)
    assert abs(m - m_ex) < 4.5 * dm, (m, m_ex, dm)


@pytest.mark.parametrize("beta,nstrips", [(0.3, 1), (0.6, 3), (BETA_TC, 14)])
def test_paper_words_match_kaufman_L42(beta, nstrips):
    """The paper's 21-spin words (L = 42, N = 2): the mean energy per spin
    against Kaufman's exact partition function of the 42 x 42 torus."""
    vals = load_exact()
    e_ex = vals[("kaufman_e_per_spin", "42", beta)]
    s = oracle.init_hot(42, 13)
    oracle.rw_run(s, 13, beta, 0, 300, nstrips)
    E, _ = oracle.rw_run(s, 13, beta, 300, 4000, nstrips)
    e, de = exact.binned_error(E / (42 * 42), 40)
    assert abs(e - e_ex) < 4.5 * de, (e, e_ex, de)


def test_one_word_update_follows_its_draws():
    """One update re-derived from its six Philox blocks: the chosen word
    (block 0, words 0 and 1), then for its spin k (site (I + kN, J)) the
    number a of anti-aligned neighbours counted here on the torus, and the
    flip rule of Sec. 2 / Table 1 with draw word 2 + k of the 24."""
    rng = np.random.default_rng(4)
    L, F = 84, 21
    N = L // F
    seed, t, phase, strip, col0, h = 0xC0FFEE, 5, 1, 2, 49, 7
    thr0, thr1 = 1 << 30, 3 << 30        # 1/4 and 3/4: both outcomes occur
    for step in range(40):
        s = np.where(rng.random((L, L)) < 0.5, 1, -1).astype(np.int8)
        before = s.copy()
        oracle.rw_step(s, seed, t, phase, strip, step, col0, h, thr0, thr1, F=F)
        ctr = np.array([[step, 8 * strip + b, t, 0x80000000 | phase] for b in range(6)], dtype=np.uint32)
        w = oracle.philox4x32_10_many(ctr, [seed & 0xFFFFFFFF, seed >> 32]).reshape(-1)
        I = int(w[0]) * N >> 32
        J = col0 + (int(w[1]) * h >> 32)
        expected = before.copy()
        for k in range(F):
            i = I + k * N
            me = before[i, J]
            nb = [before[(i - 1) % L, J], before[(i + 1) % L, J], before[i, (J - 1) % L], before[i, (J + 1) % L]]
            a = sum(1 for v in nb if v != me)
            if a >= 2 or int(w[2 + k]) < (thr0, thr1)[a]:
                expected[i, J] = -me
        np.testing.assert_array_equal(s, expected)
