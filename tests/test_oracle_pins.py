"""Pins of the oracle (CPU only) to facts fixed by the paper or by the
mathematics, chosen so that a dropped term, a wrong sign or index, or a
transposed operand in oracle.c fails at least one of them.

Pins by part:
- Philox: the 64-bit member, written with the same round structure as the
  32-bit one, equals numpy's independent Philox4x64-10; the 32-bit member is a
  bijection of the counter with uniform output.
- Thresholds: limits (beta = 0, large beta) and exp(-8b) = exp(-4b)^2.
- Group value and dE: Table 1 of the paper, exhaustively over the 32 local
  configurations, and against the change of the total energy of Eq. 1.
- Energy and magnetisation: closed forms of structured configurations.
- Chain: exact enumeration of the 4x4 torus, Kaufman's finite torus, Onsager
  and Yang, acceptance frequencies, and exact invariants of the dynamics.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import exact

BETA_TC = 1.0 / 2.269


def load_exact(golden_dir):
    vals = {}
    with open(os.path.join(golden_dir, "exact_values.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            kind, L, beta, value = line.split()
            vals[(kind, L, float(beta))] = float(value)
    return vals


# ----------------------------------------------------------------------------- Philox

def test_philox4x64_matches_numpy():
    rng = np.random.default_rng(12345)
    for _ in range(200):
        key = rng.integers(0, 2**64, size=2, dtype=np.uint64)
        ctr = rng.integers(0, 2**64, size=4, dtype=np.uint64)
        # numpy's Philox increments its counter before producing a block.
        bg = np.random.Philox(key=key, counter=ctr.copy())
        ref = bg.random_raw(4)
        c1 = ctr.copy()
        c1[0] = np.uint64((int(c1[0]) + 1) % 2**64)
        if int(ctr[0]) == 2**64 - 1:
            continue  # carry into ctr[1]; not this test's concern
        got = oracle.philox4x64_10(c1, key)
        np.testing.assert_array_equal(got, ref)


def test_philox4x32_is_a_keyed_bijection_with_uniform_output():
    rng = np.random.default_rng(7)
    key = [0x12345678, 0x9ABCDEF0]
    outs = set()
    top = np.zeros(16, dtype=np.int64)
    n = 20000
    for k in range(n):
        ctr = [k & 0xFFFF, k >> 16, 3, 5]
        o = oracle.philox4x32_10(ctr, key)
        outs.add(tuple(int(x) for x in o))
        for x in o:
            top[int(x) >> 28] += 1
    assert len(outs) == n  # distinct counters -> distinct blocks
    expected = 4 * n / 16
    chi2 = float(((top - expected) ** 2 / expected).sum())
    assert chi2 < 45.0  # 15 dof: P(chi2 > 45) ~ 1e-4
    # The key matters and every output word depends on every counter word.
    base = oracle.philox4x32_10([1, 2, 3, 4], key)
    assert not np.array_equal(base, oracle.philox4x32_10([1, 2, 3, 4], [key[0] ^ 1, key[1]]))
    for w in range(4):
        c = [1, 2, 3, 4]
        c[w] ^= 1
        diff = oracle.philox4x32_10(c, key) ^ base
        assert all(int(d) != 0 for d in diff)
    del rng


def test_site_draw_keying():
    # (i>>2, j>>1, c, i&3) is a bijection of the sites: all draws of one sweep
    # differ (with overwhelming probability) and change with t and seed.
    L = 16
    d = {(i, j): oracle.site_draw(5, 3, i, j) for i in range(L) for j in range(L)}
    assert len(set(d.values())) == L * L
    assert oracle.site_draw(5, 4, 2, 3) != d[(2, 3)]
    assert oracle.site_draw(6, 3, 2, 3) != d[(2, 3)]
    # the high word of t enters the counter
    assert oracle.site_draw(5, 3 + (1 << 32), 2, 3) != d[(2, 3)]
    # one Philox call serves the four rows 4g..4g+3 at one column pair
    i, j = 4, 6
    c = (i + j) & 1
    block = oracle.philox4x32_10([i >> 2, j >> 1, 3, c], [5, 0])
    for rr in range(4):
        jj = j if ((i + rr + j) & 1) == c else j + 1
        assert oracle.site_draw(5, 3, i + rr, jj) == int(block[rr])


# ----------------------------------------------------------------------------- thresholds

def test_threshold_limits_and_identity():
    assert oracle.thresholds(0.0) == (2**32, 2**32)
    assert oracle.thresholds(100.0) == (0, 0)
    # thr0 = 0 exactly when 2^32 exp(-8b) < 1, i.e. b > 32 ln2 / 8
    b0 = 32 * math.log(2) / 8
    assert oracle.thresholds(b0 * 1.001)[0] == 0
    assert oracle.thresholds(b0 * 0.999)[0] == 1
    b1 = 32 * math.log(2) / 4
    assert oracle.thresholds(b1 * 1.001) == (0, 0)
    assert oracle.thresholds(b1 * 0.999)[1] == 1
    prev = (2**32 + 1, 2**32 + 1)
    for b in np.linspace(0.0, 3.0, 61):
        t0, t1 = oracle.thresholds(float(b))
        assert t0 <= t1 <= 2**32
        assert t0 <= prev[0] and t1 <= prev[1]
        # exp(-8b) = exp(-4b)^2, so thr0 ~ thr1^2 / 2^32 up to the two floors
        assert abs(t0 - t1 * t1 / 2**32) <= 2.0
        prev = (t0, t1)
    # at T = 2.269 (a regression value of the closed form)
    assert oracle.thresholds(BETA_TC) == (126395633, 736793806)


# ----------------------------------------------------------------------------- Table 1

def _star(me, nb):
    """A 5x5 torus with spin `me` at (2,2) and neighbours nb = (up, down, left,
    right); every other spin is +1."""
    s = np.ones((5, 5), dtype=np.int8)
    s[2, 2] = me
    s[1, 2], s[3, 2], s[2, 1], s[2, 3] = nb
    return s


def test_table1_rows(golden_dir):
    rows = np.loadtxt(os.path.join(golden_dir, "table1.txt"), comments="#", dtype=np.int64)
    assert rows.shape == (10, 7)
    for cfg, me, n_up, E_b, E_a, dE, group in rows:
        nb = tuple([1] * n_up + [-1] * (4 - n_up))
        s = _star(me, nb)
        assert oracle.group_value(s, 2, 2) == group, cfg
        assert oracle.delta_energy(s, 2, 2) == dE, cfg
        # E and E' of the table are the selected spin's four bonds
        assert -me * sum(nb) == E_b and me * sum(nb) == E_a


def test_group_value_and_delta_exhaustive():
    """All 2^5 local configurations: dE = 8 - 4a (Table 1), and dE equals the
    change of the total energy of Eq. 1 when the spin is flipped."""
    for bits in range(32):
        vals = [1 if (bits >> k) & 1 else -1 for k in range(5)]
        s = _star(vals[0], tuple(vals[1:]))
        a = oracle.group_value(s, 2, 2)
        assert a == sum(1 for v in vals[1:] if v != vals[0])
        dE = oracle.delta_energy(s, 2, 2)
        assert dE == 8 - 4 * a
        E0 = oracle.energy(s)
        s2 = s.copy()
        s2[2, 2] = -s2[2, 2]
        assert oracle.energy(s2) - E0 == dE


# ----------------------------------------------------------------------------- E and M

@pytest.mark.parametrize("L", [4, 6, 10, 64])
def test_energy_closed_forms(L):
    up = np.ones((L, L), dtype=np.int8)
    assert oracle.energy(up) == -2 * L * L and oracle.magnetization(up) == L * L
    assert oracle.energy(-up) == -2 * L * L and oracle.magnetization(-up) == -L * L
    ii, jj = np.indices((L, L))
    afm = np.where((ii + jj) % 2 == 0, 1, -1).astype(np.int8)
    assert oracle.energy(afm) == 2 * L * L and oracle.magnetization(afm) == 0
    # vertical stripes of width 1: horizontal bonds anti, vertical aligned
    stripes = np.where(jj % 2 == 0, 1, -1).astype(np.int8)
    assert oracle.energy(stripes) == 0
    # two domains (top half up): 2 interfaces of L bonds each
    dom = np.where(ii < L // 2, 1, -1).astype(np.int8)
    assert oracle.energy(dom) == -2 * L * L + 4 * L
    # one flipped spin in the ground state: 4 broken bonds
    one = up.copy()
    one[1, 2] = -1
    assert oracle.energy(one) == -2 * L * L + 8
    assert oracle.magnetization(one) == L * L - 2
    # a single down column next to a single down row (corner shared)
    cr = up.copy()
    cr[:, 0] = -1
    cr[0, :] = -1
    assert oracle.energy(cr) == -2 * L * L + 2 * (2 * L + 2 * L - 4)


def test_energy_counts_every_bond_once():
    # random lattice: E = (#anti) - (#aligned) over the 2L^2 bonds, counted here
    # through the group values: sum_sites a = 2 * #anti.
    rng = np.random.default_rng(3)
    for L in (4, 6, 8):
        s = np.where(rng.random((L, L)) < 0.5, 1, -1).astype(np.int8)
        anti2 = sum(oracle.group_value(s, i, j) for i in range(L) for j in range(L))
        assert anti2 % 2 == 0
        anti = anti2 // 2
        assert oracle.energy(s) == anti - (2 * L * L - anti)
        assert oracle.magnetization(s) == int(s.astype(np.int64).sum())


# ----------------------------------------------------------------------------- init

def test_hot_start():
    L = 64
    s = oracle.init_hot(L, 1)
    assert set(np.unique(s)) <= {-1, 1}
    frac = (s == 1).mean()
    assert abs(frac - 0.5) < 4 * 0.5 / L  # 4 sigma
    assert not np.array_equal(s, oracle.init_hot(L, 2))
    np.testing.assert_array_equal(s, oracle.init_hot(L, 1))
    draws = np.array([[oracle.site_draw(1, 0, i, j) for j in range(L)] for i in range(L)])
    np.testing.assert_array_equal(s, np.where(draws < 2**31, 1, -1))
    big = oracle.init_hot(512, 17)
    assert abs((big == 1).mean() - 0.5) < 4 * 0.5 / 512
    c = oracle.init_cold(L, -1)
    assert (c == -1).all()


# ----------------------------------------------------------------------------- invariants

def test_ground_state_is_frozen_at_low_temperature():
    L = 8
    s = oracle.init_cold(L, 1)
    E, M = oracle.run(s, seed=9, beta=5.6, t0=0, n=50)
    assert (E == -2 * L * L).all() and (M == L * L).all()


@pytest.mark.parametrize("L", [4, 6, 8])
def test_infinite_temperature_negates_every_spin(L):
    s0 = oracle.init_hot(L, 4)
    s = s0.copy()
    E0, M0 = oracle.energy(s0), oracle.magnetization(s0)
    E, M = oracle.run(s, seed=4, beta=0.0, t0=0, n=7)
    assert (E == E0).all()
    np.testing.assert_array_equal(M, [M0 * (-1) ** t for t in range(1, 8)])
    np.testing.assert_array_equal(s, -s0)


def test_global_flip_symmetry():
    L = 10
    s = oracle.init_hot(L, 11)
    m = -s
    E1, M1 = oracle.run(s, seed=2, beta=0.35, t0=0, n=40)
    E2, M2 = oracle.run(m, seed=2, beta=0.35, t0=0, n=40)
    np.testing.assert_array_equal(E1, E2)
    np.testing.assert_array_equal(M1, -M2)
    np.testing.assert_array_equal(s, -m)


def test_incremental_bookkeeping_matches_recompute():
    L = 12
    s = oracle.init_hot(L, 21)
    beta = 0.42
    for t in range(1, 6):
        for c in (0, 1):
            before = s.copy()
            a = np.array([[oracle.group_value(before, i, j) for j in range(L)] for i in range(L)])
            E_b, M_b = oracle.energy(before), oracle.magnetization(before)
            oracle.half_sweep(s, seed=21, t=t, c=c, beta=beta)
            flipped = s != before
            ii, jj = np.indices((L, L))
            assert not (flipped & (((ii + jj) & 1) != c)).any()   # only colour c moves
            assert (flipped[(a >= 2) & (((ii + jj) & 1) == c)]).all()  # downhill always
            assert oracle.energy(s) - E_b == int((8 - 4 * a[flipped]).sum())
            assert oracle.magnetization(s) - M_b == int((-2 * before[flipped].astype(np.int64)).sum())


def test_antiferromagnet_half_sweep_flips_all_of_colour_zero():
    L = 8
    ii, jj = np.indices((L, L))
    afm = np.where((ii + jj) % 2 == 0, 1, -1).astype(np.int8)
    s = afm.copy()
    oracle.half_sweep(s, seed=1, t=1, c=0, beta=2.0)
    assert (s == -1).all()  # colour 0 all flipped (a = 4) -> all down


def test_resume_equals_uninterrupted_run():
    L = 12
    a = oracle.init_hot(L, 8)
    b = a.copy()
    Ea, Ma = oracle.run(a, seed=8, beta=0.44, t0=0, n=30, every=3)
    Eb1, Mb1 = oracle.run(b, seed=8, beta=0.44, t0=0, n=12, every=3)
    Eb2, Mb2 = oracle.run(b, seed=8, beta=0.44, t0=12, n=18, every=3)
    np.testing.assert_array_equal(Ea, np.concatenate([Eb1, Eb2]))
    np.testing.assert_array_equal(Ma, np.concatenate([Mb1, Mb2]))
    np.testing.assert_array_equal(a, b)


def test_recording_interval():
    L = 6
    a = oracle.init_hot(L, 3)
    b = a.copy()
    E1, M1 = oracle.run(a, seed=3, beta=0.3, t0=0, n=20, every=1)
    E5, M5 = oracle.run(b, seed=3, beta=0.3, t0=0, n=20, every=5)
    np.testing.assert_array_equal(E5, E1[4::5])
    np.testing.assert_array_equal(M5, M1[4::5])
    assert oracle.energy(a) == E1[-1] and oracle.magnetization(a) == M1[-1]


def test_flip_set_is_the_site_draw_below_threshold():
    """Sec. 2 step 3 with integer thresholds: an uphill site flips exactly when
    its own draw at this sweep, r(seed, t, i, j), is below thr[a]."""
    L = 8
    seed, t = 31, 6
    thr0, thr1 = 2**31, 3 * 2**30
    for c in (0, 1):
        s = oracle.init_cold(L, 1)          # every site has a = 0
        oracle.half_sweep_thr(s, seed, t, c, thr0, thr1)
        for i in range(L):
            for j in range(L):
                want = ((i + j) & 1) == c and oracle.site_draw(seed, t, i, j) < thr0
                assert (s[i, j] == -1) == want, (c, i, j)
    # a = 1 sites use thr[1]: one down spin in colour 1 gives its four colour-0
    # neighbours a = 1
    s = oracle.init_cold(L, 1)
    s[3, 2] = -1
    oracle.half_sweep_thr(s, seed, t, 0, 0, thr1)
    for (i, j) in [(2, 2), (4, 2), (3, 1), (3, 3)]:
        assert (s[i, j] == -1) == (oracle.site_draw(seed, t, i, j) < thr1)
    assert (s[(np.indices((L, L)).sum(0) % 2 == 0)] == -1).sum() <= 4


def test_run_numbers_sweeps_from_t0_plus_one():
    """Sweep t = colour-0 half-sweep then colour-1 half-sweep, both with the
    draws of sweep t; run() starting at t0 performs sweeps t0+1, t0+2, ..."""
    L = 8
    beta = 0.5
    thr0, thr1 = oracle.thresholds(beta)
    a = oracle.init_hot(L, 40)
    b = a.copy()
    oracle.run(a, seed=40, beta=beta, t0=4, n=2)
    for t in (5, 6):
        oracle.half_sweep_thr(b, 40, t, 0, thr0, thr1)
        oracle.half_sweep_thr(b, 40, t, 1, thr0, thr1)
    np.testing.assert_array_equal(a, b)


def test_strict_threshold_boundary():
    """P(accept) = thr / 2^32 for a uniform 32-bit draw needs a strict r < thr:
    a draw equal to the threshold is rejected, one below it accepted, and a
    zero threshold never accepts."""
    L = 8
    seed, t = 12, 3
    i, j = 2, 4                            # colour 0
    r = oracle.site_draw(seed, t, i, j)
    for thr, flips in ((r, False), (r + 1, True), (0, False)):
        s = oracle.init_cold(L, 1)
        oracle.half_sweep_thr(s, seed, t, 0, thr, thr)
        assert (s[i, j] == -1) == flips, thr


# ----------------------------------------------------------------------------- chain law

def test_acceptance_frequencies_match_thresholds():
    L = 32
    s = oracle.init_hot(L, 5)
    beta = 0.3
    t0, t1 = oracle.thresholds(beta)
    stats = np.zeros(10, dtype=np.int64)
    for t in range(1, 201):
        oracle.sweep(s, seed=5, t=t, beta=beta, stats=stats)
    for a, thr in ((0, t0), (1, t1)):
        n, k = stats[a], stats[5 + a]
        p = thr / 2**32
        assert n > 1000
        assert abs(k / n - p) < 5 * math.sqrt(p * (1 - p) / n)
    for a in (2, 3, 4):
        assert stats[5 + a] == stats[a]


@pytest.mark.parametrize("beta", [0.2, BETA_TC, 0.7])
def test_4x4_chain_matches_exact_enumeration(beta, golden_dir):
    vals = load_exact(golden_dir)
    e_ex = vals[("enum_e_per_spin", "4", beta)]
    m_ex = vals[("enum_absm_per_spin", "4", beta)]
    s = oracle.init_hot(4, 77)
    oracle.run(s, seed=77, beta=beta, t0=0, n=1000)
    E, M = oracle.run(s, seed=77, beta=beta, t0=1000, n=200000)
    e, de = exact.binned_error(E / 16.0, 50)
    m, dm = exact.binned_error(np.abs(M) / 16.0, 50)
    assert abs(e - e_ex) < 4.5 * de, (e, e_ex, de)
    assert abs(m - m_ex) < 4.5 * dm, (m, m_ex, dm)
    # the distribution over energy levels (detailed balance)
    _, _, levels, probs = exact.exact_means(4, beta)
    for lv, p in zip(levels, probs):
        if p < 1e-3:
            continue
        f, df = exact.binned_error((E == lv).astype(np.float64), 50)
        assert abs(f - p) < 5 * df + 1e-4, (lv, f, p, df)


def test_finite_torus_matches_kaufman(golden_dir):
    vals = load_exact(golden_dir)
    L = 16
    beta = BETA_TC
    e_ex = vals[("kaufman_e_per_spin", "16", beta)]
    s = oracle.init_hot(L, 123)
    oracle.run(s, seed=123, beta=beta, t0=0, n=2000)
    E, _ = oracle.run(s, seed=123, beta=beta, t0=2000, n=60000)
    e, de = exact.binned_error(E / (L * L), 40)
    assert abs(e - e_ex) < 4.5 * de, (e, e_ex, de)


@pytest.mark.parametrize("T", [1.5, 2.0, 3.0, 3.5])
def test_onsager_and_yang(T, golden_dir):
    vals = load_exact(golden_dir)
    beta = 1.0 / T
    u = vals[("onsager_e_per_spin", "inf", beta)]
    m_y = vals[("yang_m_per_spin", "inf", beta)]
    L = 48
    s = oracle.init_cold(L, 1)
    oracle.run(s, seed=7, beta=beta, t0=0, n=1000)
    E, M = oracle.run(s, seed=7, beta=beta, t0=1000, n=8000)
    e, de = exact.binned_error(E / (L * L), 40)
    assert abs(e - u) < 4.5 * de + 2e-4, (e, u, de)
    if T < 2.2:
        m, dm = exact.binned_error(np.abs(M) / (L * L), 40)
        assert abs(m - m_y) < 4.5 * dm + 2e-3, (m, m_y, dm)


# ----------------------------------------------------------------------------- Philox rounds (opt-in scheme)

def test_philox_round_count_family():
    """The R-round member is the same iteration stopped after R rounds: R = 10
    equals the pinned Philox4x32-10, and rounds compose (one round applied to
    the R-round output with the round-R key equals R + 1 rounds)."""
    rng = np.random.default_rng(21)
    W0, W1 = 0x9E3779B9, 0xBB67AE85
    M0, M1 = 0xD2511F53, 0xCD9E8D57
    for _ in range(200):
        ctr = rng.integers(0, 2**32, size=4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2**32, size=2, dtype=np.uint64).astype(np.uint32)
        np.testing.assert_array_equal(oracle.philox4x32_r(ctr, key, 10), oracle.philox4x32_10(ctr, key))
        x = [int(v) for v in oracle.philox4x32_r(ctr, key, 7)]
        k0 = (int(key[0]) + 7 * W0) % 2**32
        k1 = (int(key[1]) + 7 * W1) % 2**32
        p0, p1 = M0 * x[0], M1 * x[2]
        step = [(p1 >> 32) ^ x[1] ^ k0, p1 & 0xFFFFFFFF, (p0 >> 32) ^ x[3] ^ k1, p0 & 0xFFFFFFFF]
        np.testing.assert_array_equal(oracle.philox4x32_r(ctr, key, 8), np.array(step, dtype=np.uint32))
    assert not np.array_equal(oracle.philox4x32_r([1, 2, 3, 4], [5, 6], 7), oracle.philox4x32_10([1, 2, 3, 4], [5, 6]))


def test_seven_round_chain_keeps_the_boltzmann_law(golden_dir):
    """The opt-in 7-round scheme drives the same Metropolis rule: the 4x4 chain
    still matches exact enumeration, and its flips use the 7-round draws."""
    vals = load_exact(golden_dir)
    beta = BETA_TC
    e_ex = vals[("enum_e_per_spin", "4", beta)]
    m_ex = vals[("enum_absm_per_spin", "4", beta)]
    with oracle.sweep_rounds(7):
        s = oracle.init_hot(4, 3)
        oracle.run(s, 3, beta, 0, 1000)
        E, M = oracle.run(s, 3, beta, 1000, 200000)
        # the flip set of one half-sweep uses the 7-round draw of each site
        L = 8
        c = oracle.init_cold(L, 1)
        oracle.half_sweep_thr(c, 9, 4, 0, 2**31, 2**31)
        for i in range(L):
            for j in range(L):
                want = ((i + j) & 1) == 0 and oracle._load().ora_site_draw_r(9, 4, i, j, 7) < 2**31
                assert (c[i, j] == -1) == want
    e, de = exact.binned_error(E / 16.0, 50)
    m, dm = exact.binned_error(np.abs(M) / 16.0, 50)
    assert abs(e - e_ex) < 4.5 * de
    assert abs(m - m_ex) < 4.5 * dm
    # outside the context the default (10 rounds) is back
    s10 = oracle.init_cold(8, 1)
    oracle.half_sweep_thr(s10, 9, 4, 0, 2**31, 2**31)
    assert not np.array_equal(s10, c)
