"""Small-lattice parity battery run against the checked build of the library
(ISING_LIBRARY pointing at libising_checked.so): every kernel family, each
result compared with the oracle, then the device's out-of-range record read
back.  Prints one JSON line; exits non-zero on a mismatch."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import paper_1811_04384_gb300 as p  # noqa: E402
from paper_1811_04384_gb300 import serving  # noqa: E402

BETA = 1.0 / 2.269


def check(name, got, want):
    for g, w in zip(got, want):
        if not np.array_equal(np.asarray(g), np.asarray(w)):
            print(json.dumps({"ok": False, "case": name}))
            sys.exit(1)


def lattice_case(L, n, path=None, lanes=None, tiling=None, every=1):
    with p.Lattice(L, 11 + L) as lat:
        if path is not None:
            lat.set_path(path)
        if lanes is not None:
            lat.set_item_lanes(lanes)
        if tiling is not None:
            lat.set_tiling(*tiling)
        lat.init_hot()
        lat.set_beta(BETA)
        E, M = lat.sweep_record(n, every)
        S = lat.get_spins()
    s = oracle.init_hot(L, 11 + L)
    Eo, Mo = oracle.run(s, 11 + L, BETA, 0, n, every)
    check(f"lattice L={L} path={path} lanes={lanes} tiling={tiling}", (E, M, S), (Eo, Mo, s))


def main():
    checked, _ = p.check_status()
    cases = 0
    for L in (4, 6, 10, 12, 34, 42, 44, 46, 64, 130, 260):
        lattice_case(L, 6)                                       # on-chip up to 512 items
        lattice_case(L, 6, path=p.ISING_PATH_LAUNCHES)
        cases += 2
    lattice_case(300, 34, path=p.ISING_PATH_LAUNCHES)            # graph replays, masks drawn first
    lattice_case(130, 33, path=p.ISING_PATH_LAUNCHES, every=3)
    lattice_case(260, 5, path=p.ISING_PATH_RESIDENT)             # on-chip, draws inside the block
    for F in (2, 4, 8):
        lattice_case(64, 5, path=p.ISING_PATH_LAUNCHES, lanes=F)
    lattice_case(130, 5, path=p.ISING_PATH_LAUNCHES, lanes=1, tiling=(4, 16, 8))
    cases += 7
    # the cluster path: automatic at L = 300 (one word per thread, 8 mask
    # slabs), forced at L = 64 (phases of 4), L = 700 (two words per thread)
    # and L = 1500 (four words per thread, two slabs)
    lattice_case(300, 14)
    lattice_case(64, 9, path=p.ISING_PATH_CLUSTER, every=3)
    lattice_case(700, 6, every=2)
    lattice_case(1500, 3, path=p.ISING_PATH_CLUSTER)
    cases += 4
    # batch of uneven replicas
    Ls = [6, 44, 130, 64, 12]
    seeds = [3, 4, 5, 6, 7]
    E, M = p.Batch(Ls, [BETA] * 5, seeds, [1] * 5).sweep([7, 5, 6, 7, 4], every=1)
    for k, L in enumerate(Ls):
        s = oracle.init_hot(L, seeds[k])
        Eo, Mo = oracle.run(s, seeds[k], BETA, 0, [7, 5, 6, 7, 4][k], 1)
        check(f"batch replica L={L}", (E[k], M[k]), (Eo, Mo))
    cases += 1
    # the paper's column-interleaved layout: checkerboard chain on its
    # cluster path (automatic here) and on the graph replays, random-word chain
    for L in (84, 168):
        for path in (p.ISING_PATH_AUTO, p.ISING_PATH_LAUNCHES):
            with p.Lattice(L, 9, layout=p.ISING_LAYOUT_COLUMN_INTERLEAVED) as lat:
                lat.set_path(path)
                lat.init_hot()
                lat.set_beta(BETA)
                E, M = lat.sweep_record(34, 2)
                S = lat.get_spins()
            s = oracle.init_hot(L, 9)
            Eo, Mo = oracle.run(s, 9, BETA, 0, 34, 2)
            check(f"interleaved L={L} path={path}", (E, M, S), (Eo, Mo, s))
            cases += 1
        for nstrips in (1, 6, L // 2):
            with p.Lattice(L, 5, layout=p.ISING_LAYOUT_COLUMN_INTERLEAVED) as lat:
                lat.init_hot()
                lat.set_chain(p.ISING_CHAIN_RANDOM_WORDS, nstrips)
                lat.set_beta(BETA)
                E, M = lat.sweep_record(2, 1)
                S = lat.get_spins()
            s = oracle.init_hot(L, 5)
            Eo, Mo = oracle.rw_run(s, 5, BETA, 0, 2, nstrips)
            check(f"random words L={L} strips={nstrips}", (E, M, S), (Eo, Mo, s))
        cases += 4
    # a served job
    with serving.Server(16 << 20) as srv:
        r = serving.Request(46, BETA, 21, 12, 3, want_spins=True)
        srv.submit(r)
        assert srv.wait(r.id).status == 0
    s = oracle.init_hot(46, 21)
    Eo, Mo = oracle.run(s, 21, BETA, 0, 12, 3)
    check("served job", (r.E, r.M, r.spins), (Eo, Mo, s))
    cases += 1
    checked_after, violation = p.check_status()
    print(json.dumps({"ok": violation == 0, "checked": checked and checked_after, "violation": violation,
                      "cases": cases}))
    sys.exit(0 if violation == 0 else 2)


if __name__ == "__main__":
    main()
