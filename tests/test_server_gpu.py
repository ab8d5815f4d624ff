"""Serving (continuous batching): every job's result is bit-identical alone
and in the mix; jobs that arrive while others run are admitted and overlap;
admission respects the HBM budget and the slot limit; cancellation,
timeouts and bad jobs are reported without touching the device."""
import time

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serving():
    import paper_1811_04384_gb300 as p
    p.load()
    from paper_1811_04384_gb300 import serving
    return serving


def alone(L, beta, seed, sweeps, every, hot=True):
    import paper_1811_04384_gb300 as p
    with p.Lattice(L, seed) as lat:
        if hot:
            lat.init_hot()
        lat.set_beta(beta)
        E, M = lat.sweep_record(sweeps, every)
        return E, M, lat.get_spins()


def test_mix_equals_alone(serving):
    rng = np.random.default_rng(3)
    specs = []
    for k in range(12):
        L = int(rng.choice([6, 32, 64, 130, 256, 512]))
        specs.append((L, float(rng.uniform(0.28, 0.66)), int(rng.integers(1, 2**62)), int(rng.integers(1, 120)),
                      int(rng.choice([1, 3, 7])), bool(k % 3)))
    reqs = [serving.Request(L, b, s, n, e, hot, want_spins=True) for (L, b, s, n, e, hot) in specs]
    with serving.Server(64 << 20, max_jobs=8, epoch_sweeps=17) as srv:
        for r in reqs:
            srv.submit(r)
        for r in reqs:
            res = srv.wait(r.id)
            assert res.status == 0 and serving.STATES[res.state] == "done"
            assert res.sweeps_done == r.sweeps
    # every served job (all L <= 512) against the oracle, and against the same job alone
    ora = oracle.run_jobs([(L, s, b, hot, n, e) for (L, b, s, n, e, hot) in specs])
    for r, (L, b, s, n, e, hot), (Eo, Mo, so) in zip(reqs, specs, ora):
        np.testing.assert_array_equal(r.E, Eo)
        np.testing.assert_array_equal(r.M, Mo)
        np.testing.assert_array_equal(r.spins, so)
        E, M, S = alone(L, b, s, n, e, hot)
        np.testing.assert_array_equal(r.E, E)
        np.testing.assert_array_equal(r.spins, S)


def test_large_served_jobs_equal_oracle(serving):
    """Sixteen served jobs of L = 1024 .. 4096 (the serving stream's large
    sizes), 4 to 8 sweeps each, run in one mix with small jobs and compared
    with the oracle: E, M every sweep and the final spins."""
    rng = np.random.default_rng(17)
    specs = []
    for k in range(16):
        L = [1024, 2048, 4096][k % 3] if k < 15 else 4096
        n = 8 if L == 1024 else (6 if L == 2048 else 4)
        specs.append((L, float(rng.uniform(1 / 3.5, 1 / 1.5)), int(rng.integers(1, 2**62)), n, 1, bool(k % 4)))
    small = [serving.Request(64, 0.44, 100 + k, 300, 10) for k in range(6)]
    reqs = [serving.Request(L, b, s, n, e, hot, want_spins=True) for (L, b, s, n, e, hot) in specs]
    with serving.Server(2 << 30, max_jobs=32, epoch_sweeps=3) as srv:
        for k, r in enumerate(reqs):
            srv.submit(r)
            if k < len(small):
                srv.submit(small[k])
        for r in reqs + small:
            assert srv.wait(r.id).status == 0
    ora = oracle.run_jobs([(L, s, b, hot, n, e) for (L, b, s, n, e, hot) in specs])
    for r, (Eo, Mo, so) in zip(reqs, ora):
        np.testing.assert_array_equal(r.E, Eo)
        np.testing.assert_array_equal(r.M, Mo)
        np.testing.assert_array_equal(r.spins, so)


def test_jobs_arriving_while_others_run_overlap(serving):
    with serving.Server(256 << 20, max_jobs=16, epoch_sweeps=20) as srv:
        long = serving.Request(2048, 0.44, 1, 3000, 100)
        srv.submit(long)
        for _ in range(2000):
            if serving.STATES[srv.poll(long.id).state] == "running":
                break
            time.sleep(0.001)
        late = [serving.Request(128, 0.4, 10 + k, 200, 10) for k in range(4)]
        for r in late:
            srv.submit(r)
        res_long = srv.wait(long.id)
        res_late = [srv.wait(r.id) for r in late]
    for r, res in zip(late, res_late):
        assert res.status == 0
        assert res.start_s < res_long.done_s      # admitted while the long job ran
        E, M, _ = alone(128, 0.4, r.seed, 200, 10)
        np.testing.assert_array_equal(r.E, E)
    E, M, _ = alone(2048, 0.44, 1, 3000, 100)
    np.testing.assert_array_equal(long.E, E)
    np.testing.assert_array_equal(long.M, M)


def test_admission_respects_budget_and_slots(serving):
    import paper_1811_04384_gb300 as p
    per_job = 2 * 512 * 14 * 8            # L = 512: W = 13, pitch 14, both colours
    budget = 2 * per_job + 4096            # room for two L = 512 jobs at a time
    reqs = [serving.Request(512, 0.5, k + 1, 150, 50) for k in range(5)]
    with serving.Server(budget, max_jobs=8, epoch_sweeps=10) as srv:
        for r in reqs:
            srv.submit(r)
        res = [srv.wait(r.id) for r in reqs]
        with pytest.raises(p.IsingError):   # larger than the whole arena
            srv.submit(serving.Request(2048, 0.5, 1, 10))
    spans = [(x.start_s, x.done_s) for x in res]
    for t in [s for s, _ in spans]:
        assert sum(1 for (a, b) in spans if a <= t < b) <= 2
    for r in reqs:
        E, _, _ = alone(512, 0.5, r.seed, 150, 50)
        np.testing.assert_array_equal(r.E, E)


def test_cancel_timeout_and_bad_jobs(serving):
    import paper_1811_04384_gb300 as p
    with serving.Server(256 << 20, max_jobs=1, epoch_sweeps=10) as srv:
        long = serving.Request(1024, 0.44, 1, 4000, 1000)
        queued = serving.Request(64, 0.44, 2, 10)
        srv.submit(long)
        srv.submit(queued)
        srv.cancel(queued.id)
        assert serving.STATES[srv.poll(queued.id).state] == "cancelled"
        res = srv.wait(long.id, timeout_ms=0)
        assert serving.STATES[res.state] in ("queued", "running")
        with pytest.raises(p.IsingError):
            srv.submit(serving.Request(63, 0.4, 1, 10))
        with pytest.raises(p.IsingError):
            srv.submit(serving.Request(64, -1.0, 1, 10))
        with pytest.raises(p.IsingError):
            srv.poll(987654)
        res = srv.wait(long.id)
        assert res.status == 0
        srv.release(long.id)
        with pytest.raises(p.IsingError):
            srv.poll(long.id)


def test_boundary_create_form_serves_a_job(serving):
    """ising_server_create(budget, &srv): the two-argument form of the
    boundary, with the default limits, serves a job bit-exactly."""
    with serving.Server(64 << 20) as srv:
        r = serving.Request(96, 0.4, 21, 60, 4, want_spins=True)
        srv.submit(r)
        res = srv.wait(r.id)
        assert res.status == 0 and res.sweeps_done == 60
    so = oracle.init_hot(96, 21)
    Eo, Mo = oracle.run(so, 21, 0.4, 0, 60, 4)
    np.testing.assert_array_equal(r.E, Eo)
    np.testing.assert_array_equal(r.M, Mo)
    np.testing.assert_array_equal(r.spins, so)


def test_cancel_then_release_keeps_serving(serving):
    """A queued job that is cancelled and then released leaves no trace: the
    worker skips its id, later jobs still run, and the totals count only the
    jobs that ran."""
    with serving.Server(256 << 20, max_jobs=1, epoch_sweeps=10) as srv:
        long = serving.Request(1024, 0.44, 1, 4000, 1000)
        queued = serving.Request(64, 0.44, 2, 10)
        srv.submit(long)
        srv.submit(queued)
        srv.cancel(queued.id)
        srv.release(queued.id)
        after = serving.Request(64, 0.44, 3, 20, 2)
        srv.submit(after)
        assert srv.wait(long.id).status == 0
        assert srv.wait(after.id).status == 0
        st = srv.stats()
        assert st["jobs_done"] == 2
        assert st["spin_updates"] == 1024 * 1024 * 4000 + 64 * 64 * 20
    so = oracle.init_hot(64, 3)
    Eo, Mo = oracle.run(so, 3, 0.44, 0, 20, 2)
    np.testing.assert_array_equal(after.E, Eo)
    np.testing.assert_array_equal(after.M, Mo)


def test_injected_worker_fault(serving):
    """A host exception thrown in the worker between epochs (the test hook;
    nothing faults on the device): the running jobs are reported failed with
    ISING_EINTERNAL, their arena blocks come back, the queued job is then
    admitted and runs bit-exactly, and destroy returns."""
    import paper_1811_04384_gb300 as p
    per_job = 2 * 512 * 14 * 8                 # L = 512: both colours, pitch 14
    budget = 2 * per_job + 4096                # room for two such jobs at a time
    srv = serving.Server(budget, max_jobs=4, epoch_sweeps=10)
    try:
        a = serving.Request(512, 0.44, 1, 100000, 1000)
        b = serving.Request(512, 0.44, 2, 100000, 1000)
        c = serving.Request(512, 0.44, 3, 40, 4)
        srv.submit(a)
        srv.submit(b)
        for _ in range(5000):
            if all(serving.STATES[srv.poll(r.id).state] == "running" for r in (a, b)):
                break
            time.sleep(0.001)
        assert all(serving.STATES[srv.poll(r.id).state] == "running" for r in (a, b))
        srv.submit(c)                          # no arena room until a or b leaves
        assert serving.STATES[srv.poll(c.id).state] == "queued"
        srv.inject_fault(0)
        for r in (a, b):
            res = srv.wait(r.id, timeout_ms=60000)
            assert serving.STATES[res.state] == "failed"
            assert res.status == p.ISING_EINTERNAL
        res = srv.wait(c.id, timeout_ms=60000)
        assert res.status == 0 and serving.STATES[res.state] == "done"
        assert srv.stats()["jobs_done"] == 1
    finally:
        t0 = time.perf_counter()
        srv.close()
        assert time.perf_counter() - t0 < 30
    so = oracle.init_hot(512, 3)
    Eo, Mo = oracle.run(so, 3, 0.44, 0, 40, 4)
    np.testing.assert_array_equal(c.E, Eo)
    np.testing.assert_array_equal(c.M, Mo)
