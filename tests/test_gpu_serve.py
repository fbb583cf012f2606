"""Serving loop: continuous batching of resultant and gcd jobs.

Each served result must be bit-identical to the same job computed alone through the
blocking entry points (and to the oracle where the oracle is quick)."""

import threading

import numpy as np
import pytest

import paper_1201_1548_gb300 as bs
from oracle import gcd as G
from oracle import resultant as R
from workloads import cfg5_stream, dense_curve

pytestmark = pytest.mark.gpu


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _small_stream(seed, jobs, deg_hi=12, bits_hi=96):
    return cfg5_stream(seed=seed, jobs=jobs, deg_lo=3, deg_hi=deg_hi, bits_lo=8,
                       bits_hi=bits_hi)


def _alone(ctx, job):
    if job["kind"] == "gcd":
        return ctx.gcd_z(job["a"], job["b"])
    return ctx.resultant(job["f"], job["g"], job.get("var", 1))


def _submit(srv, job):
    if job["kind"] == "gcd":
        return srv.submit(bs.JOB_GCD, job["a"], job["b"])
    return srv.submit(bs.JOB_RESULTANT, job["f"], job["g"], var=job.get("var", 1))


@pytest.fixture
def server():
    srv = bs.Context(0)
    yield srv
    srv.serve_stop()
    srv.close()


def test_served_results_equal_alone_and_oracle(ctx, server):
    stream = _small_stream(seed=5, jobs=48)
    for i, job in enumerate(stream):
        if job["kind"] == "resultant" and i % 3 == 0:
            job["var"] = 0
    server.serve_start(slots=3, max_batch=8)
    tickets = [_submit(server, job) for job in stream]
    for job, t in zip(stream, tickets):
        assert server.wait(t, 120000)
        status, coeffs, q_ms, lat_ms = server.poll(t)
        assert status == 0
        assert lat_ms >= q_ms >= 0.0
        assert coeffs == _alone(ctx, job)
        if job["kind"] == "gcd":
            assert coeffs == G.gcd_z(job["a"], job["b"])
    st = server.serve_stats()
    assert st["completed"] == len(stream) and st["queued"] == 0 and st["inflight"] == 0
    assert st["arena_used"] == 0


def test_served_small_resultants_match_oracle(server):
    rng = _rng(51)
    jobs = []
    for _ in range(10):
        f = dense_curve(rng, int(rng.integers(2, 5)), int(rng.integers(4, 24)))
        g = dense_curve(rng, int(rng.integers(2, 5)), int(rng.integers(4, 24)))
        jobs.append((f, g))
    server.serve_start(slots=2, max_batch=4)
    tickets = [server.submit(bs.JOB_RESULTANT, f, g) for f, g in jobs]
    for (f, g), t in zip(jobs, tickets):
        assert server.wait(t, 60000)
        status, coeffs, _, _ = server.poll(t)
        assert status == 0 and coeffs == R.res_y(f, g)


def test_admission_by_arena_memory(ctx, server):
    stream = [j for j in _small_stream(seed=6, jobs=40, deg_hi=16, bits_hi=64)]
    probe = bs.Context(0)
    # the arena holds about three of the largest jobs: batches must wait for memory
    sizes = []
    probe.serve_start(slots=1, max_batch=1, arena_bytes=1 << 30)
    for job in stream:
        t = _submit(probe, job)
        probe.wait(t)
        probe.poll(t)
    peak_one = probe.serve_stats()["arena_peak"]
    probe.serve_stop()
    probe.close()
    arena = 3 * peak_one
    server.serve_start(slots=3, max_batch=16, arena_bytes=arena)
    tickets = [_submit(server, job) for job in stream]
    for job, t in zip(stream, tickets):
        assert server.wait(t, 120000)
        status, coeffs, _, _ = server.poll(t)
        assert status == 0 and coeffs == _alone(ctx, job)
    st = server.serve_stats()
    assert st["arena_peak"] <= st["arena_bytes"]
    assert st["batches"] > 1
    del sizes


def test_oversized_job_is_refused(server):
    rng = _rng(52)
    server.serve_start(slots=1, max_batch=4, arena_bytes=1 << 20)
    f = dense_curve(rng, 24, 64)
    g = dense_curve(rng, 24, 64)
    with pytest.raises(bs.BsError) as e:
        server.submit(bs.JOB_RESULTANT, f, g)
    assert e.value.code == 2
    t = server.submit(bs.JOB_GCD, [1, 2, 1], [1, 1])   # small jobs still run
    assert server.wait(t, 60000)
    assert server.poll(t)[1] == [1, 1]


def test_batches_overlap_and_context_is_reserved(server):
    rng = _rng(53)
    server.serve_start(slots=3, max_batch=1)
    with pytest.raises(bs.BsError):
        server.resultant([[1, 2], [3]], [[1], [1]])       # reserved for the serving loop
    jobs = [(dense_curve(rng, 20, 48), dense_curve(rng, 20, 48)) for _ in range(12)]
    tickets = [server.submit(bs.JOB_RESULTANT, f, g) for f, g in jobs]
    for t in tickets:
        assert server.wait(t, 120000)
        assert server.poll(t)[0] == 0
    st = server.serve_stats()
    assert st["max_inflight"] >= 2
    # the per-phase wall times cover the 12 batches: some device work, no negative phase
    assert st["batches"] == 12 and st["device_ms"] > 0.0
    assert st["host_plan_ms"] >= 0.0 and st["host_finish_ms"] >= 0.0


def test_submit_from_several_threads(ctx, server):
    stream = _small_stream(seed=7, jobs=24)
    server.serve_start(slots=2, max_batch=6)
    tickets = [None] * len(stream)

    def worker(lo):
        for i in range(lo, len(stream), 4):
            tickets[i] = _submit(server, stream[i])

    ths = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    for job, t in zip(stream, tickets):
        assert server.wait(t, 120000)
        status, coeffs, _, _ = server.poll(t)
        assert status == 0 and coeffs == _alone(ctx, job)
    with pytest.raises(bs.BsError):
        server.poll(tickets[0])                              # released after collection


def test_work_classes_and_priorities(ctx, server):
    """A large resultant (more than 2e9 multiply-reduces) and tiny ones submitted together:
    every result equals the same call alone, and the tiny jobs, which take other slots and
    the high-priority stream, complete before the large one."""
    import time
    rng = _rng(59)
    big = (dense_curve(rng, 44, 200), dense_curve(rng, 44, 200))
    p = bs.bs_plan(*big)
    assert p["k_total"] * p["N"] * p["m_e"] * p["n_e"] > 2e9
    tiny = [(dense_curve(rng, 4, 16), dense_curve(rng, 4, 16)) for _ in range(8)]
    want_big = ctx.resultant(*big)
    want_tiny = [ctx.resultant(f, g) for f, g in tiny]
    server.serve_start(slots=4, max_batch=4)
    tb = server.submit(bs.JOB_RESULTANT, *big)
    time.sleep(0.001)
    tt = [server.submit(bs.JOB_RESULTANT, f, g) for f, g in tiny]
    done_tiny = []
    for t in tt:
        assert server.wait(t, 120000)
        done_tiny.append(server.poll(t))
    assert server.wait(tb, 120000)
    st_b, coeffs_b, _, lat_b = server.poll(tb)
    assert st_b == 0 and coeffs_b == want_big
    for (st, coeffs, _, lat), want in zip(done_tiny, want_tiny):
        assert st == 0 and coeffs == want
        assert lat < lat_b
