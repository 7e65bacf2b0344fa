"""Serving loop and autotuner on the GPU.

Serving: jobs of different sizes, decompositions and iteration counts are
submitted while others run; each result must equal the oracle and the same
job solved alone, bit for bit (the jobs overlap on the device, their state
never does).  Admission respects the HBM budget and the slot limit.

Autotuner: the tuned context computes the same bits, reports that it was
tuned, and a second context with the same decomposition takes the choice
from the cache."""
import os
import time

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def od():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.empty_cache()  # the server's pool is its own allocation: return earlier tests' cached blocks
    from paper_2605_12734_gb300 import build
    build.build()
    import paper_2605_12734_gb300 as pkg
    return pkg


def same(a, b):
    return np.array_equal(np.ascontiguousarray(a).view(np.uint64), np.ascontiguousarray(b).view(np.uint64))


JOBS = [  # (edge, split, iters, seed, init_mode)
    (40, (2, 2, 2), 12, 11, 1), (33, (3, 3, 3), 7, 12, 0), (64, (4, 4, 4), 20, 13, 1),
    (27, (3, 3, 3), 1, 14, 1), (48, (2, 2, 2), 0, 15, 1), (56, (4, 4, 4), 9, 16, 1),
    (64, (2, 2, 2), 15, 17, 1), (35, (2, 2, 2), 25, 18, 0),
]


@pytest.mark.parametrize("batch_steps,job_streams", [(0, 0), (1, 0), (3, 0), (0, 2), (0, 8)])
def test_jobs_in_the_mix_match_alone_and_oracle(od, batch_steps, job_streams):
    # 0: the default persistent batches of 8 steps; 1: one fused step per
    # launch; 3: batches that end inside most jobs' step counts; job_streams:
    # one persistent launch per job, on 2 streams (jobs share a stream) or 8
    results = {}
    with od.Server(256 << 20, max_active=4, batch_steps=batch_steps, job_streams=job_streams) as srv:
        ids = []
        for k, (e, sp, it, seed, mode) in enumerate(JOBS):
            ids.append(srv.submit(e, e, e, it, split=sp, seed=seed, init_mode=mode))
            if k % 3 == 2:
                time.sleep(0.002)  # arrivals spread while earlier jobs run
        for jid, (e, sp, it, seed, mode) in zip(ids, JOBS):
            assert srv.wait(jid, 60.0) == od._native.OD_JOB_DONE, srv.info(jid)
            results[jid] = srv.fetch(jid)
            info = srv.info(jid)
            assert info["t_submit"] <= info["t_admit"] <= info["t_done"]
            srv.release(jid)
        st = srv.stats()
        assert st["done"] == len(JOBS) and st["failed"] == 0
        assert st["pool_used"] == 0
        if batch_steps == 1 and not job_streams:
            assert st["launches"] >= max(j[2] for j in JOBS)
        if job_streams:  # one launch per job that has steps
            assert st["launches"] == sum(1 for j in JOBS if j[2] > 0)
        assert 0 < st["busy_seconds"] <= st["seconds"]
    for jid, (e, sp, it, seed, mode) in zip(ids, JOBS):
        want = oracle.solve(e, e, e, seed, mode, it)
        assert same(results[jid], want), (e, sp, it)
        with od.Jacobi3D(e, e, e, split=sp, seed=seed, init_mode=mode, path="fused") as alone:
            alone.step(it)
            assert same(results[jid], alone.read())


@pytest.mark.parametrize("job_streams", [0, 16])
def test_serving_stream_at_full_job_sizes(od, job_streams):
    # jobs from the serving workload's own ranges -- edges up to 384, ODF up
    # to 216 with balanced splits that do not divide the edge (100 = 6 x 16 +
    # 4, 203 = 3 x 67 + 2, 250 = 4 x 62 + 2), 10..200 iterations -- submitted
    # while the others run; each result equals the job alone and the oracle
    jobs = [(384, 6, 30, 61), (100, 6, 200, 62), (203, 3, 57, 63), (64, 2, 10, 64), (250, 4, 41, 65),
            (384, 2, 12, 66), (77, 3, 133, 67), (128, 6, 88, 68)]
    results = {}
    with od.Server(24 << 30, job_streams=job_streams) as srv:
        ids = []
        for k, (e, p, it, seed) in enumerate(jobs):
            ids.append(srv.submit(e, e, e, it, split=(p, p, p), seed=seed))
            if k % 2 == 1:
                time.sleep(0.005)
        for jid in ids:
            assert srv.wait(jid, 300.0) == od._native.OD_JOB_DONE, srv.info(jid)
            results[jid] = srv.fetch(jid)
            srv.release(jid)
    threads = oracle.max_threads()
    for jid, (e, p, it, seed) in zip(ids, jobs):
        if (e, it, seed) not in _FULL_SIZE_WANT:  # the oracle's results, shared by both modes
            _FULL_SIZE_WANT[(e, it, seed)] = oracle.solve(e, e, e, seed, 1, it, threads=threads)
        assert same(results[jid], _FULL_SIZE_WANT[(e, it, seed)]), (e, p, it)
        if job_streams:
            continue  # the job alone: once
        with od.Jacobi3D(e, e, e, split=(p, p, p), seed=seed, init_mode=1, path="persistent") as alone:
            alone.step(it)
            assert same(results[jid], alone.read()), (e, p, it)


_FULL_SIZE_WANT = {}


@pytest.mark.parametrize("batch_steps", [0, 1])
def test_jobs_of_three_cta_shapes_in_one_step(od, batch_steps):
    # the planner gives these jobs 128 x 4, 256 x 4 and 128 x 2 CTAs; every
    # batch (8 steps, or 1) runs one batched launch per shape, and each result
    # is still the oracle's
    jobs = [((240, 240, 240), (2, 2, 2), 6, 21), ((600, 20, 16), (2, 1, 1), 9, 22), ((40, 40, 40), (2, 2, 2), 7, 23),
            ((600, 20, 16), (2, 1, 1), 4, 24)]
    for dims, sp, _, _ in jobs[:3]:
        assert od.plan(*dims, split=sp)["threads"] * od.plan(*dims, split=sp)["cells_per_thread"] in (256, 512, 1024)
    with od.Server(1 << 30, batch_steps=batch_steps, job_streams=0) as srv:
        ids = [srv.submit(*dims, it, split=sp, seed=seed) for dims, sp, it, seed in jobs]
        got = []
        for jid in ids:
            assert srv.wait(jid, 120.0) == od._native.OD_JOB_DONE, srv.info(jid)
            got.append(srv.fetch(jid))
            srv.release(jid)
        st = srv.stats()
    # more than one launch per batch while shapes overlap
    steps = 1 if batch_steps == 1 else 8
    assert st["launches"] > -(-max(j[2] for j in jobs) // steps)
    for res, (dims, sp, it, seed) in zip(got, jobs):
        assert same(res, oracle.solve(*dims, seed, 1, it)), dims


@pytest.mark.parametrize("job_streams", [0, 3])
def test_jobs_with_uneven_cut_lists(od, job_streams):
    # explicit cut lists (1-wide blocks, blocks of one plane, uneven edges),
    # copied at submit: the caller's arrays are gone when the job is admitted
    jobs = [((70, 45, 38), ([0, 13, 40, 70], [0, 24, 45], [0, 5, 6, 38]), 8, 71),
            ((33, 31, 29), ([0, 1, 2, 32, 33], [0, 30, 31], [0, 14, 15, 29]), 13, 72),
            ((96, 64, 48), ([0, 24, 25, 96], [0, 32, 64], [0, 1, 47, 48]), 5, 73)]
    with od.Server(1 << 30, job_streams=job_streams) as srv:
        ids = []
        for dims, cuts, it, seed in jobs:
            ids.append(srv.submit(*dims, it, cuts=tuple(list(c) for c in cuts), seed=seed))
        got = []
        for jid in ids:
            assert srv.wait(jid, 120.0) == od._native.OD_JOB_DONE, srv.info(jid)
            got.append(srv.fetch(jid))
            srv.release(jid)
    for res, (dims, cuts, it, seed) in zip(got, jobs):
        assert same(res, oracle.solve(*dims, seed, 1, it)), (dims, cuts)


@pytest.mark.parametrize("job_streams", [0, 4])
def test_completion_queue_releases_as_jobs_end(od, job_streams):
    # a budget for two jobs and six submitted at once: the client takes each
    # ended job from the completion queue (every job exactly once, a 0-step
    # job included) and releases it, which admits the next; results stay exact
    e, sp = 48, (2, 2, 2)
    need = od.plan(e, e, e, split=sp, path="persistent")["arena_bytes"]
    jobs = [(11, 5), (12, 0), (13, 9), (14, 3), (15, 7), (16, 1)]
    with od.Server(int(need * 2.5), job_streams=job_streams) as srv:
        ids = {srv.submit(e, e, e, it, split=sp, seed=seed): (seed, it) for seed, it in jobs}
        got, order = {}, []
        t0 = time.time()
        while len(order) < len(jobs):
            assert time.time() - t0 < 120
            jid = srv.next_completion(1.0)
            if jid is None:
                continue
            assert jid in ids and jid not in got
            assert srv.info(jid)["state"] == od._native.OD_JOB_DONE
            got[jid] = srv.fetch(jid)
            order.append(jid)
            srv.release(jid)
        assert srv.next_completion(0.0) is None
        assert srv.stats()["pool_used"] == 0
    for jid, (seed, it) in ids.items():
        assert same(got[jid], oracle.solve(e, e, e, seed, 1, it)), (seed, it)


def test_budget_admission_and_release(od):
    e, sp = 48, (2, 2, 2)
    need = od.plan(e, e, e, split=sp, threads=128, cells_per_thread=4, stages=4, arith=7)["arena_bytes"]
    budget = int(need * 2.5)  # room for two jobs at a time
    with od.Server(budget) as srv:
        with pytest.raises(od.ODError) as ei:
            srv.submit(200, 200, 200, 1, split=(1, 1, 1))
        assert ei.value.status == od._native.OD_EBUDGET
        ids = [srv.submit(e, e, e, 30, split=sp, seed=s) for s in range(5)]
        peak = 0
        for jid in ids:
            assert srv.wait(jid, 60.0) == od._native.OD_JOB_DONE
            peak = max(peak, srv.stats()["pool_peak"])
            srv.release(jid)
        assert peak <= budget
        # a queued job can be released (cancelled) before it runs
        with od.Server(budget, max_active=1) as srv2:
            a = srv2.submit(e, e, e, 200, split=sp, seed=1)
            b = srv2.submit(e, e, e, 200, split=sp, seed=2)
            c = srv2.submit(e, e, e, 5, split=sp, seed=3)
            srv2.release(c)
            assert srv2.wait(a, 60.0) == od._native.OD_JOB_DONE
            assert srv2.wait(b, 60.0) == od._native.OD_JOB_DONE
    want = oracle.solve(e, e, e, 4, 1, 30)
    with od.Server(budget) as srv:
        j = srv.submit(e, e, e, 30, split=sp, seed=4)
        assert srv.wait(j, 60.0) == od._native.OD_JOB_DONE
        assert same(srv.fetch(j), want)


def test_autotune_same_bits_and_cache(od, tmp_path, monkeypatch):
    monkeypatch.setenv("OD_TUNE_CACHE", str(tmp_path / "tune.txt"))
    nx, ny, nz = 96, 64, 48
    want = oracle.solve(nx, ny, nz, 8, 1, 6)
    with od.Jacobi3D(nx, ny, nz, split=(3, 2, 2), seed=8, path="persistent", autotune=True) as s:
        st = s.stats()
        assert st["tuned"] == 1 and st["tune_ms_per_step"] > 0
        s.step(6)
        assert same(s.read(), want)
    lines = (tmp_path / "tune.txt").read_text().splitlines()
    assert len(lines) == 1
    t0 = time.perf_counter()
    with od.Jacobi3D(nx, ny, nz, split=(3, 2, 2), seed=8, path="persistent", autotune=True) as s2:
        assert abs(s2.stats()["tune_ms_per_step"] - st["tune_ms_per_step"]) < 1e-9  # from the cache
        assert s2.stats()["plan"]["threads"] == st["plan"]["threads"]
    assert len((tmp_path / "tune.txt").read_text().splitlines()) == 1


def test_short_serving_names(od):
    # od_submit / od_poll / od_fetch: the serving loop's short entry points
    import ctypes
    import time
    from paper_2605_12734_gb300 import _native
    e, it = 40, 7
    want = oracle.solve(e, e, e, 9, 1, it)
    with od.Server(256 << 20) as srv:
        cfg, keep = od.make_config(e, e, e, split=(2, 2, 2), seed=9, init_mode=1)
        jid = ctypes.c_uint64()
        assert od.lib().od_submit(srv._h, ctypes.byref(cfg), it, ctypes.byref(jid)) == _native.OD_OK
        t0 = time.time()
        while not srv.poll(jid.value):
            assert time.time() - t0 < 60
            time.sleep(0.001)
        got = np.empty(e ** 3)
        assert od.lib().od_fetch(srv._h, jid.value, got.ctypes.data, 0) == _native.OD_OK
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
        srv.release(jid.value)
