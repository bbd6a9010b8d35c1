"""Serving loop (sl_server): continuous batching with admission by device
footprint.  Each request's result in the mix must equal the request run
alone (bit for bit: every request is an independent solver context); the
budget bounds the memory held by running requests; an oversized request is
rejected; latency statistics are reported."""

import time

import numpy as np
import pytest

import sl_inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sl():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_07340_gb300 import build

    build.build()
    import paper_2009_07340_gb300 as sl

    return sl


def _requests(orc):
    reqs = []
    for i, (K, N, M) in enumerate([(64, 6, 40), (300, 4, 8), (20, 8, 100), (100, 5, 16)]):
        pb = I.config2(N=N, M=M, steps=9, K=K)
        pb["seed"] = 500 + i
        pb["dt"] = 0.5 * orc.dt_max(pb)
        reqs.append(pb)
    # the last two are heavy (E M n^3 > 2e9 per step): one heavy slot serves them in turn
    for i, (K, N, M) in enumerate([((5, 5), 4, 6), ((8, 4), 3, 10), ((8, 8), 8, 600), ((8, 8), 7, 900)]):
        pb = I.problem(2, K, (0.0, 0.0), (1.0, 1.0), N, M, 9, 0.0, 600 + i,
                       ("rotation", [2 * np.pi, 0.5, 0.5]), ("const", [0.003]), ("gauss", [1.0, 0.2, 0.5, 0.5]))
        pb["dt"] = 0.5 * orc.dt_max(pb)
        reqs.append(pb)
    return reqs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mix_equals_alone(sl, orc, precision):
    reqs = _requests(orc)
    with sl.Server(budget_bytes=2 << 30, slice_steps=2, heavy_slots=1, precision=precision) as srv:
        tickets = [srv.submit(pb) for pb in reqs[:3]]
        time.sleep(0.02)  # the rest arrive while the first ones run
        tickets += [srv.submit(pb) for pb in reqs[3:]]
        srv.wait_idle(300)
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["rejected"] == 0 and st["failed"] == 0
        assert 0 < st["p50_s"] <= st["p99_s"] and st["esu_per_s"] > 0
        for t, pb in zip(tickets, reqs):
            state, res = srv.poll(t)
            assert state == 2
            mean, m2, lat = res
            assert lat > 0
            ph = srv.timing(t)  # queued, creation wait, creation, running, completion wait, moments, release
            assert min(ph[:7]) >= 0 and ph[7] == pytest.approx(lat, rel=1e-12)
            assert sum(ph[:7]) == pytest.approx(ph[7], rel=1e-9)
            assert 0 < ph[8] <= ph[3]  # the longest slice lies within the running phase
            with sl.Solver(pb, precision) as s:
                s.step()
                am, aq = s.moments()
            assert np.array_equal(mean, am.ravel()) and np.array_equal(m2, aq.ravel())


def test_budget_admission_and_rejection(sl, orc):
    reqs = _requests(orc)[:4]
    big = I.config2(N=16, M=4096, steps=5, K=256)  # ~140 MB of state
    big["dt"] = I.DT_CFG2_HALF
    budget = 40 << 20
    with sl.Server(budget_bytes=budget, slice_steps=3, heavy_slots=0, precision="fp64") as srv:
        tickets = [srv.submit(pb) for pb in reqs]
        tb = srv.submit(big)
        srv.wait_idle(300)
        st = srv.stats()
        assert st["rejected"] == 1 and st["completed"] == len(reqs)
        assert 0 < st["memory_peak"] <= budget
        assert srv.poll(tb, want=False)[0] == -3  # SL_ERR_OOM
        for t in tickets:
            assert srv.poll(t, want=False)[0] == 2


def test_max_active_one_at_a_time(sl, orc):
    reqs = _requests(orc)[:4]
    with sl.Server(budget_bytes=1 << 30, slice_steps=4, max_active=1, precision="fp64") as srv:
        tickets = [srv.submit(pb) for pb in reqs]
        srv.wait_idle(300)
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["slices"] >= len(reqs)
        assert st["launch_s"] <= st["sched_busy_s"] and st["launch_max_s"] > 0
        for t, pb in zip(tickets, reqs):
            state, (mean, _, _) = srv.poll(t)
            assert state == 2
            with sl.Solver(pb, "fp64") as s:
                s.step()
                am, _ = s.moments()
            assert np.array_equal(mean, am.ravel())
        # one request at a time: every later request waited in the queue
        assert all(srv.timing(t)[0] > 0 for t in tickets[1:])


def test_preload(sl):
    sl.sl_preload()  # idempotent: every kernel is already prepared by the solvers above
    sl.sl_preload(0)
