"""Batched uneven instances in one graph-captured launch sequence (sl_batch).

Every instance's samples after batched steps must equal the same instance
run alone through sl_init / sl_step, bit for bit (the per-sample arithmetic
is the same code); the graph is replayed across calls; the autotuner leaves
every instance's state unchanged."""

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


def _mix1d(orc):
    out = []
    for i, (K, N, M) in enumerate([(8, 4, 70), (48, 6, 9), (200, 4, 5), (300, 5, 3), (13, 6, 33), (48, 4, 1)]):
        pb = I.config2(N=N, M=M, steps=0, K=K)
        pb["seed"] = 100 + i
        pb["dt"] = (0.3 + 0.1 * i) * orc.dt_max(pb)
        out.append(pb)
    return out


def _mix2d(orc):
    out = []
    for i, (K, N, M, drift) in enumerate([((4, 4), 3, 5, ("rotation", [2 * np.pi, 0.5, 0.5])),
                                          ((6, 3), 4, 3, ("const", [0.6, -0.3])),
                                          ((3, 3), 4, 7, ("rotation", [2 * np.pi, 0.5, 0.5]))]):
        pb = I.problem(2, K, (0.0, 0.0), (1.0, 1.0), N, M, 0, 0.0, 200 + i, drift,
                       ("const", [0.004 + 0.001 * i]), ("gauss", [1.0, 0.2, 0.5, 0.5]))
        pb["dt"] = 0.4 * orc.dt_max(pb)
        out.append(pb)
    return out


def _alone(sl, pb, precision, steps):
    with sl.Solver(pb, precision) as s:
        s.step(pb["dt"], steps)
        return s.samples().reshape(pb["M"], -1)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_batch_equals_alone_1d(sl, orc, precision):
    pbs = _mix1d(orc)
    with sl.Batch(pbs, precision) as b:
        b.step(4)
        b.step(4)  # graph replay
        b.step(3)  # a second graph
        for i, pb in enumerate(pbs):
            assert np.array_equal(b.samples(i), _alone(sl, pb, precision, 11)), i


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_batch_equals_alone_2d_and_mixed_dims(sl, orc, precision):
    pbs = _mix2d(orc) + _mix1d(orc)[:2]
    with sl.Batch(pbs, precision) as b:
        b.step(3)
        b.step(3)
        for i, pb in enumerate(pbs):
            assert np.array_equal(b.samples(i), _alone(sl, pb, precision, 6)), i


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_batch_high_orders_equal_alone(sl, orc, precision):
    # 2D orders whose Gram rows are split over several lanes (FP64 N = 9..11,
    # FP32 N = 11), batched with a one-lane order
    pbs = []
    for i, (K, N, M) in enumerate([((2, 2), 9, 3), ((3, 2), 11, 2), ((2, 3), 4, 4)]):
        pb = I.problem(2, K, (0.0, 0.0), (1.0, 1.0), N, M, 0, 0.0, 300 + i, ("rotation", [2 * np.pi, 0.5, 0.5]),
                       ("const", [0.004]), ("gauss", [1.0, 0.2, 0.5, 0.5]))
        pb["dt"] = 0.4 * orc.dt_max(pb)
        pbs.append(pb)
    with sl.Batch(pbs, precision) as b:
        b.step(2)
        for i, pb in enumerate(pbs):
            assert np.array_equal(b.samples(i), _alone(sl, pb, precision, 2)), i


def test_tuner_restores_state_and_picks_grids(sl, orc):
    pbs = _mix1d(orc)
    with sl.Batch(pbs, "fp32") as b:
        b.step(2)
        before = [b.samples(i) for i in range(len(pbs))]
        ms = b.tune(probe_steps=3)
        assert ms > 0
        grids = b.grids()
        assert len(grids) == 2  # orders 4 and 6 (the N=5, K=300 instance runs as a cluster launch)
        assert all(g[1] > 0 for g in grids)
        for i in range(len(pbs)):
            assert np.array_equal(b.samples(i), before[i])
        b.step(2)
        for i, pb in enumerate(pbs):
            assert np.array_equal(b.samples(i), _alone(sl, pb, "fp32", 4)), i


def test_batch_moments_match_oracle(sl, orc):
    pbs = _mix1d(orc)[:3]
    with sl.Batch(pbs, "fp64") as b:
        b.step(5)
        for i, pb in enumerate(pbs):
            mean, _ = b.moments(i)
            ref = orc.run(I.with_(pb, steps=5), nthreads=8)
            rm = ref["sum"] / pb["M"]
            assert np.abs(mean - rm).max() / np.abs(rm).max() <= 1e-10


def test_parallel_branches_equal_alone(sl, orc):
    # order classes spread over the tuned number of parallel graph branches:
    # every instance still equals its solo run bit for bit
    pbs = _mix2d(orc) + _mix1d(orc)
    with sl.Batch(pbs, "fp32") as b:
        assert b.lanes() == 1
        ms = b.tune(probe_steps=1)
        assert ms > 0 and b.lanes() in (1, 2, 4)
        b.step(3)
        for i, pb in enumerate(pbs):
            assert np.array_equal(b.samples(i), _alone(sl, pb, "fp32", 3)), i
