"""The multi-rank host logic of bench.py, on CPU: two gloo ranks.

Each rank runs its own disjoint range of global samples (shard_sample0) with
no collective on the data path; the job's time is the slowest rank's
(max_over_ranks) and its rate counts every rank's units (whole_job_rate).
Because the Wiener increments are keyed on the global sample index, the
ranks' samples together must give the moments of one run over all samples.
The per-rank solver here is the FP64 oracle (the GPU path is the same call
with sample0 set)."""

import os
import socket

import numpy as np
import pytest

import sl_inputs as I

WORLD = 2
PER_RANK = 6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_dir):
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(WORLD))
    import torch
    import bench
    import oracle

    dist, r, world = bench._dist("gloo")
    assert (r, world) == (rank, WORLD)
    pb = I.config1()
    pb = I.with_(pb, steps=5)
    s0 = bench.shard_sample0(r, PER_RANK)
    res = oracle.run(pb, s0=s0, ns=PER_RANK, want_sums=True)
    sums = torch.tensor(np.stack([res["sum"], res["sumsq"]]))
    dist.all_reduce(sums)  # test only: combine the shards to compare with one run
    slowest = bench.max_over_ranks(1.0 + r, dist)
    rate = bench.whole_job_rate(100.0, world, slowest)
    np.save(os.path.join(out_dir, f"rank{r}.npy"), np.concatenate([sums.numpy().ravel(), [slowest, rate]]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_samples_and_take_the_slowest(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    import oracle

    oracle.build()  # once, before the ranks load it
    port = _free_port()
    mp.start_processes(_rank_main, args=(port, str(tmp_path)), nprocs=WORLD, start_method="spawn", join=True)
    pb = I.with_(I.config1(), steps=5)
    whole = oracle.run(pb, s0=0, ns=WORLD * PER_RANK, want_sums=True)
    ref = np.concatenate([whole["sum"].ravel(), whole["sumsq"].ravel()])
    for r in range(WORLD):
        got = np.load(tmp_path / f"rank{r}.npy")
        sums, slowest, rate = got[:-2], got[-2], got[-1]
        np.testing.assert_allclose(sums, ref, rtol=1e-13, atol=1e-13)
        assert slowest == 2.0  # the slower of the two ranks (1 s and 2 s)
        assert rate == WORLD * 100.0 / 2.0
