"""The multi-rank path on CPU: two gloo ranks.

Each rank holds a contiguous range of the global samples
(``shard.sample_range``) and advances it with no collective on the data
path; the job's time is the slowest rank's (``bench.max_over_ranks``) and
its rate counts every rank's units (``bench.whole_job_rate``).  The moments
take one exchange: every rank's chunk partial sums (64 samples per chunk),
gathered in rank order by the product's ``shard.gather_partials`` over
torch.distributed.  Because the Wiener increments are keyed on the global
sample index, the gathered table must equal the table of one run over all
samples, chunk for chunk and bit for bit, and its chunks added in order give
that run's moments.  The per-rank states come from the FP64 oracle here (no
GPU on this machine); ``tests/test_gpu_shard.py`` runs the same exchange on
the library's partial and combine kernels."""

import os
import socket

import numpy as np
import pytest

import sl_inputs as I

WORLD = 2
M_TOTAL = 150  # chunks of 64, 64, 22: rank 0 holds the first, rank 1 the other two
STEPS = 5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _chunk_table(states, chunk=64):
    """[nchunks][V] sums and sums of squares over consecutive sample chunks."""
    M = states.shape[0]
    flat = states.reshape(M, -1)
    ps, pq = [], []
    for c0 in range(0, M, chunk):
        blk = flat[c0:c0 + chunk]
        ps.append(blk.sum(axis=0))
        pq.append((blk * blk).sum(axis=0))
    return np.array(ps), np.array(pq)


def _rank_main(rank, port, out_dir):
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(WORLD))
    import torch
    import bench
    import oracle
    from paper_2009_07340_gb300 import shard

    dist, r, world = bench._dist("gloo")
    assert (r, world) == (rank, WORLD)
    pb = I.with_(I.config1(), steps=STEPS)
    s0, m = shard.sample_range(r, world, M_TOTAL)
    states = oracle.run(pb, s0=s0, ns=m, want_states=True, want_sums=False)["states"]
    ps, pq = _chunk_table(states)
    gs, gq = shard.gather_partials(torch.from_numpy(ps), torch.from_numpy(pq), dist)
    slowest = bench.max_over_ranks(1.0 + r, dist)
    rate = bench.whole_job_rate(100.0, world, slowest)
    np.savez(os.path.join(out_dir, f"rank{r}.npz"), psum=gs.numpy(), psq=gq.numpy(), slowest=slowest, rate=rate,
             s0=s0, m=m)
    dist.barrier()
    dist.destroy_process_group()


def test_sample_ranges():
    from paper_2009_07340_gb300 import shard

    assert [shard.sample_range(r, 2, 150) for r in range(2)] == [(0, 64), (64, 86)]
    assert [shard.sample_range(r, 4, 4096 * 4) for r in range(4)] == [(4096 * r, 4096) for r in range(4)]
    for world, M in ((3, 1000), (8, 8 * 64 + 5), (1, 7)):
        ranges = [shard.sample_range(r, world, M) for r in range(world)]
        assert ranges[0][0] == 0 and sum(m for _, m in ranges) == M
        for (a, m), (b, _) in zip(ranges, ranges[1:]):
            assert a + m == b and b % 64 == 0
    with pytest.raises(ValueError):
        shard.sample_range(3, 4, 130)  # three chunks cannot give four ranks one each


def test_two_gloo_ranks_gather_moment_partials(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    import oracle

    oracle.build()  # once, before the ranks load it
    port = _free_port()
    mp.start_processes(_rank_main, args=(port, str(tmp_path)), nprocs=WORLD, start_method="spawn", join=True)
    pb = I.with_(I.config1(), steps=STEPS)
    whole = oracle.run(pb, s0=0, ns=M_TOTAL, want_states=True, want_sums=True)
    ref_s, ref_q = _chunk_table(whole["states"])
    for r in range(WORLD):
        got = np.load(tmp_path / f"rank{r}.npz")
        # every rank holds the whole table, in global sample order, bit for bit
        assert got["psum"].shape == (3, ref_s.shape[1])
        assert np.array_equal(got["psum"], ref_s) and np.array_equal(got["psq"], ref_q)
        # its chunks added in order are the moments of one run over all samples
        a = np.zeros(ref_s.shape[1])
        for row in got["psum"]:
            a = a + row
        np.testing.assert_allclose(a / M_TOTAL, whole["sum"].ravel() / M_TOTAL, rtol=1e-14, atol=1e-15)
        assert float(got["slowest"]) == 2.0  # the slower of the two ranks (1 s and 2 s)
        assert float(got["rate"]) == WORLD * 100.0 / 2.0
