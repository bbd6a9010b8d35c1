"""Samples split over processes (one GPU each) and the one exchange it needs.

The Monte-Carlo samples are independent: each draws its own Wiener increment
per step and dimension, shared by all of its elements (Section 5.2), and
they meet only in the average of Eq. (averaged) (Section 5.4).  A solve over
M_total samples therefore splits into contiguous sample ranges, one per rank,
each advanced through the whole horizon with no communication (the Philox
counter is keyed on the global sample index, ``sl_options.sample0``).

The moments then take one exchange.  Every rank computes its chunk partial
sums (``sl_moments_partial``: sums over 64 consecutive samples); the ranks'
tables are gathered in rank order, which is ascending global sample order;
and the library's combine kernel (``sl_moments_combine``) adds the chunks in
that order and divides by M_total.  When every rank's first sample is a
multiple of 64 this is exactly the summation a single context over all
samples performs, so the result equals it bit for bit.

torch.distributed only moves the partial tables (NCCL for CUDA tensors, gloo
for CPU ones); every addition runs in the library's kernels.
"""

from __future__ import annotations

CHUNK = 64  # samples per partial-sum chunk (sl_moment_chunk)


def sample_range(rank, world, M_total):
    """(sample0, M_local) of `rank`: contiguous ranges in rank order, each
    starting at a multiple of CHUNK, the chunks split as evenly as possible
    (the last chunk may be short)."""
    if world < 1 or not 0 <= rank < world or M_total < 1:
        raise ValueError("need 0 <= rank < world and M_total >= 1")
    chunks = -(-M_total // CHUNK)
    if chunks < world:
        raise ValueError(f"{M_total} samples make {chunks} chunks of {CHUNK}: too few for {world} ranks")
    c0, c1 = rank * chunks // world, (rank + 1) * chunks // world
    s0, s1 = c0 * CHUNK, min(c1 * CHUNK, M_total)
    return s0, s1 - s0


def n_chunks(M):
    return -(-int(M) // CHUNK)


def gather_partials(psum, psq, dist=None, group=None):
    """All ranks' chunk tables [nchunks_r][V] in rank order, concatenated
    ([sum_r nchunks_r][V]); every rank receives the whole table.  psum and
    psq are torch tensors on the rank's device (CUDA under NCCL, CPU under
    gloo).  Without a process group (dist None or uninitialised) the local
    tables are returned as they are."""
    import torch

    if dist is None or not dist.is_available() or not dist.is_initialized():
        return psum, psq
    world = dist.get_world_size(group)
    dev = psum.device
    # ranks may hold different chunk counts: exchange the counts, pad to the
    # largest, gather, then drop the padding
    cnt = torch.tensor([psum.shape[0]], dtype=torch.int64, device=dev)
    counts = [torch.zeros_like(cnt) for _ in range(world)]
    dist.all_gather(counts, cnt, group=group)
    counts = [int(c.item()) for c in counts]
    cmax = max(counts)
    V = psum.shape[1]
    out = []
    for t in (psum, psq):
        pad = torch.zeros((cmax, V), dtype=torch.float64, device=dev)
        pad[: t.shape[0]] = t
        parts = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(parts, pad, group=group)
        out.append(torch.cat([p[:c] for p, c in zip(parts, counts)], dim=0).contiguous())
    return out[0], out[1]


def global_moments(solver, M_total, dist=None, group=None, stream=None):
    """Moments of Eq. (averaged) over every rank's samples: (mean, m2) as
    float64 CUDA tensors of the solver's node layout (flattened), the same
    on every rank.  `solver` is this rank's ``Solver`` (its sample0 a
    multiple of CHUNK); `stream` the CUDA stream (torch) to run on."""
    import torch

    from . import sl_moments_combine

    V = solver.V
    nc = n_chunks(solver.M)
    psum = torch.empty((nc, V), dtype=torch.float64, device="cuda")
    psq = torch.empty((nc, V), dtype=torch.float64, device="cuda")
    solver.moments_partial(psum, psq)
    # the partials were written on the solver's stream: finish them before
    # the collective and the combine, which run on torch's current stream
    torch.cuda.synchronize()
    apsum, apsq = gather_partials(psum, psq, dist, group)
    mean = torch.empty(V, dtype=torch.float64, device="cuda")
    m2 = torch.empty(V, dtype=torch.float64, device="cuda")
    if stream is None:  # the gathered tables are ordered on torch's current stream
        stream = torch.cuda.current_stream().cuda_stream
    sl_moments_combine(apsum.data_ptr(), apsq.data_ptr(), apsum.shape[0], V, int(M_total), mean.data_ptr(),
                       m2.data_ptr(), stream)
    return mean, m2
