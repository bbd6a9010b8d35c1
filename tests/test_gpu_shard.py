"""Samples split over contexts (as over GPUs) and recombined by the library:
chunk partial sums (sl_moments_partial) of disjoint sample ranges, taken in
global sample order and added by sl_moments_combine, reproduce the moments
of one context holding every sample, bit for bit (Eq. averaged)."""

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


@pytest.mark.parametrize("precision,pb", [
    ("fp64", I.config2(N=8, M=150, steps=12, K=24)),
    ("fp32", I.config2(N=8, M=150, steps=12, K=24)),
    ("fp64", I.config3(M=70, steps=2, K=6, N=5)),
])
def test_shards_recombine_bitwise(sl, precision, pb):
    import torch

    from paper_2009_07340_gb300 import shard

    M = pb["M"]
    with sl.Solver(pb, precision) as whole:
        whole.step()
        ref_mean, ref_m2 = whole.moments()
        mean1, m21 = shard.global_moments(whole, M)  # one rank: no exchange
        assert np.array_equal(mean1.cpu().numpy(), ref_mean.ravel())
        assert np.array_equal(m21.cpu().numpy(), ref_m2.ravel())
    world = 2
    parts_s, parts_q = [], []
    for r in range(world):
        s0, m = shard.sample_range(r, world, M)
        with sl.Solver(I.with_(pb, M=m), precision, sample0=s0) as s:
            s.step()
            nc = shard.n_chunks(m)
            ps = torch.empty((nc, s.V), dtype=torch.float64, device="cuda")
            pq = torch.empty_like(ps)
            s.moments_partial(ps, pq)
            torch.cuda.synchronize()
            parts_s.append(ps)
            parts_q.append(pq)
    aps, apq = torch.cat(parts_s).contiguous(), torch.cat(parts_q).contiguous()
    V = aps.shape[1]
    mean = torch.empty(V, dtype=torch.float64, device="cuda")
    m2 = torch.empty_like(mean)
    sl.sl_moments_combine(aps.data_ptr(), apq.data_ptr(), aps.shape[0], V, M, mean.data_ptr(), m2.data_ptr())
    torch.cuda.synchronize()
    assert np.array_equal(mean.cpu().numpy(), ref_mean.ravel())
    assert np.array_equal(m2.cpu().numpy(), ref_m2.ravel())


def test_partial_and_combine_arguments(sl):
    import torch

    pb = I.with_(I.config1(), M=70, steps=1)
    with sl.Solver(pb) as s:
        bad = torch.empty((1, s.V), dtype=torch.float64, device="cuda")  # 70 samples need 2 chunks
        with pytest.raises(ValueError):
            s.moments_partial(bad, bad)
    assert sl.sl_moment_chunk() == 64
    with pytest.raises(sl.SLError):
        sl.sl_moments_combine(0, 0, 1, 4, 4, 0)
