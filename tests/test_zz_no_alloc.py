"""The allocation-free moments entry point (sl_moments_static), through the C ABI.

It serves callers that cannot call cudaMalloc when they need the moments (a
serving loop with its HBM budget reserved up front, code that must not let an
allocation synchronise the device, a framework owning all device memory).  The
test is the caller: it owns the input and output device buffers; the entry
point itself must allocate nothing and must agree with the context-based
sl_moments_device on two calls in a row (the second with different data, so a
stale scratch array would show).  This file sorts last so that a run stopping
at the first failure has already run every other test.
"""

import numpy as np
import pytest

import sl_inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-13  # moments of the same FP64 samples: summation order differences only


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_07340_gb300 import build

    build.build()
    import paper_2009_07340_gb300 as sl

    return torch, sl


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_matches_context_moments_on_two_calls(env):
    torch, sl = env
    pb = I.config2(N=8, M=300, steps=25, K=40)  # M not a multiple of the 64-sample chunk
    stream = torch.cuda.current_stream()
    with sl.Solver(pb, "fp64", stream=stream.cuda_stream) as s:
        V, M = s.V, s.M
        for call, nsteps in enumerate((10, 15)):
            s.step(steps=nsteps)
            ref_mean = torch.zeros(V, dtype=torch.float64, device="cuda")
            ref_m2 = torch.zeros(V, dtype=torch.float64, device="cuda")
            s.moments_device(ref_mean, ref_m2)
            samples = torch.from_numpy(s.samples().reshape(M, V)).cuda()
            out_mean = torch.full((V,), float("nan"), dtype=torch.float64, device="cuda")
            out_m2 = torch.full((V,), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            sl.sl_moments_static(samples.data_ptr(), M, V, out_mean.data_ptr(), out_m2.data_ptr(),
                                 stream.cuda_stream)
            torch.cuda.synchronize()
            assert _rel(out_mean.cpu().numpy(), ref_mean.cpu().numpy()) <= TOL, call
            assert _rel(out_m2.cpu().numpy(), ref_m2.cpu().numpy()) <= TOL, call


def test_long_chunks_and_size_limit(env):
    torch, sl = env
    # V = 2^16 nodes: only 16 chunks fit in the fixed scratch, so the
    # samples are summed in chunks of 188
    g = torch.Generator(device="cuda").manual_seed(7)
    M, V = 3000, 1 << 16
    x = torch.rand((M, V), dtype=torch.float64, device="cuda", generator=g)
    mean = torch.empty(V, dtype=torch.float64, device="cuda")
    m2 = torch.empty(V, dtype=torch.float64, device="cuda")
    for _ in range(2):
        sl.sl_moments_static(x.data_ptr(), M, V, mean.data_ptr(), m2.data_ptr())
        torch.cuda.synchronize()
        ref = x.mean(0).cpu().numpy()
        ref2 = (x * x).mean(0).cpu().numpy()
        assert _rel(mean.cpu().numpy(), ref) <= TOL
        assert _rel(m2.cpu().numpy(), ref2) <= TOL
    # sizes beyond the fixed scratch are refused before any launch
    with pytest.raises(sl.SLError) as e:
        sl.sl_moments_static(x.data_ptr(), 1, (1 << 20) + 1, mean.data_ptr())
    assert e.value.code == -1


def test_calls_allocate_no_device_memory(env):
    # after a first call (which looks up the scratch array's address), further
    # calls must leave the device's free memory and torch's allocator untouched
    torch, sl = env
    M, V = 500, 4096
    x = torch.rand((M, V), dtype=torch.float64, device="cuda")
    mean = torch.empty(V, dtype=torch.float64, device="cuda")
    m2 = torch.empty(V, dtype=torch.float64, device="cuda")
    sl.sl_moments_static(x.data_ptr(), M, V, mean.data_ptr(), m2.data_ptr())
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0, reserved0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    for _ in range(3):
        sl.sl_moments_static(x.data_ptr(), M, V, mean.data_ptr(), m2.data_ptr())
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert (torch.cuda.memory_allocated(), torch.cuda.memory_reserved()) == (alloc0, reserved0)
    assert _rel(mean.cpu().numpy(), x.mean(0).cpu().numpy()) <= TOL
