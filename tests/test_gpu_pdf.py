"""PDF recovery by binning the samples at each node (sl_pdf) on the GPU,
against the oracle's binning of the same generated values: the counts are
integers decided in FP64 by the same formula, so they must agree bit for
bit."""

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


def _values(M, E, n, lo, hi, B, seed):
    """Float32-representable values (exact in the FP32 pair state too): a
    spread around [lo, hi], exact bin edges, lo, hi, out-of-range values and
    NaN."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(lo - 0.5, hi + 0.5, size=(M, E, n)).astype(np.float32).astype(np.float64)
    edges = np.linspace(lo, hi, B + 1)
    flat = x.reshape(-1)
    k = rng.choice(flat.size, size=min(flat.size, 40), replace=False)
    flat[k[:30]] = edges[rng.integers(0, B + 1, size=30)]
    flat[k[30:35]] = np.nan
    flat[k[35:]] = hi + 1.0
    return flat.reshape(M, E, n)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("B", [7, 64])
def test_pdf_counts_bit_exact(sl, orc, precision, B):
    pb = I.config2(N=6, M=37, steps=0, K=11)
    lo, hi = -1.0, 2.5
    x = _values(pb["M"], 11, 6, lo, hi, B, seed=B)
    with sl.Solver(pb, precision) as s:
        s.set_samples(0, x)
        got = s.pdf(B, lo, hi)
    assert np.array_equal(got, orc.pdf(x, B, lo, hi))


def test_pdf_at_scale_totals(sl, orc):
    # the config-2 field after a few steps: every sample lies in [0.4, 1.6]
    # (phi0 in [0.5, 1.5]), so every node counts all M samples
    pb = I.config2(N=8, M=4096, steps=5, K=256)
    pb["dt"] = I.DT_CFG2_HALF
    with sl.Solver(pb, "fp32") as s:
        s.step()
        c = s.pdf(100, 0.4, 1.6)
    assert c.shape == (256, 8, 100) and np.all(c.sum(axis=-1) == 4096)


def test_pdf_arguments(sl):
    with sl.Solver(I.config2(N=4, M=2, steps=0, K=4), "fp64") as s:
        for bad in [(0, 0.0, 1.0), (5000, 0.0, 1.0), (8, 1.0, 1.0), (8, 0.0, np.inf)]:
            with pytest.raises(sl.SLError) as e:
                s.pdf(*bad)
            assert e.value.code == -1
