"""Edge cases of the 1D path on the GPU, through the C ABI: the largest mesh
(a cluster of 8 CTAs), degenerate fields (no diffusion, no drift), an empty
step, a single sample."""

import numpy as np
import pytest

import sl_inputs as I

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


@pytest.fixture(scope="module")
def sl():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_07340_gb300 import build

    build.build()
    import paper_2009_07340_gb300 as sl

    return sl


def _vs_oracle(sl, orc, pb, precision="fp64"):
    ref = orc.run(pb, want_states=True, nthreads=8, ns=pb["M"])
    with sl.Solver(pb, precision) as s:
        s.step()
        st = s.samples()
        mean, _ = s.moments()
    scale = np.abs(ref["states"]).max()
    return (float(np.abs(st - ref["states"].reshape(st.shape)).max() / scale),
            float(np.abs(mean.ravel() - ref["sum"].ravel() / pb["M"]).max() / scale), st, mean)


def test_largest_mesh_2048_elements(sl, orc):
    pb = I.config2(N=4, M=2, steps=4, K=2048)
    pb["dt"] = 0.5 * orc.dt_max(pb)
    e_st, e_mean, _, m64 = _vs_oracle(sl, orc, pb)
    assert e_st <= FP64_TOL and e_mean <= FP64_TOL
    with sl.Solver(pb, "fp32") as s:
        s.step()
        m32, _ = s.moments()
    assert np.abs(m32 - m64).max() / np.abs(m64).max() <= 1e-5


def test_no_diffusion_every_sample_identical(sl, orc):
    pb = I.config2(N=8, M=5, steps=20, K=16)
    pb["diffusion"] = ("cos", [0.0, 0.5, 1.0])  # D = 0: the Wiener increments have no effect
    pb["dt"] = 0.5 * orc.dt_max(pb)
    e_st, e_mean, st, _ = _vs_oracle(sl, orc, pb)
    assert e_st <= FP64_TOL and e_mean <= FP64_TOL
    assert all(np.array_equal(st[0], st[s]) for s in range(1, pb["M"]))


def test_no_drift_pure_diffusion(sl, orc):
    pb = I.config2(N=6, M=7, steps=15, K=12)
    pb["drift"] = ("const", [0.0, 0.0])
    pb["dt"] = 0.5 * orc.dt_max(pb)
    e_st, e_mean, _, _ = _vs_oracle(sl, orc, pb)
    assert e_st <= FP64_TOL and e_mean <= FP64_TOL


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_zero_steps_changes_nothing(sl, orc, precision):
    pb = I.config2(N=5, M=3, steps=0, K=9)
    with sl.Solver(pb, precision) as s:
        before = s.samples()
        s.step(dt=1e-6, steps=0)
        assert s.step_count == 0
        assert np.array_equal(s.samples(), before)


def test_single_sample_moments(sl, orc):
    pb = I.config2(N=7, M=1, steps=6, K=10)
    pb["dt"] = 0.5 * orc.dt_max(pb)
    with sl.Solver(pb, "fp64") as s:
        s.step()
        mean, m2 = s.moments()
        q = s.samples()[0]
    assert np.array_equal(mean, q)
    np.testing.assert_allclose(m2, q * q, rtol=1e-15, atol=0)


@pytest.mark.parametrize("dim,precision", [(1, "fp64"), (1, "fp32"), (1, "mixed"), (2, "fp64"), (2, "fp32")])
def test_nonfinite_remap_reports_singular_and_poisons(sl, orc, dim, precision):
    """A non-finite value in the state makes that element's remap non-finite:
    the step reports SL_ERR_SINGULAR (-5) at the next synchronising call
    instead of returning NaN moments, and the context then refuses further
    calls with SL_ERR_STATE (-7)."""
    if dim == 1:
        pb = I.config2(N=6, M=3, steps=2, K=8)
        pb["dt"] = 0.5 * orc.dt_max(pb)
    else:
        pb = I.problem(2, (2, 2), (0.0, 0.0), (1.0, 1.0), 4, 3, 2, 0.0, 5, ("const", [0.3, -0.2]),
                       ("const", [0.004]), ("gauss", [1.0, 0.2, 0.5, 0.5]))
        pb["dt"] = 0.5 * orc.dt_edge(pb)
    q = orc.init_state(pb)
    q[1, 2] = np.nan
    with sl.Solver(pb, precision, phi0_nodal=q) as s:
        s.step()
        with pytest.raises(sl.SLError) as e:
            s.moments()
        assert e.value.code == -5
        with pytest.raises(sl.SLError) as e:
            s.step()
        assert e.value.code == -7
