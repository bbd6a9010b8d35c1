"""The boundary-row weight w of the remap (sl_options.bc_weight) on the GPU,
against the FP64 oracle: weighted rows in 1D and 2D, and hard face
constraints (w = inf) in 1D."""

import numpy as np
import pytest

import sl_inputs as I

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-5


@pytest.fixture(scope="module")
def sl():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_07340_gb300 import build

    build.build()
    import paper_2009_07340_gb300 as sl

    return sl


def _pb1(orc, w, N=6, K=24, M=7, steps=10):
    pb = I.config2(N=N, M=M, steps=steps, K=K)
    pb["bc_weight"] = w
    pb["dt"] = 0.5 * orc.dt_max(pb)
    return pb


def _rel_vs_oracle(sl, orc, pb, precision="fp64"):
    ref = orc.run(pb, want_states=True, nthreads=8, ns=pb["M"])
    with sl.Solver(pb, precision) as s:
        s.step()
        st = s.samples()
    ref_st = ref["states"].reshape(st.shape)
    return float(np.abs(st - ref_st).max() / np.abs(ref_st).max())


@pytest.mark.parametrize("w", [np.inf, 0.5, 3.0])
@pytest.mark.parametrize("N", [4, 9])
def test_1d_weighted_and_hard_fp64(sl, orc, w, N):
    assert _rel_vs_oracle(sl, orc, _pb1(orc, w, N=N)) <= FP64_TOL


def test_1d_hard_fp32_vs_fp64(sl, orc):
    pb = _pb1(orc, np.inf, N=8, K=64, M=64, steps=40)
    with sl.Solver(pb, "fp64") as s:
        s.step()
        m64, _ = s.moments()
    for precision in ("fp32", "mixed"):
        with sl.Solver(pb, precision) as s:
            s.step()
            m, _ = s.moments()
        assert np.abs(m - m64).max() / np.abs(m64).max() <= MIXED_TOL, precision


def test_batch_with_a_hard_instance_equals_alone(sl, orc):
    pbs = [_pb1(orc, np.inf, N=5, K=16, M=4), _pb1(orc, 0.0, N=5, K=40, M=3)]
    with sl.Batch(pbs, "fp64") as b:
        b.step(6)
        for i, pb in enumerate(pbs):
            with sl.Solver(pb, "fp64") as s:
                s.step(pb["dt"], 6)
                assert np.array_equal(b.samples(i), s.samples().reshape(pb["M"], -1)), i


def _pb2(orc, w, N=4):
    pb = I.problem(2, (4, 3), (0.0, 0.0), (1.0, 1.0), N, 5, 4, 0.0, 77, ("rotation", [2 * np.pi, 0.5, 0.5]),
                   ("const", [0.003]), ("gauss", [1.0, 0.2, 0.5, 0.5]))
    pb["bc_weight"] = w
    pb["dt"] = 0.5 * orc.dt_edge(pb)
    return pb


@pytest.mark.parametrize("N", [3, 5])
def test_2d_weighted_fp64(sl, orc, N):
    assert _rel_vs_oracle(sl, orc, _pb2(orc, 2.5, N=N)) <= FP64_TOL


def test_2d_hard_constraints_unsupported(sl, orc):
    with pytest.raises(sl.SLError) as e:
        sl.Solver(_pb2(orc, np.inf), "fp64")
    assert e.value.code == -8
