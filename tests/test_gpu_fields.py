"""Fields changed between steps (sl_set_fields: a time-dependent or coupled
flow) on the GPU, against the oracle run segment by segment with the same
fields, continuing the step counter."""

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


def _segments_1d():
    return [(("sin", [1.0, 0.5, 1.0]), ("cos", [0.01, 0.5, 1.0])),
            (("sin", [0.8, -0.3, 2.0]), ("const", [0.02])),
            (("const", [-0.5, 0.0]), ("cos", [0.005, -0.5, 2.0]))]


def _oracle_chain(orc, pb, segments, k):
    st = None
    for i, (u, D) in enumerate(segments):
        q = I.with_(pb, drift=u, diffusion=D)
        st = orc.run(q, nsteps=k, step0=i * k, state_in=st, want_states=True, ns=pb["M"])["states"]
    return st


def _gpu_chain(sl, pb, segments, k, precision):
    with sl.Solver(I.with_(pb, drift=segments[0][0], diffusion=segments[0][1]), precision) as s:
        for i, (u, D) in enumerate(segments):
            if i:
                s.set_fields(u, D)
            s.step(pb["dt"], k)
        return s.samples(), s.dt_max


def test_1d_fields_switched_between_steps(sl, orc):
    segs = _segments_1d()
    pb = I.config2(N=8, M=5, steps=0, K=32)
    pb["dt"] = 0.4 * min(orc.dt_max(I.with_(pb, drift=u, diffusion=D)) for u, D in segs)
    ref = _oracle_chain(orc, pb, segs, 5)
    st, dtmax = _gpu_chain(sl, pb, segs, 5, "fp64")
    assert np.abs(st - ref).max() / np.abs(ref).max() <= FP64_TOL
    assert dtmax == pytest.approx(orc.dt_max(I.with_(pb, drift=segs[-1][0], diffusion=segs[-1][1])), rel=1e-12)
    st32, _ = _gpu_chain(sl, pb, segs, 5, "fp32")
    assert np.abs(st32 - st).max() / np.abs(st).max() <= MIXED_TOL


def test_2d_fields_switched_between_steps(sl, orc):
    segs = [(("rotation", [2 * np.pi, 0.5, 0.5]), ("const", [0.003])),
            (("const", [0.4, -0.7]), ("sinsin", [0.004, 0.3, 2.0, 2.0]))]
    pb = I.problem(2, (4, 3), (0.0, 0.0), (1.0, 1.0), 4, 3, 0, 0.0, 8, segs[0][0], segs[0][1],
                   ("gauss", [1.0, 0.2, 0.5, 0.5]))
    pb["dt"] = 0.4 * min(orc.dt_edge(I.with_(pb, drift=u, diffusion=D)) for u, D in segs)
    ref = _oracle_chain(orc, pb, segs, 3)
    st, _ = _gpu_chain(sl, pb, segs, 3, "fp64")
    assert np.abs(st - ref).max() / np.abs(ref).max() <= FP64_TOL


def test_invalid_fields_rejected(sl):
    with sl.Solver(I.config2(N=4, M=2, steps=0, K=4), "fp64") as s:
        with pytest.raises(sl.SLError) as e:
            s.set_fields(("rotation", [1.0, 0.5, 0.5]), ("const", [0.01]))  # 2D drift on a 1D mesh
        assert e.value.code == -1
        with pytest.raises(sl.SLError):
            s.set_fields(("const", [1.0, 0.0]), ("const", [-0.01]))  # D < 0
