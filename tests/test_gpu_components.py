"""Two scalar fields per sample sharing the particles and so the remap
factorization (sl_options.components = 2), in 1D and in 2D.  The components do not interact,
so each must be exactly the single-field run started from that component's
initial values: same Wiener increments, same shared arithmetic."""

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


def _pair_of_fields(orc, K, N, M, steps):
    pa = I.config2(N=N, M=M, steps=steps, K=K)
    pa["dt"] = 0.5 * orc.dt_max(pa)
    pb = I.with_(pa, phi0=I.fourier_phi0(7))  # a second initial field, same particles
    return pa, orc.init_state(pa), orc.init_state(pb)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("K,N,M", [(24, 6, 9), (64, 12, 5), (300, 5, 3), (16, 16, 4)])
def test_two_components_equal_two_single_runs(sl, orc, precision, K, N, M):
    pa, qa, qb = _pair_of_fields(orc, K, N, M, 12)
    with sl.Solver(pa, precision, phi0_nodal=qa) as s:
        s.step()
        ref_a = s.samples()
    with sl.Solver(pa, precision, phi0_nodal=qb) as s:
        s.step()
        ref_b = s.samples()
    with sl.Solver(I.with_(pa, components=2), precision) as s:
        s.set_samples(0, np.stack([np.stack([qa, qb])] * M))
        s.step()
        st = s.samples()
        mean, _ = s.moments()
    assert st.shape == (M, 2, K, N)
    assert np.array_equal(st[:, 0], ref_a) and np.array_equal(st[:, 1], ref_b)
    np.testing.assert_allclose(mean[1], ref_b.mean(axis=0), rtol=1e-12, atol=0)
    if precision == "fp64":
        ref = orc.run(pa, want_states=True, nthreads=8, ns=M)["states"]
        assert np.abs(st[:, 0] - ref).max() / np.abs(ref).max() <= FP64_TOL


def _pair_of_fields_2d(orc, K, N, M, steps):
    pa = I.problem(2, K, (0.0, 0.0), (1.0, 1.0), N, M, steps, 0.0, 41, ("rotation", [2 * np.pi, 0.5, 0.5]),
                   ("sinsin", [0.004, 0.3, 2.0, 2.0]), ("gauss", [1.0, 0.15, 0.5, 0.6]))
    pa["dt"] = 0.5 * orc.dt_edge(pa)
    pb = I.with_(pa, phi0=("sinsin", [1.0, 0.4, 1.0]))  # a second initial field, same particles
    return pa, orc.init_state(pa), orc.init_state(pb)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("K,N,M", [((3, 2), 4, 5), ((2, 3), 6, 3), ((2, 2), 8, 3)])
def test_two_components_2d_equal_two_single_runs(sl, orc, precision, K, N, M):
    """2D: one Gram matrix and one elimination serve both fields; each field
    is bit for bit its own single-field run."""
    pa, qa, qb = _pair_of_fields_2d(orc, K, N, M, 4)
    refs = []
    for q in (qa, qb):
        with sl.Solver(pa, precision, phi0_nodal=q) as s:
            s.step()
            refs.append(s.samples())
    with sl.Solver(I.with_(pa, components=2), precision) as s:
        s.set_samples(0, np.stack([np.stack([qa, qb])] * M))
        s.step()
        st = s.samples()
        mean, _ = s.moments()
    E, n = K[0] * K[1], N * N
    assert st.shape == (M, 2, E, n)
    assert np.array_equal(st[:, 0], refs[0]) and np.array_equal(st[:, 1], refs[1])
    np.testing.assert_allclose(mean[1], refs[1].mean(axis=0), rtol=1e-12, atol=0)
    if precision == "fp64":
        ref = orc.run(pa, want_states=True, nthreads=8, ns=M)["states"]
        assert np.abs(st[:, 0] - ref).max() / np.abs(ref).max() <= FP64_TOL


def test_components_unsupported_combinations(sl, orc):
    pa, _, _ = _pair_of_fields(orc, 8, 4, 2, 1)
    for pb, precision in [(I.with_(pa, components=2), "mixed"), (I.with_(pa, components=3), "fp64"),
                          (I.with_(pa, components=2, periodic=False), "fp64")]:
        with pytest.raises(sl.SLError) as e:
            sl.Solver(pb, precision)
        assert e.value.code == -8
    p2 = I.problem(2, (2, 2), (0.0, 0.0), (1.0, 1.0), 9, 2, 1, 1e-4, 1, ("const", [0.1, 0.2]), ("const", [0.01]),
                   ("gauss", [1.0, 0.2, 0.5, 0.5]))
    for pb in (I.with_(p2, components=2), I.with_(p2, N=4, components=2, periodic=False)):  # 2D: N <= 8, periodic
        with pytest.raises(sl.SLError) as e:
            sl.Solver(pb, "fp64")
        assert e.value.code == -8
