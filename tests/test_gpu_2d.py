"""GPU parity of the 2D path (tensor-product elements) against the FP64 CPU
oracle, through the C ABI.  SL_FP64 within 1e-10 of the oracle; the FP32
path (float-pair state, FP32 Gram solve, one refinement step) within 1e-5 of
the FP64 path on the moments.  Orders up to 12 (FP32) and 11 (FP64), the
high ones with each Gram row split over several lanes."""

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


def _rel(a, b, scale=None):
    scale = np.abs(b).max() if scale is None else scale
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / scale)


def _rot(K=(4, 4), N=4, M=3, steps=4, frac=0.5, orc=None):
    pb = I.problem(2, K, (0.0, 0.0), (1.0, 1.0), N, M, steps, 0.0, 31,
                   ("rotation", [2 * np.pi, 0.5, 0.5]), ("sinsin", [0.005, 0.3, 2.0, 2.0]),
                   ("gauss", [1.0, 0.15, 0.5, 0.65]))
    pb["dt"] = frac * orc.dt_max(pb)
    return pb


def _pair(sl, orc, pb, precision="fp64", states=None):
    states = pb["M"] if states is None else states
    ref = orc.run(pb, want_states=True, nthreads=8, ns=pb["M"])
    with sl.Solver(pb, precision) as s:
        s.step()
        mean, m2 = s.moments()
        st = s.samples(0, states)
    M = pb["M"]
    rm = ref["sum"] / M
    scale = np.abs(rm).max()
    return _rel(mean, rm, scale), _rel(m2, ref["sumsq"] / M), _rel(st, ref["states"][:states], scale)


@pytest.mark.parametrize("N", [2, 3, 4, 6, 8])
def test_rotation_fp64(sl, orc, N):
    pb = _rot(N=N, orc=orc)
    e_mean, e_m2, e_st = _pair(sl, orc, pb)
    assert e_mean <= FP64_TOL and e_m2 <= FP64_TOL and e_st <= FP64_TOL


def test_constant_drift_nonsquare_fp64(sl, orc):
    pb = I.problem(2, (5, 3), (0.0, -1.0), (2.0, 1.0), 5, 7, 6, 0.0, 9, ("const", [0.7, -0.4]),
                   ("const", [0.002]), ("gauss", [1.0, 0.3, 1.0, 0.2]))
    pb["dt"] = 0.5 * orc.dt_max(pb)
    e_mean, e_m2, e_st = _pair(sl, orc, pb)
    assert e_mean <= FP64_TOL and e_st <= FP64_TOL


def test_config3_mesh_fp64_sampled(sl, orc):
    # the full 64x64, N=8 mesh of the 2D workload at its dt, 2 samples, 2 steps
    pb = I.config3(M=2, steps=2)
    e_mean, _, e_st = _pair(sl, orc, pb)
    assert e_mean <= FP64_TOL and e_st <= FP64_TOL


@pytest.mark.parametrize("N", [4, 6, 8])
def test_fp32_vs_fp64(sl, orc, N):
    pb = _rot(K=(12, 12), N=N, M=64, steps=40, orc=orc)
    with sl.Solver(pb, "fp64") as s:
        s.step()
        m64, _ = s.moments()
    with sl.Solver(pb, "fp32") as s:
        s.step()
        m32, _ = s.moments()
    assert _rel(m32, m64) <= MIXED_TOL


def test_config3_mesh_fp32_vs_fp64_edge_dt(sl, orc):
    # the 64x64, N=8 mesh at the edge-distance dt, 32 samples, 20 steps
    pb = I.config3(M=32, steps=20, dt=I.DT_CFG3_EDGE)
    with sl.Solver(pb, "fp64") as s:
        assert s.dt_edge == pytest.approx(orc.dt_edge(pb), rel=1e-12)
        assert s.dt_max == pytest.approx(orc.dt_max(pb), rel=1e-12)
        s.step()
        m64, _ = s.moments()
        s0 = s.samples(0, 1)[0]
    with sl.Solver(pb, "fp32") as s:
        s.step()
        m32, _ = s.moments()
    assert _rel(m32, m64) <= MIXED_TOL
    ref = orc.run(I.with_(pb, steps=3), ns=1, want_states=True)["states"][0]
    with sl.Solver(pb, "fp64") as s:
        s.step(steps=3)
        assert _rel(s.samples(0, 1)[0], ref) <= FP64_TOL


def test_config3_full_mesh_fp32_vs_oracle(sl, orc):
    # the full 64x64, N=8 mesh at the edge-distance dt: 16 samples, 6 steps,
    # FP32 moments and states against the oracle
    pb = I.config3(M=16, steps=6, dt=I.DT_CFG3_EDGE)
    e_mean, e_m2, e_st = _pair(sl, orc, pb, precision="fp32", states=16)
    assert e_mean <= MIXED_TOL and e_m2 <= MIXED_TOL and e_st <= MIXED_TOL


_ORACLE_CFG3_HALF = {}


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
def test_config3_full_mesh_at_half_node_gap_vs_oracle(sl, orc, precision):
    # the full mesh at config 3's time step (half the particle-gap bound: the
    # bound itself is unstable in 2D), 16 samples, 6 steps.  The mixed form
    # factors the remap's capacitance matrix in FP64 (the rest in FP32).
    pb = I.config3(M=16, steps=6, dt=I.DT_CFG3_HALF)
    if "ref" not in _ORACLE_CFG3_HALF:
        _ORACLE_CFG3_HALF["ref"] = orc.run(pb, want_states=True, nthreads=8, ns=pb["M"])
    ref = _ORACLE_CFG3_HALF["ref"]
    with sl.Solver(pb, precision) as s:
        s.step()
        mean, m2 = s.moments()
        st = s.samples()
    rm = ref["sum"] / pb["M"]
    scale = np.abs(rm).max()
    assert _rel(mean, rm, scale) <= MIXED_TOL
    assert _rel(m2, ref["sumsq"] / pb["M"]) <= MIXED_TOL
    assert _rel(st, ref["states"], scale) <= MIXED_TOL


@pytest.mark.parametrize("N", [4, 8, 12])
def test_mixed_factor_in_fp64_vs_oracle(sl, orc, N):
    # the mixed form runs its own remap kernel (the capacitance matrix in
    # FP64): its states differ from the FP32 form's in the last bits, and
    # both are within the mixed tolerance of the oracle
    pb = _rot(K=(8, 8), N=N, M=8, steps=3, orc=orc)
    pb["dt"] = 0.5 * orc.dt_edge(pb)
    ref = orc.run(pb, want_states=True, nthreads=8, ns=pb["M"])["states"]
    out = {}
    for precision in ("mixed", "fp32"):
        with sl.Solver(pb, precision) as s:
            s.step()
            out[precision] = s.samples()
            assert s.fallbacks == (0, 0)
        assert _rel(out[precision], ref, np.abs(ref).max()) <= MIXED_TOL
    assert not np.array_equal(out["mixed"], out["fp32"])


@pytest.mark.parametrize("precision,N", [("fp32", 9), ("fp32", 10), ("fp32", 11), ("fp32", 12),
                                         ("fp64", 9), ("fp64", 10), ("fp64", 11)])
def test_high_order_launch_geometry_vs_oracle(sl, orc, precision, N):
    # an 8x8 mesh with 8 samples: 512 element-sample groups, more CTAs than
    # SMs at every order, several groups per CTA where the order allows it
    # (FP32 per-sample states at half the edge-distance bound: at the node-gap
    # bound a sample with a large increment leaves FP32 far less accurate)
    pb = _rot(K=(8, 8), N=N, M=8, steps=3, orc=orc)
    if precision == "fp32":
        pb["dt"] = 0.5 * orc.dt_edge(pb)
    e_mean, e_m2, e_st = _pair(sl, orc, pb, precision=precision, states=8)
    tol = FP64_TOL if precision == "fp64" else MIXED_TOL
    assert e_mean <= tol and e_m2 <= tol and e_st <= tol


@pytest.mark.parametrize("precision,N", [("fp32", 8), ("fp32", 9), ("fp32", 12), ("fp64", 10), ("fp64", 11)])
def test_fast_path_finishes_every_group_at_half_edge_dt(sl, orc, precision, N):
    # particles a fraction of the node gap from their nodes: the tensor-
    # preconditioned iteration converges for every element-sample in both
    # phases, and no group goes to the direct solve
    pb = _rot(K=(8, 8), N=N, M=8, steps=3, orc=orc)
    pb["dt"] = 0.5 * orc.dt_edge(pb)
    with sl.Solver(pb, precision) as s:
        s.step()
        assert s.fallbacks == (0, 0)


@pytest.mark.parametrize("N", [4, 10])
def test_fast_and_direct_solves_mix_vs_oracle(sl, orc, N):
    # at the node-gap bound the conditioning test sends a share of the
    # element-samples to the direct solve (in both phases at N = 4, in the
    # remap at N = 10): each step runs both kernels on disjoint groups, the
    # remap's iteration starting from interpolants either kernel formed, and
    # still matches the oracle
    pb = _rot(K=(8, 8), N=N, M=8, steps=3, orc=orc)
    pb["dt"] = orc.dt_max(pb)
    ref = orc.run(pb, want_states=True, nthreads=8, ns=pb["M"])
    with sl.Solver(pb, "fp64") as s:
        s.step()
        f1, f2 = s.fallbacks
        st = s.samples()
    groups = 64 * pb["M"] * pb["steps"]
    assert 0 < f2 < groups and (N > 4 or 0 < f1 < groups)
    assert _rel(st, ref["states"], np.abs(ref["states"]).max()) <= FP64_TOL


@pytest.mark.parametrize("N", [9, 10, 11, 12])
def test_fp32_high_order_vs_oracle(sl, orc, N):
    # N = 11, 12: each Gram row split over four lanes
    pb = _rot(K=(3, 3), N=N, M=2, steps=3, orc=orc)
    e_mean, _, e_st = _pair(sl, orc, pb, precision="fp32")
    assert e_mean <= MIXED_TOL and e_st <= MIXED_TOL


@pytest.mark.parametrize("N", [9, 10, 11])
def test_fp64_high_order_vs_oracle(sl, orc, N):
    # N = 9, 10: each Gram row split over two lanes; N = 11: four
    pb = _rot(K=(3, 2), N=N, M=3, steps=3, orc=orc)
    e_mean, e_m2, e_st = _pair(sl, orc, pb)
    assert e_mean <= FP64_TOL and e_m2 <= FP64_TOL and e_st <= FP64_TOL


@pytest.mark.parametrize("N", [10, 11])
def test_fp32_vs_fp64_high_order(sl, orc, N):
    pb = _rot(K=(4, 4), N=N, M=16, steps=10, orc=orc)
    with sl.Solver(pb, "fp64") as s:
        s.step()
        m64, _ = s.moments()
    with sl.Solver(pb, "fp32") as s:
        s.step()
        m32, _ = s.moments()
    assert _rel(m32, m64) <= MIXED_TOL


def test_order_limits(sl, orc):
    pb = _rot(K=(2, 2), N=12, M=1, steps=1, orc=orc)
    with pytest.raises(sl.SLError) as e:
        sl.Solver(pb, "fp64")
    assert e.value.code == -8
    pb = _rot(K=(2, 2), N=13, M=1, steps=1, orc=orc)
    with pytest.raises(sl.SLError) as e:
        sl.Solver(pb, "fp32")
    assert e.value.code == -8


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_launch_chunk_is_bitwise_neutral(sl, orc, precision):
    # a step split into launches of 7 element-sample groups (ragged: 4*4*5 = 80
    # groups, at most 2 launches queued) equals the step in one launch per
    # phase, bit for bit
    pb = _rot(K=(4, 4), N=5, M=5, steps=6, orc=orc)
    with sl.Solver(pb, precision) as s:
        s.step()
        whole = s.samples()
    for chunk in (7, 80, 1000):
        with sl.Solver(pb, precision, launch_chunk=chunk) as s:
            s.step()
            assert np.array_equal(s.samples(), whole), chunk
