"""Dirichlet boundaries (ghost values in the upwind rule at the domain
boundaries, Eq. bnd_update) and reseeding (Eq. re-seed) on the GPU, through
the C ABI, against the FP64 oracle."""

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


def _fourier(p, x):
    f = p[0] + 0 * x
    for m in range(int(p[2])):
        f = f + p[3 + 2 * m] * np.cos((m + 1) * p[1] * np.pi * x) + p[4 + 2 * m] * np.sin((m + 1) * p[1] * np.pi * x)
    return f


def _advection(u, M=3, steps=400, dt=1e-3, K=6, N=10):
    p = [1.0, 1.0, 2.0, 0.3, -0.2, 0.1, 0.15]
    pb = I.problem(1, (K,), (0.0,), (1.5,), N, M, steps, dt, 2, ("const", [u, 0.0]), ("const", [0.0]), ("fourier", p))
    pb["periodic"] = False
    t = dt * np.arange(1, steps + 1)
    pb["ghost"] = np.stack([_fourier(p, 0.0 - u * t), _fourier(p, 1.5 - u * t)], axis=1)
    return pb, p


@pytest.mark.parametrize("u", [1.0, -1.0])
def test_inflow_advection_fp64_vs_oracle_and_exact(sl, orc, u):
    pb, p = _advection(u)
    ref = orc.run(pb, ns=pb["M"], want_states=True)["states"]
    with sl.Solver(pb, "fp64") as s:
        s.step()
        st = s.samples()
    assert np.abs(st - ref).max() / np.abs(ref).max() <= FP64_TOL
    x, _ = orc.node_coords(pb)
    assert np.abs(st[0] - _fourier(p, x - u * pb["steps"] * pb["dt"])).max() <= 1e-7
    for precision in ("fp32", "mixed"):
        with sl.Solver(pb, precision) as s:
            s.step()
            assert np.abs(s.samples() - st).max() / np.abs(st).max() <= MIXED_TOL, precision


def _heat(x, t):
    return np.exp(-x * x / (4 * t)) / np.sqrt(4 * np.pi * t)


def _heat_problem(orc, M, steps, reseed, K=4, N=8):
    t0, dt = 0.05, 1e-5
    pb = I.problem(1, (K,), (-1.0,), (1.0,), N, M, steps, dt, 21, ("const", [0.0, 0.0]), ("const", [1.0]),
                   ("gauss", [1.0, 0.3, 0.0, 0.0]))
    pb["periodic"] = False
    pb["reseed_every"] = reseed
    t = t0 + dt * np.arange(1, steps + 1)
    pb["ghost"] = np.stack([_heat(-1.0, t), _heat(1.0, t)], axis=1)
    x, _ = orc.node_coords(pb)
    return pb, _heat(x, t0)


@pytest.mark.parametrize("reseed", [0, 50, 30])
def test_heat_kernel_with_reseeding(sl, orc, reseed):
    pb, phi0 = _heat_problem(orc, 64, 100, reseed)
    ref = orc.run(pb, ns=pb["M"], want_states=True, state_in=np.broadcast_to(phi0, (pb["M"],) + phi0.shape).copy(),
                  nthreads=8)["states"]
    with sl.Solver(pb, "fp64", phi0_nodal=phi0) as s:
        s.step()
        st = s.samples()
        mean64, _ = s.moments()
    assert np.abs(st - ref).max() / np.abs(ref).max() <= FP64_TOL
    if reseed and pb["steps"] % reseed == 0:  # the last step reseeded: every sample is the mean
        assert all(np.array_equal(st[0], st[k]) for k in range(1, pb["M"]))
    for precision in ("fp32", "mixed"):
        with sl.Solver(pb, precision, phi0_nodal=phi0) as s:
            s.step()
            m, _ = s.moments()
        assert np.abs(m - mean64).max() / np.abs(mean64).max() <= MIXED_TOL, precision


def test_dirichlet_on_a_cluster_mesh(sl, orc):
    pb = I.config2(N=5, M=3, steps=15, K=300)
    pb["periodic"] = False
    pb["dt"] = 0.5 * orc.dt_max(pb)
    pb["ghost"] = np.tile([0.8, 1.3], (15, 1))  # fixed boundary values
    ref = orc.run(pb, ns=3, want_states=True)["states"]
    with sl.Solver(pb, "fp64") as s:
        s.step()
        assert np.abs(s.samples() - ref).max() / np.abs(ref).max() <= FP64_TOL


def test_boundary_table_and_reseed_calls(sl, orc):
    pb, phi0 = _heat_problem(orc, 8, 10, 0)
    with sl.Solver(I.with_(pb, ghost=None), "fp64", phi0_nodal=phi0) as s:
        with pytest.raises(sl.SLError) as e:  # no boundary values yet
            s.step()
        assert e.value.code == -1
        s.set_boundary(pb["ghost"][:4])
        s.step(steps=4)
        with pytest.raises(sl.SLError):  # the table covers 4 steps only
            s.step(steps=1)
        s.set_boundary(pb["ghost"][4:])  # steps 4 .. 9
        s.step(steps=6)
        before, _ = s.moments()
        s.reseed()
        st = s.samples()
        mean, m2 = s.moments()
    assert all(np.array_equal(st[0], st[k]) for k in range(1, 8))
    assert np.abs(mean - before).max() <= 1e-15 * np.abs(before).max()
    np.testing.assert_allclose(m2, mean * mean, rtol=1e-14)
    with sl.Solver(I.config2(N=4, M=2, steps=1, K=8), "fp64") as s:  # periodic: no boundary table
        with pytest.raises(sl.SLError):
            s.set_boundary([[1.0, 1.0]])


def test_batch_and_server_reject_dirichlet(sl, orc):
    pb, _ = _advection(1.0, steps=2)
    pb["dt"] = 1e-3
    with pytest.raises(sl.SLError) as e:
        sl.Batch([pb], "fp64")
    assert e.value.code == -8
    with sl.Server(budget_bytes=1 << 26, precision="fp64") as srv:
        with pytest.raises(sl.SLError) as e:
            srv.submit(pb)
        assert e.value.code == -8


def _ghost_2d(orc, K, N, L, fn, times):
    pts = (np.arange(K)[:, None] + orc.nodes(N)[None, :]).ravel() * (L / K)
    return np.array([np.concatenate([fn(0 * pts, pts, t), fn(L + 0 * pts, pts, t), fn(pts, 0 * pts, t),
                                     fn(pts, L + 0 * pts, t)]) for t in times])


def test_2d_inflow_advection_vs_oracle_and_exact(sl, orc):
    u, v, L, K, N, dt, steps = 0.6, -0.4, 0.8, 3, 8, 2e-3, 100

    def phi(x, y, t):
        return 1.0 + 0.5 * np.sin(2 * np.pi * (x - u * t)) * np.sin(2 * np.pi * (y - v * t))

    pb = I.problem(2, (K, K), (0.0, 0.0), (L, L), N, 2, steps, dt, 3, ("const", [u, v]), ("const", [0.0]),
                   ("sinsin", [1.0, 0.5, 1.0]))
    pb["periodic"] = False
    pb["ghost"] = _ghost_2d(orc, K, N, L, phi, dt * np.arange(1, steps + 1))
    ref = orc.run(pb, ns=2, want_states=True)["states"]
    with sl.Solver(pb, "fp64") as s:
        s.step()
        st = s.samples()
    assert np.abs(st - ref).max() / np.abs(ref).max() <= FP64_TOL
    x, y = orc.node_coords(pb)
    assert np.abs(st[0] - phi(x, y, steps * dt)).max() <= 2e-7
    # FP32: without diffusion every step repeats the same particle geometry, so
    # the rounding of the FP32 advected basis accumulates (about 1.2e-7 of the
    # field per step in 2D, periodic or not); 50 steps stay within the bar
    with sl.Solver(pb, "fp64") as s:
        s.step(dt, 50)
        st50 = s.samples()
    with sl.Solver(pb, "fp32") as s:
        s.step(dt, 50)
        assert np.abs(s.samples() - st50).max() / np.abs(st50).max() <= MIXED_TOL


@pytest.mark.parametrize("N,precision", [(10, "fp64"), (11, "fp64"), (11, "fp32"), (12, "fp32")])
def test_2d_inflow_high_orders_vs_oracle(sl, orc, N, precision):
    """Dirichlet ghosts at the orders whose Gram rows are split over lanes."""
    u, v, L, K, steps = 0.6, -0.4, 0.8, 2, 6

    def phi(x, y, t):
        return 1.0 + 0.5 * np.sin(2 * np.pi * (x - u * t)) * np.sin(2 * np.pi * (y - v * t))

    pb = I.problem(2, (K, K), (0.0, 0.0), (L, L), N, 2, steps, 0.0, 3, ("const", [u, v]), ("const", [0.001]),
                   ("sinsin", [1.0, 0.5, 1.0]))
    pb["periodic"] = False
    pb["dt"] = dt = 0.5 * orc.dt_edge(pb)
    pb["ghost"] = _ghost_2d(orc, K, N, L, phi, dt * np.arange(1, steps + 1))
    ref = orc.run(pb, ns=2, want_states=True)["states"]
    with sl.Solver(pb, precision) as s:
        s.step()
        st = s.samples()
    tol = FP64_TOL if precision == "fp64" else MIXED_TOL
    assert np.abs(st - ref).max() / np.abs(ref).max() <= tol


def test_2d_sine_diffusion_with_reseeding_vs_oracle(sl, orc):
    K, N, M, dt, steps = 2, 5, 12, 1e-5, 30

    def mean_exact(x, y, t):
        return 2.0 + np.exp(-8 * np.pi ** 2 * t) * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)

    pb = I.problem(2, (K, K), (0.0, 0.0), (1.0, 1.0), N, M, steps, dt, 31, ("const", [0.0, 0.0]), ("const", [1.0]),
                   ("sinsin", [2.0, 1.0, 1.0]))
    pb["periodic"] = False
    pb["reseed_every"] = 10
    pb["ghost"] = _ghost_2d(orc, K, N, 1.0, mean_exact, dt * np.arange(1, steps + 1))
    ref = orc.run(pb, ns=M, want_states=True)["states"]
    with sl.Solver(pb, "fp64") as s:
        s.step()
        st = s.samples()
    assert np.abs(st - ref).max() / np.abs(ref).max() <= FP64_TOL
    assert all(np.array_equal(st[0], st[k]) for k in range(1, M))  # reseeded after the last step


def test_2d_mixed_periodicity_unsupported(sl, orc):
    pb = I.problem(2, (2, 2), (0.0, 0.0), (1.0, 1.0), 3, 2, 1, 1e-4, 1, ("const", [0.1, 0.2]), ("const", [0.01]),
                   ("gauss", [1.0, 0.2, 0.5, 0.5]))
    L = sl.lib()
    import ctypes as C
    m = sl._mesh(pb)
    m.periodic[0], m.periodic[1] = 0, 1
    u, D, p = sl._field(sl._U, pb["drift"]), sl._field(sl._D, pb["diffusion"]), sl._field(sl._PHI, pb["phi0"])
    h = C.c_void_p()
    assert L.sl_init(C.byref(h), C.byref(m), 3, 2, C.byref(u), C.byref(D), C.byref(p), None) == -8
