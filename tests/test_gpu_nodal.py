"""Nodal drift and diffusion on the GPU (node values handed over by a field
solver, Section 5.2), through the C ABI, against the FP64 oracle: interface
tables given or derived from the neighbouring traces, periodic and Dirichlet
meshes, 1D and 2D, fields switched between steps (from host or device
memory), batched instances and served requests (whose tables the server must
copy)."""

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


def _n_iface(pb):
    if pb["dim"] == 1:
        return pb["K"][0] + 1
    Kx, Ky, N = pb["K"][0], pb["K"][1], pb["N"]
    return Ky * (Kx + 1) * N + (Ky + 1) * Kx * N


def _nodal_1d(orc, pb, seed, table):
    """u = 1 + 0.5 sin(pi x) and D = 0.01 (1 + 0.5 cos(pi x)) on the nodes,
    each with a seeded per-node perturbation (so the fields jump between
    elements and the derived interface values are real means); optional
    interface tables of seeded values."""
    rng = np.random.default_rng(seed)
    x, _ = orc.node_coords(pb)
    u = 1.0 + 0.5 * np.sin(np.pi * x) + 0.05 * rng.uniform(-1, 1, x.shape)
    D = 0.01 * (1.0 + 0.5 * np.cos(np.pi * x)) * (1.0 + 0.2 * rng.uniform(-1, 1, x.shape))
    nf = _n_iface(pb)
    uf = 1.0 + 0.5 * rng.uniform(-1, 1, nf) if table else None
    Df = 0.01 * rng.uniform(0.5, 1.5, nf) if table else None
    return ("nodal", u, uf), ("nodal", D, Df)


def _nodal_2d(orc, pb, seed, table):
    """Rotation about (0.5, 0.5) and D = 0.004 on the nodes, perturbed per
    node (seeded); optional seeded interface tables."""
    rng = np.random.default_rng(seed)
    x, y = orc.node_coords(pb)
    w = 2.0 * np.pi
    u = np.stack([-w * (y - 0.5), w * (x - 0.5)]) + 0.1 * rng.uniform(-1, 1, (2,) + x.shape)
    D = 0.004 * (1.0 + 0.3 * rng.uniform(-1, 1, x.shape))
    nf = _n_iface(pb)
    uf = rng.uniform(-3.0, 3.0, nf) if table else None
    Df = 0.004 * rng.uniform(0.5, 1.5, nf) if table else None
    return ("nodal", u, uf), ("nodal", D, Df)


def _ghost(pb, steps, seed):
    rng = np.random.default_rng(seed)
    width = 2 if pb["dim"] == 1 else 2 * (pb["K"][0] + pb["K"][1]) * pb["N"]
    return 1.0 + 0.2 * rng.uniform(-1, 1, (steps, width))


def _problem_1d(orc, periodic, table, steps=6):
    pb = I.with_(I.config2(N=8, M=5, steps=steps, K=16), periodic=periodic)
    u, D = _nodal_1d(orc, pb, 7, table)
    pb = I.with_(pb, drift=u, diffusion=D)
    pb["dt"] = 0.4 * orc.dt_max(pb)
    if not periodic:
        pb["ghost"] = _ghost(pb, steps, 8)
    return pb


def _problem_2d(orc, periodic, table, steps=3):
    pb = I.problem(2, (4, 3), (0.0, 0.0), (1.0, 1.0), 4, 3, steps, 0.0, 8, ("const", [0.0, 0.0]),
                   ("const", [0.0]), ("gauss", [1.0, 0.2, 0.5, 0.5]))
    pb["periodic"] = periodic
    u, D = _nodal_2d(orc, pb, 9, table)
    pb = I.with_(pb, drift=u, diffusion=D)
    pb["dt"] = 0.4 * orc.dt_edge(pb)
    if not periodic:
        pb["ghost"] = _ghost(pb, steps, 10)
    return pb


def _gpu(sl, pb, precision):
    with sl.Solver(pb, precision) as s:
        s.step()
        return s.samples()


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("table", [False, True])
def test_1d_nodal_fields_vs_oracle(sl, orc, periodic, table):
    pb = _problem_1d(orc, periodic, table)
    ref = orc.run(pb, want_states=True)["states"]
    st = _gpu(sl, pb, "fp64")
    assert np.abs(st - ref).max() / np.abs(ref).max() <= FP64_TOL
    for precision in ("mixed", "fp32"):
        assert np.abs(_gpu(sl, pb, precision) - st).max() / np.abs(st).max() <= MIXED_TOL, precision


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("table", [False, True])
def test_2d_nodal_fields_vs_oracle(sl, orc, periodic, table):
    pb = _problem_2d(orc, periodic, table)
    ref = orc.run(pb, want_states=True)["states"]
    st = _gpu(sl, pb, "fp64")
    assert np.abs(st - ref).max() / np.abs(ref).max() <= FP64_TOL
    assert np.abs(_gpu(sl, pb, "fp32") - st).max() / np.abs(st).max() <= MIXED_TOL


def test_time_step_bounds_follow_the_nodal_fields(sl, orc):
    for pb in (_problem_1d(orc, True, True), _problem_2d(orc, True, False)):
        with sl.Solver(pb, "fp64") as s:
            assert s.dt_max == pytest.approx(orc.dt_max(pb), rel=1e-12)
            assert s.dt_edge == pytest.approx(orc.dt_edge(pb), rel=1e-12)


def test_nodal_fields_switched_between_steps(sl, orc):
    """An analytic flow, then nodal flows (derived, then tabled interfaces)
    set with sl_set_fields, the step counter running on."""
    pb = I.config2(N=8, M=4, steps=0, K=16)
    segs = [(pb["drift"], pb["diffusion"]), _nodal_1d(orc, pb, 11, False), _nodal_1d(orc, pb, 12, True)]
    pb["dt"] = 0.4 * min(orc.dt_max(I.with_(pb, drift=u, diffusion=D)) for u, D in segs)
    k = 4
    ref = None
    for i, (u, D) in enumerate(segs):
        q = I.with_(pb, drift=u, diffusion=D)
        ref = orc.run(q, nsteps=k, step0=i * k, state_in=ref, want_states=True, ns=pb["M"])["states"]
    with sl.Solver(pb, "fp64") as s:
        for i, (u, D) in enumerate(segs):
            if i:
                s.set_fields(u, D)
            s.step(pb["dt"], k)
        st = s.samples()
    assert np.abs(st - ref).max() / np.abs(ref).max() <= FP64_TOL


def test_negative_nodal_diffusion_rejected(sl, orc):
    pb = _problem_1d(orc, True, False)
    with sl.Solver(pb, "fp64") as s:
        u, D = pb["drift"], pb["diffusion"]
        bad = D[1].copy()
        bad[0, 0] = -1e-4
        with pytest.raises(sl.SLError) as e:
            s.set_fields(u, ("nodal", bad))
        assert e.value.code == -1


def test_batch_with_nodal_instances_equals_alone(sl, orc):
    pbs = [_problem_1d(orc, True, False), _problem_1d(orc, True, True), I.config2(N=8, M=5, steps=6, K=16),
           _problem_2d(orc, True, True)]
    pbs[2]["dt"] = 0.4 * orc.dt_max(pbs[2])
    with sl.Batch(pbs, "fp64") as b:
        b.step(3)
        for i, pb in enumerate(pbs):
            with sl.Solver(pb, "fp64") as s:
                s.step(pb["dt"], 3)
                alone = s.samples().reshape(pb["M"], -1)
            assert np.array_equal(b.samples(i), alone), i


def test_server_copies_the_nodal_tables(sl, orc):
    """The caller's arrays are overwritten right after submission; the
    request, created later behind a queued one, must still run the fields
    it was submitted with."""
    first = I.with_(I.config2(N=8, M=256, steps=30, K=64), dt=I.DT_CFG2_HALF)
    pb = _problem_1d(orc, True, True)
    with sl.Solver(pb, "fp64") as s:
        s.step()
        want, _ = s.moments()
    with sl.Server(budget_bytes=1 << 30, slice_steps=3, max_active=1, precision="fp64") as srv:
        srv.submit(first)
        t = srv.submit(pb)
        for arr in (pb["drift"][1], pb["drift"][2], pb["diffusion"][1], pb["diffusion"][2]):
            arr[...] = np.nan
        srv.wait_idle(300)
        state, (mean, _, _) = srv.poll(t)
    assert state == 2
    assert np.array_equal(mean, want.ravel())


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("table", [False, True])
def test_device_tables_equal_host_tables(sl, orc, dim, table):
    """sl_set_fields_device reads the nodal tables in place from device
    memory: the same steps, bit for bit, as sl_set_fields with the same values
    from the host; the time-step bounds follow when next asked for."""
    import torch

    if dim == 1:
        pb = I.config2(N=8, M=4, steps=0, K=16)
        u, D = _nodal_1d(orc, pb, 21, table)
    else:
        pb = I.problem(2, (3, 4), (0.0, 0.0), (1.0, 1.0), 5, 3, 0, 0.0, 8, ("rotation", [2 * np.pi, 0.5, 0.5]),
                       ("const", [0.004]), ("gauss", [1.0, 0.2, 0.5, 0.5]))
        u, D = _nodal_2d(orc, pb, 23, table)
    q = I.with_(pb, drift=u, diffusion=D)
    dt = 0.4 * (orc.dt_max(q) if dim == 1 else orc.dt_edge(q))
    with sl.Solver(pb, "fp64") as s:
        s.step(dt, 3)
        s.set_fields(u, D)
        s.step(dt, 4)
        want = s.samples()
    dev = lambda spec: (spec[0],) + tuple(None if a is None else torch.tensor(a, dtype=torch.float64, device="cuda")
                                          for a in spec[1:])  # noqa: E731
    with sl.Solver(pb, "fp64") as s:
        s.step(dt, 3)
        s.set_fields_device(dev(u), dev(D))
        assert s.dt_max == pytest.approx(orc.dt_max(q), rel=1e-12)
        s.step(dt, 4)
        got = s.samples()
    assert np.array_equal(got, want)


def test_device_tables_negative_diffusion_is_reported(sl, orc):
    import torch

    pb = I.config2(N=6, M=2, steps=0, K=8)
    u, D = _nodal_1d(orc, pb, 22, False)
    bad = torch.tensor(D[1], dtype=torch.float64, device="cuda")
    bad[3, 2] = -1e-3
    with sl.Solver(pb, "fp64") as s:
        s.set_fields_device(("nodal", torch.tensor(u[1], device="cuda")), ("nodal", bad))
        s.step(1e-5, 1)
        with pytest.raises(sl.SLError) as e:
            s.moments()
        assert e.value.code == -1
        with pytest.raises(sl.SLError) as e:
            s.step(1e-5, 1)
        assert e.value.code == -7
