"""Pins of the oracle's nodal drift and diffusion: the form in which a field
solver hands its velocity and diffusivity over (Section 5.2 takes du/dx from
the DSEM field solver).

Reading: the values at the Gauss nodes are given; du_j/dx_j is the spectral
derivative of the nodal drift in each element; the values at the interface
points are given, or else the mean of the traces of the two neighbouring
elements' interpolants (the inside trace at a Dirichlet boundary), with a
derived D clipped at 0.  Each pin compares with something fixed outside the
nodal code: the analytic fields at the same points, traces that are exact for
polynomials, or hand-computed means.
"""

import numpy as np
import pytest

import oracle as orc
import sl_inputs as I


def _node_xy(pb):
    """Physical node coordinates [E][n] (x, y) in the element-major layout."""
    N, dim = pb["N"], pb["dim"]
    xi = orc.nodes(N)
    Kx = pb["K"][0]
    hx = (pb["hi"][0] - pb["lo"][0]) / Kx
    if dim == 1:
        x = pb["lo"][0] + (np.arange(Kx)[:, None] + xi[None, :]) * hx
        return x, np.zeros_like(x)
    Ky = pb["K"][1]
    hy = (pb["hi"][1] - pb["lo"][1]) / Ky
    kx = np.arange(Kx * Ky) % Kx
    ky = np.arange(Kx * Ky) // Kx
    i = np.arange(N * N) % N
    j = np.arange(N * N) // N
    x = pb["lo"][0] + (kx[:, None] + xi[None, i]) * hx
    y = pb["lo"][1] + (ky[:, None] + xi[None, j]) * hy
    return x, y


def _iface_xy(pb):
    """Interface points in the interface-table layout: 1D x_f = lo + f h
    (f = 0..K); 2D vertical [Ky][Kx+1][N] then horizontal [Ky+1][Kx][N].
    Returns (x, y, normal direction)."""
    N = pb["N"]
    xi = orc.nodes(N)
    Kx = pb["K"][0]
    hx = (pb["hi"][0] - pb["lo"][0]) / Kx

    def at(k, K, lo, hi, h):
        return hi if k == K else lo + k * h

    if pb["dim"] == 1:
        x = np.array([at(f, Kx, pb["lo"][0], pb["hi"][0], hx) for f in range(Kx + 1)])
        return x, np.zeros_like(x), np.zeros(Kx + 1, dtype=int)
    Ky = pb["K"][1]
    hy = (pb["hi"][1] - pb["lo"][1]) / Ky
    xs, ys, ds = [], [], []
    for ky in range(Ky):
        for f in range(Kx + 1):
            for jj in range(N):
                xs.append(at(f, Kx, pb["lo"][0], pb["hi"][0], hx))
                ys.append(pb["lo"][1] + (ky + xi[jj]) * hy)
                ds.append(0)
    for g in range(Ky + 1):
        for kx in range(Kx):
            for ii in range(N):
                xs.append(pb["lo"][0] + (kx + xi[ii]) * hx)
                ys.append(at(g, Ky, pb["lo"][1], pb["hi"][1], hy))
                ds.append(1)
    return np.array(xs), np.array(ys), np.array(ds)


def _sin_u(x):
    return 1.0 + 0.5 * np.sin(np.pi * x)


def _cos_D(x):
    return 0.01 * (1.0 + 0.5 * np.cos(np.pi * x))


def _rot(x, y, w=2.0 * np.pi, c=(0.5, 0.5)):
    return -w * (y - c[1]), w * (x - c[0])


def _sinsin_D(x, y):
    return 0.005 * (1.0 + 0.3 * np.sin(2.0 * np.pi * x) * np.sin(2.0 * np.pi * y))


def _small_1d():
    pb = I.with_(I.config2(N=6, M=6, steps=4, K=6), periodic=True)
    return I.with_(pb, dt=0.5 * orc.dt_max(pb))


def _small_2d(periodic=True):
    pb = I.config3(M=3, steps=3, K=3, N=4)
    pb = I.with_(pb, periodic=periodic)
    return I.with_(pb, dt=0.5 * orc.dt_edge(pb))


def test_nodal_1d_with_interface_table_is_the_analytic_problem():
    """Node values and interface values taken from u = 1 + 0.5 sin(pi x),
    D = 0.01 (1 + 0.5 cos(pi x)): the nodal problem is the analytic one, so
    coefficients and samples agree to rounding."""
    pb = _small_1d()
    x, _ = _node_xy(pb)
    xf, _, _ = _iface_xy(pb)
    nod = I.with_(pb, drift=("nodal", _sin_u(x), _sin_u(xf)), diffusion=("nodal", _cos_D(x), _cos_D(xf)))
    for A, B in zip(orc.coeffs(pb), orc.coeffs(nod)):
        np.testing.assert_allclose(B, A, rtol=1e-14, atol=1e-17)
    for A, B in zip(orc.face_coeffs(pb), orc.face_coeffs(nod)):
        np.testing.assert_allclose(B, A, rtol=1e-14, atol=1e-17)
    ref = orc.run(pb, want_states=True)["states"]
    got = orc.run(nod, want_states=True)["states"]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


def test_nodal_1d_derived_faces_are_exact_for_a_linear_drift():
    """Traces of a degree-1 field are exact, so away from a periodic seam the
    interface drift is the field itself; at the seam of a periodic line it is
    the mean of the two one-sided values u(hi) and u(lo)."""
    for periodic in (False, True):
        pb = I.with_(_small_1d(), K=(4,), N=5, periodic=periodic)
        x, _ = _node_xy(pb)
        u = lambda z: 0.5 + 0.25 * z  # noqa: E731
        nod = I.with_(pb, drift=("nodal", u(x)), diffusion=("const", [0.01]))
        a, _ = orc.face_coeffs(nod)
        xf, _, _ = _iface_xy(pb)
        want = u(xf)
        if periodic:
            want[0] = want[-1] = 0.5 * (u(pb["lo"][0]) + u(pb["hi"][0]))
        np.testing.assert_allclose(a / nod["dt"], want, rtol=1e-13, atol=1e-15)
        # the divergence of the nodal field is its spectral derivative: 0.25
        c = orc.coeffs(nod)[3]
        np.testing.assert_allclose((1.0 - c) / nod["dt"], 0.25, rtol=1e-10)


def test_nodal_1d_piecewise_constant_diffusion_means():
    """D = 1, 2, 4 on three elements: interface values are the means of the
    neighbours (periodic: 2.5, 1.5, 3, 2.5) or the inside value at a
    Dirichlet boundary (1, 1.5, 3, 4)."""
    for periodic, want in ((True, [2.5, 1.5, 3.0, 2.5]), (False, [1.0, 1.5, 3.0, 4.0])):
        pb = I.with_(_small_1d(), K=(3,), N=4, periodic=periodic)
        Dn = np.repeat(np.array([1.0, 2.0, 4.0])[:, None], 4, axis=1)
        nod = I.with_(pb, drift=("const", [1.0, 0.0]), diffusion=("nodal", Dn))
        _, b = orc.face_coeffs(nod)
        np.testing.assert_allclose(b, np.sqrt(2.0 * np.array(want)), rtol=1e-14)


def test_nodal_derived_diffusion_is_clipped_at_zero():
    """D = (0, 1, 0) on the three Gauss nodes: the parabola through them is
    negative at the element's faces, and the derived D there is 0."""
    pb = I.with_(_small_1d(), K=(1,), N=3, periodic=False)
    xi = orc.nodes(3)
    trace = (0 - xi[0]) * (0 - xi[2]) / ((xi[1] - xi[0]) * (xi[1] - xi[2]))
    assert trace < 0.0
    nod = I.with_(pb, diffusion=("nodal", np.array([[0.0, 1.0, 0.0]])))
    _, b = orc.face_coeffs(nod)
    assert np.all(b == 0.0)


def test_nodal_negative_diffusion_is_refused():
    pb = I.with_(_small_1d(), K=(2,), N=3)
    with pytest.raises(ValueError):
        orc.coeffs(I.with_(pb, diffusion=("nodal", np.full((2, 3), -1e-3))))
    face = np.full(3, 0.01)
    face[1] = -0.01
    with pytest.raises(ValueError):
        orc.coeffs(I.with_(pb, diffusion=("nodal", np.full((2, 3), 0.01), face)))


def test_nodal_2d_with_interface_table_is_the_analytic_problem():
    """Rotation and the sin-sin diffusion sampled on the nodes and on the
    interface table: the same coefficients and samples as the analytic
    problem.  The table entries of the last interface of each periodic line
    are NaN: they must not be read."""
    pb = _small_2d(periodic=True)
    x, y = _node_xy(pb)
    xf, yf, dn = _iface_xy(pb)
    ux, uy = _rot(x, y)
    fux, fuy = _rot(xf, yf)
    un = np.where(dn == 0, fux, fuy)
    Df = _sinsin_D(xf, yf)
    Kx, Ky, N = pb["K"][0], pb["K"][1], pb["N"]
    last = np.zeros(len(xf), dtype=bool)
    vert = np.arange(Ky * (Kx + 1) * N)
    last[vert[(vert // N) % (Kx + 1) == Kx]] = True
    last[Ky * (Kx + 1) * N + Ky * Kx * N:] = True
    un[last] = np.nan
    Df[last] = np.nan
    nod = I.with_(pb, drift=("nodal", np.stack([ux, uy]), un), diffusion=("nodal", _sinsin_D(x, y), Df))
    A, B = orc.coeffs(pb), orc.coeffs(nod)
    for a, b in zip(A, B):
        np.testing.assert_allclose(b, a, rtol=1e-13, atol=1e-15)
    ref = orc.run(pb, want_states=True)["states"]
    got = orc.run(nod, want_states=True)["states"]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("periodic", [True, False])
def test_nodal_2d_derived_faces_of_the_rotation(periodic):
    """The rotation's normal components do not vary along the normal (u_x
    depends on y only, u_y on x only) and are linear, so every derived trace
    is exact, including at periodic seams: the interface coefficients equal
    the analytic ones, and the spectral divergence vanishes."""
    pb = _small_2d(periodic=periodic)
    x, y = _node_xy(pb)
    ux, uy = _rot(x, y)
    nod = I.with_(pb, drift=("nodal", np.stack([ux, uy])))
    a0, b0 = orc.face_coeffs(pb)
    a1, b1 = orc.face_coeffs(nod)
    np.testing.assert_allclose(a1, a0, rtol=1e-12, atol=1e-16)
    np.testing.assert_array_equal(b1, b0)
    c = orc.coeffs(nod)[3]
    assert np.abs(1.0 - c).max() < 1e-12
