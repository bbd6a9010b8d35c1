"""Pins of the oracle's per-element remap (Section 5.3) against polynomial
reproduction, brute-force least squares built independently in numpy (basis
from a Chebyshev-Vandermonde solve, not the oracle's product formula), and the
algebraically equivalent reduced (Woodbury) form of the 1D remap."""

import numpy as np
import pytest

import sl_inputs as I


def _basis_np(nodes, x):
    """Lagrange basis on `nodes` at points x, [len(x)][len(nodes)], from a
    Chebyshev-Vandermonde solve (independent of the product formula)."""
    N = len(nodes)
    cv = np.polynomial.chebyshev.chebvander
    Vn = cv(2.0 * np.asarray(nodes, float) - 1.0, N - 1)
    Vx = cv(2.0 * np.atleast_1d(np.asarray(x, float)) - 1.0, N - 1)
    return np.linalg.solve(Vn.T, Vx.T).T


def _advected(orc, N, rng, scale=0.3):
    xi = orc.nodes(N)
    gap = np.min(np.diff(xi))
    return xi, xi + rng.uniform(-scale, scale) * gap + rng.uniform(-0.05, 0.05, N) * gap


@pytest.mark.parametrize("N", [2, 3, 4, 6, 8, 12])
def test_1d_polynomial_reproduction(orc, N):
    rng = np.random.default_rng(10 + N)
    for _ in range(5):
        xi, xs = _advected(orc, N, rng)
        c = rng.normal(size=N)
        poly = np.polynomial.Polynomial(c)
        e0, e1 = orc.faces_1d(xs, poly(xs))
        assert e0 == pytest.approx(poly(0.0), abs=1e-9)
        assert e1 == pytest.approx(poly(1.0), abs=1e-9)
        q = orc.remap_1d(xs, poly(xs), poly(0.0), poly(1.0))
        assert np.allclose(q, poly(xi), atol=1e-9)


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6])
def test_1d_remap_brute_force(orc, N):
    rng = np.random.default_rng(20 + N)
    for _ in range(10):
        xi, xs = _advected(orc, N, rng, 0.5)
        phs = rng.normal(size=N)
        gL, gR = rng.normal(size=2)
        V = _basis_np(xi, xs)
        B = _basis_np(xi, [0.0, 1.0])
        A = np.vstack([V, B])
        rhs = np.concatenate([phs, [gL, gR]])
        ref = np.linalg.lstsq(A, rhs, rcond=None)[0]
        q = orc.remap_1d(xs, phs, gL, gR)
        assert np.allclose(q, ref, rtol=1e-10, atol=1e-10)
        # face values of the advected interpolant (Eq. remap_bnd)
        Hs = _basis_np(xs, [0.0, 1.0])
        e0, e1 = orc.faces_1d(xs, phs)
        assert np.allclose([e0, e1], Hs @ phs, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("N", [3, 6, 8, 12, 16])
def test_1d_reduced_form_identity(orc, N):
    # q = H*(phi* - E^T mu), mu = (I + E E^T)^{-1}(E phi* - g), with H* the
    # advected basis at the Gauss nodes and E the advected basis at the faces,
    # equals the stacked least-squares solution (Woodbury identity)
    rng = np.random.default_rng(30 + N)
    for _ in range(5):
        xi, xs = _advected(orc, N, rng, 0.4)
        phs = 1.0 + 0.1 * rng.normal(size=N)
        g = np.array(orc.faces_1d(xs, phs)) + 1e-3 * rng.normal(size=2)
        Hs = _basis_np(xs, xi)
        E = _basis_np(xs, [0.0, 1.0])
        mu = np.linalg.solve(np.eye(2) + E @ E.T, E @ phs - g)
        red = Hs @ (phs - E.T @ mu)
        q = orc.remap_1d(xs, phs, g[0], g[1])
        assert np.allclose(q, red, rtol=1e-11, atol=1e-11)


def _advected_2d(orc, N, rng, scale=0.3):
    xi = orc.nodes(N)
    gap = np.min(np.diff(xi))
    X, Y = np.meshgrid(xi, xi)  # [j][i] -> p = j*N + i
    xs = X.ravel() + rng.uniform(-scale, scale, N * N) * gap
    ys = Y.ravel() + rng.uniform(-scale, scale, N * N) * gap
    return xi, xs, ys


def _B2(xi):
    N = len(xi)
    h0, h1 = _basis_np(xi, [0.0, 1.0])
    B = np.zeros((4 * N, N * N))
    for j in range(N):
        B[j, j * N:(j + 1) * N] = h0
        B[N + j, j * N:(j + 1) * N] = h1
    for i in range(N):
        B[2 * N + i, i::N] = h0
        B[3 * N + i, i::N] = h1
    return B


def _V2(xi, xs, ys):
    Hx = _basis_np(xi, xs)
    Hy = _basis_np(xi, ys)
    return np.einsum("pj,pi->pji", Hy, Hx).reshape(len(xs), -1)


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_2d_remap_brute_force(orc, N):
    rng = np.random.default_rng(40 + N)
    for _ in range(4):
        xi, xs, ys = _advected_2d(orc, N, rng)
        phs = rng.normal(size=N * N)
        g = rng.normal(size=4 * N)
        A = np.vstack([_V2(xi, xs, ys), _B2(xi)])
        ref = np.linalg.lstsq(A, np.concatenate([phs, g]), rcond=None)[0]
        q = orc.remap_2d(xs, ys, phs, g)
        assert np.allclose(q, ref, rtol=1e-9, atol=1e-9)
        alpha = np.linalg.solve(_V2(xi, xs, ys), phs)
        assert np.allclose(orc.faces_2d(xs, ys, phs), _B2(xi) @ alpha, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("N", [2, 4, 6, 8])
def test_2d_polynomial_reproduction(orc, N):
    rng = np.random.default_rng(50 + N)
    xi, xs, ys = _advected_2d(orc, N, rng)
    C = rng.normal(size=(N, N))

    def P(x, y):
        return np.polynomial.polynomial.polyval2d(x, y, C)

    X, Y = np.meshgrid(xi, xi)
    f = orc.faces_2d(xs, ys, P(xs, ys))
    want = np.concatenate([P(0 * xi, xi), P(1 + 0 * xi, xi), P(xi, 0 * xi), P(xi, 1 + 0 * xi)])
    assert np.allclose(f, want, atol=1e-8)
    q = orc.remap_2d(xs, ys, P(xs, ys), want)
    assert np.allclose(q, P(X, Y).ravel(), atol=1e-8)


@pytest.mark.parametrize("N", [3, 6, 10, 16])
def test_split_forms_equal_absolute_forms(orc, N):
    # particles given as node + displacement evaluate the same polynomials as
    # particles given by absolute position (up to the rounding of xi + d)
    rng = np.random.default_rng(60 + N)
    xi = orc.nodes(N)
    gap = np.min(np.diff(xi))
    d = rng.uniform(-0.4, 0.4, N) * gap
    phs = 1 + 0.2 * rng.normal(size=N)
    e_abs = orc.faces_1d(xi + d, phs)
    e_spl = orc.faces_1d_split(d, phs)
    assert np.allclose(e_abs, e_spl, rtol=1e-12, atol=1e-12)
    g = np.array(e_spl) + 1e-3
    assert np.allclose(orc.remap_1d(xi + d, phs, *g), orc.remap_1d_split(d, phs, *g), rtol=1e-12, atol=1e-12)
    for j in range(N):
        assert orc.lagrange_split(xi, d, j, 0.3, 0.0) == pytest.approx(orc.lagrange(xi + d, j, 0.3), rel=1e-11, abs=1e-13)


@pytest.mark.parametrize("N", [3, 5, 8])
def test_split_forms_2d(orc, N):
    rng = np.random.default_rng(70 + N)
    xi = orc.nodes(N)
    gap = np.min(np.diff(xi))
    X, Y = np.meshgrid(xi, xi)
    dx = rng.uniform(-0.3, 0.3, N * N) * gap
    dy = rng.uniform(-0.3, 0.3, N * N) * gap
    C = rng.normal(size=(N, N))

    def P(x, y):
        return np.polynomial.polynomial.polyval2d(x, y, C)

    xs, ys = X.ravel() + dx, Y.ravel() + dy
    f = orc.faces_2d_split(dx, dy, P(xs, ys))
    want = np.concatenate([P(0 * xi, xi), P(1 + 0 * xi, xi), P(xi, 0 * xi), P(xi, 1 + 0 * xi)])
    assert np.allclose(f, want, atol=1e-8)
    assert np.allclose(orc.remap_2d_split(dx, dy, P(xs, ys), want), P(X, Y).ravel(), atol=1e-8)
    phs = rng.normal(size=N * N)
    g = rng.normal(size=4 * N)
    assert np.allclose(orc.remap_2d_split(dx, dy, phs, g), orc.remap_2d(xs, ys, phs, g), rtol=1e-9, atol=1e-9)


def test_small_displacement_keeps_precision(orc):
    # a displacement of 1e-6 of the element: the split form reproduces the
    # first-order shift exactly to ~1e-10 relative, the absolute form loses
    # digits to the rounding of xi + d
    N = 8
    xi = orc.nodes(N)
    d = np.full(N, 1e-6)
    c = np.array([0.3, -1.2, 0.7, 0.25, -0.4, 0.1, 0.05, -0.02])
    poly = np.polynomial.Polynomial(c)
    dpoly = poly.deriv()
    phs = poly(xi)  # values carried by the particles (deg N-1 field)
    e0, e1 = orc.faces_1d_split(d, phs)
    # the advected polynomial is p(x - d): its face values
    want0, want1 = poly(0.0 - 1e-6), poly(1.0 - 1e-6)
    assert abs(e0 - want0) < 1e-13 and abs(e1 - want1) < 1e-13
    # and the shift itself is resolved to 1e-7 relative
    assert abs((e0 - poly(0.0)) / (-1e-6 * dpoly(0.0)) - 1) < 1e-6


# ---------------------------------------------------------------- boundary-row weight w
# (Section 5.3's least squares with the face rows weighted by w; w = inf is the
# hard-constrained problem, min |V q - phi*| subject to B q = g)

@pytest.mark.parametrize("N", [3, 6, 9])
@pytest.mark.parametrize("w", [0.5, 3.0])
def test_1d_weighted_remap_brute_force(orc, N, w):
    rng = np.random.default_rng(60 + N)
    for _ in range(5):
        xi, xs = _advected(orc, N, rng, 0.4)
        phs = rng.normal(size=N)
        gL, gR = rng.normal(size=2)
        A = np.vstack([_basis_np(xi, xs), w * _basis_np(xi, [0.0, 1.0])])
        ref = np.linalg.lstsq(A, np.concatenate([phs, [w * gL, w * gR]]), rcond=None)[0]
        q = orc.remap_1d_split(xs - xi, phs, gL, gR, w=w)
        assert np.allclose(q, ref, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("N", [3, 6, 9, 12])
def test_1d_hard_constraints(orc, N):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(70 + N)
    for _ in range(5):
        xi, xs = _advected(orc, N, rng, 0.4)
        phs = rng.normal(size=N)
        g = rng.normal(size=2)
        V, B = _basis_np(xi, xs), _basis_np(xi, [0.0, 1.0])
        q = orc.remap_1d_split(xs - xi, phs, g[0], g[1], w=np.inf)
        # the constraints hold exactly (to rounding)
        assert np.allclose(B @ q, g, rtol=0, atol=1e-11)
        # null-space solution of the equality-constrained least squares
        qp = np.linalg.lstsq(B, g, rcond=None)[0]
        Z = scipy_linalg.null_space(B)
        y = np.linalg.lstsq(V @ Z, phs - V @ qp, rcond=None)[0]
        assert np.allclose(q, qp + Z @ y, rtol=1e-9, atol=1e-9)
        # and it is the limit of large weights
        q_big = orc.remap_1d_split(xs - xi, phs, g[0], g[1], w=1e5)
        assert np.abs(q_big - q).max() <= 1e-7 * max(1.0, np.abs(q).max())


@pytest.mark.parametrize("N", [4, 8, 16])
@pytest.mark.parametrize("w", [0.5, 2.0, np.inf])
def test_1d_reduced_form_with_weight(orc, N, w):
    # q = H*(phi* - E^T mu), mu = (I / w^2 + E E^T)^{-1}(E phi* - g) (zero
    # diagonal for w = inf) equals the weighted / constrained remap
    rng = np.random.default_rng(80 + N)
    xi, xs = _advected(orc, N, rng, 0.4)
    phs = 1.0 + 0.1 * rng.normal(size=N)
    g = np.array(orc.faces_1d(xs, phs)) + 1e-3 * rng.normal(size=2)
    Hs, E = _basis_np(xs, xi), _basis_np(xs, [0.0, 1.0])
    mu = np.linalg.solve(np.eye(2) / w ** 2 + E @ E.T, E @ phs - g)
    q = orc.remap_1d_split(xs - xi, phs, g[0], g[1], w=w)
    assert np.allclose(q, Hs @ (phs - E.T @ mu), rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("N", [2, 4, 6])
def test_2d_weighted_remap_brute_force(orc, N):
    rng = np.random.default_rng(90 + N)
    w = 2.5
    xi, xs, ys = _advected_2d(orc, N, rng)
    X, Y = np.meshgrid(xi, xi)
    phs = rng.normal(size=N * N)
    g = rng.normal(size=4 * N)
    A = np.vstack([_V2(xi, xs, ys), w * _B2(xi)])
    ref = np.linalg.lstsq(A, np.concatenate([phs, w * g]), rcond=None)[0]
    q = orc.remap_2d_split(xs - X.ravel(), ys - Y.ravel(), phs, g, w=w)
    assert np.allclose(q, ref, rtol=1e-9, atol=1e-9)


def test_hard_constraints_are_1d_only(orc):
    pb = I.problem(2, (2, 2), (0.0, 0.0), (1.0, 1.0), 3, 2, 1, 1e-4, 1, ("const", [0.1, 0.2]),
                   ("const", [0.01]), ("gauss", [1.0, 0.2, 0.5, 0.5]))
    pb["bc_weight"] = np.inf
    with pytest.raises(Exception):
        orc.run(pb, ns=2)
