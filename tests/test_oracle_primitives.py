"""Pins of the oracle's numerical primitives against facts fixed outside it:
published known-answer vectors, libm / mpmath, closed forms and numpy."""

import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                v = [int(t, 16) for t in line.split()]
                rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert orc.philox4x32_10(ctr, key) == want


def test_philox_counter_sensitivity(orc):
    # every counter word and key word changes every output word
    base = orc.philox4x32_10([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        out = orc.philox4x32_10(c, [5, 6])
        assert all(a != b for a, b in zip(out, base))
    out = orc.philox4x32_10([1, 2, 3, 4], [5, 7])
    assert all(a != b for a, b in zip(out, base))


def test_log_against_libm(orc):
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.uniform(0, 1, 20000), 10.0 ** rng.uniform(-16, 0, 5000),
                         [2.0 ** -53, 1 - 2.0 ** -53, 0.5, 0.25, 0.70710678118654752, 0.7071067811865476]])
    worst = 0.0
    for x in xs:
        ref = math.log(x)
        got = orc.log(x)
        worst = max(worst, abs(got - ref) / math.ulp(ref) if ref != 0 else abs(got))
    assert worst <= 2.0
    assert orc.log(1.0) == 0.0
    assert abs(orc.log(0.5) + math.log(2.0)) <= math.ulp(math.log(2.0))


def test_sincospi_against_mpmath(orc):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 200
    rng = np.random.default_rng(2)
    worst = 0.0
    for y in np.concatenate([rng.uniform(0, 2, 3000), [1e-300, 0.125, 0.25, 0.375, 1.75, 2.0 - 2 ** -52]]):
        s, c = orc.sincospi(y)
        es = float(mpmath.sin(mpmath.pi * mpmath.mpf(float(y))))
        ec = float(mpmath.cos(mpmath.pi * mpmath.mpf(float(y))))
        for got, ref in ((s, es), (c, ec)):
            if abs(ref) > 1e-300:
                # absolute error in units of ulp(1) near zeros, relative elsewhere
                worst = max(worst, abs(got - ref) / math.ulp(max(abs(ref), 2.0 ** -4)))
    assert worst <= 2.0
    # quadrant points are exact
    assert orc.sincospi(0.0) == (0.0, 1.0)
    assert orc.sincospi(0.5) == (1.0, 0.0) or orc.sincospi(0.5) == (1.0, -0.0)
    s, c = orc.sincospi(1.0)
    assert s == 0.0 and c == -1.0
    s, c = orc.sincospi(1.5)
    assert s == -1.0 and c == 0.0


def test_normals_distribution(orc):
    scipy_stats = pytest.importorskip("scipy.stats")
    z = np.array([orc.normals(11, st, s) for st in range(4) for s in range(25000)])
    z1, z2 = z[:, 0], z[:, 1]
    for v in (z1, z2):
        assert abs(v.mean()) < 4.0 / math.sqrt(len(v))
        assert abs(v.var() - 1.0) < 4.0 * math.sqrt(2.0 / len(v))
        assert scipy_stats.kstest(v, "norm").pvalue > 1e-4
    assert abs(np.corrcoef(z1, z2)[0, 1]) < 4.0 / math.sqrt(len(z1))


def test_normals_follow_box_muller_of_philox(orc):
    # rebuild z from the raw Philox words with numpy/libm (different ln and
    # trig implementations): equal to a few ulp
    seed, step, sample, tag = 0x123456789ABCDEF, 17, 42, 0
    w = orc.philox4x32_10([step, sample, tag, 0], [seed & 0xFFFFFFFF, seed >> 32])
    x1 = ((w[0] << 32) | w[1]) >> 12
    x2 = ((w[2] << 32) | w[3]) >> 12
    u1 = (2 * x1 + 1) * 2.0 ** -53
    u2 = (2 * x2 + 1) * 2.0 ** -53
    r = math.sqrt(-2.0 * math.log(u1))
    z = orc.normals(seed, step, sample, tag)
    assert abs(z[0] - r * math.cos(2 * math.pi * u2)) < 1e-14 * max(1.0, r)
    assert abs(z[1] - r * math.sin(2 * math.pi * u2)) < 1e-14 * max(1.0, r)


def test_wiener_is_sqrt_dt_times_normal(orc):
    dW = orc.wiener(5, 2, 7, 3, 4, 2.5e-3)
    for n in range(4):
        for s in range(7):
            z = orc.normals(5, 3 + n, s, 0)
            assert dW[n, s, 0] == math.sqrt(2.5e-3) * z[0]
            assert dW[n, s, 1] == math.sqrt(2.5e-3) * z[1]


@pytest.mark.parametrize("N", [2, 3, 4, 6, 8, 12, 16])
def test_nodes_are_chebyshev_gauss(orc, N):
    xi = orc.nodes(N)
    assert np.all(np.diff(xi) > 0) and xi[0] > 0 and xi[-1] < 1
    # roots of T_N(2 xi - 1)
    coef = np.zeros(N + 1)
    coef[N] = 1.0
    assert np.max(np.abs(np.polynomial.chebyshev.chebval(2 * xi - 1, coef))) < 1e-12 * N
    # symmetric, and each lies between consecutive Lobatto nodes
    assert np.allclose(xi + xi[::-1], 1.0, atol=1e-15)
    lob = 0.5 * (1 - np.cos(np.arange(N + 1) * np.pi / N))
    assert np.all(lob[:-1] < xi) and np.all(xi < lob[1:])


@pytest.mark.parametrize("N", [3, 5, 8, 12, 16])
def test_lagrange_basis(orc, N):
    xi = orc.nodes(N)
    for j in range(N):
        for i in range(N):
            assert orc.lagrange(xi, j, xi[i]) == pytest.approx(1.0 if i == j else 0.0, abs=1e-14)
    rng = np.random.default_rng(N)
    x = rng.uniform(-0.2, 1.2, 7)
    # reproduces every monomial of degree <= N-1, and the derivative of it
    for k in range(N):
        for xv in x:
            v = sum(xi[j] ** k * orc.lagrange(xi, j, xv) for j in range(N))
            d = sum(xi[j] ** k * orc.lagrange_deriv(xi, j, xv) for j in range(N))
            assert v == pytest.approx(xv ** k, abs=1e-11)
            assert d == pytest.approx(k * xv ** (k - 1) if k else 0.0, abs=1e-9 * N * N)


@pytest.mark.parametrize("N", [2, 4, 7, 8, 16])
def test_quadrature_weights_exact(orc, N):
    w = orc.quad_weights(N)
    xi = orc.nodes(N)
    assert np.all(w > 0)
    for k in range(N):
        assert float(w @ xi ** k) == pytest.approx(1.0 / (k + 1), rel=1e-13)


def test_lu_and_lstsq_against_numpy(orc):
    rng = np.random.default_rng(3)
    for n in (1, 2, 5, 17):
        A = rng.normal(size=(n, n)) + n * np.eye(n) * 0.1
        b = rng.normal(size=n)
        assert np.allclose(orc.lu_solve(A, b), np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)
    for m, n in ((3, 2), (8, 6), (18, 16), (96, 64)):
        A = rng.normal(size=(m, n))
        b = rng.normal(size=m)
        ref = np.linalg.lstsq(A, b, rcond=None)[0]
        assert np.allclose(orc.lstsq(A, b), ref, rtol=1e-10, atol=1e-11)
    with pytest.raises(np.linalg.LinAlgError):
        orc.lu_solve(np.zeros((3, 3)), np.ones(3))


def test_pdf_binning_against_numpy_histogram(orc):
    # recovery of the PDF at each node by binning the samples (Section 5.4)
    rng = np.random.default_rng(12)
    lo, hi, B = -1.0, 2.5, 7
    x = rng.uniform(lo - 0.5, hi + 0.5, size=(50, 2, 3))
    edges = np.linspace(lo, hi, B + 1)
    x[np.min(np.abs(x[..., None] - edges), axis=-1) < 1e-9] = 0.123  # keep away from the edges
    counts = orc.pdf(x, B, lo, hi)
    for e in range(2):
        for p in range(3):
            ref, _ = np.histogram(x[:, e, p], bins=B, range=(lo, hi))
            assert np.array_equal(counts[e, p], ref)
    # the edge rules: lo in the first bin, hi in the last, outside and NaN not counted
    y = np.array([lo, hi, lo - 1e-12, hi + 1e-12, np.nan, 0.0]).reshape(6, 1, 1)
    c = orc.pdf(y, B, lo, hi)[0, 0]
    assert c[0] == 1 and c[-1] == 1 and c.sum() == 3 and c[2] == 1  # 0.0 = lo + 2 widths
