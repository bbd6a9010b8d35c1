"""Python access to the plain FP64 CPU oracle (``sl_oracle.c``).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_2009_07340_gb300``) and never imports it.

The C source is compiled on first use (``gcc -O2 -ffp-contract=off``) into
``oracle/liboracle.so`` next to it.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sl_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_DRIFT = {"const": 0, "sin": 1, "rotation": 2, "nodal": 3}
_DIFF = {"const": 0, "cos": 1, "sinsin": 2, "nodal": 3}
_PHI0 = {"gauss": 0, "fourier": 1, "sine": 2, "sinsin": 3}


def build(force=False):
    """Compile the oracle shared library (idempotent)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [("dim", C.c_int), ("K", C.c_int * 2), ("lo", C.c_double * 2),
                ("hi", C.c_double * 2), ("N", C.c_int), ("drift_kind", C.c_int),
                ("drift_p", C.c_double * 8), ("diff_kind", C.c_int), ("diff_p", C.c_double * 8),
                ("phi0_kind", C.c_int), ("phi0_p", C.c_double * 40), ("seed", C.c_ulonglong),
                ("dt", C.c_double), ("omega", C.c_double), ("periodic", C.c_int), ("reseed_every", C.c_int),
                ("drift_nodal", C.POINTER(C.c_double)), ("drift_face", C.POINTER(C.c_double)),
                ("diff_nodal", C.POINTER(C.c_double)), ("diff_face", C.POINTER(C.c_double))]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            dp = C.POINTER(C.c_double)
            u32p = C.POINTER(C.c_uint32)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_log.restype = C.c_double
            L.orc_log.argtypes = [C.c_double]
            L.orc_sincospi.argtypes = [C.c_double, dp, dp]
            L.orc_normals.argtypes = [C.c_ulonglong, C.c_uint32, C.c_uint32, C.c_uint32, dp]
            L.orc_wiener.argtypes = [C.c_ulonglong, C.c_int, C.c_int, C.c_long, C.c_int, C.c_double, dp]
            L.orc_nodes.argtypes = [C.c_int, dp]
            L.orc_lagrange.restype = C.c_double
            L.orc_lagrange.argtypes = [C.c_int, dp, C.c_int, C.c_double]
            L.orc_lagrange_deriv.restype = C.c_double
            L.orc_lagrange_deriv.argtypes = [C.c_int, dp, C.c_int, C.c_double]
            L.orc_quad_weights.argtypes = [C.c_int, dp]
            L.orc_lu_solve.argtypes = [C.c_int, dp, dp, dp]
            L.orc_lstsq.argtypes = [C.c_int, C.c_int, dp, dp, dp]
            L.orc_faces_1d.argtypes = [C.c_int, dp, dp, dp, dp]
            L.orc_remap_1d.argtypes = [C.c_int, dp, dp, dp, C.c_double, C.c_double, dp]
            L.orc_faces_2d.argtypes = [C.c_int, dp, dp, dp, dp, dp]
            L.orc_lagrange_split.restype = C.c_double
            L.orc_lagrange_split.argtypes = [C.c_int, dp, dp, C.c_int, C.c_double, C.c_double]
            L.orc_faces_1d_split.argtypes = [C.c_int, dp, dp, dp, dp, dp]
            L.orc_remap_1d_split.argtypes = [C.c_int, dp, dp, dp, C.c_double, C.c_double, dp]
            L.orc_remap_1d_split_w.argtypes = [C.c_int, dp, dp, dp, C.c_double, C.c_double, C.c_double, dp]
            L.orc_faces_2d_split.argtypes = [C.c_int, dp, dp, dp, dp, dp]
            L.orc_remap_2d_split.argtypes = [C.c_int, dp, dp, dp, dp, dp, dp]
            L.orc_remap_2d_split_w.argtypes = [C.c_int, dp, dp, dp, dp, dp, C.c_double, dp]
            L.orc_remap_2d.argtypes = [C.c_int, dp, dp, dp, dp, dp, dp]
            L.orc_init_state.argtypes = [C.POINTER(_Problem), dp]
            L.orc_get_coeffs.argtypes = [C.POINTER(_Problem), dp, dp, dp, dp]
            L.orc_get_face_coeffs.argtypes = [C.POINTER(_Problem), dp, dp]
            L.orc_run.argtypes = [C.POINTER(_Problem), C.c_long, C.c_int, C.c_int, C.c_int, C.c_int,
                                  dp, dp, dp, dp, dp]
            L.orc_dt_max.restype = C.c_double
            L.orc_dt_max.argtypes = [C.POINTER(_Problem)]
            L.orc_dt_edge.restype = C.c_double
            L.orc_dt_edge.argtypes = [C.POINTER(_Problem)]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _problem(pb, dt=None):
    p = _Problem()
    p.dim = pb["dim"]
    for d in range(pb["dim"]):
        p.K[d] = pb["K"][d]
        p.lo[d] = pb["lo"][d]
        p.hi[d] = pb["hi"][d]
    if pb["dim"] == 1:
        p.K[1] = 1
        p.lo[1], p.hi[1] = 0.0, 1.0
    p.N = pb["N"]
    keep = []

    def nodal(spec):
        # ("nodal", values at the nodes[, values at the interface points])
        arrs = [_f64(a).ravel() if a is not None else None for a in (list(spec[1:]) + [None])[:2]]
        keep.extend(a for a in arrs if a is not None)
        return _dp(arrs[0]), _dp(arrs[1])

    p.drift_kind = _DRIFT[pb["drift"][0]]
    if pb["drift"][0] == "nodal":
        p.drift_nodal, p.drift_face = nodal(pb["drift"])
    else:
        for i, v in enumerate(pb["drift"][1]):
            p.drift_p[i] = v
    p.diff_kind = _DIFF[pb["diffusion"][0]]
    if pb["diffusion"][0] == "nodal":
        p.diff_nodal, p.diff_face = nodal(pb["diffusion"])
    else:
        for i, v in enumerate(pb["diffusion"][1]):
            p.diff_p[i] = v
    p._keep = keep  # the nodal arrays live as long as the struct
    p.phi0_kind = _PHI0[pb["phi0"][0]]
    for i, v in enumerate(pb["phi0"][1]):
        p.phi0_p[i] = v
    p.seed = pb["seed"]
    p.dt = float(dt if dt is not None else (pb["dt"] or 0.0))
    p.omega = float(pb.get("bc_weight", 1.0) or 1.0)
    p.periodic = 1 if pb.get("periodic", True) else 0
    p.reseed_every = int(pb.get("reseed_every", 0) or 0)
    return p


def shape(pb):
    """(elements, nodes per element) of a problem."""
    E = int(np.prod(pb["K"]))
    n = pb["N"] ** pb["dim"]
    return E, n


# --------------------------------------------------------------------------- primitives
def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def log(x):
    return lib().orc_log(float(x))


def sincospi(y):
    s, c = C.c_double(), C.c_double()
    lib().orc_sincospi(float(y), C.byref(s), C.byref(c))
    return s.value, c.value


def normals(seed, step, sample, tag=0):
    z = np.zeros(2)
    lib().orc_normals(seed, step, sample, tag, _dp(z))
    return z


def wiener(seed, dim, M, step0, nsteps, dt):
    """dW[step][sample][dim] (float64)."""
    out = np.zeros((nsteps, M, dim))
    lib().orc_wiener(seed, dim, M, step0, nsteps, dt, _dp(out))
    return out


def nodes(N):
    xi = np.zeros(N)
    lib().orc_nodes(N, _dp(xi))
    return xi


def lagrange(pts, j, x):
    pts = _f64(pts)
    return lib().orc_lagrange(len(pts), _dp(pts), j, float(x))


def lagrange_deriv(pts, j, x):
    pts = _f64(pts)
    return lib().orc_lagrange_deriv(len(pts), _dp(pts), j, float(x))


def quad_weights(N):
    w = np.zeros(N)
    lib().orc_quad_weights(N, _dp(w))
    return w


def lu_solve(A, b):
    A, b = _f64(A), _f64(b)
    x = np.zeros(len(b))
    rc = lib().orc_lu_solve(len(b), _dp(A), _dp(b), _dp(x))
    if rc != 0:
        raise np.linalg.LinAlgError("singular")
    return x


def lstsq(A, b):
    A, b = _f64(A), _f64(b)
    x = np.zeros(A.shape[1])
    rc = lib().orc_lstsq(A.shape[0], A.shape[1], _dp(A), _dp(b), _dp(x))
    if rc != 0:
        raise np.linalg.LinAlgError("rank deficient")
    return x


def faces_1d(xs, phs):
    xs, phs = _f64(xs), _f64(phs)
    e0, e1 = C.c_double(), C.c_double()
    lib().orc_faces_1d(len(xs), _dp(xs), _dp(phs), C.byref(e0), C.byref(e1))
    return e0.value, e1.value


def remap_1d(xs, phs, gL, gR):
    xs, phs = _f64(xs), _f64(phs)
    N = len(xs)
    xi = nodes(N)
    q = np.zeros(N)
    if lib().orc_remap_1d(N, _dp(xi), _dp(xs), _dp(phs), gL, gR, _dp(q)) != 0:
        raise np.linalg.LinAlgError("remap failed")
    return q


def faces_2d(xs, ys, phs):
    xs, ys, phs = _f64(xs), _f64(ys), _f64(phs)
    N = int(round(np.sqrt(len(xs))))
    xi = nodes(N)
    f = np.zeros(4 * N)
    if lib().orc_faces_2d(N, _dp(xi), _dp(xs), _dp(ys), _dp(phs), _dp(f)) != 0:
        raise np.linalg.LinAlgError("singular")
    return f


def remap_2d(xs, ys, phs, g):
    xs, ys, phs, g = _f64(xs), _f64(ys), _f64(phs), _f64(g)
    N = int(round(np.sqrt(len(xs))))
    xi = nodes(N)
    q = np.zeros(N * N)
    if lib().orc_remap_2d(N, _dp(xi), _dp(xs), _dp(ys), _dp(phs), _dp(g), _dp(q)) != 0:
        raise np.linalg.LinAlgError("remap failed")
    return q


def lagrange_split(base, off, j, xb, xo):
    base, off = _f64(base), _f64(off)
    return lib().orc_lagrange_split(len(base), _dp(base), _dp(off), j, float(xb), float(xo))


def faces_1d_split(d, phs):
    """Face values with the particles at the Gauss nodes plus d."""
    d, phs = _f64(d), _f64(phs)
    xi = nodes(len(d))
    e0, e1 = C.c_double(), C.c_double()
    lib().orc_faces_1d_split(len(d), _dp(xi), _dp(d), _dp(phs), C.byref(e0), C.byref(e1))
    return e0.value, e1.value


def remap_1d_split(d, phs, gL, gR, w=None):
    """1D remap; w weights the boundary rows (None: the unweighted form,
    inf: hard constraints)."""
    d, phs = _f64(d), _f64(phs)
    N = len(d)
    xi = nodes(N)
    q = np.zeros(N)
    rc = (lib().orc_remap_1d_split(N, _dp(xi), _dp(d), _dp(phs), gL, gR, _dp(q)) if w is None else
          lib().orc_remap_1d_split_w(N, _dp(xi), _dp(d), _dp(phs), gL, gR, float(w), _dp(q)))
    if rc != 0:
        raise np.linalg.LinAlgError("remap failed")
    return q


def faces_2d_split(dx, dy, phs):
    dx, dy, phs = _f64(dx), _f64(dy), _f64(phs)
    N = int(round(np.sqrt(len(dx))))
    xi = nodes(N)
    f = np.zeros(4 * N)
    if lib().orc_faces_2d_split(N, _dp(xi), _dp(dx), _dp(dy), _dp(phs), _dp(f)) != 0:
        raise np.linalg.LinAlgError("singular")
    return f


def remap_2d_split(dx, dy, phs, g, w=None):
    dx, dy, phs, g = _f64(dx), _f64(dy), _f64(phs), _f64(g)
    N = int(round(np.sqrt(len(dx))))
    xi = nodes(N)
    q = np.zeros(N * N)
    rc = (lib().orc_remap_2d_split(N, _dp(xi), _dp(dx), _dp(dy), _dp(phs), _dp(g), _dp(q)) if w is None else
          lib().orc_remap_2d_split_w(N, _dp(xi), _dp(dx), _dp(dy), _dp(phs), _dp(g), float(w), _dp(q)))
    if rc != 0:
        raise np.linalg.LinAlgError("remap failed")
    return q


# --------------------------------------------------------------------------- problems
def init_state(pb):
    E, n = shape(pb)
    out = np.zeros((E, n))
    p = _problem(pb, dt=0.0)
    if lib().orc_init_state(C.byref(p), _dp(out)) != 0:
        raise ValueError("bad problem")
    return out


def coeffs(pb, dt=None):
    """Node coefficients (a_x, a_y, b, c), each [E][n]."""
    E, n = shape(pb)
    ax, ay, b, c = (np.zeros((E, n)) for _ in range(4))
    p = _problem(pb, dt)
    if lib().orc_get_coeffs(C.byref(p), _dp(ax), _dp(ay), _dp(b), _dp(c)) != 0:
        raise ValueError("bad problem")
    return ax, ay, b, c


def n_interface_points(pb):
    """Length of the interface table of a nodal field: K+1 in 1D; in 2D
    Ky (Kx+1) N vertical then (Ky+1) Kx N horizontal interface points."""
    if pb["dim"] == 1:
        return pb["K"][0] + 1
    Kx, Ky, N = pb["K"][0], pb["K"][1], pb["N"]
    return Ky * (Kx + 1) * N + (Ky + 1) * Kx * N


def face_coeffs(pb, dt=None):
    """Interface coefficients (a = u_normal dt, b = sqrt(2 D)) in the interface
    layout of ``n_interface_points`` (the last interface of a periodic line
    repeats the first)."""
    nf = n_interface_points(pb)
    a, b = np.zeros(nf), np.zeros(nf)
    p = _problem(pb, dt)
    if lib().orc_get_face_coeffs(C.byref(p), _dp(a), _dp(b)) != 0:
        raise ValueError("bad problem")
    return a, b


def dt_max(pb):
    p = _problem(pb, dt=0.0)
    return lib().orc_dt_max(C.byref(p))


def dt_edge(pb):
    p = _problem(pb, dt=0.0)
    return lib().orc_dt_edge(C.byref(p))


def run(pb, nsteps=None, step0=0, s0=0, ns=None, nthreads=1, state_in=None,
        want_states=False, want_sums=True, dt=None, ghost=None):
    """Run samples [s0, s0+ns) through steps [step0, step0+nsteps).
    ghost: [nsteps][width] Dirichlet values after each step (pb["periodic"]
    False; default pb["ghost"] when present): 1D x = lo, hi (width 2); 2D the
    face points of the left, right, bottom and top boundaries (width
    2 (Kx + Ky) N).

    Returns dict with 'states' ([ns][E][n], if asked) and 'sum', 'sumsq'
    ([E][n], sums over the ns samples)."""
    E, n = shape(pb)
    nsteps = pb["steps"] if nsteps is None else nsteps
    ns = pb["M"] if ns is None else ns
    p = _problem(pb, dt)
    sin = None if state_in is None else _f64(state_in).reshape(ns, E, n)
    st = np.zeros((ns, E, n)) if want_states else None
    sm = np.zeros((E, n)) if want_sums else None
    sq = np.zeros((E, n)) if want_sums else None
    if ghost is None:
        ghost = pb.get("ghost")
    width = 2 if pb["dim"] == 1 else 2 * (pb["K"][0] + pb["K"][1]) * pb["N"]
    gh = None if ghost is None else np.ascontiguousarray(np.asarray(ghost, dtype=np.float64).reshape(-1, width)[:nsteps])
    if gh is not None and gh.shape[0] < nsteps:
        raise ValueError("ghost values cover fewer steps than the run")
    rc = lib().orc_run(C.byref(p), step0, nsteps, s0, ns, nthreads, _dp(gh), _dp(sin), _dp(st), _dp(sm), _dp(sq))
    if rc != 0:
        raise RuntimeError("oracle run failed (singular remap or bad problem)")
    return {"states": st, "sum": sm, "sumsq": sq}


def moments(pb, **kw):
    """(mean, m2) over all M samples: (1/M) sum_s Q^s and (1/M) sum_s (Q^s)^2
    (Eq. averaged)."""
    r = run(pb, **kw)
    M = pb["M"] if kw.get("ns") is None else kw["ns"]
    return r["sum"] / M, r["sumsq"] / M


def pdf(states, nbins, lo, hi):
    """The PDF at every node recovered by binning the samples (Section 5.4):
    states [M][E][n] -> counts [E][n][nbins] (uint32); bin b = floor((x - lo)
    * (nbins / (hi - lo))) in FP64, x = hi in the last bin, x outside [lo, hi]
    or NaN not counted."""
    x = np.asarray(states, dtype=np.float64)
    M = x.shape[0]
    flat = x.reshape(M, -1)
    scale = float(nbins) / (hi - lo)
    counts = np.zeros((flat.shape[1], nbins), dtype=np.uint32)
    for v in range(flat.shape[1]):
        for s in range(M):
            xv = flat[s, v]
            if not (xv >= lo and xv <= hi):
                continue
            b = int(np.floor((xv - lo) * scale))
            counts[v, min(b, nbins - 1)] += 1
    return counts.reshape(x.shape[1:] + (nbins,))


def node_coords(pb):
    """Physical coordinates of every node, [E][n] (x) and [E][n] (y, 2D)."""
    xi = nodes(pb["N"])
    N = pb["N"]
    if pb["dim"] == 1:
        K = pb["K"][0]
        h = (pb["hi"][0] - pb["lo"][0]) / K
        x = pb["lo"][0] + (np.arange(K)[:, None] + xi[None, :]) * h
        return x, None
    Kx, Ky = pb["K"]
    hx = (pb["hi"][0] - pb["lo"][0]) / Kx
    hy = (pb["hi"][1] - pb["lo"][1]) / Ky
    E = Kx * Ky
    x = np.zeros((E, N * N))
    y = np.zeros((E, N * N))
    for e in range(E):
        kx, ky = e % Kx, e // Kx
        for p in range(N * N):
            i, j = p % N, p // N
            x[e, p] = pb["lo"][0] + (kx + xi[i]) * hx
            y[e, p] = pb["lo"][1] + (ky + xi[j]) * hy
    return x, y
