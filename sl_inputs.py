"""Seeded synthetic workloads for the semi-Lagrangian Monte-Carlo solver.

This module only describes inputs: mesh sizes, sample counts, step counts,
time steps, seeds and the parameters of the prescribed drift, diffusion and
initial-condition fields.  It holds none of the method's arithmetic, so both
the FP64 CPU oracle (tests) and the CUDA library (tests, benchmark) can take
their inputs from it without sharing any computation.

A problem is a plain dict::

    {"dim": 1, "K": (8,), "lo": (0.0,), "hi": (2.0,), "N": 6, "M": 256,
     "steps": 100, "dt": 6.510e-4, "seed": 1,
     "drift": ("const", [1.0]), "diffusion": ("const", [0.01]),
     "phi0": ("gauss", [1.0, 0.1, 1.0, 0.0])}

Field kinds (parameters p0, p1, ...):

drift      "const"    u = (p0, p1)
           "sin"      u = p0 + p1 sin(p2 pi x)                         (1D)
           "rotation" u = p0 (-(y - p2), x - p1)                        (2D)
diffusion  "const"    D = p0
           "cos"      D = p0 (1 + p1 cos(p2 pi x))
           "sinsin"   D = p0 (1 + p1 sin(p2 pi x) sin(p3 pi y))
phi0       "gauss"    p0 exp(-|x - (p2, p3)|^2 / (2 p1^2)), with the nearest
                      periodic images in each direction
           "fourier"  p0 + sum_{k=1}^{p2} (a_k cos(k p1 pi x) + b_k sin(k p1 pi x)),
                      a_k = p[3 + 2(k-1)], b_k = p[4 + 2(k-1)]        (1D)
           "sine"     p0 + p1 sin(2 pi p2 x)                            (1D)
           "sinsin"   p0 + p1 sin(2 pi p2 x) sin(2 pi p2 y)             (2D)

The workloads stand in for the paper's own synthetic analytic tests
(Section 6); the paper uses no dataset.
"""

from __future__ import annotations

import copy

import numpy as np

# Stable time steps from the particle-gap condition of Eq. (1d_timestep),
# stated once here as plain numbers so that every consumer runs the same dt.
DT_CFG1 = 6.510e-4  # K=8, N=6, u=1, D=0.01, edge gap: particles stay in-element at 1 sigma
DT_CFG2 = 7.33e-7   # K=256, N=16 node gap, |u|max=1.5, Dmax=0.015 (used for every N)
DT_CFG2_HALF = 3.665e-7  # half of it: at DT_CFG2 itself the N=16 step amplifies perturbations
DT_CFG3 = 6.93e-5   # 64x64, N=8 node gap, |u_j|max=pi, Dmax=0.0065
DT_CFG3_HALF = 3.465e-5  # half of it: at DT_CFG3 itself the 2D step amplifies perturbations ~12 %/step
DT_CFG3_EDGE = 1.618e-6  # the same with the first node's distance to the face (particles stay inside)


def problem(dim, K, lo, hi, N, M, steps, dt, seed, drift, diffusion, phi0):
    """Normalised problem dict (tuples for the mesh, lists for parameters)."""
    return {
        "dim": int(dim), "K": tuple(int(k) for k in K), "lo": tuple(float(v) for v in lo),
        "hi": tuple(float(v) for v in hi), "N": int(N), "M": int(M), "steps": int(steps),
        "dt": float(dt), "seed": int(seed),
        "drift": (drift[0], [float(v) for v in drift[1]]),
        "diffusion": (diffusion[0], [float(v) for v in diffusion[1]]),
        "phi0": (phi0[0], [float(v) for v in phi0[1]]),
    }


def with_(pb, **kw):
    """Copy of a problem with some entries replaced."""
    q = copy.deepcopy(pb)
    q.update(kw)
    return q


def config1():
    """1D constant drift-diffusion, periodic [0,2], K=8, N=6, M=256, u=1,
    D=0.01, Gaussian pulse (centre 1.0, sigma 0.1), 100 steps."""
    return problem(1, (8,), (0.0,), (2.0,), 6, 256, 100, DT_CFG1, 1,
                   ("const", [1.0, 0.0]), ("const", [0.01]), ("gauss", [1.0, 0.1, 1.0, 0.0]))


def fourier_phi0(seed=2, modes=8):
    """phi0 = 1 + 0.5 sum_k (a_k cos k pi x + b_k sin k pi x) / sum_k(|a_k|+|b_k|),
    a_k, b_k ~ U(-1, 1) (numpy PCG64, seeded), so phi0 lies in [0.5, 1.5]."""
    rng = np.random.default_rng(seed)
    ab = rng.uniform(-1.0, 1.0, size=(modes, 2))
    scale = 0.5 / np.abs(ab).sum()
    p = [1.0, 1.0, float(modes)]
    for k in range(modes):
        p += [float(ab[k, 0] * scale), float(ab[k, 1] * scale)]
    return ("fourier", p)


def config2(N=16, M=4096, steps=1000, K=256, dt=DT_CFG2):
    """1D non-constant drift-diffusion, periodic [0,2], K=256, N in {4,8,12,16},
    M=4096, u = 1 + 0.5 sin(pi x), D = 0.01 (1 + 0.5 cos(pi x)), random
    8-mode Fourier phi0 (seed 2), 1000 steps at the N=16 particle-gap dt (or
    the dt given)."""
    return problem(1, (K,), (0.0,), (2.0,), N, M, steps, dt, 2,
                   ("sin", [1.0, 0.5, 1.0]), ("cos", [0.01, 0.5, 1.0]), fourier_phi0(2))


def config3(M=1024, steps=500, K=64, N=8, dt=DT_CFG3):
    """2D periodic [0,1]^2, 64x64 elements, N=8, M=1024, solid-body rotation
    (omega = 2 pi) about (0.5, 0.5), D = 0.005 (1 + 0.3 sin 2 pi x sin 2 pi y),
    Gaussian blob (0.5, 0.75), sigma 0.05, 500 steps (node-gap dt, or the
    dt given)."""
    return problem(2, (K, K), (0.0, 0.0), (1.0, 1.0), N, M, steps, dt, 3,
                   ("rotation", [2.0 * np.pi, 0.5, 0.5]), ("sinsin", [0.005, 0.3, 2.0, 2.0]),
                   ("gauss", [1.0, 0.05, 0.5, 0.75]))


def sine_diffusion_1d(K=1, N=8, M=1000, steps=50):
    """The paper's first test (Section 6.1): u = 0, D = 1, phi0 = sin(2 pi x) + 2
    on periodic [0,1], dt = 1e-5, 50 steps."""
    return problem(1, (K,), (0.0,), (1.0,), N, M, steps, 1e-5, 11,
                   ("const", [0.0, 0.0]), ("const", [1.0]), ("sine", [2.0, 1.0, 1.0]))


def batch_instances(count=512, seed=4, steps=100):
    """Uneven 2D instances: side K ~ U{16..64}, N ~ U{4..12},
    M ~ U{256, 512, 1024, 2048}, drift constant (u ~ U[-1,1]^2) or rotation
    (omega = 2 pi) with probability 1/2, constant D ~ U[1e-3, 1e-2], Gaussian
    blob phi0.  dt is left as None (the caller takes a fraction of the
    stable dt); each instance has its own seed."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        K = int(rng.integers(16, 65))
        N = int(rng.integers(4, 13))
        M = int(rng.choice([256, 512, 1024, 2048]))
        if rng.random() < 0.5:
            drift = ("const", [float(rng.uniform(-1, 1)), float(rng.uniform(-1, 1))])
        else:
            drift = ("rotation", [2.0 * np.pi, 0.5, 0.5])
        D = float(rng.uniform(1e-3, 1e-2))
        cx, cy = (float(v) for v in rng.uniform(0.35, 0.65, size=2))
        pb = problem(2, (K, K), (0.0, 0.0), (1.0, 1.0), N, M, steps, 0.0, 1000 + i,
                     drift, ("const", [D]), ("gauss", [1.0, 0.05, cx, cy]))
        pb["dt"] = None
        out.append(pb)
    return out


def small_instances_1d(count=256, seed=46, steps=20):
    """Many small uneven 1D instances (the case batching is for): K ~ U{8..64},
    N ~ U{4..8}, M ~ U{16..128}, the fields of config 2, each its own seed.
    dt is left as None."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        pb = config2(N=int(rng.integers(4, 9)), M=int(rng.integers(16, 129)), steps=steps,
                     K=int(rng.integers(8, 65)))
        pb["seed"] = 9000 + i
        pb["dt"] = None
        out.append(pb)
    return out


def serving_requests(rate=200.0, duration=60.0, seed=5, steps=20):
    """Poisson arrivals (mean `rate` per second) over `duration` seconds.  Each
    request is, with probability 1/2, a 2D instance drawn like
    `batch_instances`, else a 1D instance with K ~ U{64..1024},
    N ~ U{4..16}, M ~ U{256..2048} and the drift / diffusion of config 2.
    Returns a list of (arrival_time_s, problem); dt is left as None."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    i = 0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            break
        if rng.random() < 0.5:
            pb = batch_instances(1, seed=int(rng.integers(1 << 31)), steps=steps)[0]
        else:
            K = int(rng.integers(64, 1025))
            N = int(rng.integers(4, 17))
            M = int(rng.integers(256, 2049))
            pb = problem(1, (K,), (0.0,), (2.0,), N, M, steps, 0.0, 50000 + i,
                         ("sin", [1.0, 0.5, 1.0]), ("cos", [0.01, 0.5, 1.0]),
                         fourier_phi0(int(rng.integers(1 << 31))))
            pb["dt"] = None
        reqs.append((t, pb))
        i += 1
    return reqs
