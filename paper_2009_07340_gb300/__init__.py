"""GB300 (sm_103a) semi-Lagrangian Monte-Carlo solver -- Python binding.

Thin ctypes marshalling over the C ABI of ``include/sl.h`` (``libsl.so``):
every step of the method runs in the library's CUDA kernels; this module
only converts Python arguments to the C structs and buffers.  There is no
CPU fallback: if ``libsl.so`` has not been built, or no CUDA device is
present, calls raise.

Problems are the plain dicts of ``sl_inputs`` (mesh, N, M, field kinds and
parameters, dt, seed).
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = ["SL_FP64", "SL_MIXED", "SL_FP32", "SLError", "Solver", "lib", "sl_init", "sl_step",
           "sl_moments", "sl_moments_device", "sl_dt_max", "sl_step_count", "sl_get_samples",
           "sl_set_samples", "sl_set_step_count", "sl_wiener", "sl_dt_edge", "sl_profile", "sl_profile_read",
           "sl_fallback_count",
           "sl_moments_static", "sl_moments_partial", "sl_moment_chunk", "sl_moments_combine", "sl_free",
           "sl_strerror"]

SL_FP64, SL_MIXED, SL_FP32 = 0, 1, 2
PRECISIONS = {"fp64": SL_FP64, "mixed": SL_MIXED, "fp32": SL_FP32}

_U = {"const": 1, "sin": 2, "rotation": 3, "nodal": 4}
_D = {"const": 11, "cos": 12, "sinsin": 13, "nodal": 14}
_PHI = {"gauss": 21, "fourier": 22, "sine": 23, "sinsin": 24, "nodal": 25}


class SLError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {sl_strerror(code)} ({code})")


class sl_field(C.Structure):
    _fields_ = [("kind", C.c_int), ("p", C.c_double * 40), ("nodal", C.POINTER(C.c_double)),
                ("face", C.POINTER(C.c_double))]


class sl_mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("K", C.c_int * 2), ("lo", C.c_double * 2), ("hi", C.c_double * 2),
                ("periodic", C.c_int * 2)]


class sl_options(C.Structure):
    _fields_ = [("seed", C.c_ulonglong), ("precision", C.c_int), ("strict_dt", C.c_int),
                ("stream", C.c_void_p), ("device", C.c_int), ("sample0", C.c_longlong),
                ("bc_weight", C.c_double), ("launch_chunk", C.c_longlong), ("components", C.c_int),
                ("reseed_every", C.c_int)]


class sl_instance(C.Structure):
    _fields_ = [("mesh", sl_mesh), ("N", C.c_int), ("M", C.c_int), ("drift", sl_field),
                ("diffusion", sl_field), ("phi0", sl_field), ("dt", C.c_double), ("dt_rule", C.c_int),
                ("seed", C.c_ulonglong), ("bc_weight", C.c_double)]


class sl_server_config(C.Structure):
    _fields_ = [("budget_bytes", C.c_size_t), ("slice_steps", C.c_int), ("heavy_slots", C.c_int),
                ("precision", C.c_int), ("device", C.c_int), ("max_active", C.c_int)]


class sl_server_stats(C.Structure):
    _fields_ = [(n, C.c_longlong) for n in ("submitted", "completed", "rejected", "failed", "running", "queued",
                                             "esu_completed", "memory_in_use", "memory_peak")] + \
               [(n, C.c_double) for n in ("p50_s", "p99_s", "mean_s", "span_s", "esu_per_s")] + \
               [("slices", C.c_longlong)] + [(n, C.c_double) for n in ("sched_busy_s", "launch_s", "launch_max_s")]


_lib = None
_dp = C.POINTER(C.c_double)


def lib():
    """Loads libsl.so (built in-tree by ``build.build()``); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libsl.so is not built: run paper_2009_07340_gb300.build.build() "
                               "(nvcc, sm_103a); there is no CPU fallback")
        L = C.CDLL(_build.LIB)
        vp = C.c_void_p
        L.sl_init.argtypes = [C.POINTER(vp), C.POINTER(sl_mesh), C.c_int, C.c_int, C.POINTER(sl_field),
                              C.POINTER(sl_field), C.POINTER(sl_field), C.POINTER(sl_options)]
        L.sl_step.argtypes = [vp, C.c_double, C.c_int]
        L.sl_preload.argtypes = [C.c_int]
        L.sl_set_boundary.argtypes = [vp, C.c_int, _dp]
        L.sl_reseed.argtypes = [vp]
        L.sl_set_fields.argtypes = [vp, C.POINTER(sl_field), C.POINTER(sl_field)]
        L.sl_set_fields_device.argtypes = [vp, C.POINTER(sl_field), C.POINTER(sl_field)]
        L.sl_pdf.argtypes = [vp, C.c_int, C.c_double, C.c_double, C.POINTER(C.c_uint32)]
        L.sl_pdf_device.argtypes = [vp, C.c_int, C.c_double, C.c_double, vp]
        L.sl_moments.argtypes = [vp, _dp, _dp]
        L.sl_moments_device.argtypes = [vp, vp, vp]
        L.sl_dt_max.argtypes = [vp, _dp]
        L.sl_dt_edge.argtypes = [vp, _dp]
        L.sl_step_count.argtypes = [vp, C.POINTER(C.c_longlong)]
        L.sl_fallback_count.argtypes = [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
        L.sl_set_step_count.argtypes = [vp, C.c_longlong]
        L.sl_get_samples.argtypes = [vp, C.c_int, C.c_int, _dp]
        L.sl_set_samples.argtypes = [vp, C.c_int, C.c_int, _dp]
        L.sl_wiener.argtypes = [vp, C.c_longlong, C.c_int, C.c_double, _dp]
        L.sl_profile.argtypes = [vp, C.c_int]
        L.sl_profile_read.argtypes = [vp, _dp, C.POINTER(C.c_longlong)]
        L.sl_moments_static.argtypes = [vp, C.c_int, C.c_longlong, vp, vp, vp]
        L.sl_moments_partial.argtypes = [vp, vp, vp]
        L.sl_moment_chunk.argtypes = []
        L.sl_moments_combine.argtypes = [vp, vp, C.c_int, C.c_longlong, C.c_longlong, vp, vp, vp]
        L.sl_batch_create.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(sl_instance), C.POINTER(sl_options)]
        L.sl_batch_step.argtypes = [vp, C.c_int]
        L.sl_batch_tune.argtypes = [vp, C.c_int, _dp]
        L.sl_batch_grid.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.sl_batch_lanes.argtypes = [vp, C.POINTER(C.c_int)]
        L.sl_batch_moments.argtypes = [vp, C.c_int, _dp, _dp]
        L.sl_batch_samples.argtypes = [vp, C.c_int, C.c_int, C.c_int, _dp]
        L.sl_batch_free.argtypes = [vp]
        L.sl_batch_free.restype = None
        L.sl_server_create.argtypes = [C.POINTER(vp), C.POINTER(sl_server_config)]
        L.sl_server_submit.argtypes = [vp, C.POINTER(sl_instance), C.c_int, C.POINTER(C.c_longlong)]
        L.sl_server_poll.argtypes = [vp, C.c_longlong, C.POINTER(C.c_int), _dp, _dp, _dp]
        L.sl_server_wait_idle.argtypes = [vp, C.c_double]
        L.sl_server_timing.argtypes = [vp, C.c_longlong, _dp]
        L.sl_server_stats_get.argtypes = [vp, C.POINTER(sl_server_stats)]
        L.sl_server_free.argtypes = [vp]
        L.sl_server_free.restype = None
        L.sl_free.argtypes = [vp]
        L.sl_free.restype = None
        L.sl_strerror.argtypes = [C.c_int]
        L.sl_strerror.restype = C.c_char_p
        _lib = L
    return _lib


def sl_strerror(code):
    try:
        return lib().sl_strerror(int(code)).decode()
    except RuntimeError:
        return f"error {code}"


def _check(rc, where):
    if rc != 0:
        raise SLError(rc, where)


def _field(kind_map, spec):
    """sl_field of a problem-dict field: (kind, parameters), or ("nodal",
    node values[, interface values]) with host arrays the struct keeps alive."""
    f = sl_field()
    f.kind = kind_map[spec[0]]
    if spec[0] == "nodal":
        f._keep = [np.ascontiguousarray(np.asarray(a, dtype=np.float64).ravel()) for a in spec[1:3] if a is not None]
        f.nodal = _f64p(f._keep[0])
        if len(f._keep) > 1:
            f.face = _f64p(f._keep[1])
        return f
    for i, v in enumerate(spec[1]):
        f.p[i] = float(v)
    return f


def _mesh(pb):
    m = sl_mesh()
    m.dim = pb["dim"]
    for d in range(pb["dim"]):
        m.K[d] = pb["K"][d]
        m.lo[d] = pb["lo"][d]
        m.hi[d] = pb["hi"][d]
        m.periodic[d] = 1 if pb.get("periodic", True) else 0
    return m


def _f64p(a):
    return a.ctypes.data_as(_dp)


# ------------------------------------------------------------------ C-named wrappers
def sl_init(pb, precision=SL_FP64, seed=None, stream=None, strict_dt=False, device=-1, phi0_nodal=None,
            sample0=0, launch_chunk=0):
    """Returns an opaque context handle (int).  `stream` is a cudaStream_t
    handle (int) or None."""
    mesh = _mesh(pb)
    u = _field(_U, pb["drift"])
    D = _field(_D, pb["diffusion"])
    keep = None
    if phi0_nodal is not None:
        keep = np.ascontiguousarray(phi0_nodal, dtype=np.float64)
        phi = sl_field()
        phi.kind = _PHI["nodal"]
        phi.nodal = _f64p(keep)
    else:
        phi = _field(_PHI, pb["phi0"])
    opt = sl_options()
    opt.seed = int(pb["seed"] if seed is None else seed)
    opt.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    opt.strict_dt = 1 if strict_dt else 0
    opt.stream = C.c_void_p(stream) if stream else None
    opt.device = device
    opt.sample0 = int(sample0)
    opt.launch_chunk = int(launch_chunk)
    opt.bc_weight = float(pb.get("bc_weight", 0.0) or 0.0)
    opt.reseed_every = int(pb.get("reseed_every", 0) or 0)
    opt.components = int(pb.get("components", 1) or 1)
    h = C.c_void_p()
    _check(lib().sl_init(C.byref(h), C.byref(mesh), pb["N"], pb["M"], C.byref(u), C.byref(D), C.byref(phi),
                         C.byref(opt)), "sl_init")
    return h.value


def sl_preload(device=-1):
    """Prepares every kernel of the library on `device` (once per process)."""
    _check(lib().sl_preload(int(device)), "sl_preload")


def sl_step(ctx, dt, steps):
    _check(lib().sl_step(C.c_void_p(ctx), float(dt), int(steps)), "sl_step")


def sl_moments(ctx, V, want_m2=True):
    mean = np.zeros(V)
    m2 = np.zeros(V) if want_m2 else None
    _check(lib().sl_moments(C.c_void_p(ctx), _f64p(mean), _f64p(m2) if want_m2 else None), "sl_moments")
    return mean, m2


def sl_moments_device(ctx, d_mean_ptr, d_m2_ptr=None):
    _check(lib().sl_moments_device(C.c_void_p(ctx), C.c_void_p(d_mean_ptr),
                                   C.c_void_p(d_m2_ptr) if d_m2_ptr else None), "sl_moments_device")


def sl_moments_partial(ctx, d_psum_ptr, d_psq_ptr):
    """Chunk partial sums [ceil(M/64)][V] into caller-owned device memory."""
    _check(lib().sl_moments_partial(C.c_void_p(ctx), C.c_void_p(d_psum_ptr), C.c_void_p(d_psq_ptr)),
           "sl_moments_partial")


def sl_moment_chunk():
    return int(lib().sl_moment_chunk())


def sl_moments_combine(d_psum_ptr, d_psq_ptr, nchunks, V, M_total, d_mean_ptr, d_m2_ptr=None, stream=None):
    """Moments from gathered chunk partials (device pointers), asynchronous on `stream`."""
    _check(lib().sl_moments_combine(C.c_void_p(d_psum_ptr), C.c_void_p(d_psq_ptr), int(nchunks), int(V),
                                    int(M_total), C.c_void_p(d_mean_ptr),
                                    C.c_void_p(d_m2_ptr) if d_m2_ptr else None,
                                    C.c_void_p(stream) if stream else None), "sl_moments_combine")


def sl_dt_max(ctx):
    v = C.c_double()
    _check(lib().sl_dt_max(C.c_void_p(ctx), C.byref(v)), "sl_dt_max")
    return v.value


def sl_dt_edge(ctx):
    v = C.c_double()
    _check(lib().sl_dt_edge(C.c_void_p(ctx), C.byref(v)), "sl_dt_edge")
    return v.value


def sl_step_count(ctx):
    v = C.c_longlong()
    _check(lib().sl_step_count(C.c_void_p(ctx), C.byref(v)), "sl_step_count")
    return v.value


def sl_fallback_count(ctx):
    """(phase 1, phase 2) element-sample groups the 2D iterative solve handed
    to the direct one since the context was created."""
    a, b = C.c_longlong(), C.c_longlong()
    _check(lib().sl_fallback_count(C.c_void_p(ctx), C.byref(a), C.byref(b)), "sl_fallback_count")
    return a.value, b.value


def sl_set_step_count(ctx, n):
    _check(lib().sl_set_step_count(C.c_void_p(ctx), int(n)), "sl_set_step_count")


def sl_get_samples(ctx, s0, count, V):
    out = np.zeros((count, V))
    _check(lib().sl_get_samples(C.c_void_p(ctx), s0, count, _f64p(out)), "sl_get_samples")
    return out


def sl_set_samples(ctx, s0, states):
    a = np.ascontiguousarray(states, dtype=np.float64)
    _check(lib().sl_set_samples(C.c_void_p(ctx), s0, a.shape[0], _f64p(a)), "sl_set_samples")


def sl_wiener(ctx, step0, nsteps, dt, M, dim):
    out = np.zeros((nsteps, M, dim))
    _check(lib().sl_wiener(C.c_void_p(ctx), int(step0), int(nsteps), float(dt), _f64p(out)), "sl_wiener")
    return out


def sl_profile(ctx, enable):
    _check(lib().sl_profile(C.c_void_p(ctx), 1 if enable else 0), "sl_profile")


def sl_profile_read(ctx):
    ms = C.c_double()
    n = C.c_longlong()
    _check(lib().sl_profile_read(C.c_void_p(ctx), C.byref(ms), C.byref(n)), "sl_profile_read")
    return ms.value, n.value


def sl_moments_static(d_samples_ptr, M, V, d_mean_ptr, d_m2_ptr=None, stream=None):
    """Allocation-free moments of caller-owned device FP64 samples [M][V]
    (see include/sl.h: for callers that cannot allocate device memory)."""
    _check(lib().sl_moments_static(C.c_void_p(d_samples_ptr), int(M), int(V), C.c_void_p(d_mean_ptr),
                                   C.c_void_p(d_m2_ptr) if d_m2_ptr else None,
                                   C.c_void_p(stream) if stream else None), "sl_moments_static")


def sl_free(ctx):
    if ctx:
        lib().sl_free(C.c_void_p(ctx))


def _instance(pb, dt=None, seed=None):
    inst = sl_instance()
    inst.mesh = _mesh(pb)
    inst.N = pb["N"]
    inst.M = pb["M"]
    fields = (_field(_U, pb["drift"]), _field(_D, pb["diffusion"]), _field(_PHI, pb["phi0"]))
    inst.drift, inst.diffusion, inst.phi0 = fields
    inst._keep = fields  # the assignment copies the structs, not the nodal arrays they point to
    d = pb["dt"] if dt is None else dt
    # a problem's dt may be ("node", f) / ("edge", f): f times sl_dt_max / sl_dt_edge
    if isinstance(d, (tuple, list)):
        inst.dt_rule = {"node": 1, "edge": 2}[d[0]]
        inst.dt = float(d[1])
    else:
        inst.dt_rule = 0
        inst.dt = float(d)
    inst.seed = int(pb["seed"] if seed is None else seed)
    inst.bc_weight = float(pb.get("bc_weight", 0.0) or 0.0)
    return inst


def sl_batch_create(problems, precision=SL_FP64, stream=None, strict_dt=False, device=-1):
    insts = [_instance(pb) for pb in problems]  # alive until the call returns (nodal arrays)
    arr = (sl_instance * len(problems))(*insts)
    opt = sl_options()
    opt.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    opt.strict_dt = 1 if strict_dt else 0
    opt.stream = C.c_void_p(stream) if stream else None
    opt.device = device
    h = C.c_void_p()
    _check(lib().sl_batch_create(C.byref(h), len(problems), arr, C.byref(opt)), "sl_batch_create")
    return h.value


def sl_batch_step(b, steps):
    _check(lib().sl_batch_step(C.c_void_p(b), int(steps)), "sl_batch_step")


def sl_batch_tune(b, probe_steps=2):
    ms = C.c_double()
    _check(lib().sl_batch_tune(C.c_void_p(b), int(probe_steps), C.byref(ms)), "sl_batch_tune")
    return ms.value


def sl_batch_grid(b, cls):
    N, g, k = C.c_int(), C.c_int(), C.c_int()
    rc = lib().sl_batch_grid(C.c_void_p(b), int(cls), C.byref(N), C.byref(g), C.byref(k))
    return None if rc != 0 else (N.value, g.value, k.value)


def sl_batch_lanes(b):
    v = C.c_int()
    _check(lib().sl_batch_lanes(C.c_void_p(b), C.byref(v)), "sl_batch_lanes")
    return v.value


def sl_batch_moments(b, i, V):
    mean, m2 = np.zeros(V), np.zeros(V)
    _check(lib().sl_batch_moments(C.c_void_p(b), int(i), _f64p(mean), _f64p(m2)), "sl_batch_moments")
    return mean, m2


def sl_batch_samples(b, i, s0, count, V):
    out = np.zeros((count, V))
    _check(lib().sl_batch_samples(C.c_void_p(b), int(i), int(s0), int(count), _f64p(out)), "sl_batch_samples")
    return out


def sl_batch_free(b):
    if b:
        lib().sl_batch_free(C.c_void_p(b))


class Batch:
    """Many independent problems advanced together (see include/sl.h)."""

    def __init__(self, problems, precision="fp64", stream=None, strict_dt=False):
        self.problems = problems
        self.V = [int(np.prod(pb["K"])) * pb["N"] ** pb["dim"] for pb in problems]
        self.h = sl_batch_create(problems, precision, stream, strict_dt)

    def step(self, steps):
        sl_batch_step(self.h, steps)

    def tune(self, probe_steps=2):
        return sl_batch_tune(self.h, probe_steps)

    def grids(self):
        out, c = [], 0
        while True:
            g = sl_batch_grid(self.h, c)
            if g is None:
                return out
            out.append(g)
            c += 1

    def lanes(self):
        """Parallel graph branches of a step (chosen by tune())."""
        return sl_batch_lanes(self.h)

    def moments(self, i):
        pb = self.problems[i]
        E, n = int(np.prod(pb["K"])), pb["N"] ** pb["dim"]
        mean, m2 = sl_batch_moments(self.h, i, self.V[i])
        return mean.reshape(E, n), m2.reshape(E, n)

    def samples(self, i, s0=0, count=None):
        pb = self.problems[i]
        count = pb["M"] - s0 if count is None else count
        return sl_batch_samples(self.h, i, s0, count, self.V[i])

    def close(self):
        if self.h:
            sl_batch_free(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server of drift-diffusion solves (see include/sl.h)."""

    def __init__(self, budget_bytes, slice_steps=10, heavy_slots=2, precision="fp32", device=-1, max_active=0):
        cfg = sl_server_config()
        cfg.budget_bytes = int(budget_bytes)
        cfg.slice_steps = int(slice_steps)
        cfg.heavy_slots = int(heavy_slots)
        cfg.max_active = int(max_active)
        cfg.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        cfg.device = device
        h = C.c_void_p()
        _check(lib().sl_server_create(C.byref(h), C.byref(cfg)), "sl_server_create")
        self.h = h.value
        self.V = {}

    def submit(self, pb, steps=None):
        inst = _instance(pb)
        t = C.c_longlong()
        _check(lib().sl_server_submit(C.c_void_p(self.h), C.byref(inst), int(pb["steps"] if steps is None else steps),
                                      C.byref(t)), "sl_server_submit")
        self.V[t.value] = int(np.prod(pb["K"])) * pb["N"] ** pb["dim"]
        return t.value

    def poll(self, ticket, want=True):
        st = C.c_int()
        lat = C.c_double()
        V = self.V[ticket]
        mean = np.zeros(V) if want else None
        m2 = np.zeros(V) if want else None
        _check(lib().sl_server_poll(C.c_void_p(self.h), int(ticket), C.byref(st), _f64p(mean) if want else None,
                                    _f64p(m2) if want else None, C.byref(lat)), "sl_server_poll")
        return st.value, (mean, m2, lat.value) if st.value == 2 else None

    def timing(self, ticket):
        """Phases of a completed request in seconds: (queued, creation wait,
        creation, running, completion wait, moments, release, total, longest
        slice)."""
        out = np.zeros(9)
        _check(lib().sl_server_timing(C.c_void_p(self.h), int(ticket), _f64p(out)), "sl_server_timing")
        return tuple(float(v) for v in out)

    def wait_idle(self, timeout_s=600.0):
        _check(lib().sl_server_wait_idle(C.c_void_p(self.h), float(timeout_s)), "sl_server_wait_idle")

    def stats(self):
        st = sl_server_stats()
        _check(lib().sl_server_stats_get(C.c_void_p(self.h), C.byref(st)), "sl_server_stats_get")
        return {f: getattr(st, f) for f, _ in sl_server_stats._fields_}

    def close(self):
        if self.h:
            lib().sl_server_free(C.c_void_p(self.h))
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ convenience
class Solver:
    """One solver context for a problem dict (see ``sl_inputs``)."""

    def __init__(self, pb, precision="fp64", seed=None, stream=None, strict_dt=False, phi0_nodal=None,
                 sample0=0, launch_chunk=0):
        self.pb = pb
        self.E = int(np.prod(pb["K"]))
        self.n = pb["N"] ** pb["dim"]
        self.ncomp = int(pb.get("components", 1) or 1)
        self.V = self.ncomp * self.E * self.n  # values per sample
        self.M = pb["M"]
        self.dim = pb["dim"]
        self._shape = (self.E, self.n) if self.ncomp == 1 else (self.ncomp, self.E, self.n)
        self.ctx = sl_init(pb, precision, seed, stream, strict_dt, phi0_nodal=phi0_nodal, sample0=sample0,
                           launch_chunk=launch_chunk)
        if not pb.get("periodic", True) and pb.get("ghost") is not None:
            self.set_boundary(pb["ghost"])

    def set_boundary(self, values):
        """Dirichlet values after each of the next steps: [steps][2] in 1D (x = lo,
        hi); [steps][2 (Kx + Ky) N] in 2D (left, right, bottom, top face points)."""
        pb = self.pb
        width = 2 if pb["dim"] == 1 else 2 * (pb["K"][0] + pb["K"][1]) * pb["N"]
        v = np.ascontiguousarray(np.asarray(values, dtype=np.float64).reshape(-1, width))
        _check(lib().sl_set_boundary(C.c_void_p(self.ctx), v.shape[0], _f64p(v)), "sl_set_boundary")

    def pdf(self, nbins, lo, hi):
        """Per-node histogram of the samples, uint32 [E][n][nbins] (see sl_pdf)."""
        out = np.zeros(self._shape + (int(nbins),), dtype=np.uint32)
        _check(lib().sl_pdf(C.c_void_p(self.ctx), int(nbins), float(lo), float(hi),
                            out.ctypes.data_as(C.POINTER(C.c_uint32))), "sl_pdf")
        return out

    def set_fields(self, drift, diffusion):
        """New drift and diffusion (problem-dict form, e.g. ("sin", [...])) for the following steps."""
        u, D = _field(_U, drift), _field(_D, diffusion)
        _check(lib().sl_set_fields(C.c_void_p(self.ctx), C.byref(u), C.byref(D)), "sl_set_fields")
        self.pb = dict(self.pb, drift=drift, diffusion=diffusion)

    def set_fields_device(self, drift, diffusion):
        """New drift and diffusion from device memory (sl_set_fields_device):
        ("nodal", tensor[, tensor]) with contiguous float64 CUDA tensors (or
        an analytic form).  Stream-ordered, no copy; the tensors must stay
        alive and unchanged until the next step has run."""
        import torch

        def dev_field(kind_map, spec):
            if spec[0] != "nodal":
                return _field(kind_map, spec)
            f = sl_field()
            f.kind = kind_map["nodal"]
            tabs = [t for t in spec[1:3] if t is not None]
            for t in tabs:
                if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                    raise TypeError("nodal tables must be contiguous float64 CUDA tensors")
            f.nodal = C.cast(C.c_void_p(tabs[0].data_ptr()), _dp)
            if len(tabs) > 1:
                f.face = C.cast(C.c_void_p(tabs[1].data_ptr()), _dp)
            return f

        u, D = dev_field(_U, drift), dev_field(_D, diffusion)
        _check(lib().sl_set_fields_device(C.c_void_p(self.ctx), C.byref(u), C.byref(D)), "sl_set_fields_device")
        self.pb = dict(self.pb, drift=drift, diffusion=diffusion)

    def reseed(self):
        """Every sample set to the current sample mean (Eq. re-seed)."""
        _check(lib().sl_reseed(C.c_void_p(self.ctx)), "sl_reseed")

    def step(self, dt=None, steps=None):
        sl_step(self.ctx, self.pb["dt"] if dt is None else dt, self.pb["steps"] if steps is None else steps)

    def moments(self, want_m2=True):
        mean, m2 = sl_moments(self.ctx, self.V, want_m2)
        return mean.reshape(self._shape), (m2.reshape(self._shape) if m2 is not None else None)

    def moments_device(self, mean_t, m2_t=None):
        sl_moments_device(self.ctx, mean_t.data_ptr(), m2_t.data_ptr() if m2_t is not None else None)

    def moments_partial(self, psum_t, psq_t):
        """Chunk partial sums into float64 CUDA tensors [ceil(M/64)][V]
        (sl_moments_partial), asynchronous on the solver's stream."""
        nc = -(-self.M // 64)
        for t in (psum_t, psq_t):
            if tuple(t.shape) != (nc, self.V) or not t.is_contiguous() or str(t.dtype) != "torch.float64" \
                    or not t.is_cuda:
                raise ValueError(f"need contiguous float64 CUDA tensors of shape ({nc}, {self.V})")
        sl_moments_partial(self.ctx, psum_t.data_ptr(), psq_t.data_ptr())

    def samples(self, s0=0, count=None):
        count = self.M - s0 if count is None else count
        return sl_get_samples(self.ctx, s0, count, self.V).reshape((count,) + self._shape)

    def set_samples(self, s0, states):
        sl_set_samples(self.ctx, s0, np.asarray(states).reshape(-1, self.V))

    def wiener(self, step0, nsteps, dt=None):
        return sl_wiener(self.ctx, step0, nsteps, self.pb["dt"] if dt is None else dt, self.M, self.dim)

    def profile(self, enable=True):
        sl_profile(self.ctx, enable)

    def profile_read(self):
        """(summed step-kernel milliseconds, launches) since the last read."""
        return sl_profile_read(self.ctx)

    @property
    def dt_max(self):
        return sl_dt_max(self.ctx)

    @property
    def dt_edge(self):
        return sl_dt_edge(self.ctx)

    @property
    def step_count(self):
        return sl_step_count(self.ctx)

    @step_count.setter
    def step_count(self, n):
        sl_set_step_count(self.ctx, n)

    @property
    def fallbacks(self):
        """(phase 1, phase 2) groups the 2D fast path left to the direct solve."""
        return sl_fallback_count(self.ctx)

    def close(self):
        if self.ctx:
            sl_free(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
