"""CPU checks of the C ABI: the library builds for sm_103a, loads without a GPU,
exports every entry point that include/sl.h declares, and rejects invalid
arguments before touching the device."""

import ctypes as C
import os
import re

import pytest

import sl_inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def sl():
    from paper_2009_07340_gb300 import build

    build.build()
    import paper_2009_07340_gb300 as sl

    return sl


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(sl_\w+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(sl):
    names = _declared()
    assert {"sl_init", "sl_step", "sl_moments", "sl_moments_device", "sl_free"} <= names
    L = C.CDLL(os.path.join(ROOT, "paper_2009_07340_gb300", "libsl.so"))
    for n in sorted(names):
        assert hasattr(L, n), n


def test_strerror(sl):
    assert sl.sl_strerror(0) == "ok"
    assert "argument" in sl.sl_strerror(-1)
    assert sl.sl_strerror(-999) == "unknown error"


@pytest.mark.parametrize("bad", [
    dict(N=1), dict(N=17), dict(M=0), dict(K=(0,)), dict(hi=(0.0,)),
    dict(diffusion=("cos", [0.01, 1.5, 1.0])), dict(diffusion=("const", [-1.0])),
    dict(drift=("rotation", [1.0, 0.5, 0.5])), dict(phi0=("sinsin", [1.0, 1.0, 1.0])),
])
def test_invalid_arguments_rejected_before_device(sl, bad):
    pb = I.config1()
    pb.update(bad)
    with pytest.raises(sl.SLError) as e:
        sl.sl_init(pb)
    assert e.value.code == -1


def test_invalid_precision_and_null(sl):
    with pytest.raises(sl.SLError) as e:
        sl.sl_init(I.config1(), precision=7)
    assert e.value.code == -1
    L = sl.lib()
    assert L.sl_step(None, 1e-3, 1) == -1
    assert L.sl_moments(None, None, None) == -1
    L.sl_free(None)  # no-op
    assert L.sl_moments_partial(None, None, None) == -1
    assert L.sl_moments_combine(None, None, 1, 4, 4, None, None, None) == -1
    assert L.sl_moment_chunk() == 64
    assert L.sl_fallback_count(None, None, None) == -1


@pytest.mark.parametrize("bad,precision,code", [
    (dict(K=(2049,)), "fp64", -8),                          # 1D beyond the largest cluster (8 x 256 elements)
    (dict(dim=2, K=(2, 2), lo=(0.0, 0.0), hi=(1.0, 1.0), N=12, drift=("const", [0.1, 0.2]),
          diffusion=("const", [0.01]), phi0=("gauss", [1.0, 0.2, 0.5, 0.5])), "fp64", -8),   # 2D FP64 N > 11
    (dict(dim=2, K=(2, 2), lo=(0.0, 0.0), hi=(1.0, 1.0), N=13, drift=("const", [0.1, 0.2]),
          diffusion=("const", [0.01]), phi0=("gauss", [1.0, 0.2, 0.5, 0.5])), "fp32", -8),   # 2D FP32 N > 12
    (dict(dim=2, K=(2, 2), lo=(0.0, 0.0), hi=(1.0, 1.0), N=9, components=2, drift=("const", [0.1, 0.2]),
          diffusion=("const", [0.01]), phi0=("gauss", [1.0, 0.2, 0.5, 0.5])), "fp32", -8),   # 2D two fields N > 8
    (dict(dim=2, K=(2, 2), lo=(0.0, 0.0), hi=(1.0, 1.0), N=4, components=2, periodic=False,
          drift=("const", [0.1, 0.2]), diffusion=("const", [0.01]), phi0=("gauss", [1.0, 0.2, 0.5, 0.5])),
     "fp64", -8),                                                                          # two fields: periodic only
    (dict(components=2), "mixed", -8),                                                     # 1D two fields: not mixed
])
def test_unsupported_sizes_rejected_before_device(sl, bad, precision, code):
    pb = I.config1()
    pb.update(bad)
    with pytest.raises(sl.SLError) as e:
        sl.sl_init(pb, precision)
    assert e.value.code == code


def test_sample_range_and_batch_server_arguments(sl):
    with pytest.raises(sl.SLError) as e:  # sample0 + M beyond the 2^32 Philox sample counter
        sl.sl_init(I.config1(), sample0=(1 << 32) - 10)
    assert e.value.code == -1
    L = sl.lib()
    h = C.c_void_p()
    assert L.sl_batch_create(C.byref(h), 0, None, None) == -1
    cfg = sl.sl_server_config()
    cfg.budget_bytes, cfg.slice_steps, cfg.precision, cfg.device = 1 << 20, 0, 0, -1
    assert L.sl_server_create(C.byref(h), C.byref(cfg)) == -1  # slice_steps < 1
    cfg.slice_steps, cfg.max_active = 1, -1
    assert L.sl_server_create(C.byref(h), C.byref(cfg)) == -1  # negative cap
    cfg.max_active, cfg.budget_bytes = 0, 0
    assert L.sl_server_create(C.byref(h), C.byref(cfg)) == -1  # no budget


def _nodal_init_rc(sl, pb, drift, diffusion):
    """sl_init's return code for the given sl_field structs (a context that
    was created, on a machine with a GPU, is freed)."""
    mesh = sl._mesh(pb)
    phi = sl._field(sl._PHI, pb["phi0"])
    opt = sl.sl_options()
    opt.device = -1
    h = C.c_void_p()
    rc = sl.lib().sl_init(C.byref(h), C.byref(mesh), pb["N"], pb["M"], C.byref(drift), C.byref(diffusion),
                          C.byref(phi), C.byref(opt))
    if rc == 0:
        sl.lib().sl_free(h)
    return rc


def test_nodal_fields_are_checked_before_device(sl):
    """Nodal drift / diffusion: a missing node table, a negative or NaN D at a
    node, or a negative D in a read interface entry is SL_ERR_ARG; on a
    periodic line the last interface entry is not read, so a NaN there passes
    the checks (and the call goes on to the device)."""
    import numpy as np

    pb = I.with_(I.config1(), K=(3,), N=4)
    u = sl._field(sl._U, pb["drift"])
    D = sl._field(sl._D, pb["diffusion"])
    none = sl.sl_field()
    none.kind = sl._U["nodal"]
    assert _nodal_init_rc(sl, pb, none, D) == -1
    none.kind = sl._D["nodal"]
    assert _nodal_init_rc(sl, pb, u, none) == -1
    good = np.full((3, 4), 0.01)
    for bad in (-1e-3, np.nan):
        nodes = good.copy()
        nodes[1, 2] = bad
        assert _nodal_init_rc(sl, pb, u, sl._field(sl._D, ("nodal", nodes))) == -1
    face = np.full(4, 0.01)
    face[1] = -0.01
    assert _nodal_init_rc(sl, pb, u, sl._field(sl._D, ("nodal", good, face))) == -1
    face[1], face[3] = 0.01, np.nan  # the periodic line's last interface: not read
    assert _nodal_init_rc(sl, pb, u, sl._field(sl._D, ("nodal", good, face))) != -1
    dirichlet = I.with_(pb, periodic=False)  # ... but read at a Dirichlet boundary
    assert _nodal_init_rc(sl, dirichlet, u, sl._field(sl._D, ("nodal", good, face))) == -1


def test_header_is_self_contained_c_and_matches_the_binding(sl, tmp_path):
    """include/sl.h compiles as plain C99 on its own, and every struct of the
    C ABI has the same size and field offsets in C as in the ctypes binding."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [sl.sl_field, sl.sl_mesh, sl.sl_options, sl.sl_instance, sl.sl_server_config, sl.sl_server_stats]
    lines = ['#include "sl.h"', "#include <stdio.h>", "#include <stddef.h>", "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c99", "-Wall", "-pedantic", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe)])
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()
    got = {tuple(l.split()[:-1]): int(l.split()[-1]) for l in out}
    for st in structs:
        name = st.__name__
        assert got[(name, "size")] == C.sizeof(st), name
        for field, _ in st._fields_:
            assert got[(name, field)] == getattr(st, field).offset, (name, field)
