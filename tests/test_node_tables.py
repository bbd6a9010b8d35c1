"""CPU check of the compile-time node tables of the FP32 1D kernels
(NodeTab1D<N> in sl_step1d.cuh, folded into the instructions): every entry,
4 (xi_i - xi_m), -4 xi_m and 4 (1 - xi_m) with xi_i = (1 - cos((i + 1/2)
pi / N)) / 2, must equal the float of the same expression evaluated with
libm's cos.  The tables are printed by a host program built with nvcc."""

import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROG = r"""
#include <cstdio>
#include "sl_step1d.cuh"
template <int N> void dump() {
    constexpr sl::NodeTab1D<N> t{};
    for (int i = 0; i < N; ++i)
        for (int m = 0; m < N; ++m) printf("%d z %d %d %.9e\n", N, i, m, (double)t.z[i][m]);
    for (int m = 0; m < N; ++m) printf("%d f %d %.9e %.9e\n", N, m, (double)t.f0[m], (double)t.f1[m]);
}
template <int... Ns> void dump_all() { (dump<Ns>(), ...); }
int main() { dump_all<2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16>(); }
"""


def test_compile_time_node_tables_equal_libm_values(tmp_path):
    nvcc = shutil.which(os.environ.get("NVCC", "nvcc"))
    if nvcc is None:
        pytest.skip("nvcc not found")
    src = tmp_path / "tables.cu"
    src.write_text(PROG)
    exe = tmp_path / "tables"
    subprocess.check_call([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                           "-I", os.path.join(ROOT, "paper_2009_07340_gb300", "csrc"),
                           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in filter(None, out):
        f = line.split()
        N = int(f[0])
        xi = 0.5 * (1.0 - np.cos(np.pi * ((np.arange(N) + 0.5) / N)))
        if f[1] == "z":
            i, m, v = int(f[2]), int(f[3]), float(f[4])
            assert np.float32(v) == np.float32(4.0 * (xi[i] - xi[m])), (N, i, m)
        else:
            m, v0, v1 = int(f[2]), float(f[3]), float(f[4])
            assert np.float32(v0) == np.float32(-4.0 * xi[m]) and np.float32(v1) == np.float32(4.0 * (1.0 - xi[m]))
        seen += 1
    assert seen == sum(N * N + N for N in range(2, 17))
