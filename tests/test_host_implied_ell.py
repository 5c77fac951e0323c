"""The implied-column layout of K's FP32 copy, checked on the host (no GPU).

The mixed-precision solves stream K's FP32 copy. When every 32-row slice's rows share a short
increasing table of relative columns (col - row), the library stores no columns at all
(build_implied_ell); absent neighbours hold 0 and the slices at the two ends of the numbering
clamp their columns. tests/host/implied_ell_check.cpp assembles K from a machine's meshes with
the library's own host assembly, builds both the stored-column layout and the implied one, and
runs the row loop of both GPU forms on the host (fmaf chains in storage order, 6 and 4 entries
a chunk). It must find every index in bounds and every row sum bitwise equal, which is what
lets the GPU forms be compared bit for bit (tests/test_gpu_matrix_columns.py). A scrambled node
numbering must be refused (its slices' tables would be long).
"""

import os
import shutil
import subprocess
from dataclasses import replace

import numpy as np
import pytest

from synth import machine_config, tiny_machine

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1707_03581_gb300", "csrc")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        p = os.path.join(d, "include")
        if d and os.path.exists(os.path.join(p, "cuda_runtime.h")):
            return p
    nvcc = shutil.which("nvcc")
    if nvcc:
        p = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
        if os.path.exists(os.path.join(p, "cuda_runtime.h")):
            return p
    return None


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    inc = _cuda_include()
    if not gxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("implied") / "implied_ell_check")
    cmd = [gxx, "-std=c++17", "-O2", "-fopenmp", "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", inc,
           os.path.join(ROOT, "tests", "host", "implied_ell_check.cpp"), os.path.join(CSRC, "host_fem.cpp"),
           "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return exe


def _write(mach, path):
    with open(path, "wb") as f:
        for b in (mach.stand, mach.stock):
            xyz = np.ascontiguousarray(b.mesh.xyz, dtype=np.float64)
            hx = np.ascontiguousarray(b.mesh.hex8, dtype=np.int64)
            kh = np.ascontiguousarray(b.k_per_hex if b.k_per_hex is not None else np.zeros(0), dtype=np.float64)
            f.write(np.array([xyz.shape[0], hx.shape[0], kh.size], dtype=np.int64).tobytes())
            f.write(np.array([b.k, b.rho, b.c], dtype=np.float64).tobytes())
            f.write(xyz.tobytes())
            f.write(hx.tobytes())
            f.write(kh.tobytes())


def _run(checker, mach, tmp_path):
    path = str(tmp_path / "mesh.bin")
    _write(mach, path)
    r = subprocess.run([checker, path], capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout


@pytest.mark.parametrize("case", ["tiny", "config0", "config1", "batch_r16"])
def test_implied_rows_bitwise_equal_stored_rows(checker, tmp_path, case):
    mach = {"tiny": lambda: tiny_machine(z0=0.37, amp=0.2, period=2.5),
            "config0": lambda: machine_config(0),
            "config1": lambda: machine_config(1),
            "batch_r16": lambda: machine_config(3)[6]}[case]()
    rc, out = _run(checker, mach, tmp_path)
    assert rc == 0, out
    assert out.startswith("implied 1"), out
    assert "bad 0 mismatches 0" in out, out


def test_scrambled_numbering_is_refused(checker, tmp_path):
    mach = machine_config(0)
    st = mach.stand
    nf = st.mesh.n_nodes
    perm = np.random.default_rng(5).permutation(nf)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(nf)
    mesh = replace(st.mesh, xyz=st.mesh.xyz[perm], hex8=inv[st.mesh.hex8])
    scr = replace(mach, stand=replace(st, mesh=mesh))
    rc, out = _run(checker, scr, tmp_path)
    assert rc == 0 and out.startswith("implied 0"), out
