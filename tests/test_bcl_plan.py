"""Host logic of the fused baroclinic kernel: its patch plan (csrc/tiles.cu,
build_bcl_plan) is checked on the CPU by a C++ harness
(tests/bcl_plan_check.cpp) on meshes numbered the way the library numbers
them: ownership of every edge, every local index the kernel dereferences in
range (or the zero slot), every neighbour and coefficient the one the global
mesh names, and the plan's maxima above every patch."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2105_13484_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    out = str(tmp_path_factory.mktemp("bclplan") / "bcl_plan_check")
    # tiles.cu is plain host C++ (no device code): compile it as C++
    subprocess.run([gxx, "-O2", "-std=c++17", "-o", out, os.path.join(HERE, "bcl_plan_check.cpp"),
                    "-x", "c++", os.path.join(ROOT, "paper_2105_13484_gb300", "csrc", "tiles.cu")],
                   check=True, capture_output=True)
    return out


def dump(m, d):
    os.makedirs(d, exist_ok=True)
    with open(os.path.join(d, "hdr.txt"), "w") as f:
        f.write(f"{m.nCells} {m.nEdges} {m.maxEdges} {m.maxEdges2} {m.nVertices}")
    for name, x in (("coe", m.cellsOnEdge), ("voe", m.verticesOnEdge), ("neoc", m.nEdgesOnCell),
                    ("eoc", m.edgesOnCell), ("neoe", m.nEdgesOnEdge), ("eoe", m.edgesOnEdge),
                    ("eov", m.edgesOnVertex), ("cov", m.cellsOnVertex)):
        np.ascontiguousarray(x, dtype=np.int32).tofile(os.path.join(d, name + ".bin"))


@pytest.mark.parametrize("name,pc", [("channel_10km", 128), ("channel_10km", 32), ("sphere_l4", 128),
                                     ("sphere_l4", 48), ("channel_1km", 128), ("sphere_l7", 128)])
def test_bcl_plan_invariants(checker, tmp_path, name, pc):
    m = inputs.workload(name)[0]
    d = str(tmp_path / name)
    dump(m, d)
    r = subprocess.run([checker, d, str(pc)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
