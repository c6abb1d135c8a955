"""Host logic of the tiled sub-cycle: the tile plan (csrc/tiles.cu) is
checked on the CPU by a small C++ harness (tests/tile_plan_check.cpp) for
ownership, local order and the closure that makes the scheme exact (each
sub-stage reads only entries exact after the one before; the interior edges
computed while the halo exchange is in flight read only owned values)."""
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
    out = str(tmp_path_factory.mktemp("tileplan") / "tile_plan_check")
    # tiles.cu is plain host C++ (no device code): compile it as C++
    subprocess.run([gxx, "-O2", "-std=c++17", "-o", out, os.path.join(HERE, "tile_plan_check.cpp"),
                    "-x", "c++", os.path.join(ROOT, "paper_2105_13484_gb300", "csrc", "tiles.cu")],
                   check=True, capture_output=True)
    return out


def dump(m, d):
    os.makedirs(d, exist_ok=True)
    with open(os.path.join(d, "hdr.txt"), "w") as f:
        f.write(f"{m.nCells} {m.nEdges} {m.maxEdges} {m.maxEdges2}")
    m.cellsOnEdge.astype(np.int32).tofile(os.path.join(d, "coe.bin"))
    m.nEdgesOnCell.astype(np.int32).tofile(os.path.join(d, "neoc.bin"))
    m.edgesOnCell.astype(np.int32).tofile(os.path.join(d, "eoc.bin"))
    m.nEdgesOnEdge.astype(np.int32).tofile(os.path.join(d, "neoe.bin"))
    m.edgesOnEdge.astype(np.int32).tofile(os.path.join(d, "eoe.bin"))


@pytest.mark.parametrize("name,patches", [("channel_10km", 1), ("channel_10km", 8),
                                          ("sphere_l4", 7), ("sphere_l4", 40),
                                          ("channel_1km", 152)])
def test_tile_plan_invariants(checker, tmp_path, name, patches):
    m = inputs.workload(name)[0]
    d = str(tmp_path / name)
    dump(m, d)
    r = subprocess.run([checker, d, str(patches)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
