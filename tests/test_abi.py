"""CPU checks of the C ABI: the library builds, loads and exports every entry
point include/sse.h declares; argument validation that runs before any CUDA
call rejects bad input with the documented codes."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

from paper_2105_13484_gb300 import binding, build, mesh as meshgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "sse.h")).read()
    return sorted(set(re.findall(r"\b(sse_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert "sse_step" in syms and "sse_mesh_create" in syms
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) <= set(binding.EXPORTS)


def test_strerror(lib):
    assert lib.sse_strerror(0) == b"ok"
    assert b"mesh" in lib.sse_strerror(-2)
    # every code the header defines has its own message
    codes = {}
    with open(os.path.join(ROOT, "include", "sse.h")) as f:
        for line in f:
            mm = re.match(r"#define (SSE_(?:OK|ERR_\w+)) \(?(-?\d+)\)?", line)
            if mm:
                codes[mm.group(1)] = int(mm.group(2))
    assert codes["SSE_ERR_INTERNAL"] == -10 and len(codes) == 11
    msgs = {lib.sse_strerror(c) for c in codes.values()}
    assert len(msgs) == len(codes) and b"unknown error" not in msgs


def test_null_arguments(lib):
    out = ct.c_void_p()
    assert lib.sse_mesh_create(None, ct.byref(out)) == -1
    assert lib.sse_step(None, 3, 60.0, 10, 1) == -1
    assert lib.sse_state_create(None, None, None, ct.byref(out)) == -1
    assert lib.sse_state_inject(None, 1, 1) == -1
    assert lib.sse_state_set_f32(None, 0, None) == -1
    assert lib.sse_state_get_f32(None, 0, None) == -1
    assert lib.sse_state_graphs(None, None) == -1
    assert lib.sse_state_transfer(None, 0, None, 0) == -1
    assert lib.sse_state_sync(None) == -1


def _desc(m, L):
    d = binding.Mesh.__new__(binding.Mesh)
    d.lib = binding.load()
    keep = []

    def ia(x):
        a = np.ascontiguousarray(x, dtype=np.int32)
        keep.append(a)
        return a.ctypes.data_as(ct.POINTER(ct.c_int32))

    def da(x):
        a = np.ascontiguousarray(x, dtype=np.float64)
        keep.append(a)
        return a.ctypes.data_as(ct.POINTER(ct.c_double))

    desc = binding.MeshDesc(m.nCells, m.nEdges, m.nVertices, m.maxEdges, m.maxEdges2, L,
                            ia(m.cellsOnEdge), ia(m.verticesOnEdge), ia(m.nEdgesOnCell),
                            ia(m.edgesOnCell), ia(m.cellsOnVertex), ia(m.edgesOnVertex),
                            ia(m.nEdgesOnEdge), ia(m.edgesOnEdge), da(m.weightsOnEdge),
                            da(m.dcEdge), da(m.dvEdge), da(m.areaCell), da(m.areaTriangle),
                            da(m.kiteAreasOnVertex), da(m.fEdge), da(m.fVertex),
                            da(m.bottomDepth), da(np.full(L, 1.0 / L)))
    return desc, keep


@pytest.mark.parametrize("corrupt,code", [
    (lambda m: m.cellsOnEdge.__setitem__((3, 1), m.nCells), -2),
    (lambda m: m.edgesOnEdge.__setitem__((5, 0), -1), -2),
    (lambda m: m.dcEdge.__setitem__(7, 0.0), -2),
    (lambda m: m.areaCell.__setitem__(2, -1.0), -2),
    (lambda m: m.edgesOnCell.__setitem__((4, 0), 0), -2),
    (lambda m: m.cellsOnVertex.__setitem__((1, 0), m.nCells + 5), -2),
])
def test_bad_mesh_rejected_before_any_device_work(lib, corrupt, code):
    m = meshgen.planar_hex(6, 8, 1e4)
    corrupt(m)
    desc, keep = _desc(m, 3)
    out = ct.c_void_p()
    assert lib.sse_mesh_create(ct.byref(desc), ct.byref(out)) == code
    assert not out.value


def test_limits(lib):
    m = meshgen.planar_hex(6, 8, 1e4)
    desc, keep = _desc(m, 3)
    desc.nLayers = 65
    out = ct.c_void_p()
    assert lib.sse_mesh_create(ct.byref(desc), ct.byref(out)) == -7
    desc.nLayers = 0
    assert lib.sse_mesh_create(ct.byref(desc), ct.byref(out)) == -1


@pytest.mark.parametrize("field", ["nCells", "nEdges", "nVertices"])
def test_empty_mesh_is_an_invalid_argument(lib, field):
    m = meshgen.planar_hex(6, 8, 1e4)
    desc, keep = _desc(m, 3)
    setattr(desc, field, 0)
    out = ct.c_void_p()
    assert lib.sse_mesh_create(ct.byref(desc), ct.byref(out)) == -1
    assert not out.value


def test_valid_mesh_without_device_memory_fails_cleanly(lib):
    """A valid mesh passes validation and builds its host plans; where no
    device memory can be had (this CPU-only machine) the call returns an
    error code, hands out nothing and frees what it built."""
    m = meshgen.planar_hex(6, 8, 1e4)
    desc, keep = _desc(m, 3)
    out = ct.c_void_p()
    rc = lib.sse_mesh_create(ct.byref(desc), ct.byref(out))
    if rc == 0:      # a machine with a GPU: the mesh exists
        lib.sse_mesh_destroy(out)
        return
    assert rc in (-3, -4) and not out.value
    for _ in range(3):   # repeated failures stay failures, nothing crashes
        assert lib.sse_mesh_create(ct.byref(desc), ct.byref(out)) == rc and not out.value


def test_rest_fractions_must_sum_to_one(lib):
    m = meshgen.planar_hex(6, 8, 1e4)
    desc, keep = _desc(m, 3)
    rf = np.array([0.3, 0.3, 0.3])
    keep.append(rf)
    desc.restThicknessFrac = rf.ctypes.data_as(ct.POINTER(ct.c_double))
    out = ct.c_void_p()
    assert lib.sse_mesh_create(ct.byref(desc), ct.byref(out)) == -2


def test_partial_bottom_arrays_are_validated(lib):
    """maxLevelCell and restThickness come together, K in 1..L, thickness > 0
    above the column's bottom and 0 below it, summing to bottomDepth."""
    from paper_2105_13484_gb300 import inputs
    m = meshgen.planar_hex(6, 8, 1e4, depth=lambda x, y: 300.0 + 600.0 * y / y.max())
    L = 4
    K, rest = inputs.partial_bottom(m, L)
    out = ct.c_void_p()

    def try_with(Kx, rx):
        desc, keep = _desc(m, L)
        if Kx is not None:
            Kx = np.ascontiguousarray(Kx, dtype=np.int32)
            keep.append(Kx)
            desc.maxLevelCell = Kx.ctypes.data_as(ct.POINTER(ct.c_int32))
        if rx is not None:
            rx = np.ascontiguousarray(rx, dtype=np.float64)
            keep.append(rx)
            desc.restThickness = rx.ctypes.data_as(ct.POINTER(ct.c_double))
        return lib.sse_mesh_create(ct.byref(desc), ct.byref(out))

    assert try_with(K, None) == -1
    assert try_with(None, rest) == -1
    bad = K.copy(); bad[3] = L + 1
    assert try_with(bad, rest) == -2
    bad = K.copy(); bad[3] = 0
    assert try_with(bad, rest) == -2
    r2 = rest.copy(); r2[5, K[5] - 1] *= 1.01            # no longer sums to the depth
    assert try_with(K, r2) == -2
    r2 = rest.copy(); r2[5, K[5] - 1] = 0.0; r2[5, 0] += rest[5, K[5] - 1]   # empty active layer
    assert try_with(K, r2) == -2
    if K.min() < L:
        i = int(np.argmin(K))
        r2 = rest.copy(); r2[i, L - 1] = 1.0; r2[i, 0] -= 1.0     # water below the bottom
        assert try_with(K, r2) == -2


@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++17")])
def test_header_compiles_on_its_own(tmp_path, lang, std):
    """include/sse.h is self-contained for C and C++ callers."""
    import shutil
    import subprocess
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    src = tmp_path / ("t.c" if lang == "c" else "t.cpp")
    src.write_text('#include "sse.h"\nint main(void) { return 0; }\n')
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-fsyntax-only",
                        "-I", os.path.join(root, "include"), str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
