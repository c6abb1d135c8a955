"""The link between the committed ncu summaries and the kernel sources (CPU).

bench.py reports a kernel's DRAM traffic from a committed capture only while
the kernels' code hashes to the values recorded with it; the hash is taken
over the code without comments, so that editing a comment keeps the capture.
"""
import os
import re

import pytest

import bench


def test_code_of_drops_comments_and_keeps_literals():
    src = ('int a = 1;  // trailing\n/* block\n   comment */ const char *s = "x // y /* z */";\n'
           "char q = '/';\tint b = a /2;\n")
    assert bench.code_of(src) == ('int a = 1; const char *s = "x // y /* z */"; '
                                  "char q = '/'; int b = a /2;")


def test_comment_edits_keep_the_hash_and_code_edits_change_it():
    a = "__global__ void k(float *x) {\n    x[0] = 1.f;   // one\n}\n"
    b = "// the kernel\n__global__ void k(float *x) {\n    /* set */ x[0] = 1.f;\n}\n"
    c = "__global__ void k(float *x) {\n    x[0] = 2.f;\n}\n"
    assert bench.code_of(a) == bench.code_of(b) != bench.code_of(c)


def test_every_ncu_summary_names_each_kernel_source_once():
    names = {os.path.basename(p) for p in bench.KERNEL_SOURCES}
    root = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles")
    for f in sorted(os.listdir(root)):
        with open(os.path.join(root, f)) as fh:
            text = fh.read()
        if "- oracle sha256 " in text:
            continue   # a count taken in the oracle, keyed to the oracle's sources
        hashes = {}
        for line in text.splitlines():
            bench.capture_hashes(line, hashes)
        assert set(hashes) == names, f
        assert all(re.fullmatch(r"[0-9a-f]{16}", v) for v in hashes.values()), f


def test_a_code_edit_voids_only_the_captures_of_the_kernels_built_from_that_source(monkeypatch):
    names = {os.path.basename(p) for p in bench.KERNEL_SOURCES}
    for workload, classes in bench.PROFILE_OF.items():
        for cls in classes:
            assert set(bench.SOURCES_OF[cls]) <= names
    real = bench.source_hashes()
    # pretend the recorded hashes are the current ones, then change one source
    recorded = {}
    for cls, name in bench.PROFILE_OF["sphere_l7"].items():
        with open(os.path.join(bench.ROOT, "profiles", name)) as fh:
            h = {}
            for line in fh:
                bench.capture_hashes(line, h)
        recorded[cls] = h
    for edited in names:
        for cls, h in recorded.items():
            now = dict(h)
            now[edited] = "0" * 16
            monkeypatch.setattr(bench, "source_hashes", lambda now=now: now)
            traffic, why = bench.ncu_traffic(cls, True, "sphere_l7")
            if edited in bench.SOURCES_OF[cls]:
                assert traffic is None and "changed" in why
            else:
                assert traffic is not None and traffic > 0, (cls, edited)
    monkeypatch.setattr(bench, "source_hashes", lambda: real)


def test_the_step_launch_list_is_valid_only_while_every_kernel_source_is_unchanged(monkeypatch):
    with open(os.path.join(bench.ROOT, "profiles", "launches_sphere_l7_mixed.md")) as fh:
        h = {}
        for line in fh:
            bench.capture_hashes(line, h)
    monkeypatch.setattr(bench, "source_hashes", lambda: dict(h))
    traffic, src = bench.step_traffic("sphere_l7", True)
    assert traffic > 0 and src.endswith("launches_sphere_l7_mixed.md")
    for edited in h:
        now = dict(h)
        now[edited] = "0" * 16
        monkeypatch.setattr(bench, "source_hashes", lambda now=now: now)
        assert bench.step_traffic("sphere_l7", True)[0] is None


def test_the_subcycle_traffic_follows_the_subcycle_sources(monkeypatch):
    class Mesh:
        nEdges, nCells = 343016, 163842
    with open(os.path.join(bench.ROOT, "profiles", "btr_tiled_sphere_l7.md")) as fh:
        h = {}
        for line in fh:
            bench.capture_hashes(line, h)
    run = {"order": 3, "M": 40}
    for edited in h:
        now = dict(h)
        now[edited] = "0" * 16
        monkeypatch.setattr(bench, "source_hashes", lambda now=now: now)
        out = bench.subcycle_of({"btr": (3 * 1.7, 3)}, Mesh(), run, 1, 152, "sphere_l7", True)
        assert out["grid_barriers_per_step"] == 120
        if edited in bench.SOURCES_OF["btr"]:
            assert out["l2_bytes_per_launch"] is None
        else:
            assert out["l2_bytes_per_launch"] > 0 and out["dram_bytes_per_launch"] > 0


def test_fp64_alu_roofline_uses_the_oracle_count():
    class Mesh:
        nCells = 114689
    out = bench.fp64_alu_of(Mesh(), 60, 47.0, 1.06, "sphere_l7")
    per_cl = bench.oracle_flops("sphere_l7")
    assert per_cl > 0 and out["flops_per_cell_layer_step"] == per_cl
    assert out["achieved"] == pytest.approx(per_cl * 114689 * 60 / 0.047 / 1e12)
    assert out["frac"] == pytest.approx(out["achieved"] / 1.06)
    assert bench.oracle_flops("channel_1km") > 0
    # a variant of the workload (another level, partial bottom) has no count of its own
    assert "frac" not in bench.fp64_alu_of(Mesh(), 60, 47.0, 1.06, "sphere_l7 (variant)")


def test_step_bytes_agree_with_the_fused_stage_launches():
    """The step's algorithmic bytes per cell-layer (each 3-D array read or
    written once per stage) against the sum of the six fused stage launches
    of one SSPRK3-SE step, on a mesh with E = 3 C exactly and the 2-D terms
    set aside: equal in the FP64 form; in the mixed form the launches also
    move the FP32 copy of h, which the step's figure does not count."""
    assert bench.step_bytes_per_cell_layer(True, 2) == 308.0
    assert bench.step_bytes_per_cell_layer(False, 2) == 528.0
    C, L = 1000, 60
    E = 3 * C
    for nT in (1, 2):
        for mixed in (False, True):
            sR = 4 if mixed else 8
            total = 0
            for stage in range(3):
                old = stage > 0
                total += bench.fused_stage_bytes("bcl_edge", C, E, L, nT, sR, old, mixed) - (
                    3 * E * sR + 8 * C)
                total += bench.fused_stage_bytes("thickness", C, E, L, nT, sR, old, mixed) - (
                    E * (2 * sR + 8) + 8 * C)
            step = bench.step_bytes_per_cell_layer(mixed, nT) * C * L
            if not mixed:
                assert total == step
            else:
                # bcl reads the 4-byte copy instead of the 8-byte h (3 stages:
                # -4 B each); thickness stages read and write h with its copy
                # (stage 1: 2 h words, stages 2-3: 3 h words, +4 B each)
                assert total == step + 4 * C * L * (-3 + 2 + 3 + 3)
