"""Pins of the oracle's operation-counting build (oracle/flop_count.cpp).

The counting build compiles the oracle's own source with every double an
8-byte wrapper that counts its arithmetic.  It must (a) compute exactly what
the plain build computes, and (b) count each operation once: the TRiSK
operators below have closed-form operation counts that follow from their
definitions (Sec. 5 cites TRiSK; the operators are written out in the
oracle), so a missed or double-counted operator shows up as a wrong count.
The committed summary the benchmark reads must come from the current
sources and reproduce.
"""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2105_13484_gb300 import inputs
from paper_2105_13484_gb300 import mesh as meshgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUMMARY = os.path.join(ROOT, "profiles", "fp64_flops_oracle.md")


@pytest.fixture(scope="module")
def channel():
    """A walled channel (boundary edges, cells with all six edges) on a beta plane."""
    m = meshgen.planar_hex(9, 8, 7e3, f0=1e-4, beta=2e-11)
    return m, oracle.Oracle(m, 3, counting=True)


def test_counting_build_steps_bit_identically(channel_small):
    m, L, p, (u, h, tr), run = channel_small
    a = oracle.Oracle(m, L, p).step(3, run["dt"], run["M"], u, h, tr, n_steps=2)
    c = oracle.Oracle(m, L, p, counting=True)
    b = c.step(3, run["dt"], run["M"], u, h, tr, n_steps=2)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert c.flops() > 0


def test_counts_of_the_trisk_operators(channel):
    m, o = channel
    L = 3
    rng = np.random.default_rng(5)
    F = rng.standard_normal((m.nEdges, L))
    phi = rng.standard_normal((m.nCells, L))
    ne = np.asarray(m.nEdgesOnCell)
    nee = np.asarray(m.nEdgesOnEdge)
    nev = (np.asarray(m.edgesOnVertex) >= 0).sum(1)
    o.flops(reset=True)
    o.div(F)      # per cell and layer: sign * l_e * F_e and a sum per edge, one division
    assert o.flops(reset=True) == L * int((3 * ne + 1).sum())
    o.grad(phi)   # per edge and layer: a difference and a division
    assert o.flops(reset=True) == 2 * L * m.nEdges
    o.curl(F)     # per vertex and layer: sign * d_e * u_e and a sum per edge, one division
    assert o.flops(reset=True) == L * int((3 * nev + 1).sum())
    o.tangential(F)   # per edge and layer: w * l * u and a sum per neighbour, one division
    assert o.flops(reset=True) == L * int((3 * nee + 1).sum())
    # the counter follows the calls, not the data
    o.grad(2.0 * phi)
    assert o.flops(reset=True) == 2 * L * m.nEdges


def test_flops_needs_the_counting_build(channel_small):
    m, L, p, _, _ = channel_small
    with pytest.raises(RuntimeError):
        oracle.Oracle(m, L, p).flops()


def _summary():
    with open(SUMMARY) as f:
        text = f.read()
    rows = {}
    for line in text.splitlines():
        cells = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cells) == 9 and cells[0] in ("sphere_l7", "channel_1km"):
            rows[cells[0]] = (int(cells[7]), float(cells[8]))
    hashes = dict(re.findall(r"^- oracle sha256 (\S+): ([0-9a-f]{16})$", text, re.M))
    return rows, hashes


def test_the_committed_count_is_current_and_reproduces():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "count_flops", os.path.join(ROOT, "oracle", "count_flops.py"))
    cf = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(cf)
    rows, hashes = _summary()
    assert set(rows) == {"sphere_l7", "channel_1km"}
    assert hashes == cf.source_hashes()
    r = cf.count_step("channel_1km")
    assert rows["channel_1km"][0] == r["flops_per_step"]
    assert rows["channel_1km"][1] == pytest.approx(r["flops_per_cell_layer_step"], abs=0.051)
    # the parts: each row reproduces, and three calls of each part plus the
    # rest make up the whole step
    with open(SUMMARY) as f:
        parts = dict(re.findall(r"^\| channel_1km: (.+?) \| \d+ \| (\d+) \|", f.read(), re.M))
    assert {k: int(v) for k, v in parts.items()} == dict(
        r["parts"], **{"split, layer fluxes, reconciliation, combinations": r["rest"]})
    assert r["rest"] > 0 and 3 * sum(r["parts"].values()) + r["rest"] == r["flops_per_step"]
