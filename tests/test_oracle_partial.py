"""Partial bottom cells (maxLevelCell) in the oracle: each column keeps the
layers that reach its depth, the last one cut to the bottom.

* With every column full and rest thickness = fraction x depth, the result
  is the one without partial-bottom data.
* Volume and tracer content are conserved; inactive layers stay empty.
* z-star: every active layer of a column keeps the same ratio h_k / rest_k.
* Lake at rest over partial-bottom bathymetry with uniform density stays at
  rest (the layer pressure gradient reduces to g grad zeta in every column).
* A constant tracer stays constant.
"""
import numpy as np
import pytest

import oracle
from paper_2105_13484_gb300 import inputs


def _depth(x, y):
    return 200.0 + 700.0 * (y / y.max()) ** 1.5 + 80.0 * np.sin(x / 2e4)


def _case(**kw):
    return inputs.partial_case(12, 14, 10e3, 8, depth=_depth, **kw)


def test_full_columns_reduce_to_the_plain_oracle():
    m, L, p, (u, h, tr) = inputs.channel_case(8, 10, 10e3, 5, perturb=True,
                                              depth=lambda x, y: 900.0 + 50 * np.sin(x / 2e4))
    frac = np.full(L, 1.0 / L)
    rest = m.bottomDepth[:, None] * frac[None, :]
    a = oracle.Oracle(m, L, p).step(3, 200.0, 8, u, h, tr, n_steps=3)
    b = oracle.Oracle(m, L, p, max_level=np.full(m.nCells, L, np.int32),
                      rest_thickness=rest).step(3, 200.0, 8, u, h, tr, n_steps=3)
    for x, y in zip(a, b):
        assert np.abs(x - y).max() <= 1e-13 * (1 + np.abs(x).max())


@pytest.mark.parametrize("order", [2, 3])
def test_conservation_zstar_and_empty_layers(order):
    m, L, p, (u, h, tr), (K, rest) = _case(nTracers=2, kappa_h=10.0, kappa_v=1e-4)
    assert K.min() < K.max() and (rest[np.arange(m.nCells), K - 1] < rest.max()).any()
    o = oracle.Oracle(m, L, p, max_level=K, rest_thickness=rest)
    A = m.areaCell
    v0, c0 = A @ h.sum(1), [A @ (h * t).sum(1) for t in tr]
    u1, h1, t1 = o.step(order, 200.0, 10, u, h, tr, n_steps=6)
    assert abs(A @ h1.sum(1) - v0) / v0 < 1e-13
    for t, c in zip(t1, c0):
        assert abs(A @ (h1 * t).sum(1) - c) / c < 1e-13
    act = np.arange(L)[None, :] < K[:, None]
    assert np.abs(h1[~act]).max() == 0.0 and np.abs(t1[:, ~act]).max() == 0.0
    Ke = np.minimum(K[m.cellsOnEdge[:, 0]], K[m.cellsOnEdge[:, 1]])
    assert np.abs(u1[np.arange(L)[None, :] >= Ke[:, None]]).max() == 0.0
    ratio = np.where(act, h1 / np.where(rest > 0, rest, 1.0), np.nan)
    assert np.nanmax(np.nanmax(ratio, 1) - np.nanmin(ratio, 1)) < 1e-14
    assert np.abs(u1 - u).max() > 1e-3


@pytest.mark.parametrize("order", [2, 3])
def test_lake_at_rest_over_partial_bottom_cells(order):
    m, L, p, (u, h, tr), (K, rest) = _case(perturb=False)
    act = np.arange(L)[None, :] < K[:, None]
    tr = np.where(act[None], 12.0, 0.0)
    h = rest.copy()
    o = oracle.Oracle(m, L, p, max_level=K, rest_thickness=rest)
    u1, h1, t1 = o.step(order, 300.0, 10, np.zeros_like(u), h, tr, n_steps=3)
    assert np.abs(u1).max() < 1e-12
    assert np.abs(h1 - h).max() < 1e-10


def test_constant_tracer_over_partial_bottom_cells():
    m, L, p, (u, h, tr), (K, rest) = _case(nTracers=2, kappa_h=10.0, kappa_v=1e-4)
    act = np.arange(L)[None, :] < K[:, None]
    tr = tr.copy()
    tr[1] = np.where(act, 34.5, 0.0)
    o = oracle.Oracle(m, L, p, max_level=K, rest_thickness=rest)
    u1, h1, t1 = o.step(3, 200.0, 10, u, h, tr, n_steps=4)
    assert np.abs(t1[1][act] - 34.5).max() < 1e-12
