"""Pins of the full SSPRK2-SE / SSPRK3-SE steps of the oracle.

* exact volume and tracer conservation (flux form, Sec. 3.4);
* SSH reconciliation identities (Sec. 3.4): with the consistent reading the
  thickness-derived SSH equals the corrector sub-cycle's SSH; with the
  printed F^h it differs by exactly -(dt/2) div D_1 (SSPRK2-SE) or
  -(dt/6) div(D_1 + D_2) (SSPRK3-SE);
* lake at rest, with and without bathymetry;
* a constant tracer stays constant under an arbitrary flow;
* temporal self-convergence of both schemes at second order (Theorem 1 and
  the remark after it: SSPRK3-SE is only second order).
"""
import numpy as np
import pytest

import oracle
from paper_2105_13484_gb300 import inputs


def _content(m, h, tr):
    A = m.areaCell
    return A @ h.sum(1), A @ (h * tr[0]).sum(1)


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("recon", ["off", "paper", "consistent"])
def test_conservation(order, recon, channel_small):
    m, L, p, (u, h, tr), run = channel_small
    q = dict(p, recon=recon)
    o = oracle.Oracle(m, L, q)
    u1, h1, tr1 = o.step(order, 120.0, 8, u, h, tr, n_steps=6)
    v0, c0 = _content(m, h, tr)
    v1, c1 = _content(m, h1, tr1)
    assert abs(v1 - v0) / v0 < 1e-13
    assert abs(c1 - c0) / c0 < 1e-13


@pytest.mark.parametrize("order", [2, 3])
def test_reconciliation_identities(order, channel_small):
    m, L, p, (u, h, tr), run = channel_small
    dt, M = run["dt"], run["M"]
    o = oracle.Oracle(m, L, dict(p, recon="consistent"))
    _, h1, _, aux = o.step(order, dt, M, u, h, tr, aux=True)
    zs = aux["zeta_sub"]
    H = m.bottomDepth
    assert np.abs(h1.sum(1) - H - zs).max() < 1e-11
    o = oracle.Oracle(m, L, dict(p, recon="paper"))
    _, h1, _, aux = o.step(order, dt, M, u, h, tr, aux=True)
    if order == 2:
        resid = -0.5 * dt * o.div(aux["D1"])
    else:
        resid = -dt / 6.0 * o.div(aux["D1"] + aux["D2"])
    got = h1.sum(1) - H - aux["zeta_sub"]
    assert np.abs(resid).max() > 1e-9          # the printed form is not consistent
    assert np.abs(got - resid).max() < 1e-11


@pytest.mark.parametrize("order", [2, 3])
def test_lake_at_rest_flat(order):
    m, L, p, (u, h, tr) = inputs.channel_case(8, 10, 10e3, 5)
    tr[:] = 12.0
    o = oracle.Oracle(m, L, p)
    u1, h1, tr1 = o.step(order, 300.0, 10, np.zeros_like(u), h, tr, n_steps=3)
    assert np.abs(u1).max() == 0.0
    assert np.abs(h1 - h).max() < 1e-12     # convex weights 1/3, 2/3 round


@pytest.mark.parametrize("order", [2, 3])
def test_lake_at_rest_bathymetry(order):
    """Uniform density over a seamount: the layer PGF (grad p + g rho grad z)
    cancels g grad zeta exactly, so nothing moves (to roundoff)."""
    def depth(x, y):
        return 1000.0 - 400.0 * np.exp(-((x - 40e3) ** 2 + (y - 40e3) ** 2) / (20e3) ** 2)
    m, L, p, (u, h, tr) = inputs.channel_case(8, 10, 10e3, 6, depth=depth)
    tr[:] = 12.0
    o = oracle.Oracle(m, L, p)
    u1, h1, tr1 = o.step(order, 300.0, 10, np.zeros_like(u), h, tr, n_steps=3)
    # the residual is the rounding of grad p / rho0 ~ 0.14 m s^-2 against
    # g rho grad z: eps * 0.14 * dt * stages * steps ~ 1e-12
    assert np.abs(u1).max() < 1e-12
    assert np.abs(h1 - h).max() < 1e-11


@pytest.mark.parametrize("order", [2, 3])
def test_constant_tracer_preserved(order):
    m, L, p, (u, h, tr) = inputs.channel_case(8, 10, 10e3, 5, perturb=True, nTracers=2,
                                              kappa_h=5.0, kappa_v=1e-5)
    tr[1] = 34.5
    o = oracle.Oracle(m, L, p)
    u1, h1, tr1 = o.step(order, 200.0, 10, u, h, tr, n_steps=4)
    assert np.abs(tr1[1] - 34.5).max() < 1e-12
    assert np.abs(u1 - u).max() > 1e-4   # the flow did evolve


def _rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.slow
@pytest.mark.parametrize("order", [2, 3])
def test_temporal_self_convergence(order):
    """Relative l2 of u_1 and h_1 (Sec. 5 metric) vs a dt/8 reference of the
    finest run: rate 2 for both schemes."""
    m, L, p, (u, h, tr) = inputs.channel_case(12, 16, 10e3, 6, perturb=True)
    o = oracle.Oracle(m, L, p)
    T, M = 1920.0, 8
    ref = o.step(order, T / 512, M, u, h, tr, n_steps=512)
    eu, eh = [], []
    for n in (16, 32, 64):
        r = o.step(order, T / n, M, u, h, tr, n_steps=n)
        eu.append(_rel_l2(r[0][:, 0], ref[0][:, 0]))
        eh.append(_rel_l2(r[1][:, 0], ref[1][:, 0]))
    ru = np.log2(np.array(eu[:-1]) / np.array(eu[1:]))
    rh = np.log2(np.array(eh[:-1]) / np.array(eh[1:]))
    # SSPRK3-SE approaches 2 from above in u_1 and from below in h_1
    assert np.all(ru > 1.75) and np.all(rh > 1.75), (ru, rh)
    assert np.all(ru < 2.6) and np.all(rh < 2.6), (ru, rh)
