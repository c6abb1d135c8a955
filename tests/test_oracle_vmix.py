"""Pins of Algorithm 2 (Baroclinic_FEuler_Mixing, implicit vertical mixing)
in the oracle.

* The solve (I - dt D^u) x = r: a vertical cosine mode on uniform layers is
  an eigenvector of the discrete operator with zero-flux ends, so backward
  Euler divides it by 1 + dt (4 nu / h^2) sin^2(pi m / 2L); interior mixing
  conserves sum_k h_e,k x_k; a one-layer column with drag only gives
  r / (1 + dt c_d |u| / h); the solution satisfies the explicit D^u of the
  oracle's Algorithm 1 to rounding.
* Algorithm 2 without viscosity, drag and wind equals Algorithm 1.
* With mixing the scheme still conserves volume and tracers, and it stays
  stable at a vertical viscosity where the explicit form blows up.
"""
import numpy as np
import pytest

import oracle
from paper_2105_13484_gb300 import inputs
from paper_2105_13484_gb300 import mesh as meshgen


def _col_case(L, nu_v, c_drag=0.0, wind=None, H=400.0):
    m = meshgen.planar_hex(4, 4, 10e3, periodic_y=True, depth=H)
    p = dict(inputs.PHYS, nu_v=nu_v, c_drag=c_drag, windStress=wind, vmix=1)
    return m, oracle.Oracle(m, L, p)


@pytest.mark.parametrize("mode", [1, 2, 5])
def test_vertical_cosine_mode_closed_form(mode):
    L, H, nu, dt = 10, 400.0, 0.05, 600.0
    m, o = _col_case(L, nu, H=H)
    h = np.full((m.nCells, L), H / L)
    k = np.arange(L)
    prof = np.cos(np.pi * mode * (k + 0.5) / L)
    r = np.outer(np.linspace(0.5, 1.5, m.nEdges), prof)
    x = o.vertical_mixing_solve(np.zeros((m.nEdges, L)), h, r, dt)
    dz = H / L
    lam = 4 * nu / dz ** 2 * np.sin(np.pi * mode / (2 * L)) ** 2
    assert np.abs(x - r / (1 + dt * lam)).max() < 1e-14


def test_mixing_conserves_column_momentum_and_solves_the_system():
    L, nu, dt = 7, 0.02, 900.0
    m, o = _col_case(L, nu)
    rng = np.random.default_rng(1)
    h = 30.0 + 40.0 * rng.random((m.nCells, L))
    r = rng.standard_normal((m.nEdges, L))
    x = o.vertical_mixing_solve(np.zeros((m.nEdges, L)), h, r, dt)
    he = o.edge_thickness(h)
    assert np.abs((he * x).sum(1) - (he * r).sum(1)).max() < 1e-12 * np.abs(he * r).sum(1).max()
    # the residual with the explicit vertical operator: x - dt D^u(x) = r
    D = np.zeros_like(x)
    hi = 0.5 * (he[:, :-1] + he[:, 1:])
    X = np.zeros((m.nEdges, L + 1))
    X[:, 1:L] = nu * (x[:, :-1] - x[:, 1:]) / hi
    D = (X[:, :L] - X[:, 1:]) / he
    assert np.abs(x - dt * D - r).max() < 1e-12


def test_one_layer_drag_closed_form():
    m, o = _col_case(1, 0.0, c_drag=2e-3)
    rng = np.random.default_rng(2)
    h = np.full((m.nCells, 1), 50.0)
    ud = 0.3 * rng.standard_normal((m.nEdges, 1))
    r = rng.standard_normal((m.nEdges, 1))
    x = o.vertical_mixing_solve(ud, h, r, 300.0)
    speed = np.sqrt(ud[:, 0] ** 2 + o.tangential(ud)[:, 0] ** 2)
    assert np.abs(x[:, 0] - r[:, 0] / (1 + 300.0 * 2e-3 * speed / 50.0)).max() < 1e-15


def test_wind_enters_the_top_layer_explicitly():
    L = 3
    m = meshgen.planar_hex(4, 4, 10e3, periodic_y=True, depth=300.0)
    wind = np.linspace(-0.1, 0.1, m.nEdges)
    p = dict(inputs.PHYS, nu_v=0.0, windStress=wind, vmix=1)
    o = oracle.Oracle(m, L, p)
    h = np.full((m.nCells, L), 100.0)
    r = np.zeros((m.nEdges, L))
    x = o.vertical_mixing_solve(np.zeros_like(r), h, r, 100.0)
    assert np.abs(x[:, 0] - 100.0 * wind / p["rho0"] / 100.0).max() < 1e-18
    assert np.abs(x[:, 1:]).max() == 0.0


def test_alg2_equals_alg1_without_vertical_terms(channel_small):
    m, L, p, (u, h, tr), run = channel_small
    p = dict(p, nu_v=0.0, c_drag=0.0, windStress=None)
    o1 = oracle.Oracle(m, L, dict(p, vmix=0))
    o2 = oracle.Oracle(m, L, dict(p, vmix=1))
    ubar, ut = o1.split(u, h)
    zeta = o1.ssh(h)
    a1, G1 = o1.baroclinic_feuler(u, ut, zeta, h, tr, 300.0)
    a2, G2 = o2.baroclinic_feuler_mixing(u, ut, ubar, zeta, h, tr, 300.0)
    assert np.abs(G2 - G1).max() == 0.0
    assert np.abs(a2 - a1).max() < 1e-15 * (1 + np.abs(ubar).max())


@pytest.mark.parametrize("order", [2, 3])
def test_mixing_scheme_conserves_and_is_stable_where_explicit_is_not(order):
    m, L, p, (u, h, tr) = inputs.channel_case(8, 10, 10e3, 10, depth=100.0, perturb=True,
                                              nu_v=0.5, c_drag=2e-3)
    A = m.areaCell
    v0 = A @ h.sum(1)
    c0 = A @ (h * tr[0]).sum(1)
    dt, M = 300.0, 10                     # 10 m layers: nu_v dt / dz^2 = 1.5
    o = oracle.Oracle(m, L, dict(p, vmix=1))
    u1, h1, t1 = o.step(order, dt, M, u, h, tr, n_steps=10)
    assert np.isfinite(u1).all() and np.abs(u1).max() < 2.0
    assert abs(A @ h1.sum(1) - v0) / v0 < 1e-13
    assert abs(A @ (h1 * t1[0]).sum(1) - c0) / c0 < 1e-13
    ox = oracle.Oracle(m, L, dict(p, vmix=0))
    ue, _, _ = ox.step(order, dt, M, u, h, tr, n_steps=10)
    assert not (np.isfinite(ue).all() and np.abs(ue).max() < 2.0)
