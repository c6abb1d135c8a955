"""Brute-force pin of the oracle: on tiny meshes the C oracle's SSPRK2-SE and
SSPRK3-SE steps equal a second FP64 implementation written with dense
operator matrices (tests/dense_scheme.py), which shares no code with it.

Every term is switched on (beta plane, bathymetry, walls, T and S, wind
stress, bottom drag, horizontal, biharmonic and vertical viscosity and
diffusion), so a
dropped term, a wrong sign, a wrong index or a transposed operand in either
implementation shows up as a mismatch far above rounding.
"""
import numpy as np
import pytest

import oracle
from paper_2105_13484_gb300 import inputs, mesh as meshmod
from dense_scheme import DenseScheme


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def tiny_case(kind, L, seed):
    rng = np.random.default_rng(seed)
    if kind == "torus":
        m = meshmod.planar_hex(4, 4, 20e3, periodic_y=True, f0=1e-4, beta=2e-10)
    else:
        # 4 x 4 ocean cells between land rows, seamount-like bottom
        m = meshmod.planar_hex(4, 4, 20e3, land_rows=2, f0=1e-4, beta=2e-10,
                               depth=lambda x, y: 800.0 + 150.0 * np.cos(x / 13e3) * np.sin(y / 9e3))
    C, E = m.nCells, m.nEdges
    s = np.full(L, 1.0 / L)
    zeta = 0.3 * rng.standard_normal(C)
    h = (m.bottomDepth + zeta)[:, None] * s[None, :] * (1 + 0.05 * rng.standard_normal((C, L)))
    u = 0.2 * rng.standard_normal((E, L))
    T = 15 + 3 * rng.standard_normal((C, L))
    S = 35 + 0.5 * rng.standard_normal((C, L))
    p = dict(inputs.PHYS)
    p.update(nTracers=2, nu_h=40.0, nu_v=1e-2, kappa_h=30.0, kappa_v=5e-3, c_drag=2e-3,
             nu_4=1e12, windStress=0.1 * rng.standard_normal(E))
    return m, L, p, (u, h, np.stack([T, S]))


@pytest.mark.parametrize("kind", ["torus", "walls"])
@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("recon", ["consistent", "paper", "off"])
def test_oracle_equals_dense_matrix_scheme(kind, order, recon):
    L = 3
    m, L, p, (u, h, tr) = tiny_case(kind, L, seed=11 + order)
    p["recon"] = recon
    dt, M, nsteps = 120.0, 4, 2
    o = oracle.Oracle(m, L, p)
    uo, ho, to = o.step(order, dt, M, u.copy(), h.copy(), tr.copy(), n_steps=nsteps)
    d = DenseScheme(m, L, p)
    ud, hd, td = u.copy(), h.copy(), tr.copy()
    for _ in range(nsteps):
        ud, hd, td = d.step(order, dt, M, ud, hd, td)
    # the state moved well away from the initial one: the comparison is not trivial
    assert rel(ud, u) > 1e-3 and rel(hd, h) > 1e-8
    assert rel(uo, ud) < 1e-12
    assert rel(ho, hd) < 1e-14
    assert rel(to, td) < 1e-13


def test_dense_matrices_pin_operator_identities():
    """The dense operators obey the TRiSK identities on their own (doubly
    periodic mesh: every vertex and cell is interior)."""
    m, L, p, _ = tiny_case("torus", 2, seed=3)
    d = DenseScheme(m, L, p)
    # curl grad = 0 and div of the discrete curl (dual) field = 0
    assert np.abs(d.Curl @ d.Grad).max() < 1e-12 * np.abs(d.Curl).max() * np.abs(d.Grad).max()
    assert np.abs(d.Div @ d.Rot).max() < 1e-12 * np.abs(d.Div).max() * np.abs(d.Rot).max()
    m, L, p, _ = tiny_case("walls", 2, seed=3)
    d = DenseScheme(m, L, p)
    # the Coriolis operator does no work: l d * Cor is antisymmetric
    W = (m.dvEdge * m.dcEdge)[:, None] * d.Cor
    assert np.abs(W + W.T).max() < 1e-12 * np.abs(W).max()


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("vmix", [0, 1])
def test_oracle_equals_dense_with_partial_bottom_cells(order, vmix):
    """Partial bottom cells (1 to 4 active layers, cut bottom layers) with every
    term on, Algorithm 1 and Algorithm 2: the oracle against the dense-matrix
    implementation."""
    rng = np.random.default_rng(21 + order)
    m = meshmod.planar_hex(4, 4, 20e3, land_rows=2, f0=1e-4, beta=2e-10,
                           depth=lambda x, y: 120.0 + 700.0 * (0.5 + 0.5 * np.sin(x / 9e3 + y / 7e3)))
    L = 4
    K, rest = inputs.partial_bottom(m, L)
    assert K.min() < K.max()
    C, E = m.nCells, m.nEdges
    zeta = 0.3 * rng.standard_normal(C)
    h = rest * ((m.bottomDepth + zeta) / m.bottomDepth)[:, None]
    Ke = np.minimum(K[m.cellsOnEdge[:, 0]], K[m.cellsOnEdge[:, 1]])
    u = np.where(np.arange(L)[None, :] < Ke[:, None], 0.2 * rng.standard_normal((E, L)), 0.0)
    act = np.arange(L)[None, :] < K[:, None]
    tr = np.stack([np.where(act, 15 + 3 * rng.standard_normal((C, L)), 0.0),
                   np.where(act, 35 + 0.5 * rng.standard_normal((C, L)), 0.0)])
    p = dict(inputs.PHYS)
    p.update(nTracers=2, nu_h=40.0, nu_v=1e-2, kappa_h=30.0, kappa_v=5e-3, c_drag=2e-3,
             nu_4=1e12, windStress=0.1 * rng.standard_normal(E), vmix=vmix, recon="consistent")
    o = oracle.Oracle(m, L, p, max_level=K, rest_thickness=rest)
    uo, ho, to = o.step(order, 120.0, 4, u.copy(), h.copy(), tr.copy(), n_steps=2)
    d = DenseScheme(m, L, p, max_level=K, rest_thickness=rest)
    ud, hd, td = u.copy(), h.copy(), tr.copy()
    for _ in range(2):
        ud, hd, td = d.step(order, 120.0, 4, ud, hd, td)
    assert rel(ud, u) > 1e-3
    assert rel(uo, ud) < 1e-12
    assert rel(ho, hd) < 1e-14
    assert rel(to, td) < 1e-13
    # inactive layers stay empty
    assert np.abs(ho[~act]).max() == 0 and np.abs(to[:, ~act]).max() == 0
    assert np.abs(uo[np.arange(L)[None, :] >= Ke[:, None]]).max() == 0


def test_every_term_is_exercised_by_the_brute_force_case():
    """The brute-force comparison pins a term only if the case exercises it:
    removing any one physics term moves the two-step result by orders of
    magnitude more than the comparison's tolerance."""
    m, L, p, (u, h, tr) = tiny_case("walls", 3, seed=14)
    base = oracle.Oracle(m, L, p).step(3, 120.0, 4, u.copy(), h.copy(), tr.copy(), n_steps=2)
    for term, off, field, least in [("c_drag", 0.0, 0, 1e-5), ("windStress", None, 0, 1e-6),
                                    ("nu_h", 0.0, 0, 1e-6), ("nu_v", 0.0, 0, 1e-7),
                                    ("nu_4", 0.0, 0, 1e-4), ("kappa_h", 0.0, 2, 1e-7),
                                    ("kappa_v", 0.0, 2, 1e-7)]:
        q = dict(p)
        q[term] = off
        out = oracle.Oracle(m, L, q).step(3, 120.0, 4, u.copy(), h.copy(), tr.copy(), n_steps=2)
        assert rel(out[field], base[field]) > least, term
