"""Pins of the oracle's TRiSK operators against closed forms and identities.

The paper (Sec. 5) uses the TRiSK scheme without writing it out; these tests
fix the discrete operators against properties that hold exactly on any
TRiSK mesh, or exactly on a regular periodic hexagonal mesh.
"""
import numpy as np
import pytest

import oracle
from paper_2105_13484_gb300 import mesh as meshgen


@pytest.fixture(scope="module")
def torus():
    """Fully periodic regular hex mesh (no walls), 12 x 10 cells, 5 km."""
    m = meshgen.planar_hex(12, 10, 5e3, periodic_y=True, f0=1e-4)
    return m, oracle.Oracle(m, 1)


@pytest.fixture(scope="module")
def channel():
    """Channel with walls on a beta plane."""
    m = meshgen.planar_hex(10, 12, 8e3, f0=1e-4, beta=2e-11)
    return m, oracle.Oracle(m, 1)


def test_mesh_regular_geometry(torus):
    m, _ = torus
    d = 5e3
    assert np.allclose(m.dcEdge, d, rtol=1e-13)
    assert np.allclose(m.dvEdge, d / np.sqrt(3), rtol=1e-13)
    assert np.allclose(m.areaCell, np.sqrt(3) / 2 * d * d, rtol=1e-13)
    assert np.allclose(m.areaTriangle, np.sqrt(3) / 4 * d * d, rtol=1e-13)
    assert (m.nEdgesOnEdge == 10).all()


def test_curl_of_grad_is_zero(torus, channel):
    rng = np.random.default_rng(1)
    for m, o in (torus, channel):
        phi = rng.standard_normal(m.nCells)
        c = o.curl(o.grad(phi))
        full = (m.edgesOnVertex >= 0).all(axis=1)   # vertices with all 3 edges
        scale = np.abs(o.grad(phi)).max() / m.dvEdge.min()
        assert np.abs(c[full]).max() < 1e-13 * scale


def test_div_of_discrete_curl_field_is_zero(torus):
    """u_e = (psi_v1 - psi_v2)/l_e is discretely non-divergent."""
    m, o = torus
    rng = np.random.default_rng(2)
    psi = rng.standard_normal(m.nVertices)
    u = (psi[m.verticesOnEdge[:, 0]] - psi[m.verticesOnEdge[:, 1]]) / m.dvEdge
    assert np.abs(o.div(u)).max() < 1e-13 * np.abs(u).max() / m.dcEdge.min()


def test_divergence_theorem(channel):
    m, o = channel
    F = np.random.default_rng(3).standard_normal(m.nEdges)
    total = m.areaCell @ o.div(F)
    assert abs(total) < 1e-12 * np.abs(F * m.dvEdge).sum()


def test_coriolis_does_no_work(torus, channel):
    """Energy neutrality of the TRiSK Coriolis term for any u (beta plane too)."""
    rng = np.random.default_rng(4)
    for m, o in (torus, channel):
        u = rng.standard_normal(m.nEdges)
        cf = o.coriolis(u)
        work = np.sum(m.dvEdge * m.dcEdge * u * cf)
        assert abs(work) < 1e-12 * np.sum(m.dvEdge * m.dcEdge * np.abs(u * cf))


def test_weights_antisymmetric(channel):
    m, _ = channel
    W = {}
    for e in range(m.nEdges):
        for j in range(m.nEdgesOnEdge[e]):
            W[(e, m.edgesOnEdge[e, j])] = m.weightsOnEdge[e, j]
    for (a, b), w in W.items():
        assert abs(w + W[(b, a)]) < 1e-14


def test_pv_flux_does_no_work(channel):
    """sum_e l_e d_e (h_e u_e) Q_e = 0: the PV flux conserves energy."""
    m, _ = channel
    o = oracle.Oracle(m, 3)
    rng = np.random.default_rng(5)
    u = rng.standard_normal((m.nEdges, 3))
    h = 50.0 + rng.random((m.nCells, 3))
    Q = o.pv_flux(u, h)
    he = o.edge_thickness(h)
    work = np.sum((m.dvEdge * m.dcEdge)[:, None] * he * u * Q, axis=0)
    scale = np.sum((m.dvEdge * m.dcEdge)[:, None] * np.abs(he * u * Q), axis=0)
    assert np.all(np.abs(work) < 1e-12 * scale)


def test_tangential_exact_for_uniform_flow(torus):
    m, o = torus
    for U in ((1.0, 0.0), (0.3, -0.7)):
        U = np.array(U)
        n = m.normalEdge
        t = np.stack([-n[:, 1], n[:, 0]], axis=1)
        ut = o.tangential(n @ U)
        assert np.abs(ut - t @ U).max() < 1e-13


def test_kinetic_energy_uniform_flow(torus):
    m, o = torus
    U = np.array([0.4, -0.25])
    K = o.kinetic_energy(m.normalEdge @ U)
    assert np.abs(K - 0.5 * U @ U).max() < 1e-14


def test_laplacian_of_hex_fourier_mode_closed_form(torus):
    """div(grad(cos k.x)) = lambda(k) cos(k.x) exactly on the regular hex grid,
    lambda = (2 / 3 d^2) sum_j (cos(k.r_j) - 1) over the 6 neighbour offsets."""
    m, o = torus
    d = 5e3
    Lx, Ly = 12 * d, 10 * d * np.sqrt(3) / 2
    r = d * np.array([[np.cos(a), np.sin(a)] for a in np.arange(6) * np.pi / 3])
    for kx, ky in ((2 * np.pi / Lx, 0.0), (4 * np.pi / Lx, 2 * np.pi / Ly),
                   (2 * np.pi / Lx, -4 * np.pi / Ly)):
        k = np.array([kx, ky])
        phi = np.cos(m.xCell @ k)
        lam = 2.0 / (3 * d * d) * np.sum(np.cos(r @ k) - 1.0)
        got = o.div(o.grad(phi))
        assert np.abs(got - lam * phi).max() < 1e-12 * abs(lam)


def test_vector_laplacian_identities(torus):
    """Lap(grad phi) = grad(div grad phi) (curl grad = 0) and uniform flow has
    zero Laplacian."""
    m, o = torus
    rng = np.random.default_rng(6)
    phi = rng.standard_normal(m.nCells)
    g = o.grad(phi)
    assert np.allclose(o.laplacian(g), o.grad(o.div(g)), rtol=0, atol=1e-12 * np.abs(g).max() / 1e6)
    assert np.abs(o.laplacian(m.normalEdge @ np.array([1.0, 2.0]))).max() < 1e-18


def test_grad_second_order_convergence():
    """grad of a smooth field converges at second order at edge midpoints."""
    errs = []
    for n in (8, 16, 32):
        d = 100e3 / n
        m = meshgen.planar_hex(n, n, d, periodic_y=True)
        o = oracle.Oracle(m, 1)
        Lx = n * d
        k = 2 * np.pi / Lx
        phi = np.sin(k * m.xCell[:, 0])
        exact = k * np.cos(k * m.xEdge[:, 0]) * m.normalEdge[:, 0]
        errs.append(np.abs(o.grad(phi) - exact).max() / k)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.9)


def test_vertex_thickness_uniform(channel):
    m, _ = channel
    o = oracle.Oracle(m, 2)
    h = np.full((m.nCells, 2), 37.5)
    assert np.allclose(o.vertex_thickness(h), 37.5, rtol=1e-15)


def test_biharmonic_of_gradient_mode_is_lambda_squared(torus):
    """del^4 (grad phi) = lambda^2 grad phi for a hex Fourier mode phi: the
    vector Laplacian of a gradient field is grad(div), and div(grad phi) =
    lambda phi exactly (closed form above)."""
    m, o = torus
    d = 5e3
    Lx, Ly = 12 * d, 10 * d * np.sqrt(3) / 2
    r = d * np.array([[np.cos(a), np.sin(a)] for a in np.arange(6) * np.pi / 3])
    for kx, ky in ((2 * np.pi / Lx, 0.0), (4 * np.pi / Lx, 2 * np.pi / Ly)):
        k = np.array([kx, ky])
        phi = np.cos(m.xCell @ k)
        lam = 2.0 / (3 * d * d) * np.sum(np.cos(r @ k) - 1.0)
        u = o.grad(phi)
        got = o.biharmonic(u)
        assert np.abs(got - lam * lam * u).max() < 1e-11 * lam * lam * np.abs(u).max()


def test_biharmonic_is_self_adjoint_and_dissipative(torus):
    """<u, del^4 u> = <del^2 u, del^2 u> >= 0 in the l d inner product, for
    any u (the Laplacian is symmetric there, so -nu_4 del^4 removes energy)."""
    m, o = torus
    rng = np.random.default_rng(7)
    W = m.dvEdge * m.dcEdge
    for _ in range(3):
        u = rng.standard_normal(m.nEdges)
        a = np.sum(W * u * o.biharmonic(u))
        lu = o.laplacian(u)
        b = np.sum(W * lu * lu)
        assert b > 0 and abs(a - b) < 1e-12 * b
