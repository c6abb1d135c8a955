"""Pins of the oracle's Algorithms 1, 3 and 4 against closed forms.

* Algorithm 1: the thickness-weighted mean of the baroclinic output vanishes
  and G is the thickness-weighted mean tendency (Alg. 1, lines 2-3).
* Algorithms 3 / 4: the sub-cycle is textbook SSPRK2 / SSPRK3 (Eqs. SSPRK2,
  SSPRK3) applied M times; on a single hexagonal Fourier mode of the linear
  f = 0 system it reproduces the SSPRK stability polynomial with the exact
  semi-discrete frequency; the accumulated flux of Sec. 3.4 reproduces the
  sub-cycle's own SSH; SSPRK3 sub-cycling is third order.
* Proposition 1: the third-order term of M SSPRK2 sub-steps.
* Linear inertia-gravity waves on an f-plane: eigenvalues of the assembled
  linear barotropic operator vs omega^2 = f^2 + g H k^2.
"""
import numpy as np
import pytest

import oracle
from paper_2105_13484_gb300 import inputs
from paper_2105_13484_gb300 import mesh as meshgen

G_ACC = 9.80616


def _r2(z):
    return 1 + z + z * z / 2


def _r3(z):
    return 1 + z + z * z / 2 + z ** 3 / 6


def test_split_mean_free(channel_small):
    m, L, p, (u, h, tr), run = channel_small
    o = oracle.Oracle(m, L, p)
    ubar, ut = o.split(u, h)
    he = o.edge_thickness(h)
    assert np.abs((he * ut).sum(1)).max() < 1e-12 * np.abs(he * u).sum(1).max()
    assert np.allclose(ubar[:, None] + ut, u, rtol=0, atol=1e-15)


def test_alg1_mean_free_and_G(channel_small):
    m, L, p, (u, h, tr), run = channel_small
    o = oracle.Oracle(m, L, p)
    ubar, ut = o.split(u, h)
    zeta = o.ssh(h)
    dt = run["dt"]
    ut1, G = o.baroclinic_feuler(u, ut, zeta, h, tr, dt)
    he = o.edge_thickness(h)
    # line 3: mass-weighted mean of the output is zero
    assert np.abs((he * ut1).sum(1)).max() < 1e-12 * np.abs(he * ut).sum(1).max()
    # line 2: G = mean of (ut + dt * rhs) / dt
    rhs = o.baroclinic_rhs(u, ut, zeta, h, tr)
    Gref = ((he * (ut + dt * rhs)).sum(1) / he.sum(1)) / dt
    assert np.allclose(G, Gref, rtol=1e-12, atol=1e-14 * np.abs(Gref).max())
    assert np.abs(G).max() > 0


def _torus_case(n=12, d=5e3, H=1000.0, f=0.0):
    m = meshgen.planar_hex(n, n, d, periodic_y=True, f0=f, depth=H)
    return m, oracle.Oracle(m, 1, dict(g=G_ACC))


@pytest.mark.parametrize("order", [2, 3])
def test_subcycle_matches_ssprk_polynomial_on_fourier_mode(order):
    """Standing gravity wave zeta = eps cos(k.x), u = 0 on the f = 0 torus: the
    sub-cycle returns zeta * Re(R(i omega tau)^M), R the SSPRK polynomial and
    omega^2 = -g H lambda(k), lambda the exact hex Laplacian eigenvalue."""
    n, d, H = 12, 5e3, 1000.0
    m, o = _torus_case(n, d, H)
    Lx = n * d
    k = np.array([2 * np.pi / Lx, 0.0])
    r = d * np.array([[np.cos(a), np.sin(a)] for a in np.arange(6) * np.pi / 3])
    lam = 2.0 / (3 * d * d) * np.sum(np.cos(r @ k) - 1.0)
    omega = np.sqrt(-G_ACC * H * lam)
    eps = 1e-6
    zeta0 = eps * np.cos(m.xCell @ k)
    dt, M = 200.0, 10
    tau = dt / M
    _, Fz, z1 = o.barotropic_substep(order, np.zeros(m.nEdges), zeta0, np.zeros(m.nEdges), dt, M)
    R = (_r2 if order == 2 else _r3)(1j * omega * tau)
    pred = zeta0 * np.real(R ** M)
    assert np.abs(z1 - pred).max() < 1e-9 * eps
    # continuous-limit frequency: relative error O((k d)^2)
    assert abs(omega / (np.sqrt(G_ACC * H) * k[0]) - 1) < (k[0] * d) ** 2


@pytest.mark.parametrize("order", [2, 3])
def test_accumulated_flux_reproduces_subcycle_ssh(order, channel_small):
    """Sec. 3.4: zeta^{M/M} = zeta^0 - dt div(F^zeta)."""
    m, L, p, (u, h, tr), run = channel_small
    o = oracle.Oracle(m, L, p)
    ubar, _ = o.split(u, h)
    zeta = o.ssh(h)
    G = 1e-6 * np.sin(np.arange(m.nEdges))
    dt, M = 300.0, 7
    u1, Fz, z1 = o.barotropic_substep(order, ubar, zeta, G, dt, M)
    assert np.abs(z1 - (zeta - dt * o.div(Fz))).max() < 1e-13 * (1 + np.abs(zeta).max())


@pytest.mark.parametrize("order,rate", [(2, 2.0), (3, 3.0)])
def test_subcycle_temporal_order(order, rate):
    """Global error of M sub-steps over a fixed dt vs the exact cos(omega dt)."""
    n, d, H = 12, 5e3, 1000.0
    m, o = _torus_case(n, d, H)
    k = np.array([2 * np.pi / (n * d), 0.0])
    r = d * np.array([[np.cos(a), np.sin(a)] for a in np.arange(6) * np.pi / 3])
    lam = 2.0 / (3 * d * d) * np.sum(np.cos(r @ k) - 1.0)
    omega = np.sqrt(-G_ACC * H * lam)
    eps = 1e-6
    zeta0 = eps * np.cos(m.xCell @ k)
    dt = 200.0
    errs = []
    for M in (16, 32, 64):
        _, _, z1 = o.barotropic_substep(order, np.zeros(m.nEdges), zeta0, np.zeros(m.nEdges), dt, M)
        errs.append(np.abs(z1 - zeta0 * np.cos(omega * dt)).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    # the phase error (next order) still shows at M = 16; the last rate is asymptotic
    assert abs(rates[0] - rate) < 0.3 and abs(rates[-1] - rate) < 0.15, rates


def test_proposition1_third_order_term():
    """Prop. 1: ubar after M SSPRK2 sub-steps vs its Taylor expansion.

    Direct expansion of (1 + a + a^2/2)^M gives the Delta t^3 coefficient
    (M^2 - 1) / (6 M^2); with it the residual falls as Delta t^4.  The
    printed coefficient (M^2 - 1) / (3 M^2) leaves a Delta t^3 residual."""
    m = meshgen.planar_hex(10, 10, 10e3, periodic_y=True, f0=1e-4, depth=1000.0)
    o = oracle.Oracle(m, 1, dict(g=G_ACC))
    rng = np.random.default_rng(7)
    eps = 1e-7
    ubar = eps * rng.standard_normal(m.nEdges) * 30
    zeta = eps * 1000 * rng.standard_normal(m.nCells)
    Gs = eps * 1e-3 * rng.standard_normal(m.nEdges)
    H = m.bottomDepth
    M = 4

    def avg(c):
        return 0.5 * (c[m.cellsOnEdge[:, 0]] + c[m.cellsOnEdge[:, 1]])

    F = -(o.coriolis(ubar) - G_ACC * o.grad(zeta) + Gs)
    P = o.div(ubar * avg(zeta + H))
    E = -o.coriolis(F) + G_ACC * o.grad(P)
    Q = o.div(ubar * avg(P) + avg(zeta + H) * F)
    X = -o.coriolis(E) + G_ACC * o.grad(Q)
    res_fixed, res_printed = [], []
    dts = np.array([240.0, 120.0, 60.0, 30.0])
    for dt in dts:
        u1, _, _ = o.barotropic_substep(2, ubar, zeta, Gs, dt, M)
        base = ubar - dt * F + dt * dt / 2 * E
        res_fixed.append(np.abs(u1 - (base - (M * M - 1) / (6 * M * M) * dt ** 3 * X)).max())
        res_printed.append(np.abs(u1 - (base - (M * M - 1) / (3 * M * M) * dt ** 3 * X)).max())
    r_fixed = np.log2(np.array(res_fixed[:-1]) / np.array(res_fixed[1:]))
    r_printed = np.log2(np.array(res_printed[:-1]) / np.array(res_printed[1:]))
    assert np.all(r_fixed > 3.7), r_fixed
    assert abs(r_printed[-1] - 3.0) < 0.2, r_printed
    assert res_printed[-1] > 20 * res_fixed[-1]


def _linear_operator(m, o):
    """Assemble the linear barotropic operator at rest (G = 0) column by column."""
    E, C = m.nEdges, m.nCells
    A = np.zeros((E + C, E + C))
    for j in range(E + C):
        x = np.zeros(E + C)
        x[j] = 1.0
        u1, z1, _ = o.barotropic_fe(x[:E], x[E:], np.zeros(E), 1.0)
        A[:, j] = np.concatenate([u1 - x[:E], z1 - x[E:]])
    return A


def test_inertia_gravity_wave_frequencies():
    """f-plane, flat bottom: the linear operator is skew (energy-neutral) and
    its lowest inertia-gravity frequency converges to sqrt(f^2 + g H k^2)
    at second order in k d."""
    f, H, Lx = 1e-4, 1000.0, 400e3
    errs = []
    for n in (6, 12):
        d = Lx / n
        m = meshgen.planar_hex(n, n, d, periodic_y=True, f0=f, depth=H)
        o = oracle.Oracle(m, 1, dict(g=G_ACC))
        A = _linear_operator(m, o)
        ev = np.linalg.eigvals(A)
        assert np.abs(ev.real).max() < 1e-9 * np.abs(ev).max()
        k = 2 * np.pi / Lx
        w_exact = np.sqrt(f * f + G_ACC * H * k * k)
        w = np.abs(ev.imag)
        w_num = w[np.argmin(np.abs(w - w_exact))]
        # inertial floor: no IG frequency below f
        assert w[w > 0.5 * f].min() > f * (1 - 1e-9)
        errs.append(abs(w_num / w_exact - 1))
    assert errs[1] < errs[0] / 3.0
    assert errs[1] < 0.02


@pytest.mark.parametrize("order", [2, 3])
def test_full_scheme_gravity_wave_ten_layers(order):
    """The whole SSPRK-SE step with 10 layers, uniform density rho, flat bottom,
    f = 0 and a small SSH Fourier mode at rest: the depth-mean flow obeys the
    linear shallow-water equations with the reduced gravity g rho / rho0 of
    the Boussinesq pressure gradient, whose exact semi-discrete solution is the
    standing wave zeta(t) = eta0 cos(omega t) on the mode, omega^2 = g (rho /
    rho0) H lambda', lambda' = -lambda the hex Laplacian eigenvalue.  The error of the
    fully discrete scheme falls at second order under dt refinement (M
    fixed); every layer keeps its rest share of the column (z-star) and the
    baroclinic velocity stays zero."""
    n, d, H, f0, L = 12, 5e3, 1000.0, 0.0, 10
    m = meshgen.planar_hex(n, n, d, periodic_y=True, f0=f0, depth=H)
    Lx = n * d
    k = np.array([2 * np.pi / Lx, 0.0])
    r = d * np.array([[np.cos(a), np.sin(a)] for a in np.arange(6) * np.pi / 3])
    lam = -2.0 / (3 * d * d) * np.sum(np.cos(r @ k) - 1.0)
    P = inputs.PHYS
    rho = P["eos_rho_ref"] - P["eos_alpha"] * (12.0 - P["eos_T_ref"])
    geff = G_ACC * rho / P["rho0"]
    omega = np.sqrt(f0 ** 2 + geff * H * lam)
    eta0 = 1e-3
    mode = np.cos(m.xCell @ k)
    h = (H + eta0 * mode)[:, None] * np.full(L, 1.0 / L)[None, :]
    tr = np.full((1, m.nCells, L), 12.0)
    u = np.zeros((m.nEdges, L))
    p = dict(inputs.PHYS, nTracers=1)
    o = oracle.Oracle(m, L, p)

    def run(dt, M=10, T=1600.0):
        uu, hh, tt = u.copy(), h.copy(), tr.copy()
        nper = int(round(200.0 / dt))
        worst, t = 0.0, 0.0
        while t < T - 1e-9:
            uu, hh, tt = o.step(order, dt, M, uu, hh, tt, n_steps=nper)
            t += nper * dt
            a = ((hh.sum(1) - H) @ mode) / (mode @ mode)
            exact = eta0 * np.cos(omega * t)
            worst = max(worst, abs(a - exact) / eta0)
        return worst, uu, hh

    w40, _, _ = run(40.0)
    w20, u, h = run(20.0)
    # the time error (a phase error growing over ~2.6 periods) falls at about
    # second order: the discrete frequency is the closed-form one
    assert w20 < w40 / 3.0 and w20 < 2e-3, (w40, w20)
    assert np.abs(h - h.sum(1, keepdims=True) / L).max() < 1e-12 * H
    assert np.abs(u - u.mean(1, keepdims=True)).max() < 1e-12
