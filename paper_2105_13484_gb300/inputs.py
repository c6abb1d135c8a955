"""Seeded synthetic workloads shaped like the paper's test cases.

Input generation only: meshes (from ``mesh.py``), physical parameters and
initial states.  Nothing here performs any step of the time-stepping method;
both the CUDA path and the CPU oracle are fed from these generators.

Workloads (the paper's MPAS meshes and data are not available, so these
stand in for them):

* ``channel_10km``  16 x 32 hexagonal channel, 10 km spacing, 10 layers x 100 m,
  flat 1000 m bottom, f-plane f = 1.2e-4, temperature-only linear EOS,
  tanh temperature front across y plus a 1 K sinusoidal perturbation with a
  seeded phase (the baroclinic-eddies setup of Sec. 5.1 in miniature).
  SSPRK2-SE, dt = 300 s, M = 20, 10 steps.
* ``channel_1km``   160 x 578 cells at 1 km (160 km x 500 km, 92,480 cells),
  20 layers x 50 m, beta plane, same front.  SSPRK3-SE, dt = 60 s, M = 30.
* ``sphere_l7``     icosahedral geodesic sphere at level 7 (163,842 cells before
  the land mask), 60 z-star layers, seeded bathymetry 100-5000 m, ~30 % land,
  T and S with the linear EOS, f = 2 Omega sin(lat), seeded zonal wind stress.
  SSPRK3-SE, dt = 600 s, M = 40, 144 steps.  ``sphere_l4`` is the same
  recipe at level 4 (2,562 cells) with 12 layers for parity tests.
"""
from __future__ import annotations

import math

import numpy as np

from . import mesh as _mesh

PHYS = dict(g=9.80616, rho0=1000.0, eos_rho_ref=1000.0, eos_alpha=0.2, eos_beta=0.8,
            eos_T_ref=10.0, eos_S_ref=35.0)


def channel_state(m, L, *, seed=0, width=40e3, dT=5.0, amp=1.0, perturb=False,
                  nTracers=1):
    """Initial (u [E,L], h [C,L], tracers [nT,C,L]) on a planar channel mesh.

    Temperature: linear from 20 C at the surface to 10 C at the bottom, a tanh
    front of height dT across the channel middle and an amp-K perturbation
    cos(2 pi m x / Lx + phase) (m in {1, 2}, seeded phase) confined to the
    front.  With ``perturb`` a smooth seeded velocity field and SSH
    perturbation are added so that every term of the tendencies is active.
    """
    rng = np.random.default_rng(seed)
    xc, yc = m.xCell[:, 0], m.xCell[:, 1]
    Lx = _channel_lx(m)
    y0 = 0.5 * (yc.min() + yc.max())
    mode = int(rng.integers(1, 3))
    phase = float(rng.uniform(0, 2 * np.pi))
    s = np.full(L, 1.0 / L)
    zeta = np.zeros(m.nCells)
    if perturb:
        kx = 2 * np.pi / Lx
        zeta = 0.2 * np.cos(kx * xc + rng.uniform(0, 6.3)) * np.exp(-((yc - y0) / (2 * width)) ** 2)
    H = m.bottomDepth
    h = (H + zeta)[:, None] * s[None, :]
    # layer mid depths as fractions of the column (at rest)
    zfrac = -(np.cumsum(s) - 0.5 * s)
    eta = (yc - y0) / width
    T = (20.0 + 10.0 * zfrac[None, :]
         - 0.5 * dT * np.tanh(eta)[:, None]
         + amp * (np.cos(mode * 2 * np.pi * xc / Lx + phase) / np.cosh(eta) ** 2)[:, None])
    tr = [T]
    if nTracers >= 2:
        S = 35.0 + 0.5 * np.tanh(eta)[:, None] - 0.2 * zfrac[None, :] + 0.0 * T[:, :1]
        tr.append(S)
    tr = np.stack(tr)
    u = np.zeros((m.nEdges, L))
    if perturb:
        xe, ye = m.xEdge[:, 0], m.xEdge[:, 1]
        n = m.normalEdge
        ky = np.pi / (yc.max() - yc.min())
        prof = np.exp(zfrac)  # decays with depth
        a, b = rng.uniform(0, 6.3, 2)
        U = 0.3 * np.sin(2 * np.pi * xe / Lx + a) * np.sin(ky * (ye - yc.min()))
        Vv = 0.3 * np.cos(4 * np.pi * xe / Lx + b) * np.sin(ky * (ye - yc.min()))
        un = U * n[:, 0] + Vv * n[:, 1]
        u = un[:, None] * prof[None, :] + 0.05 * np.sin(3 * ky * ye)[:, None] * (s[None, :] - s.mean())
    return u, h, tr


def _channel_lx(m):
    dc = float(np.median(m.dcEdge))
    return float(round((m.xCell[:, 0].max() - m.xCell[:, 0].min()) / dc + 0.5)) * dc


def channel_case(nx, ny, dc, L, *, depth=1000.0, f0=1.2e-4, beta=0.0, seed=0, perturb=False,
                 nTracers=1, **params):
    """(mesh, L, params, (u, h, tr)) for a planar channel."""
    m = _mesh.planar_hex(nx, ny, dc, depth=depth, f0=f0, beta=beta)
    u, h, tr = channel_state(m, L, seed=seed, perturb=perturb, nTracers=nTracers)
    p = dict(PHYS)
    p.update(nTracers=nTracers, recon="consistent", nu_h=10.0, nu_v=1e-4, kappa_h=0.0, kappa_v=0.0,
             c_drag=1e-3)
    p.update(params)
    return m, L, p, (u, h, tr)


def _low_degree_field(rng, deg=4):
    """Seeded smooth field on the unit sphere: a random polynomial of degree
    <= deg in (x, y, z), i.e. a combination of spherical harmonics of degree
    <= deg, returned as a function of unit vectors [n, 3]."""
    terms = [(a, b, c) for a in range(deg + 1) for b in range(deg + 1 - a)
             for c in range(deg + 1 - a - b)]
    coef = rng.standard_normal(len(terms)) / (1.0 + np.array([sum(t) for t in terms]))

    def field(p):
        x, y, z = p[:, 0], p[:, 1], p[:, 2]
        return sum(k * x ** a * y ** b * z ** c for k, (a, b, c) in zip(coef, terms))
    return field


# meshes already built, by (level, seed, land fraction, depth range): a mesh
# does not depend on the layer count or on the state drawn after it
_SPHERE_MESHES = {}


def sphere_case(level, L, *, seed=0, land_frac=0.3, dmin=100.0, dmax=5000.0, nTracers=2,
                wind=0.1, perturb=False, **params):
    """(mesh, L, params, (u, h, tr)) for the global-ocean-like sphere.

    Land: the cells where a seeded low-degree field is below its land_frac
    quantile (largest ocean basin kept).  Bathymetry: a second seeded field
    mapped linearly onto [dmin, dmax] over the ocean.  T decreases with
    latitude and depth (about 25 C at the equator surface to 5 C at depth), S
    between 34 and 36; u = 0 and zeta = 0 at rest (``perturb`` adds a seeded
    smooth SSH bump).  Wind stress: zonal, amplitude ``wind`` N m^-2, a seeded
    mix of cos(2 lat)-type bands, projected on the edge normals.
    """
    rng = np.random.default_rng(seed)
    f_land, f_dep = _low_degree_field(rng), _low_degree_field(rng)

    def land(p):
        v = f_land(p)
        return v < np.quantile(v, land_frac)

    def depth(p):
        v = f_dep(p)
        v = (v - v.min()) / max(v.max() - v.min(), 1e-300)
        return dmin + (dmax - dmin) * v

    key = (level, seed, land_frac, dmin, dmax)
    m = _SPHERE_MESHES.get(key)
    if m is None:
        m = _SPHERE_MESHES[key] = _mesh.geodesic_sphere(level, land=land, depth=depth)
    R = float(np.linalg.norm(m.xCell[0]))
    lat = m.latCell
    s = np.full(L, 1.0 / L)
    zfrac = -(np.cumsum(s) - 0.5 * s)            # 0 at the surface, -1 at the bottom
    dz = m.bottomDepth[:, None] * zfrac[None, :]  # mid-layer depth (negative), m
    zeta = np.zeros(m.nCells)
    if perturb:
        c0 = m.xCell[rng.integers(m.nCells)] / R
        zeta = 0.5 * np.exp(-((1.0 - m.xCell @ c0 / R) / 0.02))
    h = (m.bottomDepth + zeta)[:, None] * s[None, :]
    T = 5.0 + 20.0 * (np.cos(lat) ** 2)[:, None] * np.exp(dz / 800.0)
    S = 34.0 + 2.0 * (np.cos(lat) ** 2)[:, None] * np.exp(dz / 1500.0)
    tr = np.stack([T, S][:nTracers])
    u = np.zeros((m.nEdges, L))
    xe = m.xEdge / R
    late = np.arcsin(np.clip(xe[:, 2], -1, 1))
    east = np.cross(np.array([0.0, 0.0, 1.0]), xe)
    east /= np.maximum(np.linalg.norm(east, axis=1, keepdims=True), 1e-300)
    a1, a2 = rng.uniform(0.5, 1.0, 2)
    prof = -a1 * np.cos(3.0 * late) + a2 * np.cos(5.0 * late) * np.cos(late)
    tau = wind * prof / np.abs(prof).max() * np.sum(east * m.normalEdge, axis=1)
    p = dict(PHYS)
    p.update(nTracers=nTracers, recon="consistent", nu_h=1.0e3, nu_v=1e-4, kappa_h=0.0,
             kappa_v=0.0, c_drag=1e-3, windStress=tau)
    p.update(params)
    return m, L, p, (u, h, tr)


WORKLOADS = {
    "channel_10km": dict(nx=16, ny=32, dc=10e3, L=10, depth=1000.0, f0=1.2e-4, beta=0.0,
                         order=2, dt=300.0, M=20, steps=10),
    "channel_1km": dict(nx=160, ny=578, dc=1e3, L=20, depth=1000.0, f0=1.2e-4, beta=1.6e-11,
                        order=3, dt=60.0, M=30, steps=200),
    "sphere_l7": dict(kind="sphere", level=7, L=60, order=3, dt=600.0, M=40, steps=144),
    "sphere_l4": dict(kind="sphere", level=4, L=12, order=3, dt=600.0, M=40, steps=10),
}


def workload(name, *, seed=0, perturb=False, **override):
    """Build a named workload: returns (mesh, L, params, state, run)."""
    w = dict(WORKLOADS[name])
    w.update(override)
    run = {k: w.pop(k) for k in ("order", "dt", "M", "steps")}
    partial = w.pop("partial", False)
    if w.pop("kind", "channel") == "sphere":
        m, L, p, st = sphere_case(w.pop("level"), w.pop("L"), seed=seed, perturb=perturb, **w)
    else:
        m, L, p, st = channel_case(w.pop("nx"), w.pop("ny"), w.pop("dc"), w.pop("L"), seed=seed,
                                   perturb=perturb, **w)
    if partial:
        # partial bottom cells: the state remapped to each column's own layers;
        # the layer data travel in params (maxLevelCell, restThickness)
        u, h, tr = st
        K, rest = partial_bottom(m, L)
        H = m.bottomDepth
        h = rest * (h.sum(1) / H)[:, None]
        act = np.arange(L)[None, :] < K[:, None]
        tr = np.where(act[None], tr, 0.0)
        Ke = np.minimum(K[m.cellsOnEdge[:, 0]], K[m.cellsOnEdge[:, 1]])
        u = np.where(np.arange(L)[None, :] < Ke[:, None], u, 0.0)
        st = (u, h, tr)
        p = dict(p, maxLevelCell=K, restThickness=rest)
    return m, L, p, st, run


# ----------------------------------------------------------------------------
# ensembles and request streams (specifications only; meshes and states are
# built from them with the generators above)
# ----------------------------------------------------------------------------
def planar_shape(n_cells, rng):
    """(nx, ny) of a channel with about n_cells ocean cells, ny even."""
    aspect = rng.uniform(0.5, 2.0)
    nx = max(8, int(round(math.sqrt(n_cells * aspect))))
    ny = max(8, int(round(n_cells / nx)))
    ny += ny % 2
    return nx, ny


def ensemble_members(n=64, seed=0, size_classes=8, cells=(2000, 60000), layers=(10, 40),
                     substeps=(20, 40), steps=100):
    """Batched-ensemble members: planar channels with seeded sizes (log-uniform
    in `cells`, drawn once per size class and shared by the members of the
    class), seeded layer counts, fronts, dt and sub-step counts; SSPRK3-SE,
    mixed precision, `steps` large steps each."""
    rng = np.random.default_rng(seed)
    shapes = [planar_shape(int(math.exp(rng.uniform(math.log(cells[0]), math.log(cells[1])))), rng)
              for _ in range(size_classes)]
    out = []
    for k in range(n):
        nx, ny = shapes[k % size_classes]
        out.append(dict(kind="planar", nx=nx, ny=ny, dc=5e3,
                        L=int(rng.integers(layers[0], layers[1] + 1)),
                        order=3, dt=float(rng.choice([90.0, 120.0, 150.0])),
                        M=int(rng.integers(substeps[0], substeps[1] + 1)), steps=steps,
                        seed=int(rng.integers(1 << 30))))
    return out


def serving_requests(n=32, seed=0, rate=20.0, cells=(2000, 60000), levels=(5, 7),
                     layers=(10, 60), horizon=(50, 500)):
    """A Poisson stream of solves: arrival times with mean rate `rate` per
    second, each an SSPRK2-SE or SSPRK3-SE solve on a planar channel (cells
    log-uniform in `cells`) or a geodesic sphere of a level in `levels`, with
    a seeded layer count and horizon."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n):
        t += float(rng.exponential(1.0 / rate))
        order = int(rng.choice([2, 3]))
        L = int(rng.integers(layers[0], layers[1] + 1))
        steps = int(rng.integers(horizon[0], horizon[1] + 1))
        if rng.random() < 0.5:
            nx, ny = planar_shape(int(math.exp(rng.uniform(math.log(cells[0]),
                                                           math.log(cells[1])))), rng)
            spec = dict(kind="planar", nx=nx, ny=ny, dc=5e3, dt=120.0, M=20)
        else:
            lev = int(rng.integers(levels[0], levels[1] + 1))
            spec = dict(kind="sphere", level=lev, dt=1200.0 / 2 ** (lev - 5), M=40)
        spec.update(L=L, order=order, steps=steps, arrival=t, seed=int(rng.integers(1 << 30)))
        out.append(spec)
    return out


def build_spec(spec):
    """(mesh, L, params, (u, h, tr)) for an ensemble member or request spec."""
    if spec["kind"] == "sphere":
        return sphere_case(spec["level"], spec["L"], seed=spec["seed"] % 7, perturb=True)
    return channel_case(spec["nx"], spec["ny"], spec["dc"], spec["L"], beta=1.6e-11,
                        seed=spec["seed"], perturb=True)


def partial_bottom(m, L, min_frac=0.25):
    """Partial bottom cells for the depths of mesh m on a uniform reference
    grid of L layers reaching the deepest cell: cell i keeps the K_i layers
    that reach its depth, the last one cut to the depth (merged into the layer
    above when thinner than min_frac of a layer).  Returns (maxLevelCell [C]
    int32, restThickness [C, L], 0 below maxLevelCell)."""
    H = np.asarray(m.bottomDepth, dtype=np.float64)
    dz = H.max() / L
    K = np.minimum(np.ceil(H / dz - 1e-12).astype(np.int64), L)
    K = np.maximum(K, 1)
    rest = np.zeros((m.nCells, L))
    for i in range(m.nCells):
        k = int(K[i])
        bottom = H[i] - (k - 1) * dz
        if k > 1 and bottom < min_frac * dz:
            k -= 1
            bottom += dz
        K[i] = k
        rest[i, :k - 1] = dz
        rest[i, k - 1] = H[i] - (k - 1) * dz
    return K.astype(np.int32), rest


def partial_case(nx, ny, dc, L, *, depth, seed=0, perturb=True, nTracers=1, **params):
    """A channel over the bathymetry `depth(x, y)` with partial bottom cells:
    (mesh, L, params, (u, h, tr), (maxLevelCell, restThickness)).  The state is
    the channel state remapped to z-star layers proportional to the rest
    thickness (h_k = rest_k (H + zeta) / H); inactive layers hold h = 0, u = 0
    and tracer 0."""
    m, L, p, (u, h, tr) = channel_case(nx, ny, dc, L, depth=depth, seed=seed, perturb=perturb,
                                       nTracers=nTracers, **params)
    K, rest = partial_bottom(m, L)
    H = m.bottomDepth
    zeta = h.sum(1) - H
    h = rest * ((H + zeta) / H)[:, None]
    active = np.arange(L)[None, :] < K[:, None]
    tr = np.where(active[None], tr, 0.0)
    Ke = np.minimum(K[m.cellsOnEdge[:, 0]], K[m.cellsOnEdge[:, 1]])
    u = np.where(np.arange(L)[None, :] < Ke[:, None], u, 0.0)
    return m, L, p, (u, h, tr), (K, rest)
