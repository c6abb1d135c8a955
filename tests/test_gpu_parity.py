"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances: FP64 path relative L2 <= 1e-11 per field (the bar stated for the
FP64 form); mixed path per-field bounds stated below, volume conserved to
1e-13 relative.
"""
import numpy as np
import pytest

import oracle
from paper_2105_13484_gb300 import binding, build, inputs
from paper_2105_13484_gb300 import mesh as meshgen

pytestmark = pytest.mark.gpu

TOL64 = 1e-11


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    binding.load()


def _gpu(m, L, p, u, h, tr, precision="fp64", rest_frac=None):
    dm = binding.Mesh(m, L, rest_frac)
    st = binding.State(dm, p, precision)
    st.load_state(u, h, tr)
    return dm, st


def _compare(gpu, ref, tol, names=("u", "h", "tr")):
    errs = {n: rel(a, b) for n, a, b in zip(names, gpu, ref)}
    for n, e in errs.items():
        assert e < tol, errs
    return errs


def test_alg1_baroclinic_feuler(channel_small):
    m, L, p, (u, h, tr), run = channel_small
    o = oracle.Oracle(m, L, p)
    ubar, ut = o.split(u, h)
    zeta = o.ssh(h)
    ut1, G = o.baroclinic_feuler(u, ut, zeta, h, tr, run["dt"])
    dm, st = _gpu(m, L, p, u, h, tr)
    st.set("ubar", ubar)
    st.set("utilde", ut)
    st.baroclinic_feuler(run["dt"])
    assert rel(st.get("utilde"), ut1) < TOL64
    assert rel(st.get("G"), G) < TOL64


@pytest.mark.parametrize("order", [2, 3])
def test_alg34_barotropic_substep(order, channel_small):
    m, L, p, (u, h, tr), run = channel_small
    o = oracle.Oracle(m, L, p)
    ubar, _ = o.split(u, h)
    zeta = o.ssh(h)
    G = 1e-6 * np.sin(np.arange(m.nEdges) * 0.37)
    u1, Fz, z1 = o.barotropic_substep(order, ubar, zeta, G, run["dt"], run["M"])
    dm, st = _gpu(m, L, p, u, h, tr)
    st.set("ubar", ubar)
    st.set("G", G)
    st.barotropic_substep(order, run["dt"], run["M"])
    assert rel(st.get("ubar"), u1) < TOL64
    assert rel(st.get("Fzeta"), Fz) < TOL64
    assert np.abs(st.get("zeta_sub") - z1).max() < 1e-11 * (1 + np.abs(z1).max())


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("recon", ["off", "paper", "consistent"])
def test_full_step_channel_10km(order, recon):
    """The 16 x 32 channel workload, 10 steps, every reconciliation mode.

    SSPRK2-SE without reconciliation or with the printed F^h is unstable at
    the workload's dt = 300 s, M = 20 (both the oracle and the GPU grow to
    NaN, as the paper's N/A entries do); those modes run at dt = 100 s."""
    m, L, p, (u, h, tr), run = inputs.workload("channel_10km", perturb=True)
    p = dict(p, recon=recon)
    if order == 2 and recon == "consistent":
        dt, M, n = run["dt"], run["M"], run["steps"]
    elif order == 2:
        dt, M, n = 100.0, 10, 10
    else:
        dt, M, n = 150.0, 10, 10
    o = oracle.Oracle(m, L, p)
    ref = o.step(order, dt, M, u, h, tr, n_steps=n)
    dm, st = _gpu(m, L, p, u, h, tr)
    st.step(order, dt, M, n)
    _compare(st.read_state(), ref, TOL64)
    zeta = st.get("zeta")
    assert np.abs(zeta - (ref[1].sum(1) - m.bottomDepth)).max() < 1e-9


def test_full_step_all_terms():
    """Two tracers, tracer diffusion, bathymetry, beta plane, wind stress,
    bottom drag, a ragged mesh size (13 x 18 cells) and uneven rest layers."""
    def depth(x, y):
        return 900.0 - 300.0 * np.exp(-((x - 60e3) ** 2 + (y - 70e3) ** 2) / (30e3) ** 2)
    m, L, p, (u, h, tr) = inputs.channel_case(13, 18, 9e3, 7, depth=depth, beta=2e-11,
                                              perturb=True, nTracers=2, kappa_h=20.0,
                                              kappa_v=1e-4, c_drag=3e-3, nu_h=50.0,
                                              nu_v=1e-3)
    rf = np.array([0.05, 0.08, 0.1, 0.14, 0.18, 0.2, 0.25])
    H = m.bottomDepth
    h = (H + (h.sum(1) - H))[:, None] * rf[None, :]
    p["windStress"] = 0.1 * np.cos(m.xEdge[:, 1] / 40e3) * m.normalEdge[:, 0]
    o = oracle.Oracle(m, L, p, rest_frac=rf)
    ref = o.step(3, 200.0, 12, u, h, tr, n_steps=4)
    dm, st = _gpu(m, L, p, u, h, tr, rest_frac=rf)
    st.step(3, 200.0, 12, 4)
    _compare(st.read_state(), ref, TOL64)


@pytest.mark.parametrize("L", [1, 64])
def test_layer_count_extremes(L):
    m, _, p, (u, h, tr) = inputs.channel_case(8, 10, 10e3, L, perturb=True)
    o = oracle.Oracle(m, L, p)
    ref = o.step(2, 200.0, 8, u, h, tr, n_steps=3)
    dm, st = _gpu(m, L, p, u, h, tr)
    st.step(2, 200.0, 8, 3)
    _compare(st.read_state(), ref, TOL64)


def test_mixed_precision_bounds_and_volume():
    m, L, p, (u, h, tr), run = inputs.workload("channel_10km", perturb=True)
    o = oracle.Oracle(m, L, p)
    ref = o.step(3, 150.0, 10, u, h, tr, n_steps=10)
    dm, st = _gpu(m, L, p, u, h, tr, "mixed")
    d0 = st.diagnostics()
    st.step(3, 150.0, 10, 10)
    d1 = st.diagnostics()
    gu, gh, gt = st.read_state()
    assert rel(gu, ref[0]) < 1e-4
    assert rel(gh, ref[1]) < 1e-9
    assert rel(gt, ref[2]) < 1e-6
    assert abs(d1["volume"] - d0["volume"]) / d0["volume"] < 1e-13


def test_diagnostics_and_conservation_fp64(channel_small):
    m, L, p, (u, h, tr), run = channel_small
    dm, st = _gpu(m, L, p, u, h, tr)
    d0 = st.diagnostics()
    A = m.areaCell
    assert abs(d0["volume"] - A @ h.sum(1)) / d0["volume"] < 1e-14
    assert abs(d0["tracer_content"][0] - A @ (h * tr[0]).sum(1)) / d0["tracer_content"][0] < 1e-14
    st.step(3, 150.0, 10, 5)
    d1 = st.diagnostics()
    assert abs(d1["volume"] - d0["volume"]) / d0["volume"] < 1e-13
    assert abs(d1["tracer_content"][0] - d0["tracer_content"][0]) / d0["tracer_content"][0] < 1e-13
    assert d1["step"] == 5 and not d1["nonfinite"]


def test_invalid_arguments_on_device(channel_small):
    m, L, p, (u, h, tr), run = channel_small
    dm, st = _gpu(m, L, p, u, h, tr)
    for args in ((4, 100.0, 10, 1), (3, -1.0, 10, 1), (3, 100.0, 0, 1), (2, float("nan"), 5, 1)):
        with pytest.raises(binding.SSEError) as ei:
            st.step(*args)
        assert ei.value.code == -1
    with pytest.raises(binding.SSEError):
        st.set("tracer1", tr[0])      # nTracers = 1
    # the state is still usable after rejected calls
    st.step(2, 100.0, 5, 1)
    assert not st.diagnostics()["nonfinite"]


@pytest.mark.slow
def test_channel_1km_full_size_two_steps():
    """The 92,480-cell, 20-layer workload: two SSPRK3-SE steps, whole fields."""
    m, L, p, (u, h, tr), run = inputs.workload("channel_1km", perturb=True)
    o = oracle.Oracle(m, L, p)
    ref = o.step(run["order"], run["dt"], run["M"], u, h, tr, n_steps=2)
    dm, st = _gpu(m, L, p, u, h, tr)
    st.step(run["order"], run["dt"], run["M"], 2)
    _compare(st.read_state(), ref, TOL64)


@pytest.mark.parametrize("precision,order", [("mixed", 3), ("mixed", 2), ("fp64", 3)])
def test_tiled_subcycle_matches_global_kernel(precision, order, monkeypatch):
    """The shared-memory tiled sub-cycle (halo of 3 rings, one exchange per
    sub-step) against the global-memory one on the 92,480-cell channel (the
    mixed form uses tiles there) and on the 16 x 32 channel (FP64 tiles)."""
    name = "channel_1km" if precision == "mixed" else "channel_10km"
    m, L, p, (u, h, tr), run = inputs.workload(name, perturb=True)
    rng = np.random.default_rng(3)
    ubar = 0.05 * rng.standard_normal(m.nEdges)
    G = 1e-6 * rng.standard_normal(m.nEdges)
    out = {}
    for kern in ("global", "tiled"):
        if kern == "global":
            monkeypatch.setenv("SSE_BTR_KERNEL", "global")
        else:
            monkeypatch.delenv("SSE_BTR_KERNEL", raising=False)
        dm, st = _gpu(m, L, p, u, h, tr, precision)
        st.set("ubar", ubar)
        st.set("G", G)
        st.barotropic_substep(order, run["dt"], run["M"])
        out[kern] = (st.get("ubar"), st.get("Fzeta"), st.get("zeta_sub"))
        st.close()
        dm.close()
    tol = 1e-5 if precision == "mixed" else 1e-13
    for a, b in zip(out["tiled"], out["global"]):
        assert rel(a, b) < tol


@pytest.mark.parametrize("order", [3, 2])
def test_tiled_subcycle_tensor_memory_keeps_the_bits(order, monkeypatch):
    """The FP32 tiled sub-cycle with each thread's edge coefficients and
    edgesOnEdge offsets held in tensor memory (the 1024-thread patches of the
    92,480-cell channel) against the same sub-cycle streaming them from L2
    (SSE_BTR_TMEM=0): the same arithmetic on the same values, so the same
    bits, for the sub-cycle alone and for whole steps."""
    m, L, p, (u, h, tr), run = inputs.workload("channel_1km", perturb=True, L=4)
    rng = np.random.default_rng(5)
    ubar = 0.05 * rng.standard_normal(m.nEdges)
    G = 1e-6 * rng.standard_normal(m.nEdges)
    out = {}
    for tmem in (True, False):
        if tmem:
            monkeypatch.delenv("SSE_BTR_TMEM", raising=False)
        else:
            monkeypatch.setenv("SSE_BTR_TMEM", "0")
        dm, st = _gpu(m, L, p, u, h, tr, "mixed")
        assert st.subcycle_shape() == (1024, tmem)
        st.set("ubar", ubar)
        st.set("G", G)
        st.barotropic_substep(order, run["dt"], run["M"])
        res = [st.get("ubar"), st.get("Fzeta"), st.get("zeta_sub")]
        st.load_state(u, h, tr)
        st.step(order, run["dt"], run["M"], 2)
        res += list(st.read_state())
        out[tmem] = res
        st.close()
        dm.close()
    for a, b in zip(out[True], out[False]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("order", [2, 3])
def test_full_step_sphere(order):
    """Icosahedral sphere at level 4 with ~30 % land, bathymetry 100-5000 m,
    12 layers, T and S, wind stress, pentagons: 3 steps, FP64."""
    m, L, p, (u, h, tr), run = inputs.workload("sphere_l4", perturb=True)
    o = oracle.Oracle(m, L, p)
    ref = o.step(order, run["dt"], run["M"], u, h, tr, n_steps=3)
    dm, st = _gpu(m, L, p, u, h, tr)
    st.step(order, run["dt"], run["M"], 3)
    _compare(st.read_state(), ref, TOL64)


def test_mixed_precision_sphere():
    m, L, p, (u, h, tr), run = inputs.workload("sphere_l4", perturb=True)
    o = oracle.Oracle(m, L, p)
    ref = o.step(3, run["dt"], run["M"], u, h, tr, n_steps=6)
    dm, st = _gpu(m, L, p, u, h, tr, "mixed")
    d0 = st.diagnostics()
    st.step(3, run["dt"], run["M"], 6)
    d1 = st.diagnostics()
    gu, gh, gt = st.read_state()
    # the barotropic pair (ubar, zeta) is advanced in FP32 in the mixed form, so
    # the SSH carries the velocity's relative error; under z-star every layer
    # thickness is s_k (H + zeta), so h follows zeta
    H = m.bottomDepth
    errs = {"u": rel(gu, ref[0]), "zeta": rel(gh.sum(1) - H, ref[1].sum(1) - H),
            "T": rel(gt[0], ref[2][0]), "S": rel(gt[1], ref[2][1])}
    assert errs["u"] < 1e-4 and errs["zeta"] < 1e-4, errs
    assert errs["T"] < 1e-6 and errs["S"] < 1e-6, errs
    assert np.abs(gh - (gh.sum(1, keepdims=True) / L)).max() < 1e-10 * H.max()
    assert abs(d1["volume"] - d0["volume"]) / d0["volume"] < 1e-13


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_tiled_subcycle_sphere(precision, monkeypatch):
    """Tiled against global sub-cycle on the level-7 sphere (mixed: patches of
    up to 3 owned entries per thread) and the level-4 sphere (FP64)."""
    name = "sphere_l7" if precision == "mixed" else "sphere_l4"
    m, L, p, (u, h, tr), run = inputs.workload(name, perturb=True, L=4)
    rng = np.random.default_rng(4)
    ubar = 0.05 * rng.standard_normal(m.nEdges)
    G = 1e-6 * rng.standard_normal(m.nEdges)
    out = {}
    for kern in ("global", "tiled"):
        if kern == "global":
            monkeypatch.setenv("SSE_BTR_KERNEL", "global")
        else:
            monkeypatch.delenv("SSE_BTR_KERNEL", raising=False)
        dm, st = _gpu(m, L, p, u, h, tr, precision)
        st.set("ubar", ubar)
        st.set("G", G)
        st.barotropic_substep(3, run["dt"], run["M"])
        out[kern] = (st.get("ubar"), st.get("Fzeta"), st.get("zeta_sub"))
        st.close()
        dm.close()
    tol = 1e-5 if precision == "mixed" else 1e-13
    for a, b in zip(out["tiled"], out["global"]):
        assert rel(a, b) < tol


def _pgf_rounding(m, p, h, tr, edge_layers=None):
    """L2 norm of the rounding of the layer pressure gradient as the oracle
    writes it, (grad p + g rho_e grad z_mid) / rho0: two terms of size
    g |grad z| that cancel over bathymetry.  Estimated against the same
    quantity in anomaly form, (rho_ref/rho0) g grad zeta + (grad p' +
    g rho'_e grad z) / rho0, whose terms are ~300 times smaller."""
    g, rho0, rref = p["g"], p["rho0"], p["eos_rho_ref"]
    rho = rref - p["eos_alpha"] * (tr[0] - p["eos_T_ref"]) + p["eos_beta"] * (tr[1] - p["eos_S_ref"])
    c1, c2 = m.cellsOnEdge[:, 0], m.cellsOnEdge[:, 1]

    def grad(x):
        return (x[c2] - x[c1]) / m.dcEdge[:, None]

    def pres(r):
        rh = r * h
        return g * (np.cumsum(rh, 1) - 0.5 * rh)
    zmid = -m.bottomDepth[:, None] + np.cumsum(h[:, ::-1], 1)[:, ::-1] - 0.5 * h
    zeta = (h.sum(1) - m.bottomDepth)[:, None]
    full = (grad(pres(rho)) + g * 0.5 * (rho[c1] + rho[c2]) * grad(zmid)) / rho0
    ra = rho - rref
    anom = rref / rho0 * g * grad(zeta) + (grad(pres(ra)) + g * 0.5 * (ra[c1] + ra[c2]) * grad(zmid)) / rho0
    if edge_layers is not None:      # only the layers the edges have
        full, anom = full * edge_layers, anom * edge_layers
    return float(np.linalg.norm(full - anom))


@pytest.mark.slow
def test_sphere_l7_full_size_one_step():
    """The level-7 sphere, 60 layers, one SSPRK3-SE step, whole fields, FP64.

    h and the tracers match to 1e-11.  For u the bar is the oracle's own
    rounding: over 100-5000 m bathymetry its full-form pressure gradient
    rounds at ~1e-16 m s^-2 while u after one step is only ~5e-4 m s^-1, so
    the comparison allows twice the PGF rounding integrated over the three
    stages of the step (the CUDA path uses the anomaly form)."""
    m, L, p, (u, h, tr), run = inputs.workload("sphere_l7", perturb=True)
    o = oracle.Oracle(m, L, p)
    ref = o.step(run["order"], run["dt"], run["M"], u, h, tr, n_steps=1)
    dm, st = _gpu(m, L, p, u, h, tr)
    st.step(run["order"], run["dt"], run["M"], 1)
    gu, gh, gt = st.read_state()
    assert rel(gh, ref[1]) < TOL64 and rel(gt, ref[2]) < TOL64
    bound = 2.0 * 3 * run["dt"] * _pgf_rounding(m, p, ref[1], ref[2])
    assert np.linalg.norm(gu - ref[0]) < bound, (np.linalg.norm(gu - ref[0]), bound)
    assert rel(gu, ref[0]) < 1e-8


def _vmix_case():
    # 10 m layers and nu_v = 0.5: nu_v dt / dz^2 = 1.5, beyond explicit stability
    return inputs.channel_case(10, 12, 10e3, 10, depth=100.0, perturb=True, nTracers=2,
                               nu_v=0.5, c_drag=2e-3, vmix=True)


def test_alg2_baroclinic_feuler_mixing():
    m, L, p, (u, h, tr) = _vmix_case()
    p["windStress"] = 0.1 * np.cos(m.xEdge[:, 1] / 30e3) * m.normalEdge[:, 0]
    o = oracle.Oracle(m, L, p)
    ubar, ut = o.split(u, h)
    zeta = o.ssh(h)
    ut1, G = o.baroclinic_feuler_mixing(u, ut, ubar, zeta, h, tr, 300.0)
    dm, st = _gpu(m, L, p, u, h, tr)
    st.set("ubar", ubar)
    st.set("utilde", ut)
    st.baroclinic_feuler(300.0)
    assert rel(st.get("utilde"), ut1) < TOL64
    assert rel(st.get("G"), G) < TOL64


@pytest.mark.parametrize("order", [2, 3])
def test_full_step_vertical_mixing(order):
    m, L, p, (u, h, tr) = _vmix_case()
    p["windStress"] = 0.1 * np.cos(m.xEdge[:, 1] / 30e3) * m.normalEdge[:, 0]
    o = oracle.Oracle(m, L, p)
    ref = o.step(order, 300.0, 10, u, h, tr, n_steps=5)
    dm, st = _gpu(m, L, p, u, h, tr)
    st.step(order, 300.0, 10, 5)
    _compare(st.read_state(), ref, TOL64)
    dm, st = _gpu(m, L, p, u, h, tr, "mixed")
    st.step(order, 300.0, 10, 5)
    gu, gh, gt = st.read_state()
    assert rel(gu, ref[0]) < 1e-4 and rel(gt, ref[2]) < 1e-6


@pytest.mark.parametrize("order", [2, 3])
def test_full_step_biharmonic_viscosity(order):
    """-nu_4 del^4 u (with Laplacian viscosity and walls) on a 12 x 14 channel."""
    m, L, p, (u, h, tr) = inputs.channel_case(12, 14, 10e3, 6, perturb=True, beta=2e-11,
                                              nu_h=20.0, nu_4=2e10)
    o = oracle.Oracle(m, L, p)
    ref = o.step(order, 200.0, 10, u, h, tr, n_steps=4)
    ref0 = oracle.Oracle(m, L, dict(p, nu_4=0.0)).step(order, 200.0, 10, u, h, tr, n_steps=4)
    assert rel(ref[0], ref0[0]) > 1e-4          # the term matters at this nu_4
    dm, st = _gpu(m, L, p, u, h, tr)
    assert st.kernels_per_step(order) == (17 if order == 2 else 25)   # + 1 per stage
    st.step(order, 200.0, 10, 4)
    _compare(st.read_state(), ref, TOL64)
    dm, st = _gpu(m, L, p, u, h, tr, "mixed")
    st.step(order, 200.0, 10, 4)
    gu, gh, gt = st.read_state()
    assert rel(gu, ref[0]) < 1e-4 and rel(gt, ref[2]) < 1e-6


def _partial_case(vmix=False):
    def depth(x, y):
        return 200.0 + 700.0 * (y / y.max()) ** 1.5 + 80.0 * np.sin(x / 2e4)
    m, L, p, st, (K, rest) = inputs.partial_case(12, 14, 10e3, 8, depth=depth, nTracers=2,
                                                 kappa_h=10.0, kappa_v=1e-4, nu_4=1e10,
                                                 c_drag=2e-3, vmix=vmix)
    p["windStress"] = 0.1 * np.cos(m.xEdge[:, 1] / 30e3) * m.normalEdge[:, 0]
    return m, L, p, st, K, rest


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("vmix", [False, True])
def test_full_step_partial_bottom_cells(order, vmix):
    """Columns of 1-8 layers with cut bottom layers, every term on (T and S,
    diffusion, wind, drag, Laplacian and biharmonic viscosity), Algorithm 1
    or 2: FP64 parity, mixed bounds, missing layers read back as 0."""
    m, L, p, (u, h, tr), K, rest = _partial_case(vmix)
    o = oracle.Oracle(m, L, p, max_level=K, rest_thickness=rest)
    ref = o.step(order, 200.0, 10, u, h, tr, n_steps=4)
    dm = binding.Mesh(m, L, max_level=K, rest_thickness=rest)
    st = binding.State(dm, p, "fp64")
    st.load_state(u, h, tr)
    st.step(order, 200.0, 10, 4)
    got = st.read_state()
    _compare(got, ref, TOL64)
    act = np.arange(L)[None, :] < K[:, None]
    Ke = np.minimum(K[m.cellsOnEdge[:, 0]], K[m.cellsOnEdge[:, 1]])
    assert np.abs(got[1][~act]).max() == 0.0 and np.abs(got[2][:, ~act]).max() == 0.0
    assert np.abs(got[0][np.arange(L)[None, :] >= Ke[:, None]]).max() == 0.0
    st = binding.State(dm, p, "mixed")
    st.load_state(u, h, tr)
    d0 = st.diagnostics()
    st.step(order, 200.0, 10, 4)
    d1 = st.diagnostics()
    gu, gh, gt = st.read_state()
    assert rel(gu, ref[0]) < 1e-4 and rel(gt, ref[2]) < 1e-6
    assert abs(d1["volume"] - d0["volume"]) / d0["volume"] < 1e-13
    assert d1["min_thickness"] > 0.0


def test_partial_bottom_sphere_fp64():
    """The level-4 sphere (100-5000 m) on 20 reference layers with partial
    bottom cells: 2 SSPRK3-SE steps, FP64."""
    m, L, p, (u, h, tr), run = inputs.workload("sphere_l4", perturb=True, L=20)
    K, rest = inputs.partial_bottom(m, L)
    H = m.bottomDepth
    h = rest * (h.sum(1) / H)[:, None]
    act = np.arange(L)[None, :] < K[:, None]
    tr = np.where(act[None], tr, 0.0)
    o = oracle.Oracle(m, L, p, max_level=K, rest_thickness=rest)
    ref = o.step(3, run["dt"], run["M"], u, h, tr, n_steps=2)
    dm = binding.Mesh(m, L, max_level=K, rest_thickness=rest)
    st = binding.State(dm, p, "fp64")
    st.load_state(u, h, tr)
    st.step(3, run["dt"], run["M"], 2)
    gu, gh, gt = st.read_state()
    assert rel(gh, ref[1]) < TOL64 and rel(gt, ref[2]) < TOL64
    # u against the oracle's own pressure-gradient rounding over bathymetry
    Ke = np.minimum(K[m.cellsOnEdge[:, 0]], K[m.cellsOnEdge[:, 1]])
    me = (np.arange(L)[None, :] < Ke[:, None]).astype(float)
    bound = 2.0 * 3 * 2 * run["dt"] * _pgf_rounding(m, p, ref[1], ref[2], me)
    assert np.linalg.norm(gu - ref[0]) < bound, (np.linalg.norm(gu - ref[0]), bound)


@pytest.mark.parametrize("order", [2, 3])
def test_gpu_temporal_convergence_fp64(order):
    """The GPU path's own dt-refinement sweep (M fixed): the paper's relative
    l2 error of u_1 and h_1 against a run with dt/8 of the finest falls at
    rate 2, like the oracle's."""
    m, L, p, (u, h, tr) = inputs.channel_case(12, 16, 10e3, 6, perturb=True)
    dm = binding.Mesh(m, L)
    T, M = 1920.0, 8

    def solve(n):
        st = binding.State(dm, p, "fp64")
        st.load_state(u, h, tr)
        st.step(order, T / n, M, n)
        out = st.read_state()
        st.close()
        return out

    ref = solve(512)
    eu, eh = [], []
    for n in (16, 32, 64):
        r = solve(n)
        eu.append(rel(r[0][:, 0], ref[0][:, 0]))
        eh.append(rel(r[1][:, 0], ref[1][:, 0]))
    ru = np.log2(np.array(eu[:-1]) / np.array(eu[1:]))
    rh = np.log2(np.array(eh[:-1]) / np.array(eh[1:]))
    assert np.all(ru > 1.75) and np.all(rh > 1.75), (ru, rh)
    assert np.all(ru < 2.6) and np.all(rh < 2.6), (ru, rh)
