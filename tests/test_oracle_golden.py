"""The oracle against the coefficients the paper prints (tests/golden/
ssprk_se_weights.txt): the SSPRK2/SSPRK3 convex weights (Eqs. SSPRK2,
SSPRK3), the corrector forcings Interp_2 / Interp_3 (Eqs. force2, force3),
the accumulated-flux weights and the reconciliation factors of Sec. 3.4.
Each check rebuilds the quantity from the printed numbers and from the
oracle's separately exposed pieces (forward-Euler stages, aux records)."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2105_13484_gb300 import inputs
from paper_2105_13484_gb300 import mesh as meshgen

HERE = os.path.dirname(os.path.abspath(__file__))


def golden():
    out = {}
    with open(os.path.join(HERE, "golden", "ssprk_se_weights.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                out[k.strip()] = [float(Fraction(x)) for x in v.split()]
    return out


W = golden()


def test_golden_weights_are_convex():
    for k in ("ssprk2_final", "ssprk3_stage2", "ssprk3_final", "interp2", "interp3", "fzeta2",
              "fzeta3"):
        assert abs(sum(W[k]) - 1.0) < 1e-15 and min(W[k]) > 0


def _torus(n=8, d=5e3, H=1000.0, f0=1e-4):
    m = meshgen.planar_hex(n, n, d, periodic_y=True, f0=f0, depth=H)
    return m, oracle.Oracle(m, 1, dict(g=9.80616))


@pytest.mark.parametrize("order", [2, 3])
def test_subcycle_is_printed_ssprk_with_printed_flux_weights(order):
    """One sub-step (M = 1) equals the printed convex combination of forward-
    Euler stages, and F^zeta the printed weighted sum of the stage fluxes."""
    m, o = _torus()
    rng = np.random.default_rng(5)
    ub = 0.1 * rng.standard_normal(m.nEdges)
    z = 0.5 * rng.standard_normal(m.nCells)
    G = 1e-5 * rng.standard_normal(m.nEdges)
    dt = 30.0
    u1, F, z1 = o.barotropic_substep(order, ub, z, G, dt, 1)
    ua, za, fa = o.barotropic_fe(ub, z, G, dt)
    ubb, zb, fb = o.barotropic_fe(ua, za, G, dt)
    if order == 2:
        a, b = W["ssprk2_final"]
        ue, ze = a * ub + b * ubb, a * z + b * zb
        Fe = W["fzeta2"][0] * fa + W["fzeta2"][1] * fb
    else:
        a, b = W["ssprk3_stage2"]
        uh, zh = a * ub + b * ubb, a * z + b * zb
        uc, zc, fc = o.barotropic_fe(uh, zh, G, dt)
        a, b = W["ssprk3_final"]
        ue, ze = a * ub + b * uc, a * z + b * zc
        w = W["fzeta3"]
        Fe = w[0] * fa + w[1] * fb + w[2] * fc
    assert np.abs(u1 - ue).max() < 1e-15 * (1 + np.abs(ue).max())
    assert np.abs(z1 - ze).max() < 1e-15 * (1 + np.abs(ze).max())
    assert np.abs(F - Fe).max() < 1e-12 * np.abs(Fe).max()


@pytest.mark.parametrize("order", [2, 3])
def test_corrector_forcing_is_printed_interp(order):
    """The corrector sub-cycle of a full step is driven by Interp_2 / Interp_3
    of the stage forcings: re-running it with the printed weights on the
    aux G records reproduces its accumulated flux."""
    m, L, p, (u, h, tr), run = inputs.workload("channel_10km", perturb=True)
    o = oracle.Oracle(m, L, p)
    dt, M = 150.0, 6
    _, _, _, aux = o.step(order, dt, M, u.copy(), h.copy(), tr.copy(), aux=True)
    ubar, _ = o.split(u, h)
    zeta = o.ssh(h)
    if order == 2:
        Gi = W["interp2"][0] * aux["G0"] + W["interp2"][1] * aux["G1"]
        ref = aux["Fz2"]
    else:
        w = W["interp3"]
        Gi = w[0] * aux["G0"] + w[1] * aux["G1"] + w[2] * aux["G2"]
        ref = aux["Fz3"]
    _, F, _ = o.barotropic_substep(order, ubar, zeta, Gi, dt, M)
    assert np.abs(F - ref).max() < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("order", [2, 3])
def test_reconciliation_factors_close_the_ssh(order):
    """With the printed factors c_i (u^A = c_i D_i / sum h) and the
    already-adjusted fluxes in F^h, sum h - H after the step equals the
    corrector's own SSH; any other final factor leaves a residual."""
    m, L, p, (u, h, tr), run = inputs.workload("channel_10km", perturb=True)
    p = dict(p, recon="consistent")
    o = oracle.Oracle(m, L, p)
    dt, M = 150.0, 6
    _, h1, _, aux = o.step(order, dt, M, u.copy(), h.copy(), tr.copy(), aux=True)
    assert np.abs(o.ssh(h1) - aux["zeta_sub"]).max() < 1e-11
    # the printed factor of the last stage undoes the weight of the final
    # convex average (its deficit enters h^{n+1} scaled by that weight)
    if order == 2:
        assert W["recon2"][-1] * W["ssprk2_final"][1] == 1.0
    else:
        assert W["recon3"][-1] * W["ssprk3_final"][1] == 1.0
