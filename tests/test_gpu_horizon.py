"""Parity at each full-size workload's horizon (Sec. 3.3, SSPRK3-SE, with the
Sec. 3.4 reconciliation): the 92,480-cell channel after its 200 steps and the
level-7 sphere after its 144 steps, on the GPU through the C ABI, against the
FP64 oracle's results stored by tests/golden/make_horizon.py (a seeded sample
of each final field; the full fields are 10^7-10^8 values).

FP64 form: relative L2 error over the sampled entries <= 1e-11 for every
prognostic field (u, h, the tracers), or twice the field's spread where that
is larger: the distance the oracle's own result moves when its input
thicknesses are moved by one unit in the last place, stored with the
results.  On the sphere the SSH gradient turns an ulp of column depth into a
velocity change of order g eps H dt / dc per step while u stays O(1e-2 m/s),
so u's spread there (about 1e-10) is above 1e-11 and no FP64 evaluation
order other than the oracle's own can meet 1e-11 on it.  The SSH is
diagnosed as zeta = sum h - H: its error is h's, and relative to zeta itself
it is amplified by H/|zeta| (about 10^4 on the sphere), so it is held to
1e-13 of the depth instead.
Mixed form: the per-field bounds stated below, and volume conserved to 1e-13
relative over the whole run.  The stored digest of the inputs must match the
inputs generated here, else the comparison would be between different runs.
"""
import os
import sys

import numpy as np
import pytest

from paper_2105_13484_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_horizon  # noqa: E402

TOL64 = 1e-11
SPREAD_FACTOR = 2.0
# mixed form against the FP64 oracle at the horizon (relative L2 over the
# sampled entries), per workload and field: about 2.5 times the measured
# errors (channel: u 1.0e-5, h 9.9e-9, zeta 1.6e-5, T 3.8e-7; sphere: u
# 5.8e-5, h 3.1e-10, zeta 3.9e-6, T 4.9e-7, S 1.9e-8)
MIXED_BOUND = {
    "channel_1km": {"u": 3e-5, "h": 3e-8, "zeta": 5e-5, "tracer0": 1e-6},
    "sphere_l7": {"u": 1.5e-4, "h": 1e-9, "zeta": 1e-5, "tracer0": 1.5e-6, "tracer1": 1e-7},
}


def _run(name, precision):
    path = make_horizon.path_of(name)
    assert os.path.exists(path), f"{path} missing: run tests/golden/make_horizon.py"
    g = np.load(path)
    m, L, p, (u, h, tr), run = inputs.workload(name, perturb=True)
    digest = make_horizon.input_digest(m, L, p, (u, h, tr))
    assert str(g["digest"]) == digest, (
        "the stored oracle results were made from other inputs than this host generates "
        "(regenerate them on this platform with tests/golden/make_horizon.py)")
    assert int(g["steps"]) == run["steps"]
    dm = binding.Mesh(m, L)
    st = binding.State(dm, p, precision)
    st.load_state(u, h, tr)
    vol0 = st.diagnostics()["volume"]
    st.step(run["order"], run["dt"], run["M"], run["steps"])
    d = st.diagnostics()
    gu, gh, gt = st.read_state()
    st.close()
    dm.close()
    got = {"u": gu.ravel(), "h": gh.ravel(), "zeta": gh.sum(1) - m.bottomDepth}
    for k in range(gt.shape[0]):
        got[f"tracer{k}"] = gt[k].ravel()
    err = {}
    for f, x in got.items():
        idx, val = g[f + "_idx"], g[f + "_val"]
        err[f] = float(np.linalg.norm(x[idx] - val) / np.linalg.norm(val))
        if f == "zeta":   # relative to the depth
            err["zeta_of_depth"] = float(np.linalg.norm(x[idx] - val) /
                                         np.linalg.norm(m.bottomDepth[idx]))
    spread = {f: float(g[f + "_spread"]) for f in got}
    print(name, precision, "error", err, "oracle spread", spread)
    return err, abs(d["volume"] - vol0) / vol0, spread


@pytest.mark.parametrize("name", ["channel_1km", "sphere_l7"])
def test_fp64_matches_oracle_at_horizon(name):
    err, dvol, spread = _run(name, "fp64")
    for f in ("u", "h", "tracer0", "tracer1"):
        if f in err:
            bound = max(TOL64, SPREAD_FACTOR * spread[f])
            assert err[f] <= bound, (f, bound, err, spread)
    assert err["zeta_of_depth"] <= 1e-13, err
    assert dvol < 1e-13


@pytest.mark.parametrize("name", ["channel_1km", "sphere_l7"])
def test_mixed_bounds_at_horizon(name):
    err, dvol, _ = _run(name, "mixed")
    for f, b in MIXED_BOUND[name].items():
        if f in err:
            assert err[f] <= b, (f, err)
    assert dvol < 1e-13
