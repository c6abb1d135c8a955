"""Checkpoint and resume through the C ABI.  The state between steps is
(ubar, utilde, h, tracers): saved with sse_state_get and loaded into a fresh
state with sse_state_set, it continues bit for bit like the state that never
stopped in FP64.  Saving u = ubar + utilde instead is a valid restart (each
step re-splits u), equal to rounding; so is the mixed form, whose FP32 copy
of h is rebuilt from the FP64 h on load."""
import numpy as np
import pytest

from paper_2105_13484_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def save(st):
    return {n: st.get(n) for n in ("ubar", "utilde", "h", "tracer0")}


def load(st, ck):
    st.set("h", ck["h"])
    st.set("tracer0", ck["tracer0"])
    st.set("utilde", ck["utilde"])
    st.set("ubar", ck["ubar"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_resume_continues_the_run(precision):
    m, L, p, (u, h, tr), run = inputs.workload("channel_10km", perturb=True)
    dm = binding.Mesh(m, L)
    order, dt, M = 3, run["dt"], run["M"]
    a = binding.State(dm, p, precision)
    a.load_state(u, h, tr)
    a.step(order, dt, M, 3)
    ck = save(a)
    ck_u = a.read_state()
    a.step(order, dt, M, 3)
    want = a.read_state()
    b = binding.State(dm, p, precision)
    load(b, ck)
    b.step(order, dt, M, 3)
    got = b.read_state()
    c = binding.State(dm, p, precision)   # restart from u = ubar + utilde
    c.load_state(*ck_u)
    c.step(order, dt, M, 3)
    got_u = c.read_state()
    for x, y, z, n in zip(got, want, got_u, ("u", "h", "tracers")):
        if precision == "fp64":
            assert np.array_equal(x, y), n
            assert np.linalg.norm(z - y) <= 1e-13 * np.linalg.norm(y), n
        else:
            assert np.linalg.norm(x - y) <= 1e-5 * np.linalg.norm(y), n
            assert np.linalg.norm(z - y) <= 1e-5 * np.linalg.norm(y), n
    for st in (a, b, c):
        st.close()
