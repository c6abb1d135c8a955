"""Failure path of the sub-cycle's grid barriers, exercised without a GPU
fault: a host-set stall (sse_state_inject) makes every barrier wait for one
arrival more than its grid has.  Each wait then runs out its bounded budget
(2 s), the kernel records the error in the state's error word and returns;
the host reads SSE_ERR_SYNC_TIMEOUT, the CUDA context stays usable, and the
state, once re-set, steps on bit-identically to a fresh one."""
import time

import numpy as np
import pytest

from paper_2105_13484_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

SYNC_TIMEOUT = -6


@pytest.mark.parametrize("kernel", ["tiled", "global"])
def test_barrier_timeout_is_reported_and_the_state_recovers(kernel, monkeypatch):
    if kernel == "global":
        monkeypatch.setenv("SSE_BTR_KERNEL", "global")
    else:
        monkeypatch.delenv("SSE_BTR_KERNEL", raising=False)
    m, L, p, (u, h, tr), run = inputs.workload("channel_10km", perturb=True)
    dm = binding.Mesh(m, L)
    st = binding.State(dm, p, "mixed")
    assert (st.patches() > 0) == (kernel == "tiled")
    st.load_state(u, h, tr)

    st.inject_barrier_stall(True)
    t0 = time.time()
    with pytest.raises(binding.SSEError) as e:
        st.step(run["order"], run["dt"], run["M"], 1)
        st.read_state()
    assert e.value.code == SYNC_TIMEOUT
    assert time.time() - t0 < 60
    assert st.diagnostics(check=False)["rc"] == SYNC_TIMEOUT

    # the context is usable: the same state, re-set, matches a fresh one bit for bit
    st.inject_barrier_stall(False)
    st.load_state(u, h, tr)
    st.step(run["order"], run["dt"], run["M"], 2)
    got = st.read_state()
    ref = binding.State(dm, p, "mixed")
    ref.load_state(u, h, tr)
    ref.step(run["order"], run["dt"], run["M"], 2)
    want = ref.read_state()
    for a, b in zip(got, want):
        assert np.array_equal(a, b)
    assert st.diagnostics()["rc"] == 0
    st.close()
    ref.close()


def test_barrier_timeout_in_the_tensor_memory_subcycle():
    """The FP32 1024-thread sub-cycle holds its SM's tensor memory: on a
    barrier timeout every block frees it before returning, so the launches
    that follow (which allocate it again on the same SMs) run, and the state
    recovers bit for bit."""
    m, L, p, (u, h, tr), run = inputs.workload("channel_1km", perturb=True, L=4)
    dm = binding.Mesh(m, L)
    st = binding.State(dm, p, "mixed")
    assert st.subcycle_shape() == (1024, True)
    st.load_state(u, h, tr)
    st.inject_barrier_stall(True)
    with pytest.raises(binding.SSEError) as e:
        st.step(run["order"], run["dt"], run["M"], 1)
        st.read_state()
    assert e.value.code == SYNC_TIMEOUT
    st.inject_barrier_stall(False)
    st.load_state(u, h, tr)
    st.step(run["order"], run["dt"], run["M"], 2)
    got = st.read_state()
    ref = binding.State(dm, p, "mixed")
    ref.load_state(u, h, tr)
    ref.step(run["order"], run["dt"], run["M"], 2)
    for a, b in zip(got, ref.read_state()):
        assert np.array_equal(a, b)
    st.close()
    ref.close()
    dm.close()


def test_inject_rejects_unknown_hooks():
    m, L, p, _, _ = inputs.workload("channel_10km")
    st = binding.State(binding.Mesh(m, L), p, "mixed")
    lib = binding.load()
    assert lib.sse_state_inject(st.handle, 2, 1) == -1
    assert lib.sse_state_inject(st.handle, 1, 5) == -1
    st.close()
