"""sse_step with n_steps >= 2 replays pairs of large steps from a CUDA graph
captured from the same launches; it must give the same bits as stepping one
step per call, across orders, a state reset, a later wind stress (which
changes the step's kernel arguments) and profiling."""
import numpy as np
import pytest

from paper_2105_13484_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_graph_steps_equal_single_steps(precision):
    torch = pytest.importorskip("torch")
    m, L, p, (u, h, tr), run = inputs.workload("channel_10km", perturb=True)
    dm = binding.Mesh(m, L)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    a = binding.State(dm, p, precision, stream=sa.cuda_stream)   # launch by launch
    b = binding.State(dm, p, precision, stream=sb.cuda_stream)   # pairs from graphs
    rng = np.random.default_rng(5)
    wind = 0.05 * rng.standard_normal(m.nEdges)
    dt, M = run["dt"], run["M"]
    for st in (a, b):
        st.load_state(u, h, tr)

    def both(order, n):
        for _ in range(n):
            a.step(order, dt, M, 1)
        b.step(order, dt, M, n)

    both(3, 4)
    assert b.graphs() == 1 and a.graphs() == 0
    both(2, 3)            # an odd count leaves the buffers rotated
    both(3, 2)
    for st in (a, b):
        st.set("wind", wind)
    assert b.graphs() == 0   # the wind stress changed the step's kernel arguments
    both(3, 4)
    b.profile(True)       # profiling steps launch by launch
    both(3, 2)
    b.profile(False)
    both(2, 2)
    for x, y in zip(a.read_state(), b.read_state()):
        assert np.array_equal(x, y)
    # a reset state replays the cached graphs from the new initial state
    for st in (a, b):
        st.load_state(u, h, tr)
    both(3, 4)
    for x, y in zip(a.read_state(), b.read_state()):
        assert np.array_equal(x, y)
    a.close()
    b.close()


def test_no_graphs_on_the_legacy_default_stream():
    m, L, p, (u, h, tr), run = inputs.workload("channel_10km", perturb=True)
    st = binding.State(binding.Mesh(m, L), p, "mixed")   # NULL stream
    st.load_state(u, h, tr)
    st.step(run["order"], run["dt"], run["M"], 2)
    assert st.graphs() == 0
    assert st.diagnostics()["rc"] == 0
    st.close()
