"""Packed launches of several states (sse_step_batch): uneven meshes, layer
counts, time steps and sub-step counts advance in lock-step with one 3-D
launch per kernel and stage; each state's result equals the state stepped
alone with sse_step."""
import numpy as np
import pytest

from paper_2105_13484_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def _members(order):
    specs = [
        (inputs.workload("channel_10km", perturb=True), 300.0, 20),
        (inputs.workload("sphere_l4", perturb=True), 600.0, 40),
        ((*inputs.channel_case(24, 40, 8e3, 15, beta=1.6e-11, seed=3, perturb=True),
          dict(order=order)), 240.0, 24),
        ((*inputs.channel_case(12, 18, 12e3, 7, seed=5, perturb=True), dict(order=order)),
         360.0, 16),
    ]
    return [(w[0], w[1], w[2], w[3], dt, M) for w, dt, M in specs]


@pytest.mark.parametrize("precision,order", [("mixed", 3), ("fp64", 3), ("mixed", 2)])
def test_batched_steps_equal_steps_alone(precision, order):
    torch = pytest.importorskip("torch")
    members = _members(order)
    nsteps = 3
    meshes, alone, states = [], [], []
    for m, L, p, (u, h, tr), dt, M in members:
        dm = binding.Mesh(m, L)
        meshes.append(dm)
        a = binding.State(dm, p, precision)
        a.load_state(u, h, tr)
        a.step(order, dt, M, nsteps)
        alone.append(a.read_state())
        a.close()
    streams = [torch.cuda.Stream() for _ in members]
    for (m, L, p, (u, h, tr), dt, M), dm, s in zip(members, meshes, streams):
        st = binding.State(dm, p, precision, stream=s.cuda_stream)
        st.load_state(u, h, tr)
        states.append(st)
    main = torch.cuda.Stream()
    binding.step_batch(states, order, [x[4] for x in members], [x[5] for x in members], nsteps,
                       stream=main.cuda_stream)
    for st, ref in zip(states, alone):
        got = st.read_state()
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
        st.close()
    for dm in meshes:
        dm.close()
