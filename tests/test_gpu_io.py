"""Host transfers of the state: page-locked host buffers are read and written
by the conversion kernels directly, any other host buffer goes through the
device staging array; both must give the same bits."""
import numpy as np
import pytest

from paper_2105_13484_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_pinned_and_pageable_host_buffers_agree(precision):
    torch = pytest.importorskip("torch")
    m, L, p, (u, h, tr), run = inputs.workload("channel_10km", perturb=True)
    dm = binding.Mesh(m, L)
    a = binding.State(dm, p, precision)
    b = binding.State(dm, p, precision)
    fields = [("u", u), ("h", h), ("tracer0", tr[0])]
    pinned = {n: torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for n, x in fields}
    for n, x in fields:
        a.set(n, x)                                   # pageable: staged
        b.set_ptr(n, pinned[n].data_ptr())            # page-locked: direct
    for st in (a, b):
        st.step(run["order"], run["dt"], run["M"], 2)
    for n in ("u", "h", "tracer0", "zeta", "Fzeta"):
        want = a.get(n)
        out = torch.empty(want.size, dtype=torch.float64).pin_memory()
        b.get_ptr(n, out.data_ptr())
        assert np.array_equal(out.numpy().reshape(want.shape), want), n
    a.close()
    b.close()
