"""The allocation-free sub-cycle entry point (sse_barotropic_substep_noalloc).

It serves callers that must not allocate device memory where they run the
sub-cycle (inside an allocator or memory-pool callback, or in a runtime that
reserves its device memory up front).  The test calls it through the C ABI on
caller-owned device arrays, twice in a row with different inputs (the shared
work array keeps the previous call's contents), and checks each result
against sse_barotropic_substep.  This file
is collected last so that a failure here leaves every other test run.
"""
import numpy as np
import pytest

from paper_2105_13484_gb300 import binding, build, inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-11


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_noalloc_matches_substep_twice_in_a_row():
    torch = pytest.importorskip("torch")
    build.build()
    m, L, p, (u, h, tr), run = inputs.workload("channel_10km", perturb=True)
    dm = binding.Mesh(m, L)
    st = binding.State(dm, p, "fp64")
    st.load_state(u, h, tr)
    zeta = h.sum(1) - m.bottomDepth
    rng = np.random.default_rng(11)
    dev = torch.device("cuda:0")
    for call, order in enumerate((3, 2)):
        ubar = 0.05 * rng.standard_normal(m.nEdges)
        G = 1e-6 * rng.standard_normal(m.nEdges)
        # reference: the allocating entry point on the state
        st.set("ubar", ubar)
        st.set("G", G)
        st.barotropic_substep(order, run["dt"], run["M"])
        ref_u, ref_F, ref_z = st.get("ubar"), st.get("Fzeta"), st.get("zeta_sub")
        # allocation-free: caller-owned device arrays
        d_u = torch.tensor(ubar, dtype=torch.float64, device=dev)
        d_z = torch.tensor(zeta, dtype=torch.float64, device=dev)
        d_G = torch.tensor(G, dtype=torch.float64, device=dev)
        o_u = torch.full((m.nEdges,), float("nan"), dtype=torch.float64, device=dev)
        o_F = torch.full((m.nEdges,), float("nan"), dtype=torch.float64, device=dev)
        o_z = torch.full((m.nCells,), float("nan"), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        binding.barotropic_substep_noalloc(dm, order, run["dt"], run["M"], p["g"],
                                           d_u.data_ptr(), d_z.data_ptr(), d_G.data_ptr(),
                                           o_u.data_ptr(), o_F.data_ptr(), o_z.data_ptr())
        torch.cuda.synchronize()
        got_u, got_F, got_z = (x.cpu().numpy() for x in (o_u, o_F, o_z))
        assert rel(got_u, ref_u) < TOL64, call
        assert rel(got_F, ref_F) < TOL64, call
        assert np.abs(got_z - ref_z).max() < 1e-11 * (1 + np.abs(ref_z).max()), call
    st.close()
    dm.close()
