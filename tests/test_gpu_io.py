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


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_fp32_transfers_match_the_fp64_ones(precision):
    """sse_state_set_f32/get_f32 move the same values as the FP64 calls for the
    fields held in the tendency precision; h and the other FP64 fields refuse
    them."""
    torch = pytest.importorskip("torch")
    m, L, p, (u, h, tr), run = inputs.workload("channel_10km", perturb=True)
    dm = binding.Mesh(m, L)
    u32, t32 = u.astype(np.float32), tr[0].astype(np.float32)
    a = binding.State(dm, p, precision)
    b = binding.State(dm, p, precision)
    a.set("u", u32.astype(np.float64))
    a.set("h", h)
    a.set("tracer0", t32.astype(np.float64))
    b.set_f32("u", u32)                                             # pageable
    b.set("h", h)
    pin = torch.from_numpy(t32.copy()).pin_memory()
    b.set_ptr_f32("tracer0", pin.data_ptr())                        # page-locked
    for st in (a, b):
        st.step(run["order"], run["dt"], run["M"], 2)
    for n in ("u", "tracer0"):
        want = a.get(n)
        assert np.array_equal(b.get(n), want), n
        assert np.array_equal(b.get_f32(n), want.astype(np.float32)), n
        out = torch.empty(want.size, dtype=torch.float32).pin_memory()
        b.get_ptr_f32(n, out.data_ptr())
        assert np.array_equal(out.numpy().reshape(want.shape), want.astype(np.float32)), n
    assert np.array_equal(b.get("h"), a.get("h"))
    for n in ("h", "zeta", "Fzeta"):
        with pytest.raises(binding.SSEError) as e:
            b.get_f32(n)
        assert e.value.code == -1
    with pytest.raises(binding.SSEError):
        b.set_f32("h", h.astype(np.float32))
    a.close()
    b.close()


def test_stream_ordered_transfers_match_the_synchronous_ones():
    """sse_state_transfer with SSE_XFER_ASYNC: sets, steps and gets queued in
    stream order without a synchronisation give the same bits as the
    synchronous calls once sse_state_sync returns."""
    torch = pytest.importorskip("torch")
    m, L, p, (u, h, tr), run = inputs.workload("channel_10km", perturb=True)
    dm = binding.Mesh(m, L)
    stream = torch.cuda.Stream()
    a = binding.State(dm, p, "mixed")
    b = binding.State(dm, p, "mixed", stream=stream.cuda_stream)
    # b is given FP32 copies of u and T; a starts from the same values in FP64,
    # so that both hold the same FP32 state (the tracer as its anomaly from
    # the EOS reference, rounded once)
    u32, t32 = u.astype(np.float32), tr[0].astype(np.float32)
    tr_a = tr.copy()
    tr_a[0] = t32
    a.load_state(u32.astype(np.float64), h, tr_a)
    a.step(run["order"], run["dt"], run["M"], 2)
    want = a.read_state()
    src = {"u": torch.from_numpy(u32).pin_memory(),
           "h": torch.from_numpy(np.ascontiguousarray(h)).pin_memory(),
           "tracer0": torch.from_numpy(t32).pin_memory()}
    out = {n: torch.empty_like(x).pin_memory() for n, x in src.items()}
    for _ in range(2):   # twice in a row from the same buffers
        for n, x in src.items():
            b.transfer_ptr(n, x.data_ptr(), get=False, f32=(n != "h"), asynchronous=True)
        b.step(run["order"], run["dt"], run["M"], 2)
        for n, x in out.items():
            b.transfer_ptr(n, x.data_ptr(), get=True, f32=(n != "h"), asynchronous=True)
        b.sync()
    assert np.array_equal(out["u"].numpy(), want[0].astype(np.float32))
    assert np.array_equal(out["h"].numpy(), want[1])
    assert np.array_equal(out["tracer0"].numpy(), want[2][0].astype(np.float32))
    import ctypes
    lib = binding.load()
    assert lib.sse_state_transfer(b.handle, 0, ctypes.c_void_p(out["u"].data_ptr()), 8) == -1
    a.close()
    b.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_state_init_equals_create_and_set(precision):
    """sse_state_init (create + set of u, h, tracers and wind in one call) gives
    the state sse_state_create + sse_state_set give: the same bits after two
    steps, on the sphere (two tracers, wind stress, the internal numbering
    far from the caller's)."""
    m, L, p, (u, h, tr), run = inputs.workload("sphere_l4", perturb=True)
    dm = binding.Mesh(m, L)
    a = binding.State(dm, p, precision)
    a.load_state(u, h, tr)
    b = binding.State.init(dm, p, precision, u, h, tr)
    for st in (a, b):
        st.step(run["order"], run["dt"], run["M"], 2)
    for n in ("u", "h", "tracer0", "tracer1", "zeta", "Fzeta", "ubar", "G"):
        assert np.array_equal(a.get(n), b.get(n)), n
    a.close()
    b.close()
    dm.close()
