"""The request runtime (sse_server_*): continuous batching of independent
solves on one GPU.

* A request's result is bit-identical alone, in a mix of concurrent
  requests, and through a plain state (the same kernels in the same order).
* Admission never exceeds the HBM budget or the slot limit, follows arrival
  order, and admits waiting requests as others finish.
* Concurrent small requests overlap: the mix finishes sooner than the same
  requests one at a time.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2105_13484_gb300 import binding, build, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    binding.load()


def _cases():
    out = []
    for k, (nx, ny, L, nT) in enumerate([(16, 32, 10, 1), (13, 18, 7, 2), (24, 20, 12, 1)]):
        m, L, p, st = inputs.channel_case(nx, ny, 10e3, L, perturb=True, nTracers=nT, seed=k)
        out.append((binding.Mesh(m, L), m, L, p, st))
    m, L, p, st, run = inputs.workload("sphere_l4", perturb=True)
    out.append((binding.Mesh(m, L), m, L, p, st))
    return out


def test_same_result_alone_in_the_mix_and_through_a_state():
    cases = _cases()
    dm, m, L, p, (u, h, tr) = cases[0]
    steps = 12
    # alone
    srv = binding.Server(hbm_budget=8 << 30, max_active=1)
    r = srv.submit(dm, p, "mixed", u, h, tr, 3, 200.0, 10, steps)
    assert r.wait(120)["status"] == "done"
    alone = (r.u.copy(), r.h.copy(), r.tr.copy())
    srv.close()
    # in a mix of eight concurrent requests (the same one twice)
    srv = binding.Server(hbm_budget=8 << 30, max_active=8, steps_per_launch=3)
    reqs = []
    for k in range(8):
        dmk, mk, Lk, pk, (uk, hk, tk) = cases[k % len(cases)]
        reqs.append(srv.submit(dmk, pk, "mixed" if k % 3 else "fp64", uk, hk, tk,
                               2 + k % 2, 200.0, 10, 6 + 2 * k))
    again = srv.submit(dm, p, "mixed", u, h, tr, 3, 200.0, 10, steps)
    for q in reqs + [again]:
        assert q.wait(300)["status"] == "done"
    assert srv.stats()["max_active_seen"] > 1
    srv.close()
    for a, b in zip(alone, (again.u, again.h, again.tr)):
        assert np.array_equal(a, b)
    # through a plain state on the default stream
    st = binding.State(dm, p, "mixed")
    st.load_state(u, h, tr)
    st.step(3, 200.0, 10, steps)
    for a, b in zip(alone, st.read_state()):
        assert np.array_equal(a, b)


def test_fp64_request_matches_the_oracle():
    dm, m, L, p, (u, h, tr) = _cases()[1]
    srv = binding.Server(hbm_budget=4 << 30, max_active=4)
    r = srv.submit(dm, p, "fp64", u, h, tr, 3, 200.0, 12, 4)
    assert r.wait(120)["status"] == "done"
    srv.close()
    ref = oracle.Oracle(m, L, p).step(3, 200.0, 12, u, h, tr, n_steps=4)
    for a, b in zip((r.u, r.h, r.tr), ref):
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-11


def test_admission_budget_order_and_backfill():
    cases = _cases()
    dm, m, L, p, (u, h, tr) = cases[0]
    fp = binding.footprint(dm, p, "mixed")
    srv = binding.Server(hbm_budget=int(2.5 * fp), max_active=16)
    reqs = [srv.submit(dm, p, "mixed", u, h, tr, 3, 200.0, 10, 5 + k) for k in range(7)]
    infos = [q.wait(300) for q in reqs]
    st = srv.stats()
    reqs[0].release()                                    # the record is gone afterwards
    with pytest.raises(binding.SSEError):
        reqs[0].info()
    srv.close()
    assert all(i["status"] == "done" for i in infos)
    assert all(i["footprint"] == fp for i in infos)
    assert st["max_active_seen"] <= 2 and st["peak_bytes"] <= int(2.5 * fp)
    t_admit = [i["t_admit"] for i in infos]
    assert t_admit == sorted(t_admit)                     # arrival order
    # the third request waited for one of the first two to finish
    assert infos[2]["t_admit"] >= min(infos[0]["t_done"], infos[1]["t_done"]) - 1e-6


def test_request_larger_than_budget_is_rejected_and_close_drains():
    dm, m, L, p, (u, h, tr) = _cases()[0]
    fp = binding.footprint(dm, p, "fp64")
    srv = binding.Server(hbm_budget=fp - 1, max_active=4)
    with pytest.raises(binding.SSEError) as ei:
        srv.submit(dm, p, "fp64", u, h, tr, 3, 200.0, 10, 2)
    assert ei.value.code == -3
    srv.close()
    srv = binding.Server(hbm_budget=fp, max_active=1)
    reqs = [srv.submit(dm, p, "fp64", u, h, tr, 3, 200.0, 10, 40) for _ in range(3)]
    first = reqs[0].wait(300)
    assert first["status"] == "done"
    assert reqs[2].info()["status"] in ("pending", "active")   # still queued behind the second
    srv.close()                    # the admitted one finishes, a waiting one is cancelled


def test_concurrent_small_requests_overlap():
    dm, m, L, p, (u, h, tr) = _cases()[0]
    n, steps = 12, 20

    def makespan(max_active):
        srv = binding.Server(hbm_budget=16 << 30, max_active=max_active, steps_per_launch=4)
        t0 = time.perf_counter()
        reqs = [srv.submit(dm, p, "mixed", u, h, tr, 3, 200.0, 10, steps) for _ in range(n)]
        for q in reqs:
            assert q.wait(300)["status"] == "done"
        t = time.perf_counter() - t0
        srv.close()
        return t

    makespan(4)                                           # warm up
    t1, t8 = makespan(1), makespan(8)
    assert t8 < t1 / 1.2, (t1, t8)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_patch_size_keeps_results_within_rounding_and_the_tuner_picks_a_candidate():
    """The partition of the tiled sub-cycle only changes which code path (an
    owned or a halo copy of an edge) rounds a value first, so results with
    three different patch counts (and 512- or 1024-thread patches) agree to the
    mixed form's rounding, far inside its error bounds against the oracle
    (u 1e-4, h 1e-9, tracers 1e-6)."""
    m, L, p, (u, h, tr), run = inputs.workload("sphere_l4", perturb=True)
    dm = binding.Mesh(m, L)
    outs, patches = [], []
    for pc in (0, 256, 2000):
        st = binding.State(dm, p, "mixed", patch_cells=pc)
        patches.append(st.patches())
        st.load_state(u, h, tr)
        st.step(3, run["dt"], run["M"], 3)
        outs.append(st.read_state())
        st.close()
    assert len(set(patches)) == 3 and min(patches) >= 1
    for o in outs[1:]:
        assert _rel(o[0], outs[0][0]) < 1e-5
        assert _rel(o[1], outs[0][1]) < 1e-10
        assert _rel(o[2], outs[0][2]) < 1e-7
    for obj in ("latency", "throughput"):
        pc = binding.tune(dm, p, "mixed", obj)
        assert pc in (64, 128, 256, 384, 512, 768, 1024, 1536)
    # a server that tunes for throughput: bit-identical to a state with its patch size
    pc = binding.tune(dm, p, "mixed", "throughput")
    srv = binding.Server(hbm_budget=4 << 30, max_active=4, tune="throughput")
    r = srv.submit(dm, p, "mixed", u, h, tr, 3, run["dt"], run["M"], 3)
    assert r.wait(120)["status"] == "done"
    srv.close()
    st = binding.State(dm, p, "mixed", patch_cells=pc)
    st.load_state(u, h, tr)
    st.step(3, run["dt"], run["M"], 3)
    for a, b in zip(st.read_state(), (r.u, r.h, r.tr)):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_baroclinic_patch_size_keeps_the_bits_and_the_tuner_picks_a_candidate(precision):
    """sse_tuning.bcl_patch_cells sets the fused baroclinic kernel's patch
    size; every size computes each edge, cell and vertex with the same
    arithmetic, so the results are the same bits.  sse_tune returns one of the
    candidate sizes (or 0), and a size the ABI does not know is refused."""
    m, L, p, (u, h, tr), run = inputs.workload("sphere_l4", perturb=True)
    dm = binding.Mesh(m, L)
    outs = []
    for pc in (0, 32, 64, 160):
        st = binding.State(dm, p, precision, bcl_patch_cells=pc)
        st.load_state(u, h, tr)
        st.step(3, run["dt"], run["M"], 2)
        outs.append(st.read_state())
        st.close()
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)
    for obj in ("latency", "throughput"):
        shapes = binding.tune_shapes(dm, p, precision, obj)
        assert shapes["bcl_patch_cells"] in (0, 160, 128, 112, 96, 80, 64, 48, 32)
        assert shapes["patch_cells"] in (0, 64, 128, 256, 384, 512, 768, 1024, 1536)
    with pytest.raises(binding.SSEError):
        binding.State(dm, p, precision, bcl_patch_cells=33)
    dm.close()


def test_packed_mode_same_result_as_alone():
    """SSE_SERVER_PACKED: the active requests of one precision and order run
    in rounds of one sse_step_batch call; each result equals the request run
    alone, whatever else joins or leaves the rounds (uneven meshes, layer
    counts, time steps and horizons, both precisions and orders)."""
    cases = _cases()
    runs = [(k % len(cases), "mixed" if k % 3 else "fp64", 2 + k % 2, 150.0 + 25 * k, 8 + k % 5,
             4 + 3 * k) for k in range(9)]
    alone = []
    srv = binding.Server(hbm_budget=8 << 30, max_active=1)
    for c, prec, order, dt, M, steps in runs:
        dm, m, L, p, (u, h, tr) = cases[c]
        r = srv.submit(dm, p, prec, u, h, tr, order, dt, M, steps)
        assert r.wait(300)["status"] == "done"
        alone.append((r.u.copy(), r.h.copy(), r.tr.copy()))
        r.release()
    srv.close()
    srv = binding.Server(hbm_budget=8 << 30, max_active=16, steps_per_launch=3, packed=True)
    reqs = []
    for c, prec, order, dt, M, steps in runs:
        dm, m, L, p, (u, h, tr) = cases[c]
        reqs.append(srv.submit(dm, p, prec, u, h, tr, order, dt, M, steps))
    for q in reqs:
        assert q.wait(300)["status"] == "done"
    assert srv.stats()["max_active_seen"] > 1
    srv.close()
    for q, ref in zip(reqs, alone):
        for a, b in zip((q.u, q.h, q.tr), ref):
            assert np.array_equal(a, b)
