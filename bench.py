#!/usr/bin/env python
"""Throughput of one SSPRK3-SE large step on the level-7 icosahedral sphere.

Workload (the synthetic stand-in for the paper's global-ocean runs): the
level-7 geodesic sphere (163,842 cells; 114,689 ocean cells and 343,016
edges after the seeded land mask), 60 z-star layers over seeded bathymetry
of 100-5000 m, T and S with a linear EOS, f = 2 Omega sin(lat), seeded zonal
wind stress; SSPRK3-SE with dt = 600 s and M = 40 barotropic sub-steps,
reconciliation "consistent", 144 steps (one day).  A "step" is one large
step: three baroclinic stages, three sub-cycles and three thickness stages.

Metric: cell-layer-steps/s = ocean cells x layers x steps / device time.
The headline form is the mixed-precision path; the FP64 path is measured in
the same run and reported under "forms", with per-step p50/p99 latency.  L2
is flushed (a 512 MB write) between timed steps and the flush is excluded
from the per-step CUDA-event times.  The same run also measures, under
"also": the 92,480-cell channel (both forms); the sphere with partial bottom
cells and biharmonic viscosity; the channel with Algorithm 2 (implicit
vertical mixing); the dt-refinement sweep of the channel (FP64 and mixed); a
64-member uneven ensemble packed into one launch per kernel and stage
against one member at a time; and a seeded Poisson request stream, mixed
precision with continuous batching against FP64 one request at a time
(p50/p99 time-to-horizon).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload sphere_l7|channel_1km] [--no-also] [--no-serving]
                    [--study convergence]

Under torchrun with N > 1 every rank runs an independent replica (the method
has no cross-replica exchange): value = N x per-replica units / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import re
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-layer-steps/s"
WORKLOAD = "sphere_l7"

# algorithmic HBM bytes per launch of each kernel class (inputs read once,
# outputs written once); sR = 8 (FP64) or 4 (mixed); h and zeta are FP64
# except the FP32 copy of h the mixed form's tendency kernels read.


def kernel_bytes(cls, C, E, V, L, nT, sR, stage_has_old=True, mixed=False):
    CL, EL, VL = C * L, E * L, V * L
    if cls == "cell_diag":
        return (EL + E + CL + nT * CL) * sR + 6 * CL * sR
    if cls == "vertex":
        return (EL + E + CL) * sR + 2 * VL * sR
    if cls == "edge_pre":
        return (EL + E + CL + VL) * sR + 2 * EL * sR
    if cls == "bcl_edge":
        ins = (EL + (EL if stage_has_old else 0) + E + CL + 6 * CL + VL + 2 * EL) * sR + 8 * C
        return ins + (EL + E) * sR
    if cls == "btr":
        return (3 * E + E) * sR + 8 * C + 8 * E
    if cls == "transport":
        return 8 * CL + 2 * EL * sR + 2 * E * sR + 3 * 8 * E + EL * sR
    if cls == "thickness":
        # flux, column flux, h_s (+ its FP32 copy), tracers; h^n, its copy and
        # tracers^n only in stages that combine with the old level; writes h
        # (+ copy), tracers, zeta
        h_words = 8 * CL + (sR * CL if mixed else 0)
        old = (h_words + nT * CL * sR) if stage_has_old else 0
        return (EL * sR + 8 * E + h_words + nT * CL * sR + old +
                h_words + nT * CL * sR + 8 * C)
    if cls == "combine":
        return 4 * E * sR
    return 0


def fused_stage_bytes(cls, C, E, L, nT, sR, stage_has_old, mixed):
    """Algorithmic HBM bytes of one launch of a fused 3-D stage kernel: each
    3-D array the stage needs read once, each it produces written once.
    Baroclinic stage: utilde in, utilde^n (stages that combine with the old
    level), h (the FP32 copy in the mixed form), nT tracers; utilde out; the
    2-D ubar, column transport, G and SSH.  Thickness/tracer stage: the
    transport velocity's utilde, h and its FP32 copy, nT tracers, and h^n, its
    copy and nT tracers^n where the stage combines with the old level; h, its
    copy and nT tracers out; the 2-D u^A, column flux, ubar and SSH."""
    CL, EL = C * L, E * L
    hw = 8 * CL + (4 * CL if mixed else 0)          # h (+ the FP32 copy)
    if cls == "bcl_edge":
        hr = 4 * CL if mixed else 8 * CL
        return (2 * EL * sR + (EL * sR if stage_has_old else 0) + hr + nT * CL * sR +
                3 * E * sR + 8 * C)
    if cls == "thickness":
        old = (hw + nT * CL * sR) if stage_has_old else 0
        return (EL * sR + hw + nT * CL * sR + old + hw + nT * CL * sR +
                E * (2 * sR + 8) + 8 * C)
    return None


def step_bytes_per_cell_layer(mixed: bool, nT: int = 1) -> float:
    """Algorithmic bytes per cell-layer of one SSPRK3-SE step: every 3-D
    array read or written once per stage (E ~ 3C counts 3 words per cell):
    baroclinic stages 7+nT, 10+nT, 10+nT words, thickness stages 5+2nT,
    6+3nT, 6+3nT words; mixed: h 8 B, everything else 4 B."""
    if not mixed:
        return 8.0 * ((7 + nT) + 2 * (10 + nT) + (5 + 2 * nT) + 2 * (6 + 3 * nT))
    # mixed: h words (8 B): bcl reads h once per stage (3), thickness stages
    # read h_stage + h^n and write h (stage 1: 2 words, stages 2-3: 3 words)
    h_words = 3 + 2 + 3 + 3
    total_words = (7 + nT) + 2 * (10 + nT) + (5 + 2 * nT) + 2 * (6 + 3 * nT)
    return 8.0 * h_words + 4.0 * (total_words - h_words)


# ncu summaries under profiles/ per kernel class (mixed form, this workload);
# each records DRAM traffic per launch and the hashes of the sources it was
# captured from, so a figure taken from an older kernel is not reported
PROFILE_OF = {  # committed ncu summaries by workload and kernel class (mixed form)
    "sphere_l7": {"btr": "btr_tiled_sphere_l7.md", "bcl_edge": "bcl_fused_sphere_l7.md",
                  "thickness": "thick_fused_sphere_l7.md"},
}
KERNEL_SOURCES = ("paper_2105_13484_gb300/csrc/btr_kernel.cu",
                  "paper_2105_13484_gb300/csrc/stage_kernels.cu",
                  "paper_2105_13484_gb300/csrc/bcl_fused.cu",
                  "paper_2105_13484_gb300/csrc/thick_fused.cu",
                  "paper_2105_13484_gb300/csrc/sse_internal.cuh")
# the sources a kernel class's device code is compiled from: a capture of one
# class stays valid while these are unchanged (ncu flushes the caches before
# each captured launch, so its DRAM bytes do not depend on the other kernels)
SOURCES_OF = {"btr": ("btr_kernel.cu", "sse_internal.cuh"),
              "bcl_edge": ("bcl_fused.cu", "sse_internal.cuh"),
              "thickness": ("thick_fused.cu", "sse_internal.cuh")}


_CXX_TOKENS = re.compile(r'//[^\n]*|/\*.*?\*/|"(?:\\.|[^"\\\n])*"|\'(?:\\.|[^\'\\\n])*\'',
                         re.S)


def code_of(text):
    """A C++/CUDA source without its comments (string and character literals
    kept) and with every run of blank space made one space: what compiles,
    so that a comment-only edit keeps the hash of the kernels an ncu capture
    was taken from."""
    text = _CXX_TOKENS.sub(lambda m: " " if m.group(0)[0] == "/" else m.group(0), text)
    return " ".join(text.split())


def source_hashes():
    """sha256 (16 hex digits) of the code of each kernel source."""
    import hashlib
    out = {}
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
            out[os.path.basename(rel)] = hashlib.sha256(code_of(f.read()).encode()).hexdigest()[:16]
    return out


def capture_hashes(line, hashes):
    """Collect a profile summary's '- code sha256 <file>: <hash>' line."""
    if line.startswith("- code sha256 "):
        k, v = line[len("- code sha256 "):].strip().split(": ")
        hashes[k] = v


def ncu_traffic(cls, mixed, workload):
    """DRAM bytes per launch from the committed ncu capture of `cls`, or
    (None, reason) when there is none or the kernel sources have changed."""
    name = PROFILE_OF.get(workload, {}).get(cls)
    if not mixed or name is None:
        return None, "no ncu capture of this kernel/form/workload"
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None, "no ncu capture of this kernel/form"
    traffic, hashes = None, {}
    with open(path) as f:
        for line in f:
            if line.startswith("| DRAM bytes read + written"):
                traffic = float(line.split("|")[2].split()[0]) * 1e6
            capture_hashes(line, hashes)
    if traffic is None or not hashes:
        return None, "capture summary incomplete"
    now = source_hashes()
    if any(hashes.get(f) != now.get(f) for f in SOURCES_OF[cls]):
        return None, "kernel sources changed since the ncu capture"
    return traffic, f"profiles/{name}"


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the GPU works."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go to SSE_CLOCKS_DIR (default: the system temp folder);
        # the JSON line carries their summary
        d = os.environ.get("SSE_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": float(np.median(busy)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(torch, dist, value, device):
    """Max of a per-rank float over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, world, max_ms):
    """Whole-job throughput of `world` independent replicas timed together."""
    return world * units_per_rank / (max_ms / 1e3)


def build_workload(seed=0, scale=None, name=WORKLOAD, **over):
    from paper_2105_13484_gb300 import inputs
    if scale is not None:
        over = dict(over, nx=scale[0], ny=scale[1])
    m, L, p, st, run = inputs.workload(name, seed=seed, perturb=True, **over)
    return m, L, p, st, run


# ---------------------------------------------------------------------------
# the oracle (CPU baseline / reference arm)
# ---------------------------------------------------------------------------
def host_info():
    """CPU model and core count of this host (the oracle baseline's machine)."""
    import oracle
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
            else:
                f.seek(0)
                parts = {}
                for line in f:
                    if ":" in line:
                        k, v = line.split(":", 1)
                        parts.setdefault(k.strip().lower(), v.strip())
                if "cpu implementer" in parts:
                    model = (f"{platform.machine()} implementer {parts['cpu implementer']} "
                             f"part {parts.get('cpu part', '?')}")
    except OSError:
        pass
    return {"cpu_model": model, "nproc": os.cpu_count(), "threads_available": oracle.host_threads(),
            "machine": platform.machine()}


def time_oracle(steps, warmup, name=WORKLOAD, threads=1, **over):
    """The FP64 C oracle on `threads` host threads (its OpenMP build above 1,
    bit-identical results), `steps` timed steps of the named workload after
    `warmup` untimed ones.  Returns (cell-layer-steps/s, ms per step, sample)."""
    import oracle
    m, L, p, (u, h, tr), run = build_workload(name=name, **over)
    o = oracle.Oracle(m, L, p, threads=threads)
    for _ in range(warmup):
        u, h, tr = o.step(run["order"], run["dt"], run["M"], u, h, tr)
    t0 = time.perf_counter()
    for _ in range(steps):
        u, h, tr = o.step(run["order"], run["dt"], run["M"], u, h, tr)
    dt = time.perf_counter() - t0
    units = m.nCells * L * steps
    desc = (f"{name}: {m.nCells} cells x {L} layers, {steps} SSPRK{run['order']}-SE steps "
            f"(dt {run['dt']} s, M {run['M']}), {threads} thread{'s' if threads > 1 else ''}")
    return units / dt, dt / steps * 1e3, desc


def cpu_baseline_of(name, horizon, omp_steps=3, single_steps=1):
    """The oracle as it stands on this host's cores: all threads (OpenMP
    build) and one thread, each on a few steps of the full workload; the
    time for the configuration's horizon is extrapolated from them."""
    info = host_info()
    nt = info["threads_available"]
    v_all, ms_all, s_all = time_oracle(omp_steps, 0, name=name, threads=nt)
    v_one, ms_one, s_one = time_oracle(single_steps, 0, name=name, threads=1)
    return {"value": v_all, "unit": METRIC, "cores": nt, "kind": "oracle", "sample": s_all,
            "horizon_steps": horizon,
            "horizon_s_extrapolated": ms_all * horizon / 1e3,
            "single_thread": {"value": v_one, "unit": METRIC, "cores": 1, "sample": s_one,
                              "horizon_s_extrapolated": ms_one * horizon / 1e3},
            **info}


def run_reference(args):
    """The reference arm: the FP64 oracle (the only implementation of the
    method besides this one) on every host core, on the headline workload;
    each timed step is one full step of the level-7 sphere when the whole run
    stays within minutes (about 1.1 s a step on 16 Arm cores: the default 144
    + 5 steps take about three minutes), else of the same recipe at level 6."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    steps, warmup = args.steps, args.warmup
    nt = oracle.host_threads()
    over = {} if steps + warmup <= 160 else {"level": 6}
    value, ms, sample = time_oracle(steps, warmup, name=args.workload, threads=nt, **over)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC,
            "n_gpus": args.gpus, "steps": steps, "warmup": warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload + ("" if not over else " at level 6 (bounded sample)"),
                       "sample": sample, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": nt, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "host": host_info()}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def measure_form(torch, binding, dm, m, L, p, state0, run, precision, steps, warmup, stream,
                 flush, sampler=None):
    u, h, tr = state0
    st = binding.State(dm, p, precision, stream=stream.cuda_stream)
    st.load_state(u, h, tr)
    order, dt, M = run["order"], run["dt"], run["M"]
    for _ in range(warmup):
        st.step(order, dt, M, 1)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    st.profile(True)
    if sampler:
        sampler.start()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    with torch.cuda.stream(stream):
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            st.step(order, dt, M, 1)
            ev[i][1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop() if sampler else None
    prof = st.profile_read()
    st.profile(False)
    per = np.array([a.elapsed_time(b) for a, b in ev])
    ms = float(per.sum())
    d = st.diagnostics(check=False)
    res = {"device_ms": ms, "ms_per_step": ms / steps, "wall_s": t_wall, "prof": prof,
           "patches": st.patches(), "fused_bcl": st.kernels_per_step(order) < 20,
           "latency_ms": {"p50": float(np.percentile(per, 50)), "p99": float(np.percentile(per, 99))},
           "clocks": clocks, "diag": d, "kernels_per_step": st.kernels_per_step(order)}
    gu, gh, gt = st.read_state()
    res["final"] = (gu, gh, gt)
    st.close()
    return res


def measure_e2e(torch, binding, dm, p, state0, run, precision, steps, stream, native=True):
    """Through the public C ABI with pinned host buffers: per step, H2D of
    (u, h, T), one large step, D2H of (u, h, T), queued in stream order
    (sse_state_transfer with SSE_XFER_ASYNC) and one sse_state_sync, after
    which the step's result is in host memory.  Each field crosses in the
    precision the state holds it in: FP32 u and T for the mixed form, FP64 h
    always, FP64 everything for the FP64 form."""
    u, h, tr = state0
    st = binding.State(dm, p, precision, stream=stream.cuda_stream)
    fields = [("u", u), ("h", h)] + [(f"tracer{k}", tr[k]) for k in range(tr.shape[0])]
    # native: each field in the precision the state holds it in; else all FP64
    f32 = {n: native and precision == "mixed" and n != "h" for n, _ in fields}
    hin = [(n, torch.from_numpy(np.ascontiguousarray(
        x, dtype=np.float32 if f32[n] else np.float64)).pin_memory()) for n, x in fields]
    hout = [(n, torch.empty_like(x).pin_memory()) for n, x in hin]
    order, dt, M = run["order"], run["dt"], run["M"]

    def put(n, x):
        st.transfer_ptr(n, x.data_ptr(), get=False, f32=f32[n], asynchronous=True)

    def take(n, x):
        st.transfer_ptr(n, x.data_ptr(), get=True, f32=f32[n], asynchronous=True)

    for n, x in hin:
        put(n, x)
    st.step(order, dt, M, 1)
    st.sync()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        for n, x in hin:
            put(n, x)
        st.step(order, dt, M, 1)
        for n, x in hout:
            take(n, x)
        st.sync()   # the step's result is in host memory
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    nbytes = sum(x.numel() * x.element_size() for _, x in hin)
    dtypes = {n: ("f32" if f32[n] else "f64") for n, _ in fields}
    st.close()
    return ms, nbytes, dtypes


def kernel_roofline_of(prof, m, L, nT, mixed, order, fused):
    """The dominant kernel of the HBM-bound 3-D phase: the longest kernel
    class other than the barotropic sub-cycle, whose bound is its grid
    synchronisations and on-chip latency (reported under "subcycle").  Its
    algorithmic bytes per launch (averaged over the step's stages; the first
    stage has no old-level input) over its average launch time, against the
    measured HBM copy peak."""
    peaks, peak_kind = measured_peaks()
    sR = 4 if mixed else 8
    total = sum(v[0] for v in prof.values()) or 1.0
    overall = max(prof, key=lambda k: prof[k][0])
    dom = max((k for k in prof if k != "btr" and prof[k][1]), key=lambda k: prof[k][0])
    nlaunch = prof[dom][1]
    per_launch_ms = prof[dom][0] / max(nlaunch, 1)
    C, E, V = m.nCells, m.nEdges, m.nVertices

    def stage_bytes(has_old):
        b = fused_stage_bytes(dom, C, E, L, nT, sR, has_old, mixed) if fused else None
        return b if b is not None else kernel_bytes(dom, C, E, V, L, nT, sR, has_old, mixed)
    if dom in ("bcl_edge", "thickness"):
        b = (stage_bytes(False) + (order - 1) * stage_bytes(True)) / order
    else:
        b = kernel_bytes(dom, C, E, V, L, nT, sR, True, mixed)
    achieved = b / (per_launch_ms / 1e3) / 1e9
    names = {"bcl_edge": "k_bcl_fused" if fused else "k_bcl_edge",
             "thickness": "k_thick_fused" if fused else "k_thickness"}
    return {"kernel": names.get(dom, dom), "class": dom, "bound": "hbm", "achieved": achieved,
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
            "peak_source": f"{peak_kind} hbm_gbs (copy), burst", "bytes_per_launch": b,
            "ms_per_launch": per_launch_ms, "share_of_step": prof[dom][0] / total,
            "longest_overall": {"class": overall, "share_of_step": prof[overall][0] / total,
                                "bound": "grid synchronisation and L2 latency (see subcycle)"
                                if overall == "btr" else "hbm"}}


def step_roofline_of(m, L, nT, mixed, ms_per_step, workload):
    """The whole step against the HBM copy peak: the algorithmic bytes of one
    large step (every 3-D array read or written once per stage) over the
    step's device time; traffic from the committed launch list with DRAM
    counters when one exists for this workload and form."""
    peaks, peak_kind = measured_peaks()
    per_cl = step_bytes_per_cell_layer(mixed, nT)
    step_b = per_cl * m.nCells * L
    gbs = step_b / (ms_per_step / 1e3) / 1e9
    traffic, src = step_traffic(workload, mixed)
    return {"kernel": "step (all launches of one large step)", "bound": "hbm", "achieved": gbs,
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
            "peak_source": f"{peak_kind} hbm_gbs (copy)", "bytes_per_step": step_b,
            "bytes_per_cell_layer": per_cl, "ms_per_step": ms_per_step,
            "traffic": traffic, "traffic_source": src}


def step_traffic(workload, mixed):
    """DRAM bytes (read + write) of one large step from the committed ncu
    launch list of this workload and form, while the kernel sources match."""
    name = f"launches_{workload}_{'mixed' if mixed else 'fp64'}.md"
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None, "no ncu launch list with DRAM counters for this workload/form"
    traffic, hashes = None, {}
    with open(path) as f:
        for line in f:
            if line.startswith("| DRAM bytes per step"):
                traffic = float(line.split("|")[2].split()[0]) * 1e6
            capture_hashes(line, hashes)
    if traffic is None or not hashes:
        return None, "launch list incomplete"
    if hashes != source_hashes():
        return None, "kernel sources changed since the ncu capture"
    return traffic, f"profiles/{name}"


def subcycle_of(prof, m, run, steps, tiled_patches, workload, mixed):
    """The barotropic sub-cycle, which is bound by its grid synchronisations
    and on-chip latency rather than by HBM: its time per step, grid barriers
    per step (the tiled kernel: one per sub-step; the global-memory kernel:
    one per forward-Euler sub-stage), the time per barrier interval, and its
    L2/DRAM traffic per launch from the committed ncu capture."""
    order, M = run["order"], run["M"]
    calls = 3 if order == 3 else 2
    ms, launches = prof.get("btr", (0.0, 0))
    ms_step = ms / steps
    per_call_syncs = M if tiled_patches else order * M
    syncs = calls * per_call_syncs
    out = {"ms_per_step": ms_step, "launches_per_step": launches / steps,
           "substeps_per_step": calls * M, "fe_substages_per_step": calls * order * M,
           "grid_barriers_per_step": syncs,
           "us_per_barrier_interval": ms_step * 1e3 / syncs if syncs else None,
           "kernel": "k_btr_tiled (one patch per SM in shared memory)" if tiled_patches
           else "k_btr (global memory)", "patches": tiled_patches,
           "state_bytes_2d": (4 if mixed else 8) * 4 * m.nEdges + 8 * m.nCells}
    name = PROFILE_OF.get(workload, {}).get("btr")
    l2 = dram = None
    src = "no ncu capture of the sub-cycle for this workload/form"
    if name and mixed and os.path.exists(os.path.join(ROOT, "profiles", name)):
        hashes = {}
        with open(os.path.join(ROOT, "profiles", name)) as f:
            for line in f:
                if line.startswith("| L2 bytes"):
                    l2 = float(line.split("|")[2].split()[0]) * 1e6
                if line.startswith("| DRAM bytes read + written"):
                    dram = float(line.split("|")[2].split()[0]) * 1e6
                capture_hashes(line, hashes)
        src = f"profiles/{name}"
        now = source_hashes()
        if any(hashes.get(f) != now.get(f) for f in SOURCES_OF["btr"]):
            l2 = dram = None
            src = "kernel sources changed since the ncu capture"
    out.update({"l2_bytes_per_launch": l2, "dram_bytes_per_launch": dram, "traffic_source": src})
    return out


def oracle_flops(workload):
    """FP64 operations per cell-layer-step of one large step of the workload as
    the oracle computes it: the committed summary written by
    oracle/count_flops.py from the oracle's counting build (a file read here;
    no oracle code runs in this leg)."""
    path = os.path.join(ROOT, "profiles", "fp64_flops_oracle.md")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        for line in f:
            cells = [c.strip() for c in line.strip().strip("|").split("|")]
            if len(cells) == 9 and cells[0] == workload:
                return float(cells[8])
    return None


def fp64_alu_of(m, L, ms_per_step, fp64_tflops, workload):
    """The FP64 form against its arithmetic bound, the FMA rate measured by
    sse_probe_fma_rate: the algorithmic FP64 operations of a step (counted in
    the oracle) x cell-layers / step time; beside it, while its capture
    matches the kernel sources, the FP64 operations the GPU kernels executed
    (ncu: dadd + dmul + 2 dfma over every launch of one step of the sphere
    recipe)."""
    per_cl = oracle_flops(workload)
    src = ("profiles/fp64_flops_oracle.md (oracle counting build)" if per_cl is not None
           else "no oracle operation count for this workload")
    out = {"bound": "alu", "unit": "TFLOP/s", "peak": fp64_tflops,
           "peak_source": "measured FP64 FMA rate (sse_probe_fma_rate)",
           "flops_per_cell_layer_step": per_cl, "flops_source": src}
    if per_cl is not None and fp64_tflops:
        ach = per_cl * m.nCells * L / (ms_per_step / 1e3) / 1e12
        out.update({"achieved": ach, "frac": ach / fp64_tflops})
    path = os.path.join(ROOT, "profiles", "fp64_ops_per_cell_layer_step.md")
    ex, ex_src = None, "no committed hardware count of the FP64 kernels for this workload"
    if workload.startswith("sphere") and os.path.exists(path):
        hashes = {}
        with open(path) as f:
            for line in f:
                if line.startswith("| FP64 flops per cell-layer-step"):
                    ex = float(line.split("|")[2].split()[0])
                capture_hashes(line, hashes)
        ex_src = "profiles/fp64_ops_per_cell_layer_step.md"
        if hashes != source_hashes():
            ex, ex_src = None, "kernel sources changed since the FP64 operation count"
    out.update({"executed_flops_per_cell_layer_step": ex, "executed_flops_source": ex_src})
    if ex is not None and fp64_tflops:
        ach = ex * m.nCells * L / (ms_per_step / 1e3) / 1e12
        out.update({"executed_achieved": ach, "executed_frac": ach / fp64_tflops})
    return out


def measure_workload(torch, binding, name, forms_todo, headline, steps, warmup, rank, stream,
                     flush, sampler=None, e2e=True, world=1, dist=None, fp64_tflops=None,
                     **over):
    """Every requested precision form of one named workload on this GPU."""
    m, L, p, state0, run = build_workload(seed=rank, name=name, **over)
    nT = int(p.get("nTracers", 1))
    dm = binding.Mesh(m, L, max_level=p.get("maxLevelCell"), rest_thickness=p.get("restThickness"))
    forms = {}
    for prec in forms_todo:
        forms[prec] = measure_form(torch, binding, dm, m, L, p, state0, run, prec, steps, warmup,
                                   stream, flush, sampler if prec == headline else None)
    head = forms[headline]
    mixed = headline == "mixed"
    out = {"mesh": m, "L": L, "p": p, "run": run, "nT": nT, "forms": forms, "head": head}
    out["t_max"] = max_over_ranks(torch, dist, head["device_ms"], "cuda")
    out["value"] = replica_throughput(m.nCells * L * steps, world, out["t_max"])
    # error of the mixed form against the FP64 form at the horizon (per field)
    out["mixed_err"] = None
    if "fp64" in forms and "mixed" in forms:
        fu, fh, ft = forms["fp64"]["final"]
        mu, mh, mt = forms["mixed"]["final"]

        def rel(a, b):
            return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
        err = {"u": rel(mu, fu), "h": rel(mh, fh),
               "zeta": rel(mh.sum(1) - m.bottomDepth, fh.sum(1) - m.bottomDepth)}
        for k, nm in zip(range(nT), ("T", "S")):
            err[nm] = rel(mt[k], ft[k])
        out["mixed_err"] = err
    prof = head["prof"]
    tag = name if not over else name + " (variant)"
    kroof = kernel_roofline_of(prof, m, L, nT, mixed, run["order"], head["fused_bcl"])
    traffic, traffic_src = ncu_traffic(kroof["class"], mixed, name) if not over else \
        (None, "no ncu capture of this variant of the workload")
    kroof["traffic"], kroof["traffic_source"] = traffic, traffic_src
    out["roofline"] = kroof
    out["step_roofline"] = step_roofline_of(m, L, nT, mixed, head["ms_per_step"], tag)
    out["subcycle"] = subcycle_of(prof, m, run, steps, head["patches"], tag, mixed)
    out["kernels"] = {k: {"ms_per_step": v[0] / steps, "share": v[0] / max(head["device_ms"], 1e-9),
                          "launches_per_step": v[1] / steps} for k, v in prof.items() if v[1]}
    vol0 = float(m.areaCell @ state0[1].sum(1))
    out["forms_summary"] = {}
    for k, v in forms.items():
        fs = {"value": world * m.nCells * L * steps / (v["device_ms"] / 1e3),
              "ms_per_step": v["ms_per_step"], "latency_ms": v["latency_ms"],
              "volume_rel_change": abs(v["diag"]["volume"] - vol0) / vol0,
              "hbm_roofline": step_roofline_of(m, L, nT, k == "mixed", v["ms_per_step"], tag),
              "fused_baroclinic": v["fused_bcl"]}
        if k == "fp64":
            fs["alu_roofline"] = fp64_alu_of(m, L, v["ms_per_step"], fp64_tflops, tag)
            fs["kernels"] = {c: {"ms_per_step": x[0] / steps,
                                 "share": x[0] / max(v["device_ms"], 1e-9)}
                             for c, x in v["prof"].items() if x[1]}
        out["forms_summary"][k] = fs
    out["e2e"] = None
    if e2e:
        e2e_steps = min(steps, 20)
        e2e_ms, nbytes, dtypes = measure_e2e(torch, binding, dm, p, state0, run, headline,
                                             e2e_steps, stream)
        e2e_val = replica_throughput(m.nCells * L * e2e_steps, world,
                                     max_over_ranks(torch, dist, e2e_ms, "cuda"))
        out["e2e"] = {"value": e2e_val, "unit": METRIC, "h2d_bytes_per_step": nbytes,
                      "d2h_bytes_per_step": nbytes, "host_dtypes": dtypes}
        if headline == "mixed":
            # the same loop with every field crossing as FP64 host data
            ms64, nb64, dt64 = measure_e2e(torch, binding, dm, p, state0, run, headline,
                                           e2e_steps, stream, native=False)
            out["e2e_fp64_host"] = {
                "value": replica_throughput(m.nCells * L * e2e_steps, world,
                                            max_over_ranks(torch, dist, ms64, "cuda")),
                "unit": METRIC, "h2d_bytes_per_step": nb64, "d2h_bytes_per_step": nb64,
                "host_dtypes": dt64}
    dm.close()
    return out


def _build_requests(binding, specs):
    """Meshes (shared where the spec repeats) and initial states of request specs."""
    from paper_2105_13484_gb300 import inputs
    cache, out = {}, []
    for sp in specs:
        key = (sp["kind"], sp.get("level"), sp.get("nx"), sp.get("ny"), sp["L"],
               sp["seed"] % 7 if sp["kind"] == "sphere" else sp["seed"])
        if key not in cache:
            m, L, p, st = inputs.build_spec(sp)
            dm = binding.Mesh(m, L)
            for prec in ("mixed", "fp64"):      # plans and tuning before the clock runs
                for obj in ("latency", "throughput"):
                    sh = binding.tune_shapes(dm, p, prec, obj)
                    binding.footprint(dm, p, prec, sh["patch_cells"], sh["bcl_patch_cells"])
            cache[key] = (m, L, p, st, dm)
        out.append(cache[key])
    return out


def run_stream(binding, specs, built, precision, max_active, budget, chunk, realtime=True,
               tune="throughput", packed=False):
    """Submit the specs (at their arrival times when realtime) to one server
    (packed: SSE_SERVER_PACKED); returns per-request latency and the makespan."""
    srv = binding.Server(hbm_budget=budget, max_active=max_active, steps_per_launch=chunk,
                         tune=tune, packed=packed)
    t0 = time.perf_counter()
    handles = []
    for sp, (m, L, p, (u, h, tr), dm) in zip(specs, built):
        if realtime:
            wait = t0 + sp.get("arrival", 0.0) - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
        handles.append((srv.submit(dm, p, precision, u, h, tr, sp["order"], sp["dt"], sp["M"],
                                   sp["steps"]), m.nCells * L * sp["steps"]))
    lat, units = [], 0
    for hd, un in handles:
        inf = hd.wait(-1)
        if inf["status"] != "done":
            raise RuntimeError(f"request {inf['id']} ended with {inf['status']}")
        hd.release()
        lat.append(inf["t_done"] - inf["t_submit"])
        units += un
    makespan = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    lat = np.array(lat)
    return {"requests": len(specs), "makespan_s": makespan, "value": units / makespan,
            "unit": METRIC, "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "max_active_seen": st["max_active_seen"],
            "peak_bytes": st["peak_bytes"], "latencies_s": [float(x) for x in lat]}


def measure_ensemble(binding, seed=0):
    """64 uneven channel members (SSPRK3-SE, mixed, 100 steps each) batched
    through the request runtime against the same members one at a time."""
    from paper_2105_13484_gb300 import inputs
    specs = inputs.ensemble_members(seed=seed)
    built = _build_requests(binding, specs)
    packed = run_stream(binding, specs, built, "mixed", 64, 200 << 30, 10, realtime=False,
                        tune="throughput", packed=True)
    batched = run_stream(binding, specs, built, "mixed", 64, 200 << 30, 10, realtime=False,
                         tune="throughput")
    single = run_stream(binding, specs, built, "mixed", 1, 200 << 30, 10, realtime=False,
                        tune="latency")
    tuned = sorted({(b[0].nCells, *binding.tune_shapes(b[4], b[2], "mixed", obj).values(), obj)
                    for b in built for obj in ("throughput", "latency")})
    for r in (packed, batched, single):
        r.pop("latencies_s", None)
    return {"members": len(specs), "cells": sorted({b[0].nCells for b in built}),
            "tuned_shapes": {"columns": ["cells", "sub-cycle patch cells",
                                         "baroclinic patch cells", "objective"],
                             "rows": tuned},
            "layers": [int(min(b[1] for b in built)), int(max(b[1] for b in built))],
            "packed": packed, "batched": batched, "one_at_a_time": single,
            "speedup_packed": single["makespan_s"] / packed["makespan_s"],
            "speedup": single["makespan_s"] / batched["makespan_s"]}


def measure_serving(binding, seed=0, n_fp64=8):
    """A seeded Poisson stream (20 requests/s, 32 requests) of SSPRK2/3-SE
    solves on planar channels and geodesic spheres of levels 5-7, 10-60
    layers, 50-500 steps: mixed precision with continuous batching against
    the FP64 path one request at a time on the same arrival times.  The FP64
    arm serves only the first `n_fp64` requests (one at a time it would take
    minutes); the mixed arm's latencies on those same requests are reported
    beside it."""
    from paper_2105_13484_gb300 import inputs
    specs = inputs.serving_requests(seed=seed)
    built = _build_requests(binding, specs)
    mixed = run_stream(binding, specs, built, "mixed", 64, 200 << 30, 4, tune="throughput",
                       packed=True)
    streams = run_stream(binding, specs, built, "mixed", 64, 200 << 30, 4, tune="throughput")
    fp64 = run_stream(binding, specs[:n_fp64], built[:n_fp64], "fp64", 1, 200 << 30, 4,
                      tune="latency")
    lat8 = np.array(mixed["latencies_s"][:n_fp64])
    for r in (mixed, streams, fp64):
        r.pop("latencies_s", None)
    mixed_first = {"requests": n_fp64, "p50_s": float(np.percentile(lat8, 50)),
                   "p99_s": float(np.percentile(lat8, 99))}
    cells = sorted({b[0].nCells for b in built})
    return {"requests": len(specs), "rate_per_s": 20.0,
            "mix": "planar 2k-60k cells and geodesic levels 5-7 (up to 163,842 cells), "
                   "10-60 layers, 50-500 steps, SSPRK2-SE and SSPRK3-SE",
            "cells": [cells[0], cells[-1]],
            "mixed_batched": mixed, "mixed_streams": streams, "fp64_one_at_a_time": fp64,
            "batching": "mixed_batched: SSE_SERVER_PACKED rounds (one 3-D launch per kernel "
                        "and stage for all active requests); mixed_streams: one stream per "
                        "request",
            "fp64_requests": f"the first {n_fp64} of the {len(specs)} (same arrival times)",
            "mixed_batched_first": mixed_first,
            "throughput_ratio": mixed["value"] / fp64["value"],
            "p99_ratio_same_requests": fp64["p99_s"] / mixed_first["p99_s"]}


def measure_convergence(binding, T=960.0, n_list=(16, 32, 64, 128, 256), n_ref=2048,
                        hold="M", recon=None, forms=("fp64", "mixed"), M0=None):
    """The dt-refinement sweep of the 1 km channel: SSPRK3-SE, the paper's
    relative l2 error of the top-layer velocity u_1 and thickness h_1 at time T
    against a run with T / n_ref, on the GPU.  hold = "M": the sub-step count
    is fixed (dt and the sub-step shrink together); hold = "tau": the
    sub-step length tau = dt / M is fixed (M shrinks with dt).  recon: the
    reconciliation mode (default: the workload's)."""
    m, L, p, (u, h, tr), run = build_workload(name="channel_1km")
    if recon is not None:
        p = dict(p, recon=recon)
    dm = binding.Mesh(m, L)
    M0 = M0 or run["M"]
    dt0 = T / n_list[0]
    tau = dt0 / M0

    def M_of(n):
        return M0 if hold == "M" else max(1, int(round((T / n) / tau)))

    def solve(prec, n):
        st = binding.State(dm, p, prec)
        st.load_state(u, h, tr)
        st.step(3, T / n, M_of(n), n)
        gu, gh, _ = st.read_state()
        st.close()
        return gu[:, 0], gh[:, 0]

    ru, rh = solve("fp64", n_ref)
    out = {"T_s": T, "hold": hold, "recon": p.get("recon"), "dt_s": [T / n for n in n_list],
           "M": [M_of(n) for n in n_list], "reference_dt_s": T / n_ref,
           "reference_M": M_of(n_ref)}
    for prec in forms:
        eu, eh = [], []
        for n in n_list:
            a, b = solve(prec, n)
            eu.append(float(np.linalg.norm(a - ru) / np.linalg.norm(ru)))
            eh.append(float(np.linalg.norm(b - rh) / np.linalg.norm(rh)))
        out[prec] = {"err_u1": eu, "err_h1": eh,
                     "rate_u1": [float(np.log2(eu[i] / eu[i + 1])) for i in range(len(eu) - 1)],
                     "rate_h1": [float(np.log2(eh[i] / eh[i + 1])) for i in range(len(eh) - 1)]}
    dm.close()
    return out


def convergence_study(binding):
    """The longer study of the channel's observed order (run with --study):
    T = 3840 s (64 steps at dt = 60 s) against dt = 0.9375 s, FP64, with M
    fixed and with tau fixed, in the consistent and the printed
    reconciliation; and with a sub-step of about 0.125 s at every dt
    (M = 480 at dt = 60 s, 8 at the reference), so that the sub-cycle's own
    error is negligible and the rate is the large step's."""
    res = {}
    n_list, n_ref = (64, 128, 256, 512), 4096
    for hold in ("M", "tau"):
        for recon in ("consistent", "paper"):
            res[f"{hold}_{recon}"] = measure_convergence(binding, T=3840.0, n_list=n_list,
                                                         n_ref=n_ref, hold=hold, recon=recon,
                                                         forms=("fp64",))
    res["small_tau_consistent"] = measure_convergence(binding, T=3840.0, n_list=n_list,
                                                      n_ref=n_ref, hold="tau",
                                                      recon="consistent", forms=("fp64",),
                                                      M0=480)
    return res


def config_of(name, w, precision, world):
    m, L, run, p = w["mesh"], w["L"], w["run"], w["p"]
    return {"workload": name, "cells": m.nCells, "edges": m.nEdges, "layers": L,
            "tracers": w["nT"], "scheme": f"SSPRK{run['order']}-SE", "dt": run["dt"],
            "M": run["M"], "recon": p.get("recon"), "precision": precision,
            "l2": "flushed (512 MB write) between timed steps, flush excluded",
            "parallelism": f"replicas x{world}"}


def run_ours(args):
    import torch
    from paper_2105_13484_gb300 import binding, build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device (the CUDA path has no CPU fallback)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    binding.load()
    stream = torch.cuda.Stream()
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    # measured arithmetic rates (denominators of the FP64 form's ALU roofline)
    rates = {"fp64_tflops": binding.fma_rate("fp64"), "fp32_tflops": binding.fma_rate("mixed")}
    todo = ("mixed", "fp64") if args.forms == "both" else (args.forms,)
    if args.precision not in todo:
        todo = todo + (args.precision,)
    over = {"level": args.level} if args.level else {}
    w = measure_workload(torch, binding, args.workload, todo, args.precision, args.steps,
                         args.warmup, rank, stream, flush, sampler, not args.no_e2e, world, dist,
                         fp64_tflops=rates["fp64_tflops"], **over)
    head = w["head"]
    also = {}
    extra = args.workload == WORKLOAD and not args.no_also and not args.level
    if extra:
        # the 92,480-cell channel (SSPRK3-SE, dt 60 s, M 30), both forms
        nc = min(args.steps, 200)
        ch = measure_workload(torch, binding, "channel_1km", ("mixed", "fp64"), "mixed", nc,
                              args.warmup, rank, stream, flush, None, False, world, dist,
                              fp64_tflops=rates["fp64_tflops"])
        also["channel_1km"] = {
            "value": ch["value"], "unit": METRIC, "steps": nc, "ms_per_step": ch["t_max"] / nc,
            "latency_ms": ch["head"]["latency_ms"],
            "config": config_of("channel_1km", ch, "mixed", world), "roofline": ch["roofline"],
            "step_roofline": ch["step_roofline"],
            "subcycle": ch["subcycle"], "kernels": ch["kernels"], "forms": ch["forms_summary"],
            "mixed_vs_fp64_rel_l2": ch["mixed_err"]}
        # the same sphere as a global-ocean setup: partial bottom cells on the
        # 60 reference layers and biharmonic viscosity
        ns = min(args.steps, 144)
        pb = measure_workload(torch, binding, "sphere_l7", ("mixed",), "mixed", ns, args.warmup,
                              rank, stream, flush, None, False, world, dist, partial=True,
                              nu_4=1e11)
        K = pb["p"]["maxLevelCell"]
        active = int(K.sum())
        also["sphere_l7_partial_bottom"] = {
            "value": active * ns / (pb["t_max"] / 1e3), "unit": METRIC + " (active cell-layers)",
            "steps": ns, "ms_per_step": pb["t_max"] / ns, "latency_ms": pb["head"]["latency_ms"],
            "active_cell_layers": active, "cell_layers": int(pb["mesh"].nCells * pb["L"]),
            "config": dict(config_of("sphere_l7", pb, "mixed", world), partial_bottom=True,
                           nu_4=1e11),
            "kernels": pb["kernels"],
            "volume_rel_change": pb["forms_summary"]["mixed"]["volume_rel_change"]}
        # the channel with Algorithm 2 (implicit vertical mixing) in every stage
        vm = measure_workload(torch, binding, "channel_1km", ("mixed",), "mixed", nc,
                              args.warmup, rank, stream, flush, None, False, world, dist,
                              vmix=True)
        also["channel_1km_vmix"] = {
            "value": vm["value"], "unit": METRIC, "steps": nc,
            "ms_per_step": vm["t_max"] / nc, "latency_ms": vm["head"]["latency_ms"],
            "config": dict(config_of("channel_1km", vm, "mixed", world), baroclinic="Algorithm 2"),
            "kernels": vm["kernels"],
            "volume_rel_change": vm["forms_summary"]["mixed"]["volume_rel_change"]}
        also["convergence"] = measure_convergence(binding)
    if extra and not args.no_serving:
        also["ensemble"] = measure_ensemble(binding, seed=rank)
        also["serving"] = measure_serving(binding, seed=rank)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_of(args.workload, w["run"]["steps"])

    line = {
        "metric": METRIC, "value": w["value"], "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": w["t_max"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": config_of(args.workload + (f" at level {args.level}" if args.level else ""), w,
                            args.precision, world),
        "roofline": w["roofline"], "step_roofline": w["step_roofline"],
        "subcycle": w["subcycle"], "kernels": w["kernels"],
        "latency_ms": head["latency_ms"],
        "forms": w["forms_summary"],
        "mixed_vs_fp64_rel_l2": w["mixed_err"],
        "measured_rates": rates,
        "e2e": w["e2e"],
        "e2e_fp64_host": w.get("e2e_fp64_host"),
        "gpu_launches": head["kernels_per_step"] * args.steps,
        "clocks": head["clocks"],
        "cpu_baseline": cpu,
        "also": also or None,
    }
    if dist:
        dist.barrier()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=144)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--forms", default="both", choices=["both", "mixed", "fp64"],
                    help="precision forms to measure (the headline form is always measured)")
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, "channel_1km"],
                    help="headline workload (default: the level-7 sphere, 60 layers)")
    ap.add_argument("--no-also", "--no-sphere", dest="no_also", action="store_true",
                    help="skip the channel, partial-bottom, Algorithm 2 and convergence "
                         "measurements")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the batched-ensemble and request-stream measurements")
    ap.add_argument("--study", choices=["convergence"],
                    help="run only the named longer study and print its JSON")
    ap.add_argument("--level", type=int, default=0,
                    help="the sphere recipe at another geodesic level (a smaller case for "
                         "profiling; not a bench line of the workload)")
    args = ap.parse_args()
    if args.level and args.workload != WORKLOAD:
        ap.error("--level applies to the sphere workload")
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.study == "convergence":
        from paper_2105_13484_gb300 import binding, build
        build.build()
        binding.load()
        print(json.dumps({"study": "convergence", "channel_1km": convergence_study(binding)}),
              flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
