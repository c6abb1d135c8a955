"""Count the FP64 operations of one large step of the named workloads with the
oracle's counting build and write the summary the benchmark reads.

    python oracle/count_flops.py > profiles/fp64_flops_oracle.md

Test infrastructure, like the rest of ``oracle/``: it runs only the oracle
(serial, counting build) on the seeded inputs of
``paper_2105_13484_gb300.inputs``; nothing from the CUDA path is involved.
The count is the method's algorithmic work as the oracle writes it (one per
+, -, *, / and sqrt on FP64 values), divided by the workload's cell-layers.
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2105_13484_gb300 import inputs  # noqa: E402

WORKLOADS = ("sphere_l7", "channel_1km")
SOURCES = ("sse_oracle.c", "sse_oracle.h", "flop_count.cpp")


def source_hashes() -> dict:
    """sha256 (16 hex digits) of each source the counting build compiles."""
    out = {}
    for f in SOURCES:
        with open(os.path.join(HERE, f), "rb") as fh:
            out[f] = hashlib.sha256(fh.read()).hexdigest()[:16]
    return out


def count_step(name: str) -> dict:
    """FP64 operations of one large step of the workload, from its seeded
    perturbed initial state."""
    m, L, p, (u, h, tr), run = inputs.workload(name, perturb=True)
    o = oracle.Oracle(m, L, p, counting=True)
    o.flops(reset=True)
    t0 = time.perf_counter()
    o.step(run["order"], run["dt"], run["M"], u, h, tr)
    secs = time.perf_counter() - t0
    n = o.flops(reset=True)
    cl = int(m.nCells) * int(L)
    # the three parts of a step, each called alone on the initial state (the
    # counts do not depend on the values); SSPRK3-SE calls each three times
    # (SSPRK2-SE twice), the rest of the step is the split, the layer fluxes,
    # the reconciliation and the stage combinations
    calls = 3 if run["order"] == 3 else 2
    ubar, ut = o.split(u, h)
    zeta = o.ssh(h)
    o.flops(reset=True)
    o.baroclinic_feuler(u, ut, zeta, h, tr, run["dt"])
    n_bcl = o.flops(reset=True)
    o.barotropic_substep(run["order"], ubar, zeta, 0.0 * ubar, run["dt"], run["M"])
    n_btr = o.flops(reset=True)
    o.thickness_tracer_fe(h, tr, u, run["dt"])
    n_thk = o.flops(reset=True)
    parts = {"baroclinic stage (Algorithm 1)": n_bcl,
             f"barotropic sub-cycle (Algorithm {4 if run['order'] == 3 else 3}, M = {run['M']})":
                 n_btr,
             "thickness and tracer stage": n_thk}
    return {"workload": name, "cells": int(m.nCells), "edges": int(m.nEdges), "layers": int(L),
            "tracers": int(p.get("nTracers", 1)), "order": run["order"], "M": run["M"],
            "flops_per_step": n, "flops_per_cell_layer_step": n / cl, "seconds": secs,
            "calls": calls, "parts": parts,
            "rest": n - calls * (n_bcl + n_btr + n_thk), "cell_layers": cl}


def main() -> int:
    rows = [count_step(w) for w in WORKLOADS]
    print("# FP64 operations per cell-layer-step, counted in the oracle\n")
    print("Command (from the repository root, on the CPU; no GPU involved):\n")
    print("```\npython oracle/count_flops.py > profiles/fp64_flops_oracle.md\n```\n")
    print("One large step of each workload from its seeded perturbed state, run by the "
          "oracle's counting build (`oracle/flop_count.cpp`: the oracle's source with every "
          "double an operation-counting wrapper; results bit-identical to the plain build).  "
          "One count per +, -, *, / and sqrt on FP64 values (a product and a sum are two, as "
          "an FMA is); comparisons, sign changes and fabs count nothing.  This is the "
          "method's work as the oracle writes it, each operator evaluated on its own; the "
          "GPU kernels execute a different number (they form shared intermediate quantities "
          "once per stage and, in the patch-tiled kernels, repeat halo work), which only a "
          "hardware count of their launches measures.\n")
    print("| workload | cells | edges | layers | tracers | scheme | M | FP64 flops per step "
          "| FP64 flops per cell-layer-step |")
    print("|---|---:|---:|---:|---:|---|---:|---:|---:|")
    for r in rows:
        print(f"| {r['workload']} | {r['cells']} | {r['edges']} | {r['layers']} | "
              f"{r['tracers']} | SSPRK{r['order']}-SE | {r['M']} | {r['flops_per_step']} | "
              f"{r['flops_per_cell_layer_step']:.1f} |")
    print("\nBy part (each part's function of the oracle called alone; calls per step "
          "from the scheme):\n")
    print("| workload / part | calls per step | FP64 flops per call | share of the step |")
    print("|---|---:|---:|---:|")
    for r in rows:
        for part, k in r["parts"].items():
            print(f"| {r['workload']}: {part} | {r['calls']} | {k} | "
                  f"{r['calls'] * k / r['flops_per_step']:.3f} |")
        print(f"| {r['workload']}: split, layer fluxes, reconciliation, combinations | 1 | "
              f"{r['rest']} | {r['rest'] / r['flops_per_step']:.3f} |")
    print("\nSources the count was taken from (sha256 of each file, 16 hex digits):\n")
    for f, v in source_hashes().items():
        print(f"- oracle sha256 {f}: {v}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
