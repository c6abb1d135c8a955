"""Write the stored oracle results at each full-size workload's horizon.

The FP64 oracle (``oracle/``, nothing else) runs the workload from its seeded
initial state for the configuration's whole step count -- the 92,480-cell
channel: SSPRK3-SE, dt = 60 s, M = 30, 200 steps; the level-7 sphere:
SSPRK3-SE, dt = 600 s, M = 40, 144 steps -- and a seeded sample of the final
fields (u, h, zeta, and each tracer) is stored with its indices, next to a
digest of the inputs, in ``horizon_<workload>.npz``.  The oracle also runs
once more from the same state with every thickness moved by one unit in the
last place (a seeded sign per entry), and the relative L2 distance between
the two results over each field's sampled entries is stored as that field's
spread: how far the FP64 solution itself moves under a rounding-sized change
of its input, the floor below which no two FP64 evaluation orders can be
expected to agree.  The GPU tests step the
same inputs on the device for the same number of steps and compare the
sampled entries element by element (the full fields are 10^7-10^8 values,
too large to store).  The digest lets a test refuse to compare results whose
inputs were generated differently.

    python tests/golden/make_horizon.py [channel_1km|sphere_l7 ...] [--threads N] [--out DIR]

Takes minutes per workload (two runs) on a multi-core host (the OpenMP build of the
oracle; results are bit-identical to the serial build).
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NSAMPLE = 4096


def input_digest(m, L, p, state) -> str:
    """SHA-256 over every array that defines the run's inputs."""
    h = hashlib.sha256()
    for name in ("cellsOnEdge", "edgesOnEdge", "weightsOnEdge", "dcEdge", "dvEdge", "areaCell",
                 "areaTriangle", "kiteAreasOnVertex", "fEdge", "fVertex", "bottomDepth"):
        h.update(np.ascontiguousarray(getattr(m, name)).tobytes())
    for x in state:
        h.update(np.ascontiguousarray(x, dtype=np.float64).tobytes())
    ws = p.get("windStress")
    if ws is not None:
        h.update(np.ascontiguousarray(ws, dtype=np.float64).tobytes())
    h.update(repr(L).encode())
    return h.hexdigest()


def ulp_perturbed(h: np.ndarray, seed: int = 7) -> np.ndarray:
    """h with every entry moved to its neighbouring double, up or down by a
    seeded sign."""
    up = np.random.default_rng(seed).random(h.shape) < 0.5
    return np.where(up, np.nextafter(h, np.inf), np.nextafter(h, -np.inf))


def sample_indices(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(NSAMPLE, n), replace=False))


def path_of(name: str, out_dir: str = HERE) -> str:
    return os.path.join(out_dir, f"horizon_{name}.npz")


def make(name: str, threads: int, out_dir: str = HERE) -> None:
    import oracle
    from paper_2105_13484_gb300 import inputs

    m, L, p, (u, h, tr), run = inputs.workload(name, perturb=True)
    digest = input_digest(m, L, p, (u, h, tr))
    o = oracle.Oracle(m, L, p, threads=threads)
    t0 = time.time()

    def fields_of(h0):
        uo, ho, tro = o.step(run["order"], run["dt"], run["M"], u, h0, tr, n_steps=run["steps"])
        fl = {"u": uo.ravel(), "h": ho.ravel(), "zeta": ho.sum(1) - m.bottomDepth}
        for k in range(tro.shape[0]):
            fl[f"tracer{k}"] = tro[k].ravel()
        return fl

    fields = fields_of(h)
    moved = fields_of(ulp_perturbed(h))
    secs = time.time() - t0
    out = {"digest": np.array(digest), "steps": np.array(run["steps"]),
           "order": np.array(run["order"]), "dt": np.array(run["dt"]), "M": np.array(run["M"])}
    for seed, (f, x) in enumerate(fields.items()):
        idx = sample_indices(x.size, seed)
        out[f"{f}_idx"] = idx.astype(np.int64)
        out[f"{f}_val"] = x[idx]
        out[f"{f}_norm"] = np.array(np.linalg.norm(x))   # full-field L2 norm
        out[f"{f}_spread"] = np.array(np.linalg.norm(moved[f][idx] - x[idx]) / np.linalg.norm(x[idx]))
    np.savez_compressed(path_of(name, out_dir), **out)
    print(f"{name}: 2 x {run['steps']} steps in {secs:.0f} s on {threads} threads -> "
          f"{path_of(name, out_dir)}; spread " +
          " ".join(f"{f} {float(out[f + '_spread']):.2e}" for f in fields), flush=True)


def main() -> None:
    import oracle
    ap = argparse.ArgumentParser()
    ap.add_argument("workloads", nargs="*", default=["channel_1km", "sphere_l7"])
    ap.add_argument("--threads", type=int, default=oracle.host_threads())
    ap.add_argument("--out", default=HERE, help="folder for the .npz files (default: here)")
    a = ap.parse_args()
    os.makedirs(a.out, exist_ok=True)
    for w in a.workloads:
        make(w, a.threads, a.out)


if __name__ == "__main__":
    main()
