"""The OpenMP build of the oracle (same source, -fopenmp) returns the same
bits as the serial build: every threaded loop writes only its own entity's
outputs.  It is what times the oracle over all host cores and what makes
full-horizon oracle runs affordable."""
import numpy as np

import oracle
from paper_2105_13484_gb300 import inputs


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def test_threads_bit_identical_sphere():
    m, L, p, (u, h, tr), run = inputs.workload("sphere_l4", perturb=True)
    a = oracle.Oracle(m, L, p).step(3, run["dt"], run["M"], u, h, tr, n_steps=2)
    b = oracle.Oracle(m, L, p, threads=4).step(3, run["dt"], run["M"], u, h, tr, n_steps=2)
    assert _same(a, b)


def test_threads_bit_identical_every_term():
    """Algorithm 2, biharmonic viscosity, tracer diffusion, drag and the
    printed reconciliation, SSPRK2-SE."""
    m, L, p, (u, h, tr), run = inputs.workload("channel_10km", perturb=True)
    p = dict(p, vmix=1, nu_4=1e9, kappa_h=50.0, kappa_v=1e-4, nu_v=1e-3, c_drag=1e-3,
             nu_h=20.0, recon="paper")
    a = oracle.Oracle(m, L, p).step(2, run["dt"], run["M"], u, h, tr, n_steps=2)
    b = oracle.Oracle(m, L, p, threads=3).step(2, run["dt"], run["M"], u, h, tr, n_steps=2)
    assert _same(a, b)
