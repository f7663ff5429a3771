"""Test-side helpers: interaction matrix and reconstructor built with the oracle, and shared
workloads.  Only the tests use this module."""
import functools

import numpy as np

import oracle
from paper_1608_00386_gb300 import inputs


@functools.lru_cache(maxsize=None)
def scao_tiny_inputs():
    """Screens and a truncated least-squares reconstructor R = -pinv(D) of the 8 m case.

    D is the push-pull interaction matrix (poke 0.1 rad) measured noise-free by the oracle with
    the DM subtracted from a flat wavefront; singular values below 1e-2 of the largest are
    dropped (piston and waffle), as a truncated LSE control matrix."""
    cfg = inputs.scao_tiny()
    screens = inputs.make_screens(cfg)
    zero = [np.zeros_like(s) for s in screens]
    sim = oracle.Sim(cfg, zero)
    n = sim.n_cmd
    d = 0.1
    D = np.zeros((sim.n_slopes, n))
    for j in range(n):
        c = np.zeros(n)
        c[j] = d
        sim.set_commands(c)
        sp = sim.measure()
        c[j] = -d
        sim.set_commands(c)
        D[:, j] = (sp - sim.measure()) / (2 * d)
    U, S, Vt = np.linalg.svd(D, full_matrices=False)
    keep = S > 1e-2 * S[0]
    R = -(Vt[keep].T / S[keep]) @ U[:, keep].T
    return cfg, screens, R.astype(np.float32)


@functools.lru_cache(maxsize=None)
def eelt_inputs(n_layers: int = 10):
    cfg = inputs.eelt_mcao(n_layers=n_layers)
    screens = inputs.make_screens(cfg)
    n_cmd = inputs.n_commands(cfg)
    return cfg, screens, n_cmd
