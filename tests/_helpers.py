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


def mcao_small():
    """8 m two-sensor case for the adjoint tests: one side-launched laser star (8 x 8
    subapertures of 8 samples, FFT 16, bin 2, elongated spots) and one natural star (2 x 2 of 32,
    FFT 64, bin 4), two layers, a ground DM and a 5 km DM; noise off."""
    a = inputs.ARCSEC
    cfg = {
        "name": "mcao_small_8m",
        "D": 8.0, "obstruction": 0.0, "lambda_ref": 500e-9,
        "dt": 2e-3, "gain": 0.5, "seed": 11, "noise": False, "psf_every": 1, "n_steps": 10,
        "wfs": [inputs._wfs("lgs", (10 * a, 0.0), 8, 8, 16, 2, 589e-9, 1000.0, height=90e3, na_fwhm=10e3,
                            launch=(4.2, 0.0)),
                inputs._wfs("ngs", (0.0, 15 * a), 2, 32, 64, 4, 1.65e-6, 500.0)],
        "science": [{"theta": (0.0, 0.0), "lambda": 2.2e-6, "n_px": 64, "pad": 2}],
        "layers": [{"n": 256, "pixel": 0.0625, "alt": 0.0, "vx": 8.0, "vy": 2.0, "r0": 0.2, "L0": 25.0,
                    "seed": 3},
                   {"n": 256, "pixel": 0.0625, "alt": 5000.0, "vx": -5.0, "vy": 12.0, "r0": 0.35, "L0": 25.0,
                    "seed": 4}],
    }
    cfg["dms"] = [inputs.dm_spec(cfg, 0.0, 1.0, 0.3), inputs.dm_spec(cfg, 5000.0, 1.4, 0.3)]
    return cfg


def wide_lgs():
    """8 m case with a wide-field laser star: 4 x 4 subapertures of 16 samples (twice the field
    of view of 8-sample subapertures), FFT 32, bin 2, side launch, 5 km sodium layer (elongated
    spots on the block-per-subaperture route); one layer, one ground DM; noise off."""
    cfg = {
        "name": "wide_lgs_8m",
        "D": 8.0, "obstruction": 0.0, "lambda_ref": 500e-9,
        "dt": 2e-3, "gain": 0.5, "seed": 13, "noise": False, "psf_every": 1, "n_steps": 10,
        "wfs": [inputs._wfs("lgs", (0.0, 0.0), 4, 16, 32, 2, 589e-9, 2000.0, height=90e3, na_fwhm=5e3,
                            launch=(4.2, 0.0))],
        "science": [{"theta": (0.0, 0.0), "lambda": 2.2e-6, "n_px": 64, "pad": 2}],
        "layers": [{"n": 256, "pixel": 0.0625, "alt": 0.0, "vx": 8.0, "vy": 2.0, "r0": 0.15, "L0": 25.0,
                    "seed": 5}],
    }
    cfg["dms"] = [inputs.dm_spec(cfg, 0.0, 1.0, 0.3)]
    return cfg
