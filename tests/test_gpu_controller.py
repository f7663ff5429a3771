"""Closed-loop options through the C ABI against the oracle (float32 tolerances: slopes 1e-4
pixel RMS, commands 1e-5 relative, Strehl 1e-3): the second-order controller (single and
batched) and the sodium layer evolution of the laser sensors."""
import numpy as np
import pytest

import oracle
from paper_1608_00386_gb300 import build, inputs, mcao

from _helpers import scao_tiny_inputs

pytestmark = pytest.mark.gpu

# low-pass-filtered integrator: beta = 0.6, g = 0.5; and a general biquad
CASES = [(1.4, -0.4, 0.3, 0.0), (1.2, -0.25, 0.35, 0.05)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build.build()
    oracle.build()


def _rms(a):
    return float(np.sqrt(np.mean(np.square(a))))


@pytest.mark.parametrize("ctl", CASES)
def test_controller_loop_matches_oracle(ctl):
    cfg, screens, R = scao_tiny_inputs()
    g = mcao.make_sim(cfg, screens, R)
    o = oracle.Sim(cfg, screens, R)
    g.step(5)
    o.step(5)
    g.set_controller(*ctl)
    o.set_controller(*ctl)
    worst = 0.0
    for _ in range(9):
        g.step(5)
        o.step(5)
        worst = max(worst, _rms(g.slopes() - o.slopes()))
    assert worst <= 1e-4
    cg, co = g.commands(), o.commands()
    assert np.linalg.norm(cg - co) / np.linalg.norm(co) <= 1e-5
    _, srg, _ = g.psf()
    _, sro, _ = o.psf()
    assert abs(srg - sro) <= 1e-3


def test_controller_batched_matches_oracle():
    cfg, _, R = scao_tiny_inputs()
    n = 2
    screens = [inputs.make_screens(cfg, realization=r) for r in range(n)]
    g = mcao.make_sim(cfg, screens, R, n_real=n)
    orc = [oracle.Sim(dict(cfg, seed=cfg["seed"] + r), screens[r], R) for r in range(n)]
    g.set_controller(*CASES[0])
    for o in orc:
        o.set_controller(*CASES[0])
    g.step(50)
    for o in orc:
        o.step(50)
    for r in range(n):
        g.set_realization(r)
        cg, co = g.commands(), orc[r].commands()
        assert np.linalg.norm(cg - co) / np.linalg.norm(co) <= 1e-5


def test_integrator_coefficients_equal_default():
    cfg, screens, R = scao_tiny_inputs()
    a = mcao.make_sim(cfg, screens, R)
    b = mcao.make_sim(cfg, screens, R)
    b.set_controller(1.0, 0.0, cfg["gain"], 0.0)
    a.step(20)
    b.step(20)
    ca, cb = a.commands(), b.commands()
    assert np.linalg.norm(ca - cb) / np.linalg.norm(ca) <= 1e-6


def test_controller_rejects_non_finite():
    cfg, screens, R = scao_tiny_inputs()
    g = mcao.make_sim(cfg, screens, R)
    with pytest.raises(mcao.McaoError):
        g.set_controller(float("nan"), 0.0, 0.5, 0.0)


def test_sodium_evolution_matches_oracle():
    from _helpers import eelt_inputs
    cfg, screens, n_cmd = eelt_inputs(10)
    R = inputs.random_reconstructor(n_cmd, 55608, 1e-4, 3)
    g = mcao.make_sim(cfg, screens, R)
    o = oracle.Sim(cfg, screens, R)
    g.step(1)
    o.step(1)
    for w in range(6):                      # the six laser stars: layer 3 km higher, 40 % thicker
        g.set_sodium(w, 93e3, 14e3)
        o.set_sodium(w, 93e3, 14e3)
    for _ in range(2):
        g.step(1)
        o.step(1)
        assert _rms(g.slopes() - o.slopes()) <= 1e-4
    with pytest.raises(mcao.McaoError):
        g.set_sodium(7, 90e3, 10e3)         # a natural star
