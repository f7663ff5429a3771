"""Wide-field laser star on the block-per-subaperture FFT route (16 samples per subaperture,
FFT 32, bin 2, elongated spots from a side launch) through the C ABI against the oracle:
noise-free intensities and slopes, bit-exact noise given the intensities, a short noisy loop,
the interaction matrix, and a sodium-layer update."""
import numpy as np
import pytest

import oracle
from paper_1608_00386_gb300 import build, inputs, mcao

from _helpers import wide_lgs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build.build()
    oracle.build()


def _rms(a):
    return float(np.sqrt(np.mean(np.square(a))))


def _sims(noise=False, keep_frames=False):
    cfg = dict(wide_lgs(), noise=noise)
    screens = inputs.make_screens(cfg)
    n_cmd = inputs.n_commands(cfg)
    o = oracle.Sim(cfg, screens)
    R = inputs.random_reconstructor(n_cmd, o.n_slopes, 0.02, 4)
    o.close()
    g = mcao.make_sim(cfg, screens, R, keep_frames=keep_frames)
    o = oracle.Sim(cfg, screens, R)
    return cfg, g, o


def test_wide_lgs_uses_elongation_and_matches_oracle():
    cfg, g, o = _sims(keep_frames=True)
    sig, _ = o.elongation(0)
    assert sig.max() > 2.0                           # visibly elongated spots
    for _ in range(3):
        g.step(1)
        o.step(1)
        assert _rms(g.slopes() - o.slopes()) <= 1e-4
    lam_g, _ = g.frames(0)
    lam_o, _ = o.frames(0)
    assert np.abs(lam_g - lam_o).max() <= 1e-4 * lam_o.max()
    c_o = o.commands()
    assert np.abs(g.commands() - c_o).max() <= 1e-5 * np.abs(c_o).max() + 1e-7


def test_wide_lgs_noise_bit_exact_given_lambda_and_noisy_loop():
    cfg, g, o = _sims(noise=True, keep_frames=True)
    g.step(2)
    o.step(2)
    lam, fr = g.frames(0)
    w = cfg["wfs"][0]
    ref = oracle.noise_frame(lam.ravel(), w["read_noise"], 0, 1, 0, cfg["seed"], frame_px=(w["n_fft"] // w["n_bin"]) ** 2)
    assert np.array_equal(fr.ravel(), ref)
    _, fo = o.frames(0)
    flips = int(np.sum(fr != fo))
    assert flips <= max(3, fr.size // 2000)
    assert _rms(g.slopes() - o.slopes()) <= 3e-4 * max(1, flips)


def test_wide_lgs_interaction_matrix_and_sodium_update():
    cfg, g, o = _sims()
    Dg = g.interaction_matrix().cpu().numpy().astype(np.float64)
    Do = oracle.jacobian_fd(o, 1e-3)
    assert np.linalg.norm(Dg - Do) <= 1e-5 * np.linalg.norm(Do)
    g.set_sodium(0, 95e3, 8e3)
    o.set_sodium(0, 95e3, 8e3)
    g.step(2)
    o.step(2)
    assert _rms(g.slopes() - o.slopes()) <= 1e-4
