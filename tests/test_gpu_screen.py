"""Phase screens generated on the device (mcao_generate_screen, "The atmospheric layers
generation") against the oracle's FFT-method screens from the same Philox coefficients:
element by element within float32 FFT rounding (max |diff| <= 1e-4 of the screen RMS), across
radix-2/3/5 sizes, odd sizes and the largest size; and a closed loop on device-generated layers
against the oracle on its own screens."""
import numpy as np
import pytest

import oracle
from paper_1608_00386_gb300 import build, inputs, mcao

from _helpers import scao_tiny_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build.build()
    oracle.build()


@pytest.mark.parametrize("n,pixel,r0,L0,seed", [
    (2, 0.5, 0.2, 20.0, 3),
    (64, 0.1, 0.15, 25.0, 1),
    (75, 0.08, 0.1, 10.0, 2),          # 3 * 5^2: odd size, no radix 2
    (96, 0.1, 0.15, 25.0, 0x1234_5678_9ABC),  # seed above 32 bits
    (120, 0.05, 0.3, 40.0, 7),
    (250, 0.04, 0.15, 25.0, 11),
    (1024, 0.05, 0.157, 25.0, 5),
    (4096, 0.025, 0.157, 25.0, 9),     # largest size
])
def test_screen_matches_oracle(n, pixel, r0, L0, seed):
    import torch
    got = mcao.generate_screen(n, pixel, r0, L0, seed)
    torch.cuda.synchronize()
    got = got.cpu().numpy().astype(np.float64)
    want = oracle.phase_screen(n, pixel, r0, L0, seed)
    rms = float(np.sqrt(np.mean(want ** 2)))
    assert rms > 0
    err = np.abs(got - want)
    assert err.max() <= 1e-4 * rms, (err.max() / rms)
    assert np.sqrt(np.mean(err ** 2)) <= 1e-5 * rms


def test_screen_seed_and_stream_order():
    import torch
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = mcao.generate_screen(128, 0.1, 0.15, 25.0, 42, stream=s)
        b = mcao.generate_screen(128, 0.1, 0.15, 25.0, 42, stream=s)
        c = mcao.generate_screen(128, 0.1, 0.15, 25.0, 43, stream=s)
    s.synchronize()
    assert torch.equal(a, b)
    assert not torch.allclose(a, c)
    assert float(a.double().mean().abs()) < 1e-5 * float(a.double().std())


def test_closed_loop_on_generated_layers_matches_oracle():
    # noise off: the two sides' screens differ by float32 FFT rounding, which may flip photon
    # counts; the deterministic loop is compared within float32 tolerances
    cfg, _, R = scao_tiny_inputs()
    cfg = dict(cfg, noise=False)
    g = mcao.Sim(cfg)
    scr = g.generate_atmosphere()
    g.load_dms()
    g.load_reconstructor(R)
    ref = [oracle.phase_screen(l["n"], l["pixel"], l["r0"], l["L0"], l["seed"]) for l in cfg["layers"]]
    for a, b in zip(scr, ref):
        assert np.abs(a.cpu().numpy() - b).max() <= 1e-4 * np.sqrt(np.mean(b ** 2))
    o = oracle.Sim(cfg, [r.astype(np.float32) for r in ref], R)
    g.step(10)
    o.step(10)
    ds = g.slopes() - o.slopes()
    assert float(np.sqrt(np.mean(ds ** 2))) < 1e-4
    c_o = o.commands()
    assert np.abs(g.commands() - c_o).max() <= 1e-5 * np.abs(c_o).max() + 1e-7
    o.close()
