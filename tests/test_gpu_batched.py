"""Several Monte-Carlo realizations advanced together (cfg.n_real > 1) through the C ABI.

Realization r has its own screens (layer seeds + 1000 r), its own noise key (seed + r) and its
own commands, slopes and accumulators; the reconstructor is shared and the product of all
realizations is one matrix product.  Each realization must match the oracle run alone on its
inputs (float32 tolerances: slopes 1e-4 pixel RMS, commands 1e-5 relative, Strehl 1e-3), the
noise frames must be bit-exact given the intensities, and a realization inside the batch must
match the same realization simulated alone.
"""
import numpy as np
import pytest

import oracle
from paper_1608_00386_gb300 import build, inputs, mcao

from _helpers import eelt_inputs, scao_tiny_inputs

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


def _batch(cfg, R, n, **kw):
    screens = [inputs.make_screens(cfg, realization=r) for r in range(n)]
    return mcao.make_sim(cfg, screens, R, n_real=n, **kw), screens


def test_batched_realizations_match_oracle():
    cfg, _, R = scao_tiny_inputs()
    n = 3
    g, screens = _batch(cfg, R, n)
    assert g.query(mcao.Q_REALIZATIONS) == n
    orc = [oracle.Sim(dict(cfg, seed=cfg["seed"] + r), screens[r], R) for r in range(n)]
    for _ in range(10):
        g.step(10)
        for o in orc:
            o.step(10)
        for r in range(n):
            g.set_realization(r)
            assert _rms(g.slopes() - orc[r].slopes()) <= 1e-4
    srs = []
    for r in range(n):
        g.set_realization(r)
        cg, co = g.commands(), orc[r].commands()
        assert np.linalg.norm(cg - co) / np.linalg.norm(co) <= 1e-5
        _, srg, _ = g.psf()
        _, sro, _ = orc[r].psf()
        assert abs(srg - sro) <= 1e-3
        srs.append(srg)
    assert len(set(np.round(srs, 6))) == n    # independent realizations differ


def test_batched_noise_frames_bit_exact():
    cfg, _, R = scao_tiny_inputs()
    cfg = dict(cfg, noise=True)
    n = 2
    g, screens = _batch(cfg, R, n, keep_frames=True)
    g.step(2)
    wfs = 0
    for r in range(n):
        g.set_realization(r)
        lam, frames = g.frames(wfs)
        k = g.step_index - 1
        ww = cfg["wfs"][wfs]
        ref = oracle.noise_frame(lam.ravel(), ww["read_noise"], 0, k, wfs, cfg["seed"] + r,
                                 frame_px=(ww["n_fft"] // ww["n_bin"]) ** 2)
        assert np.array_equal(frames.ravel(), ref)


def test_realization_in_batch_equals_alone():
    cfg, _, R = scao_tiny_inputs()
    g, screens = _batch(cfg, R, 3)
    alone = mcao.make_sim(dict(cfg, seed=cfg["seed"] + 2), screens[2], R)
    g.step(100)
    alone.step(100)
    g.set_realization(2)
    assert _rms(g.slopes() - alone.slopes()) <= 1e-5
    ca, cb = g.commands(), alone.commands()
    assert np.linalg.norm(ca - cb) / np.linalg.norm(cb) <= 1e-5


def test_batched_full_size_step():
    cfg, _, n_cmd = eelt_inputs(10)
    R = inputs.random_reconstructor(n_cmd, 55608, 1e-4, 3)
    g, screens = _batch(cfg, R, 2)
    o = oracle.Sim(dict(cfg, seed=cfg["seed"] + 1), screens[1], R)
    for _ in range(2):
        g.step(1)
        o.step(1)
    g.set_realization(1)
    assert _rms(g.slopes() - o.slopes()) <= 1e-4
    cg, co = g.commands(), o.commands()
    assert np.linalg.norm(cg - co) / np.linalg.norm(co) <= 1e-5


def test_batched_bf16_strehl_within_one_percent():
    """bfloat16 reconstructor and bfloat16 slopes in the batched product (tensor-core matrix
    product, float32 accumulation): long-exposure Strehl within 1 % of the float32 batch."""
    cfg, _, R = scao_tiny_inputs()
    n = 2
    ref, _ = _batch(cfg, R, n)
    red, _ = _batch(cfg, R, n, r_dtype=mcao.DTYPE_BF16)
    ref.step(100)
    red.step(100)
    for r in range(n):
        ref.set_realization(r)
        red.set_realization(r)
        _, a, _ = ref.psf()
        _, b, _ = red.psf()
        assert abs(b - a) <= 0.01 * a


def test_checkpoint_covers_all_realizations():
    cfg, _, R = scao_tiny_inputs()
    g, screens = _batch(cfg, R, 2)
    g.step(5)
    blob = g.get_state()
    g.set_realization(1)
    c5 = g.commands()
    g.step(5)
    g.set_state(blob)
    g.step(5)
    h, _ = _batch(cfg, R, 2)
    h.step(10)
    for r in range(2):
        g.set_realization(r)
        h.set_realization(r)
        assert np.array_equal(g.commands(), h.commands())
    assert c5.shape == g.commands().shape


def test_realization_index_checked():
    cfg, _, R = scao_tiny_inputs()
    g, _ = _batch(cfg, R, 2)
    with pytest.raises(mcao.McaoError):
        g.set_realization(2)
    with pytest.raises(mcao.McaoError):
        g.set_realization(-1)
