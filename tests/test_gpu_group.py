"""Group stepping (mcao_step_group): simulations of different configurations advanced by one
graph launch per step give bit-identical slopes and commands to stepping each alone; the
argument checks."""
import numpy as np
import pytest

import oracle
from paper_1608_00386_gb300 import build, inputs, mcao

from _helpers import mcao_small, scao_tiny_inputs, wide_lgs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build.build()
    oracle.build()


def _make():
    cfg0, screens0, R0 = scao_tiny_inputs()
    sims = [mcao.make_sim(dict(cfg0, noise=True), screens0, R0)]
    # a batched member: two realizations with a bfloat16 reconstructor
    scr2 = [screens0, inputs.make_screens(cfg0, realization=1)]
    sims.append(mcao.make_sim(dict(cfg0, noise=True), scr2, R0, r_dtype=mcao.DTYPE_BF16, n_real=2))
    for k, cfg in enumerate((dict(mcao_small(), noise=True), wide_lgs())):
        screens = inputs.make_screens(cfg)
        n_cmd = inputs.n_commands(cfg)
        g = mcao.Sim(cfg)
        n_slopes = g.query(mcao.Q_SLOPES)
        g.close()
        R = inputs.random_reconstructor(n_cmd, n_slopes, 0.02, 5 + k)
        sims.append(mcao.make_sim(cfg, screens, R))
    return sims


def test_group_step_is_bit_identical_to_single_steps():
    a = _make()
    b = _make()
    mcao.step_group(a, 4)
    mcao.step_group(a, 3)
    for s in b:
        s.step(7)
    for x, y in zip(a, b):
        assert x.step_index == y.step_index == 7
        for r in range(x.query(mcao.Q_REALIZATIONS)):
            x.set_realization(r)
            y.set_realization(r)
            assert np.array_equal(x.slopes(), y.slopes())
            assert np.array_equal(x.commands(), y.commands())
            q1, q2 = x.psf(0, with_image=False), y.psf(0, with_image=False)
            assert q1[1:] == q2[1:]


def test_group_step_argument_checks():
    sims = _make()
    with pytest.raises(mcao.McaoError):
        mcao.step_group([sims[0], sims[0]], 1)
    sims[1].set_profiling(True)
    with pytest.raises(mcao.McaoError):
        mcao.step_group(sims, 1)
    sims[1].set_profiling(False)
    mcao.step_group(sims, 0)
    mcao.step_group(sims, 1)
    assert all(s.step_index == 1 for s in sims)


def test_read_async_matches_synchronous_reads():
    import torch
    cfg, screens, R = scao_tiny_inputs()
    g = mcao.make_sim(dict(cfg, noise=True), screens, R)
    n = g.query(mcao.Q_COMMANDS)
    ring_c = torch.zeros((4, n), dtype=torch.float32).pin_memory()
    ring_s = torch.zeros((4, 1, 2), dtype=torch.float64).pin_memory()
    ref = []
    for k in range(4):
        g.step(1)
        g.read_async(ring_c[k], ring_s[k])
    g.sync()
    h = mcao.make_sim(dict(cfg, noise=True), screens, R)
    for k in range(4):
        h.step(1)
        _, sl, sn = h.psf(0, with_image=False)
        assert np.array_equal(ring_c[k].numpy(), h.commands())
        assert ring_s[k, 0, 0].item() == sl and ring_s[k, 0, 1].item() == sn
    with pytest.raises(mcao.McaoError):
        g.read_async(None, None)


def test_read_async_ring_reuse_and_partial_reads():
    """More reads in flight than the 64 device ring slots (a slot is reused once its copy is
    done) and reads of the commands or the Strehl ratios alone: every value equals the
    synchronous reads of a twin run."""
    import torch
    cfg, screens, R = scao_tiny_inputs()
    cfg = dict(cfg, noise=True)
    g = mcao.make_sim(cfg, screens, R)
    n = g.query(mcao.Q_COMMANDS)
    steps = 150
    ring_c = torch.zeros((steps, n), dtype=torch.float32).pin_memory()
    ring_s = torch.zeros((steps, 1, 2), dtype=torch.float64).pin_memory()
    for k in range(steps):
        g.step(1)
        if k % 3 == 0:
            g.read_async(ring_c[k], ring_s[k])
        elif k % 3 == 1:
            g.read_async(ring_c[k], None)
        else:
            g.read_async(None, ring_s[k])
    g.sync()
    h = mcao.make_sim(cfg, screens, R)
    for k in range(steps):
        h.step(1)
        _, sl, sn = h.psf(0, with_image=False)
        if k % 3 != 2:
            assert np.array_equal(ring_c[k].numpy(), h.commands()), k
        if k % 3 != 1:
            assert ring_s[k, 0, 0].item() == sl and ring_s[k, 0, 1].item() == sn, k
