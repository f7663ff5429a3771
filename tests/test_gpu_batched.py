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
    """bfloat16 reconstructor in the batched product (tensor cores, float32 slopes, float32
    accumulation): long-exposure Strehl within 1 % of the float32 batch."""
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


# ------------------------------------------------------------------------------------------ product
def _eelt_product_sim(n_real, dtype, seed):
    """39 m configuration with n_real realizations, DMs and a random R on the device (no
    atmosphere: the product needs only the reconstructor).  For bfloat16 the float32 entries
    have their low 16 bits cleared, so R is exactly representable and the stored codes are R."""
    import torch
    cfg, _, n_cmd = eelt_inputs(10)
    g = torch.Generator(device="cuda").manual_seed(seed)
    R = torch.randn((n_cmd, 55608), generator=g, device="cuda", dtype=torch.float32)
    if dtype == mcao.DTYPE_BF16:
        R = (R.view(torch.int32) & -65536).view(torch.float32)
    sim = mcao.Sim(cfg, n_real=n_real)
    sim.load_dms()
    sim.load_reconstructor(R, dtype=dtype)
    return sim, R, g


@pytest.mark.parametrize("dtype,n_real,n_rhs", [(mcao.DTYPE_BF16, 2, 1), (mcao.DTYPE_BF16, 16, 16),
                                                (mcao.DTYPE_BF16, 17, 17), (mcao.DTYPE_BF16, 64, 64),
                                                (mcao.DTYPE_BF16, 80, 80), (mcao.DTYPE_F32, 17, 17)])
def test_batched_product_full_size_matches_float64(dtype, n_real, n_rhs):
    """The batched step's product at the 39 m size (8051 x 55608) against a float64 product:
    bfloat16 R on the tensor cores with float32 slopes (1, 16, 17 and 64 realizations in one pass
    over R, 80 in two passes), float32 R on the CUDA cores in groups of 16.  Each element within
    1e-5 |R_i| |s_r| (float32 accumulation), which also bounds the whole-vector error."""
    import torch
    sim, R, g = _eelt_product_sim(n_real, dtype, 100 + n_rhs)
    S = torch.randn((n_rhs, 55608), generator=g, device="cuda", dtype=torch.float32)
    for _ in range(2):                                  # a second call reuses every scratch buffer
        D = sim.reconstruct_batch(S)
        ref = (S.double() @ R.double().t())             # [n_rhs][n_cmd]
        bound = 1e-5 * S.double().norm(dim=1)[:, None] * R.double().norm(dim=1)[None, :]
        err = (D.double() - ref).abs()
        assert bool((err <= bound).all()), float((err / bound).max())
        rel = float((D.double() - ref).norm() / ref.norm())
        assert rel <= 1e-5
        S = S.flip(0).contiguous()


def _bf16_loop_against_oracle(n, steps):
    # The 8 m loop passes a sensitive transient near step 30 (an edge actuator's command swings
    # from -200 to -129 rad) where even the single-realization float32 loop differs from the oracle
    # by 1.2e-5 relative; at 10, 20 and 50 steps every path is within 1.5e-6.  The comparisons
    # are made away from it.
    cfg, _, R = scao_tiny_inputs()
    g, screens = _batch(cfg, R, n, r_dtype=mcao.DTYPE_BF16)
    orc = [oracle.Sim(dict(cfg, seed=cfg["seed"] + r), screens[r], R, r_dtype=oracle.DTYPE_BF16) for r in range(n)]
    g.step(steps)
    for o in orc:
        o.step(steps)
    for r in range(n):
        g.set_realization(r)
        assert _rms(g.slopes() - orc[r].slopes()) <= 1e-4, r
        cg, co = g.commands(), orc[r].commands()
        assert np.linalg.norm(cg - co) / np.linalg.norm(co) <= 1e-5, r
        _, srg, _ = g.psf()
        _, sro, _ = orc[r].psf()
        assert abs(srg - sro) <= 1e-3, r


def test_batched_bf16_loop_17_realizations_matches_oracle_bf16():
    """17 realizations (more than one 16-wide group) with a bfloat16 R, every realization against
    the oracle's bfloat16 variant (represented values of R, float slopes, double product) run
    alone on its inputs, at the float32 tolerances."""
    _bf16_loop_against_oracle(17, 50)


def test_batched_bf16_loop_64_realizations_matches_oracle_bf16():
    """The batched configuration's 64 realizations with a bfloat16 R, every realization against
    the oracle's bfloat16 variant."""
    _bf16_loop_against_oracle(64, 12)


def test_batched_f32_loop_17_realizations_matches_oracle():
    """17 realizations with a float32 R (two passes of the CUDA-core product), every realization
    against the oracle."""
    cfg, _, R = scao_tiny_inputs()
    n = 17
    g, screens = _batch(cfg, R, n)
    orc = [oracle.Sim(dict(cfg, seed=cfg["seed"] + r), screens[r], R) for r in range(n)]
    g.step(20)
    for o in orc:
        o.step(20)
    for r in range(n):
        g.set_realization(r)
        assert _rms(g.slopes() - orc[r].slopes()) <= 1e-4, r
        cg, co = g.commands(), orc[r].commands()
        assert np.linalg.norm(cg - co) / np.linalg.norm(co) <= 1e-5, r


def test_reconstruct_batch_checks_its_arguments():
    import torch
    cfg, _, R = scao_tiny_inputs()
    g, _ = _batch(cfg, R, 2)
    S = torch.zeros((3, 416), device="cuda")
    with pytest.raises(mcao.McaoError):
        g.reconstruct_batch(S)                       # more vectors than realizations
    with pytest.raises(mcao.McaoError):
        g.reconstruct_batch(torch.zeros((2, 415), device="cuda"))
    one = mcao.make_sim(cfg, inputs.make_screens(cfg), R)
    with pytest.raises(mcao.McaoError):
        one.reconstruct_batch(torch.zeros((1, 416), device="cuda"))


def test_batched_product_fp8_full_size_matches_oracle_dequantized():
    """FP8 E4M3 R in the batched product (code values on the tensor cores, row scales after the
    sum), 17 realizations at the 39 m size, against float64 products of the oracle's own
    quantization of R (codes and per-row scales): every element within 1e-5 |R_i||s_r|."""
    import torch
    cfg, _, n_cmd = eelt_inputs(10)
    g = torch.Generator(device="cuda").manual_seed(71)
    R = torch.randn((n_cmd, 55608), generator=g, device="cuda", dtype=torch.float32) * 0.01
    sim = mcao.Sim(cfg, n_real=17)
    sim.load_dms()
    sim.load_reconstructor(R, dtype=mcao.DTYPE_FP8_E4M3)
    codes, scales = oracle.quantize_rows(R.cpu().numpy(), oracle.DTYPE_FP8_E4M3)
    Rq = torch.from_numpy(oracle.dequantize_rows(codes, scales, oracle.DTYPE_FP8_E4M3)).cuda()
    del codes
    S = torch.randn((17, 55608), generator=g, device="cuda", dtype=torch.float32)
    D = sim.reconstruct_batch(S).double()
    ref = S.double() @ Rq.double().t()
    bound = 1e-5 * S.double().norm(dim=1)[:, None] * Rq.double().norm(dim=1)[None, :]
    assert bool(((D - ref).abs() <= bound).all())
    assert float((D - ref).norm() / ref.norm()) <= 1e-5


def test_batched_fp8_loop_17_realizations_matches_oracle_fp8():
    """17 realizations with an FP8 E4M3 R, every realization against the oracle's FP8 variant
    (the represented values scale x code, float slopes, double product) at the float32
    tolerances."""
    cfg, _, R = scao_tiny_inputs()
    n = 17
    g, screens = _batch(cfg, R, n, r_dtype=mcao.DTYPE_FP8_E4M3)
    orc = [oracle.Sim(dict(cfg, seed=cfg["seed"] + r), screens[r], R, r_dtype=oracle.DTYPE_FP8_E4M3)
           for r in range(n)]
    g.step(50)
    for o in orc:
        o.step(50)
    for r in range(n):
        g.set_realization(r)
        assert _rms(g.slopes() - orc[r].slopes()) <= 1e-4, r
        cg, co = g.commands(), orc[r].commands()
        assert np.linalg.norm(cg - co) / np.linalg.norm(co) <= 1e-5, r
