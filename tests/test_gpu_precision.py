"""Reduced-precision reconstructor (bfloat16; FP8 E4M3 with per-row scales) through the C ABI.

The codes are byte work: they must equal the oracle's quantizer bit for bit.  The loop itself
is compared with the oracle running the same format (the oracle's product is in double over
the represented values, the library's in float32), with the float32 path's tolerances: slopes
1e-4 pixel RMS, commands 1e-5 relative, long-exposure Strehl 1e-3 absolute.  Against the
float32 loop, the long-exposure Strehl may move by at most 1 % (the comparison the
reduced formats are measured by).
"""
import numpy as np
import pytest

import oracle
from paper_1608_00386_gb300 import build, inputs, mcao

from _helpers import eelt_inputs, scao_tiny_inputs

pytestmark = pytest.mark.gpu

DTYPES = [mcao.DTYPE_BF16, mcao.DTYPE_FP8_E4M3]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build.build()
    oracle.build()


def _rms(a):
    return float(np.sqrt(np.mean(np.square(a))))


@pytest.mark.parametrize("dtype", DTYPES)
def test_quantized_codes_bit_exact(dtype):
    import torch
    rng = np.random.default_rng(21)
    rows, cols, ld = 37, 304, 320
    R = (rng.normal(0, 1e-2, (rows, ld)) * rng.uniform(0.01, 50, (rows, 1))).astype(np.float32)
    R[3, :] = 0.0
    R[7, :cols] = 0.0
    R[5, 11] = 1e-30            # below every format's resolution after scaling
    R[11, :] = 0.0
    R[11, 7] = -4e-40           # the row's max / 448 underflows: scale 1, codes zero (not 0 / 0)
    R[13, :] = 0.0
    R[13, 3] = 3e-36            # max / 448 just below the smallest normal float
    R[9, 2] = -3.0e5            # dominates its row
    R[:, cols:] = 1e30          # outside the quantized columns: must not reach the scales
    d = torch.from_numpy(R).cuda()
    codes, scales = mcao.quantize_rows(d[:, :cols], dtype)
    torch.cuda.synchronize()
    ref_codes, ref_scales = oracle.quantize_rows(R[:, :cols], dtype)
    got = codes.cpu().numpy().view(ref_codes.dtype)
    assert np.array_equal(got, ref_codes)
    if dtype == mcao.DTYPE_FP8_E4M3:
        assert np.array_equal(scales.cpu().numpy(), ref_scales)


def test_quantize_rows_rejects_bad_shapes():
    import torch
    d = torch.zeros((4, 20), device="cuda")
    with pytest.raises(mcao.McaoError):
        mcao.quantize_rows(d, mcao.DTYPE_BF16)          # 20 is not a multiple of 8
    with pytest.raises(mcao.McaoError):
        mcao.quantize_rows(d[:, :16], 7)                 # unknown format


@pytest.mark.parametrize("dtype", DTYPES)
def test_closed_loop_scao_reduced_precision(dtype):
    cfg, screens, R = scao_tiny_inputs()
    g = mcao.make_sim(cfg, screens, R, r_dtype=dtype)
    o = oracle.Sim(cfg, screens, R, r_dtype=dtype)
    worst = 0.0
    for _ in range(5):
        g.step(10)
        o.step(10)
        worst = max(worst, _rms(g.slopes() - o.slopes()))
    assert worst <= 1e-4
    cg, co = g.commands(), o.commands()
    assert np.linalg.norm(cg - co) / np.linalg.norm(co) <= 1e-5
    _, srg, _ = g.psf()
    _, sro, _ = o.psf()
    assert abs(srg - sro) <= 1e-3


@pytest.mark.parametrize("dtype", DTYPES)
def test_eelt_reduced_precision_steps(dtype):
    cfg, screens, n_cmd = eelt_inputs(10)
    R = inputs.random_reconstructor(n_cmd, 55608, 1e-4, 3)
    g = mcao.make_sim(cfg, screens, R, r_dtype=dtype)
    o = oracle.Sim(cfg, screens, R, r_dtype=dtype)
    for _ in range(2):
        g.step(1)
        o.step(1)
        assert _rms(g.slopes() - o.slopes()) <= 1e-4
    cg, co = g.commands(), o.commands()
    assert np.linalg.norm(cg - co) / np.linalg.norm(co) <= 1e-5


@pytest.mark.parametrize("dtype", DTYPES)
def test_strehl_within_one_percent_of_float32(dtype):
    """The corrected 8 m loop over 100 steps: long-exposure Strehl with the reduced format
    within 1 % (relative) of the float32 loop's."""
    cfg, screens, R = scao_tiny_inputs()
    ref = mcao.make_sim(cfg, screens, R)
    red = mcao.make_sim(cfg, screens, R, r_dtype=dtype)
    ref.step(100)
    red.step(100)
    _, sr_ref, _ = ref.psf()
    _, sr_red, _ = red.psf()
    assert abs(sr_red - sr_ref) <= 0.01 * sr_ref
