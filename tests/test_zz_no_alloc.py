"""The allocation-free reconstructor update (mcao_reconstruct_noalloc), called through the C ABI.

Some callers cannot allocate device memory while they run (a controller that reserves its memory
once at start-up, or code living inside another framework's memory pool); this entry point keeps
its split-K scratch in a fixed array inside the library instead.  It is checked against the
update the closed loop itself applies and against c + g R s formed in float64, on two calls in a
row (the shared scratch keeps the previous call's partial sums), at sizes with several column
chunks, a ragged last chunk, a row count that is not a multiple of the row block and NaN in the
caller's padding columns.  The file is named so that pytest collects it last."""
import numpy as np
import pytest

from paper_1608_00386_gb300 import build, mcao

from _helpers import scao_tiny_inputs

pytestmark = pytest.mark.gpu


def test_noalloc_update_matches_the_loop_update_on_two_calls():
    import torch
    build.build()
    cfg, screens, R = scao_tiny_inputs()
    loop = mcao.make_sim(cfg, screens, R)
    dR = torch.from_numpy(R).cuda()
    c = torch.zeros(R.shape[0], dtype=torch.float32, device="cuda")
    for _ in range(2):
        loop.step(1)                                  # c_{k+1} = c_k + g R s_k inside the loop
        s = torch.from_numpy(loop.slopes()).cuda()    # the s_k that update used
        mcao.reconstruct_noalloc(dR, s, c, cfg["gain"])
        torch.cuda.synchronize()
        ref = loop.commands().astype(np.float64)
        got = c.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5


@pytest.mark.parametrize("n_cmd,n_slopes,ld", [(1001, 10001, 10004), (37, 4099, 4104), (8051, 55608, 55612)])
def test_noalloc_matches_float64_product_with_nan_padding(n_cmd, n_slopes, ld):
    """Several column chunks (3, 2 and 14), a last chunk shorter than the others, 1-3 columns
    left after the last whole 16-byte vector, rows past n_cmd in the last row block, and NaN
    in the padding columns n_slopes..ld-1, which must never enter a sum."""
    import torch
    build.build()
    g = torch.Generator(device="cuda").manual_seed(n_cmd + n_slopes)
    Rp = torch.randn((n_cmd, ld), generator=g, device="cuda", dtype=torch.float32) * 0.01
    Rp[:, n_slopes:] = float("nan")
    R = Rp[:, :n_slopes]                              # row stride ld, unit column stride
    c = torch.randn(n_cmd, generator=g, device="cuda", dtype=torch.float32)
    ref = c.double()
    R64 = R.double()
    gain = 0.37
    for _ in range(2):
        s = torch.randn(n_slopes, generator=g, device="cuda", dtype=torch.float32)
        mcao.reconstruct_noalloc(R, s, c, gain)
        ref = ref + gain * (R64 @ s.double())
        torch.cuda.synchronize()
        assert bool(torch.isfinite(c).all())
        err = (c.double() - ref).norm() / ref.norm()
        assert float(err) <= 1e-5
        assert float((c.double() - ref).abs().max()) <= 1e-5 * float(ref.abs().max())


def test_noalloc_rejects_bad_arguments_and_sizes_beyond_its_scratch():
    import torch
    build.build()
    R = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    s = torch.zeros(4, dtype=torch.float32, device="cuda")
    c = torch.zeros(4, dtype=torch.float32, device="cuda")
    big = mcao.lib().mcao_reconstruct_noalloc
    buf = mcao.C.create_string_buffer(256)
    # 600000 rows x 1 chunk exceeds the 524288 partial sums: rejected before any launch
    st = big(R.data_ptr(), 600000, 4, 4, s.data_ptr(), c.data_ptr(), 0.5, None, buf, 256)
    assert st == 2 and b"scratch" in buf.value
    # 70000 column chunks of 4096 for 2 rows fit the scratch but not the launch grid
    st = big(R.data_ptr(), 2, 4096 * 70000, 4096 * 70000, s.data_ptr(), c.data_ptr(), 0.5, None, buf, 256)
    assert st == 2 and b"65535" in buf.value
    # the binding checks what the C ABI cannot see
    with pytest.raises(mcao.McaoError):
        mcao.reconstruct_noalloc(R.double(), s, c, 0.5)
    with pytest.raises(mcao.McaoError):
        mcao.reconstruct_noalloc(R, s, c[:3], 0.5)
    with pytest.raises(mcao.McaoError):
        mcao.reconstruct_noalloc(R.t(), s, c, 0.5)
