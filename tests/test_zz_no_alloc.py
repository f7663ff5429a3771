"""The allocation-free reconstructor update (mcao_reconstruct_noalloc), called through the C ABI,
against the update the closed loop itself applies.

Some callers cannot allocate device memory while they run (a controller that reserves its memory
once at start-up, or code living inside another framework's memory pool); this entry point keeps
its split-K scratch in a fixed array inside the library instead.  The file is named so that pytest
collects it last."""
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


def test_noalloc_rejects_sizes_beyond_its_scratch():
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
