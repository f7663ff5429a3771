"""Tikhonov-regularised control matrix computed in FP64 on the GPU (mcao_tikhonov_reconstructor),
called through the C ABI.

R = -(D^T D + lam I)^-1 D^T with lam = alpha tr(D^T D) / n_cmd.  The oracle's definition
(oracle.tikhonov_reconstructor: the normal equations in double, solved by LAPACK) is pinned on
the CPU against the SVD filter form and the pseudo-inverse limit.  Here:

* a seeded banded matrix with zero tiles, ragged sizes and NaN in the padding columns: the FP64
  result within 1e-10 of the oracle's, the float32 result equal to it rounded once;
* the 8 m case: the GPU inversion of the oracle's own finite-difference interaction matrix equals
  the oracle's control matrix; a closed loop with the GPU's R (from the GPU's exact Jacobian)
  reaches the Strehl of the oracle's loop with the oracle's R;
* the 39 m workload (55608 x 8051 from the exact Jacobian at a flat wavefront): the FP64 normal
  equations hold to 1e-9 on sampled columns.
"""
import time

import numpy as np
import pytest

import oracle
from paper_1608_00386_gb300 import build, inputs, mcao

from _helpers import eelt_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build.build()
    oracle.build()


def _banded(n_slopes, n_cmd, seed):
    """Interaction-matrix-like D: each slope sees a band of 40 commands around a position that
    moves with the slope index (so the 64 x 64 tiles away from the band are zero), random values."""
    rng = np.random.default_rng(seed)
    D = np.zeros((n_slopes, n_cmd))
    for s in range(n_slopes):
        c0 = int(s * n_cmd / n_slopes)
        lo, hi = max(0, c0 - 20), min(n_cmd, c0 + 20)
        D[s, lo:hi] = rng.standard_normal(hi - lo)
    return D.astype(np.float32)


@pytest.mark.parametrize("n_slopes,n_cmd,alpha", [(700, 200, 1e-2), (130, 64, 1e-3), (1000, 333, 0.3)])
def test_tikhonov_matches_oracle_banded(n_slopes, n_cmd, alpha):
    import torch
    D = _banded(n_slopes, n_cmd, n_cmd)
    if n_cmd > 64:
        assert not D[:64, -64:].any()                       # at least one zero tile
    ld = n_cmd + 5
    Dp = np.full((n_slopes, ld), np.nan, np.float32)       # padding columns must never be read
    Dp[:, :n_cmd] = D
    dD = torch.from_numpy(Dp).cuda()[:, :n_cmd]
    R64, lam = mcao.tikhonov_reconstructor(dD, alpha, fp64=True)
    R32, lam32 = mcao.tikhonov_reconstructor(dD, alpha)
    ref, lam_ref = oracle.tikhonov_reconstructor(D, alpha)
    assert lam == pytest.approx(lam_ref, rel=1e-12) and lam32 == lam
    got = R64.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
    assert np.array_equal(R32.cpu().numpy(), got.astype(np.float32))     # rounded once, at the store


def test_tikhonov_of_oracle_interaction_matrix_8m():
    """The GPU inversion of the oracle's finite-difference D (an oracle output used as the
    input of both sides) equals the oracle's control matrix."""
    import torch
    cfg = inputs.scao_tiny()
    zero = [np.zeros((256, 256), np.float32)]
    o = oracle.Sim(cfg, zero)
    D = oracle.jacobian_fd(o, 1e-3)
    ref, _ = oracle.tikhonov_reconstructor(D, 1e-2)
    got, _ = mcao.tikhonov_reconstructor(torch.from_numpy(D.astype(np.float32)).cuda(), 1e-2, fp64=True)
    # the input is D rounded to float32: compare with the oracle's R of the same rounded matrix
    ref32, _ = oracle.tikhonov_reconstructor(D.astype(np.float32), 1e-2)
    assert np.max(np.abs(got.cpu().numpy() - ref32)) <= 1e-10 * np.max(np.abs(ref32))
    assert np.max(np.abs(ref32 - ref)) <= 1e-4 * np.max(np.abs(ref))


def test_tikhonov_loop_8m_reaches_oracle_strehl():
    """Closed loop with R built on the GPU from the GPU's exact Jacobian at a flat wavefront,
    against the oracle's loop with R from the oracle's finite-difference Jacobian: both close, and
    the long-exposure Strehl agrees within 1e-3 after 60 steps."""
    import torch
    cfg = inputs.scao_tiny()
    screens = inputs.make_screens(cfg)
    zero = [np.zeros_like(s) for s in screens]
    cal = mcao.Sim(cfg)
    cal.load_atmosphere(zero)
    cal.load_dms()
    Dg = cal.interaction_matrix()
    Rg, _ = mcao.tikhonov_reconstructor(Dg, 1e-2)
    cal.close()
    o = oracle.Sim(cfg, zero)
    Ro, _ = oracle.tikhonov_reconstructor(oracle.jacobian_fd(o, 1e-3), 1e-2)
    g = mcao.make_sim(cfg, screens, Rg.cpu().numpy())
    ol = oracle.Sim(cfg, screens, Ro.astype(np.float32))
    g.step(60)
    ol.step(60)
    _, srg, _ = g.psf(0, with_image=False)
    _, sro, _ = ol.psf(0)
    assert sro > 0.3                          # the loop closes (open loop: about 0.003)
    assert abs(srg - sro) <= 1e-3


def test_tikhonov_full_size_normal_equations():
    """The 39 m workload's exact Jacobian at a flat wavefront (55608 x 8051): the FP64 result
    satisfies (D^T D + lam I) r_s = -d_s to 1e-9 relative on 64 sampled columns s."""
    import torch
    cfg, _, n_cmd = eelt_inputs(10)
    sim = mcao.Sim(cfg)
    sim.load_atmosphere([torch.zeros((l["n"], l["n"]), device="cuda") for l in cfg["layers"]])
    sim.load_dms()
    D = sim.interaction_matrix()
    sim.close()
    torch.cuda.synchronize()
    t0 = time.time()
    R, lam = mcao.tikhonov_reconstructor(D, 1e-2, fp64=True)
    torch.cuda.synchronize()
    elapsed = time.time() - t0
    assert lam > 0.0
    D64 = D.double()
    g = torch.Generator(device="cuda").manual_seed(3)
    cols = torch.randint(0, D.shape[0], (64,), generator=g, device="cuda")
    r = R[:, cols]                                          # [n_cmd][64]
    res = D64.t() @ (D64 @ r) + lam * r + D64[cols].t()     # (D^T D + lam I) r + d
    scale = D64[cols].norm(dim=1)
    rel = (res.norm(dim=0) / scale).max().item()
    assert rel <= 1e-9, rel
    # the float32 matrix is the FP64 one rounded once
    R32, _ = mcao.tikhonov_reconstructor(D, 1e-2)
    assert torch.equal(R32, R.float())
    print(f"39 m Tikhonov control matrix: {elapsed:.2f} s, lambda {lam:.4g}, max rel residual {rel:.2e}")
