"""Derivatives of the noise-free sensing through the C ABI against the oracle's central
differences (fp64, h = 1e-3 rad, O(h^2) truncation far below the float32 bar): the interaction
matrix (mcao_interaction_matrix), command and pupil-phase vector-Jacobian products
(mcao_slopes_vjp), the autograd function built on them, and the noise-free measurement."""
import numpy as np
import pytest

import oracle
from paper_1608_00386_gb300 import build, inputs, mcao

from _helpers import mcao_small, scao_tiny_inputs

pytestmark = pytest.mark.gpu

# float32 forward and adjoint (FFTs of 16..64 points: about 2 log2 N roundings of 6e-8 per
# value, a few hundred terms per centroid sum) against fp64 central differences: relative
# Frobenius error of the matrix, and largest element error over the largest element
# (measured 2.4e-7 / 8.5e-7 on the 8 m cases)
TOL_FRO, TOL_MAX = 1e-5, 2e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build.build()
    oracle.build()


def _case(name, seed=1):
    if name == "scao_tiny":
        cfg, screens, _ = scao_tiny_inputs()
        cfg = dict(cfg, noise=False)
    else:
        cfg = mcao_small()
        screens = inputs.make_screens(cfg)
    g = mcao.Sim(cfg)
    g.load_atmosphere(screens)
    g.load_dms()
    o = oracle.Sim(cfg, screens)
    c = np.random.default_rng(seed).normal(0.0, 0.3, o.n_cmd).astype(np.float32)
    g.set_commands(c)
    o.set_commands(c.astype(np.float64))
    return cfg, g, o


@pytest.mark.parametrize("name", ["scao_tiny", "mcao_small"])
def test_noise_free_measure_matches_oracle(name):
    _, g, o = _case(name)
    k0 = g.step_index
    s = g.measure()
    assert g.step_index == k0
    assert float(np.sqrt(np.mean((s - o.measure()) ** 2))) <= 1e-4


@pytest.mark.parametrize("name", ["scao_tiny", "mcao_small"])
def test_interaction_matrix_matches_oracle(name):
    _, g, o = _case(name)
    Dg = g.interaction_matrix().cpu().numpy().astype(np.float64)
    Do = oracle.jacobian_fd(o, 1e-3)
    n = np.linalg.norm
    assert n(Dg - Do) <= TOL_FRO * n(Do), n(Dg - Do) / n(Do)
    assert np.abs(Dg - Do).max() <= TOL_MAX * np.abs(Do).max()


def test_interaction_matrix_after_steps_matches_oracle():
    # frozen flow moved the layers (step 3) and the loop changed the commands
    cfg, screens, R = scao_tiny_inputs()
    cfg = dict(cfg, noise=False)
    g = mcao.make_sim(cfg, screens, R)
    o = oracle.Sim(cfg, screens, R)
    g.step(3)
    o.step(3)
    c = g.commands()
    o.set_commands(c.astype(np.float64))
    g.set_commands(c)
    Dg = g.interaction_matrix().cpu().numpy().astype(np.float64)
    Do = oracle.jacobian_fd(o, 1e-3)
    assert np.linalg.norm(Dg - Do) <= TOL_FRO * np.linalg.norm(Do)


@pytest.mark.parametrize("name", ["scao_tiny", "mcao_small"])
def test_command_vjp_is_transposed_interaction_matrix(name):
    import torch
    _, g, o = _case(name)
    G = np.random.default_rng(4).normal(size=(3, o.n_slopes)).astype(np.float32)
    gc, gp = g.slopes_vjp(torch.from_numpy(G).cuda(), phase=True)
    gc = gc.cpu().numpy().astype(np.float64)
    Dg = g.interaction_matrix().cpu().numpy().astype(np.float64)
    want = G.astype(np.float64) @ Dg
    assert np.abs(gc - want).max() <= 1e-5 * np.abs(want).max()
    Do = oracle.jacobian_fd(o, 1e-3)
    ref = G.astype(np.float64) @ Do
    assert np.linalg.norm(gc - ref) <= TOL_FRO * np.linalg.norm(ref)
    # a single vector gives the same row
    g1, _ = g.slopes_vjp(torch.from_numpy(G[1]).cuda())
    assert np.abs(g1.cpu().numpy() - gc[1]).max() <= 1e-5 * np.abs(gc[1]).max()
    assert gp.shape == (3, sum(g.query(mcao.Q_WFS_PHASE, w) for w in range(len(g.cfg["wfs"]))))


@pytest.mark.parametrize("name,w,ranks", [("scao_tiny", 0, (0, 57, -1)), ("mcao_small", 0, (0, 20, -1)),
                                          ("mcao_small", 1, (0, 3))])
def test_phase_vjp_matches_subaperture_fd(name, w, ranks):
    # unit vectors on a subaperture's two slopes: the pupil-phase gradient equals the oracle's
    # central differences of cog(bin(sh_image)) on that subaperture (times lambda_ref / lambda),
    # is zero elsewhere and sums to zero (piston)
    import torch
    cfg, g, o = _case(name)
    ww = cfg["wfs"][w]
    npx, N = ww["n_px"], ww["n_sub"] * ww["n_px"]
    scale = cfg["lambda_ref"] / ww["lambda"]
    valid = o.valid(w)
    nv = valid.size
    slope0 = sum(2 * o.n_valid(q) for q in range(w))
    off = sum((cfg["wfs"][q]["n_sub"] * cfg["wfs"][q]["n_px"]) ** 2 for q in range(w))
    amp = oracle.pupil(cfg["D"], cfg["obstruction"], N)
    phase = o.wfs_phase(w) * scale
    sig, dirs = o.elongation(w)
    for r in ranks:
        r = r % nv
        G = np.zeros((2, o.n_slopes), np.float32)
        G[0, slope0 + r] = 1.0
        G[1, slope0 + nv + r] = 1.0
        _, gp = g.slopes_vjp(torch.from_numpy(G).cuda(), commands=False, phase=True)
        gp = gp.cpu().numpy()[:, off:off + N * N].reshape(2, N, N).astype(np.float64)
        sx, sy = valid[r] % ww["n_sub"], valid[r] // ww["n_sub"]
        sl = (slice(sy * npx, (sy + 1) * npx), slice(sx * npx, (sx + 1) * npx))
        J = oracle.subap_jacobian_fd(amp[sl], phase[sl], ww["n_fft"], ww["n_bin"], sig[r], tuple(dirs[r]),
                                     h=1e-4) * scale
        patch = gp[:, sl[0], sl[1]]
        assert np.abs(patch - J).max() <= TOL_MAX * np.abs(J).max(), (r, np.abs(patch - J).max() / np.abs(J).max())
        rest = gp.copy()
        rest[:, sl[0], sl[1]] = 0.0
        assert not rest.any()
        assert abs(patch[0].sum()) <= 1e-4 * np.abs(patch[0]).sum()


def test_autograd_sensing_function():
    import torch
    _, g, o = _case("mcao_small")
    c = torch.tensor(g.commands(), dtype=torch.float32, device="cuda", requires_grad=True)
    s = mcao.sensing(g, c)
    assert float(torch.sqrt(torch.mean((s.detach().cpu().double() - torch.from_numpy(o.measure())) ** 2))) <= 1e-4
    wv = torch.from_numpy(np.random.default_rng(9).normal(size=o.n_slopes).astype(np.float32)).cuda()
    (s * wv).sum().backward()
    Dg = g.interaction_matrix()
    want = (wv @ Dg).cpu().numpy()
    assert np.abs(c.grad.cpu().numpy() - want).max() <= 1e-5 * np.abs(want).max()


def test_vjp_argument_errors():
    import torch
    _, g, _ = _case("scao_tiny")
    G = torch.zeros((1, g.query(mcao.Q_SLOPES)), device="cuda")
    with pytest.raises(mcao.McaoError):
        g.slopes_vjp(G, commands=False, phase=False)
    L = mcao.lib()
    assert L.mcao_interaction_matrix(g.h, None, 10) == 1
    assert L.mcao_interaction_matrix(g.h, G.data_ptr(), 1) == 2      # ld < n_commands


@pytest.mark.parametrize("name", ["scao_tiny", "mcao_small"])
def test_layer_vjp_matches_directional_derivative(name):
    # <g_layers, delta> equals g^T (s(screens + e delta) - s(screens - e delta)) / 2e of the oracle,
    # with delta the perturbation the float32 screens actually carry
    import torch
    if name == "scao_tiny":
        cfg, screens, _ = scao_tiny_inputs()
        cfg = dict(cfg, noise=False)
    else:
        cfg = mcao_small()
        screens = inputs.make_screens(cfg)
    _, g, o = _case(name)
    c = o.commands()
    rng = np.random.default_rng(8)
    G = rng.normal(size=(2, o.n_slopes)).astype(np.float32)
    _, _, gl = g.slopes_vjp(torch.from_numpy(G).cuda(), commands=False, layers=True)
    gl = gl.cpu().numpy().astype(np.float64)
    eps = 1e-3
    delta = [rng.normal(size=s.shape) for s in screens]
    plus = [(s.astype(np.float64) + eps * d).astype(np.float32) for s, d in zip(screens, delta)]
    minus = [(s.astype(np.float64) - eps * d).astype(np.float32) for s, d in zip(screens, delta)]
    act = np.concatenate([(p.astype(np.float64) - m.astype(np.float64)).ravel() / 2.0 for p, m in zip(plus, minus)])
    sp = oracle.Sim(cfg, plus)
    sm = oracle.Sim(cfg, minus)
    sp.set_commands(c)
    sm.set_commands(c)
    ds = (sp.measure() - sm.measure()) / 2.0
    for v in range(2):
        want = float(G[v].astype(np.float64) @ ds)
        got = float(gl[v] @ act)
        assert got == pytest.approx(want, rel=1e-4, abs=1e-6 * np.abs(G[v]).sum() * eps)
    # samples outside every beam get nothing; the total over a layer is the derivative of a
    # uniform (piston) layer change, which the centroids ignore
    n0 = cfg["layers"][0]["n"] ** 2
    assert np.count_nonzero(gl[0, :n0]) < n0
    assert abs(gl[0, :n0].sum()) <= 1e-4 * np.abs(gl[0, :n0]).sum()
    sp.close()
    sm.close()
