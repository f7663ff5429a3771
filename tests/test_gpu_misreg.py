"""Misregistered DMs through the C ABI against the oracle's direct sum over actuators: surfaces,
noise-free slopes and interaction matrices for a shifted and magnified DM (transform folded
into the separable tables) and for a rotated one (per-sample evaluation); the Gauss-Newton fit
recovers a misregistration from an oracle interaction matrix."""
import numpy as np
import pytest

import oracle
from paper_1608_00386_gb300 import build, calibration, inputs, mcao

from _helpers import mcao_small

pytestmark = pytest.mark.gpu

# (dm, shift x m, shift y m, rotation rad, magnification)
CASES = [(0, 0.3, -0.2, 0.0, 1.012), (0, 0.25, 0.1, np.radians(0.8), 0.985), (1, -0.4, 0.35, np.radians(-1.0), 1.02)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build.build()
    oracle.build()


def _pair(case=None):
    cfg = mcao_small()
    screens = inputs.make_screens(cfg)
    g = mcao.Sim(cfg)
    g.load_atmosphere(screens)
    g.load_dms()
    o = oracle.Sim(cfg, screens)
    c = np.random.default_rng(5).normal(0.0, 0.3, o.n_cmd).astype(np.float32)
    g.set_commands(c)
    o.set_commands(c.astype(np.float64))
    if case is not None:
        g.set_misregistration(*case)
        o.set_misregistration(*case)
    return cfg, g, o


@pytest.mark.parametrize("case", CASES)
def test_misregistered_surface_and_slopes_match_oracle(case):
    cfg, g, o = _pair(case)
    m = case[0]
    s_g = g.measure()
    s_o = o.measure()
    Sg = g.dm_surface(m).astype(np.float64)
    So = o.dm_surface(m)
    assert np.abs(Sg - So).max() <= 1e-5 * np.abs(So).max()
    assert float(np.sqrt(np.mean((s_g - s_o) ** 2))) <= 1e-4


@pytest.mark.parametrize("case", CASES)
def test_misregistered_interaction_matrix_matches_oracle(case):
    cfg, g, o = _pair(case)
    Dg = g.interaction_matrix().cpu().numpy().astype(np.float64)
    Do = oracle.jacobian_fd(o, 1e-3)
    n = np.linalg.norm
    assert n(Dg - Do) <= 1e-5 * n(Do), n(Dg - Do) / n(Do)
    assert np.abs(Dg - Do).max() <= 2e-5 * np.abs(Do).max()


def test_identity_restores_the_nominal_dm():
    cfg, g, o = _pair()
    s0 = g.measure()
    g.set_misregistration(0, 0.2, 0.1, 0.01, 1.01)
    assert np.abs(g.measure() - s0).max() > 1e-3
    g.set_misregistration(0, 0.0, 0.0, 0.0, 1.0)
    assert np.array_equal(g.measure(), s0)
    for bad in ((5, 0.0, 0.0, 0.0, 1.0), (0, 0.0, 0.0, 4.0, 1.0), (0, 0.0, 0.0, 0.0, 0.0),
                (0, float("nan"), 0.0, 0.0, 1.0)):
        with pytest.raises(mcao.McaoError):
            g.set_misregistration(*bad)
    assert np.array_equal(g.measure(), s0)


@pytest.mark.parametrize("true", [(0, 0.35, -0.25, np.radians(0.7), 1.015), (1, -0.3, 0.2, np.radians(-0.9), 0.985)])
def test_fit_recovers_misregistration_from_oracle_matrix(true):
    # measured matrix: the oracle's central differences with the true misregistration; the fit
    # starts from the nominal DM
    import torch
    cfg, g, o = _pair()
    o.set_misregistration(*true)
    D_meas = torch.from_numpy(oracle.jacobian_fd(o, 1e-3).astype(np.float32)).cuda()
    p, hist = calibration.fit_misregistration(g, D_meas, true[0], iters=12)
    pitch = cfg["dms"][true[0]]["pitch"]
    # measured: |error| about 5e-8 m, 2e-8 rad, 4e-8 after four iterations (float32 model
    # matrices against fp64 central differences)
    assert abs(p[0] - true[1]) <= 1e-5 * pitch and abs(p[1] - true[2]) <= 1e-5 * pitch
    assert abs(p[2] - true[3]) <= 1e-6
    assert abs(p[3] - true[4]) <= 1e-6
    assert hist[-1] <= 1e-5 < hist[0]


@pytest.mark.parametrize("case", CASES)
def test_normal_equations_model_equals_interaction_matrix(case):
    """The model matrix the Gauss-Newton kernel forms (influence functions at the bilinear corners
    of each pupil sample, in the DM's frame) is the interaction matrix of the misregistered DM:
    against mcao_interaction_matrix at the same misregistration the cost vanishes (float32
    rounding of two summation orders) and the gradient with it."""
    cfg, g, _ = _pair(case)
    D = calibration.dm_columns(g, g.interaction_matrix(), case[0])
    JtJ, Jte, cost, msq = g.misreg_normal_equations(case[0], D)
    assert msq > 0.0
    assert np.sqrt(cost / msq) <= 1e-5
    assert np.all(np.abs(Jte) <= 1e-5 * np.sqrt(np.diag(JtJ) * msq))


@pytest.mark.parametrize("case", CASES)
def test_normal_equations_gradient_is_the_derivative(case):
    """2 Jte is the gradient of the cost: against central differences of the call's own cost in
    each parameter (steps 1e-3 pitch, 1e-4 rad, 1e-4), measured 0.3 pitch / 1 deg / 1 % away from
    the matrix's misregistration; JtJ is symmetric positive semidefinite."""
    cfg, g, _ = _pair(case)
    dm = case[0]
    pitch = cfg["dms"][dm]["pitch"]
    D = calibration.dm_columns(g, g.interaction_matrix(), dm).clone()
    p = np.array(case[1:], dtype=np.float64) + np.array([0.3 * pitch, -0.2 * pitch, np.radians(1.0), 0.01])
    g.set_misregistration(dm, *p)
    JtJ, Jte, cost, _ = g.misreg_normal_equations(dm, D)
    h = np.array([1e-3 * pitch, 1e-3 * pitch, 1e-4, 1e-4])
    for i in range(4):
        e = np.zeros(4)
        e[i] = h[i]
        g.set_misregistration(dm, *(p + e))
        cp = g.misreg_normal_equations(dm, D)[2]
        g.set_misregistration(dm, *(p - e))
        cm = g.misreg_normal_equations(dm, D)[2]
        fd = (cp - cm) / (2.0 * h[i])
        assert abs(2.0 * Jte[i] - fd) <= 2e-3 * abs(fd) + 1e-6 * cost / h[i], (i, 2.0 * Jte[i], fd)
    assert np.allclose(JtJ, JtJ.T)
    assert np.min(np.linalg.eigvalsh(JtJ)) >= -1e-9 * np.max(np.abs(JtJ))
