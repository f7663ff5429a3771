"""Host-side checks of the C ABI that need no GPU: the library builds, loads and exports every
function include/mcao.h declares; configuration validation rejects bad inputs before any CUDA
call; the product path does not reach the oracle."""
import os
import re

import numpy as np
import pytest

from paper_1608_00386_gb300 import build, inputs, mcao

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mcao.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mcao_[a-z_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    build.build()
    L = mcao.lib()
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(L, n)]
    assert missing == []
    assert sorted(mcao.EXPORTS) == names


def _expect(status, cfg):
    with pytest.raises(mcao.McaoError) as ei:
        mcao.Sim(cfg)
    assert ei.value.status == status, str(ei.value)


@pytest.mark.parametrize("mutate,status", [
    (lambda c: c.update(D=-1.0), 1),
    (lambda c: c.update(obstruction=1.0), 1),
    (lambda c: c.update(lambda_ref=0.0), 1),
    (lambda c: c.update(gain=float("nan")), 1),
    (lambda c: c.update(psf_every=-1), 1),
    (lambda c: c.update(wfs=[]), 1),
    (lambda c: c["wfs"][0].update(n_fft=8), 7),            # pad < 2
    (lambda c: c["wfs"][0].update(n_bin=3), 1),            # bin must divide n_fft
    (lambda c: c["wfs"][0].update(n_px=6, n_fft=12), 7),   # no kernel variant
    (lambda c: c["wfs"][0].update(valid_thr=1.5), 1),
    (lambda c: c["wfs"][0].update(type="lgs", height=-1.0), 1),
    (lambda c: c["science"][0].update(n_px=100), 7),       # not a multiple of 8
    (lambda c: c["science"][0].update(pad=7), 7),          # FFT size 896 = 2^7 * 7
])
def test_config_validation_rejects(mutate, status):
    build.build()
    cfg = inputs.scao_tiny()
    mutate(cfg)
    _expect(status, cfg)


def test_product_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1608_00386_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "mcao_oracle" not in text and "liboracle" not in text, f
    for f in ("mcao_oracle.c", "__init__.py"):
        text = open(os.path.join(ROOT, "oracle", f)).read()
        assert "paper_1608_00386_gb300" not in text and "mcao.h" not in text


@pytest.mark.parametrize("n,pixel,r0,L0,null_out,status", [
    (64, 0.1, 0.15, 25.0, True, 1),     # null output
    (64, 0.0, 0.15, 25.0, False, 1),    # pixel <= 0
    (64, 0.1, -1.0, 25.0, False, 1),    # r0 <= 0
    (64, 0.1, 0.15, float("inf"), False, 1),
    (1, 0.1, 0.15, 25.0, False, 2),     # n < 2
    (77, 0.1, 0.15, 25.0, False, 2),    # 7 * 11: no radix-2/3/5 factorisation
    (8192, 0.1, 0.15, 25.0, False, 2),  # above 4096
])
def test_generate_screen_rejects_before_any_device_call(n, pixel, r0, L0, null_out, status):
    # argument checks run on the host first; the pointer is never dereferenced
    import ctypes as C
    build.build()
    err = C.create_string_buffer(128)
    out = None if null_out else C.c_void_p(16)
    st = mcao.lib().mcao_generate_screen(n, pixel, r0, L0, 1, out, None, err, 128)
    assert st == status and err.value


def test_misregistration_fit_host_logic_on_a_linear_model():
    # the Gauss-Newton loop against a fake simulation whose matrix is linear in the parameters
    # (D(p) = D0 + sum_k (p_k - n_k) A_k, n the nominal parameters): one step lands on the truth,
    # only the DM's own columns are used, and the DM is left at the fitted parameters
    torch = pytest.importorskip("torch")
    from paper_1608_00386_gb300 import calibration
    rng = np.random.default_rng(0)
    n_slopes, cols = 40, (3, 9)          # DM 1 owns columns 3..8 of 12
    D0 = torch.from_numpy(rng.normal(size=(n_slopes, 12))).float()
    A = [torch.from_numpy(rng.normal(size=(n_slopes, 12))).float() for _ in range(4)]
    nominal = np.array([0.0, 0.0, 0.0, 1.0])

    class FakeSim:
        cfg = {"dms": [{"pitch": 1.0, "valid": np.ones(3, np.uint8)}, {"pitch": 0.5, "valid": np.ones(6, np.uint8)},
                       {"pitch": 2.0, "valid": np.ones(3, np.uint8)}]}

        def __init__(self):
            self.p = nominal.copy()

        def set_misregistration(self, dm, *p):
            assert dm == 1
            self.p = np.array(p)

        def interaction_matrix(self):
            D = D0.clone()
            for k in range(4):
                D += float(self.p[k] - nominal[k]) * A[k]
            return D

        def misreg_normal_equations(self, dm, Dm):
            # what the library returns for this linear model: dD/dp_k = A_k on the DM's columns
            assert dm == 1 and Dm.shape[1] == cols[1] - cols[0]
            e = (self.interaction_matrix()[:, cols[0]:cols[1]] - Dm).double().numpy()
            J = [a[:, cols[0]:cols[1]].double().numpy() for a in A]
            JtJ = np.array([[np.sum(J[i] * J[j]) for j in range(4)] for i in range(4)])
            Jte = np.array([np.sum(J[i] * e) for i in range(4)])
            return JtJ, Jte, float(np.sum(e * e)), float(np.sum(Dm.double().numpy() ** 2))

    truth = np.array([0.2, -0.1, 0.01, 1.02])
    sim = FakeSim()
    sim.set_misregistration(1, *truth)
    D_meas = sim.interaction_matrix()
    D_meas[:, :cols[0]] += 5.0            # other DMs' columns must not matter
    sim.set_misregistration(1, *nominal)
    p, hist = calibration.fit_misregistration(sim, D_meas, 1, iters=4)
    assert np.allclose(p, truth, atol=1e-4)
    assert hist[-1] < 1e-5 < hist[0]
    assert np.allclose(sim.p, p)
