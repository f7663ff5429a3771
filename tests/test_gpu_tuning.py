"""Launch shapes and the autotuner (mcao_get_tuning / mcao_set_tuning / mcao_autotune) through the
C ABI.  The shapes change how work is laid on the GPU, not what is computed: the sensing grid,
the reconstructor slices' grid, the science ordering, the batched float32 product's grid and the
steps per graph launch leave
every result bit-identical; the tensor-core product's chunk regroups float32 sums only.  The
autotuner's trials run on a checkpoint of the simulation, so a tuned run continues exactly as an
untuned one."""
import numpy as np
import pytest

from paper_1608_00386_gb300 import build, inputs, mcao

from _helpers import mcao_small, scao_tiny_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build.build()


def _mcao_small_sim(noise=True, n_real=1, r_dtype=mcao.DTYPE_F32):
    cfg = dict(mcao_small(), noise=noise)
    n_cmd = inputs.n_commands(cfg)
    g = mcao.Sim(cfg, n_real=n_real)
    for r in range(n_real):
        g.load_atmosphere(inputs.make_screens(cfg, realization=r), realization=r)
    g.set_realization(0)
    g.load_dms()
    R = inputs.random_reconstructor(n_cmd, g.query(mcao.Q_SLOPES), 1e-3, 4)
    g.load_reconstructor(R, dtype=r_dtype)
    return g


def test_tuning_round_trip_and_checks():
    g = _mcao_small_sim()
    t = g.tuning()
    assert t == {"sense_blocks_per_sm": 4, "recon_ctas_pct": 85, "science_after_aux": 1, "tc_chunk": 8,
                 "multi_blocks_per_sm": 2, "steps_per_graph": 1}
    g.set_tuning(sense_blocks_per_sm=2, recon_ctas_pct=150)
    assert g.tuning()["sense_blocks_per_sm"] == 2 and g.tuning()["recon_ctas_pct"] == 150
    for bad in ({"sense_blocks_per_sm": 0}, {"recon_ctas_pct": 1000}, {"science_after_aux": 2}, {"tc_chunk": 0},
                {"steps_per_graph": 17}):
        with pytest.raises(mcao.McaoError):
            g.set_tuning(**bad)
    with pytest.raises(mcao.McaoError):
        g.autotune(steps_per_trial=0)


def test_shapes_leave_results_bit_identical():
    """A laser star and a natural star, noise on: default shapes against the sensing grid at 2
    blocks per SM, the slices at 50 % of the SMs, the science started at the step's start and
    four steps per graph."""
    a = _mcao_small_sim()
    b = _mcao_small_sim()
    b.set_tuning(sense_blocks_per_sm=2, recon_ctas_pct=50, science_after_aux=0, steps_per_graph=4)
    a.step(15)
    b.step(15)   # three launches of the four-step graph, then three one-step launches
    assert np.array_equal(a.slopes(), b.slopes())
    assert np.array_equal(a.commands(), b.commands())
    assert a.psf(0, with_image=False) == b.psf(0, with_image=False)


def test_autotune_restores_the_run():
    a = _mcao_small_sim()
    b = _mcao_small_sim()
    a.step(5)
    b.step(5)
    chosen, report = a.autotune(steps_per_trial=10)
    assert chosen["sense_blocks_per_sm"] in (2, 3, 4, 6)
    assert chosen["recon_ctas_pct"] in (50, 75, 80, 85, 90, 95, 100, 125)
    assert chosen["science_after_aux"] in (0, 1) and chosen["steps_per_graph"] in (1, 2, 4, 8)
    for name in ("sense_blocks_per_sm:", "recon_ctas_pct:", "science_after_aux:", "steps_per_graph:", "chosen"):
        assert name in report
    assert a.tuning() == chosen
    assert a.step_index == b.step_index == 5
    a.step(10)
    b.step(10)
    assert np.array_equal(a.commands(), b.commands())
    assert np.array_equal(a.slopes(), b.slopes())


def test_autotune_batched_tensor_core_chunk():
    """Batched bfloat16 (tensor-core product): the tuner picks the TMEM chunk among its candidates,
    and any chunk gives the product within float32 rounding of the default."""
    g = _mcao_small_sim(noise=False, n_real=3, r_dtype=mcao.DTYPE_BF16)
    ref = _mcao_small_sim(noise=False, n_real=3, r_dtype=mcao.DTYPE_BF16)
    chosen, report = g.autotune(steps_per_trial=5)
    assert chosen["tc_chunk"] in (4, 8, 16) and "tc_chunk:" in report
    g.set_tuning(tc_chunk=1)
    g.step(10)
    ref.step(10)
    for r in range(3):
        g.set_realization(r)
        ref.set_realization(r)
        cg, cr = g.commands().astype(np.float64), ref.commands().astype(np.float64)
        assert np.linalg.norm(cg - cr) <= 1e-5 * np.linalg.norm(cr)


def test_autotune_batched_float32_grid():
    cfg, screens, R = scao_tiny_inputs()
    g = mcao.make_sim(cfg, [inputs.make_screens(cfg, realization=r) for r in range(4)], R, n_real=4)
    chosen, report = g.autotune(steps_per_trial=5)
    assert chosen["multi_blocks_per_sm"] in (1, 2) and "multi_blocks_per_sm:" in report


def test_profiler_stage_mask_and_graph_nodes_leave_results_bit_identical():
    """The stage profiler's event-record nodes are in the step graph only for the stages asked
    (mcao_set_profiling_stages): timing the product alone records only its launches, timing
    every stage records all of them, and neither changes what a step computes."""
    a = _mcao_small_sim()
    b = _mcao_small_sim()
    b.set_profiling(True, stages=["recon"])
    b.step(3)
    tl = b.get_timeline()
    assert tl and {name for _, name, _, _ in tl} == {"recon"}
    ms, cnt, lps = b.get_profile()
    assert cnt["recon"] > 0 and cnt["dm"] == 0 and cnt["wfs_main"] == 0 and lps > 0
    b.set_profiling(True)
    b.step(2)
    names = {name for _, name, _, _ in b.get_timeline()}
    assert {"dm", "wfs_main", "recon", "recon_reduce"} <= names
    b.set_profiling(False)
    b.step(5)
    a.step(10)
    assert np.array_equal(a.slopes(), b.slopes())
    assert np.array_equal(a.commands(), b.commands())
    assert mcao.lib().mcao_set_profiling_stages(b.h, 1 << len(mcao.STAGES)) == 1   # MCAO_E_INVALID_ARG
