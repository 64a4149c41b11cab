"""End to end on a small scale: autotune training regions, train the MLP on
the GPU with the library's kernels, and rank unseen regions' schedules.  The
trained model must beat the method without it (the paper's default CUDA
geometry) in mean regret against the exhaustive autotuner."""
import pytest

pytestmark = pytest.mark.gpu

U = pytest.importorskip("paper_2209_10643_b300")


def test_cost_model_beats_the_default_geometry():
    from paper_2209_10643_b300 import costmodel as CM
    ctx = U.upir_init(0)
    try:
        rep = CM.run_protocol(ctx, n_train=150, n_eval=60, epochs=150, eval_t_hi=2e6, reps=2)
    finally:
        U.upir_finalize(ctx)
    assert rep["regions"] == 60
    assert rep["loss_last"] < rep["loss_first"]
    assert rep["model_regret"]["mean"] < rep["heuristic_regret"]["mean"]
