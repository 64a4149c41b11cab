"""The learned schedule cost model end to end: autotune training regions
exhaustively, train the MLP on the GPU with the library's kernels, and rank
the candidate schedules of unseen regions against the exhaustive autotuner.

- small scale: the trained model beats the method without it (the paper's
  default CUDA geometry) in mean regret;
- the target scale: over 300 unseen regions (240 drawn like the batched-region
  workload, 60 FP32 GEMM loops) the model's mean regret is at most 10 %, and
  every loop kind, GEMM included, is ranked.  Each candidate's label is the
  median of five timed runs, so that measurement noise cannot carry the mean
  over the bound."""
import pytest

pytestmark = pytest.mark.gpu

U = pytest.importorskip("paper_2209_10643_b300")


def test_cost_model_beats_the_default_geometry():
    from paper_2209_10643_b300 import costmodel as CM
    ctx = U.upir_init(0)
    try:
        rep = CM.run_protocol(ctx, n_train=150, n_eval=60, epochs=150, eval_t_hi=2e6, reps=2,
                              n_train_gemm=20, n_eval_gemm=10)
    finally:
        U.upir_finalize(ctx)
    assert rep["regions"] == 70
    assert rep["loss_last"] < rep["loss_first"]
    assert rep["model_regret"]["mean"] < rep["heuristic_regret"]["mean"]


def test_cost_model_regret_within_ten_percent():
    from paper_2209_10643_b300 import costmodel as CM
    ctx = U.upir_init(0)
    try:
        rep = CM.run_protocol(ctx, n_train=800, n_eval=240, epochs=300, reps=5,
                              n_train_gemm=120, n_eval_gemm=60)
    finally:
        U.upir_finalize(ctx)
    assert rep["regions"] == 300
    assert set(rep["model_regret_by_op"]) == {"axpy", "jacobi", "matvec", "gemm"}
    assert rep["model_regret_by_op"]["gemm"]["regions"] == 60
    assert rep["model_regret"]["mean"] <= 0.10, rep["model_regret"]


def test_batch_split_by_predicted_cost():
    """Longest-processing-time split of the 512-region batch over 2-4 ranks
    by the trained model's predicted times (each region's best candidate):
    every region lands on one rank, and the predicted loads differ by at most
    the largest single prediction."""
    import numpy as np

    import upir_inputs as I
    from paper_2209_10643_b300 import costmodel as CM
    from paper_2209_10643_b300.sharding import shard_lpt
    ctx = U.upir_init(0)
    try:
        specs = CM.training_specs(150, gemm=0)
        tr, _ = CM.train(ctx, CM.pool_for(ctx, specs), specs, epochs=150, reps=2)
        batch = I.batched_region_specs(512, seed=6)
        cost = tr.predict_us(batch)
    finally:
        U.upir_finalize(ctx)
    assert cost.shape == (512,) and np.all(np.isfinite(cost)) and np.all(cost > 0)
    # larger regions of one kind are predicted slower (the smallest AXPY
    # regions take the launch's latency, ~8 us; the largest ~20-30 us)
    ax = [(sp["n"], c) for sp, c in zip(batch, cost) if sp["op"] == I.OP_AXPY_DOT]
    ax.sort()
    assert np.mean([c for _, c in ax[-20:]]) > 1.5 * np.mean([c for _, c in ax[:20]])
    for world in (2, 3, 4):
        parts = shard_lpt(cost.tolist(), world)
        assert sorted(i for p in parts for i in p) == list(range(512))
        loads = [float(sum(cost[i] for i in p)) for p in parts]
        assert max(loads) - min(loads) <= float(cost.max())


def test_auto_schedule_scores_the_features_the_model_was_trained_on():
    """schedule(auto) on recorded loops: the candidate the runtime takes has
    the smallest prediction the trained model gives over all candidates, with
    each candidate's features built from the geometry the planner launches it
    with (the features of the training data)."""
    import numpy as np

    from paper_2209_10643_b300 import costmodel as CM
    ctx = U.upir_init(0)
    try:
        specs = CM.training_specs(120, gemm=12)
        pool = CM.pool_for(ctx, specs + [{"op": CM.OP_GEMM, "m": 512, "n": 384, "k": 256}])
        tr, _ = CM.train(ctx, pool, specs, epochs=120, reps=2)
        CM.install(ctx, tr.model, tr.mean, tr.std)
        for sp in [{"op": CM.OP_AXPY, "n": 3_000_000}, {"op": CM.OP_AXPY, "n": 5000},
                   {"op": CM.OP_JACOBI, "side": 700}, {"op": CM.OP_MATVEC, "rows": 3000, "cols": 900},
                   {"op": CM.OP_GEMM, "m": 512, "n": 384, "k": 256}]:
            pb = CM.Problem(pool, sp)
            rows, cands = [], []
            for cand in CM.candidates(sp["op"]):
                try:
                    r = pb.region(cand)
                except U.UpirError:
                    continue  # a candidate that cannot run this loop (the runtime skips it too)
                teams, units = U.upir_region_loop_geometry(r, 0)
                U.upir_region_destroy(r)
                rows.append(CM.features(pb.op, pb.trip, pb.bpi, pb.fpi, cand["sched"], cand["chunk"], units, teams))
                cands.append(cand)
            pred = tr.model.predict(CM.standardize(np.stack(rows), tr.mean, tr.std)[0]).cpu().numpy()
            r = pb.region(dict(sched=U.UPIR_SCHED_AUTO, chunk=0, units=0, teams=0))
            sched, chunk, _ = U.upir_region_loop_schedule(r, 0)
            teams, units = U.upir_region_loop_geometry(r, 0)
            U.upir_region_destroy(r)
            picked = [i for i, c in enumerate(cands)
                      if (c["sched"], c["chunk"], c["units"]) == (sched, chunk, units)]
            assert picked, (sp, sched, chunk, units)
            assert pred[picked[0]] <= pred.min() + 1e-3, (sp, float(pred[picked[0]]), float(pred.min()))
            pb.close()
    finally:
        U.upir_finalize(ctx)
