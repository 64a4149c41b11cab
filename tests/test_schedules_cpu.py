"""Host-side parts of the schedule policies (no GPU): the auto schedule's
candidate lists, its features against the cost model's, and its pick with
hand-made models whose preference is known."""
import math

import numpy as np
import pytest

U = pytest.importorskip("paper_2209_10643_b300")
from paper_2209_10643_b300 import costmodel as CM  # noqa: E402


def test_candidate_lists():
    ax = U.upir_auto_candidates(U.UPIR_BODY_AXPY)
    ja = U.upir_auto_candidates(U.UPIR_BODY_JACOBI5)
    mv = U.upir_auto_candidates(U.UPIR_BODY_MATVEC)
    gm = U.upir_auto_candidates(U.UPIR_BODY_GEMM_F32)
    assert (len(ax), len(ja), len(mv), len(gm)) == (28, 15, 20, 6)
    assert all(un == 256 for _, _, un in gm)
    assert U.upir_auto_candidates(U.UPIR_BODY_GEMM_BF16) == []
    for lst in (ax, ja, mv):
        assert len(set(lst)) == len(lst)
        assert {sc for sc, _, _ in lst} == {U.UPIR_SCHED_STATIC, U.UPIR_SCHED_DYNAMIC}
    assert (U.UPIR_SCHED_DYNAMIC, 65536, 1024) in ax and (U.UPIR_SCHED_STATIC, 0, 128) == ja[0]
    assert CM.candidates(CM.OP_AXPY)[0] == dict(sched=U.UPIR_SCHED_STATIC, chunk=0, units=128, teams=0)


@pytest.mark.parametrize("op,body,trip,cols,bpi,fpi,ftrip", [
    (CM.OP_AXPY, U.UPIR_BODY_AXPY, 1 << 20, 0, 12.0, 4.0, 1 << 20),
    (CM.OP_JACOBI, U.UPIR_BODY_JACOBI5, 510, 512, 8.0, 6.0, 510 * 510),
    (CM.OP_MATVEC, U.UPIR_BODY_MATVEC, 3000, 700, 2800.0, 1400.0, 3000),
    (CM.OP_GEMM, U.UPIR_BODY_GEMM_F32, 512 * 640, 384, 24.0, 768.0, 512 * 640)])
def test_runtime_features_match_the_cost_models(op, body, trip, cols, bpi, fpi, ftrip):
    for sched, chunk, units, teams in [(0, 0, 256, 0), (1, 4096, 1024, 37), (0, 7, 128, 1)]:
        want = CM.features(op, ftrip, bpi, fpi, sched, chunk, units, teams)
        got = np.array(U.upir_auto_features(body, trip, cols, sched, chunk, units, teams), np.float32)
        assert np.allclose(got, want, rtol=1e-6, atol=0), (sched, chunk, units, teams)


def crafted(weights_on):
    """An MLP whose prediction is -sum(features[i] for i in weights_on) for
    standardised features that are >= 0 (all here, with mean 0, std 1)."""
    p = np.zeros(U.UPIR_MLP_NPARAM, np.float32)
    w1 = p[:64 * 12].reshape(64, 12)
    for i in weights_on:
        w1[0, i] = 1.0
    off_w2 = 64 * 12 + 64
    p[off_w2 + 0] = 1.0                      # W2[0][0]
    off_w3 = off_w2 + 64 * 64 + 64
    p[off_w3 + 0] = -1.0                     # W3[0]
    return p, np.zeros(12, np.float32), np.ones(12, np.float32)


def test_auto_pick_follows_the_model():
    p, m, s = crafted([9])                   # largest chunk wins
    assert U.upir_auto_pick(p, m, s, U.UPIR_BODY_AXPY, 1 << 20) == (U.UPIR_SCHED_DYNAMIC, 65536, 128)
    assert U.upir_auto_pick(p, m, s, U.UPIR_BODY_AXPY, 1 << 20, units=512) == (U.UPIR_SCHED_DYNAMIC, 65536, 0)
    p, m, s = crafted([8, 9])                # dynamic, then the largest chunk
    assert U.upir_auto_pick(p, m, s, U.UPIR_BODY_JACOBI5, 100, 128) == (U.UPIR_SCHED_DYNAMIC, 4, 128)
    p, m, s = crafted([10])                  # most units per team
    assert U.upir_auto_pick(p, m, s, U.UPIR_BODY_MATVEC, 5000, 300) == (U.UPIR_SCHED_STATIC, 0, 1024)
    p, m, s = crafted([9])                   # GEMM_F32: largest chunk of tiles, 256-unit teams
    assert U.upir_auto_pick(p, m, s, U.UPIR_BODY_GEMM_F32, 1 << 20, 1024) == (U.UPIR_SCHED_STATIC, 8, 256)
    p, m, s = crafted([8])                   # any dynamic candidate: the first one
    assert U.upir_auto_pick(p, m, s, U.UPIR_BODY_GEMM_F32, 1 << 20, 1024) == (U.UPIR_SCHED_DYNAMIC, 1, 256)


def test_gemm_features():
    f = U.upir_auto_features(U.UPIR_BODY_GEMM_F32, 512 * 1024, 2048, U.UPIR_SCHED_DYNAMIC, 2, 256, 0)
    assert f[3] == 1.0 and sum(f[:4]) == 1.0
    assert math.isclose(f[4], 19.0) and f[5] == 128.0 and f[6] == 4096.0
    assert f[8] == 1.0 and math.isclose(f[9], math.log2(3), rel_tol=1e-6) and f[10] == 8.0


def test_auto_pick_without_model_or_candidates_is_static():
    assert U.upir_auto_pick(None, None, None, U.UPIR_BODY_AXPY, 1000) == (U.UPIR_SCHED_STATIC, 0, 0)
    p, m, s = crafted([9])
    assert U.upir_auto_pick(p, m, s, U.UPIR_BODY_GEMM_BF16, 1000) == (U.UPIR_SCHED_STATIC, 0, 0)
    assert U.upir_auto_pick(p, m, s, U.UPIR_BODY_AXPY, 1000, units=96) == (U.UPIR_SCHED_STATIC, 0, 0)


def test_auto_pick_standardises_features():
    # with the chunk feature's mean above every candidate, standardised it is
    # negative for all: the ReLU then zeroes it and every candidate ties, so
    # the first candidate wins
    p, m, s = crafted([9])
    m = m.copy()
    m[9] = 100.0
    assert U.upir_auto_pick(p, m, s, U.UPIR_BODY_AXPY, 1 << 20) == (U.UPIR_SCHED_STATIC, 0, 128)
    assert math.isclose(U.upir_auto_features(U.UPIR_BODY_AXPY, 1, 0, 0, 1, 1, 1)[9], 1.0)
