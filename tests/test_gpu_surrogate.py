"""The learned surrogate end to end: training data from the solver, training
with the library's FNO kernels, held-out error judged by the solver, and what
the trained network gains over the method without it -- its throughput
against the plain solver run at the same accuracy (the coarsest time step
whose error matches the surrogate's)."""
import numpy as np
import pytest

from tests.gpu_helpers import need_gpu

pytestmark = pytest.mark.gpu


def test_surrogate_trains_and_is_judged_against_the_solver():
    need_gpu()
    from paper_1007_3470_gb300 import surrogate as S
    from paper_1007_3470_gb300.fno import Fno, FnoConfig
    tr_i, tr_p, _ = S.family(4096, seed=11)
    te_i, te_p, _ = S.family(512, seed=12)
    Xtr, Xte = S.features(tr_i, tr_p), S.features(te_i, te_p)
    Ytr, Yte = S.solve(tr_i, tr_p), S.solve(te_i, te_p)
    m = Fno(FnoConfig(), max_batch=512, train=True, seed=3)
    hist = S.train(m, Xtr, Ytr, epochs=25, batch=128, lr=2e-3)
    assert hist[-1] < 0.5 * hist[0]
    err = S.rel_errors(S.predict(m, Xte, 512), Yte)
    med = float(np.median(err))
    assert med < 0.1
    # the comparison: the plain solver at the surrogate's accuracy
    dt, solver_med = S.equal_accuracy_solver(te_i, te_p, Yte, med)
    assert solver_med <= med and 0 < dt <= 0.5
    fno_rate = S.time_inference(m, Xte)
    solver_rate = S.time_solver(te_i, te_p, dt)
    assert fno_rate > 0 and solver_rate > 0
    print(f"surrogate median rel err {med:.3e}: {fno_rate:.3e} solves/s; "
          f"solver at dt={dt} (median {solver_med:.3e}): {solver_rate:.3e} solves/s")
    m.close()
