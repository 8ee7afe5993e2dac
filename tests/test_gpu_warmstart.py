"""The learned warm start end to end on a small cantilever: a trajectory from
the plain Newton step (start v_n), training with the library's MLP kernels,
and held-out steps where the MLP start begins with a much smaller residual
than the v_n start, needs no more Newton iterations and fewer linear-solver
iterations (inexact Newton), and converges to the same states (same 1e-8
residual target)."""
import numpy as np
import pytest

from paper_2604_10357_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_mlp_warm_start_beats_previous_velocity():
    from paper_2604_10357_gb300 import build, tl, warmstart
    build.build()
    rng = np.random.default_rng(60)
    m = inputs.box_t10(20, 2, 2, 2.0, 0.2, 0.2)
    f_ext = inputs.tip_load_schedule(m, 400, 50, 50.0, rng)
    g = tl.Mesh(m.X, m.conn, [dict(inputs.SVK_1E7)], precision=tl.TL_FP64)
    g.build_pattern(m.fixed_nodes)
    prm = tl.params(h=1e-3, rtol=1e-8, linear_solver=tl.TL_SOLVER_PCG, lin_adaptive=1)
    tr = warmstart.generate(g, m.X, f_ext, 330, prm)
    train_idx = np.arange(1, 270)
    test_idx = np.arange(282, 330)
    model, hist = warmstart.train(g, tr, m.X, m.fixed_nodes, train_idx, iters=1500, lr=3e-3, log_every=500)
    assert min(h[2] for h in hist) <= hist[0][2]
    summary, _ = warmstart.evaluate(g, tr, test_idx, prm, model)
    print(summary)
    assert summary["mlp"]["median_g0_ratio"] < 0.2 * summary["v_n"]["median_g0_ratio"]
    assert summary["mlp"]["mean_iters"] <= summary["v_n"]["mean_iters"]
    assert summary["mlp"]["mean_lin_iters"] < summary["v_n"]["mean_lin_iters"]
    for mode in summary:
        assert summary[mode]["max_rel_dev"] < 1e-6, (mode, summary[mode])
