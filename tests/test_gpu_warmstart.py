"""The learned warm start end to end on a small cantilever: a trajectory from
the plain Newton step (start v_n), training with the library's MLP kernels,
and held-out steps where the network's start (a learned correction of the
cubic extrapolation of the velocity history) begins with a smaller residual
than the linear extrapolation 2 v_n - v_{n-1} (its free two-velocity base)
and than v_n, needs no more Newton iterations, fewer linear-solver iterations
and less time, and converges to the same states (same 1e-8 residual target).
The cubic extrapolation itself is reported beside it."""
import numpy as np
import pytest

from paper_2604_10357_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_mlp_warm_start_beats_linear_extrapolation():
    from paper_2604_10357_gb300 import build, tl, warmstart
    build.build()
    rng = np.random.default_rng(60)
    m = inputs.box_t10(20, 2, 2, 2.0, 0.2, 0.2)
    f_ext = inputs.tip_load_schedule(m, 400, 50, 50.0, rng)
    g = tl.Mesh(m.X, m.conn, [dict(inputs.SVK_1E7)], precision=tl.TL_FP64)
    g.build_pattern(m.fixed_nodes)
    prm = tl.params(h=1e-3, rtol=1e-8, linear_solver=tl.TL_SOLVER_PCG, lin_adaptive=1)
    tr = warmstart.generate(g, m.X, f_ext, 330, prm)
    train_idx = np.arange(3, 270)
    test_idx = np.arange(282, 330)
    model, hist = warmstart.train(g, tr, m.fixed_nodes, train_idx, iters=1500, lr=3e-3, log_every=500)
    assert min(h[2] for h in hist) <= hist[0][2]
    warmstart.evaluate(g, tr, test_idx[:2], prm, model)          # first-use allocations, untimed
    summary, _ = warmstart.evaluate(g, tr, test_idx, prm, model)
    print({k: {kk: round(vv, 6) for kk, vv in v.items()} for k, v in summary.items()})
    mlp, lin, vn = summary["mlp"], summary["linear"], summary["v_n"]
    assert mlp["median_g0_ratio"] < 0.5 * lin["median_g0_ratio"] < 0.5 * vn["median_g0_ratio"]
    assert mlp["mean_iters"] <= lin["mean_iters"] <= vn["mean_iters"]
    assert mlp["mean_lin_iters"] < lin["mean_lin_iters"]
    assert mlp["mean_ms"] < lin["mean_ms"]
    for mode in summary:
        assert summary[mode]["max_rel_dev"] < 1e-6, (mode, summary[mode])
