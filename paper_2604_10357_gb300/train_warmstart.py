"""Train the learned Newton warm start on the 103,680-element cantilever.

    python -m paper_2604_10357_gb300.train_warmstart [--steps 1300] [--holdout 200]
        [--iters 4000] [--out PATH] [--report PATH]
    python -m paper_2604_10357_gb300.train_warmstart --collapse-log PATH [--steps 1400]

Box 12 x 1.2 x 1.2 m (120 x 12 x 12 hexes x 6 T10, SVK E = 1e7, nu = 0.3,
rho = 1000), clamped at x = 0, gravity plus a seeded tip load U(0, 500) N in a
random direction redrawn every 100 steps, h = 1e-3.  The trajectory comes from
the plain Newton step (FP64 element form, start v_n, PCG inner solve); the
network is trained on the first steps and evaluated on held-out steps after
them, where it is compared with the v_n start and with the linear and cubic
extrapolations of the velocity history in both element precisions.  Writes
the model (npz) and a JSON report.

With E = 1e7 Pa the 12 m beam cannot carry its own weight: it falls almost
freely about the clamp, the root is compressed until the SVK energy loses
convexity (min corner J 0.58 at step 1350), elements invert from step ~1358
on and Newton stops converging at step ~1370.  The default trajectory is
therefore 1,300 steps (min J about 0.67 at its end), not 2,000.
--collapse-log runs the trajectory only (no training) and writes one JSON line
per step: Newton / PCG iterations, convergence, ||g(v_n)||, mean tip
deflection and the smallest deformed / reference volume ratio of the corner
tetrahedra (torch reductions on the device, diagnostics only).
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import build, inputs, tl, warmstart

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_MODEL = os.path.join(HERE, "data", "warmstart_box120x12x12.npz")


def collapse_log(nsteps, path):
    import torch
    build.build()
    w = inputs.workload_warm_start_svk()
    m = w["mesh"]
    g = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP64)
    g.build_pattern(m.fixed_nodes)
    prm = tl.params(h=w["h"], rtol=1e-8, linear_solver=tl.TL_SOLVER_PCG, use_graph=1)
    X = torch.as_tensor(m.X, device="cuda")
    corners = torch.as_tensor(m.conn[:, :4].astype(np.int64), device="cuda")

    def signed_vol(P):
        return torch.linalg.det(torch.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], 1))

    V0 = signed_vol(X[corners])
    tip = torch.as_tensor(np.nonzero(np.isclose(m.X[:, 0], m.X[:, 0].max()))[0], device="cuda")
    q = X.reshape(-1).clone()
    v = torch.zeros_like(q)
    lam = torch.zeros(3 * g.nfixed, dtype=torch.float64, device="cuda")
    with open(path, "w") as out:
        for step in range(nsteps):
            fe = torch.as_tensor(w["f_ext"](step), dtype=torch.float64, device="cuda")
            v_new, q_new, st = g.newton_step(prm, q, v, lam, f_ext=fe, raise_on_nonconvergence=False)
            qn = q_new.view(-1, 3)
            row = dict(step=step, newton=st["inner_iters"], outer=st["outer_iters"], converged=st["converged"],
                       g_ref=st["g_ref"], pcg=st["lin_iters"],
                       tip=(qn[tip] - X[tip]).mean(0).tolist(),
                       min_volume_ratio=(signed_vol(qn[corners]) / V0).min().item())
            out.write(json.dumps(row) + "\n")
            if step % 100 == 0:
                print(row, flush=True)
            q, v = q_new.clone(), v_new.clone()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=1300)
    ap.add_argument("--holdout", type=int, default=200)
    ap.add_argument("--iters", type=int, default=4000)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--out", default=DEFAULT_MODEL)
    ap.add_argument("--report", default=None)
    ap.add_argument("--eval-steps", type=int, default=100)
    ap.add_argument("--collapse-log", default=None)
    args = ap.parse_args()
    if args.collapse_log:
        collapse_log(args.steps, args.collapse_log)
        return
    import torch
    build.build()
    w = inputs.workload_warm_start_svk()
    m = w["mesh"]
    g64 = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP64)
    g64.build_pattern(m.fixed_nodes)
    prm_plain = tl.params(h=w["h"], rtol=1e-8, linear_solver=tl.TL_SOLVER_PCG)
    prm_gen = tl.params(h=w["h"], rtol=1e-8, linear_solver=tl.TL_SOLVER_PCG, use_graph=1)
    t0 = time.time()
    tr = warmstart.generate(g64, m.X, w["f_ext"], args.steps, prm_gen, log_every=200)
    t_gen = time.time() - t0
    print(f"trajectory: {args.steps} steps in {t_gen:.1f} s", flush=True)
    ntrain = args.steps - args.holdout
    train_idx = np.arange(1, ntrain)
    test_idx = np.arange(ntrain + 1, min(args.steps, ntrain + 1 + args.eval_steps))
    assert len(test_idx) > 0
    t0 = time.time()
    model, hist = warmstart.train(g64, tr, m.fixed_nodes, train_idx, iters=args.iters, lr=args.lr,
                                  log_every=500)
    print(f"validation loss {model.val_loss:.4e} (zero-correction loss 1 by the target scale), "
          f"output shrinkage alpha {model.alpha:.3f}", flush=True)
    t_train = time.time() - t0
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    model.to_npz(args.out)
    g32 = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP32_ELEM)
    g32.build_pattern(m.fixed_nodes)
    prm_chosen = tl.params(h=w["h"], rtol=1e-8, linear_solver=tl.TL_SOLVER_PCG, lin_adaptive=1)
    prm_chosen_graph = tl.params(h=w["h"], rtol=1e-8, linear_solver=tl.TL_SOLVER_PCG, lin_adaptive=1,
                                 use_graph=1)
    plain, _ = warmstart.evaluate(g64, tr, test_idx, prm_plain, model, modes=["v_n"])
    fp64_starts, _ = warmstart.evaluate(g64, tr, test_idx, prm_chosen, model)
    fp32_starts, _ = warmstart.evaluate(g32, tr, test_idx, prm_chosen, model)
    fp32_graph, _ = warmstart.evaluate(g32, tr, test_idx, prm_chosen_graph, model)
    report = dict(workload=w["name"], steps=args.steps, holdout=args.holdout, eval_steps=len(test_idx),
                  train_steps=[int(train_idx[0]), int(train_idx[-1])],
                  test_steps=[int(test_idx[0]), int(test_idx[-1])],
                  generation_s=t_gen, training_s=t_train, loss_history=hist,
                  val_loss=model.val_loss, alpha=model.alpha,
                  plain_fp64_vn_pcg=plain["v_n"], fp64_adaptive=fp64_starts, fp32_adaptive=fp32_starts,
                  fp32_adaptive_graph=fp32_graph,
                  speedup_chosen_vs_plain=plain["v_n"]["mean_ms"] / fp32_graph["mlp"]["mean_ms"])
    print(json.dumps(report, indent=1))
    if args.report:
        with open(args.report, "w") as f:
            json.dump(report, f, indent=1)


if __name__ == "__main__":
    main()
