"""Learned Newton warm start: generate backward-Euler trajectories with the
plain Newton step (start v_n), train the per-node MLP with the library's own
kernels, and compare Newton iterations / time to the same 1e-8 residual from
the starts v_n (the paper's), the polynomial extrapolations of the velocity
history (linear from v_n, v_{n-1}; cubic from v_n .. v_{n-3}) and the MLP,
which learns a correction of the cubic extrapolation from the backward
differences of the history.  The inner tolerance is relative to the residual
at v_n in every case, so all starts converge to the same state within the
Newton tolerance.

Orchestration only: every array operation of the method (Newton steps,
features, training targets, normalisation statistics, forward / backward
passes, loss gradient, Adam) runs in the CUDA kernels behind include/tl.h;
torch provides device memory, random minibatch choice and timing events, and
the host turns a handful of float64 sums into scales.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import tl

NPARAM = tl.MLP_NPARAM


@dataclass
class Trajectory:
    q: list = field(default_factory=list)       # q_n per step (device float64)
    v: list = field(default_factory=list)       # v_n per step
    lam: list = field(default_factory=list)     # lambda at the start of the step
    f_ext: list = field(default_factory=list)
    stats: list = field(default_factory=list)


def generate(g, X, f_ext_fn, nsteps, prm, q0=None, v0=None, record_from=0, log_every=0):
    """Run nsteps of the plain Newton step from (q0, v0) (default: rest).
    Returns a Trajectory with the states at the start of steps
    record_from .. nsteps (one more state than steps)."""
    import torch
    nd = g.ndof
    q = torch.as_tensor(np.asarray(X).reshape(-1) if q0 is None else q0, dtype=torch.float64, device="cuda").clone()
    v = torch.zeros(nd, dtype=torch.float64, device="cuda") if v0 is None else v0.clone()
    lam = torch.zeros(max(3 * g.nfixed, 1), dtype=torch.float64, device="cuda")
    tr = Trajectory()
    for step in range(nsteps + 1):
        fe = torch.as_tensor(f_ext_fn(step), dtype=torch.float64, device="cuda") if f_ext_fn else None
        if step >= record_from:
            tr.q.append(q.clone())
            tr.v.append(v.clone())
            tr.lam.append(lam.clone())
            tr.f_ext.append(fe)
        if step == nsteps:
            break
        v_new, q_new, st = g.newton_step(prm, q, v, lam, f_ext=fe)
        if step >= record_from:
            tr.stats.append(st)
        q, v = q_new.clone(), v_new.clone()
        if log_every and step % log_every == 0:
            print(f"  step {step}: {st['inner_iters']} Newton iterations, {st['ms_total']:.1f} ms", flush=True)
    return tr


@dataclass
class WarmStartModel:
    params: object          # int16 CUDA tensor of bf16 bits (9219)
    s1: float               # scales of the first, second and third backward differences
    s2: float
    s3: float
    s_out: float            # output scale (shrinkage included)
    alpha: float = 1.0      # shrinkage factor chosen on the validation steps
    val_loss: float = float("nan")

    @property
    def scales(self):
        return (self.s1, self.s2, self.s3)

    def to_npz(self, path):
        np.savez(path, params=self.params.cpu().numpy(), s1=self.s1, s2=self.s2, s3=self.s3, s_out=self.s_out,
                 alpha=self.alpha, val_loss=self.val_loss)

    @classmethod
    def from_npz(cls, path):
        import torch
        d = np.load(path)
        return cls(torch.as_tensor(d["params"], device="cuda"), float(d["s1"]), float(d["s2"]), float(d["s3"]),
                   float(d["s_out"]), float(d["alpha"]), float(d["val_loss"]))


def history(tr, t, order=4):
    """(v_t, v_{t-1}, ..., ) of length `order` from a trajectory (None before its start)."""
    return tuple(tr.v[t - k] if t - k >= 0 else None for k in range(order))


def _scales(g, tr, idx, rounds=4):
    """Scales of the inputs and the output from the library's feature / target
    kernels and column sums over the steps idx.  s1, s2, s3 balance the three
    backward differences: each round divides s_k by the square root of group
    k's share of the nodes' (unit) input vectors times three, so that the three
    groups end with equal shares; s_out is the RMS of the resulting target."""
    import torch
    nn = g.nn
    feats = torch.empty(nn, 10, dtype=torch.float32, device="cuda")
    target = torch.empty(nn, 3, dtype=torch.float32, device="cuda")
    sc = np.ones(3)
    pick = idx[np.linspace(0, len(idx) - 1, min(20, len(idx))).astype(int)]
    for _ in range(rounds):
        sf = torch.zeros(10, dtype=torch.float64, device="cuda")
        for t in pick:
            g.mlp_features(history(tr, t), tuple(sc), feats)
            tl.mlp_col_sumsq(feats, sf)
        e = sf.cpu().numpy()[:9].reshape(3, 3).sum(axis=1)
        share = e / max(e.sum(), 1e-300)
        sc = sc * np.sqrt(np.maximum(3.0 * share, 1e-12))
    st = torch.zeros(3, dtype=torch.float64, device="cuda")
    for t in idx:
        g.mlp_target(tr.v[t + 1], history(tr, t), tuple(sc), 1.0, target)
        tl.mlp_col_sumsq(target, st)
    s_out = np.sqrt(st.cpu().numpy().sum() / (3.0 * nn * len(idx)))
    return tuple(float(max(x, 1e-30)) for x in (*sc, s_out))


def _glorot_init(rng):
    sizes = [(64, 10), (64,), (64, 64), (64,), (64, 64), (64,), (3, 64), (3,)]
    out = []
    for sz in sizes:
        if len(sz) == 2:
            lim = np.sqrt(6.0 / (sz[0] + sz[1]))
            out.append(rng.uniform(-lim, lim, size=sz).astype(np.float32).ravel())
        else:
            out.append(np.zeros(sz, np.float32))
    return np.concatenate(out)


def train(g, tr, fixed_nodes, train_idx, iters=2000, lr=2e-3, seed=0, log_every=0, val_frac=0.1,
          eval_every=100):
    """Fit the MLP to predict (v_{t+1} - b_t) / (s_out r_I), b_t the cubic
    extrapolation of v_t .. v_{t-3} (the error of that extrapolation), from the
    node-normalised backward differences at step t (mean squared error over
    free nodes).  Each
    iteration uses every node of one randomly drawn training step; Adam on a
    float32 master copy.

    Model selection on the last `val_frac` of the training steps (never
    trained on): the parameters with the lowest validation loss are kept, and
    the output scale is shrunk by the least-squares factor alpha in [0, 1] of
    the network output against the validation targets, so a network that does
    not generalise falls back towards the extrapolation itself (alpha = 0)."""
    import torch
    rng = np.random.default_rng(seed)
    train_idx = np.asarray(train_idx)
    train_idx = train_idx[train_idx >= 3]
    n_val = max(1, int(round(val_frac * len(train_idx))))
    fit_idx, val_idx = train_idx[:-n_val], train_idx[-n_val:]
    s1, s2, s3, s_out = _scales(g, tr, fit_idx)
    scales = (s1, s2, s3)
    nn = g.nn
    master = torch.as_tensor(_glorot_init(rng), device="cuda")
    P = torch.empty(NPARAM, dtype=torch.int16, device="cuda")
    m1 = torch.zeros(NPARAM, dtype=torch.float32, device="cuda")
    m2 = torch.zeros_like(m1)
    grads = torch.zeros_like(m1)
    tl.mlp_adam(master, P, grads, m1, m2, lr=0.0, step=1)          # P <- bf16(master)
    fixed = np.zeros(nn, bool)
    fixed[np.asarray(fixed_nodes, dtype=np.int64)] = True
    weight = torch.as_tensor(np.where(fixed, 0.0, 1.0 / max(1, (~fixed).sum())).astype(np.float32), device="cuda")
    feats = torch.empty(nn, 10, dtype=torch.float32, device="cuda")
    acts = torch.empty(nn, 192, dtype=torch.int16, device="cuda")
    out = torch.empty(nn, 3, dtype=torch.float32, device="cuda")
    target = torch.empty(nn, 3, dtype=torch.float32, device="cuda")
    zeros3 = torch.zeros(nn, 3, dtype=torch.float32, device="cuda")
    dout = torch.empty_like(out)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")

    def prepare(t):
        g.mlp_features(history(tr, t), scales, feats)
        g.mlp_target(tr.v[t + 1], history(tr, t), scales, s_out, target)

    val_pick = val_idx[np.linspace(0, len(val_idx) - 1, min(10, len(val_idx))).astype(int)]

    def weighted_sq(a, b):
        loss.zero_()
        tl.mlp_mse_grad(a, b, weight, dout, loss)
        return loss.item()

    def val_loss():
        tot = 0.0
        for t in val_pick:
            prepare(t)
            tl.mlp_forward(P, feats, out=out)
            tot += weighted_sq(out, target)
        return tot / len(val_pick)

    history_ = []
    best = (val_loss(), P.clone())
    history_.append((0, float("nan"), best[0]))
    for it in range(iters):
        t = int(rng.choice(fit_idx))
        prepare(t)
        tl.mlp_forward(P, feats, out=out, acts=acts)
        loss.zero_()
        tl.mlp_mse_grad(out, target, weight, dout, loss)
        grads.zero_()
        tl.mlp_backward(P, feats, acts, dout, grads)
        tl.mlp_adam(master, P, grads, m1, m2, lr=lr * (0.1 ** (it / max(1, iters))), step=it + 1)
        if (it + 1) % eval_every == 0 or it == iters - 1:
            vl = val_loss()
            history_.append((it + 1, loss.item(), vl))
            if vl < best[0]:
                best = (vl, P.clone())
            if log_every and ((it + 1) % log_every == 0 or it == iters - 1):
                print(f"  iter {it + 1}: train loss {loss.item():.4e}, validation loss {vl:.4e}", flush=True)
    P.copy_(best[1])
    # output shrinkage alpha = argmin sum w |alpha out - target|^2 = B / A on the
    # validation steps, from weighted squared norms the loss kernel forms:
    # A = |out|^2_w, C = |target|^2_w, L = |out - target|^2_w, B = (A + C - L) / 2
    A = B = 0.0
    for t in val_pick:
        prepare(t)
        tl.mlp_forward(P, feats, out=out)
        a_, c_, l_ = weighted_sq(out, zeros3), weighted_sq(target, zeros3), weighted_sq(out, target)
        A += a_
        B += 0.5 * (a_ + c_ - l_)
    alpha = float(min(1.0, max(0.0, B / A))) if A > 0 else 0.0
    model = WarmStartModel(P, s1, s2, s3, alpha * s_out)
    model.alpha, model.val_loss = alpha, best[0]
    return model, history_


START_ORDERS = {"v_n": 1, "linear": 2, "quadratic": 3, "cubic": 4}


def evaluate(g, tr, test_idx, prm, model=None, modes=None):
    """Newton iterations and time to the same tolerance on the stored test
    steps, from the starts in `modes`: "v_n" (the paper's), "linear",
    "quadratic", "cubic" (polynomial extrapolations of the last 2, 3, 4
    velocities) and "mlp" (needs model; its base is the cubic).  g may be a
    handle of either element precision; prm selects the linear solver."""
    import torch
    if modes is None:
        modes = ["v_n", "linear", "cubic"] + (["mlp"] if model is not None else [])
    res = {m: dict(iters=[], ms=[], ms_start=[], dev=[], g0=[], lin=[], ls=[]) for m in modes}
    work = torch.empty(13 * g.nn, dtype=torch.float32, device="cuda")
    vinit = torch.empty(g.ndof, dtype=torch.float64, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for t in test_idx:
        ref = tr.v[t + 1]
        for mode in modes:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e0.record()
            if mode == "v_n":
                vi = None
            elif mode == "mlp":
                g.warm_start(model.params, history(tr, t), model.scales, model.s_out, work=work, v_init=vinit)
                vi = vinit
            else:
                g.warm_start(None, history(tr, t, START_ORDERS[mode]), v_init=vinit)
                vi = vinit
            e1.record()
            lam = tr.lam[t].clone()
            v_new, _, st = g.newton_step(prm, tr.q[t], tr.v[t], lam, v_init=vi, f_ext=tr.f_ext[t])
            ms = 1e3 * (time.perf_counter() - t0)
            r = res[mode]
            r["iters"].append(st["inner_iters"])
            r["ms"].append(ms)
            r["ms_start"].append(e0.elapsed_time(e1))
            r["dev"].append((torch.linalg.norm(v_new - ref) / torch.linalg.norm(ref)).item())
            r["g0"].append(st["g_init"] / st["g_ref"])
            r["lin"].append(st["lin_iters"])
            r["ls"].append(st["ls_trials"])
    summary = {m: dict(mean_iters=float(np.mean(r["iters"])), mean_ms=float(np.mean(r["ms"])),
                       median_ms=float(np.median(r["ms"])),
                       mean_ms_start=float(np.mean(r["ms_start"])), max_rel_dev=float(np.max(r["dev"])),
                       median_g0_ratio=float(np.median(r["g0"])), mean_lin_iters=float(np.mean(r["lin"])),
                       mean_ls_trials=float(np.mean(r["ls"])), steps=len(r["ms"]))
               for m, r in res.items()}
    return summary, res
