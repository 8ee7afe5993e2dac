"""Benchmark of the T10 force + tangent + CSR-assembly hot path on GB300.

One step = one pass of the hot path over the 960,000-element box
(20 x 4 x 2 m, 200 x 40 x 20 hexes x 6 T10, SVK + Kelvin-Voigt, FP32 element
form, float64-class residual): the fused element kernel (internal force +
30x30 tangent + scatter into the fixed-pattern CSR Hessian, values zeroed
first), the clamp-penalty diagonal and the residual g with its norm (float64,
its mass product in double-float arithmetic when the autotuner picks it).

Prints ONE JSON line (rank 0).  Under torchrun every rank runs an independent
replica of the workload (the assembly needs no exchange; weak scaling).  At N = 1
the line also carries the Newton comparison (`newton`), the cost of general
constraint rows (`constraints`) and the ANCF3243 beam / ANCF3443 shell passes at the
paper's largest resolutions with their Newton steps (`ancf`).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "T10 force+tangent+assembly elems/s; Newton step ms to 1e-8, chosen vs plain"
UNIT = "elems/s"

# Algorithmic FP32 flops per element of the fused pass (force + tangent +
# assembly), counted from the formulas the kernel evaluates (FMA = 2), once
# per element, without the kernel's own redundancy.  Per quadrature point
# (SVK + KV): grad N 92, H 180, Fdot 180, J - 1 37, E 54, S 11, Edot 72,
# S_v 11, S_tot 6, B 36, P 64, f 180, tangent entries 278 (45 unique),
# A n per node 1,620, 55 blocks x 9 x 3 FMA 2,970 = 5,791; x 5 plus the
# force and tangent reductions and the mass term (457) = 29,412.
FLOPS_PER_ELEM = {("svk", False): 28_067, ("svk", True): 29_412,
                  ("mr", False): 33_782, ("mr", True): 36_477}

SM_COUNT, FP32_LANES_PER_SM, SM_MAX_MHZ = 152, 128, 2070.0


def fp32_alu_peak_tflops():
    """152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz max SM clock."""
    return SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12


def algorithmic_bytes_per_elem(ne, nn, nnz, value_bytes):
    """Minimal DRAM bytes of one pass, per element: every H value written once,
    node data (X, q_n, v) read once and f written once, per-element
    connectivity (40 B), geometry (13 values) and slot indices (100 B) read
    once, node row pointers read once."""
    per_node = 72 + 24 + 4
    per_elem = 40 + 13 * value_bytes + 100
    return (nnz * value_bytes + nn * per_node + ne * per_elem) / ne


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        self.gpu_id = gpu_id
        self.t_marks = {}

    def start(self):
        try:
            self.f = open(self.path, "w")
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id:
                cmd += ["-i", self.gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def mark(self, name):
        self.t_marks[name] = time.time()

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            rows = []
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if sm:
            loaded = [x for x in sm if x > 0.5 * max(sm)] or sm
            out.update(sm_mhz=statistics.median(loaded), sm_max_mhz=max(smax), samples=len(sm))
        out["reasons"] = sorted(reasons)
        return out


ELEM_KERNEL_SOURCES = [os.path.join(ROOT, "paper_2604_10357_gb300", "csrc", f)
                       for f in ("tl_element_pair.cu", "tl_element_impl.cuh", "tl_element_common.cuh", "tl_tilemap.cu",
                                 "tl_internal.cuh")]


def kernel_source_hash(files=ELEM_KERNEL_SOURCES):
    hs = hashlib.sha256()
    for f in files:
        hs.update(open(f, "rb").read())
    return hs.hexdigest()


def traffic_from_profile():
    """DRAM bytes per launch of the element kernel from the committed ncu
    summary, only if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "pair_kernel_traffic_box120k.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        h = kernel_source_hash()
        if d.get("kernel_sha256") == h:
            return d["dram_bytes_per_launch_full_workload"]
    except Exception:
        pass
    return None


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, on a bounded sample
# ---------------------------------------------------------------------------

def oracle_sample_workload(nx=10, ny=4, nz=4):
    """A sub-box of the large workload: same hex size (0.1 m), material and
    field recipe, nx*ny*nz*6 elements."""
    from paper_2604_10357_gb300 import inputs
    rng = np.random.default_rng(1000 + 5)
    m = inputs.box_t10(nx, ny, nz, 0.1 * nx, 0.1 * ny, 0.1 * nz)
    q, _ = inputs.sine_mode_field(m, 0.02, rng)
    v = inputs.gaussian_velocity(m, 0.05, rng)
    mat = dict(inputs.SVK_1E7, eta_d=1e3, lambda_d=1e3)
    return m, q, v, mat


def oracle_step_rate(budget_s=12.0, min_reps=1, nx=10, ny=4, nz=4):
    """Elements/s of the oracle's force + tangent + CSR assembly + residual."""
    from oracle import assembly as asm
    m, q, v, mat = oracle_sample_workload(nx, ny, nz)
    om = asm.OracleMesh(m.X, m.conn, [mat], fixed_nodes=m.fixed_nodes)
    om.pattern()
    lam = np.zeros(3 * len(m.fixed_nodes))
    reps, t0 = 0, time.perf_counter()
    while True:
        om.hessian_values(q, v, 1e-3, 1e12)
        om.residual(v, q, v, 1e-3, None, (0, 0, -9.81), lam, 1e12)
        reps += 1
        el = time.perf_counter() - t0
        if reps >= min_reps and el >= budget_s:
            break
    return reps * m.ne / el, reps, m.ne, el


def oracle_ancf_rate(kind, budget_s=6.0, min_reps=1):
    """Elements/s of the oracle's ANCF Hessian assembly (element force +
    tangent + CSR values, the assembly pass the GPU arm times) on a bounded
    sample of the same element kind, material and state recipe: a 64-element
    beam or a 4 x 4 shell.  Reference geometry and mass are built untimed
    (precomputation, as on the device)."""
    from oracle import ancf as oancf
    from paper_2604_10357_gb300 import inputs
    if kind == "ancf3243":
        m, h, curv = inputs.beam_ancf3243(64), 1e-3, 1e-5
    else:
        m, h, curv = inputs.shell_ancf3443(4, 4), 5e-4, 0.25
    rng = np.random.default_rng(1000 + 8)
    q = inputs.ancf_perturbation(m, inputs.ancf_bend(m, curv), 0.001, rng)
    v = rng.normal(0.0, 0.01, size=q.shape)
    v[m.fixed_nodes] = 0.0
    om = oancf.OracleAncfMesh(kind, m.E0, m.conn, m.dims, [dict(inputs.SVK_7E8)], fixed_nodes=m.fixed_nodes)
    om.pattern()
    reps, t0 = 0, time.perf_counter()
    while True:
        om.hessian_values(q, v, h, 1e12)
        om.internal_force(q, v, h)
        reps += 1
        el = time.perf_counter() - t0
        if reps >= min_reps and el >= budget_s:
            break
    return reps * m.ne / el, reps, m.ne, el


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def replica_aggregate(ms, ne, steps, world, device="cuda"):
    """Max over ranks of the timed region (ms) and the whole-job rate: every
    rank assembles its own replica of ne elements per step (weak scaling)."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * ne * steps / (ms_max * 1e-3)


def run_ours(args, rank, world):
    import torch

    from paper_2604_10357_gb300 import build, inputs, tl

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    tl.load_library()

    w = inputs.workload_large_svk_kv(scale=args.scale)
    m = w["mesh"]
    prec = tl.TL_FP32_ELEM if args.precision == "fp32" else tl.TL_FP64
    stream = torch.cuda.current_stream()
    g = tl.Mesh(m.X, m.conn, [w["material"]], precision=prec, stream=stream)
    t_pat = time.perf_counter()
    nnz = g.build_pattern(m.fixed_nodes)
    t_pat = time.perf_counter() - t_pat
    h, rho = w["h"], 1e12
    prm = tl.params(h=h, rho_alm=rho)
    q = torch.as_tensor(w["q_n"].reshape(-1), device="cuda")
    v = torch.as_tensor(w["v"].reshape(-1), device="cuda")
    vdtype = torch.float32 if prec == tl.TL_FP32_ELEM else torch.float64
    values = torch.empty(nnz, dtype=vdtype, device="cuda")
    f = torch.empty(3 * m.nn, dtype=torch.float64, device="cuda")
    res = torch.empty(3 * m.nn, dtype=torch.float64, device="cuda")
    gnorm = torch.empty(1, dtype=torch.float64, device="cuda")

    def step(qd, vd):
        g.assemble_hessian(qd, vd, h, rho, values=values, f_int=f)
        g.eval_residual(prm, qd, vd, vd, f_int=f, g=res, g_norm=gnorm)

    # launch shapes picked by the library's autotuner on this mesh (untimed),
    # then any shape the command line fixes (--shape key=value)
    tune = g.autotune(q, v, h, reps=3) if not args.no_autotune else g.tune_get()
    if args.shape:
        g.tune_set(**{k: int(val) for k, val in (kv.split("=") for kv in args.shape)})
        tune.update(g.tune_get())

    for _ in range(args.warmup):
        step(q, v)
    g.sync()
    g.timing_read()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    if rank == 0:
        sampler.start()
        time.sleep(0.5)
    g.timing_enable(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        step(q, v)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = ev0.elapsed_time(ev1)
    tim = g.timing_read()
    g.timing_enable(False)
    g.sync()

    # end-to-end through the public API with host buffers: every step's inputs
    # copied H2D from pinned memory, the pass, D2H of the residual norm.  The
    # copies of step k+1 run on a copy stream into the other of two device
    # buffers while step k computes (events order a buffer's copy after the
    # step that last read it, and the step after its copy).
    e2e = None
    if not args.no_e2e:
        q_h = torch.as_tensor(w["q_n"].reshape(-1)).pin_memory()
        v_h = torch.as_tensor(w["v"].reshape(-1)).pin_memory()
        out_h = torch.empty(1, dtype=torch.float64).pin_memory()
        bufs = [(torch.empty_like(q), torch.empty_like(v)) for _ in range(2)]
        cstream = torch.cuda.Stream()
        ke = max(3, min(args.steps, 50))

        def run_e2e(nsteps):
            ready = [torch.cuda.Event() for _ in range(2)]
            free = [torch.cuda.Event() for _ in range(2)]
            cstream.wait_stream(stream)

            def upload(k):
                qd, vd = bufs[k % 2]
                with torch.cuda.stream(cstream):
                    if k >= 2:
                        cstream.wait_event(free[k % 2])
                    qd.copy_(q_h, non_blocking=True)
                    vd.copy_(v_h, non_blocking=True)
                    ready[k % 2].record(cstream)

            upload(0)
            for k in range(nsteps):
                if k + 1 < nsteps:
                    upload(k + 1)
                stream.wait_event(ready[k % 2])
                step(*bufs[k % 2])
                out_h.copy_(gnorm, non_blocking=True)
                free[k % 2].record(stream)

        run_e2e(2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run_e2e(ke)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = e0.elapsed_time(e1) / ke
        e2e = {"value": m.ne / (ms_e2e * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": int(q_h.numel() * 8 + v_h.numel() * 8),
               "d2h_bytes_per_step": int(out_h.numel() * 8), "ms_per_step": ms_e2e, "steps": ke}
    if rank == 0:
        sampler.stop()

    ms_max, value = replica_aggregate(ms, m.ne, args.steps, world)
    ms_step = ms_max / args.steps

    if rank != 0:
        return None
    kind = w["material"]["kind"]
    kv = bool(w["material"].get("eta_d") or w["material"].get("lambda_d"))
    vbytes = 4 if prec == tl.TL_FP32_ELEM else 8
    elem_ms = tim["ms_element"] / max(1, tim["n_element"])
    flops = FLOPS_PER_ELEM[(kind, kv)] * m.ne
    bpe = algorithmic_bytes_per_elem(m.ne, m.nn, nnz, vbytes)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    if prec == tl.TL_FP32_ELEM:
        peak = fp32_alu_peak_tflops()
        achieved = flops / (elem_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak,
                    "peak_source": "FP32 ALU: 152 SM x 128 lanes x 2 x 2070 MHz (derived, not measured)"}
    else:
        roofline = {"bound": "alu", "achieved": flops / (elem_ms * 1e-3) / 1e12, "peak": None,
                    "unit": "TFLOP/s", "frac": None, "peak_source": "FP64 ALU peak not yet measured"}
    roofline["traffic"] = traffic_from_profile()
    roofline["kernel"] = ("pair_kernel (closed-form SVK pair tangent, fused force + tangent + CSR scatter)"
                          if tune.get("elem_pair") and prec == tl.TL_FP32_ELEM else
                          "elem_kernel (fused force + tangent + CSR scatter)")
    roofline["kernel_ms"] = elem_ms
    roofline["residual_ms"] = tim["ms_residual"] / max(1, tim["n_residual"])
    roofline["algorithmic_bytes_per_elem"] = bpe
    roofline["hbm_frac_of_measured"] = (bpe * m.ne / (elem_ms * 1e-3)) / (hbm * 1e9)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == tl.TL_FP32_ELEM else "f64", "data": "synthetic",
        "config": {"workload": w["name"], "ne": m.ne, "nn": m.nn, "ndof": 3 * m.nn, "nnz": nnz,
                   "precision": ("FP32 element form, float64 residual (mass product double-float: "
                                 f"{'yes' if tune.get('residual_split') else 'no'})")
                                if prec == tl.TL_FP32_ELEM else "FP64",
                   "material": "SVK E=1e7 nu=0.3 + Kelvin-Voigt 1e3", "h": h,
                   "l2": "no flush: the H values written every step (%.2f GB) exceed L2" % (nnz * vbytes / 1e9),
                   "parallelism": f"replicas x{world}", "pattern_build_s": t_pat,
                   "launch_shapes": {k: tune[k] for k in ("elem_pair", "elem_ws", "elem_occ2", "elem_spread",
                                                          "elem_prefetch", "elem_xchg", "elem_full_grid", "elem_agg",
                                                          "spmv_group", "spmv_row", "residual_lanes", "residual_split")},
                   "launch_shape_ms": {k: tune[k] for k in ("ms_pair", "ms_ws", "ms_occ2", "ms_spread", "ms_element",
                                                            "ms_agg", "ms_spmv", "ms_spmv_row", "ms_residual",
                                                            "ms_residual_split")}},
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": int(tim["launches"]),
        "clocks": sampler.summary(),
    }
    return line


def run_newton(args):
    """Newton step ms to the 1e-8 relative residual on the 103,680-element
    cantilever (12 x 1.2 x 1.2 m, SVK, gravity + seeded tip loads), on the
    held-out steps of the warm-start trajectory (steps 1101.. of the trajectory
    from rest; the network was trained on steps 3..1099).  'plain' = the
    paper's step: FP64 element form, start v_n, host-driven loop (||g|| read
    back every iteration), PCG to 1e-10; 'chosen' = FP32 element form,
    inexact-Newton PCG, the whole step as one captured CUDA graph, from the
    learned start (a correction of the cubic extrapolation of the velocity
    history), beside the same arm from the linear (2 v_n - v_{n-1}) and cubic
    extrapolations.  All from the same stored states to the same target; the
    trajectory itself is generated (untimed) with the plain step in its graph
    form.  Returns (compact summary, details)."""
    import torch

    from paper_2604_10357_gb300 import inputs, tl, warmstart
    w = inputs.workload_warm_start_svk()
    m = w["mesh"]
    g64 = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP64)
    g64.build_pattern(m.fixed_nodes)
    g32 = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP32_ELEM)
    g32.build_pattern(m.fixed_nodes)
    plain = tl.params(h=w["h"], rtol=1e-8, linear_solver=tl.TL_SOLVER_PCG)
    gen = tl.params(h=w["h"], rtol=1e-8, linear_solver=tl.TL_SOLVER_PCG, use_graph=1)
    chosen = tl.params(h=w["h"], rtol=1e-8, linear_solver=tl.TL_SOLVER_PCG, lin_adaptive=1,
                       use_graph=0 if args.newton_no_graph else 1)
    t0_step, n_eval = args.newton_start, args.newton_steps
    t_gen = time.time()
    tr = warmstart.generate(g64, m.X, w["f_ext"], t0_step + n_eval + 1, gen, record_from=t0_step - 3)
    t_gen = time.time() - t_gen
    test_idx = list(range(3, n_eval + 3))          # trajectory-local indices (record_from offset)
    model_path = os.path.join(ROOT, "paper_2604_10357_gb300", "data", "warmstart_box120x12x12.npz")
    model = warmstart.WarmStartModel.from_npz(model_path) if os.path.exists(model_path) else None
    starts = ["linear", "cubic"] + (["mlp"] if model is not None else [])
    # launch shapes of both arms picked by the autotuner on the first held-out state (untimed)
    shape_keys = ("elem_pair", "elem_occ2", "elem_prefetch", "elem_xchg", "elem_full_grid", "elem_agg", "spmv_group",
                  "spmv_row", "pcg_f32", "residual_split")
    shapes = {}
    for name, g in (("plain", g64), ("chosen", g32)):
        t = g.tune_get() if args.no_autotune else g.autotune(tr.q[test_idx[0]], tr.v[test_idx[0]], w["h"], reps=3)
        shapes[name] = {k: t[k] for k in shape_keys}
    # one untimed pass of each arm first (graph capture, first-use allocations)
    warmstart.evaluate(g64, tr, test_idx[:1], plain, modes=["v_n"])
    warmstart.evaluate(g32, tr, test_idx[:1], chosen, model, modes=starts)
    p_sum, _ = warmstart.evaluate(g64, tr, test_idx, plain, modes=["v_n"])
    c_sum, _ = warmstart.evaluate(g32, tr, test_idx, chosen, model, modes=starts)
    best = "mlp" if model is not None else "cubic"
    details = {"workload": w["name"], "ndof": 3 * m.nn, "steps": [t0_step, t0_step + n_eval - 1],
               "target": "||g|| <= 1e-8 ||g(v_n)||", "trajectory_generation_s": t_gen,
               "plain": dict(p_sum["v_n"], desc="FP64 element form, start v_n, host loop, PCG 1e-10"),
               "chosen_starts": c_sum, "launch_shapes": shapes,
               "model": os.path.relpath(model_path, ROOT) if model is not None else None,
               "model_alpha": model.alpha if model is not None else None}
    # the chosen arm with the Armijo line search of eq. armijo (trial residual per Newton step)
    chosen_ls = tl.params(h=w["h"], rtol=1e-8, linear_solver=tl.TL_SOLVER_PCG, lin_adaptive=1, line_search=1,
                          use_graph=0 if args.newton_no_graph else 1)
    warmstart.evaluate(g32, tr, test_idx[:1], chosen_ls, model, modes=[best])
    l_sum, _ = warmstart.evaluate(g32, tr, test_idx[:10], chosen_ls, model, modes=[best])
    details["chosen_line_search"] = dict(l_sum[best], desc="chosen arm with the Armijo line search (10 steps)")
    # the first-order inner solver (Algorithm 2) from the first held-out state:
    # cost per AdamW update and the gradient reduction a fixed budget reaches
    t_a = test_idx[0]
    lam_a = tr.lam[t_a].clone()
    _, g0 = g32.eval_residual(tl.params(h=w["h"]), tr.q[t_a], tr.v[t_a], tr.v[t_a], f_ext=tr.f_ext[t_a], lam=lam_a)
    g0 = g0.item()
    a_prm = tl.adamw_params(lr=1e-4, max_inner=200, check_every=50)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, st_a = g32.adamw_step(tl.params(h=w["h"], max_outer=1), a_prm, tr.q[t_a], tr.v[t_a], lam_a,
                                f_ext=tr.f_ext[t_a], raise_on_nonconvergence=False)
    ms_a = 1e3 * (time.perf_counter() - t0)
    details["adamw"] = dict(inner_iters=st_a["inner_iters"], ms=ms_a, ms_per_update=ms_a / max(1, st_a["inner_iters"]),
                            g_ratio=st_a["g_norm"] / g0, converged=st_a["converged"],
                            desc="Algorithm 2, lr 1e-4, 200 updates from the first held-out state (not converged: "
                                 "a first-order rate)")
    g64.close()
    g32.close()

    def brief(d):
        return {"ms": round(d["mean_ms"], 3), "newton_its": round(d["mean_iters"], 2),
                "pcg_its": round(d["mean_lin_iters"], 1), "g0_ratio": float("%.3g" % d["median_g0_ratio"]),
                "max_rel_dev": float("%.2g" % d["max_rel_dev"])}

    summary = {"steps": n_eval, "first_step": t0_step, "ndof": 3 * m.nn,
               "plain_ms": round(p_sum["v_n"]["mean_ms"], 3),
               "chosen_ms": round(c_sum[best]["mean_ms"], 3), "chosen_start": best,
               "speedup": round(p_sum["v_n"]["mean_ms"] / c_sum[best]["mean_ms"], 2),
               "plain": brief(p_sum["v_n"]), **{f"chosen_{k}": brief(c_sum[k]) for k in starts}}
    return summary, details


class ErrorNorms:
    """Comparison norms of a GPU result against the oracle (the paper gives
    none): force error relative to the largest element force, element-tangent
    error relative to each element's own Frobenius norm, CSR values relative to
    the largest value and in the 2-norm."""

    @staticmethod
    def force_error(f_gpu, f_ora, fe_ora):
        return float(np.abs(np.asarray(f_gpu) - np.asarray(f_ora)).max() / np.abs(fe_ora).max())

    @staticmethod
    def tangent_error(K_gpu, K_ora):
        K_gpu = np.asarray(K_gpu, dtype=np.float64).reshape(-1, 900)
        K_ora = np.asarray(K_ora, dtype=np.float64).reshape(-1, 900)
        den = np.linalg.norm(K_ora, axis=1)
        num = np.linalg.norm(K_gpu - K_ora, axis=1)
        return float(np.max(num[den > 0] / den[den > 0]))

    @staticmethod
    def values_error(v_gpu, v_ora):
        d = np.asarray(v_gpu, dtype=np.float64) - np.asarray(v_ora, dtype=np.float64)
        return float(np.abs(d).max() / np.abs(v_ora).max()), float(np.linalg.norm(d) / np.linalg.norm(v_ora))


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def _oracle_rate_worker(budget_s):
    return oracle_step_rate(budget_s=budget_s)


def oracle_all_cores_rate(budget_s=8.0):
    """The oracle's element loop on every host core: one process per core, each
    assembling its own copy of the bounded sample (spawned processes, one BLAS
    thread each); the rate is the sum over processes."""
    import multiprocessing as mp
    ncores = os.cpu_count() or 1
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_keep:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(ncores) as pool:
            res = pool.map(_oracle_rate_worker, [budget_s] * ncores)
    finally:
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return sum(r[0] for r in res), ncores, res[0][2]


def _time_passes(g, fn, reps=10, warm=3):
    """Mean ms per call of fn over reps calls (CUDA events), and the library's
    element-kernel ms per launch over the same calls."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    g.timing_read()
    g.timing_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    t = g.timing_read()
    g.timing_enable(False)
    return e0.elapsed_time(e1) / reps, t["ms_element"] / max(1, t["n_element"]), t


def run_fp64_large(args):
    """The same 960,000-element step with the FP64 element form (the paper's
    precision): element kernel ms against the float64 ALU roofline."""
    import torch

    from paper_2604_10357_gb300 import inputs, tl
    w = inputs.workload_large_svk_kv(scale=args.scale)
    m = w["mesh"]
    g = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP64)
    nnz = g.build_pattern(m.fixed_nodes)
    q = torch.as_tensor(w["q_n"].reshape(-1), device="cuda")
    v = torch.as_tensor(w["v"].reshape(-1), device="cuda")
    h = w["h"]
    if not args.no_autotune:
        g.autotune(q, v, h, reps=2)
    vals = torch.empty(nnz, dtype=torch.float64, device="cuda")
    f = torch.empty(3 * m.nn, dtype=torch.float64, device="cuda")
    res = torch.empty_like(f)
    gn = torch.empty(1, dtype=torch.float64, device="cuda")
    prm = tl.params(h=h, rho_alm=1e12)

    def step():
        g.assemble_hessian(q, v, h, 1e12, values=vals, f_int=f)
        g.eval_residual(prm, q, v, v, f_int=f, g=res, g_norm=gn)

    ms, kms, _ = _time_passes(g, step, reps=5)
    g.close()
    flops = FLOPS_PER_ELEM[("svk", True)] * m.ne
    ach = flops / (kms * 1e-3) / 1e12
    return {"workload": w["name"], "dtype": "f64", "ms_per_step": ms, "elems_per_s": m.ne / (ms * 1e-3),
            "kernel_ms": kms, "roofline": {"bound": "alu", "achieved": ach, "peak": fp64_alu_peak_tflops(),
                                           "unit": "TFLOP/s", "frac": ach / fp64_alu_peak_tflops(),
                                           "peak_source": "FP64 ALU: 152 SM x 2 FMA/clk x 2 x 2070 MHz (derived)"}}


def run_mid(args):
    """The 15,360-element Mooney-Rivlin + Kelvin-Voigt box: element pass of both
    forms (elems/s), and the errors of the FP32 form (and of FP64) against the
    FP64 oracle for the internal force, the element tangents h K_t + D, the
    CSR Hessian values, and one backward-Euler Newton step: the oracle's
    residual at each form's converged velocity, and the distance between the
    two forms' velocities."""
    import torch

    from oracle import assembly as asm
    from paper_2604_10357_gb300 import inputs, tl
    he = ErrorNorms
    w = inputs.workload_mid_mr_kv()
    m = w["mesh"]
    h, rho = w["h"], 1e12
    om = asm.OracleMesh(m.X, m.conn, [w["material"]], fixed_nodes=m.fixed_nodes)
    x = w["q_n"] + h * w["v"]
    fe = om.element_forces(x, w["v"])
    f_ora = om.internal_force(w["q_n"], w["v"], h)
    K_ora = om.element_tangents(x, w["v"], h, 1.0)
    v_ora = om.hessian_values(w["q_n"], w["v"], h, rho)
    _, _, row_ptr, col = om.pattern()
    pen = asm.csr_positions(row_ptr, col, om.fixed_dofs, om.fixed_dofs)
    rest = np.ones(len(v_ora), bool)
    rest[pen] = False
    q = torch.as_tensor(w["q_n"].reshape(-1), device="cuda")
    v = torch.as_tensor(w["v"].reshape(-1), device="cuda")
    qN_h = (m.X + 0.05 * (w["q_n"] - m.X)).reshape(-1)
    qN = torch.as_tensor(qN_h, device="cuda")
    out = {"workload": w["name"], "ne": m.ne, "ndof": 3 * m.nn}
    vout = {}
    for name, prec in (("fp64", tl.TL_FP64), ("fp32", tl.TL_FP32_ELEM)):
        g = tl.Mesh(m.X, m.conn, [w["material"]], precision=prec)
        nnz = g.build_pattern(m.fixed_nodes)
        if not args.no_autotune:
            g.autotune(q, v, h, reps=2)
        vals = torch.empty(nnz, dtype=g.vdtype, device="cuda")
        f = torch.empty(3 * m.nn, dtype=torch.float64, device="cuda")
        ms, kms, _ = _time_passes(g, lambda: g.assemble_hessian(q, v, h, rho, values=vals, f_int=f), reps=10)
        f_gpu = g.eval_force(q, v, h).cpu().numpy()
        K_gpu = g.eval_tangent(q, v, h, h, 1.0).cpu().numpy()
        vals_h = g.assemble_hessian(q, v, h, rho).cpu().numpy().astype(np.float64)
        emax, e2 = he.values_error(vals_h[rest], v_ora[rest])
        out[name] = {"element_pass_ms": ms, "kernel_ms": kms, "elems_per_s": m.ne / (ms * 1e-3),
                     "err_force": he.force_error(f_gpu, f_ora, fe), "err_tangent": he.tangent_error(K_gpu, K_ora),
                     "err_values_max": emax, "err_values_2": e2}
        # one Newton step from (q_N, v_n) under gravity, start v_n (the full
        # deformed state's Newton matrix is indefinite, see newton_state)
        try:
            prm = (tl.params(h=h, rho_alm=rho, rtol=1e-8, linear_solver=tl.TL_SOLVER_PCG) if prec == tl.TL_FP64 else
                   tl.params(h=h, rho_alm=rho, rtol=1e-8, linear_solver=tl.TL_SOLVER_PCG, lin_adaptive=1,
                             use_graph=1))
            lam = torch.zeros(3 * len(m.fixed_nodes), dtype=torch.float64, device="cuda")
            g.newton_step(prm, qN, v, lam, raise_on_nonconvergence=False)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lam = torch.zeros_like(lam)
            vn, _, st = g.newton_step(prm, qN, v, lam, raise_on_nonconvergence=False)
            torch.cuda.synchronize()
            ms_newton = 1e3 * (time.perf_counter() - t0)
            vout[name] = vn.cpu().numpy()
            lam_inner = lam.cpu().numpy() - rho * om.constraint(qN_h + h * vout[name])
            g_ref = np.linalg.norm(om.residual(w["v"].reshape(-1), qN_h, w["v"].reshape(-1), h, None,
                                               (0.0, 0.0, -9.81), np.zeros(3 * len(m.fixed_nodes)), rho))
            g_at = np.linalg.norm(om.residual(vout[name], qN_h, w["v"].reshape(-1), h, None,
                                              (0.0, 0.0, -9.81), lam_inner, rho))
            out[name]["newton"] = {"status": st["status"], "its": st["inner_iters"], "pcg_its": st["lin_iters"],
                                   "ms": ms_newton, "oracle_residual_ratio": g_at / g_ref}
        except Exception as exc:
            out[name]["newton"] = {"error": f"{type(exc).__name__}: {exc}"}
        g.close()
    out["newton_fp32_vs_fp64_velocity"] = (float(np.linalg.norm(vout["fp32"] - vout["fp64"])
                                                 / np.linalg.norm(vout["fp64"])) if len(vout) == 2 else None)
    out["newton_state"] = ("q_n = X + (q - X) / 20 (the workload's sine-mode field at a twentieth of its amplitude), "
                           "v_n its velocity field, gravity, lambda = 0: in the full deformed state the "
                           "Mooney-Rivlin Newton matrix M/h + h K_t + D is indefinite at h = 1e-3 (compressive "
                           "stresses make the negative geometric part of h K_t exceed the smallest eigenvalues of "
                           "M/h), so neither the Cholesky nor the CG inner solve applies there; at a twentieth it "
                           "is positive definite (the Newton parity tests use the same state)")
    out["norms"] = ("force: max|df| / max element |f|; tangent: max over elements of ||dK||_F / ||K||_F (h K_t + D); "
                    "values: max|dH| / max|H| and ||dH|| / ||H|| without the clamp-penalty diagonal; Newton: the "
                    "oracle's residual at the GPU velocity over its residual at v_n")
    return out


def run_batched(args):
    """48 bodies of uneven size (boxes and cylinders, SVK and Mooney-Rivlin; 1k to
    60k T10 each) in one handle: the fused element pass over all bodies (one
    persistent launch per kernel kind: the SVK segments in the pair kernel, the
    Mooney-Rivlin ones in the generic kernel), and the batched Newton step of all
    bodies from rest under gravity as one captured graph (FP32 element form).  The
    bodies are independent, so H is block diagonal and one Newton loop serves all
    of them: every body takes the same iteration count."""
    import torch

    from paper_2604_10357_gb300 import inputs, tl
    w = inputs.workload_batched()
    m = w["mesh"]
    h, rho = w["h"], 1e12
    g = tl.Mesh(m.X, m.conn, w["materials"], w["mat_of_elem"], precision=tl.TL_FP32_ELEM)
    nnz = g.build_pattern(m.fixed_nodes)
    q = torch.as_tensor(w["q_n"].reshape(-1), device="cuda")
    v = torch.as_tensor(w["v"].reshape(-1), device="cuda")
    if not args.no_autotune:
        g.autotune(q, v, h, reps=2)
    vals = torch.empty(nnz, dtype=torch.float32, device="cuda")
    f = torch.empty(3 * m.nn, dtype=torch.float64, device="cuda")
    ms, kms, t = _time_passes(g, lambda: g.assemble_hessian(q, v, h, rho, values=vals, f_int=f), reps=10)
    launches = t["launches"] / 10.0
    prm = tl.params(h=h, rho_alm=rho, rtol=1e-8, linear_solver=tl.TL_SOLVER_PCG, lin_adaptive=1, use_graph=1)
    qn = torch.as_tensor(m.X.reshape(-1), device="cuda")
    vn = torch.zeros_like(qn)
    lam = torch.zeros(3 * len(m.fixed_nodes), dtype=torch.float64, device="cuda")
    steps = []
    for k in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        v1, q1, st = g.newton_step(prm, qn, vn, lam, raise_on_nonconvergence=False)
        torch.cuda.synchronize()
        steps.append({"ms": 1e3 * (time.perf_counter() - t0), "its": st["inner_iters"], "pcg_its": st["lin_iters"],
                      "converged": st["converged"], "g_ratio": st["g_norm"] / max(st["g_ref"], 1e-300)})
        qn, vn = q1.clone(), v1.clone()
    g.close()
    return {"workload": w["name"], "bodies": len(w["meshes"]), "ne": m.ne, "nnz": int(nnz),
            "element_pass_ms": ms, "kernel_ms": kms, "elems_per_s": m.ne / (ms * 1e-3),
            "kernel_launches_per_pass": launches,
            "newton_from_rest": {"first_step_incl_capture_ms": steps[0]["ms"],
                                 "ms": statistics.median(s_["ms"] for s_ in steps[1:]),
                                 "its_per_body": [s_["its"] for s_ in steps], "pcg_its": [s_["pcg_its"] for s_ in steps],
                                 "converged": [s_["converged"] for s_ in steps],
                                 "g_ratio": [float("%.3g" % s_["g_ratio"]) for s_ in steps]}}


def run_direct(args):
    """The vendor sparse direct solver (cuSOLVER Cholesky) inside the FP64 Newton
    step on the 240-element box and on the 15,360-element box (its field at a
    twentieth of the amplitude, where the Newton matrix is definite): the solver's
    time reported apart from assembly (the step's own timers), three steps each
    (the first one includes the symbolic analysis)."""
    import torch

    from paper_2604_10357_gb300 import inputs, tl
    out = {}
    for name, wf, scale in (("c1_240", inputs.workload_small_svk, 1.0), ("c2_15360", inputs.workload_mid_mr_kv, 0.05)):
        try:
            w = wf()
            m = w["mesh"]
            g = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP64)
            g.build_pattern(m.fixed_nodes)
            prm = tl.params(h=w["h"], rtol=1e-8, linear_solver=tl.TL_SOLVER_DIRECT)
            q = torch.as_tensor((m.X + scale * (w["q_n"] - m.X)).reshape(-1), device="cuda")
            v = torch.as_tensor(w["v"].reshape(-1), device="cuda")
            rows = []
            for k in range(3):
                lam = torch.zeros(3 * len(m.fixed_nodes), dtype=torch.float64, device="cuda")
                _, _, st = g.newton_step(prm, q, v, lam, raise_on_nonconvergence=False)
                rows.append({k2: st[k2] for k2 in ("ms_total", "ms_assembly", "ms_solver", "inner_iters",
                                                   "converged")})
            g.close()
            out[name] = {"ndof": 3 * m.nn, "field_scale": scale, "first": rows[0],
                         "ms_total": statistics.median(r["ms_total"] for r in rows[1:]),
                         "ms_solver": statistics.median(r["ms_solver"] for r in rows[1:]),
                         "ms_assembly": statistics.median(r["ms_assembly"] for r in rows[1:]),
                         "newton_its": rows[-1]["inner_iters"]}
        except Exception as exc:
            out[name] = {"error": f"{type(exc).__name__}: {exc}"}
    return out


def run_reference(args, rank, world):
    """The oracle on the host cores, on this arm's metric: each step a bounded
    sample (a 4x2x2-hex sub-box of the same workload, 96 elements)."""
    if rank != 0:
        return None
    from oracle import assembly as asm
    m, q, v, mat = oracle_sample_workload(4, 2, 2)
    om = asm.OracleMesh(m.X, m.conn, [mat], fixed_nodes=m.fixed_nodes)
    om.pattern()
    lam = np.zeros(3 * len(m.fixed_nodes))

    def step():
        om.hessian_values(q, v, 1e-3, 1e12)
        om.residual(v, q, v, 1e-3, None, (0, 0, -9.81), lam, 1e12)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    value = args.steps * m.ne / el
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "box 20x4x2 m, 200x40x20 hex x6 = 960,000 T10, SVK+KV",
                       "sample": f"{m.ne}-element sub-box (4x2x2 hexes, same hex size and field recipe) per step"},
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT, "cores": 1, "cpu": cpu_model(),
                             "host_cores": os.cpu_count(),
                             "sample": f"{m.ne} elements per step, {args.steps} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_constraints(args):
    """Cost of general linear constraint rows (Sec. 4.2) in the assembly and
    the residual: the 103,680-element cantilever with its tip face tied into a
    plate (each tip-face node tied to its next neighbour along y in all three
    DOFs: rows c = q_I - q_J - (X_I - X_J)), against the same handle shape
    without them; Hessian assembly (fused force) + residual per pass, CUDA
    events over 20 passes after 3 warm-ups."""
    import torch

    from paper_2604_10357_gb300 import inputs, tl
    w = inputs.workload_warm_start_svk()
    m = w["mesh"]
    X = m.X
    tip = np.nonzero(np.isclose(X[:, 0], X[:, 0].max()))[0]
    order = np.lexsort((X[tip, 1], X[tip, 2]))
    tip = tip[order]
    ny = len(np.unique(np.round(X[tip, 1], 9)))
    rows_ptr, rows_col, rows_val = [0], [], []
    for k in range(len(tip) - 1):
        if (k + 1) % ny == 0:
            continue                                      # the next node is on the next z line
        a, b = tip[k], tip[k + 1]
        for d in range(3):
            rows_col += [3 * a + d, 3 * b + d]
            rows_val += [1.0, -1.0]
            rows_ptr.append(len(rows_col))
    rows_ptr = np.array(rows_ptr, dtype=np.int32)
    rows_col = np.array(rows_col, dtype=np.int32)
    rows_val = np.array(rows_val)
    bvec = np.array([rows_val[rows_ptr[r]:rows_ptr[r + 1]] @ X.ravel()[rows_col[rows_ptr[r]:rows_ptr[r + 1]]]
                     for r in range(len(rows_ptr) - 1)])
    rng = np.random.default_rng(77)
    q = torch.as_tensor(inputs.uniform_perturbation(m, 0.01, rng).reshape(-1), device="cuda")
    v = torch.as_tensor(inputs.gaussian_velocity(m, 0.05, rng).reshape(-1), device="cuda")
    h, rho = w["h"], 1e12
    out = {"workload": w["name"], "ncon": int(len(bvec)), "rows": "tip face tied along y (3 per node pair)"}
    for tag, with_c in (("without", False), ("with", True)):
        g = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP32_ELEM)
        if with_c:
            g.set_constraints(rows_ptr, rows_col, rows_val, bvec)
        g.build_pattern(m.fixed_nodes)
        lam = torch.zeros(3 * len(m.fixed_nodes) + (len(bvec) if with_c else 0), dtype=torch.float64,
                          device="cuda")
        vals = torch.empty(g.nnz, dtype=torch.float32, device="cuda")
        f = torch.empty(3 * m.nn, dtype=torch.float64, device="cuda")
        res = torch.empty_like(f)
        gn = torch.empty(1, dtype=torch.float64, device="cuda")
        prm = tl.params(h=h, rho_alm=rho)

        def one():
            g.assemble_hessian(q, v, h, rho, values=vals, f_int=f)
            g.eval_residual(prm, q, v, v, lam=lam, f_int=f, g=res, g_norm=gn)

        for _ in range(3):
            one()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(20):
            one()
        e1.record()
        torch.cuda.synchronize()
        out[tag] = {"ms": e0.elapsed_time(e1) / 20, "nnz": int(g.nnz)}
        g.close()
    out["overhead"] = out["with"]["ms"] / out["without"]["ms"] - 1.0
    return out


# Algorithmic float64 flops per element of the ANCF passes (SVK), counted from
# the formulas the kernels evaluate (FMA = 2), n shape functions, per point:
# shape derivatives 10n, J0 18n, its inverse 41, grad S 18n, u 6n, H 18n,
# F / E / J - 1 / S / B 141, S n_a and F n_a 30n, w J0 1 = 100n + 183
# (force pass: 85n + 147 without F n_a and B); force sum 21 per (a, point);
# tangent 77 per block pair (a <= b) and point: n_a.n_b 5, n_a.S n_b 5,
# weights 4, nine entries of c1 g_a g_b^T + c2 (g_b g_a^T + (n_a.n_b) B) 60,
# diagonal 3; mass on the diagonal 3 per pair.
ANCF_SHAPE = {"ancf3243": (8, 12), "ancf3443": (16, 48)}     # shape functions, points


def ancf_flops_per_elem(kind, tangent=True):
    n, nq = ANCF_SHAPE[kind]
    npair = n * (n + 1) // 2
    force = 21 * n * nq
    if not tangent:
        return nq * (85 * n + 147) + force
    return nq * (100 * n + 183) + force + npair * nq * 77 + 3 * npair


FP64_FMA_PER_SM_CLK = 2


def fp64_alu_peak_tflops():
    """152 SMs x 2 float64 FMA per clock x 2 flop x 2.07 GHz (GB300's float64
    rate: its nominal 1.25 TFLOP/s over 152 SMs at 2.07 GHz)."""
    return SM_COUNT * FP64_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12


def run_ancf(args):
    """ANCF3243 beam and ANCF3443 shell at the largest resolutions of the
    paper's element-type scaling tables (500,000 beam elements of 0.2 x 0.1 x
    0.1 m; a 200 x 200 shell of 4 x 2 x 0.1 m), SVK 7e8 / 0.33 / 2700, bent and
    perturbed by 0.1%: the Hessian assembly pass (values zeroed, fused
    internal force + tangent + exact mass + clamp penalty) in float64 and in
    the float32 element form, and the float64 force pass,
    CUDA events over 10 passes after 3 warm-ups, the element kernel alone from
    the library's event timers, against the float64 ALU roofline.  Then one
    Newton steps from rest under the paper's tip loads (beam: F_z = 5,000 N at
    the free end; shell: -500 N spread over the free edge) at the RES0
    resolution, vendor direct solver and the captured PCG graph, inner stop
    max(1e-4, 1e-8 relative), the paper's eps_in at RES0.  The oracle's
    assembly rate on a bounded sample of each kind is reported beside the GPU
    numbers (`cpu_baseline`, skipped with --no-cpu-baseline)."""
    import torch

    from paper_2604_10357_gb300 import inputs, tl
    out = {"roofline_peak_tflops": fp64_alu_peak_tflops(), "peak_kind": "float64 ALU, derived"}
    mat = dict(inputs.SVK_7E8)
    for kind in ("ancf3243", "ancf3443"):
        rng = np.random.default_rng(1000 + 8)
        if kind == "ancf3243":
            m, h, curv = inputs.beam_ancf3243(max(8, int(round(500_000 * args.ancf_scale)))), 1e-3, 1e-5
        else:
            ns = max(2, int(round(200 * args.ancf_scale ** 0.5)))
            m, h, curv = inputs.shell_ancf3443(ns, ns), 5e-4, 0.25
        q = inputs.ancf_perturbation(m, inputs.ancf_bend(m, curv), 0.001, rng)
        v = rng.normal(0.0, 0.01, size=q.shape)
        v[m.fixed_nodes] = 0.0
        g = tl.Mesh.ancf(kind, m.E0, m.conn, m.dims, [mat])
        g.build_pattern(m.fixed_nodes)
        qd = torch.as_tensor(q.reshape(-1), device="cuda")
        vd = torch.as_tensor(v.reshape(-1), device="cuda")
        vals = torch.empty(g.nnz, dtype=torch.float64, device="cuda")
        f = torch.empty(3 * m.nn, dtype=torch.float64, device="cuda")
        res = {}
        for tag, fn in (("assembly", lambda: g.assemble_hessian(qd, vd, h, 1e12, values=vals, f_int=f)),
                        ("force", lambda: g.eval_force(qd, vd, h, out=f))):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            g.timing_read()
            g.timing_enable(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(10):
                fn()
            e1.record()
            torch.cuda.synchronize()
            tim = g.timing_read()
            g.timing_enable(False)
            ms = e0.elapsed_time(e1) / 10
            kms = tim["ms_element"] / max(1, tim["n_element"])
            fl = ancf_flops_per_elem(kind, tag == "assembly")
            res[tag] = {"ms": ms, "elems_per_s": m.ne / ms * 1e3, "kernel_ms": kms,
                        "flops_per_elem": fl, "achieved_tflops": fl * m.ne / (kms * 1e-3) / 1e12,
                        "frac": fl * m.ne / (kms * 1e-3) / 1e12 / fp64_alu_peak_tflops()}
        g.sync()
        res.update(elements=int(m.ne), coefficients=int(m.nn), dofs=int(3 * m.nn), nnz=int(g.nnz))
        g.close()
        # the float32 element form: the same assembly pass with float32 tangent and values
        g32 = tl.Mesh.ancf(kind, m.E0, m.conn, m.dims, [mat], precision=tl.TL_FP32_ELEM)
        g32.build_pattern(m.fixed_nodes)
        vals32 = torch.empty(g32.nnz, dtype=torch.float32, device="cuda")
        for _ in range(3):
            g32.assemble_hessian(qd, vd, h, 1e12, values=vals32, f_int=f)
        torch.cuda.synchronize()
        g32.timing_read()
        g32.timing_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            g32.assemble_hessian(qd, vd, h, 1e12, values=vals32, f_int=f)
        e1.record()
        torch.cuda.synchronize()
        tim = g32.timing_read()
        g32.timing_enable(False)
        g32.sync()
        ms = e0.elapsed_time(e1) / 10
        kms = tim["ms_element"] / max(1, tim["n_element"])
        fl = ancf_flops_per_elem(kind, True)
        res["assembly_fp32"] = {"ms": ms, "elems_per_s": m.ne / ms * 1e3, "kernel_ms": kms, "flops_per_elem": fl,
                                "achieved_tflops": fl * m.ne / (kms * 1e-3) / 1e12,
                                "frac_fp32_alu": fl * m.ne / (kms * 1e-3) / 1e12 / fp32_alu_peak_tflops(),
                                "speedup_vs_fp64": res["assembly"]["ms"] / ms}
        g32.close()
        if not args.no_cpu_baseline:
            rate, reps, n, el = oracle_ancf_rate(kind)
            res["cpu_baseline"] = {"kind": "oracle", "value": rate, "unit": "elems/s", "cores": 1,
                                   "sample": f"{n}-element {kind} of the same recipe, Hessian assembly + force, "
                                             f"{reps} passes in {el:.1f} s (numpy, one thread)"}
        if args.ancf_no_newton:
            out[kind] = res
            continue
        # Newton steps from rest under the tip load at the RES0 resolution of
        # the paper's tables, the vendor direct solver and the captured PCG graph
        if kind == "ancf3243":
            mn = inputs.beam_ancf3243(1_000)
            fe = np.zeros_like(mn.E0)
            fe[4 * (mn.nphys - 1), 2] = 5000.0
            res_name, paper_rtf = "RES0 (1,000 elements)", 4.85
        else:
            mn = inputs.shell_ancf3443(10, 10)
            fe = np.zeros_like(mn.E0)
            edge = np.nonzero(np.isclose(mn.phys_x[:, 0], mn.phys_x[:, 0].max()))[0]
            fe[4 * edge, 2] = -500.0 / len(edge)
            res_name, paper_rtf = "RES0 (10 x 10)", 8.11
        newton = {"resolution": res_name, "h_s": h, "paper_rtf_other_gpu": paper_rtf,
                  "tol": "max(1e-4, 1e-8 g_ref), eps_out 1e-4 (the paper's eps_in / eps_out at RES0)",
                  "note": "RTF = wall time / simulated time; the paper's stopping rule and GPU differ"}
        for arm, solver, graph in (("direct", tl.TL_SOLVER_DIRECT, 0), ("pcg_graph", tl.TL_SOLVER_PCG, 1)):
            gn = tl.Mesh.ancf(kind, mn.E0, mn.conn, mn.dims, [mat])
            gn.build_pattern(mn.fixed_nodes)
            p = tl.params(h=h, rtol=1e-8, atol=1e-4, eps_out=1e-4, linear_solver=solver, use_graph=graph)
            qn = torch.as_tensor(mn.E0.reshape(-1), device="cuda")
            vn = torch.zeros_like(qn)
            fx = torch.as_tensor(fe.reshape(-1), device="cuda")
            lam = torch.zeros(3 * len(mn.fixed_nodes), dtype=torch.float64, device="cuda")
            steps, t_ms, iters, status = 10, [], [], []
            for k in range(steps + 2):           # the first two steps include the solver / graph set-up
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                vv, qq, st = gn.newton_step(p, qn, vn, lam, f_ext=fx, raise_on_nonconvergence=False)
                torch.cuda.synchronize()
                if k >= 2:
                    t_ms.append((time.perf_counter() - t0) * 1e3)
                    iters.append(int(st["inner_iters"]))
                    status.append(int(st["status"]))
                qn, vn = qq.clone(), vv.clone()
            gn.close()
            newton[arm] = {"steps": steps, "ms_per_step": statistics.median(t_ms), "inner_iters": iters,
                           "status": status, "rtf": statistics.median(t_ms) / (h * 1e3)}
        res["newton"] = newton
        out[kind] = res
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--scale", type=float, default=1.0, help="hex-count scale of the box (1.0 = 960k T10)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-newton", action="store_true")
    ap.add_argument("--newton-steps", type=int, default=50)
    ap.add_argument("--newton-direct", action="store_true")
    ap.add_argument("--newton-start", type=int, default=1101,
                    help="first evaluated step of the cantilever trajectory (1101: the held-out window)")
    ap.add_argument("--newton-only", action="store_true", help="run only the Newton comparison and print it")
    ap.add_argument("--newton-no-graph", action="store_true",
                    help="chosen arm from the host loop (same kernels; for launch lists, which do not see "
                         "kernels inside conditional graph nodes)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-constraints", action="store_true", help="skip the general-constraint cost measurement")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64, mid-size, batched and direct-solver measurements")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--shape", action="append", default=[],
                    help="fix a launch shape of the element workload after the autotuner (key=value, repeatable)")
    ap.add_argument("--no-ancf", action="store_true", help="skip the ANCF beam / shell measurement")
    ap.add_argument("--ancf-only", action="store_true", help="run only the ANCF measurement and print it")
    ap.add_argument("--ancf-scale", type=float, default=1.0,
                    help="element-count scale of the ANCF meshes (1.0 = 500,000 beam and 200 x 200 shell elements)")
    ap.add_argument("--ancf-no-newton", action="store_true", help="skip the ANCF Newton steps")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if args.newton_only:
        if rank == 0:
            summary, details = run_newton(args)
            print("# newton_details: " + json.dumps(details), flush=True)
            print(json.dumps({"newton": summary}), flush=True)
        return
    if args.ancf_only:
        if rank == 0:
            print(json.dumps(run_ancf(args)), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group("nccl")
    line = run_ours(args, rank, world)
    if line is not None:
        if world == 1:
            # details go to lines of their own (prefixed "# "), before the JSON line
            def extra(name, fn, *a):
                try:
                    return fn(*a)
                except Exception as exc:                  # a failed extra must not lose the main line
                    return {"error": f"{type(exc).__name__}: {exc}"}
            if not args.no_extras:
                line["fp64"] = extra("fp64", run_fp64_large, args)
                line["mid_mr_kv"] = extra("mid", run_mid, args)
                line["batched"] = extra("batched", run_batched, args)
                line["direct_solver"] = extra("direct", run_direct, args)
            if not args.no_constraints:
                line["constraints"] = extra("constraints", run_constraints, args)
            if not args.no_ancf:
                anc = extra("ancf", run_ancf, args)
                print("# ancf: " + json.dumps(anc), flush=True)
                line["ancf"] = {k: {"assembly_frac_fp64_alu": v["assembly"]["frac"],
                                    "assembly_fp32_frac_fp32_alu": v["assembly_fp32"]["frac_fp32_alu"],
                                    "assembly_ms": v["assembly"]["ms"], "assembly_fp32_ms": v["assembly_fp32"]["ms"]}
                                for k, v in anc.items() if isinstance(v, dict) and "assembly" in v} \
                    if "error" not in anc else anc
            if not args.no_cpu_baseline:
                rate, reps, n, el = oracle_step_rate()
                cb = {"kind": "oracle", "value": rate, "unit": UNIT, "cores": 1, "cpu": cpu_model(),
                      "host_cores": os.cpu_count(),
                      "sample": f"{n}-element sub-box (10x4x4 hexes) of the same workload, "
                                f"{reps} passes in {el:.1f} s (numpy, one thread)"}
                try:
                    rate_all, ncores, _ = oracle_all_cores_rate()
                    cb["all_cores"] = {"value": rate_all, "cores": ncores,
                                       "sample": "one copy of the same sub-box per process, one process per core"}
                except Exception as exc:
                    cb["all_cores"] = {"error": f"{type(exc).__name__}: {exc}"}
                line["cpu_baseline"] = cb
            if not args.no_newton:
                nw = extra("newton", run_newton, args)
                if isinstance(nw, tuple):
                    print("# newton_details: " + json.dumps(nw[1]), flush=True)
                    line["newton"] = nw[0]
                else:
                    line["newton"] = nw
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
