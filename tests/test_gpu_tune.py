"""The launch-shape autotuner: it times every compiled variant on the mesh and
keeps the fastest, and every variant computes the same thing - the Hessian of
each element-pass variant matches the oracle, and the Newton step converges
to the same state with each PCG product shape."""
import numpy as np
import pytest

from oracle import assembly as asm
from paper_2604_10357_gb300 import inputs

from helpers import TOL_FP32, values_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _tl():
    from paper_2604_10357_gb300 import build, tl
    build.build()
    return tl


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(-1), device="cuda")


def test_autotune_reports_and_keeps_a_choice():
    tl = _tl()
    w = inputs.workload_mid_mr_kv()
    m = w["mesh"]
    g = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP32_ELEM)
    g.build_pattern(m.fixed_nodes)
    rep = g.autotune(_dev(w["q_n"]), _dev(w["v"]), w["h"], reps=3)
    assert rep["spmv_group"] in (4, 8, 16, 32) and rep["spmv_row"] in (0, 1)
    assert rep["elem_xchg"] in (0, 1) and rep["elem_full_grid"] in (0, 1)
    assert all(t > 0 for t in rep["ms_element"]) and all(t > 0 for t in rep["ms_spmv"]) and rep["ms_ws"] > 0
    assert rep["ms_occ2"] > 0
    assert rep["ms_agg"] > 0                                 # aggregation timed on the exchanged variants
    assert rep["ms_pair"] > 0                                # the closed-form pair kernel timed too
    best = min(min(rep["ms_element"]), rep["ms_ws"], rep["ms_occ2"], rep["ms_agg"], rep["ms_pair"])
    if rep["elem_pair"]:
        assert rep["ms_pair"] == best
    elif rep["elem_agg"]:
        assert rep["ms_agg"] == best
    elif rep["elem_ws"]:
        assert rep["ms_ws"] == best
    elif rep["elem_occ2"]:
        assert rep["ms_occ2"] == best
    else:
        k = 4 * (1 - rep["elem_prefetch"]) + 2 * (1 - rep["elem_xchg"]) + rep["elem_full_grid"]
        assert rep["ms_element"][k] == best
    # then the tile order of that variant
    if rep["ms_spread"] > 0:
        assert (rep["ms_spread"] < best) == bool(rep["elem_spread"])
    assert all(t > 0 for t in rep["ms_spmv_row"])          # the float32 iteration times the row form too
    spmv_best = min(rep["ms_spmv"] + rep["ms_spmv_row"])
    if rep["spmv_row"]:
        assert rep["ms_spmv_row"][(8, 16, 32).index(rep["spmv_group"])] == spmv_best
    else:
        assert rep["ms_spmv"][(4, 8, 16).index(rep["spmv_group"])] == spmv_best
    assert all(t > 0 for t in rep["ms_residual_split"])     # double-float residual, 1 and 4 lanes
    res_best = min(rep["ms_residual"] + rep["ms_residual_split"])
    times = rep["ms_residual_split"] if rep["residual_split"] else rep["ms_residual"]
    assert times[(1, 4).index(rep["residual_lanes"])] == res_best
    assert all(t > 0 for t in rep["ms_force"])                # float32 handle: both residual forces timed
    assert rep["force_split"] == 0                            # a precision trade: never chosen by the tuner
    cur = g.tune_get()
    keys = ("spmv_group", "elem_xchg", "elem_full_grid", "elem_prefetch", "elem_ws", "residual_lanes", "elem_occ2",
            "elem_spread", "spmv_row", "pcg_f32", "elem_agg", "residual_split", "force_split", "elem_pair",
            "elem_fold")
    assert all(cur[k] == rep[k] for k in keys)
    with pytest.raises(tl.TLError):
        g.tune_set(spmv_group=5)


@pytest.mark.parametrize("prefetch,xchg,full_grid,ws,occ2,spread,agg",
                         [(pf, x, f, 0, 0, 0, 0) for pf in (0, 1) for x in (0, 1) for f in (0, 1)]
                         + [(1, 1, 0, 1, 0, 0, 0), (0, 1, 0, 0, 1, 0, 0), (0, 1, 0, 0, 1, 1, 0), (1, 1, 0, 0, 0, 1, 0),
                            (1, 0, 0, 0, 0, 1, 0),
                            (0, 1, 0, 0, 1, 0, 1), (0, 1, 0, 0, 1, 1, 1), (1, 1, 0, 0, 0, 0, 1), (0, 1, 1, 0, 0, 0, 1),
                            (0, 1, 0, 0, 0, 0, 1)])
def test_every_element_variant_matches_oracle(xchg, full_grid, prefetch, ws, occ2, spread, agg):
    tl = _tl()
    w = inputs.workload_small_svk()
    m = w["mesh"]
    om = asm.OracleMesh(m.X, m.conn, [w["material"]], fixed_nodes=m.fixed_nodes)
    g = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP32_ELEM)
    g.build_pattern(m.fixed_nodes)
    g.tune_set(spmv_group=8, elem_xchg=xchg, elem_full_grid=full_grid, elem_prefetch=prefetch, elem_ws=ws,
               elem_occ2=occ2, elem_spread=spread, elem_agg=agg, elem_pair=0)   # the generic kernel's variants
    h, rho = w["h"], 1e12
    vals = g.assemble_hessian(_dev(w["q_n"]), _dev(w["v"]), h, rho).cpu().numpy().astype(np.float64)
    ref = om.hessian_values(w["q_n"], w["v"], h, rho)
    _, _, row_ptr, col = om.pattern()
    pen = asm.csr_positions(row_ptr, col, om.fixed_dofs, om.fixed_dofs)
    rest = np.ones(len(ref), bool)
    rest[pen] = False
    emax, e2 = values_error(vals[rest], ref[rest])
    assert emax < TOL_FP32 and e2 < TOL_FP32


@pytest.mark.parametrize("group", [4, 8, 16])
def test_every_spmv_shape_converges_to_the_same_state(group):
    tl = _tl()
    w = inputs.workload_small_svk()
    m = w["mesh"]
    g = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP64)
    g.build_pattern(m.fixed_nodes)
    p = tl.params(h=w["h"], rtol=1e-8, linear_solver=tl.TL_SOLVER_PCG)
    out = {}
    for gr in (8, group):
        g.tune_set(spmv_group=gr)
        lam = torch.zeros(3 * len(m.fixed_nodes), dtype=torch.float64, device="cuda")
        v, _, st = g.newton_step(p, _dev(w["q_n"]), _dev(w["v"]), lam)
        assert st["converged"] == 1
        out[gr] = v.cpu().numpy()
    assert np.linalg.norm(out[group] - out[8]) <= 1e-9 * np.linalg.norm(out[8])


@pytest.mark.parametrize("row,group", [(0, 4), (0, 16), (1, 8), (1, 16), (1, 32)])
def test_every_float32_spmv_shape_converges_to_the_same_state(row, group):
    """Float32 Hessian, float32 PCG iteration: each product shape (one
    neighbour per lane, or lanes along the contiguous rows) gives the same
    converged Newton step as the 8-lane neighbour form, to the residual's
    tolerance, with the same Newton count."""
    tl = _tl()
    w = inputs.workload_small_svk()
    m = w["mesh"]
    g = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP32_ELEM)
    g.build_pattern(m.fixed_nodes)
    p = tl.params(h=w["h"], rtol=1e-8, linear_solver=tl.TL_SOLVER_PCG)
    out = {}
    for key, (r, gr) in (("ref", (0, 8)), ("test", (row, group))):
        g.tune_set(spmv_group=gr, spmv_row=r)
        lam = torch.zeros(3 * len(m.fixed_nodes), dtype=torch.float64, device="cuda")
        v, _, st = g.newton_step(p, _dev(w["q_n"]), _dev(w["v"]), lam)
        assert st["converged"] == 1 and st["g_norm"] <= 1e-8 * st["g_ref"]
        out[key] = (v.cpu().numpy(), st)
    (v0, s0), (v1, s1) = out["ref"], out["test"]
    assert s1["inner_iters"] == s0["inner_iters"]
    assert np.linalg.norm(v1 - v0) <= 1e-7 * np.linalg.norm(v0)
