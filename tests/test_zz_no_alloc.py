"""GPU tests of tl_eval_residual_noalloc, the residual entry point for
callers that cannot allocate device memory while they step (their memory is
owned by a pool or a fixed budget, or a device-synchronising cudaMalloc is not
acceptable in their loop).  It must give the same g and ||g|| as
tl_eval_residual, on consecutive calls (its scratch array is shared and keeps
the previous call's contents), and refuse meshes beyond its stated limit.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

from paper_2604_10357_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-11


def _tl():
    from paper_2604_10357_gb300 import build, tl
    build.build()
    return tl


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(-1), device="cuda")


@pytest.mark.parametrize("workload", ["small_svk", "mid_mr_kv"])
def test_noalloc_residual_matches_existing_entry_point(workload):
    tl = _tl()
    w = inputs.workload_small_svk() if workload == "small_svk" else inputs.workload_mid_mr_kv()
    m = w["mesh"]
    g = tl.Mesh(m.X, m.conn, [w["material"]], precision=tl.TL_FP64)
    g.build_pattern(m.fixed_nodes)
    rng = np.random.default_rng(11)
    v_n = w["v"] + 0.01 * rng.normal(size=w["v"].shape)
    v_n[m.fixed_nodes] = 0.0
    q, v, vn = _dev(w["q_n"]), _dev(w["v"]), _dev(v_n)
    f_ext = _dev(rng.normal(size=3 * m.nn))
    lam = _dev(rng.normal(size=3 * len(m.fixed_nodes)))
    prm = tl.params(h=w["h"], rho_alm=1e6)
    f = g.eval_force(q, v, w["h"])
    g_ref, n_ref = g.eval_residual(prm, q, vn, v, f_ext=f_ext, lam=lam, f_int=f)
    g.sync()
    g_ref, n_ref = g_ref.cpu().numpy(), n_ref.item()
    out = torch.empty(3 * m.nn, dtype=torch.float64, device="cuda")
    nrm = torch.empty(1, dtype=torch.float64, device="cuda")
    for _call in range(2):
        out.fill_(np.nan)
        nrm.fill_(np.nan)
        g.eval_residual_noalloc(prm, q, vn, v, f, out, nrm, f_ext=f_ext, lam=lam)
        g.sync()
        got = out.cpu().numpy()
        assert np.abs(got - g_ref).max() <= TOL * np.abs(g_ref).max()
        assert abs(nrm.item() - n_ref) <= TOL * n_ref


def test_noalloc_rejects_meshes_beyond_its_limit():
    """4,194,305 nodes (one hexahedron's 6 elements plus unconnected nodes):
    one node past the limit of 16,384 blocks of 256 nodes."""
    tl = _tl()
    box = inputs.box_t10(1, 1, 1, 0.1, 0.1, 0.1, fixed_face_x0=False)
    n_total = 16384 * 256 + 1
    X = np.zeros((n_total, 3))
    X[: box.nn] = box.X
    X[box.nn:, 0] = 10.0 + np.arange(n_total - box.nn) * 1e-3
    g = tl.Mesh(X, box.conn, [dict(inputs.SVK_1E7)], precision=tl.TL_FP64)
    g.build_pattern(())
    zeros = torch.zeros(3 * n_total, dtype=torch.float64, device="cuda")
    out = torch.empty_like(zeros)
    nrm = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(tl.TLError) as ei:
        g.eval_residual_noalloc(tl.params(), zeros, zeros, zeros, zeros, out, nrm)
    assert ei.value.status == 10
    assert "4,194,304" in str(ei.value)
