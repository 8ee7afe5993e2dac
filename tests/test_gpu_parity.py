"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle:
bit-exact pattern and slot map; force, element tangents, CSR Hessian values
and residual within 1e-11 (FP64 element path) or 1e-5 (FP32 element form)."""
import numpy as np
import pytest

from oracle import assembly as asm
from paper_2604_10357_gb300 import inputs

from helpers import TOL_FP32, TOL_FP64, force_error, tangent_error, values_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _tl():
    from paper_2604_10357_gb300 import build, tl
    build.build()
    return tl


def ragged_mixed():
    """Three bodies (ragged element counts, two materials incl. KV) in one mesh."""
    rng = np.random.default_rng(77)
    bodies = [inputs.box_t10(3, 2, 1, 0.3, 0.2, 0.1), inputs.box_t10(2, 2, 2, 0.2, 0.2, 0.2),
              inputs.cylinder_t10(1, 3, 0.1, 0.3)]
    mesh = inputs.merge_meshes(bodies)
    q = inputs.uniform_perturbation(mesh, 0.02, rng)
    v = inputs.gaussian_velocity(mesh, 0.05, rng)
    mats = [dict(inputs.SVK_1E7, eta_d=0.0, lambda_d=0.0),
            dict(inputs.MR_C2, eta_d=1e3, lambda_d=2e3),
            dict(inputs.SVK_1E7, eta_d=5e2, lambda_d=1e3)]
    return dict(name="mixed", mesh=mesh, q_n=q, v=v, materials=mats,
                mat_of_elem=mesh.body_of_elem, h=1e-3)


def shuffled_order():
    """Elements in random order: the 32 elements of a tile share few nodes,
    so their CSR runs land in unrelated rows at every alignment of the
    vector reductions."""
    w = inputs.workload_small_svk()
    rng = np.random.default_rng(99)
    m = w["mesh"]
    perm = rng.permutation(m.ne)
    m2 = inputs.Mesh(X=m.X, conn=m.conn[perm].copy(), fixed_nodes=m.fixed_nodes, extent=m.extent,
                     hex_size=m.hex_size)
    return dict(w, name="shuffled", mesh=m2)


WORKLOADS = {
    "small_svk": inputs.workload_small_svk,
    "mid_mr_kv": inputs.workload_mid_mr_kv,
    "ragged_mixed": ragged_mixed,
    "shuffled": shuffled_order,
}


@pytest.fixture(scope="module", params=list(WORKLOADS))
def case(request):
    w = WORKLOADS[request.param]()
    m = w["mesh"]
    mats = w.get("materials", [w.get("material")])
    om = asm.OracleMesh(m.X, m.conn, mats, w.get("mat_of_elem"), fixed_nodes=m.fixed_nodes)
    return request.param, w, om


def _gpu_mesh(tl, w, precision):
    m = w["mesh"]
    mats = w.get("materials", [w.get("material")])
    g = tl.Mesh(m.X, m.conn, mats, w.get("mat_of_elem"), precision=precision)
    g.build_pattern(m.fixed_nodes)
    return g


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(-1), device="cuda")


def test_pattern_and_slot_map_bit_exact(case):
    tl = _tl()
    name, w, om = case
    g = _gpu_mesh(tl, w, tl.TL_FP64)
    node_ptr, node_col, row_ptr, col = om.pattern()
    rp, cl, sm = g.get_pattern(with_slot_map=True)
    assert g.nnz == len(col)
    assert np.array_equal(rp.cpu().numpy(), row_ptr.astype(np.int32))
    assert np.array_equal(cl.cpu().numpy(), col.astype(np.int32))
    assert np.array_equal(sm.cpu().numpy().reshape(-1, 900),
                          asm.slot_map(om.conn, row_ptr, col).astype(np.int32))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_force_parity(case, prec):
    tl = _tl()
    name, w, om = case
    g = _gpu_mesh(tl, w, tl.TL_FP64 if prec == "fp64" else tl.TL_FP32_ELEM)
    h = w["h"]
    f = g.eval_force(_dev(w["q_n"]), _dev(w["v"]), h).cpu().numpy()
    g.sync()
    x = w["q_n"] + h * w["v"]
    fe = om.element_forces(x, w["v"])
    f_ora = om.internal_force(w["q_n"], w["v"], h)
    err = force_error(f, f_ora, fe)
    assert err < (TOL_FP64 if prec == "fp64" else TOL_FP32), err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("ab", [(1.0, 0.0), (0.0, 1.0), (1e-3, 1.0)], ids=["K", "D", "hK+D"])
def test_element_tangent_parity(case, prec, ab):
    tl = _tl()
    name, w, om = case
    alpha, beta = ab
    if beta != 0.0 and not any(m.get("eta_d", 0) or m.get("lambda_d", 0)
                               for m in w.get("materials", [w.get("material")])):
        pytest.skip("no Kelvin-Voigt material in this workload")
    g = _gpu_mesh(tl, w, tl.TL_FP64 if prec == "fp64" else tl.TL_FP32_ELEM)
    h = w["h"]
    K = g.eval_tangent(_dev(w["q_n"]), _dev(w["v"]), h, alpha, beta).cpu().numpy()
    g.sync()
    x = w["q_n"] + h * w["v"]
    K_ora = om.element_tangents(x, w["v"], alpha, beta)
    err = tangent_error(K, K_ora)
    assert err < (TOL_FP64 if prec == "fp64" else TOL_FP32), err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_hessian_values_and_fused_force_parity(case, prec):
    tl = _tl()
    name, w, om = case
    g = _gpu_mesh(tl, w, tl.TL_FP64 if prec == "fp64" else tl.TL_FP32_ELEM)
    h, rho = w["h"], 1e12
    f = torch.empty(3 * w["mesh"].nn, dtype=torch.float64, device="cuda")
    vals = g.assemble_hessian(_dev(w["q_n"]), _dev(w["v"]), h, rho, f_int=f).cpu().numpy()
    g.sync()
    v_ora = om.hessian_values(w["q_n"], w["v"], h, rho)
    tol = TOL_FP64 if prec == "fp64" else TOL_FP32
    # the clamp-penalty diagonal entries (h^2 rho = 1e6 added) are compared
    # relative to their own magnitude (in float32 storage they carry a
    # rounding of ~6e-8 * 1e6); all other entries relative to max |value|
    fd = om.fixed_dofs
    _, _, row_ptr, col = om.pattern()
    pen = asm.csr_positions(row_ptr, col, fd, fd)
    v_gpu = vals.astype(np.float64)
    rest = np.ones(len(v_ora), bool)
    rest[pen] = False
    emax, e2 = values_error(v_gpu[rest], v_ora[rest])
    assert emax < tol and e2 < tol, (emax, e2)
    if len(pen):
        assert np.max(np.abs(v_gpu[pen] - v_ora[pen]) / np.abs(v_ora[pen])) < tol
    fe = om.element_forces(w["q_n"] + h * w["v"], w["v"])
    assert force_error(f.cpu().numpy(), om.internal_force(w["q_n"], w["v"], h), fe) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("split", [0, 1])
def test_residual_parity(case, prec, split):
    """The residual with its internal force evaluated here: float64
    throughout, or with the mass product and (float32 handles) the internal
    force in double-float arithmetic (48-bit significands); every combination
    within the float64 bar of the oracle (a float32 handle's residual force is
    float64-class too)."""
    tl = _tl()
    name, w, om = case
    g = _gpu_mesh(tl, w, tl.TL_FP64 if prec == "fp64" else tl.TL_FP32_ELEM)
    g.tune_set(residual_split=split, force_split=split)
    m = w["mesh"]
    rng = np.random.default_rng(5)
    v_n = w["v"] + 0.01 * rng.normal(size=w["v"].shape)
    v_n[m.fixed_nodes] = 0.0
    f_ext = rng.normal(size=3 * m.nn)
    lam = rng.normal(size=3 * len(m.fixed_nodes))
    prm = tl.params(h=w["h"], rho_alm=1e6)
    gg, gn = g.eval_residual(prm, _dev(w["q_n"]), _dev(v_n), _dev(w["v"]), _dev(f_ext), _dev(lam))
    g.sync()
    g_ora = om.residual(w["v"], w["q_n"], v_n, w["h"], f_ext, prm.gravity[:], lam, 1e6)
    fe = om.element_forces(w["q_n"] + w["h"] * w["v"], w["v"])
    assert force_error(gg.cpu().numpy(), g_ora, fe) < TOL_FP64
    assert abs(gn.item() - np.linalg.norm(g_ora)) < 1e-10 * np.linalg.norm(g_ora)


def test_inverted_element_is_reported():
    """An inverted current configuration is a valid input: the kernel flags
    det F <= 0 and tl_sync returns TL_ERR_INVERTED (no fault, no trap)."""
    tl = _tl()
    m = inputs.box_t10(2, 1, 1, 0.2, 0.1, 0.1)
    x = m.X.copy()
    x[:, 2] *= -1.0                       # mirror: every element inverted
    g = tl.Mesh(m.X, m.conn, [dict(inputs.SVK_1E7)], precision=tl.TL_FP64)
    g.build_pattern(m.fixed_nodes)
    g.eval_force(_dev(x), _dev(np.zeros_like(x)), 0.0)
    with pytest.raises(tl.TLError) as ei:
        g.sync()
    assert ei.value.status == 4
    g.sync()                               # the flag is cleared


def test_create_rejects_bad_input():
    tl = _tl()
    m = inputs.box_t10(1, 1, 1, 0.1, 0.1, 0.1)
    bad = m.conn.copy()
    bad[0, 0] = m.nn + 5
    with pytest.raises(tl.TLError):
        tl.Mesh(m.X, bad, [dict(inputs.SVK_1E7)])
    flipped = m.conn.copy()
    flipped[:, [1, 2]] = flipped[:, [2, 1]]
    with pytest.raises(tl.TLError):
        tl.Mesh(m.X, flipped, [dict(inputs.SVK_1E7)])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_residual_sliced_ell_matches_csr_rows(case, prec):
    """The default residual reads the mass rows in sliced ELL (slices of 32
    rows ordered by length within windows of 256, padded with zero mass);
    the four-lane form reads the same double-float rows in CSR order.  Both
    sum the same products of the same float32 pairs, in other orders, so g
    agrees to a few units of 2^-48 of its largest terms (1e-13), on meshes
    whose node count leaves a partial last window and whose rows differ in
    length (vertex and midside nodes, two bodies and a cylinder)."""
    tl = _tl()
    name, w, om = case
    m = w["mesh"]
    assert m.nn % 256 != 0
    g = _gpu_mesh(tl, w, tl.TL_FP64 if prec == "fp64" else tl.TL_FP32_ELEM)
    rng = np.random.default_rng(6)
    v_n = w["v"] + 0.01 * rng.normal(size=w["v"].shape)
    v_n[m.fixed_nodes] = 0.0
    f_int = _dev(rng.normal(size=3 * m.nn))
    lam = _dev(rng.normal(size=3 * len(m.fixed_nodes)))
    prm = tl.params(h=w["h"], rho_alm=1e6)
    out = {}
    for lanes in (1, 4):
        g.tune_set(residual_split=1, residual_lanes=lanes)
        gg, gn = g.eval_residual(prm, _dev(w["q_n"]), _dev(v_n), _dev(w["v"]), lam=lam, f_int=f_int)
        g.sync()
        out[lanes] = (gg.cpu().numpy(), gn.item())
    scale = np.abs(out[4][0]).max()
    assert np.abs(out[1][0] - out[4][0]).max() <= 1e-13 * scale
    assert abs(out[1][1] - out[4][1]) <= 1e-13 * out[4][1]
