"""The closed-form pair kernel of the float32 element form (St. Venant-Kirchhoff
with and without Kelvin-Voigt) against the FP64 oracle: the fused internal
force and the CSR Hessian values through the per-tile maps, and the element
tangents alpha K_t + beta D written per element, in every launch shape the
library compiles for it (prefetch on / off, persistent grid or one CTA per
tile) and in both of its forms (folded: K = c1 Q + c2 Q^T formed once per
tile; unfolded), on meshes with a ragged last tile, shuffled element order,
and a multi-material mesh whose Mooney-Rivlin segments keep the generic
kernel."""
import numpy as np
import pytest

from oracle import assembly as asm
from paper_2604_10357_gb300 import inputs

from helpers import TOL_FP32, force_error, tangent_error, values_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _tl():
    from paper_2604_10357_gb300 import build, tl
    build.build()
    return tl


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(-1), device="cuda")


def svk_kv_ragged():
    """7 x 5 x 3 hexes x 6 = 630 elements (19 full tiles and a ragged one),
    SVK + Kelvin-Voigt with unequal damping constants, sine-mode field."""
    rng = np.random.default_rng(1234)
    m = inputs.box_t10(7, 5, 3, 0.7, 0.5, 0.3)
    q, _ = inputs.sine_mode_field(m, 0.03, rng)
    v = inputs.gaussian_velocity(m, 0.5, rng)
    return dict(name="svk_kv_ragged", mesh=m, q_n=q, v=v, material=dict(inputs.SVK_1E7, eta_d=1e3, lambda_d=3e3),
                h=1e-3)


def ragged_mixed():
    rng = np.random.default_rng(77)
    bodies = [inputs.box_t10(3, 2, 1, 0.3, 0.2, 0.1), inputs.box_t10(2, 2, 2, 0.2, 0.2, 0.2),
              inputs.cylinder_t10(1, 3, 0.1, 0.3)]
    mesh = inputs.merge_meshes(bodies)
    q = inputs.uniform_perturbation(mesh, 0.02, rng)
    v = inputs.gaussian_velocity(mesh, 0.05, rng)
    mats = [dict(inputs.SVK_1E7, eta_d=0.0, lambda_d=0.0),
            dict(inputs.MR_C2, eta_d=1e3, lambda_d=2e3),
            dict(inputs.SVK_1E7, eta_d=5e2, lambda_d=1e3)]
    return dict(name="mixed", mesh=mesh, q_n=q, v=v, materials=mats, mat_of_elem=mesh.body_of_elem, h=1e-3)


def shuffled_svk_kv():
    w = svk_kv_ragged()
    rng = np.random.default_rng(98)
    m = w["mesh"]
    perm = rng.permutation(m.ne)
    m2 = inputs.Mesh(X=m.X, conn=m.conn[perm].copy(), fixed_nodes=m.fixed_nodes, extent=m.extent,
                     hex_size=m.hex_size)
    return dict(w, name="shuffled", mesh=m2)


WORKLOADS = {"small_svk": inputs.workload_small_svk, "svk_kv_ragged": svk_kv_ragged,
             "ragged_mixed": ragged_mixed, "shuffled": shuffled_svk_kv}


@pytest.fixture(scope="module", params=list(WORKLOADS))
def case(request):
    w = WORKLOADS[request.param]()
    m = w["mesh"]
    mats = w.get("materials", [w.get("material")])
    om = asm.OracleMesh(m.X, m.conn, mats, w.get("mat_of_elem"), fixed_nodes=m.fixed_nodes)
    return request.param, w, om


def _mesh(tl, w, **shape):
    m = w["mesh"]
    g = tl.Mesh(m.X, m.conn, w.get("materials", [w.get("material")]), w.get("mat_of_elem"),
                precision=tl.TL_FP32_ELEM)
    g.build_pattern(m.fixed_nodes)
    g.tune_set(elem_pair=1, elem_agg=1, elem_xchg=1, **shape)
    assert g.tune_get()["elem_pair"] == 1
    return g


@pytest.mark.parametrize("fold", [1, 0])
@pytest.mark.parametrize("prefetch,full_grid", [(1, 0), (0, 0), (1, 1), (0, 1)])
def test_pair_kernel_hessian_and_force(case, prefetch, full_grid, fold):
    tl = _tl()
    name, w, om = case
    g = _mesh(tl, w, elem_prefetch=prefetch, elem_full_grid=full_grid, elem_fold=fold)
    h, rho = w["h"], 1e12
    f = torch.empty(3 * w["mesh"].nn, dtype=torch.float64, device="cuda")
    for rep in range(2):                                  # the second pass sees values from the first: zeroed
        vals = g.assemble_hessian(_dev(w["q_n"]), _dev(w["v"]), h, rho, f_int=f).cpu().numpy()
    g.sync()
    ref = om.hessian_values(w["q_n"], w["v"], h, rho)
    _, _, row_ptr, col = om.pattern()
    pen = asm.csr_positions(row_ptr, col, om.fixed_dofs, om.fixed_dofs)
    rest = np.ones(len(ref), bool)
    rest[pen] = False
    emax, e2 = values_error(vals[rest].astype(np.float64), ref[rest])
    assert emax < TOL_FP32 and e2 < TOL_FP32, (emax, e2)
    if len(pen):
        assert np.max(np.abs(vals[pen] - ref[pen]) / np.abs(ref[pen])) < TOL_FP32
    fe = om.element_forces(w["q_n"] + h * w["v"], w["v"])
    assert force_error(f.cpu().numpy(), om.internal_force(w["q_n"], w["v"], h), fe) < TOL_FP32


@pytest.mark.parametrize("fold", [1, 0])
@pytest.mark.parametrize("ab", [(1.0, 0.0), (0.0, 1.0), (1e-3, 1.0)], ids=["K", "D", "hK+D"])
def test_pair_kernel_element_tangents(case, ab, fold):
    tl = _tl()
    name, w, om = case
    alpha, beta = ab
    if beta != 0.0 and not any(m.get("eta_d", 0) or m.get("lambda_d", 0)
                               for m in w.get("materials", [w.get("material")])):
        pytest.skip("no Kelvin-Voigt material in this workload")
    g = _mesh(tl, w, elem_fold=fold)
    h = w["h"]
    K = g.eval_tangent(_dev(w["q_n"]), _dev(w["v"]), h, alpha, beta).cpu().numpy()
    g.sync()
    K_ora = om.element_tangents(w["q_n"] + h * w["v"], w["v"], alpha, beta)
    assert tangent_error(K, K_ora) < TOL_FP32
    # symmetric to its float32 rounding (hyperelastic part and the damping tangent alike)
    Kr = K.reshape(-1, 30, 30).astype(np.float64)
    assert np.abs(Kr - Kr.transpose(0, 2, 1)).max() <= 1e-6 * np.abs(Kr).max()


def test_pair_kernel_matches_generic_kernel():
    """Both float32 kernels on the same state: the same CSR values to float32
    rounding (they sum the same terms in another order)."""
    tl = _tl()
    w = svk_kv_ragged()
    h, rho = w["h"], 1e12
    out = []
    for pair in (0, 1):
        g = _mesh(tl, w)
        g.tune_set(elem_pair=pair)
        out.append(g.assemble_hessian(_dev(w["q_n"]), _dev(w["v"]), h, rho).cpu().numpy().astype(np.float64))
        g.close()
    emax, e2 = values_error(out[1], out[0])
    assert emax < 2e-6 and e2 < 2e-6, (emax, e2)


def _svk_kv_tangents(tl, w, alpha, beta, fold):
    g = _mesh(tl, w, elem_fold=fold)
    K = g.eval_tangent(_dev(w["q_n"]), _dev(w["v"]), w["h"], alpha, beta).cpu().numpy()
    g.sync()
    g.close()
    return K


def test_pair_kernel_fold_taken_and_declined():
    """With alpha = 1, beta = 1e-3 (c1 + c2 well away from zero) the folded
    form runs: its tangents differ from the unfolded ones at float32 rounding
    and both match the oracle.  With beta chosen so that c1 + c2 nearly
    cancels (c1 = -1.4e6, c2 = 1.4e6, c1 + c2 = 2e4: below a quarter of
    max(|c1|, |c2|)) the library declines the fold: both settings give the
    same bits, and they match the oracle."""
    tl = _tl()
    w = svk_kv_ragged()
    mat = w["material"]
    E, nu = mat["E"], mat["nu"]
    lam, mu = E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))
    om = asm.OracleMesh(w["mesh"].X, w["mesh"].conn, [mat], fixed_nodes=w["mesh"].fixed_nodes)
    x = w["q_n"] + w["h"] * w["v"]
    # well conditioned: the fold is taken
    K1, K0 = (_svk_kv_tangents(tl, w, 1.0, 1e-3, f) for f in (1, 0))
    assert not np.array_equal(K1, K0)
    K_ora = om.element_tangents(x, w["v"], 1.0, 1e-3)
    assert tangent_error(K1, K_ora) < TOL_FP32 and tangent_error(K0, K_ora) < TOL_FP32
    # c1 + c2 = (lam + mu) + beta (lambda_d + eta) close to zero against c1 and c2
    beta = -(lam + mu - 2e4) / (mat["lambda_d"] + mat["eta_d"])
    c1, c2 = lam + beta * mat["lambda_d"], mu + beta * mat["eta_d"]
    assert abs(c1 + c2) < 0.25 * max(abs(c1), abs(c2))
    K1, K0 = (_svk_kv_tangents(tl, w, 1.0, beta, f) for f in (1, 0))
    assert np.array_equal(K1, K0)
    assert tangent_error(K1, om.element_tangents(x, w["v"], 1.0, beta)) < TOL_FP32
