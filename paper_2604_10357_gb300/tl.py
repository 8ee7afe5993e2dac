"""Python binding of the C ABI in include/tl.h (argument marshalling only).

Every compute step runs in the CUDA kernels of libtl_gb300.so; this module
only converts torch tensors / numpy arrays into pointers and sizes.  There is
no CPU fallback: if the shared library is missing or no GPU is present, the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtl_gb300.so")

TL_FP64, TL_FP32_ELEM = 0, 1
TL_ELEM_T10, TL_ELEM_ANCF3243, TL_ELEM_ANCF3443 = 0, 1, 2
TL_SVK, TL_MOONEY_RIVLIN = 0, 1

STATUS = {0: "TL_OK", 1: "TL_ERR_INVALID_ARG", 2: "TL_ERR_OOM", 3: "TL_ERR_CUDA", 4: "TL_ERR_INVERTED",
          5: "TL_ERR_NONFINITE", 6: "TL_ERR_NOT_CONVERGED", 7: "TL_ERR_SOLVER", 8: "TL_ERR_TIMEOUT",
          9: "TL_ERR_OVERFLOW", 10: "TL_ERR_UNSUPPORTED", 11: "TL_ERR_STATE"}


class TLError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class tl_material(C.Structure):
    _fields_ = [("kind", C.c_int32), ("_pad", C.c_int32), ("E", C.c_double), ("nu", C.c_double),
                ("rho0", C.c_double), ("C10", C.c_double), ("C01", C.c_double), ("kappa", C.c_double),
                ("eta_d", C.c_double), ("lambda_d", C.c_double)]


TL_SOLVER_DIRECT, TL_SOLVER_PCG = 0, 1


class tl_params(C.Structure):
    _fields_ = [("h", C.c_double), ("rho_alm", C.c_double), ("rtol", C.c_double), ("atol", C.c_double),
                ("eps_out", C.c_double), ("gravity", C.c_double * 3), ("max_inner", C.c_int32),
                ("max_outer", C.c_int32), ("linear_solver", C.c_int32), ("lin_max_iter", C.c_int32),
                ("lin_rtol", C.c_double), ("lin_adaptive", C.c_int32), ("use_graph", C.c_int32),
                ("line_search", C.c_int32), ("ls_max_trials", C.c_int32), ("ls_c1", C.c_double),
                ("ls_beta", C.c_double)]


class tl_newton_stats(C.Structure):
    _fields_ = [("inner_iters", C.c_int32), ("outer_iters", C.c_int32), ("converged", C.c_int32),
                ("_pad", C.c_int32), ("g_ref", C.c_double), ("g_norm", C.c_double), ("c_norm", C.c_double),
                ("ms_total", C.c_double), ("ms_assembly", C.c_double), ("ms_solver", C.c_double),
                ("lin_iters", C.c_int32), ("ls_trials", C.c_int32), ("g_init", C.c_double)]


class tl_adamw_params(C.Structure):
    _fields_ = [("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
                ("weight_decay", C.c_double), ("eps_in", C.c_double), ("eps_rel", C.c_double),
                ("max_inner", C.c_int32), ("check_every", C.c_int32)]


class tl_adamw_stats(C.Structure):
    _fields_ = [("inner_iters", C.c_int32), ("outer_iters", C.c_int32), ("converged", C.c_int32),
                ("_pad", C.c_int32), ("g_norm", C.c_double), ("c_norm", C.c_double), ("ms_total", C.c_double)]


class tl_timing(C.Structure):
    _fields_ = [("ms_element", C.c_double), ("ms_residual", C.c_double), ("n_element", C.c_int64),
                ("n_residual", C.c_int64), ("launches", C.c_int64)]


class tl_mesh_info(C.Structure):
    _fields_ = [("nn", C.c_int64), ("ne", C.c_int64), ("ndof", C.c_int64), ("nnz", C.c_int64),
                ("nnz_node", C.c_int64), ("nfixed", C.c_int64), ("precision", C.c_int32),
                ("nmat", C.c_int32), ("ncon", C.c_int64), ("element_kind", C.c_int32), ("nen", C.c_int32)]


class tl_tune_result(C.Structure):
    _fields_ = [("spmv_group", C.c_int32), ("elem_xchg", C.c_int32), ("elem_full_grid", C.c_int32),
                ("elem_prefetch", C.c_int32), ("elem_ws", C.c_int32), ("residual_lanes", C.c_int32),
                ("elem_occ2", C.c_int32), ("elem_spread", C.c_int32),
                ("ms_element", C.c_float * 8), ("ms_ws", C.c_float), ("ms_spmv", C.c_float * 3),
                ("ms_residual", C.c_float * 2), ("ms_occ2", C.c_float), ("ms_spread", C.c_float),
                ("pcg_f32", C.c_int32), ("spmv_row", C.c_int32), ("ms_spmv_row", C.c_float * 3),
                ("elem_agg", C.c_int32), ("ms_agg", C.c_float), ("residual_split", C.c_int32),
                ("ms_residual_split", C.c_float * 2), ("force_split", C.c_int32), ("ms_force", C.c_float * 2),
                ("elem_pair", C.c_int32), ("ms_pair", C.c_float), ("elem_fold", C.c_int32)]


# every symbol declared in include/tl.h, with (restype, argtypes)
_P = C.c_void_p
SIGNATURES = {
    "tl_mesh_create": (C.c_int, [_P, C.c_int64, _P, C.c_int64, _P, C.c_int32, _P, C.c_int32, _P, _P]),
    "tl_mesh_create_ancf": (C.c_int, [C.c_int32, _P, C.c_int64, _P, C.c_int64, _P, _P, C.c_int32, _P, C.c_int32,
                                      _P, _P]),
    "tl_build_pattern": (C.c_int, [_P, _P, C.c_int64, _P]),
    "tl_get_pattern": (C.c_int, [_P, _P, _P, _P]),
    "tl_eval_force": (C.c_int, [_P, _P, _P, C.c_double, _P]),
    "tl_eval_tangent": (C.c_int, [_P, _P, _P, C.c_double, C.c_double, C.c_double, _P]),
    "tl_assemble_hessian": (C.c_int, [_P, _P, _P, C.c_double, C.c_double, _P, _P]),
    "tl_eval_residual": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "tl_eval_residual_noalloc": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "tl_timing_enable": (C.c_int, [_P, C.c_int32]),
    "tl_timing_read": (C.c_int, [_P, _P]),
    "tl_newton_step": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "tl_adamw_step": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "tl_set_constraints": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P]),
    "tl_mlp_forward": (C.c_int, [_P, _P, C.c_int64, _P, _P, _P]),
    "tl_mlp_backward": (C.c_int, [_P, _P, _P, _P, C.c_int64, _P, _P]),
    "tl_mlp_mse_grad": (C.c_int, [_P, _P, _P, C.c_int64, _P, _P, _P]),
    "tl_mlp_adam": (C.c_int, [_P, _P, _P, _P, _P, C.c_int64, C.c_float, C.c_float, C.c_float, C.c_float,
                              C.c_int32, _P]),
    "tl_mlp_features": (C.c_int, [_P, _P, _P, _P, _P, C.c_double, C.c_double, C.c_double, _P]),
    "tl_warm_start": (C.c_int, [_P, _P, _P, _P, _P, _P, C.c_double, C.c_double, C.c_double, C.c_double, _P, _P]),
    "tl_mlp_target": (C.c_int, [_P, _P, _P, _P, _P, _P, C.c_double, C.c_double, C.c_double, C.c_double, _P]),
    "tl_mlp_col_sumsq": (C.c_int, [_P, C.c_int64, C.c_int32, _P, _P]),
    "tl_autotune": (C.c_int, [_P, _P, _P, C.c_double, C.c_int32, _P]),
    "tl_tune_get": (C.c_int, [_P, _P]),
    "tl_tune_set": (C.c_int, [_P, _P]),
    "tl_sync": (C.c_int, [_P]),
    "tl_mesh_info_get": (C.c_int, [_P, _P]),
    "tl_status_string": (C.c_char_p, [C.c_int]),
    "tl_last_error": (C.c_char_p, [_P]),
    "tl_mesh_destroy": (None, [_P]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libtl_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it first (paper_2604_10357_gb300.build.build())")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(t):
    """Device pointer of a CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def material(kind="svk", E=0.0, nu=0.0, rho0=1000.0, C10=0.0, C01=0.0, kappa=0.0, eta_d=0.0,
             lambda_d=0.0, **_):
    k = TL_SVK if kind in ("svk", TL_SVK) else TL_MOONEY_RIVLIN
    return tl_material(k, 0, E, nu, rho0, C10, C01, kappa, eta_d, lambda_d)


def params(h=1e-3, rho_alm=1e12, rtol=1e-8, atol=0.0, eps_out=1e-4, gravity=(0.0, 0.0, -9.81),
           max_inner=20, max_outer=5, linear_solver=TL_SOLVER_DIRECT, lin_max_iter=0, lin_rtol=0.0,
           lin_adaptive=0, use_graph=0, line_search=0, ls_max_trials=0, ls_c1=0.0, ls_beta=0.0):
    p = tl_params()
    p.h, p.rho_alm, p.rtol, p.atol, p.eps_out = h, rho_alm, rtol, atol, eps_out
    for i in range(3):
        p.gravity[i] = gravity[i]
    p.max_inner, p.max_outer = max_inner, max_outer
    p.linear_solver, p.lin_max_iter, p.lin_rtol = linear_solver, lin_max_iter, lin_rtol
    p.lin_adaptive = lin_adaptive
    p.use_graph = use_graph
    p.line_search, p.ls_max_trials, p.ls_c1, p.ls_beta = line_search, ls_max_trials, ls_c1, ls_beta
    return p


def adamw_params(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, eps_in=1e-4, eps_rel=1e-6,
                 max_inner=1000, check_every=10):
    a = tl_adamw_params()
    a.lr, a.beta1, a.beta2, a.eps, a.weight_decay = lr, beta1, beta2, eps, weight_decay
    a.eps_in, a.eps_rel, a.max_inner, a.check_every = eps_in, eps_rel, max_inner, check_every
    return a


MLP_NPARAM = 9219


def _tune_dict(r):
    return dict(spmv_group=r.spmv_group, elem_xchg=r.elem_xchg, elem_full_grid=r.elem_full_grid,
                elem_prefetch=r.elem_prefetch, elem_ws=r.elem_ws, residual_lanes=r.residual_lanes,
                elem_occ2=r.elem_occ2, elem_spread=r.elem_spread, ms_element=list(r.ms_element),
                ms_ws=r.ms_ws, ms_spmv=list(r.ms_spmv), ms_residual=list(r.ms_residual), ms_occ2=r.ms_occ2,
                ms_spread=r.ms_spread, pcg_f32=r.pcg_f32,
                spmv_row=r.spmv_row, ms_spmv_row=list(r.ms_spmv_row), elem_agg=r.elem_agg, ms_agg=r.ms_agg,
                residual_split=r.residual_split, ms_residual_split=list(r.ms_residual_split),
                force_split=r.force_split, ms_force=list(r.ms_force), elem_pair=r.elem_pair, ms_pair=r.ms_pair,
                elem_fold=r.elem_fold)


def _stream_ptr():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _chk(st, what):
    if st != 0:
        raise TLError(st, what)


def mlp_forward(params_bf16, feats, out=None, acts=None):
    """params_bf16: int16 CUDA tensor (bf16 bits, 9219); feats (n, 10) float32."""
    import torch
    lib = load_library()
    n = feats.shape[0]
    out = torch.empty(n, 3, dtype=torch.float32, device="cuda") if out is None else out
    _chk(lib.tl_mlp_forward(_ptr(params_bf16), _ptr(feats), n, _ptr(out), _ptr(acts), _stream_ptr()),
         "tl_mlp_forward")
    return out


def mlp_backward(params_bf16, feats, acts, dout, grads):
    lib = load_library()
    _chk(lib.tl_mlp_backward(_ptr(params_bf16), _ptr(feats), _ptr(acts), _ptr(dout), feats.shape[0],
                             _ptr(grads), _stream_ptr()), "tl_mlp_backward")
    return grads


def mlp_mse_grad(out, target, weight, dout, loss):
    lib = load_library()
    _chk(lib.tl_mlp_mse_grad(_ptr(out), _ptr(target), _ptr(weight), out.shape[0], _ptr(dout), _ptr(loss),
                             _stream_ptr()), "tl_mlp_mse_grad")


def mlp_col_sumsq(x, out):
    """out[c] += sum_i x[i, c]^2 (float64) for a float32 CUDA tensor x of shape (n, ncol)."""
    lib = load_library()
    _chk(lib.tl_mlp_col_sumsq(_ptr(x), x.shape[0], x.shape[1], _ptr(out), _stream_ptr()), "tl_mlp_col_sumsq")
    return out


def mlp_adam(master, params_bf16, grads, m1, m2, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
    lib = load_library()
    _chk(lib.tl_mlp_adam(_ptr(master), _ptr(params_bf16), _ptr(grads), _ptr(m1), _ptr(m2), master.numel(),
                         float(lr), float(beta1), float(beta2), float(eps), int(step), _stream_ptr()),
         "tl_mlp_adam")


class Mesh:
    """A tl_mesh handle.  Device arrays are torch CUDA tensors (float64 nodal
    vectors of length 3 nn, node-major)."""

    def __init__(self, X, conn, materials, mat_of_elem=None, precision=TL_FP64, stream=None):
        import torch
        self._torch = torch
        lib = load_library()
        self.lib = lib
        X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
        conn = np.ascontiguousarray(conn, dtype=np.int32).reshape(-1, 10)
        if isinstance(materials, dict):
            materials = [materials]
        mats = (tl_material * len(materials))(*[material(**m) for m in materials])
        moe = None if mat_of_elem is None else np.ascontiguousarray(mat_of_elem, dtype=np.int32)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        st = lib.tl_mesh_create(X.ctypes.data_as(_P), X.shape[0], conn.ctypes.data_as(_P), conn.shape[0],
                                C.cast(mats, _P), len(materials),
                                None if moe is None else moe.ctypes.data_as(_P), int(precision),
                                C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != 0:
            raise TLError(st, lib.tl_last_error(None).decode())
        self._finish(h, X.shape[0], conn.shape[0], 10, precision)

    @classmethod
    def ancf(cls, kind, E0, conn, dims, materials, mat_of_elem=None, precision=TL_FP64, stream=None):
        """tl_mesh_create_ancf: kind TL_ELEM_ANCF3243 / TL_ELEM_ANCF3443 (or
        "ancf3243" / "ancf3443"); E0 (ncoef, 3) reference coefficients, conn
        (ne, 8 | 16) coefficient ids, dims (ne, 3) element L, W, H.  Every
        "node" of the other calls is then a coefficient."""
        import torch
        if isinstance(kind, str):
            kind = {"ancf3243": TL_ELEM_ANCF3243, "ancf3443": TL_ELEM_ANCF3443}[kind]
        nen = 8 if kind == TL_ELEM_ANCF3243 else 16
        self = cls.__new__(cls)
        self._torch = torch
        lib = load_library()
        self.lib = lib
        E0 = np.ascontiguousarray(E0, dtype=np.float64).reshape(-1, 3)
        conn = np.ascontiguousarray(conn, dtype=np.int32).reshape(-1, nen)
        dims = np.ascontiguousarray(dims, dtype=np.float64).reshape(-1, 3)
        if isinstance(materials, dict):
            materials = [materials]
        mats = (tl_material * len(materials))(*[material(**m) for m in materials])
        moe = None if mat_of_elem is None else np.ascontiguousarray(mat_of_elem, dtype=np.int32)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        st = lib.tl_mesh_create_ancf(int(kind), E0.ctypes.data_as(_P), E0.shape[0], conn.ctypes.data_as(_P),
                                     conn.shape[0], dims.ctypes.data_as(_P), C.cast(mats, _P), len(materials),
                                     None if moe is None else moe.ctypes.data_as(_P), int(precision),
                                     C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != 0:
            raise TLError(st, lib.tl_last_error(None).decode())
        self._finish(h, E0.shape[0], conn.shape[0], nen, precision)
        return self

    def _finish(self, h, nn, ne, nen, precision):
        torch = self._torch
        self.h = h
        self.nn, self.ne, self.nen = nn, ne, nen
        self.ndof = 3 * self.nn
        self.precision = precision
        self.vdtype = torch.float32 if precision == TL_FP32_ELEM else torch.float64
        self.nnz = None
        self.nfixed = 0

    # -- helpers -----------------------------------------------------------
    def _check(self, st):
        if st != 0:
            raise TLError(st, self.lib.tl_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.tl_mesh_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- ABI calls -----------------------------------------------------------
    def set_constraints(self, row_ptr, col, val, b):
        """tl_set_constraints: general linear rows c = C q - b (C in CSR over
        DOFs, host arrays); before build_pattern."""
        rp = np.ascontiguousarray(np.asarray(row_ptr, dtype=np.int32).reshape(-1))
        cc = np.ascontiguousarray(np.asarray(col, dtype=np.int32).reshape(-1))
        vv = np.ascontiguousarray(np.asarray(val, dtype=np.float64).reshape(-1))
        bb = np.ascontiguousarray(np.asarray(b, dtype=np.float64).reshape(-1))
        self._check(self.lib.tl_set_constraints(self.h, len(bb), rp.ctypes.data_as(_P), cc.ctypes.data_as(_P),
                                                vv.ctypes.data_as(_P), bb.ctypes.data_as(_P)))
        self.ncon = len(bb)

    def build_pattern(self, fixed_nodes=()):
        fixed = np.ascontiguousarray(np.asarray(fixed_nodes, dtype=np.int32).reshape(-1))
        nnz = C.c_int64()
        self._check(self.lib.tl_build_pattern(self.h, fixed.ctypes.data_as(_P) if len(fixed) else None,
                                              len(fixed), C.byref(nnz)))
        self.nnz = nnz.value
        self.nfixed = len(fixed)
        return self.nnz

    def get_pattern(self, with_slot_map=False):
        torch = self._torch
        row_ptr = torch.empty(self.ndof + 1, dtype=torch.int32, device="cuda")
        col = torch.empty(self.nnz, dtype=torch.int32, device="cuda")
        slot = torch.empty(self.ne * (3 * self.nen) ** 2, dtype=torch.int32, device="cuda") if with_slot_map else None
        self._check(self.lib.tl_get_pattern(self.h, _ptr(row_ptr), _ptr(col), _ptr(slot)))
        return row_ptr, col, slot

    def eval_force(self, q_n, v, h, out=None):
        torch = self._torch
        out = torch.empty(self.ndof, dtype=torch.float64, device="cuda") if out is None else out
        self._check(self.lib.tl_eval_force(self.h, _ptr(q_n), _ptr(v), float(h), _ptr(out)))
        return out

    def eval_tangent(self, q_n, v, h, alpha=1.0, beta=0.0, out=None):
        torch = self._torch
        out = torch.empty(self.ne * (3 * self.nen) ** 2, dtype=self.vdtype, device="cuda") if out is None else out
        self._check(self.lib.tl_eval_tangent(self.h, _ptr(q_n), _ptr(v), float(h), float(alpha),
                                             float(beta), _ptr(out)))
        return out

    def assemble_hessian(self, q_n, v, h, rho_alm, values=None, f_int=None):
        torch = self._torch
        values = torch.empty(self.nnz, dtype=self.vdtype, device="cuda") if values is None else values
        self._check(self.lib.tl_assemble_hessian(self.h, _ptr(q_n), _ptr(v), float(h), float(rho_alm),
                                                 _ptr(values), _ptr(f_int)))
        return values

    def eval_residual(self, prm, q_n, v_n, v, f_ext=None, lam=None, g=None, g_norm=None, f_int=None):
        torch = self._torch
        g = torch.empty(self.ndof, dtype=torch.float64, device="cuda") if g is None else g
        g_norm = torch.empty(1, dtype=torch.float64, device="cuda") if g_norm is None else g_norm
        self._check(self.lib.tl_eval_residual(self.h, C.byref(prm), _ptr(q_n), _ptr(v_n), _ptr(v),
                                              _ptr(f_int), _ptr(f_ext), _ptr(lam), _ptr(g), _ptr(g_norm)))
        return g, g_norm

    def eval_residual_noalloc(self, prm, q_n, v_n, v, f_int, g, g_norm, f_ext=None, lam=None):
        """tl_eval_residual_noalloc: outputs g and g_norm must be given (no
        allocation anywhere on this path)."""
        self._check(self.lib.tl_eval_residual_noalloc(self.h, C.byref(prm), _ptr(q_n), _ptr(v_n), _ptr(v),
                                                      _ptr(f_int), _ptr(f_ext), _ptr(lam), _ptr(g),
                                                      _ptr(g_norm)))
        return g, g_norm

    def autotune(self, q_n, v, h, reps=5):
        """tl_autotune: time the launch-shape variants on this mesh, keep the fastest."""
        r = tl_tune_result()
        self._check(self.lib.tl_autotune(self.h, _ptr(q_n), _ptr(v), float(h), int(reps), C.byref(r)))
        return _tune_dict(r)

    def tune_get(self):
        r = tl_tune_result()
        self._check(self.lib.tl_tune_get(self.h, C.byref(r)))
        return _tune_dict(r)

    TUNE_KEYS = ("spmv_group", "spmv_row", "elem_xchg", "elem_full_grid", "elem_prefetch", "elem_ws",
                 "residual_lanes", "elem_occ2", "elem_spread", "pcg_f32", "elem_agg", "residual_split",
                 "force_split", "elem_pair", "elem_fold")

    def tune_set(self, **choice):
        """Set launch shapes by name (see tl_tune_result); the others keep
        their current values."""
        unknown = set(choice) - set(self.TUNE_KEYS)
        if unknown:
            raise TypeError(f"unknown launch-shape keys: {sorted(unknown)}")
        r = tl_tune_result()
        self._check(self.lib.tl_tune_get(self.h, C.byref(r)))
        for k, val in choice.items():
            setattr(r, k, int(val))
        self._check(self.lib.tl_tune_set(self.h, C.byref(r)))

    def timing_enable(self, on=True):
        self._check(self.lib.tl_timing_enable(self.h, 1 if on else 0))

    def timing_read(self):
        t = tl_timing()
        self._check(self.lib.tl_timing_read(self.h, C.byref(t)))
        return {f: getattr(t, f) for f, _ in tl_timing._fields_}

    def newton_step(self, prm, q_n, v_n, lam, v_init=None, f_ext=None, v_out=None, q_out=None,
                    raise_on_nonconvergence=True):
        """tl_newton_step; returns (v, q, stats dict).  lam is updated in place."""
        torch = self._torch
        v_out = torch.empty(self.ndof, dtype=torch.float64, device="cuda") if v_out is None else v_out
        q_out = torch.empty(self.ndof, dtype=torch.float64, device="cuda") if q_out is None else q_out
        st = tl_newton_stats()
        rc = self.lib.tl_newton_step(self.h, C.byref(prm), _ptr(q_n), _ptr(v_n), _ptr(v_init), _ptr(f_ext),
                                     _ptr(lam), _ptr(v_out), _ptr(q_out), C.byref(st))
        stats = {f: getattr(st, f) for f, _ in tl_newton_stats._fields_ if not f.startswith("_pad")}
        stats["status"] = rc
        if rc != 0 and (raise_on_nonconvergence or rc != 6):
            raise TLError(rc, self.lib.tl_last_error(self.h).decode())
        return v_out, q_out, stats

    def adamw_step(self, prm, aprm, q_n, v_n, lam, v_init=None, f_ext=None, v_out=None, q_out=None,
                   raise_on_nonconvergence=True):
        """tl_adamw_step; returns (v, q, stats dict).  lam is updated in place."""
        torch = self._torch
        v_out = torch.empty(self.ndof, dtype=torch.float64, device="cuda") if v_out is None else v_out
        q_out = torch.empty(self.ndof, dtype=torch.float64, device="cuda") if q_out is None else q_out
        st = tl_adamw_stats()
        rc = self.lib.tl_adamw_step(self.h, C.byref(prm), C.byref(aprm), _ptr(q_n), _ptr(v_n), _ptr(v_init),
                                    _ptr(f_ext), _ptr(lam), _ptr(v_out), _ptr(q_out), C.byref(st))
        stats = {f: getattr(st, f) for f, _ in tl_adamw_stats._fields_ if not f.startswith("_pad")}
        stats["status"] = rc
        if rc != 0 and (raise_on_nonconvergence or rc != 6):
            raise TLError(rc, self.lib.tl_last_error(self.h).decode())
        return v_out, q_out, stats

    def mlp_features(self, hist, scales, feats=None):
        """tl_mlp_features: hist = (v_n, v_{n-1}, v_{n-2}, v_{n-3}) (None for a missing
        velocity), scales = (s1, s2, s3)."""
        torch = self._torch
        feats = torch.empty(self.nn, 10, dtype=torch.float32, device="cuda") if feats is None else feats
        h = list(hist) + [None] * (4 - len(hist))
        self._check(self.lib.tl_mlp_features(self.h, _ptr(h[0]), _ptr(h[1]), _ptr(h[2]), _ptr(h[3]),
                                             float(scales[0]), float(scales[1]), float(scales[2]), _ptr(feats)))
        return feats

    def mlp_target(self, v_next, hist, scales, s_out, target=None):
        """tl_mlp_target: (v_next - extrapolation of hist) / (s_out r_I), float32 (nn, 3)."""
        torch = self._torch
        target = torch.empty(self.nn, 3, dtype=torch.float32, device="cuda") if target is None else target
        h = list(hist) + [None] * (4 - len(hist))
        self._check(self.lib.tl_mlp_target(self.h, _ptr(v_next), _ptr(h[0]), _ptr(h[1]), _ptr(h[2]), _ptr(h[3]),
                                           float(scales[0]), float(scales[1]), float(scales[2]), float(s_out),
                                           _ptr(target)))
        return target

    def warm_start(self, params_bf16, hist, scales=(1.0, 1.0, 1.0), s_out=0.0, work=None, v_init=None):
        """tl_warm_start: hist = (v_n, v_{n-1}, v_{n-2}, v_{n-3}) (None for a missing
        velocity); params None -> the extrapolation alone."""
        torch = self._torch
        if work is None and params_bf16 is not None:
            work = torch.empty(13 * self.nn, dtype=torch.float32, device="cuda")
        v_init = torch.empty(self.ndof, dtype=torch.float64, device="cuda") if v_init is None else v_init
        h = list(hist) + [None] * (4 - len(hist))
        self._check(self.lib.tl_warm_start(self.h, _ptr(params_bf16), _ptr(h[0]), _ptr(h[1]), _ptr(h[2]),
                                           _ptr(h[3]), float(scales[0]), float(scales[1]), float(scales[2]),
                                           float(s_out), _ptr(work), _ptr(v_init)))
        return v_init

    def sync(self):
        self._check(self.lib.tl_sync(self.h))

    def info(self):
        inf = tl_mesh_info()
        self._check(self.lib.tl_mesh_info_get(self.h, C.byref(inf)))
        return {f: getattr(inf, f) for f, _ in tl_mesh_info._fields_}
