"""Shared test helpers: comparison norms (the paper gives none; these are the
readings used throughout) and the oracle / GPU set-up of a workload."""
import numpy as np

# Tolerances: FP64 element path vs the FP64 oracle, and the FP32 element form.
TOL_FP64 = 1e-11
TOL_FP32 = 1e-5


def force_error(f_gpu, f_ora, fe_ora):
    """||f_gpu - f_ora||_inf / max_e ||f_e||_inf: element-level scale, so
    cancellation of element forces at a node cannot inflate the ratio."""
    scale = np.abs(fe_ora).max()
    return float(np.abs(np.asarray(f_gpu) - np.asarray(f_ora)).max() / scale)


def tangent_error(K_gpu, K_ora):
    """max_e ||K_e,gpu - K_e,ora||_F / ||K_e,ora||_F."""
    K_gpu = np.asarray(K_gpu, dtype=np.float64).reshape(-1, 900)
    K_ora = np.asarray(K_ora, dtype=np.float64).reshape(-1, 900)
    num = np.linalg.norm(K_gpu - K_ora, axis=1)
    den = np.linalg.norm(K_ora, axis=1)
    zero = den == 0.0          # e.g. the damping tangent of an undamped material
    if np.any(num[zero] != 0.0):
        return float("inf")
    if np.all(zero):
        return 0.0
    return float(np.max(num[~zero] / den[~zero]))


def values_error(v_gpu, v_ora):
    """Entry-wise error of CSR values relative to the largest |value| of the
    row-block's diagonal scale: max |dv| / max |v| and the 2-norm ratio."""
    v_gpu = np.asarray(v_gpu, dtype=np.float64)
    v_ora = np.asarray(v_ora, dtype=np.float64)
    return (float(np.abs(v_gpu - v_ora).max() / np.abs(v_ora).max()),
            float(np.linalg.norm(v_gpu - v_ora) / np.linalg.norm(v_ora)))


def material_list(w):
    return w["materials"] if "materials" in w else [w["material"]]


def first_frequencies(om, nn, nen, k=2):
    """Smallest natural frequencies of K phi = w^2 M phi (clamps eliminated),
    K the element tangents at the reference state, M the consistent mass."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    Ke = om.element_tangents(om.X, 0 * om.X, 1.0, 0.0)
    nd = 3 * nen
    dofs = (3 * om.conn[:, :, None] + np.arange(3)).reshape(om.conn.shape[0], nd)
    K = sp.coo_matrix((Ke.ravel(), (np.repeat(dofs, nd, axis=1).ravel(), np.tile(dofs, (1, nd)).ravel())),
                      shape=(3 * nn, 3 * nn)).tocsr()
    M = sp.kron(om.mass_matrix(), sp.eye(3)).tocsr()
    free = np.setdiff1d(np.arange(3 * nn), om.fixed_dofs)
    w2 = spla.eigsh(K[free][:, free].tocsc(), k=k, M=M[free][:, free].tocsc(), sigma=0.0, which="LM",
                    return_eigenvectors=False)
    return np.sqrt(np.sort(w2))
