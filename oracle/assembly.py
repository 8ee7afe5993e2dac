"""Fixed-sparsity patterns, global force, mass, residual and Hessian.

Paper passages:
  * Sec. 4.2: CSR (offsets, columns, values); coefficient-level adjacency from
    element connectivity by encoding (i, j) pairs as 64-bit keys, sorting,
    removing duplicates, counting rows and scanning; the Newton matrix pattern
    lifts each adjacent (I, J) to a 3x3 block of DOFs; clamped (Dirichlet)
    constraints are identity rows of C_q.
  * eq. fint_global: f_I = sum over elements sharing I of f_a(e,I).
  * eq. residual / eq. grad_L: g = M (v - v_n)/h + f_int(q_n + h v, v)
    - f_ext - f_ff + h C_q^T (lambda + rho c).
  * eq. hessian: H = M/h + h K_t + h^2 rho C_q^T C_q, plus the Kelvin-Voigt
    velocity tangent D (see element.py for that reading).

  * Sec. 4.2 (general constraints): C_q in CSR with a user-given fixed
    pattern; the Newton-matrix pattern also holds every DOF pair that a row
    of C_q couples, so h^2 rho C_q^T C_q causes no fill-in.

Readings: the DOF CSR stores the full symmetric matrix with ascending rows
and columns; f_ff = int rho N_a g dV = (row sums of M) x gravity; the clamp
constraint of DOF r is c_r(q) = q_r - X_r.  General constraints are linear,
c(q) = C q - b, with C (ncon x 3nn) and b given; their rows follow the clamp
rows in c, C_q and lambda.  The pattern lifts them at node level: two nodes
whose DOFs share a row of C become adjacent (their whole 3x3 block enters the
pattern).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import element as elem
from . import t10


# ---------------------------------------------------------------------------
# Sparsity (Sec. 4.2)
# ---------------------------------------------------------------------------

def node_adjacency(conn, nn, extra_pairs=None):
    """Coefficient-level CSR: 64-bit keys I*nn + J for every element-local
    pair (and every node pair in `extra_pairs`, an (k, 2) array), sorted and
    de-duplicated, then row counts and an exclusive scan."""
    nen = conn.shape[1]
    a = np.repeat(np.arange(nen), nen)
    b = np.tile(np.arange(nen), nen)
    I = conn[:, a].astype(np.int64).ravel()
    J = conn[:, b].astype(np.int64).ravel()
    if extra_pairs is not None and len(extra_pairs):
        ep = np.asarray(extra_pairs, dtype=np.int64).reshape(-1, 2)
        I = np.concatenate([I, ep[:, 0], ep[:, 1]])
        J = np.concatenate([J, ep[:, 1], ep[:, 0]])
    keys = np.unique(I * nn + J)
    rows = keys // nn
    cols = keys % nn
    counts = np.bincount(rows, minlength=nn)
    ptr = np.zeros(nn + 1, dtype=np.int64)
    np.cumsum(counts, out=ptr[1:])
    return ptr, cols


def dof_pattern(node_ptr, node_col):
    """Lift the node adjacency to DOF level: every adjacent (I, J) gives the
    3x3 block (3I+d, 3J+e).  Returns (row_ptr, col) of the full symmetric
    DOF CSR with ascending columns."""
    nn = len(node_ptr) - 1
    deg = np.diff(node_ptr)
    rows_node = np.repeat(np.arange(nn, dtype=np.int64), deg)
    keys = []
    ndof = 3 * nn
    for d in range(3):
        for e in range(3):
            keys.append((3 * rows_node + d) * ndof + 3 * node_col + e)
    keys = np.sort(np.concatenate(keys))
    rows = keys // ndof
    cols = keys % ndof
    counts = np.bincount(rows, minlength=ndof)
    row_ptr = np.zeros(ndof + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, cols


def csr_positions(row_ptr, col, rows, cols):
    """Position in `values` of entries (rows[k], cols[k]); raises if absent."""
    ndof = len(row_ptr) - 1
    nnz_rows = np.repeat(np.arange(ndof, dtype=np.int64), np.diff(row_ptr))
    keys = nnz_rows * ndof + col
    q = np.asarray(rows, dtype=np.int64) * ndof + np.asarray(cols, dtype=np.int64)
    pos = np.searchsorted(keys, q)
    if np.any(pos >= len(keys)) or np.any(keys[np.minimum(pos, len(keys) - 1)] != q):
        raise KeyError("entry not in pattern")
    return pos


def element_dofs(conn):
    """(ne, 3 nen) global DOF of local row 3a+i."""
    return (3 * conn[:, :, None].astype(np.int64) + np.arange(3)).reshape(conn.shape[0], 3 * conn.shape[1])


def slot_map(conn, row_ptr, col):
    """(ne, (3 nen)^2) CSR position of K_elem entry (r, s), r = 3a+i, s = 3b+k."""
    dofs = element_dofs(conn)
    ne, nd = dofs.shape
    R = np.repeat(dofs, nd, axis=1)
    S = np.tile(dofs, (1, nd))
    return csr_positions(row_ptr, col, R.ravel(), S.ravel()).reshape(ne, nd * nd)


# ---------------------------------------------------------------------------
# The mesh-level constants of Sec. 4.1
# ---------------------------------------------------------------------------

class OracleMesh:
    """Reference-configuration constants of one (possibly multi-material) mesh.

    materials: list of material dicts; mat_of_elem: (ne,) index (or None).
    """

    def __init__(self, X, conn, materials, mat_of_elem=None, fixed_nodes=(), constraints=None):
        self.X = np.asarray(X, dtype=np.float64)
        self.conn = np.asarray(conn, dtype=np.int64)
        self.nn = self.X.shape[0]
        self.ne = self.conn.shape[0]
        self.materials = list(materials)
        self.mat_of_elem = (np.zeros(self.ne, dtype=np.int64) if mat_of_elem is None
                            else np.asarray(mat_of_elem, dtype=np.int64))
        self.fixed_nodes = np.sort(np.asarray(fixed_nodes, dtype=np.int64))
        self.nen = self.conn.shape[1]
        rho = np.array([m["rho0"] for m in self.materials])[self.mat_of_elem]
        self._reference(rho)
        if np.any(self.J0 <= 0.0):
            raise ValueError("element with non-positive reference Jacobian")
        # general linear constraints c = C q - b (rows after the clamp rows)
        if constraints is None:
            self.C_lin = sp.csr_matrix((0, 3 * self.nn))
            self.b_lin = np.zeros(0)
        else:
            self.C_lin = sp.csr_matrix(constraints[0], shape=(len(constraints[1]), 3 * self.nn))
            self.b_lin = np.asarray(constraints[1], dtype=np.float64).reshape(-1)
        self._pattern = None

    def _reference(self, rho):
        """Sec. 4.1 constants of the T10 elements: grad_X N per quadrature
        point, J0, w_q J0 and the element mass (ne, 10, 10)."""
        self.gradN, self.J0, self.wJ0 = t10.reference_geometry(self.X, self.conn)
        self.Me = t10.element_mass(self.X, self.conn, rho)

    # --- pattern ---------------------------------------------------------
    def constraint_node_pairs(self):
        """Node pairs (I, J) whose DOFs share a row of the general C."""
        pairs = []
        C = self.C_lin.tocsr()
        for r in range(C.shape[0]):
            nodes = np.unique(C.indices[C.indptr[r]:C.indptr[r + 1]] // 3)
            pairs += [(I, J) for I in nodes for J in nodes]
        return np.array(pairs, dtype=np.int64).reshape(-1, 2)

    def pattern(self):
        if self._pattern is None:
            node_ptr, node_col = node_adjacency(self.conn, self.nn, self.constraint_node_pairs())
            row_ptr, col = dof_pattern(node_ptr, node_col)
            self._pattern = (node_ptr, node_col, row_ptr, col)
        return self._pattern

    @property
    def fixed_dofs(self):
        return (3 * self.fixed_nodes[:, None] + np.arange(3)).ravel()

    # --- mass ------------------------------------------------------------
    def mass_matrix(self):
        """Global scalar (node-level) consistent mass, scipy CSR (nn x nn)."""
        a = np.repeat(np.arange(self.nen), self.nen)
        b = np.tile(np.arange(self.nen), self.nen)
        I = self.conn[:, a].ravel()
        J = self.conn[:, b].ravel()
        return sp.coo_matrix((self.Me.reshape(-1), (I, J)), shape=(self.nn, self.nn)).tocsr()

    def gravity_force(self, gravity):
        """f_ff = int rho N_a g dV = (row sums of M) (x) g, flattened (3nn,)."""
        m_row = np.asarray(self.mass_matrix().sum(axis=1)).ravel()
        return (m_row[:, None] * np.asarray(gravity)[None, :]).ravel()

    # --- element loops -----------------------------------------------------
    def _by_material(self):
        for k, mat in enumerate(self.materials):
            idx = np.nonzero(self.mat_of_elem == k)[0]
            if len(idx):
                yield idx, mat

    def element_forces(self, x, v):
        """(ne, nen, 3) element forces at nodal positions x and velocities v (nn,3)."""
        fe = np.zeros((self.ne, self.nen, 3), dtype=np.result_type(x, v))
        for idx, mat in self._by_material():
            c = self.conn[idx]
            fe[idx] = elem.element_force(x[c], v[c], self.gradN[idx], self.wJ0[idx], mat)
        return fe

    def element_tangents(self, x, v, alpha=1.0, beta=0.0):
        nd = 3 * self.nen
        Ke = np.zeros((self.ne, nd, nd), dtype=np.result_type(x, v))
        for idx, mat in self._by_material():
            c = self.conn[idx]
            Ke[idx] = elem.element_tangent(x[c], v[c], self.gradN[idx], self.wJ0[idx],
                                           mat, alpha, beta)
        return Ke

    # --- global quantities ------------------------------------------------
    def internal_force(self, q_n, v, h):
        """f_int(q_n + h v, v) as a flat (3nn,) vector (eq. fint_global)."""
        q_n = np.asarray(q_n).reshape(-1, 3)
        v = np.asarray(v).reshape(-1, 3)
        fe = self.element_forces(q_n + h * v, v)
        f = np.zeros(3 * self.nn, dtype=fe.dtype)
        np.add.at(f, element_dofs(self.conn).ravel(), fe.reshape(-1))
        return f

    def hessian_values(self, q_n, v, h, rho_alm):
        """CSR values of H = M/h + h K_t + D + h^2 rho C_q^T C_q (full symmetric)."""
        _, _, row_ptr, col = self.pattern()
        q_n = np.asarray(q_n).reshape(-1, 3)
        v = np.asarray(v).reshape(-1, 3)
        Ke = self.element_tangents(q_n + h * v, v, alpha=h, beta=1.0)
        # mass: M_e/h on the (3I+d, 3J+d) entries
        Me = self.Me / h
        nd = 3 * self.nen
        Kfull = Ke + np.einsum("eab,ik->eaibk", Me, np.eye(3)).reshape(self.ne, nd, nd)
        values = np.zeros(len(col))
        np.add.at(values, slot_map(self.conn, row_ptr, col).ravel(), Kfull.reshape(-1))
        fd = self.fixed_dofs
        values[csr_positions(row_ptr, col, fd, fd)] += h * h * rho_alm
        if self.C_lin.shape[0]:
            CtC = (self.C_lin.T @ self.C_lin).tocoo()
            np.add.at(values, csr_positions(row_ptr, col, CtC.row, CtC.col), h * h * rho_alm * CtC.data)
        return values

    def hessian_matrix(self, q_n, v, h, rho_alm):
        _, _, row_ptr, col = self.pattern()
        vals = self.hessian_values(q_n, v, h, rho_alm)
        n = 3 * self.nn
        return sp.csr_matrix((vals, col, row_ptr), shape=(n, n))

    def internal_energy(self, q):
        """Pi_int(q) = sum_e Pi_e (hyperelastic part)."""
        q = np.asarray(q).reshape(-1, 3)
        total = 0.0
        for idx, mat in self._by_material():
            total = total + np.sum(elem.element_energy(q[self.conn[idx]], self.gradN[idx],
                                                       self.wJ0[idx], mat))
        return total

    def augmented_cost(self, v, q_n, v_n, h, f_ext, gravity, lam, rho_alm, M=None):
        """Phi_rho(v, lambda) of eq. cost (hyperelastic materials)."""
        if M is None:
            M = self.mass_matrix()
        v = np.asarray(v).reshape(-1)
        dv = (v - np.asarray(v_n).reshape(-1)).reshape(-1, 3)
        q = np.asarray(q_n).reshape(-1) + h * v
        c = self.constraint(q)
        phi = 0.5 / h * np.sum(dv * (M @ dv))
        phi = phi + self.internal_energy(q) / h
        if f_ext is not None:
            phi = phi - np.asarray(f_ext).reshape(-1) @ v
        phi = phi - self.gravity_force(gravity) @ v
        phi = phi + np.asarray(lam).reshape(-1) @ c + 0.5 * rho_alm * (c @ c)
        return phi

    def constraint(self, q):
        """c(q): the clamp rows q_r - X_r at every fixed DOF r, then the
        general rows C q - b."""
        fd = self.fixed_dofs
        q = np.asarray(q).reshape(-1)
        c = q[fd] - self.X.reshape(-1)[fd]
        if self.C_lin.shape[0]:
            c = np.concatenate([c, self.C_lin @ q - self.b_lin])
        return c

    def residual(self, v, q_n, v_n, h, f_ext, gravity, lam, rho_alm, M=None):
        """g(v, lambda) of eq. residual, flat (3nn,)."""
        if M is None:
            M = self.mass_matrix()
        v = np.asarray(v).reshape(-1)
        q_n = np.asarray(q_n).reshape(-1)
        dv = (v - np.asarray(v_n).reshape(-1)).reshape(-1, 3)
        g = (M @ dv).reshape(-1) / h
        g = g + self.internal_force(q_n, v, h)
        if f_ext is not None:
            g = g - np.asarray(f_ext).reshape(-1)
        g = g - self.gravity_force(gravity)
        q = q_n + h * v
        fd = self.fixed_dofs
        w = np.asarray(lam).reshape(-1) + rho_alm * self.constraint(q)     # lambda + rho c
        g[fd] += h * w[:len(fd)]
        if self.C_lin.shape[0]:
            g = g + h * (self.C_lin.T @ w[len(fd):])                      # h C_q^T (lambda + rho c)
        return g
