"""Plain FP64 finite-element oracle: Q1 hexahedra, 2x2x2 Gauss quadrature (TEST INFRASTRUCTURE).

Reference element: the cube [-1, 1]^3.  Corner a (a = 0..7) has reference coordinates
s_a = (+-1, +-1, +-1) with bit 0 of a -> xi, bit 1 -> eta, bit 2 -> zeta (0 -> -1, 1 -> +1), the
lexicographic order of ``paper_2308_09839_gb300.inputs``.  Shape functions
phi_a(xi) = 1/8 prod_d (1 + s_a,d xi_d).  Gauss points xi_d = +-1/sqrt(3), weights 1.

Everything here follows Sec. 2 of the paper: the element matrices of Eqs. 1 and 3 evaluated through
the isoparametric quadrature forms of Eqs. 4 and 6, with J_ij = d x_i / d xi_j and
grad phi = J^{-T} grad_ref phi.  Readings taken where the paper is silent:

* a per-cell coefficient kappa_e multiplies the Laplace integrand (the cell-wise fields of the
  abstract);
* the isotropic constitutive law is Hooke's law in Lame form, sigma = lam tr(eps) I + 2 mu eps with
  eps = sym(grad u), lam = E nu / ((1 + nu)(1 - 2 nu)), mu = E / (2 (1 + nu)), one (E, nu) pair per
  cell (two cell constants, Table 2);
* Dirichlet degrees of freedom: their columns are dropped and their rows are the identity, so
  (A x)_d = x_d.  For b_d = 0 and x0_d = 0 this is the reduced system on the free DoFs.

Triquadratic hexahedra (Q2, 27 nodes), the higher-order elements that Sec. 7 names as future work:
node a = i + 3 j + 9 k (i, j, k in {0, 1, 2}) sits at reference coordinates (i - 1, j - 1, k - 1) and
phi_a = L_i(xi) L_j(eta) L_k(zeta) with the quadratic Lagrange polynomials L_0(t) = t (t - 1) / 2,
L_1(t) = 1 - t^2, L_2(t) = t (t + 1) / 2; quadrature is the 3 x 3 x 3 Gauss rule (points 0 and
+-sqrt(3/5), weights 8/9 and 5/9; point q = i + 3 j + 9 k), exact for the stiffness integrand of
an affine Q2 element.

Linear tetrahedra (P1, 4 nodes), the simplex elements that Sec. 7 names as future work, use the
same element integrals (Eqs. 1-3) with the reference tetrahedron {xi, eta, zeta >= 0, xi + eta +
zeta <= 1}: phi_0 = 1 - xi - eta - zeta, phi_k = xi_k; the gradients are constant, so one point
with weight 1/6 (the reference volume) integrates the element matrices exactly.  Every helper below
takes the element type from the connectivity's width (8: Q1 hexahedron, 4: P1 tetrahedron, 27: Q2
hexahedron).

Parity pins live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

G = 1.0 / math.sqrt(3.0)

CHUNK = 1 << 16  # elements per vectorised block (bounds the memory of the (E, 8, 24, 24) temporaries)


def _chunk(npe: int) -> int:
    """Elements per block for elements with npe nodes (the temporaries grow as npe^2)."""
    return max(1, CHUNK * 64 // (npe * npe))


def corner_signs() -> np.ndarray:
    """(8, 3) reference coordinates s_a of the corners."""
    a = np.arange(8)
    return np.stack([(a & 1), (a >> 1) & 1, (a >> 2) & 1], axis=1).astype(np.float64) * 2.0 - 1.0


def gauss_points() -> tuple[np.ndarray, np.ndarray]:
    """Tensor 2-point Gauss rule on [-1, 1]^3: points (8, 3) and weights (8,), same corner order."""
    return corner_signs() * G, np.ones(8)


def shape_values(pts: np.ndarray) -> np.ndarray:
    """phi_a at points: (nq, 8)."""
    s = corner_signs()
    return np.prod(1.0 + pts[:, None, :] * s[None, :, :], axis=2) / 8.0


def shape_ref_grads(pts: np.ndarray) -> np.ndarray:
    """Reference gradients d phi_a / d xi_d at points: (nq, 8, 3)."""
    s = corner_signs()
    f = 1.0 + pts[:, None, :] * s[None, :, :]  # (nq, 8, 3)
    out = np.empty(f.shape)
    for d in range(3):
        o = [e for e in range(3) if e != d]
        out[:, :, d] = s[None, :, d] * f[:, :, o[0]] * f[:, :, o[1]] / 8.0
    return out


def q2_nodes() -> np.ndarray:
    """(27, 3) reference coordinates of the Q2 nodes, a = i + 3 j + 9 k at (i - 1, j - 1, k - 1)."""
    a = np.arange(27)
    return np.stack([a % 3, (a // 3) % 3, a // 9], axis=1).astype(np.float64) - 1.0


def _lagrange2(t: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Quadratic Lagrange polynomials on the nodes -1, 0, 1 and their derivatives: (n, 3) each."""
    L = np.stack([0.5 * t * (t - 1.0), 1.0 - t * t, 0.5 * t * (t + 1.0)], axis=-1)
    dL = np.stack([t - 0.5, -2.0 * t, t + 0.5], axis=-1)
    return L, dL


def gauss3_points() -> tuple[np.ndarray, np.ndarray]:
    """Tensor 3-point Gauss rule on [-1, 1]^3: points (27, 3), weights (27,), q = i + 3 j + 9 k."""
    g1 = np.array([-math.sqrt(0.6), 0.0, math.sqrt(0.6)])
    w1 = np.array([5.0, 8.0, 5.0]) / 9.0
    q = np.arange(27)
    idx = np.stack([q % 3, (q // 3) % 3, q // 9], axis=1)
    return g1[idx], w1[idx[:, 0]] * w1[idx[:, 1]] * w1[idx[:, 2]]


def q2_shape_values(pts: np.ndarray) -> np.ndarray:
    """phi_a at points: (nq, 27)."""
    n = q2_nodes().astype(int) + 1
    Ls = [_lagrange2(pts[:, d])[0] for d in range(3)]
    return Ls[0][:, n[:, 0]] * Ls[1][:, n[:, 1]] * Ls[2][:, n[:, 2]]


def q2_shape_ref_grads(pts: np.ndarray) -> np.ndarray:
    """Reference gradients d phi_a / d xi_d at points: (nq, 27, 3)."""
    n = q2_nodes().astype(int) + 1
    LL = [_lagrange2(pts[:, d]) for d in range(3)]
    out = np.empty((pts.shape[0], 27, 3))
    for d in range(3):
        f = [LL[e][1 if e == d else 0][:, n[:, e]] for e in range(3)]
        out[:, :, d] = f[0] * f[1] * f[2]
    return out


def tet_ref_grads() -> np.ndarray:
    """(4, 3) reference gradients of the P1 tetrahedron's shape functions (constant)."""
    return np.array([[-1.0, -1.0, -1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])


def reference_rule(npe: int) -> tuple[np.ndarray, np.ndarray]:
    """Quadrature weights (nq,) and reference gradients (nq, npe, 3) of the element with npe nodes:
    the 2x2x2 Gauss rule for the Q1 hexahedron, the one-point rule (weight 1/6) for the P1
    tetrahedron."""
    if npe == 8:
        pts, w = gauss_points()
        return w, shape_ref_grads(pts)
    if npe == 4:
        return np.array([1.0 / 6.0]), tet_ref_grads()[None]
    if npe == 27:
        pts, w = gauss3_points()
        return w, q2_shape_ref_grads(pts)
    raise ValueError(f"no element with {npe} nodes")


def jacobians(X: np.ndarray, dN: np.ndarray) -> np.ndarray:
    """J[e, q, i, j] = sum_a X[e, a, i] dN[q, a, j]   (Algorithm 1: J = sum_j x_j (x) grad_ref phi_j)."""
    return np.einsum("eai,qaj->eqij", X, dN)


def physical_grads(J: np.ndarray, dN: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Returns (grad phi (E, nq, 8, 3), det J (E, nq)), grad phi_a = J^{-T} grad_ref phi_a."""
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    # (J^{-T} g)_i = sum_j (J^{-1})_{ji} g_j
    g = np.einsum("eqji,qaj->eqai", Jinv, dN)
    return g, det


def lame(E: np.ndarray, nu: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def laplace_element_matrices(X: np.ndarray, kappa: np.ndarray) -> np.ndarray:
    """Eq. 4 times kappa_e:  A^e_ab = kappa_e sum_q (J^{-T} grad_ref phi_a).(J^{-T} grad_ref phi_b) w_q det J.

    X: (E, npe, 3) element node coordinates, kappa: (E,).  Returns (E, npe, npe)."""
    w, dN = reference_rule(X.shape[1])
    g, det = physical_grads(jacobians(X, dN), dN)
    return np.einsum("e,q,eq,eqai,eqbi->eab", kappa, w, det, g, g)


def vector_laplace_element_matrices(X: np.ndarray, kappa: np.ndarray) -> np.ndarray:
    """Eq. 5 times kappa_e: A^e_{3a+k, 3b+l} = kappa_e delta_kl sum_q (J^{-T} grad_ref phi_a).(J^{-T}
    grad_ref phi_b) w_q det J  (each displacement component sees the scalar operator)."""
    npe = X.shape[1]
    w, dN = reference_rule(npe)
    g, det = physical_grads(jacobians(X, dN), dN)
    gg = np.einsum("e,q,eq,eqai,eqbi->eab", kappa, w, det, g, g)
    A = np.zeros((X.shape[0], npe, 3, npe, 3))
    for k in range(3):
        A[:, :, k, :, k] = gg
    return A.reshape(X.shape[0], 3 * npe, 3 * npe)


def elasticity_element_matrices(X: np.ndarray, lam: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """Eq. 6 with Hooke's law:
    A^e_{3a+k, 3b+l} = sum_q w_q det J [lam d_k phi_a d_l phi_b + mu (d_l phi_a d_k phi_b + delta_kl grad phi_a . grad phi_b)].

    X: (E, npe, 3), lam, mu: (E,).  Returns (E, 3 npe, 3 npe) in the xyz-interleaved DoF order 3a + k."""
    npe = X.shape[1]
    w, dN = reference_rule(npe)
    g, det = physical_grads(jacobians(X, dN), dN)
    wd = det * w[None, :]
    t_lam = np.einsum("e,eq,eqak,eqbl->eakbl", lam, wd, g, g)
    t_mu1 = np.einsum("e,eq,eqal,eqbk->eakbl", mu, wd, g, g)
    dot = np.einsum("e,eq,eqai,eqbi->eab", mu, wd, g, g)
    A = t_lam + t_mu1
    for k in range(3):
        A[:, :, k, :, k] += dot
    return A.reshape(X.shape[0], 3 * npe, 3 * npe)


# --------------------------------------------------------------------------------------------------
# problem-level helpers
# --------------------------------------------------------------------------------------------------

def element_dofs(cells: np.ndarray, ndpn: int) -> np.ndarray:
    """(E, npe*ndpn) global DoF indices, xyz interleaved (DoF 3*node + k)."""
    cells = cells.astype(np.int64)
    if ndpn == 1:
        return cells
    return (cells[:, :, None] * ndpn + np.arange(ndpn)[None, None, :]).reshape(cells.shape[0], cells.shape[1] * ndpn)


def element_matrices(physics: str, coords: np.ndarray, cells: np.ndarray, mat: np.ndarray, elems=None) -> np.ndarray:
    """Element matrices of the listed elements (all if None)."""
    if elems is None:
        elems = np.arange(cells.shape[0])
    X = coords[cells[elems]]
    if physics == "laplace":
        return laplace_element_matrices(X, mat[elems])
    if physics == "vector_laplace":
        return vector_laplace_element_matrices(X, mat[elems])
    lam, mu = lame(mat[elems, 0], mat[elems, 1])
    return elasticity_element_matrices(X, lam, mu)


def _ndpn(physics: str) -> int:
    return 1 if physics == "laplace" else 3  # elasticity and vector_laplace: 3 components


def apply(physics, coords, cells, mat, dirichlet, x) -> np.ndarray:
    """y = A x by the three steps of Sec. 3: gather u^e, v^e = A^e u^e, add v^e into v.

    Dirichlet columns are zero (x_d is replaced by 0 before the gather) and Dirichlet rows are the
    identity (y_d = x_d)."""
    ndpn = _ndpn(physics)
    dmask = np.repeat(dirichlet.astype(bool), ndpn)
    xm = np.where(dmask, 0.0, x)
    y = np.zeros(x.shape[0])
    ch = _chunk(cells.shape[1])
    for s in range(0, cells.shape[0], ch):
        el = np.arange(s, min(s + ch, cells.shape[0]))
        Ae = element_matrices(physics, coords, cells, mat, el)
        dofs = element_dofs(cells[el], ndpn)
        ve = np.einsum("eij,ej->ei", Ae, xm[dofs])
        y += np.bincount(dofs.reshape(-1), weights=ve.reshape(-1), minlength=y.shape[0])
    y[dmask] = x[dmask]
    return y


def adjacent_elements_box(nodes: np.ndarray, nx: int, ny: int, nz: int) -> np.ndarray:
    """Elements of an nx x ny x nz box mesh touching any of the given nodes (sorted, unique)."""
    nodes = np.asarray(nodes, dtype=np.int64)
    i = nodes % (nx + 1)
    j = (nodes // (nx + 1)) % (ny + 1)
    k = nodes // ((nx + 1) * (ny + 1))
    out = []
    for a in range(8):
        ex, ey, ez = i - (a & 1), j - ((a >> 1) & 1), k - ((a >> 2) & 1)
        ok = (ex >= 0) & (ex < nx) & (ey >= 0) & (ey < ny) & (ez >= 0) & (ez < nz)
        out.append((ex + nx * (ey + ny * ez))[ok])
    return np.unique(np.concatenate(out))


def apply_rows(physics, coords, cells, mat, dirichlet, x, rows, elems) -> np.ndarray:
    """Selected rows of y = A x.  ``elems`` must contain every element touching the rows' nodes
    (``adjacent_elements_box`` for box meshes); the result is the same sum as ``apply`` restricted
    to those rows."""
    ndpn = _ndpn(physics)
    rows = np.asarray(rows, dtype=np.int64)
    dmask = np.repeat(dirichlet.astype(bool), ndpn)
    xm = np.where(dmask, 0.0, x)
    Ae = element_matrices(physics, coords, cells, mat, elems)
    dofs = element_dofs(cells[elems], ndpn)
    ve = np.einsum("eij,ej->ei", Ae, xm[dofs])
    pos = {int(r): t for t, r in enumerate(rows)}
    y = np.zeros(rows.shape[0])
    flat_d = dofs.reshape(-1)
    flat_v = ve.reshape(-1)
    sel = np.isin(flat_d, rows)
    for d, v in zip(flat_d[sel], flat_v[sel]):
        y[pos[int(d)]] += v
    drow = dmask[rows]
    y[drow] = x[rows[drow]]
    return y


def assemble_csr(physics, coords, cells, mat, dirichlet, n_nodes) -> sp.csr_matrix:
    """Global matrix in CSR (duplicates summed by scipy), Dirichlet rows/columns replaced by the
    identity.  This is the matrix-based operator of Sec. 3 used for the SpMV comparison (Table 1)."""
    ndpn = _ndpn(physics)
    n = n_nodes * ndpn
    dmask = np.repeat(dirichlet.astype(bool), ndpn)
    rows_l, cols_l, vals_l = [], [], []
    ch = _chunk(cells.shape[1])
    for s in range(0, cells.shape[0], ch):
        el = np.arange(s, min(s + ch, cells.shape[0]))
        Ae = element_matrices(physics, coords, cells, mat, el)
        dofs = element_dofs(cells[el], ndpn)
        r = np.broadcast_to(dofs[:, :, None], Ae.shape).reshape(-1)
        c = np.broadcast_to(dofs[:, None, :], Ae.shape).reshape(-1)
        v = Ae.reshape(-1)
        keep = ~(dmask[r] | dmask[c])
        rows_l.append(r[keep]); cols_l.append(c[keep]); vals_l.append(v[keep])
    d = np.nonzero(dmask)[0]
    rows_l.append(d); cols_l.append(d); vals_l.append(np.ones(d.shape[0]))
    A = sp.coo_matrix((np.concatenate(vals_l), (np.concatenate(rows_l), np.concatenate(cols_l))), shape=(n, n))
    A = A.tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def diagonal(physics, coords, cells, mat, dirichlet, n_nodes) -> np.ndarray:
    """diag(A) with the Dirichlet convention above (Jacobi preconditioner)."""
    ndpn = _ndpn(physics)
    dmask = np.repeat(dirichlet.astype(bool), ndpn)
    dg = np.zeros(n_nodes * ndpn)
    ch = _chunk(cells.shape[1])
    for s in range(0, cells.shape[0], ch):
        el = np.arange(s, min(s + ch, cells.shape[0]))
        Ae = element_matrices(physics, coords, cells, mat, el)
        dofs = element_dofs(cells[el], ndpn)
        dg += np.bincount(dofs.reshape(-1), weights=np.einsum("eii->ei", Ae).reshape(-1), minlength=dg.shape[0])
    dg[dmask] = 1.0
    return dg


# --------------------------------------------------------------------------------------------------
# quadrature of fields (manufactured-solution checks)
# --------------------------------------------------------------------------------------------------

def load_vector(coords, cells, dirichlet, f) -> np.ndarray:
    """b_a = sum_e sum_q phi_a(xi_q) f(x(xi_q)) w_q det J, Dirichlet entries zeroed (scalar problem)."""
    pts, w = gauss_points()
    N = shape_values(pts)
    dN = shape_ref_grads(pts)
    b = np.zeros(coords.shape[0])
    ch = _chunk(cells.shape[1])
    for s in range(0, cells.shape[0], ch):
        el = np.arange(s, min(s + ch, cells.shape[0]))
        X = coords[cells[el]]
        det = np.linalg.det(jacobians(X, dN))
        xq = np.einsum("qa,eai->eqi", N, X)
        fq = f(xq[..., 0], xq[..., 1], xq[..., 2])
        be = np.einsum("qa,eq,q,eq->ea", N, fq, w, det)
        b += np.bincount(cells[el].reshape(-1), weights=be.reshape(-1), minlength=b.shape[0])
    b[dirichlet.astype(bool)] = 0.0
    return b


def error_norms(coords, cells, uh, u, grad_u) -> tuple[float, float]:
    """(L2 error, H1-seminorm error) of the Q1 field uh against u, by 2x2x2 Gauss."""
    pts, w = gauss_points()
    N = shape_values(pts)
    dN = shape_ref_grads(pts)
    e0 = e1 = 0.0
    ch = _chunk(cells.shape[1])
    for s in range(0, cells.shape[0], ch):
        el = np.arange(s, min(s + ch, cells.shape[0]))
        X = coords[cells[el]]
        g, det = physical_grads(jacobians(X, dN), dN)
        xq = np.einsum("qa,eai->eqi", N, X)
        ue = uh[cells[el]]
        uq = np.einsum("qa,ea->eq", N, ue)
        gq = np.einsum("eqai,ea->eqi", g, ue)
        ex = u(xq[..., 0], xq[..., 1], xq[..., 2])
        gx = grad_u(xq[..., 0], xq[..., 1], xq[..., 2])
        wd = det * w[None, :]
        e0 += float(np.sum((uq - ex) ** 2 * wd))
        e1 += float(np.sum(np.sum((gq - gx) ** 2, axis=-1) * wd))
    return math.sqrt(e0), math.sqrt(e1)


def volumes(coords, cells) -> np.ndarray:
    """sum_q w_q det J per element."""
    pts, w = gauss_points()
    dN = shape_ref_grads(pts)
    out = np.empty(cells.shape[0])
    ch = _chunk(cells.shape[1])
    for s in range(0, cells.shape[0], ch):
        el = np.arange(s, min(s + ch, cells.shape[0]))
        out[el] = np.linalg.det(jacobians(coords[cells[el]], dN)) @ w
    return out
