"""Pins of the oracle's P1 tetrahedra (the simplex elements named as future work in Sec. 7), checked
against facts that do not come from the oracle's own formulas:

* the unit right tetrahedron's Laplace matrix (the textbook closed form);
* the cotangent formula: off the diagonal, A_ij = -|e_kl| cot(theta_kl) / 6 with e_kl the edge
  opposite to edge ij and theta_kl the dihedral angle at it (Duffin 1959), on distorted elements;
* the strain energy of a linear field u = F x, which P1 integrates exactly: u^T A u equals
  kappa |grad u|^2 |T| (Laplace) and (lam tr(eps)^2 + 2 mu eps:eps) |T| (elasticity), |T| the
  volume, for a general (non-symmetric) F;
* the null space: constants (Laplace) and the six rigid-body modes (elasticity);
* the patch test on a jittered mesh: A u = 0 on interior rows for a linear u and uniform material;
* the tetrahedralisation: orientation, conformity (every interior face shared by two elements),
  total volume 1;
* the convergence rates of a manufactured solution: O(h^2) in L2 and O(h) in the H1 seminorm.
"""
import math

import numpy as np
import pytest

from oracle import fem
from paper_2308_09839_gb300 import inputs


def _tets(seed, n=5, jitter=0.15):
    rng = np.random.default_rng(seed)
    base = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    X = base[None] + jitter * rng.uniform(-1, 1, size=(n, 4, 3))
    X = X @ rng.uniform(0.5, 1.5, size=(3, 3))  # general linear distortion
    vol = np.linalg.det(np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=1))
    X[vol < 0] = X[vol < 0][:, [0, 2, 1, 3]]  # orient positively
    return X


def _volume(X):
    return np.linalg.det(np.stack([X[..., 1, :] - X[..., 0, :], X[..., 2, :] - X[..., 0, :],
                                   X[..., 3, :] - X[..., 0, :]], axis=-2)) / 6.0


def test_unit_tet_laplace_closed_form():
    X = np.array([[[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]])
    A = fem.laplace_element_matrices(X, np.array([2.5]))[0]
    ref = np.array([[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]]) / 6.0 * 2.5
    assert np.allclose(A, ref, rtol=0, atol=1e-15)


def test_cotangent_formula():
    X = _tets(1, n=8)
    A = fem.laplace_element_matrices(X, np.ones(X.shape[0]))
    for e in range(X.shape[0]):
        v = X[e]
        for i in range(4):
            for j in range(i + 1, 4):
                k, l = [t for t in range(4) if t not in (i, j)]
                ed = v[l] - v[k]
                u = ed / np.linalg.norm(ed)
                pi = (v[i] - v[k]) - np.dot(v[i] - v[k], u) * u
                pj = (v[j] - v[k]) - np.dot(v[j] - v[k], u) * u
                cot = np.dot(pi, pj) / np.linalg.norm(np.cross(pi, pj))
                assert A[e, i, j] == pytest.approx(-np.linalg.norm(ed) * cot / 6.0, rel=1e-12, abs=1e-14)


def test_linear_field_energy():
    X = _tets(2, n=6)
    rng = np.random.default_rng(3)
    F = rng.normal(size=(3, 3))  # not symmetric
    kappa = rng.uniform(0.5, 2.0, size=X.shape[0])
    lam, mu = rng.uniform(0.5, 2.0, size=X.shape[0]), rng.uniform(0.5, 2.0, size=X.shape[0])
    vol = _volume(X)
    a = F[0]
    u_s = X @ a                                     # (E, 4) scalar field a.x
    AL = fem.laplace_element_matrices(X, kappa)
    assert np.allclose(np.einsum("ea,eab,eb->e", u_s, AL, u_s), kappa * (a @ a) * vol, rtol=1e-12)
    u_v = (X @ F.T).reshape(X.shape[0], 12)        # displacement F x at the nodes, xyz interleaved
    AE = fem.elasticity_element_matrices(X, lam, mu)
    eps = 0.5 * (F + F.T)
    dens = lam * np.trace(eps) ** 2 + 2.0 * mu * np.sum(eps * eps)
    assert np.allclose(np.einsum("ea,eab,eb->e", u_v, AE, u_v), dens * vol, rtol=1e-12)
    # vector Laplace: each component is the scalar operator
    AV = fem.vector_laplace_element_matrices(X, kappa)
    assert np.allclose(np.einsum("ea,eab,eb->e", u_v, AV, u_v), kappa * np.sum(F * F) * vol, rtol=1e-12)


def test_null_spaces_and_ranks():
    X = _tets(4, n=4)
    AL = fem.laplace_element_matrices(X, np.ones(4))
    AE = fem.elasticity_element_matrices(X, np.full(4, 1.3), np.full(4, 0.7))
    for e in range(4):
        assert np.allclose(AL[e] @ np.ones(4), 0, atol=1e-13)
        assert np.linalg.matrix_rank(AL[e], tol=1e-10) == 3
        assert np.allclose(AE[e], AE[e].T, atol=1e-13)
        modes = []
        for k in range(3):  # translations
            t = np.zeros((4, 3)); t[:, k] = 1.0
            modes.append(t.reshape(-1))
        for W in (np.array([[0, -1, 0], [1, 0, 0], [0, 0, 0.]]), np.array([[0, 0, 1], [0, 0, 0], [-1, 0, 0.]]),
                  np.array([[0, 0, 0], [0, 0, -1], [0, 1, 0.]])):  # rotations
            modes.append((X[e] @ W.T).reshape(-1))
        for mvec in modes:
            assert np.allclose(AE[e] @ mvec, 0, atol=1e-12)
        assert np.linalg.matrix_rank(AE[e], tol=1e-10) == 6


@pytest.mark.parametrize("physics", ["laplace", "elasticity", "vector_laplace"])
def test_patch_test_on_jittered_tet_mesh(physics):
    p = inputs.tet_box(physics, 4, ny=3, nz=5, jitter=0.15, seed=6)
    mat = np.ones(p.n_cells) if physics != "elasticity" else np.tile([1.0, 0.3], (p.n_cells, 1))
    no_bc = np.zeros_like(p.dirichlet)
    F = np.array([[0.3, -1.1, 0.4], [0.9, 0.2, -0.6], [-0.5, 0.7, 1.2]])
    if physics == "laplace":
        u = p.coords @ F[0]
    else:
        u = (p.coords @ F.T).reshape(-1)
    y = fem.apply(physics, p.coords, p.cells, mat, no_bc, u)
    c = p.coords
    interior = np.all((c > 1e-12) & (c < 1 - 1e-12), axis=1)
    nd = 1 if physics == "laplace" else 3
    rows = np.repeat(interior, nd)
    assert np.max(np.abs(y[rows])) < 1e-12 * np.max(np.abs(y))
    assert np.max(np.abs(y[~rows])) > 1e-3


def test_tetrahedralisation_is_conforming_and_oriented():
    p = inputs.tet_box("laplace", 3, ny=4, nz=2, jitter=0.15, seed=7)
    X = p.coords[p.cells]
    vol = _volume(X)
    assert np.all(vol > 0)
    assert abs(vol.sum() - 1.0) < 1e-13
    faces = {}
    for e, c in enumerate(p.cells):
        for drop in range(4):
            f = tuple(sorted(np.delete(c, drop)))
            faces.setdefault(f, []).append(e)
    on_boundary = lambda f: any(np.all(np.isclose(p.coords[list(f)][:, d], v)) for d in range(3) for v in (0.0, 1.0))
    for f, es in faces.items():
        assert len(es) == (1 if on_boundary(f) else 2), f


def _energy_error():
    X = _tets(8, n=3)
    F = np.array([[0.3, -1.1, 0.4], [0.9, 0.2, -0.6], [-0.5, 0.7, 1.2]])
    lam, mu = np.full(3, 1.7), np.full(3, 0.6)
    u_v = (X @ F.T).reshape(3, 12)
    AE = fem.elasticity_element_matrices(X, lam, mu)
    eps = 0.5 * (F + F.T)
    dens = lam * np.trace(eps) ** 2 + 2.0 * mu * np.sum(eps * eps)
    got = np.einsum("ea,eab,eb->e", u_v, AE, u_v)
    return np.max(np.abs(got - dens * _volume(X)) / (dens * _volume(X)))


def test_energy_pin_catches_planted_slips(monkeypatch):
    """The energy pin fails for plausible slips planted in the oracle (here, on the CPU)."""
    assert _energy_error() < 1e-12
    rule = fem.reference_rule
    monkeypatch.setattr(fem, "reference_rule", lambda npe: (np.ones(1), rule(npe)[1]) if npe == 4 else rule(npe))
    assert _energy_error() > 1e-3  # weight 1 instead of the reference volume 1/6
    monkeypatch.setattr(fem, "reference_rule", rule)
    monkeypatch.setattr(fem, "tet_ref_grads", lambda: np.array([[1.0, 1, 1], [1, 0, 0], [0, 1, 0], [0, 0, 1]]))
    assert _energy_error() > 1e-3  # sign of grad phi_0


def _tet_mms_errors(n):
    """P1 solution of -lap u = f for u = cos(pi x) cos(pi y) sin(pi z / 2) (u = 0 on z = 0, natural
    conditions elsewhere) on the Kuhn-split n^3 box: L2 and H1-seminorm errors.  The load vector and
    the L2 error use the 4-point rule of degree 2 (barycentric (a, b, b, b) and permutations,
    a = (5 + 3 sqrt 5) / 20, b = (5 - sqrt 5) / 20, weights |T| / 4)."""
    p = inputs.tet_box("laplace", n, jitter=0.1, seed=9)
    pi = math.pi
    u = lambda X: np.cos(pi * X[..., 0]) * np.cos(pi * X[..., 1]) * np.sin(pi * X[..., 2] / 2)
    gu = lambda X: np.stack([-pi * np.sin(pi * X[..., 0]) * np.cos(pi * X[..., 1]) * np.sin(pi * X[..., 2] / 2),
                             -pi * np.cos(pi * X[..., 0]) * np.sin(pi * X[..., 1]) * np.sin(pi * X[..., 2] / 2),
                             pi / 2 * np.cos(pi * X[..., 0]) * np.cos(pi * X[..., 1]) * np.cos(pi * X[..., 2] / 2)], -1)
    a, b = (5 + 3 * math.sqrt(5)) / 20, (5 - math.sqrt(5)) / 20
    L = np.full((4, 4), b) + np.eye(4) * (a - b)      # barycentric coordinates of the 4 points
    X = p.coords[p.cells]
    vol = _volume(X)
    Xq = np.einsum("qa,eai->eqi", L, X)
    be = np.einsum("e,qa,eq->ea", vol / 4, L, 2.25 * pi * pi * u(Xq))
    bvec = np.bincount(p.cells.reshape(-1), weights=be.reshape(-1), minlength=p.n_nodes)
    bvec[p.dirichlet.astype(bool)] = 0.0
    A = fem.assemble_csr("laplace", p.coords, p.cells, np.ones(p.n_cells), p.dirichlet, p.n_nodes)
    import scipy.sparse.linalg as spl
    uh = spl.spsolve(A.tocsc(), bvec)
    ue = uh[p.cells]
    w, dN = fem.reference_rule(4)
    J = fem.jacobians(X, dN)[:, 0]
    g = np.einsum("eji,aj,ea->ei", np.linalg.inv(J), dN[0], ue)   # constant gradient per element
    e0 = math.sqrt(np.einsum("e,eq->", vol / 4, (np.einsum("qa,ea->eq", L, ue) - u(Xq)) ** 2))
    e1 = math.sqrt(np.einsum("e,eqi->", vol / 4, (g[:, None, :] - gu(Xq)) ** 2))
    return e0, e1


def test_tet_manufactured_solution_convergence():
    """P1 on the Kuhn meshes: O(h^2) in L2 and O(h) in the H1 seminorm."""
    e = [_tet_mms_errors(n) for n in (4, 8, 16)]
    r0 = [math.log2(e[i][0] / e[i + 1][0]) for i in range(2)]
    r1 = [math.log2(e[i][1] / e[i + 1][1]) for i in range(2)]
    assert r0[-1] > 1.8, r0
    assert 0.85 < r1[-1] < 1.2, r1
