"""Pins of the oracle's triquadratic (Q2, 27-node) hexahedra, the higher-order elements named as
future work in Sec. 7, against facts that do not come from the oracle's own formulas:

* the 3-point Gauss rule integrates every monomial of degree <= 5 per variable exactly;
* the shape functions are a partition of unity, interpolate (Kronecker delta at the nodes) and
  reproduce triquadratic polynomials;
* on the axis-aligned box [0, hx] x [0, hy] x [0, hz] the Laplace matrix is the Kronecker sum of the
  textbook 1D quadratic stiffness and mass matrices, K = (1/3h)[[7,-8,1],[-8,16,-8],[1,-8,7]] and
  M = (h/30)[[4,2,-1],[2,16,2],[-1,2,4]];
* the patch test on a jittered mesh with straight edges (interior rows of A u vanish for linear u);
* the energy of a linear field u = F x on curved elements (kappa |grad u|^2 V, lam tr(eps)^2 +
  2 mu eps:eps times V), and the null spaces (constants, six rigid-body modes);
* the convergence rates of a manufactured solution: O(h^3) in L2 and O(h^2) in the H1 seminorm.
"""
import math

import numpy as np
import pytest

from oracle import fem
from paper_2308_09839_gb300 import inputs


def test_gauss3_exact_to_degree_5():
    pts, w = fem.gauss3_points()
    assert abs(w.sum() - 8.0) < 1e-14
    for a in range(6):
        for b in range(6):
            for c in range(6):
                exact = 1.0
                for e in (a, b, c):
                    exact *= 0.0 if e % 2 else 2.0 / (e + 1)
                got = np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
                assert abs(got - exact) < 1e-13, (a, b, c)


def test_q2_shape_functions():
    nodes = fem.q2_nodes()
    assert np.allclose(fem.q2_shape_values(nodes), np.eye(27), atol=1e-15)
    rng = np.random.default_rng(0)
    pts = rng.uniform(-1, 1, size=(20, 3))
    N = fem.q2_shape_values(pts)
    assert np.allclose(N.sum(axis=1), 1.0, atol=1e-14)
    f = lambda x: 1 + x[:, 0] - 2 * x[:, 1] ** 2 + 3 * x[:, 0] * x[:, 2] + x[:, 0] ** 2 * x[:, 1] ** 2 * x[:, 2] ** 2
    assert np.allclose(N @ f(nodes), f(pts), atol=1e-13)
    dN = fem.q2_shape_ref_grads(pts)
    assert np.allclose(dN.sum(axis=1), 0.0, atol=1e-13)
    # derivative of the interpolant of f equals df/dxi (f is in the space)
    dfx = 1 + 3 * pts[:, 2] + 2 * pts[:, 0] * pts[:, 1] ** 2 * pts[:, 2] ** 2
    assert np.allclose(np.einsum("qa,a->q", dN[:, :, 0], f(nodes)), dfx, atol=1e-12)


def test_q2_box_element_is_kronecker_sum():
    hx, hy, hz = 0.7, 1.3, 0.4
    X = (fem.q2_nodes() + 1.0) / 2.0 * np.array([hx, hy, hz])
    A = fem.laplace_element_matrices(X[None], np.array([1.0]))[0]
    K = lambda h: np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / (3.0 * h)
    M = lambda h: np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) * h / 30.0
    # node a = i + 3 j + 9 k: x index fastest, so the Kronecker order is z (x) y (x) x
    ref = np.kron(M(hz), np.kron(M(hy), K(hx))) + np.kron(M(hz), np.kron(K(hy), M(hx))) + \
        np.kron(K(hz), np.kron(M(hy), M(hx)))
    assert np.allclose(A, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("physics", ["laplace", "elasticity", "vector_laplace"])
def test_q2_patch_test_straight_edges(physics):
    p = inputs.q2_box(physics, 3, ny=2, nz=3, jitter=0.2, seed=3)
    mat = np.ones(p.n_cells) if physics != "elasticity" else np.tile([1.0, 0.3], (p.n_cells, 1))
    F = np.array([[0.3, -1.1, 0.4], [0.9, 0.2, -0.6], [-0.5, 0.7, 1.2]])
    u = p.coords @ F[0] if physics == "laplace" else (p.coords @ F.T).reshape(-1)
    y = fem.apply(physics, p.coords, p.cells, mat, np.zeros_like(p.dirichlet), u)
    c = p.coords
    interior = np.all((c > 1e-12) & (c < 1 - 1e-12), axis=1)
    rows = np.repeat(interior, 1 if physics == "laplace" else 3)
    assert np.max(np.abs(y[rows])) < 1e-12 * np.max(np.abs(y))
    assert np.max(np.abs(y[~rows])) > 1e-3


def test_q2_linear_field_energy_and_null_spaces_on_curved_elements():
    p = inputs.q2_box("elasticity", 2, ny=2, nz=2, jitter=0.15, curve=0.08, seed=4)
    X = p.coords[p.cells]
    w, dN = fem.reference_rule(27)
    vol = np.einsum("q,eq->e", w, np.linalg.det(fem.jacobians(X, dN)))
    assert abs(vol.sum() - 1.0) < 1e-13
    rng = np.random.default_rng(5)
    F = rng.normal(size=(3, 3))
    E = X.shape[0]
    kappa = rng.uniform(0.5, 2, size=E)
    lam, mu = rng.uniform(0.5, 2, size=E), rng.uniform(0.5, 2, size=E)
    AL = fem.laplace_element_matrices(X, kappa)
    us = X @ F[0]
    assert np.allclose(np.einsum("ea,eab,eb->e", us, AL, us), kappa * (F[0] @ F[0]) * vol, rtol=1e-11)
    AE = fem.elasticity_element_matrices(X, lam, mu)
    uv = (X @ F.T).reshape(E, 81)
    eps = 0.5 * (F + F.T)
    dens = lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps)
    assert np.allclose(np.einsum("ea,eab,eb->e", uv, AE, uv), dens * vol, rtol=1e-11)
    for e in range(E):
        assert np.allclose(AL[e] @ np.ones(27), 0, atol=1e-12)
        for W in (np.array([[0, -1, 0], [1, 0, 0], [0, 0, 0.]]), np.array([[0, 0, 1], [0, 0, 0], [-1, 0, 0.]]),
                  np.array([[0, 0, 0], [0, 0, -1], [0, 1, 0.]])):
            assert np.allclose(AE[e] @ (X[e] @ W.T).reshape(-1), 0, atol=1e-11)
        assert np.allclose(AE[e] @ np.tile([1.0, -2.0, 0.5], 27), 0, atol=1e-11)
        assert np.linalg.matrix_rank(AE[e], tol=1e-9 * np.abs(AE[e]).max()) == 81 - 6


def _q2_mms_errors(n, jitter):
    """Q2 solution of -lap u = f for u = cos(pi x) cos(pi y) sin(pi z / 2) (u = 0 on z = 0, natural
    conditions elsewhere) on the n^3 box: L2 and H1-seminorm errors.  The load vector and the error
    integrals use the 3x3x3 Gauss rule and the oracle's Q2 shape functions (pinned above)."""
    p = inputs.q2_box("laplace", n, jitter=jitter, seed=7)
    pi = math.pi
    u = lambda X: np.cos(pi * X[..., 0]) * np.cos(pi * X[..., 1]) * np.sin(pi * X[..., 2] / 2)
    gu = lambda X: np.stack([-pi * np.sin(pi * X[..., 0]) * np.cos(pi * X[..., 1]) * np.sin(pi * X[..., 2] / 2),
                             -pi * np.cos(pi * X[..., 0]) * np.sin(pi * X[..., 1]) * np.sin(pi * X[..., 2] / 2),
                             pi / 2 * np.cos(pi * X[..., 0]) * np.cos(pi * X[..., 1]) * np.cos(pi * X[..., 2] / 2)], -1)
    pts, w = fem.gauss3_points()
    N = fem.q2_shape_values(pts)                       # (27 q, 27 a)
    dN = fem.q2_shape_ref_grads(pts)                   # (27 q, 27 a, 3)
    Xe = p.coords[p.cells]                             # (E, 27, 3)
    Xq = np.einsum("qa,eai->eqi", N, Xe)
    J = fem.jacobians(Xe, dN)
    det = np.linalg.det(J)
    f = 2.25 * pi * pi * u(Xq)
    be = np.einsum("q,eq,qa,eq->ea", w, det, N, f)
    b = np.bincount(p.cells.reshape(-1), weights=be.reshape(-1), minlength=p.n_nodes)
    b[p.dirichlet.astype(bool)] = 0.0
    A = fem.assemble_csr("laplace", p.coords, p.cells, np.ones(p.n_cells), p.dirichlet, p.n_nodes)
    import scipy.sparse.linalg as spl
    uh = spl.spsolve(A.tocsc(), b)
    ue = uh[p.cells]                                   # (E, 27)
    uq = np.einsum("qa,ea->eq", N, ue)
    g_ref = np.einsum("qaj,ea->eqj", dN, ue)
    gq = np.einsum("eqji,eqj->eqi", np.linalg.inv(J), g_ref)  # J^{-T} grad_ref
    e0 = math.sqrt(np.einsum("q,eq,eq->", w, det, (uq - u(Xq)) ** 2))
    e1 = math.sqrt(np.einsum("q,eq,eqi->", w, det, (gq - gu(Xq)) ** 2))
    return e0, e1


@pytest.mark.parametrize("jitter", [0.0, 0.15])
def test_q2_manufactured_solution_convergence(jitter):
    """Q2: O(h^3) in L2 and O(h^2) in the H1 seminorm (straight-edged jittered meshes included)."""
    e = [_q2_mms_errors(n, jitter) for n in (2, 4, 8)]
    r0 = [math.log2(e[i][0] / e[i + 1][0]) for i in range(2)]
    r1 = [math.log2(e[i][1] / e[i + 1][1]) for i in range(2)]
    assert r0[-1] > 2.8, r0
    assert 1.8 < r1[-1] < 2.3, r1
