"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics (no GPU).

Each test states what it pins.  Together they are chosen so that a plausible slip in the oracle (a
transposed Jacobian, a dropped term of the stress, a wrong sign or index in the shape functions, a
wrong Dirichlet convention, a broken scatter) fails at least one of them; ``test_oracle_mutations.py``
plants such slips and checks that these pins catch them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import fem, solvers
from paper_2308_09839_gb300 import inputs
from tests import _exact

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _mesh(n, jitter, seed=3):
    coords = inputs.box_coords(n, n, n, jitter, seed)
    cells = inputs.box_cells(n, n, n)
    return coords, cells


# ---------------------------------------------------------------------------------- quadrature ----

def test_gauss_rule_exact_to_degree_3():
    """2-point Gauss integrates x^i y^j z^k (i, j, k <= 3) exactly over [-1, 1]^3."""
    pts, w = fem.gauss_points()
    for i in range(4):
        for j in range(4):
            for k in range(4):
                q = float(np.sum(w * pts[:, 0] ** i * pts[:, 1] ** j * pts[:, 2] ** k))
                ex = float(_exact.integrate({(i, j, k): Fraction(1)}))
                assert abs(q - ex) < 1e-14


def test_shape_functions_partition_of_unity_and_kronecker():
    s = fem.corner_signs()
    N = fem.shape_values(s)
    assert np.allclose(N, np.eye(8), atol=0)
    pts = np.random.default_rng(0).uniform(-1, 1, (20, 3))
    assert np.allclose(fem.shape_values(pts).sum(1), 1.0, atol=1e-15)
    assert np.allclose(fem.shape_ref_grads(pts).sum(1), 0.0, atol=1e-15)


# ----------------------------------------------------------------------------- element matrices ----

def test_laplace_cube_closed_form():
    """Eq. 4 on a cube of side h equals the textbook Q1 matrix (tests/golden/q1_laplace_unit_cube.txt)."""
    ref = np.loadtxt(os.path.join(GOLD, "q1_laplace_unit_cube.txt"))
    for h in (1.0, 0.25, 1.0 / 3.0):
        X = fem.corner_signs()[None] * (h / 2) + np.array([0.3, -1.0, 2.0])
        A = fem.laplace_element_matrices(X, np.array([1.0]))[0]
        assert np.allclose(A, ref * h / 12.0, rtol=0, atol=1e-15 * max(1, h))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_laplace_affine_exact_rational(seed):
    """On a parallelepiped x = x0 + J xi with rational, non-symmetric J the integrand of Eq. 1 is a
    polynomial; Gauss must give the exact rational integral."""
    rng = np.random.default_rng(seed)
    Jq = [[Fraction(int(v), 8) for v in row] for row in rng.integers(-3, 4, (3, 3))]
    for d in range(3):
        Jq[d][d] += 2
    kappa = Fraction(int(rng.integers(1, 9)), 3)
    exact = np.array(_exact.affine_laplace_exact(Jq, kappa), dtype=float)
    J = np.array(Jq, dtype=float)
    X = fem.corner_signs() @ J.T + rng.normal(size=3)
    if np.linalg.det(J) <= 0:
        pytest.skip("orientation")
    A = fem.laplace_element_matrices(X[None], np.array([float(kappa)]))[0]
    assert np.max(np.abs(A - exact)) <= 1e-13 * np.max(np.abs(exact))


@pytest.mark.parametrize("seed", [0, 1])
def test_elasticity_affine_exact_rational(seed):
    """Same pin for Eq. 6 with Hooke's law (exact rational integration, 24x24)."""
    rng = np.random.default_rng(10 + seed)
    Jq = [[Fraction(int(v), 8) for v in row] for row in rng.integers(-3, 4, (3, 3))]
    for d in range(3):
        Jq[d][d] += 2
    lam, mu = Fraction(7, 5), Fraction(3, 4)
    exact = np.array(_exact.affine_elasticity_exact(Jq, lam, mu), dtype=float)
    J = np.array(Jq, dtype=float)
    if np.linalg.det(J) <= 0:
        pytest.skip("orientation")
    X = fem.corner_signs() @ J.T + rng.normal(size=3)
    A = fem.elasticity_element_matrices(X[None], np.array([float(lam)]), np.array([float(mu)]))[0]
    assert np.max(np.abs(A - exact)) <= 1e-13 * np.max(np.abs(exact))


def test_lame_parameters():
    """lam = E nu/((1+nu)(1-2nu)), mu = E/(2(1+nu)): E = 5/2, nu = 1/4 -> lam = 1, mu = 1."""
    lam, mu = fem.lame(np.array([2.5]), np.array([0.25]))
    assert abs(lam[0] - 1.0) < 1e-15 and abs(mu[0] - 1.0) < 1e-15


def test_element_matrix_symmetry_and_psd_on_distorted_hex():
    coords, cells = _mesh(2, 0.2, seed=7)
    A = fem.laplace_element_matrices(coords[cells], np.full(8, 2.0))
    assert np.allclose(A, A.transpose(0, 2, 1), atol=1e-15)
    assert np.linalg.eigvalsh(A).min() > -1e-13
    lam, mu = fem.lame(np.full(8, 1.5), np.full(8, 0.3))
    B = fem.elasticity_element_matrices(coords[cells], lam, mu)
    assert np.allclose(B, B.transpose(0, 2, 1), atol=1e-14)
    ev = np.linalg.eigvalsh(B)
    # exactly 6 zero modes (rigid body), the rest positive
    assert np.all(np.abs(ev[:, :6]) < 1e-12 * ev[:, -1:]) and np.all(ev[:, 6] > 1e-6 * ev[:, -1])


# ------------------------------------------------------------------------------- global invariants ----

def test_volume_exact():
    """sum_e sum_q w det J = 1 on the jittered unit cube: det J has degree <= 2 per variable, so
    2-point Gauss integrates it exactly."""
    coords, cells = _mesh(5, 0.2)
    assert abs(fem.volumes(coords, cells).sum() - 1.0) < 1e-14


def test_laplace_constant_null_space():
    """A 1 = 0 for the Laplace operator without Dirichlet rows (rows of A^e sum to zero)."""
    coords, cells = _mesh(4, 0.2)
    kappa = inputs.lognormal_cells(cells.shape[0], 1.0, 0)
    nod = np.zeros(coords.shape[0], np.uint8)
    y = fem.apply("laplace", coords, cells, kappa, nod, np.ones(coords.shape[0]))
    assert np.max(np.abs(y)) < 1e-13 * kappa.max()


def _rigid_modes(coords):
    n = coords.shape[0]
    modes = []
    for k in range(3):
        t = np.zeros((n, 3)); t[:, k] = 1.0
        modes.append(t.reshape(-1))
    for w in np.eye(3):
        modes.append(np.cross(w[None, :], coords).reshape(-1))
    return modes


def test_elasticity_rigid_body_modes():
    """A r = 0 for the 3 translations and 3 rotations omega x x (skew gradient -> zero strain)."""
    coords, cells = _mesh(3, 0.2)
    E = inputs.lognormal_cells(cells.shape[0], 0.5, 0)
    nu = inputs.poisson_ratio(cells.shape[0], 0)
    mat = np.stack([E, nu], 1)
    nod = np.zeros(coords.shape[0], np.uint8)
    ref = np.abs(fem.apply("elasticity", coords, cells, mat, nod, inputs.uniform_vector(coords.size, 0))).max()
    for r in _rigid_modes(coords):
        y = fem.apply("elasticity", coords, cells, mat, nod, r)
        assert np.max(np.abs(y)) < 1e-13 * ref


def test_elasticity_not_singular_beyond_rigid_modes():
    """A non-rigid linear field (pure stretch) is not in the null space (guards a dropped lam term)."""
    coords, cells = _mesh(2, 0.0)
    mat = np.tile([1.0, 0.3], (cells.shape[0], 1))
    u = np.zeros_like(coords); u[:, 0] = coords[:, 0]
    y = fem.apply("elasticity", coords, cells, mat, np.zeros(coords.shape[0], np.uint8), u.reshape(-1))
    assert np.max(np.abs(y)) > 1e-3


@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
def test_symmetry_with_dirichlet(physics):
    """x^T A y = y^T A x, Dirichlet rows as identity and columns dropped."""
    p = (inputs.laplace_box if physics == "laplace" else inputs.elasticity_box)(3, jitter=0.2, seed=4)
    cells = p.cell_array()
    x = inputs.uniform_vector(p.n_dof, 1)
    y = inputs.uniform_vector(p.n_dof, 2)
    Ax = fem.apply(physics, p.coords, cells, p.mat, p.dirichlet, x)
    Ay = fem.apply(physics, p.coords, cells, p.mat, p.dirichlet, y)
    assert abs(x @ Ay - y @ Ax) < 1e-13 * abs(x @ Ay)


@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
def test_spd_on_free_dofs(physics):
    p = (inputs.laplace_box if physics == "laplace" else inputs.elasticity_box)(2, jitter=0.2, seed=5)
    A = fem.assemble_csr(physics, p.coords, p.cell_array(), p.mat, p.dirichlet, p.n_nodes).toarray()
    assert np.allclose(A, A.T, atol=1e-13 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).min() > 0.0


def test_laplace_patch_test_jittered():
    """Linear u = a.x + c, kappa = 1 on a jittered mesh: (A u)_i = 0 at every interior node, exactly
    (the cofactor integrand has degree <= 3 per variable, so Gauss reproduces the divergence
    theorem)."""
    n = 4
    coords, cells = _mesh(n, 0.2, seed=11)
    a, c = np.array([0.7, -1.3, 0.4]), 0.25
    u = coords @ a + c
    y = fem.apply("laplace", coords, cells, np.ones(cells.shape[0]), np.zeros(coords.shape[0], np.uint8), u)
    ijk = np.stack(np.unravel_index(np.arange(coords.shape[0]), (n + 1,) * 3)[::-1], 1)
    interior = np.all((ijk > 0) & (ijk < n), axis=1)
    assert np.max(np.abs(y[interior])) < 1e-14
    assert np.max(np.abs(y[~interior])) > 1e-3  # boundary rows carry the flux


def test_elasticity_patch_test_jittered():
    n = 3
    coords, cells = _mesh(n, 0.2, seed=12)
    B = np.array([[0.3, -0.2, 0.5], [0.1, 0.4, -0.3], [-0.6, 0.2, 0.1]])
    u = (coords @ B.T + np.array([1.0, 2.0, -1.0])).reshape(-1)
    mat = np.tile([2.0, 0.27], (cells.shape[0], 1))
    y = fem.apply("elasticity", coords, cells, mat, np.zeros(coords.shape[0], np.uint8), u).reshape(-1, 3)
    ijk = np.stack(np.unravel_index(np.arange(coords.shape[0]), (n + 1,) * 3)[::-1], 1)
    interior = np.all((ijk > 0) & (ijk < n), axis=1)
    assert np.max(np.abs(y[interior])) < 1e-13
    assert np.max(np.abs(y[~interior])) > 1e-3


@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
def test_csr_product_agrees_with_elementwise(physics):
    """Second product: assembled CSR (duplicates summed by scipy) times x equals the element-wise
    apply to 1e-14."""
    p = (inputs.laplace_box if physics == "laplace" else inputs.elasticity_box)(4, jitter=0.2, seed=6)
    cells = p.cell_array()
    x = p.x()
    y1 = fem.apply(physics, p.coords, cells, p.mat, p.dirichlet, x)
    A = fem.assemble_csr(physics, p.coords, cells, p.mat, p.dirichlet, p.n_nodes)
    y2 = A @ x
    assert np.linalg.norm(y1 - y2) <= 1e-14 * np.linalg.norm(y1)
    # the Laplace sparsity pattern of an n^3 box without Dirichlet is the 27-point stencil
    if physics == "laplace":
        A0 = fem.assemble_csr(physics, p.coords, cells, p.mat, np.zeros(p.n_nodes, np.uint8), p.n_nodes)
        assert A0.nnz == (3 * 4 + 1) ** 3


def test_dirichlet_rows_identity():
    p = inputs.laplace_box(3, jitter=0.1, seed=1)
    x = inputs.uniform_vector(p.n_dof, 9)  # Dirichlet entries deliberately nonzero
    y = fem.apply("laplace", p.coords, p.cell_array(), p.mat, p.dirichlet, x)
    d = p.dirichlet.astype(bool)
    assert np.array_equal(y[d], x[d])
    # columns dropped: changing x on Dirichlet nodes changes no free row
    x2 = x.copy(); x2[d] += 5.0
    y2 = fem.apply("laplace", p.coords, p.cell_array(), p.mat, p.dirichlet, x2)
    assert np.array_equal(y2[~d], y[~d])


def test_apply_rows_matches_apply():
    p = inputs.elasticity_box(4, jitter=0.2, seed=2)
    cells = p.cell_array()
    x = p.x()
    y = fem.apply("elasticity", p.coords, cells, p.mat, p.dirichlet, x)
    rows = np.random.default_rng(0).choice(p.n_dof, 40, replace=False)
    el = fem.adjacent_elements_box(rows // 3, p.nx, p.ny, p.nz)
    ys = fem.apply_rows("elasticity", p.coords, cells, p.mat, p.dirichlet, x, rows, el)
    assert np.allclose(ys, y[rows], rtol=0, atol=1e-15 * np.abs(y).max())


def test_renumbering_invariance():
    """The operator commutes with a relabelling of nodes and elements (general connectivity path)."""
    p = inputs.laplace_box(3, jitter=0.2, seed=8)
    cells = p.cell_array()
    x = p.x()
    y = fem.apply("laplace", p.coords, cells, p.mat, p.dirichlet, x)
    c2, cl2, d2, nperm, eperm = inputs.renumber(p.coords, cells, p.dirichlet, 1)
    x2 = np.empty_like(x); x2[nperm] = x
    y2 = fem.apply("laplace", c2, cl2, p.mat[eperm], d2, x2)
    assert np.allclose(y2[nperm], y, atol=1e-14 * np.abs(y).max())


# ------------------------------------------------------------------------------------ convergence ----

def _mms_error(n, jitter):
    coords, cells = _mesh(n, jitter, seed=21)
    d = inputs.dirichlet_z0(n, n, n)
    pi = math.pi
    u = lambda x, y, z: np.cos(pi * x) * np.cos(pi * y) * np.sin(pi * z / 2)
    gu = lambda x, y, z: np.stack([-pi * np.sin(pi * x) * np.cos(pi * y) * np.sin(pi * z / 2),
                                   -pi * np.cos(pi * x) * np.sin(pi * y) * np.sin(pi * z / 2),
                                   pi / 2 * np.cos(pi * x) * np.cos(pi * y) * np.cos(pi * z / 2)], -1)
    f = lambda x, y, z: 2.25 * pi * pi * u(x, y, z)
    b = fem.load_vector(coords, cells, d, f)
    A = fem.assemble_csr("laplace", coords, cells, np.ones(cells.shape[0]), d, coords.shape[0])
    import scipy.sparse.linalg as spl
    uh = spl.spsolve(A.tocsc(), b)
    return fem.error_norms(coords, cells, uh, u, gu)


@pytest.mark.parametrize("jitter", [0.0, 0.2])
def test_manufactured_solution_convergence(jitter):
    """u = cos(pi x) cos(pi y) sin(pi z / 2), -lap u = 2.25 pi^2 u, u = 0 on z = 0, natural BCs
    elsewhere: O(h^2) in L2 and O(h) in H1."""
    e = [_mms_error(n, jitter) for n in (4, 8, 16)]
    r0 = [math.log2(e[i][0] / e[i + 1][0]) for i in range(2)]
    r1 = [math.log2(e[i][1] / e[i + 1][1]) for i in range(2)]
    assert r0[-1] > 1.85, r0
    assert 0.9 < r1[-1] < 1.3, r1


# --------------------------------------------------------------------------------------- solvers ----

def test_cg_matches_direct_solve_and_residual():
    p = inputs.small_laplace_16()
    p = inputs.laplace_box(6, jitter=0.2, sigma=1.0, seed=0)
    cells = p.cell_array()
    A = fem.assemble_csr("laplace", p.coords, cells, p.mat, p.dirichlet, p.n_nodes)
    b = p.b()
    x, it, hist = solvers.cg(lambda v: A @ v, b, rtol=1e-10)
    import scipy.sparse.linalg as spl
    xd = spl.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)
    assert hist[-1] <= 1e-10 and it == len(hist) - 1


def test_cg_finite_termination_small_spd():
    """Exact-arithmetic CG terminates in <= n steps; on a tiny well-conditioned SPD system it reaches
    1e-12 within n + 2 iterations."""
    rng = np.random.default_rng(0)
    Q = np.linalg.qr(rng.normal(size=(12, 12)))[0]
    A = Q @ np.diag(np.linspace(1, 4, 12)) @ Q.T
    b = rng.normal(size=12)
    x, it, _ = solvers.cg(lambda v: A @ v, b, rtol=1e-12)
    assert it <= 14
    assert np.allclose(x, np.linalg.solve(A, b), atol=1e-10)


def test_fcg_identity_equals_cg_and_pcg_jacobi():
    p = inputs.laplace_box(5, jitter=0.2, sigma=1.0, seed=2)
    cells = p.cell_array()
    A = fem.assemble_csr("laplace", p.coords, cells, p.mat, p.dirichlet, p.n_nodes)
    b = p.b()
    _, it_cg, h_cg = solvers.cg(lambda v: A @ v, b, rtol=1e-8)
    _, it_f, h_f = solvers.fcg(lambda v: A @ v, b, lambda r: r.copy(), rtol=1e-8)
    # equal in exact arithmetic; rounding makes the two drift apart slowly
    assert abs(it_f - it_cg) <= 1
    assert np.allclose(h_f[:20], h_cg[:20], rtol=1e-8)
    dg = fem.diagonal("laplace", p.coords, cells, p.mat, p.dirichlet, p.n_nodes)
    assert np.allclose(dg, A.diagonal(), rtol=1e-14)
    x, it_j, _ = solvers.pcg(lambda v: A @ v, b, lambda r: r / dg, rtol=1e-8)
    assert np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b)
    assert it_j < it_cg  # lognormal(0, 1) coefficients: diagonal scaling helps


def test_fcg_m_special_cases_and_orthogonality():
    """FCG(m) with a fixed preconditioner is PCG (identity: CG); with a preconditioner that changes
    every iteration its directions are still A-orthogonal within the window."""
    p = inputs.laplace_box(5, jitter=0.2, sigma=1.0, seed=2)
    cells = p.cell_array()
    A = fem.assemble_csr("laplace", p.coords, cells, p.mat, p.dirichlet, p.n_nodes)
    b = p.b()
    _, it_cg, h_cg = solvers.cg(lambda v: A @ v, b, rtol=1e-8)
    _, it_m, h_m = solvers.fcg_m(lambda v: A @ v, b, lambda r: r.copy(), m=4, rtol=1e-8)
    assert abs(it_m - it_cg) <= 1 and np.allclose(h_m[:20], h_cg[:20], rtol=1e-8)
    dg = A.diagonal()
    _, it_j, h_j = solvers.pcg(lambda v: A @ v, b, lambda r: r / dg, rtol=1e-8)
    _, it_mj, h_mj = solvers.fcg_m(lambda v: A @ v, b, lambda r: r / dg, m=1, rtol=1e-8)
    assert abs(it_mj - it_j) <= 1 and np.allclose(h_mj[:20], h_j[:20], rtol=1e-8)
    # a preconditioner that varies from call to call (random positive diagonal scalings)
    rng = np.random.default_rng(5)
    var = lambda r: r / dg * rng.uniform(0.5, 2.0, size=r.size)
    x, it_v, _, pairs = solvers.fcg_m(lambda v: A @ v, b, var, m=3, rtol=1e-8, keep_directions=True)
    assert np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b)
    for k in range(len(pairs)):
        for j in range(max(0, k - 3), k):
            pk, apk = pairs[k]
            pj, apj = pairs[j]
            assert abs(pk @ apj) <= 1e-9 * np.sqrt((pk @ apk) * (pj @ apj))


def test_iterative_refinement_fp32_inner():
    """FP64 IR around an FP32 inner CG (rtol 1e-4) reaches a 1e-10 FP64 residual."""
    p = inputs.laplace_box(6, jitter=0.1, sigma=0.5, seed=3)
    cells = p.cell_array()
    A = fem.assemble_csr("laplace", p.coords, cells, p.mat, p.dirichlet, p.n_nodes)
    A32 = A.astype(np.float32)
    b = p.b()

    def inner(r):
        dot = lambda u, v: float(np.dot(u.astype(np.float32), v.astype(np.float32)))
        d, _, _ = solvers.cg(lambda v: (A32 @ v.astype(np.float32)).astype(np.float32), r.astype(np.float32), 1e-4, dot=dot)
        return d.astype(np.float64)

    x, m, hist = solvers.iterative_refinement(lambda v: A @ v, inner, b, 1e-10)
    assert hist[-1] <= 1e-10 and m <= 6


def test_vector_laplace_is_componentwise_scalar_laplace():
    """Eq. 5: the vector Laplace element matrix equals the scalar one on each component, exactly
    (checked against exact rational integration on a parallelepiped)."""
    Jq = [[Fraction(2), Fraction(1, 8), Fraction(-3, 8)],
          [Fraction(-1, 4), Fraction(17, 8), Fraction(1, 4)],
          [Fraction(3, 8), Fraction(-1, 8), Fraction(15, 8)]]
    ex = np.array(_exact.affine_laplace_exact(Jq, Fraction(5, 3)), dtype=float)
    X = fem.corner_signs() @ np.array(Jq, dtype=float).T
    A = fem.vector_laplace_element_matrices(X[None], np.array([5.0 / 3.0]))[0].reshape(8, 3, 8, 3)
    for k in range(3):
        for l in range(3):
            blk = A[:, k, :, l]
            assert np.max(np.abs(blk - (ex if k == l else 0))) <= 1e-13 * np.abs(ex).max()
    # constants per component are in the null space without Dirichlet rows
    p = inputs.elasticity_box(3, jitter=0.2, seed=2)
    cells = p.cell_array()
    for k in range(3):
        u = np.zeros((p.n_nodes, 3)); u[:, k] = 1.0
        y = fem.apply("vector_laplace", p.coords, cells, p.mat[:, 0], np.zeros(p.n_nodes, np.uint8), u.reshape(-1))
        assert np.abs(y).max() < 1e-13


def test_single_sync_cg_pins():
    """Chronopoulos-Gear CG: finite termination on a small SPD system, the exact solution of a
    direct solve, the same residual history as CG (identity preconditioner) and as Jacobi-PCG in its
    first iterations (equal in exact arithmetic), and its residual recurrence equal to b - A x."""
    rng = np.random.default_rng(5)
    Q = np.linalg.qr(rng.normal(size=(10, 10)))[0]
    A = Q @ np.diag(np.linspace(1, 3, 10)) @ Q.T
    b = rng.normal(size=10)
    x, it, _ = solvers.cg_single_sync(lambda v: A @ v, b, rtol=1e-12)
    assert it <= 12 and np.allclose(x, np.linalg.solve(A, b), atol=1e-10)
    p = inputs.laplace_box(5, jitter=0.2, sigma=1.0, seed=3)
    cells = p.cell_array()
    A = fem.assemble_csr("laplace", p.coords, cells, p.mat, p.dirichlet, p.n_nodes)
    b = p.b()
    _, it_cg, h_cg = solvers.cg(lambda v: A @ v, b, rtol=1e-8)
    x1, it_s, h_s = solvers.cg_single_sync(lambda v: A @ v, b, rtol=1e-8)
    assert abs(it_s - it_cg) <= 1
    assert np.allclose(h_s[:20], h_cg[:20], rtol=1e-8)
    assert np.linalg.norm(b - A @ x1) <= 1.01e-8 * np.linalg.norm(b)
    dg = A.diagonal()
    _, it_j, h_j = solvers.pcg(lambda v: A @ v, b, lambda r: r / dg, rtol=1e-8)
    _, it_sj, h_sj = solvers.cg_single_sync(lambda v: A @ v, b, lambda r: r / dg, rtol=1e-8)
    assert abs(it_sj - it_j) <= 1
    assert np.allclose(h_sj[:20], h_j[:20], rtol=1e-8)


def test_cg_counts_drift_under_double_word_rounding():
    """Basis of the iteration-count tolerance of the pipelined-CG GPU tests (max(3, 3 %)).  The GPU's
    fast operators round at about 2^-48 relative (double-word arithmetic) instead of 2^-53.  With the
    oracle's operator results perturbed by that much (seeded), the oracle's own classic recurrence
    and its single-synchronisation recurrence both stop a few iterations away from their unperturbed
    counts on the 10^3 jittered Laplace problem (about 130 iterations): more than 1 % for the classic
    one, and within 3 iterations for both."""
    p = inputs.laplace_box(10, jitter=0.2, seed=73)
    A = fem.assemble_csr(p.physics, p.coords, p.cell_array(), p.mat, p.dirichlet, p.n_nodes)
    b = p.b()
    _, it_c, _ = solvers.cg(lambda v: A @ v, b, rtol=1e-8)
    _, it_p, _ = solvers.cg_single_sync(lambda v: A @ v, b, None, rtol=1e-8)
    dev_c, dev_p = [], []
    for seed in range(6):
        rng = np.random.default_rng(seed)

        def op(v):
            y = A @ v
            return y * (1.0 + 2.0 ** -48 * rng.standard_normal(y.shape))

        dev_c.append(solvers.cg(op, b, rtol=1e-8)[1] - it_c)
        rng = np.random.default_rng(seed)
        dev_p.append(solvers.cg_single_sync(op, b, None, rtol=1e-8)[1] - it_p)
    tol = max(3, math.ceil(0.03 * it_p))
    assert max(abs(d) for d in dev_c + dev_p) <= tol
    assert max(abs(d) for d in dev_c) > math.ceil(0.01 * it_c)  # the 1 % window is too tight here


@pytest.mark.parametrize("physics,min_frac", [("laplace", 0.01), ("elasticity", 0.03)])
def test_q2_cg_counts_drift_under_double_word_rounding(physics, min_frac):
    """Basis of the iteration-count tolerance (5 %) of the Q2 CG tests, whose operators are the
    double-word partial-assembly kernels.  A floating-point matrix-vector product errs per row by about
    the unit roundoff times sum_j |a_ij v_j|; with the oracle's operator perturbed by 2^-48 of that
    (double-word rounding; seeded), the oracle's own CG on the 3 x 2 x 3 straight-edged Q2 problems
    stops later by more than 1 % (Laplace, about 330 iterations: 8 more) and by more than 3 %
    (elasticity, about 1030 iterations, ill-conditioned: 30 to 37 more) - more than the 1 % of the
    scope table and the 3 % that the 10^3 Q1 Laplace problem above needs - and within 5 %."""
    p = inputs.q2_box(physics, 3, ny=2, nz=3, jitter=0.1, seed=88)
    A = fem.assemble_csr(p.physics, p.coords, p.cells, p.mat, p.dirichlet, p.n_nodes)
    absA = abs(A)
    b = p.b()
    _, it0, _ = solvers.cg(lambda v: A @ v, b, rtol=1e-8)

    def drift(seed):
        rng = np.random.default_rng(seed)
        return solvers.cg(lambda v: A @ v + 2.0 ** -48 * rng.standard_normal(v.shape) * (absA @ np.abs(v)),
                          b, rtol=1e-8)[1] - it0

    dev = [drift(s) for s in range(4)]
    assert max(abs(d) for d in dev) > math.ceil(min_frac * it0)
    assert max(abs(d) for d in dev) <= math.ceil(0.05 * it0)
