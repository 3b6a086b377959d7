"""P1 tetrahedra (the simplex elements of Sec. 7's future work) through the C ABI against the CPU
oracle: apply in FP64 (<= 1e-12 relative 2-norm) and FP32, multi-RHS, CSR pattern and values,
operator diagonal, CG and Jacobi-PCG, mixed precision, and the checks of the setup call."""
import math

import numpy as np
import pytest

from oracle import fem, solvers
from paper_2308_09839_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_2308_09839_gb300 import mf  # noqa: E402

TOL64 = 1e-12


def rel2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def oracle_apply(p, x):
    return fem.apply(p.physics, p.coords, p.cells, p.mat, p.dirichlet, x)


MESHES = {
    "laplace_jitter_5x4x6": lambda: inputs.tet_box("laplace", 5, ny=4, nz=6, jitter=0.15, seed=51, sigma=1.0),
    "laplace_1x1x1": lambda: inputs.tet_box("laplace", 1, seed=52),
    "elasticity_jitter_4x5x3": lambda: inputs.tet_box("elasticity", 4, ny=5, nz=3, jitter=0.15, seed=53),
    "elasticity_renumbered_3x3x4": lambda: _renumbered(inputs.tet_box("elasticity", 3, ny=3, nz=4, jitter=0.1, seed=54)),
    "vector_laplace_jitter_4x3x5": lambda: inputs.tet_box("vector_laplace", 4, ny=3, nz=5, jitter=0.15, seed=55),
}


def _renumbered(p):
    """Random node and element numbering (orientation kept: the vertex order is unchanged)."""
    coords, cells, dirichlet, _, elem_perm = inputs.renumber(p.coords, p.cells, p.dirichlet, seed=p.seed)
    return inputs.Problem(p.name + "_renum", p.physics, p.nx, p.ny, p.nz, coords, p.mat[elem_perm], dirichlet,
                          p.seed, cells=cells, meta=p.meta, element="tet4")


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("variant", [mf.MF_VARIANT_AUTO, mf.MF_VARIANT_REFERENCE])
def test_tet_apply_matches_oracle(name, variant):
    p = MESHES[name]()
    mesh = mf.Mesh.from_problem(p)
    assert mesh.info["tetrahedral"] and not mesh.info["structured"]
    mesh.set_variant(variant)
    for seed in (0, 1):
        x = p.x(seed)
        y = mesh.apply(gpu(x))
        torch.cuda.synchronize()
        ref = oracle_apply(p, x)
        assert rel2(y.cpu().numpy(), ref) <= TOL64, (name, seed, rel2(y.cpu().numpy(), ref))
    y32 = mesh.apply(gpu(x).float())
    torch.cuda.synchronize()
    assert rel2(y32.double().cpu().numpy(), ref) < 1e-5


def test_tet_apply_larger_mesh_many_colours():
    """20 x 18 x 22 boxes (47,520 tetrahedra): every colour class of the greedy colouring is
    exercised; bitwise repeatable."""
    p = inputs.tet_box("elasticity", 20, ny=18, nz=22, jitter=0.12, seed=56)
    mesh = mf.Mesh.from_problem(p)
    x = p.x(2)
    y1 = mesh.apply(gpu(x))
    y2 = mesh.apply(gpu(x))
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    assert rel2(y1.cpu().numpy(), oracle_apply(p, x)) <= TOL64
    assert mesh.info["n_colours"] <= 64


@pytest.mark.parametrize("nrhs", [1, 3, 16])
@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
def test_tet_multi_rhs(physics, nrhs):
    p = inputs.tet_box(physics, 4, ny=5, nz=3, jitter=0.15, seed=57)
    mesh = mf.Mesh.from_problem(p)
    nd = p.ndpn
    xs = [p.x(seed=s) for s in range(nrhs)]
    X = np.stack([x.reshape(-1, nd) for x in xs], axis=1).reshape(-1)
    Y = mesh.apply_multi(gpu(X), nrhs)
    torch.cuda.synchronize()
    Y = Y.cpu().numpy().reshape(p.n_nodes, nrhs, nd)
    for r in range(nrhs):
        assert rel2(Y[:, r, :].reshape(-1), oracle_apply(p, xs[r])) <= TOL64


@pytest.mark.parametrize("physics", ["laplace", "elasticity", "vector_laplace"])
def test_tet_csr_and_diagonal(physics):
    p = inputs.tet_box(physics, 4, ny=3, nz=5, jitter=0.15, seed=58)
    mesh = mf.Mesh.from_problem(p)
    A = mesh.assemble_csr()
    G = A.to_scipy()
    R = fem.assemble_csr(p.physics, p.coords, p.cells, p.mat, p.dirichlet, p.n_nodes)
    if physics == "vector_laplace":
        # block-diagonal pattern: (3n + k, 3m + k) for every (n, m) of the scalar pattern.  Entries
        # that are exactly zero (right angles of the Kuhn tetrahedra) stay in the pattern.
        S = fem.assemble_csr("laplace", p.coords, p.cells, p.mat, p.dirichlet, p.n_nodes).tocoo()
        want = {(3 * int(r) + k, 3 * int(c) + k) for r, c in zip(S.row, S.col) for k in range(3)}
        Gc = G.tocoo()
        assert set(zip(Gc.row.tolist(), Gc.col.tolist())) == want
        assert np.max(np.abs(G.toarray() - R.toarray())) <= 1e-13 * np.max(np.abs(R.data))
    else:
        assert np.array_equal(G.indptr, R.indptr) and np.array_equal(G.indices, R.indices)
        assert np.max(np.abs(G.data - R.data)) <= 1e-13 * np.max(np.abs(R.data))
    x = p.x()
    y = A.spmv(gpu(x))
    torch.cuda.synchronize()
    assert rel2(y.cpu().numpy(), oracle_apply(p, x)) <= TOL64
    d = torch.empty(p.n_dof, dtype=torch.float64, device="cuda")
    mf.mf_operator_diagonal(mesh, d)
    torch.cuda.synchronize()
    ref = fem.diagonal(p.physics, p.coords, p.cells, p.mat, p.dirichlet, p.n_nodes)
    assert np.max(np.abs(d.cpu().numpy() - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
def test_tet_cg_and_jacobi_match_oracle(physics):
    p = inputs.tet_box(physics, 6, ny=5, nz=7, jitter=0.1, seed=59)
    A = fem.assemble_csr(p.physics, p.coords, p.cells, p.mat, p.dirichlet, p.n_nodes)
    b = p.b()
    _, it_o, _ = solvers.cg(lambda v: A @ v, b, rtol=1e-8)
    dg = fem.diagonal(p.physics, p.coords, p.cells, p.mat, p.dirichlet, p.n_nodes)
    _, it_j, _ = solvers.pcg(lambda v: A @ v, b, lambda r: r / dg, rtol=1e-8)
    mesh = mf.Mesh.from_problem(p)
    x, info = mesh.cg(gpu(b))
    torch.cuda.synchronize()
    assert info.status == mf.MF_OK
    assert abs(info.iters - it_o) <= max(2, math.ceil(0.01 * it_o)), (info.iters, it_o)
    assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 1.05e-8 * np.linalg.norm(b)
    _, ij = mesh.cg(gpu(b), precond=mf.MF_PC_JACOBI)
    assert ij.status == mf.MF_OK
    assert abs(ij.iters - it_j) <= max(2, math.ceil(0.01 * it_j)), (ij.iters, it_j)


def test_tet_mixed_precision():
    p = inputs.tet_box("elasticity", 6, jitter=0.1, seed=60)
    A = fem.assemble_csr(p.physics, p.coords, p.cells, p.mat, p.dirichlet, p.n_nodes)
    b = p.b()
    mesh = mf.Mesh.from_problem(p)
    x, info = mesh.cg(gpu(b), precision=mf.MF_PREC_MIXED_IR, rtol=1e-10, inner_rtol=1e-4)
    torch.cuda.synchronize()
    assert info.status == mf.MF_OK
    assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 1.05e-10 * np.linalg.norm(b)


def test_tet_setup_checks():
    p = inputs.tet_box("laplace", 2, seed=61)
    coords, mat, dirichlet = gpu(p.coords), gpu(p.mat), gpu(p.dirichlet)
    bad = p.cells.copy()
    bad[3, [1, 2]] = bad[3, [2, 1]]  # one negatively oriented tetrahedron
    with pytest.raises(mf.MfError):
        mf.Mesh("laplace", coords, mat, dirichlet, gpu(bad), element="tet4")
    assert "det" in mf.mf_last_error()
    out = p.cells.copy()
    out[0, 0] = p.n_nodes  # node id out of range
    with pytest.raises(mf.MfError):
        mf.Mesh("laplace", coords, mat, dirichlet, gpu(out), element="tet4")
    mesh = mf.Mesh.from_problem(p)
    for v in (mf.MF_VARIANT_GENERAL, mf.MF_VARIANT_PARTIAL):
        with pytest.raises(mf.MfError):
            mesh.set_variant(v)
