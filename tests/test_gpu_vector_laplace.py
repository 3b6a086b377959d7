"""Vector Laplace operator (Eq. 5: the scalar element matrix of Eq. 4 acting on each of three
components) through the C ABI against the CPU oracle: every apply variant, FP32 error, CSR
(block-diagonal pattern), multi-RHS, CG.  FP64 results agree with the oracle to <= 1e-12 relative
in the 2-norm."""
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
    return fem.apply(p.physics, p.coords, p.cell_array(), p.mat, p.dirichlet, x)


MESHES = {
    # jittered box: general structured kernel (auto) / colour kernel (reference, unstructured)
    "jitter_7x6x5": lambda: inputs.vector_laplace_box(7, ny=6, nz=5, jitter=0.2, seed=21),
    # graded tensor-product grid with ragged tiles: face-marching kernel
    "graded_45x19x9": lambda: inputs.vector_laplace_box(45, ny=19, nz=9, graded=0.5, seed=22),
    "cartesian_1x1x1": lambda: inputs.vector_laplace_box(1, seed=23),
    "cartesian_layers_12": lambda: inputs.vector_laplace_box(12, sigma=0.5, layered=True, seed=24),
}


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("variant", [mf.MF_VARIANT_AUTO, mf.MF_VARIANT_REFERENCE])
@pytest.mark.parametrize("structured", [True, False])
def test_vector_laplace_apply_matches_oracle(name, variant, structured):
    p = MESHES[name]()
    mesh = mf.Mesh.from_problem(p, structured=structured)
    mesh.set_variant(variant)
    for seed in (0, 1):
        x = p.x(seed)
        y = mesh.apply(gpu(x))
        torch.cuda.synchronize()
        ref = oracle_apply(p, x)
        assert rel2(y.cpu().numpy(), ref) <= TOL64, (name, seed, rel2(y.cpu().numpy(), ref))
    y32 = mesh.apply(gpu(x).float())
    torch.cuda.synchronize()
    assert rel2(y32.double().cpu().numpy(), ref) < 2e-6


def test_vector_laplace_is_the_scalar_operator_per_component():
    """A property that holds at any size: component k of A_vec x equals the GPU scalar Laplace of
    component k of x (same mesh, same kappa)."""
    pv = inputs.vector_laplace_box(40, ny=33, nz=21, graded=0.3, seed=25)
    ps = inputs.laplace_box(40, ny=33, nz=21, graded=0.3, seed=25)
    mv, ms = mf.Mesh.from_problem(pv), mf.Mesh.from_problem(ps)
    x = gpu(pv.x(3)).view(-1, 3)
    yv = mv.apply(x.reshape(-1)).view(-1, 3)
    for k in range(3):
        ys = ms.apply(x[:, k].contiguous())
        torch.cuda.synchronize()
        assert rel2(yv[:, k].cpu().numpy(), ys.cpu().numpy()) <= TOL64


@pytest.mark.parametrize("structured", [True, False])
def test_vector_laplace_csr_block_diagonal(structured):
    p = inputs.vector_laplace_box(5, ny=4, nz=6, jitter=0.2, seed=26)
    mesh = mf.Mesh.from_problem(p, structured=structured)
    A = mesh.assemble_csr()
    G = A.to_scipy()
    R = fem.assemble_csr(p.physics, p.coords, p.cell_array(), p.mat, p.dirichlet, p.n_nodes)
    R.eliminate_zeros()
    assert np.array_equal(G.indptr, R.indptr) and np.array_equal(G.indices, R.indices)
    assert np.max(np.abs(G.data - R.data)) <= 1e-13 * np.max(np.abs(R.data))
    # block-diagonal: no row couples two components
    rows = np.repeat(np.arange(G.shape[0]), np.diff(G.indptr))
    assert np.all(rows % 3 == G.indices % 3)
    x = p.x()
    y = A.spmv(gpu(x))
    torch.cuda.synchronize()
    assert rel2(y.cpu().numpy(), oracle_apply(p, x)) <= TOL64


@pytest.mark.parametrize("nrhs", [1, 4, 5])
def test_vector_laplace_multi_rhs(nrhs):
    p = inputs.vector_laplace_box(11, ny=9, nz=13, graded=0.4, seed=27)
    mesh = mf.Mesh.from_problem(p)
    xs = [p.x(seed=s) for s in range(nrhs)]
    X = np.stack([x.reshape(-1, 3) for x in xs], axis=1).reshape(-1)
    Y = mesh.apply_multi(gpu(X), nrhs)
    torch.cuda.synchronize()
    Y = Y.cpu().numpy().reshape(p.n_nodes, nrhs, 3)
    for r in range(nrhs):
        assert rel2(Y[:, r, :].reshape(-1), oracle_apply(p, xs[r])) <= TOL64


def test_vector_laplace_cg_matches_oracle():
    p = inputs.vector_laplace_box(8, jitter=0.2, sigma=1.0, seed=28)
    A = fem.assemble_csr(p.physics, p.coords, p.cell_array(), p.mat, p.dirichlet, p.n_nodes)
    b = p.b()
    xo, it_o, _ = solvers.cg(lambda v: A @ v, b, rtol=1e-8)
    mesh = mf.Mesh.from_problem(p)
    x, info = mesh.cg(gpu(b))
    torch.cuda.synchronize()
    assert info.status == mf.MF_OK
    assert abs(info.iters - it_o) <= max(2, math.ceil(0.01 * it_o)), (info.iters, it_o)
    assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 1.05e-8 * np.linalg.norm(b)


def test_vector_laplace_entry_point_checks_physics():
    p = inputs.vector_laplace_box(3, seed=29)
    mesh = mf.Mesh.from_problem(p)
    x = gpu(p.x())
    y = torch.empty_like(x)
    with pytest.raises(mf.MfError):
        mf.mf_apply_elasticity(mesh.h, x, y)
    with pytest.raises(mf.MfError):
        mf.mf_apply_laplace(mesh.h, x, y)
    mf.mf_apply_vector_laplace(mesh.h, x, y)
