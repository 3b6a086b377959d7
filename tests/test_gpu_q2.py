"""Q2 (27-node) hexahedra, the higher-order elements of Sec. 7's future work, through the C ABI
against the CPU oracle: apply in FP64 (<= 1e-12 relative 2-norm) and FP32 on straight-edged and
curved meshes, multi-RHS, CSR pattern and values, operator diagonal, CG and Jacobi-PCG, and the checks
of the setup call."""
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
    "laplace_jitter_3x4x2": lambda: inputs.q2_box("laplace", 3, ny=4, nz=2, jitter=0.2, seed=81, sigma=1.0),
    "laplace_curved_3x3x3": lambda: inputs.q2_box("laplace", 3, jitter=0.1, curve=0.08, seed=82, sigma=1.0),
    "laplace_1x1x1": lambda: inputs.q2_box("laplace", 1, seed=83),
    "elasticity_curved_2x3x2": lambda: inputs.q2_box("elasticity", 2, ny=3, nz=2, jitter=0.1, curve=0.06, seed=84),
    "vector_laplace_jitter_2x2x3": lambda: inputs.q2_box("vector_laplace", 2, ny=2, nz=3, jitter=0.15, seed=85),
}


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("variant", [mf.MF_VARIANT_AUTO, mf.MF_VARIANT_REFERENCE])
def test_q2_apply_matches_oracle(name, variant):
    """AUTO is the sum-factorised partial-assembly kernel (one thread per element for Laplace and
    vector Laplace, one warp per element for elasticity)."""
    p = MESHES[name]()
    mesh = mf.Mesh.from_problem(p)
    assert mesh.info["q2"] and not mesh.info["structured"]
    assert mesh.info["partial_assembly"]
    mesh.set_variant(variant)
    for seed in (0, 1):
        x = p.x(seed)
        y = mesh.apply(gpu(x))
        torch.cuda.synchronize()
        ref = oracle_apply(p, x)
        assert rel2(y.cpu().numpy(), ref) <= TOL64, (name, seed, rel2(y.cpu().numpy(), ref))
    y32 = mesh.apply(gpu(x).float())
    torch.cuda.synchronize()
    assert rel2(y32.double().cpu().numpy(), ref) < 2e-5


@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
def test_q2_partial_assembly_larger_mesh(physics):
    """10 x 9 x 11 curved Q2 mesh: the sum-factorised kernel against the oracle, and against the
    reference kernel of the same library."""
    p = inputs.q2_box(physics, 10, ny=9, nz=11, jitter=0.1, curve=0.05, seed=90, sigma=1.0)
    mesh = mf.Mesh.from_problem(p)
    x = p.x(3)
    y_pa = mesh.apply(gpu(x))
    mesh.set_variant(mf.MF_VARIANT_REFERENCE)
    y_ref = mesh.apply(gpu(x))
    torch.cuda.synchronize()
    ref = oracle_apply(p, x)
    assert rel2(y_pa.cpu().numpy(), ref) <= TOL64
    assert rel2(y_pa.cpu().numpy(), y_ref.cpu().numpy()) <= TOL64


@pytest.mark.parametrize("nrhs", [1, 4])
@pytest.mark.parametrize("physics", ["elasticity", "vector_laplace"])
def test_q2_multi_rhs(nrhs, physics):
    p = inputs.q2_box(physics, 2, ny=2, nz=3, jitter=0.1, seed=86)
    mesh = mf.Mesh.from_problem(p)
    xs = [p.x(seed=s) for s in range(nrhs)]
    X = np.stack([x.reshape(-1, 3) for x in xs], axis=1).reshape(-1)
    Y = mesh.apply_multi(gpu(X), nrhs)
    torch.cuda.synchronize()
    Y = Y.cpu().numpy().reshape(p.n_nodes, nrhs, 3)
    for r in range(nrhs):
        assert rel2(Y[:, r, :].reshape(-1), oracle_apply(p, xs[r])) <= TOL64


@pytest.mark.parametrize("physics", ["laplace", "elasticity", "vector_laplace"])
def test_q2_csr_and_diagonal(physics):
    p = inputs.q2_box(physics, 2, ny=3, nz=2, jitter=0.1, curve=0.05, seed=87)
    mesh = mf.Mesh.from_problem(p)
    A = mesh.assemble_csr()
    G = A.to_scipy()
    R = fem.assemble_csr(p.physics, p.coords, p.cells, p.mat, p.dirichlet, p.n_nodes)
    if physics == "vector_laplace":
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
def test_q2_cg_and_jacobi_match_oracle(physics):
    """Iteration counts within 5 % of the oracle's: the operators are the double-word partial-assembly
    kernels, and under double-word-sized rounding of its operator the oracle's own CG moves by more than
    1 % (Laplace) and 3 % (elasticity) on these problems (test_q2_cg_counts_drift_under_double_word_
    rounding in the oracle pins)."""
    p = inputs.q2_box(physics, 3, ny=2, nz=3, jitter=0.1, seed=88)
    frac = 0.05
    A = fem.assemble_csr(p.physics, p.coords, p.cells, p.mat, p.dirichlet, p.n_nodes)
    b = p.b()
    _, it_o, _ = solvers.cg(lambda v: A @ v, b, rtol=1e-8)
    dg = fem.diagonal(p.physics, p.coords, p.cells, p.mat, p.dirichlet, p.n_nodes)
    _, it_j, _ = solvers.pcg(lambda v: A @ v, b, lambda r: r / dg, rtol=1e-8)
    mesh = mf.Mesh.from_problem(p)
    x, info = mesh.cg(gpu(b))
    torch.cuda.synchronize()
    assert info.status == mf.MF_OK
    assert abs(info.iters - it_o) <= max(2, math.ceil(frac * it_o)), (info.iters, it_o)
    assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 1.05e-8 * np.linalg.norm(b)
    _, ij = mesh.cg(gpu(b), precond=mf.MF_PC_JACOBI)
    assert ij.status == mf.MF_OK
    assert abs(ij.iters - it_j) <= max(2, math.ceil(frac * it_j)), (ij.iters, it_j)


def test_q2_setup_checks():
    p = inputs.q2_box("laplace", 2, seed=89)
    coords, mat, dirichlet = gpu(p.coords), gpu(p.mat), gpu(p.dirichlet)
    bad = p.cells.copy()
    bad[1] = bad[1].reshape(3, 3, 3)[:, :, ::-1].reshape(-1)  # mirrored in x: det J < 0
    with pytest.raises(mf.MfError):
        mf.Mesh("laplace", coords, mat, dirichlet, gpu(bad), element="hex27")
    assert "det" in mf.mf_last_error()
    mesh = mf.Mesh.from_problem(p)
    with pytest.raises(mf.MfError):
        mesh.set_variant(mf.MF_VARIANT_GENERAL)
    mesh.set_variant(mf.MF_VARIANT_PARTIAL)  # Laplace: the sum-factorised partial assembly
    pe = inputs.q2_box("elasticity", 1, seed=89)
    me = mf.Mesh.from_problem(pe)
    assert me.info["partial_assembly"]
    me.set_variant(mf.MF_VARIANT_PARTIAL)  # elasticity: the warp-per-element partial assembly
    with pytest.raises(mf.MfError):
        me.set_variant(mf.MF_VARIANT_GENERAL)
