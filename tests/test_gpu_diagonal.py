"""diag(A) through the C ABI (mf_operator_diagonal, the Jacobi preconditioner of Sec. 5) against the
oracle's diagonal of the assembled element matrices (Eqs. 4/5/6), and the reuse of that diagonal
across solves on one mesh.  FP64 agreement <= 1e-13 relative (per entry, against max |diag|)."""
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

PROBLEMS = {
    "laplace_jitter_7x5x6": lambda: inputs.laplace_box(7, ny=5, nz=6, jitter=0.25, seed=41),
    "laplace_graded_1x3x2": lambda: inputs.laplace_box(1, ny=3, nz=2, graded=0.5, seed=42),
    "elasticity_jitter_5x6x4": lambda: inputs.elasticity_box(5, ny=6, nz=4, jitter=0.2, seed=43),
    "vector_laplace_jitter_4x4x5": lambda: inputs.vector_laplace_box(4, ny=4, nz=5, jitter=0.2, seed=44),
}


@pytest.mark.parametrize("name", sorted(PROBLEMS))
@pytest.mark.parametrize("structured", [True, False])
def test_operator_diagonal_matches_oracle(name, structured):
    p = PROBLEMS[name]()
    mesh = mf.Mesh.from_problem(p, structured=structured)
    d = torch.full((p.n_dof,), float("nan"), dtype=torch.float64, device="cuda")
    mf.mf_operator_diagonal(mesh, d)
    torch.cuda.synchronize()
    ref = fem.diagonal(p.physics, p.coords, p.cell_array(), p.mat, p.dirichlet, p.n_nodes)
    got = d.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    # Dirichlet rows of the constrained operator are identity rows
    assert np.all(got[p.dirichlet_dofs()] == 1.0)


def test_jacobi_diagonal_is_reused_across_solves():
    """The first Jacobi solve computes 1/diag(A); later solves on the same mesh (Jacobi-PCG and the
    flexible CG's smoother) reuse it: repeated solves are bitwise identical and keep matching the
    oracle's PCG."""
    p = inputs.laplace_box(9, ny=7, nz=8, jitter=0.2, seed=45)
    A = fem.assemble_csr(p.physics, p.coords, p.cell_array(), p.mat, p.dirichlet, p.n_nodes)
    dg = fem.diagonal(p.physics, p.coords, p.cell_array(), p.mat, p.dirichlet, p.n_nodes)
    b = p.b()
    _, it_o, _ = solvers.pcg(lambda v: A @ v, b, lambda r: r / dg, rtol=1e-8)
    mesh = mf.Mesh.from_problem(p)
    bb = torch.from_numpy(b).cuda()
    x1, i1 = mesh.cg(bb, precond=mf.MF_PC_JACOBI)
    x1 = x1.clone()
    mesh.cg(bb)  # an unpreconditioned solve in between
    x2, i2 = mesh.cg(bb, precond=mf.MF_PC_JACOBI)
    assert i1.status == mf.MF_OK and i2.status == mf.MF_OK
    assert i1.iters == i2.iters
    assert torch.equal(x1, x2)
    assert abs(i1.iters - it_o) <= max(2, math.ceil(0.01 * it_o)), (i1.iters, it_o)
