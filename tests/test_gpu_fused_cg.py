"""Classic CG with the vector updates fused into the face-marching apply (MF_CG_CLASSIC on scalar
Laplace tensor-product meshes) against the same recurrence with separate vector kernels
(MF_CG_CLASSIC_SPLIT): the fused kernels evaluate the same FP64 formulas (p = z + beta p,
x += alpha p, Table 4) on the same values and sum p.Ap over the same CTAs, so iteration counts,
residual records and solutions are bitwise equal.  Covered: Laplace with and without Jacobi (and
the vector Laplace and elasticity meshes, where MF_CG_CLASSIC takes the separate kernels), graphs
with odd and even block lengths and plain launches, several z-segments, the not-converged and
breakdown exits, right-hand sides outside the double-word window (the range fix-up kernel reads p
back from the fused kernel's output), and the oracle's CG.  The fused path's launches are counted
(2 kernels and the fix-up per iteration against 3 and the fix-up)."""
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

ANY = (mf.MF_OK, mf.MF_NOT_CONVERGED, mf.MF_ERR_BREAKDOWN, mf.MF_ERR_TIMEOUT)

CASES = {
    "laplace": lambda: inputs.laplace_box(37, ny=19, nz=23, graded=0.4, seed=81),
    "laplace_segments": lambda: inputs.laplace_box(40, ny=33, nz=70, graded=0.2, seed=82),
    "vector_laplace": lambda: inputs.vector_laplace_box(14, ny=11, nz=9, graded=0.3, seed=83),
    "elasticity": lambda: inputs.elasticity_box(33, ny=14, nz=12, graded=0.3, seed=84),
}


def _pair(mesh, b, **kw):
    x1, i1 = mesh.cg(b, ok=ANY, **kw)
    x1 = x1.clone()
    x2, i2 = mesh.cg(b, ok=ANY, recurrence=mf.MF_CG_CLASSIC_SPLIT, **kw)
    torch.cuda.synchronize()
    return (x1, i1), (x2, i2)


def _assert_same(a, b):
    (x1, i1), (x2, i2) = a, b
    assert (i1.status, i1.iters) == (i2.status, i2.iters)
    assert i1.rel_res == i2.rel_res and i1.rel_res_true == i2.rel_res_true
    assert torch.equal(x1, x2)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("jacobi", [False, True])
def test_fused_classic_cg_bitwise_equals_split_kernels(name, jacobi):
    p = CASES[name]()
    mesh = mf.Mesh.from_problem(p)
    assert mesh.info["tensor_product"]
    b = torch.from_numpy(p.b()).cuda()
    pc = mf.MF_PC_JACOBI if jacobi else mf.MF_PC_NONE
    a, s = _pair(mesh, b, precond=pc)
    assert a[1].status == mf.MF_OK and a[1].iters > 10
    _assert_same(a, s)


@pytest.mark.parametrize("use_graph,check_every", [(1, 7), (1, 16), (0, 5), (1, 1)])
def test_fused_cg_graph_blocks_and_plain_launches(use_graph, check_every):
    p = CASES["laplace"]()
    mesh = mf.Mesh.from_problem(p)
    b = torch.from_numpy(p.b()).cuda()
    a, s = _pair(mesh, b, use_graph=use_graph, check_every=check_every)
    _assert_same(a, s)
    # and the same as the default graph block length
    x3, i3 = mesh.cg(b)
    assert i3.iters == a[1].iters and torch.equal(x3, a[0])


@pytest.mark.parametrize("max_iter", [1, 2, 3, 8, 9])
def test_fused_cg_not_converged_keeps_the_last_update(max_iter):
    # the last iteration's x += alpha p is owed by the fused apply that never runs: the end of the solve
    # adds it (odd and even final iterations use different p buffers)
    p = CASES["laplace"]()
    mesh = mf.Mesh.from_problem(p)
    b = torch.from_numpy(p.b()).cuda()
    a, s = _pair(mesh, b, max_iter=max_iter, check_every=4)
    assert a[1].status == mf.MF_NOT_CONVERGED and a[1].iters == max_iter
    _assert_same(a, s)


def test_fused_cg_breakdown_and_zero_rhs():
    p = CASES["laplace"]()
    mesh = mf.Mesh.from_problem(p)
    bn = p.b()
    bn[17] = np.nan
    a, s = _pair(mesh, torch.from_numpy(bn).cuda())
    assert a[1].status == mf.MF_ERR_BREAKDOWN
    assert (a[1].status, a[1].iters) == (s[1].status, s[1].iters)
    z = torch.zeros(p.n_dof, dtype=torch.float64, device="cuda")
    a, s = _pair(mesh, z)
    assert a[1].status == mf.MF_OK and a[1].iters == 0
    _assert_same(a, s)
    assert not torch.any(a[0])


@pytest.mark.parametrize("shift", [-480, 400])
def test_fused_cg_right_hand_side_outside_the_double_word_window(shift):
    p = CASES["laplace"]()
    mesh = mf.Mesh.from_problem(p)
    b = torch.from_numpy(np.ldexp(p.b(), shift)).cuda()
    a, s = _pair(mesh, b)
    assert a[1].status == mf.MF_OK
    _assert_same(a, s)
    # CG is invariant under b -> 2^s b (exact scaling): the iterates are those of the unscaled solve
    x0, i0 = mesh.cg(torch.from_numpy(p.b()).cuda())
    assert abs(a[1].iters - i0.iters) <= max(3, math.ceil(0.03 * i0.iters))


@pytest.mark.parametrize("name", ["laplace", "elasticity"])
def test_fused_cg_matches_oracle(name):
    p = CASES[name]()
    A = fem.assemble_csr(p.physics, p.coords, p.cell_array(), p.mat, p.dirichlet, p.n_nodes)
    b = p.b()
    xo, it_o, _ = solvers.cg(lambda v: A @ v, b, rtol=1e-8)
    mesh = mf.Mesh.from_problem(p)
    x, info = mesh.cg(torch.from_numpy(b).cuda())
    x = x.cpu().numpy()
    assert info.status == mf.MF_OK
    assert abs(info.iters - it_o) <= max(1, math.ceil(0.01 * it_o)), (info.iters, it_o)
    assert np.linalg.norm(b - A @ x) <= 1.05e-8 * np.linalg.norm(b)
    assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)


def test_fused_cg_launch_counts():
    """Per iteration the fused path launches the apply, its range fix-up and the r update (3 kernels);
    the separate kernels launch the apply with the dot, the fix-up, the x/r and the p update (4); the
    fused solve adds one kernel at the end (the last x update).  On elasticity MF_CG_CLASSIC is the
    separate kernels."""
    n_it = 16
    for name, fused in (("laplace", True), ("elasticity", False)):
        p = CASES[name]()
        mesh = mf.Mesh.from_problem(p)
        b = torch.from_numpy(p.b()).cuda()
        counts = []
        for rec in (mf.MF_CG_CLASSIC, mf.MF_CG_CLASSIC_SPLIT):
            mesh.cg(b, ok=ANY, max_iter=n_it, check_every=n_it, recurrence=rec)  # graph capture
            torch.cuda.synchronize()
            c0 = mf.mf_kernel_launches()
            mesh.cg(b, ok=ANY, max_iter=n_it, check_every=n_it, recurrence=rec)
            torch.cuda.synchronize()
            counts.append(mf.mf_kernel_launches() - c0)
        assert counts[1] - counts[0] == ((n_it - 1) if fused else 0), (name, counts)
