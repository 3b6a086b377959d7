"""CG checkpoint and resume through the C ABI: a solve stopped by its iteration limit or its wall-clock
budget, saved to host memory and resumed (on the same mesh, after other solves, or on a new mesh
object built from the same problem), gives bitwise the iterations, residual record and solution of
the solve that was never interrupted; for the fused classic iteration, the split kernels, Jacobi,
the general structured kernel and CSR; plus the argument checks."""
import numpy as np
import pytest

from paper_2308_09839_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_2308_09839_gb300 import mf  # noqa: E402

STOPPED = (mf.MF_OK, mf.MF_NOT_CONVERGED, mf.MF_ERR_TIMEOUT)

PROBLEMS = {
    "laplace_tensor": lambda: inputs.laplace_box(29, ny=17, nz=21, graded=0.3, seed=91),
    "elasticity_tensor": lambda: inputs.elasticity_box(17, ny=12, nz=14, graded=0.2, seed=92),
    "laplace_jittered": lambda: inputs.laplace_box(14, jitter=0.2, seed=93),
}


def _same(a, b):
    (x1, i1), (x2, i2) = a, b
    assert (i1.status, i1.iters) == (i2.status, i2.iters)
    assert i1.rel_res == i2.rel_res and i1.rel_res_true == i2.rel_res_true
    assert torch.equal(x1, x2)


@pytest.mark.parametrize("name", sorted(PROBLEMS))
@pytest.mark.parametrize("rec", [mf.MF_CG_CLASSIC, mf.MF_CG_CLASSIC_SPLIT])
@pytest.mark.parametrize("jacobi", [False, True])
@pytest.mark.parametrize("stop", [7, 12])
def test_resume_after_iteration_limit_is_bitwise(name, rec, jacobi, stop):
    p = PROBLEMS[name]()
    mesh = mf.Mesh.from_problem(p)
    b = torch.from_numpy(p.b()).cuda()
    kw = dict(recurrence=rec, precond=mf.MF_PC_JACOBI if jacobi else mf.MF_PC_NONE, check_every=5)
    xf, inf = mesh.cg(b, **kw)
    full = (xf.clone(), inf)
    assert inf.status == mf.MF_OK and inf.iters > stop
    _, ip = mesh.cg(b, max_iter=stop, **kw)
    assert ip.status == mf.MF_NOT_CONVERGED and ip.iters == stop
    state = mesh.cg_state()
    assert len(state) == mf.mf_cg_state_bytes(mesh.h)
    mesh.cg(torch.flip(b, [0]), **kw)  # the workspace is reused in between
    xr, ir = mesh.cg_resume(state, b, **kw)
    _same((xr, ir), full)


@pytest.mark.parametrize("rec", [mf.MF_CG_CLASSIC, mf.MF_CG_CLASSIC_SPLIT])
def test_resume_after_timeout_on_a_new_mesh_object(rec):
    p = PROBLEMS["laplace_tensor"]()
    b = torch.from_numpy(p.b()).cuda()
    kw = dict(recurrence=rec, check_every=3)
    mesh = mf.Mesh.from_problem(p)
    xf, inf = mesh.cg(b, **kw)
    full = (xf.clone(), inf)
    _, it = mesh.cg(b, timeout_s=1e-9, ok=STOPPED, **kw)
    assert it.status == mf.MF_ERR_TIMEOUT and 0 < it.iters < inf.iters
    state = mesh.cg_state()
    mesh.close()
    other = mf.Mesh.from_problem(p)
    xr, ir = other.cg_resume(state, b, **kw)
    _same((xr, ir), full)


def test_resume_through_csr():
    p = PROBLEMS["laplace_jittered"]()
    mesh = mf.Mesh.from_problem(p)
    csr = mesh.assemble_csr()
    b = torch.from_numpy(p.b()).cuda()
    xf, inf = mesh.cg(b, csr=csr)
    full = (xf.clone(), inf)
    mesh.cg(b, csr=csr, max_iter=9)
    state = mesh.cg_state()
    x = torch.empty_like(b)
    o = mf.mf_solve_opts_default()
    o.op = mf.MF_OP_CSR
    o.csr = csr.h
    ir = mf.mf_cg_resume(mesh.h, o, state, b, x)
    _same((x, ir), full)


def test_state_argument_checks():
    p = PROBLEMS["laplace_tensor"]()
    mesh = mf.Mesh.from_problem(p)
    b = torch.from_numpy(p.b()).cuda()
    mesh.cg(b)  # converged: nothing to resume
    with pytest.raises(mf.MfError):
        mesh.cg_state()
    mesh.cg(b, max_iter=4)
    state = mesh.cg_state()
    with pytest.raises(mf.MfError):  # another preconditioner
        mesh.cg_resume(state, b, precond=mf.MF_PC_JACOBI)
    with pytest.raises(mf.MfError):  # the fused iteration's state through the split kernels
        mesh.cg_resume(state, b, recurrence=mf.MF_CG_CLASSIC_SPLIT)
    with pytest.raises(mf.MfError):  # the pipelined recurrence keeps no state
        mesh.cg_resume(state, b, recurrence=mf.MF_CG_PIPELINED)
    bad = bytearray(state)
    bad[0] ^= 0xFF
    with pytest.raises(mf.MfError):
        mesh.cg_resume(bytes(bad), b)
    small = mf.Mesh.from_problem(inputs.laplace_box(5, seed=94))
    with pytest.raises(mf.MfError):  # another mesh size
        small.cg_resume(state, torch.zeros(small.n_dof, dtype=torch.float64, device="cuda"))
    with pytest.raises(mf.MfError):
        mesh.cg_resume(state[:100], b)
    mesh.cg(b, recurrence=mf.MF_CG_PIPELINED, max_iter=4)
    with pytest.raises(mf.MfError):  # a pipelined solve leaves no state
        mesh.cg_state()
    # the state of a stopped solve still resumes after the failed calls
    mesh.cg(b, max_iter=4)
    xr, ir = mesh.cg_resume(mesh.cg_state(), b)
    assert ir.status == mf.MF_OK and np.isfinite(ir.rel_res_true)
