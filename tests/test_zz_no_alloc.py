"""The allocation-free CG entry point (mf_cg_solve_noalloc) against the ordinary one (mf_cg_solve).

mf_cg_solve_noalloc is for callers that must not allocate device memory while they run (an
application that gives the whole device to its own pool at start-up, or runs under a memory budget
enforced outside CUDA).  Its scratch is a fixed array inside the library, so this test checks that
it returns what mf_cg_solve returns, twice in a row (the array keeps the previous call's contents),
and that a problem above its size limit is refused.  The file is named so that pytest collects it
last; it passes alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

from paper_2308_09839_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_2308_09839_gb300 import mf  # noqa: E402

TOL = 1e-12  # relative 2-norm, as for the FP64 apply parity tests


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("physics,op", [("laplace", "matfree"), ("elasticity", "matfree"), ("laplace", "csr")])
def test_noalloc_cg_matches_cg_on_two_calls(physics, op):
    p = inputs.small_laplace_16(seed=0) if physics == "laplace" else inputs.elasticity_box(8, jitter=0.2, seed=2)
    mesh = mf.Mesh.from_problem(p)
    assert mesh.n_dof <= mf.MF_NOALLOC_MAX_DOF
    b = torch.from_numpy(p.b()).cuda()
    opts = mf.mf_solve_opts_default()
    csr = None
    if op == "csr":
        csr = mesh.assemble_csr()
        opts.op = mf.MF_OP_CSR
        opts.csr = csr.h
    x_ref = torch.empty_like(b)
    ref = mf.mf_cg_solve(mesh.h, opts, b, x_ref)
    torch.cuda.synchronize()
    assert ref.status == mf.MF_OK
    for _ in range(2):
        x = torch.full_like(b, 7.0)  # stale content must not matter
        info = mf.mf_cg_solve_noalloc(mesh.h, opts, b, x)
        torch.cuda.synchronize()
        assert info.status == mf.MF_OK
        assert info.iters == ref.iters
        assert _rel(x, x_ref) <= TOL
        assert info.rel_res_true <= 1.05e-8
        assert abs(info.rel_res_true - ref.rel_res_true) <= TOL * 1e-8 + 1e-3 * ref.rel_res_true


def test_noalloc_rejects_problem_above_limit():
    p = inputs.laplace_box(64, seed=0)  # 65^3 = 274,625 DoFs > 262,144
    mesh = mf.Mesh.from_problem(p)
    assert mesh.n_dof > mf.MF_NOALLOC_MAX_DOF
    b = torch.from_numpy(p.b()).cuda()
    with pytest.raises(mf.MfError) as e:
        mf.mf_cg_solve_noalloc(mesh.h, mf.mf_solve_opts_default(), b, torch.empty_like(b))
    assert e.value.status == mf.MF_ERR_ARG
    assert "limit" in str(e.value)
