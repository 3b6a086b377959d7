"""Degenerate cases of the operators and the solver on the GPU: a mesh whose every node is
constrained (A is the identity), zero inputs, a zero right-hand side, and the null spaces of the
unconstrained operators (constants for Laplace, the six rigid-body modes for elasticity), on every
apply variant."""
import dataclasses

import numpy as np
import pytest

from paper_2308_09839_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

from paper_2308_09839_gb300 import mf  # noqa: E402

VARIANTS = (mf.MF_VARIANT_AUTO, mf.MF_VARIANT_REFERENCE, mf.MF_VARIANT_GENERAL, mf.MF_VARIANT_PARTIAL)


def boxes(physics, constrained):
    """A tensor-product box (face-marching kernel) and a jittered one (general and partial-assembly
    kernels), with every node constrained (constrained=True) or none."""
    make = {"laplace": inputs.laplace_box, "elasticity": inputs.elasticity_box,
            "vector_laplace": inputs.vector_laplace_box}[physics]
    out = []
    for jitter in (0.0, 0.2):
        p = make(5, ny=4, nz=6, jitter=jitter, seed=31)
        d = np.ones_like(p.dirichlet) if constrained else np.zeros_like(p.dirichlet)
        out.append(dataclasses.replace(p, dirichlet=d))
    return out


def variants_of(p):
    return VARIANTS if p.meta.get("jitter", 0.0) or not np.allclose(p.coords, inputs.box_coords(p.nx, p.ny, p.nz)) \
        else (mf.MF_VARIANT_AUTO, mf.MF_VARIANT_REFERENCE)


@pytest.mark.parametrize("physics", ["laplace", "elasticity", "vector_laplace"])
def test_all_constrained_mesh_is_the_identity(physics):
    for p in boxes(physics, constrained=True):
        m = mf.Mesh.from_problem(p)
        x = torch.from_numpy(p.x()).cuda()
        for v in variants_of(p):
            m.set_variant(v)
            y = m.apply(x)
            torch.cuda.synchronize()
            assert torch.equal(y, x), (physics, v)
        m.set_variant(mf.MF_VARIANT_AUTO)
        A = m.assemble_csr()
        assert torch.equal(A.spmv(x), x)
        b = torch.from_numpy(p.x(5)).cuda()
        xs, info = m.cg(b)
        assert info.status == mf.MF_OK and info.iters <= 1
        assert torch.allclose(xs, b, rtol=0, atol=1e-15 * float(b.abs().max()))


@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
def test_zero_input_gives_zero_and_zero_rhs_gives_zero_solution(physics):
    make = inputs.laplace_box if physics == "laplace" else inputs.elasticity_box
    for jitter in (0.0, 0.2):
        p = make(6, ny=5, nz=4, jitter=jitter, seed=32)
        m = mf.Mesh.from_problem(p)
        x = torch.zeros(p.n_dof, dtype=torch.float64, device="cuda")
        for v in variants_of(p):
            m.set_variant(v)
            y = m.apply(x)
            torch.cuda.synchronize()
            assert float(y.abs().max()) == 0.0, (physics, jitter, v)
        m.set_variant(mf.MF_VARIANT_AUTO)
        xs, info = m.cg(x.clone())
        assert info.status == mf.MF_OK and info.iters == 0
        assert float(xs.abs().max()) == 0.0


def test_null_spaces_of_the_unconstrained_operators():
    """Without constraints A 1 = 0 (Laplace) and A r = 0 for the rigid-body modes r (elasticity), to
    the rounding of the element sums: |A r| <= 1e-12 |A| |r| on every variant."""
    for physics in ("laplace", "elasticity"):
        for p in boxes(physics, constrained=False):
            m = mf.Mesh.from_problem(p)
            X = p.coords
            if physics == "laplace":
                modes = [np.ones(p.n_nodes)]
            else:
                c = X - X.mean(axis=0)
                e = np.eye(3)
                modes = [np.tile(e[k], (p.n_nodes, 1)).reshape(-1) for k in range(3)]
                for k in range(3):  # rotations about axis k: r = e_k x (X - c)
                    modes.append(np.cross(np.tile(e[k], (p.n_nodes, 1)), c).reshape(-1))
            scale = np.abs(m.apply(torch.from_numpy(p.x()).cuda()).cpu().numpy()).max() / np.abs(p.x()).max()
            for v in variants_of(p):
                m.set_variant(v)
                for r in modes:
                    y = m.apply(torch.from_numpy(np.ascontiguousarray(r)).cuda()).cpu().numpy()
                    assert np.abs(y).max() <= 1e-12 * scale * np.abs(r).max() * 27, (physics, v)
