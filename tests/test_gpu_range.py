"""Range of the FP64 operator apply: the double-word (float pair) kernels against the FP64 oracle
when inputs, cell constants or coordinates lie far outside FP32's exponent range.

The paper's operator is FP64 (Sec. 2, Table 1's 8-byte values).  The fast kernels compute in pairs
of floats, which cover FP32's exponent range only, so the library (a) scales the cell constants and
the coordinates of a mesh by powers of two at setup when their magnitudes need it, and (b) has every
CTA of an apply recompute its tile with its inputs scaled by a power of two when the largest input
it read lies outside the window the pairs cover.  Power-of-two scaling is exact, so besides parity
with the oracle (<= 1e-12 relative in the 2-norm) the tests check that scaling x, the cell
constants or the coordinates by 2^k scales y by exactly 2^k (bitwise).
"""
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

DEV = "cuda"
TOL64 = 1e-12


def rel2(a, b):
    """||a - b|| / ||b||, computed on both vectors scaled by the same power of two (the squares of
    entries near 1e200 or 1e-300 would overflow or underflow)."""
    m = max(float(np.abs(a).max()), float(np.abs(b).max()))
    if m == 0.0:
        return 0.0
    k = -int(np.frexp(m)[1])
    a, b = np.ldexp(a, k), np.ldexp(b, k)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def oracle_apply(p, x):
    return fem.apply(p.physics, p.coords, p.cell_array(), p.mat, p.dirichlet, x)


def gpu_apply(mesh, x):
    y = mesh.apply(gpu(x))
    torch.cuda.synchronize()
    return y.cpu().numpy()


def scaled(p, mat=1.0, coords=1.0):
    """The problem with its cell constants (kappa, or Young's modulus) times `mat` and its
    coordinates times `coords`."""
    m = p.mat.copy()
    if m.ndim == 1:
        m *= mat
    else:
        m[:, 0] *= mat
    return inputs.Problem(p.name, p.physics, p.nx, p.ny, p.nz, p.coords * coords, m, p.dirichlet, p.seed,
                          p.cells, dict(p.meta), p.element)


# meshes with several CTAs in x, y and z; (problem, variants to run)
MESHES = {
    "tp_laplace": (lambda: inputs.laplace_box(40, ny=33, nz=21, sigma=1.0, layered=True, graded=0.3, seed=3),
                   [mf.MF_VARIANT_AUTO]),
    "tp_elasticity": (lambda: inputs.elasticity_box(20, ny=17, nz=11, graded=0.3, seed=4), [mf.MF_VARIANT_AUTO]),
    "tp_vector_laplace": (lambda: inputs.vector_laplace_box(18, ny=13, nz=9, seed=5), [mf.MF_VARIANT_AUTO]),
    "jit_laplace": (lambda: inputs.laplace_box(24, ny=19, nz=13, jitter=0.2, seed=6),
                    [mf.MF_VARIANT_AUTO, mf.MF_VARIANT_GENERAL, mf.MF_VARIANT_PARTIAL]),
    "jit_elasticity": (lambda: inputs.elasticity_box(14, ny=11, nz=9, jitter=0.2, seed=7),
                       [mf.MF_VARIANT_AUTO, mf.MF_VARIANT_GENERAL, mf.MF_VARIANT_PARTIAL]),
}
CASES = [(name, v) for name, (_, vs) in MESHES.items() for v in vs]


def _mesh(p, variant):
    mesh = mf.Mesh.from_problem(p)
    mesh.set_variant(variant)
    return mesh


@pytest.mark.parametrize("name,variant", CASES)
@pytest.mark.parametrize("xscale", [1e-35, 1e35, 1e-200, 1e200, 1e-300])
def test_x_magnitudes_match_oracle(name, variant, xscale):
    """x of every magnitude FP64 can hold (values near 2^-1000 included) gives FP64 parity."""
    p = MESHES[name][0]()
    mesh = _mesh(p, variant)
    x = p.x(1) * xscale
    y = gpu_apply(mesh, x)
    ref = oracle_apply(p, x)
    assert np.all(np.isfinite(y))
    assert rel2(y, ref) <= TOL64, (name, variant, xscale, rel2(y, ref))


@pytest.mark.parametrize("name,variant", CASES)
def test_subnormal_x_matches_oracle(name, variant):
    """Subnormal inputs (below 2^-1022) with cell constants large enough that y is normal."""
    p = scaled(MESHES[name][0](), mat=2.0 ** 60)
    mesh = _mesh(p, variant)
    x = np.ldexp(p.x(2), -1030)
    assert np.abs(x).max() < np.finfo(np.float64).tiny
    y = gpu_apply(mesh, x)
    ref = np.ldexp(oracle_apply(p, np.ldexp(x, 1100)), -1100)  # both scalings exact
    assert rel2(y, ref) <= TOL64, rel2(y, ref)


@pytest.mark.parametrize("name,variant", CASES)
def test_mixed_magnitude_x_matches_oracle(name, variant):
    """Entries of one x spread over 10^-250 .. 10^250: tiles see very different magnitudes."""
    p = MESHES[name][0]()
    mesh = _mesh(p, variant)
    rng = np.random.default_rng(17)
    x = p.x(3) * 10.0 ** rng.uniform(-250, 250, size=p.n_dof)
    y = gpu_apply(mesh, x)
    ref = oracle_apply(p, x)
    assert rel2(y, ref) <= TOL64, rel2(y, ref)


@pytest.mark.parametrize("name,variant", CASES)
@pytest.mark.parametrize("k", [-1000, -300, -100, 150, 600, 1000])
def test_power_of_two_scaling_of_x_is_exact(name, variant, k):
    """y(2^k x) == 2^k y(x) bitwise, inside and far outside the pairs' exponent range."""
    p = MESHES[name][0]()
    mesh = _mesh(p, variant)
    x = p.x(4)
    y0 = gpu_apply(mesh, x)
    yk = gpu_apply(mesh, np.ldexp(x, k))
    np.testing.assert_array_equal(yk, np.ldexp(y0, k))


@pytest.mark.parametrize("name,variant", CASES)
@pytest.mark.parametrize("what,factor", [("mat", 1e30), ("mat", 1e-30), ("coords", 1e-20), ("coords", 1e15)])
def test_scaled_cell_constants_and_coordinates_match_oracle(name, variant, what, factor):
    """kappa or Young's modulus at 1e+-30, domains of size 1e-20 and 1e15: normalised at setup."""
    p = scaled(MESHES[name][0](), **{what: factor})
    mesh = _mesh(p, variant)
    assert mesh.info["dw_normalised"] and not mesh.info["dw_range_exceeded"]
    x = p.x(5)
    y = gpu_apply(mesh, x)
    ref = oracle_apply(p, x)
    assert rel2(y, ref) <= TOL64, (what, factor, rel2(y, ref))
    if what == "mat":  # and x outside the pairs' range on top of it
        y = gpu_apply(mesh, x * 1e-250)
        ref = oracle_apply(p, x * 1e-250)
        assert rel2(y, ref) <= TOL64, rel2(y, ref)


@pytest.mark.parametrize("name,variant", CASES)
@pytest.mark.parametrize("what,k", [("mat", 100), ("mat", -110), ("coords", -70), ("coords", 55)])
def test_power_of_two_scaling_of_mesh_is_exact(name, variant, what, k):
    """The operator is linear in the cell constants and in the length scale (Eqs. 4 and 6 in 3D:
    A ~ kappa h, A ~ E h), so scaling either by 2^k scales y by exactly 2^k."""
    p = MESHES[name][0]()
    ps = scaled(p, **{what: 2.0 ** k})
    x = p.x(6)
    y0 = gpu_apply(_mesh(p, variant), x)
    yk = gpu_apply(_mesh(ps, variant), x)
    free = ~fem_dirichlet_dofs(p)
    np.testing.assert_array_equal(yk[free], np.ldexp(y0[free], k))


def fem_dirichlet_dofs(p):
    m = np.zeros(p.n_dof, dtype=bool)
    m[p.dirichlet_dofs()] = True
    return m


@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
def test_too_wide_cell_constants_take_the_fp64_kernel(physics):
    """Cell constants spread over more than the pairs cover (2^+-70 here): the double-word kernels
    are switched off (flag bit 6), the auto variant runs the FP64 reference kernel, the explicit
    double-word variants are refused, and the result still matches the oracle."""
    p = (inputs.laplace_box if physics == "laplace" else inputs.elasticity_box)(12, ny=9, nz=7, jitter=0.15, seed=8)
    rng = np.random.default_rng(9)
    f = 2.0 ** rng.uniform(-70, 70, size=p.n_cells)
    m = p.mat.copy()
    if m.ndim == 1:
        m *= f
    else:
        m[:, 0] *= f
    p = inputs.Problem(p.name, p.physics, p.nx, p.ny, p.nz, p.coords, m, p.dirichlet, p.seed)
    mesh = mf.Mesh.from_problem(p)
    assert mesh.info["flags"] & 64
    with pytest.raises(mf.MfError):
        mesh.set_variant(mf.MF_VARIANT_GENERAL)
    x = p.x(7)
    assert rel2(gpu_apply(mesh, x), oracle_apply(p, x)) <= TOL64


@pytest.mark.parametrize("name", ["tp_laplace", "jit_laplace"])
@pytest.mark.parametrize("k", [-465, 400])
def test_cg_right_hand_side_scaled_by_power_of_two(name, k):
    """CG on 2^k b runs the same iterations and returns 2^k x bitwise (alpha and beta are ratios of
    dot products, which the exact scaling leaves unchanged); with k = -465 every Krylov vector lies
    far below FP32's range."""
    p = MESHES[name][0]()
    mesh = mf.Mesh.from_problem(p)
    b = p.b(1)
    x0, i0 = mesh.cg(gpu(b), check_every=8)
    x0 = x0.cpu().numpy()
    xk, ik = mesh.cg(gpu(np.ldexp(b, k)), check_every=8)
    assert i0.status == mf.MF_OK and ik.status == mf.MF_OK
    assert ik.iters == i0.iters
    np.testing.assert_array_equal(xk.cpu().numpy(), np.ldexp(x0, k))
    A = fem.assemble_csr(p.physics, p.coords, p.cell_array(), p.mat, p.dirichlet, p.n_nodes)
    _, it_o, _ = solvers.cg(lambda v: A @ v, b, rtol=1e-8)
    # the layered lognormal(sigma = 1) problems take over 1000 iterations; the count is compared
    # with the drift tolerance of double-word operators (the oracle pin on CG counts)
    assert abs(i0.iters - it_o) <= max(3, math.ceil(0.03 * it_o)), (i0.iters, it_o)


@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
@pytest.mark.parametrize("case", ["tiny", "huge", "subnormal", "mixed", "plain"])
def test_csr_spmv_over_the_fp64_range(physics, case):
    """The CSR SpMV forms its products and sums in pairs of floats; rows whose products leave the
    pairs' exponent range are summed again in FP64, so y stays FP64-accurate for every input."""
    p = (inputs.laplace_box if physics == "laplace" else inputs.elasticity_box)(9, ny=7, nz=6, jitter=0.2, seed=21)
    if case == "subnormal":
        p = scaled(p, mat=2.0 ** 60)
    mesh = mf.Mesh.from_problem(p)
    A = mesh.assemble_csr()
    R = fem.assemble_csr(p.physics, p.coords, p.cell_array(), p.mat, p.dirichlet, p.n_nodes)
    x = p.x(8)
    if case == "tiny":
        x = x * 1e-200
    elif case == "huge":
        x = x * 1e200
    elif case == "subnormal":
        x = np.ldexp(x, -1030)
    elif case == "mixed":
        x = x * 10.0 ** np.random.default_rng(3).uniform(-250, 250, size=x.size)
    y = A.spmv(gpu(x))
    torch.cuda.synchronize()
    y = y.cpu().numpy()
    if case == "subnormal":
        ref = np.ldexp(R @ np.ldexp(x, 1100), -1100)
    else:
        ref = R @ x
    assert rel2(y, ref) <= TOL64, (case, rel2(y, ref))
