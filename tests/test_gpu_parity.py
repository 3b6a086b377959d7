"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

Tolerance: FP64 results agree with the oracle to <= 1e-12 relative in the 2-norm (rounding order
differs only); FP32 results state their error.  Integer / structural results (CSR pattern) are
compared exactly.
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
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def oracle_apply(p, x, cells=None):
    return fem.apply(p.physics, p.coords, p.cell_array() if cells is None else cells, p.mat, p.dirichlet, x)


def gpu_apply(mesh, x):
    y = mesh.apply(gpu(x))
    torch.cuda.synchronize()
    return y.cpu().numpy()


PROBLEMS = {
    "laplace16_jitter": lambda: inputs.small_laplace_16(seed=0),
    "laplace_5x7x3": lambda: inputs.laplace_box(5, ny=7, nz=3, jitter=0.2, seed=1),
    "laplace_1x1x1": lambda: inputs.laplace_box(1, jitter=0.0, seed=2),
    "laplace_1x2x3": lambda: inputs.laplace_box(1, ny=2, nz=3, jitter=0.0, seed=3),
    "laplace_cartesian_layers": lambda: inputs.laplace_box(12, jitter=0.0, sigma=0.5, layered=True, seed=4),
    "elast8_jitter": lambda: inputs.elasticity_box(8, jitter=0.2, seed=5),
    "elast_cartesian_6x5x9": lambda: inputs.elasticity_box(6, ny=5, nz=9, jitter=0.0, seed=6),
    "elast_1x1x1": lambda: inputs.elasticity_box(1, jitter=0.0, seed=7),
}


@pytest.mark.parametrize("name", sorted(PROBLEMS))
@pytest.mark.parametrize("variant", [mf.MF_VARIANT_AUTO, mf.MF_VARIANT_REFERENCE])
@pytest.mark.parametrize("structured", [True, False])
def test_apply_fp64_matches_oracle(name, variant, structured):
    p = PROBLEMS[name]()
    mesh = mf.Mesh.from_problem(p, structured=structured)
    mesh.set_variant(variant)
    for seed in (0, 1):
        x = p.x(seed)
        y = gpu_apply(mesh, x)
        ref = oracle_apply(p, x)
        assert rel2(y, ref) <= TOL64, (name, seed, rel2(y, ref))


@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
def test_apply_renumbered_mesh(physics):
    """General connectivity: randomly permuted node and element numbering (greedy colouring)."""
    p = (inputs.laplace_box if physics == "laplace" else inputs.elasticity_box)(7, jitter=0.2, seed=11)
    c2, cl2, d2, nperm, eperm = inputs.renumber(p.coords, p.cell_array(), p.dirichlet, 3)
    mat2 = p.mat[eperm]
    nd = p.ndpn
    x = p.x()
    x2 = np.empty_like(x).reshape(-1, nd)
    x2[nperm] = x.reshape(-1, nd)
    x2 = x2.reshape(-1)
    mesh = mf.Mesh(physics, gpu(c2), gpu(mat2), gpu(d2), gpu(cl2))
    assert mesh.info["n_colours"] >= 8
    y = gpu_apply(mesh, x2)
    ref = fem.apply(physics, c2, cl2, mat2, d2, x2)
    assert rel2(y, ref) <= TOL64


def test_apply_dirichlet_entries_ignored_and_identity_rows():
    p = inputs.small_laplace_16(seed=2)
    mesh = mf.Mesh.from_problem(p)
    x = inputs.uniform_vector(p.n_dof, 5)  # nonzero on Dirichlet nodes
    y = gpu_apply(mesh, x)
    d = p.dirichlet.astype(bool)
    assert np.array_equal(y[d], x[d])
    assert rel2(y, oracle_apply(p, x)) <= TOL64


@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
def test_apply_bitwise_deterministic(physics):
    p = (inputs.laplace_box if physics == "laplace" else inputs.elasticity_box)(10, jitter=0.2, seed=8)
    mesh = mf.Mesh.from_problem(p)
    x = gpu(p.x())
    y1 = mesh.apply(x).clone()
    y2 = mesh.apply(x).clone()
    assert torch.equal(y1, y2)


@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
def test_apply_fp32_error_vs_oracle(physics):
    """FP32 geometry and arithmetic: error against the FP64 oracle stated and bounded."""
    p = (inputs.laplace_box if physics == "laplace" else inputs.elasticity_box)(10, jitter=0.2, seed=9)
    mesh = mf.Mesh.from_problem(p)
    x = p.x()
    y = mesh.apply(gpu(x).float())
    torch.cuda.synchronize()
    err = rel2(y.double().cpu().numpy(), oracle_apply(p, x))
    print(f"fp32 apply rel err {physics}: {err:.2e}")
    assert err < 1e-5


@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
@pytest.mark.parametrize("nrhs", [1, 3, 16])
def test_apply_multi_rhs(physics, nrhs):
    p = (inputs.laplace_box if physics == "laplace" else inputs.elasticity_box)(6, jitter=0.2, seed=10)
    mesh = mf.Mesh.from_problem(p)
    nd = p.ndpn
    xs = [p.x(seed=s) for s in range(nrhs)]
    X = np.stack([x.reshape(-1, nd) for x in xs], axis=1).reshape(-1)  # [node][rhs][k]
    Y = mesh.apply_multi(gpu(X), nrhs)
    torch.cuda.synchronize()
    Y = Y.cpu().numpy().reshape(p.n_nodes, nrhs, nd)
    for r in range(nrhs):
        assert rel2(Y[:, r, :].reshape(-1), oracle_apply(p, xs[r])) <= TOL64


@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
@pytest.mark.parametrize("structured", [True, False])
def test_csr_matches_oracle(physics, structured):
    p = (inputs.laplace_box if physics == "laplace" else inputs.elasticity_box)(5, ny=4, nz=6, jitter=0.2, seed=12)
    mesh = mf.Mesh.from_problem(p, structured=structured)
    A = mesh.assemble_csr()
    G = A.to_scipy()
    R = fem.assemble_csr(p.physics, p.coords, p.cell_array(), p.mat, p.dirichlet, p.n_nodes)
    # identical sparsity (structural, exact)
    assert np.array_equal(G.indptr, R.indptr) and np.array_equal(G.indices, R.indices)
    assert np.max(np.abs(G.data - R.data)) <= 1e-13 * np.max(np.abs(R.data))
    x = p.x()
    y = A.spmv(gpu(x))
    torch.cuda.synchronize()
    assert rel2(y.cpu().numpy(), R @ x) <= TOL64
    assert rel2(y.cpu().numpy(), oracle_apply(p, x)) <= TOL64


def _oracle_cg(p, rtol=1e-8):
    A = fem.assemble_csr(p.physics, p.coords, p.cell_array(), p.mat, p.dirichlet, p.n_nodes)
    b = p.b()
    x, it, _ = solvers.cg(lambda v: A @ v, b, rtol=rtol)
    return A, b, x, it


@pytest.mark.parametrize("op", ["matfree", "csr"])
def test_cg_small_laplace_matches_oracle(op):
    """16^3 jittered Laplace, lognormal(0,1) kappa: iterations within +-1 % (at least +-2) of the
    oracle's, true residual <= 1e-8, solution close to the oracle's."""
    p = inputs.small_laplace_16(seed=0)
    A, b, xo, it_o = _oracle_cg(p)
    mesh = mf.Mesh.from_problem(p)
    kw = {}
    if op == "csr":
        kw["csr"] = mesh.assemble_csr()
    x, info = mesh.cg(gpu(b), **kw)
    torch.cuda.synchronize()
    x = x.cpu().numpy()
    assert info.status == mf.MF_OK
    assert abs(info.iters - it_o) <= max(2, math.ceil(0.01 * it_o)), (info.iters, it_o)
    assert info.rel_res_true <= 1.05e-8
    assert np.linalg.norm(b - A @ x) <= 1.05e-8 * np.linalg.norm(b)
    assert rel2(x, xo) <= 1e-5


def test_cg_csr_graph_after_destroy_and_reassemble():
    """A CG graph captured for one assembled matrix must never be replayed for another.  Solve with a
    CSR, destroy it (its handle's host address may then be reused by the next one), fill the freed
    device memory with NaN through another allocation, assemble a new matrix and solve again: the
    second solve must use the new matrix and match the oracle."""
    p = inputs.small_laplace_16(seed=0)
    A, b, xo, it_o = _oracle_cg(p)
    mesh = mf.Mesh.from_problem(p)
    fillers = []
    for _ in range(3):
        csr = mesh.assemble_csr()
        x, info = mesh.cg(gpu(b), csr=csr, check_every=8)
        torch.cuda.synchronize()
        assert info.status == mf.MF_OK
        assert abs(info.iters - it_o) <= max(2, math.ceil(0.01 * it_o)), (info.iters, it_o)
        assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 1.05e-8 * np.linalg.norm(b)
        assert rel2(x.cpu().numpy(), xo) <= 1e-5
        nbytes = csr.info["nnz"] * 12 + (csr.info["n_rows"] + 1) * 8
        csr.close()
        fillers.append(torch.full((2 * nbytes // 8,), float("nan"), dtype=torch.float64, device=DEV))
        torch.cuda.synchronize()


def test_cg_elasticity_matches_oracle():
    p = inputs.elasticity_box(8, jitter=0.2, seed=13)
    A, b, xo, it_o = _oracle_cg(p)
    mesh = mf.Mesh.from_problem(p)
    x, info = mesh.cg(gpu(b))
    torch.cuda.synchronize()
    assert info.status == mf.MF_OK
    assert abs(info.iters - it_o) <= max(2, math.ceil(0.01 * it_o)), (info.iters, it_o)
    assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 1.05e-8 * np.linalg.norm(b)


def test_cg_graph_and_plain_launches_agree_bitwise():
    p = inputs.small_laplace_16(seed=1)
    mesh = mf.Mesh.from_problem(p)
    b = gpu(p.b())
    x1, i1 = mesh.cg(b, use_graph=1, check_every=16)
    x1 = x1.clone()
    x2, i2 = mesh.cg(b, use_graph=0, check_every=5)
    assert i1.iters == i2.iters
    assert torch.equal(x1, x2)


def test_jacobi_pcg_matches_oracle():
    p = inputs.small_laplace_16(seed=3)
    A, b, _, _ = _oracle_cg(p)
    dg = fem.diagonal(p.physics, p.coords, p.cell_array(), p.mat, p.dirichlet, p.n_nodes)
    _, it_o, _ = solvers.pcg(lambda v: A @ v, b, lambda r: r / dg, rtol=1e-8)
    mesh = mf.Mesh.from_problem(p)
    x, info = mesh.cg(gpu(b), precond=mf.MF_PC_JACOBI)
    assert info.status == mf.MF_OK
    assert abs(info.iters - it_o) <= max(2, math.ceil(0.01 * it_o)), (info.iters, it_o)
    assert info.rel_res_true <= 1.05e-8


@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
def test_mixed_precision_ir(physics):
    """FP32 inner CG (rtol 1e-4) inside FP64 refinement reaches a 1e-10 FP64 residual; the error
    against the oracle's FP64 solution is stated."""
    p = (inputs.laplace_box if physics == "laplace" else inputs.elasticity_box)(10, jitter=0.1, seed=14)
    A, b, xo, _ = _oracle_cg(p, rtol=1e-12)
    mesh = mf.Mesh.from_problem(p)
    x, info = mesh.cg(gpu(b), precision=mf.MF_PREC_MIXED_IR, rtol=1e-10, inner_rtol=1e-4)
    torch.cuda.synchronize()
    x = x.cpu().numpy()
    assert info.status == mf.MF_OK
    assert info.rel_res_true <= 1.05e-10
    assert np.linalg.norm(b - A @ x) <= 1.05e-10 * np.linalg.norm(b)
    err = rel2(x, xo)
    print(f"mixed IR {physics}: outer {info.outer_iters} inner {info.iters} err vs oracle {err:.2e}")
    assert err < 1e-6


# ------------------------------------------------------------------------------------- errors ----

def test_setup_rejects_inverted_element():
    p = inputs.laplace_box(3, seed=0)
    c = p.coords.copy()
    inner = inputs.node_id(1, 1, 1, 3, 3)
    c[inner] = c[inputs.node_id(2, 2, 2, 3, 3)] + 0.2  # push a node through its neighbours
    with pytest.raises(mf.MfError) as e:
        mf.Mesh("laplace", gpu(c), gpu(p.mat), gpu(p.dirichlet), None, (3, 3, 3))
    assert e.value.status == mf.MF_ERR_MESH


@pytest.mark.parametrize("what", ["nan_coord", "neg_kappa", "bad_node"])
def test_setup_rejects_bad_input(what):
    p = inputs.laplace_box(3, seed=0)
    c, k, cells = p.coords.copy(), p.mat.copy(), p.cell_array().copy()
    if what == "nan_coord":
        c[5, 1] = np.nan
    elif what == "neg_kappa":
        k[3] = -1.0
    else:
        cells[2, 4] = p.n_nodes + 7
    with pytest.raises(mf.MfError) as e:
        mf.Mesh("laplace", gpu(c), gpu(k), gpu(p.dirichlet), gpu(cells) if what == "bad_node" else None, (3, 3, 3))
    assert e.value.status == mf.MF_ERR_MESH


def test_apply_rejects_aliasing_and_wrong_physics():
    p = inputs.laplace_box(3, seed=0)
    mesh = mf.Mesh.from_problem(p)
    x = gpu(p.x())
    with pytest.raises(mf.MfError) as e:
        mf.mf_apply_laplace(mesh.h, x, x)
    assert e.value.status == mf.MF_ERR_ARG
    with pytest.raises(mf.MfError) as e:
        mf.mf_apply_elasticity(mesh.h, x, torch.empty_like(x))
    assert e.value.status == mf.MF_ERR_ARG


def test_cg_not_converged_and_breakdown_statuses():
    p = inputs.small_laplace_16(seed=0)
    mesh = mf.Mesh.from_problem(p)
    b = p.b()
    _, info = mesh.cg(gpu(b), max_iter=3)
    assert info.status == mf.MF_NOT_CONVERGED and info.iters == 3
    bn = b.copy()
    bn[17] = np.nan
    with pytest.raises(mf.MfError) as e:
        mesh.cg(gpu(bn))
    assert e.value.status == mf.MF_ERR_BREAKDOWN
    # the context stays usable
    x, info = mesh.cg(gpu(b))
    assert info.status == mf.MF_OK


def test_cg_timeout_status():
    p = inputs.laplace_box(24, jitter=0.2, seed=0)
    mesh = mf.Mesh.from_problem(p)
    with pytest.raises(mf.MfError) as e:
        mesh.cg(gpu(p.b()), timeout_s=1e-9, check_every=1, rtol=1e-14)
    assert e.value.status == mf.MF_ERR_TIMEOUT


# ------------------------------------------------------------- full-size sampled parity ----

def _sampled_parity(p, n_rows=1500, seed=0):
    mesh = mf.Mesh.from_problem(p)
    x = p.x()
    y = gpu_apply(mesh, x)
    rows = np.random.default_rng(seed).choice(p.n_dof, n_rows, replace=False)
    el = fem.adjacent_elements_box(rows // p.ndpn, p.nx, p.ny, p.nz)
    cells = inputs.box_cells(p.nx, p.ny, p.nz)
    ref = fem.apply_rows(p.physics, p.coords, cells, p.mat, p.dirichlet, x, rows, el)
    return rel2(y[rows], ref)


def test_full_size_laplace_256_sampled():
    """256^3 Cartesian Laplace (the benchmarked launch configuration): sampled rows vs the oracle."""
    assert _sampled_parity(inputs.cartesian_laplace_256()) <= TOL64


def test_full_size_elasticity_160_sampled():
    assert _sampled_parity(inputs.cartesian_elasticity_160()) <= TOL64


# ------------------------------------------------------- tensor-product tile kernels (auto) ----

TILE_SHAPES = [(1, 1, 1), (2, 3, 1), (31, 7, 5), (32, 8, 3), (45, 19, 23), (62, 14, 9), (5, 70, 4)]


@pytest.mark.parametrize("shape", TILE_SHAPES)
@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
def test_tile_apply_matches_oracle(shape, physics):
    """Graded (non-uniform) tensor-product grids with ragged tiles in x, y and z segments."""
    nx, ny, nz = shape
    mk = inputs.laplace_box if physics == "laplace" else inputs.elasticity_box
    p = mk(nx, ny=ny, nz=nz, graded=0.5, seed=nx + ny + nz, sigma=1.0)
    mesh = mf.Mesh.from_problem(p)
    assert mesh.info["tensor_product"]
    for seed in (0, 3):
        x = p.x(seed)
        y = gpu_apply(mesh, x)
        ref = oracle_apply(p, x)
        assert rel2(y, ref) <= TOL64, (shape, rel2(y, ref))
    # FP32 tile path: error stated and bounded
    y32 = mesh.apply(gpu(x).float())
    torch.cuda.synchronize()
    e32 = rel2(y32.double().cpu().numpy(), ref)
    assert e32 < 2e-6, e32


@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
def test_tile_and_reference_variants_agree(physics):
    mk = inputs.laplace_box if physics == "laplace" else inputs.elasticity_box
    p = mk(20, ny=17, nz=13, graded=0.3, seed=5)
    mesh = mf.Mesh.from_problem(p)
    x = gpu(p.x())
    ya = mesh.apply(x).clone()
    mesh.set_variant(mf.MF_VARIANT_REFERENCE)
    yr = mesh.apply(x).clone()
    torch.cuda.synchronize()
    assert rel2(ya.cpu().numpy(), yr.cpu().numpy()) <= TOL64
    mesh.set_variant(mf.MF_VARIANT_AUTO)
    yb = mesh.apply(x).clone()
    assert torch.equal(ya, yb)  # bitwise reproducible


@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
def test_tile_z_segments_bitwise_identical(physics):
    """The z-segment length only changes which CTA computes a node plane (the halo element layer
    below a segment is recomputed with the same operands), so every segmentation gives the same
    bits, also through the multi-RHS entry point."""
    mk = inputs.laplace_box if physics == "laplace" else inputs.elasticity_box
    p = mk(40, ny=23, nz=19, graded=0.4, seed=8, sigma=1.0)
    mesh = mf.Mesh.from_problem(p)
    x = gpu(p.x(2))
    outs = []
    for seg in (1, 2, 3, 7, 20, 0):
        mf.mf_set_tile_segment(mesh, seg)
        outs.append(mesh.apply(x).clone())
    torch.cuda.synchronize()
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    ref = oracle_apply(p, p.x(2))
    assert rel2(outs[0].cpu().numpy(), ref) <= TOL64
    ym = mesh.apply_multi(x, 1)
    torch.cuda.synchronize()
    assert torch.equal(ym, outs[0])


def test_tile_dirichlet_rows_and_large_values():
    """Dirichlet rows copy x; inputs spanning many binades stay FP64-accurate."""
    p = inputs.laplace_box(12, ny=9, nz=11, graded=0.4, seed=6)
    mesh = mf.Mesh.from_problem(p)
    rng = np.random.default_rng(0)
    x = rng.uniform(-1, 1, p.n_dof) * 10.0 ** rng.uniform(-20, 20, p.n_dof)
    y = gpu_apply(mesh, x)
    d = p.dirichlet.astype(bool)
    assert np.array_equal(y[d], x[d])
    ref = oracle_apply(p, x)
    assert rel2(y, ref) <= TOL64


@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
def test_cg_auto_variant_matches_oracle(physics):
    mk = inputs.laplace_box if physics == "laplace" else inputs.elasticity_box
    p = mk(12, ny=10, nz=14, graded=0.3, seed=7, layered=True, sigma=0.5)
    A, b, xo, it_o = _oracle_cg(p)
    mesh = mf.Mesh.from_problem(p)
    x, info = mesh.cg(gpu(b))
    torch.cuda.synchronize()
    assert info.status == mf.MF_OK
    assert abs(info.iters - it_o) <= max(2, math.ceil(0.01 * it_o)), (info.iters, it_o)
    assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 1.05e-8 * np.linalg.norm(b)


def test_mixed_ir_auto_variant():
    p = inputs.elasticity_box(14, ny=12, nz=10, graded=0.3, seed=8)
    A, b, xo, _ = _oracle_cg(p, rtol=1e-12)
    mesh = mf.Mesh.from_problem(p)
    x, info = mesh.cg(gpu(b), precision=mf.MF_PREC_MIXED_IR, rtol=1e-10)
    assert info.status == mf.MF_OK and info.rel_res_true <= 1.05e-10
    assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 1.05e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
@pytest.mark.parametrize("nrhs", [1, 3, 4, 5, 16])
def test_tile_apply_multi_rhs(physics, nrhs):
    """Multi right-hand-side apply ([node][rhs][comp], one launch over all right-hand sides): every
    column equals the single apply bitwise and the oracle to 1e-12."""
    mk = inputs.laplace_box if physics == "laplace" else inputs.elasticity_box
    p = mk(11, ny=9, nz=13, graded=0.4, seed=nrhs)
    mesh = mf.Mesh.from_problem(p)
    nd = p.ndpn
    xs = [p.x(seed=s) for s in range(nrhs)]
    X = np.stack([x.reshape(-1, nd) for x in xs], axis=1).reshape(-1)
    Y = mesh.apply_multi(gpu(X), nrhs)
    torch.cuda.synchronize()
    Y = Y.cpu().numpy().reshape(p.n_nodes, nrhs, nd)
    for r in range(nrhs):
        single = gpu_apply(mesh, xs[r])
        assert np.array_equal(Y[:, r, :].reshape(-1), single)
        assert rel2(single, oracle_apply(p, xs[r])) <= TOL64


def _warped(n, seed):
    """A smoothly warped structured box (not a tensor-product grid, large offsets from the axis lines)."""
    p = inputs.laplace_box(n, ny=n - 1, nz=n + 1, jitter=0.1, seed=seed)
    X = p.coords.copy()
    x, y, z = X[:, 0].copy(), X[:, 1].copy(), X[:, 2].copy()
    X[:, 0] = x + 0.08 * np.sin(np.pi * y) * z
    X[:, 1] = y + 0.05 * x * z
    X[:, 2] = z + 0.06 * np.sin(np.pi * x) * y
    return p, X


@pytest.mark.parametrize("physics", ["laplace", "elasticity"])
def test_general_kernel_on_warped_mesh(physics):
    """Structured but curved mesh: the general (per-Gauss-point Jacobian) double-word kernel."""
    p, X = _warped(9, 3)
    if physics == "elasticity":
        q = inputs.elasticity_box(9, ny=8, nz=10, seed=3)
        mat = q.mat
    else:
        mat = p.mat
    cells = p.cell_array()
    nd = 1 if physics == "laplace" else 3
    mesh = mf.Mesh(physics, gpu(X), gpu(np.ascontiguousarray(mat)), gpu(p.dirichlet), None, (p.nx, p.ny, p.nz))
    assert not mesh.info["tensor_product"]
    x = inputs.uniform_vector(p.n_nodes * nd, 4, dirichlet_dofs=np.nonzero(np.repeat(p.dirichlet, nd))[0])
    y = gpu_apply(mesh, x)
    ref = fem.apply(physics, X, cells, mat, p.dirichlet, x)
    assert rel2(y, ref) <= TOL64
    mesh.set_variant(mf.MF_VARIANT_REFERENCE)
    assert rel2(gpu_apply(mesh, x), ref) <= TOL64


# ------------------------------------------ general structured kernel and partial assembly ----

@pytest.mark.parametrize("physics", ["laplace", "elasticity", "vector_laplace"])
@pytest.mark.parametrize("variant", ["general", "partial"])
def test_general_and_partial_assembly_variants(physics, variant):
    """Jittered and warped structured boxes: the general kernel (geometry at every Gauss point in
    double-word arithmetic) and partial assembly (quadrature-point data computed once in FP64 and
    stored as float pairs) both match the oracle to 1e-12; their FP32 forms state their error."""
    mk = {"laplace": inputs.laplace_box, "elasticity": inputs.elasticity_box,
          "vector_laplace": inputs.vector_laplace_box}[physics]
    p = mk(23, ny=9, nz=14, jitter=0.2, seed=31, sigma=1.0)
    mesh = mf.Mesh.from_problem(p)
    assert not mesh.info["tensor_product"]
    mesh.set_variant(mf.MF_VARIANT_GENERAL if variant == "general" else mf.MF_VARIANT_PARTIAL)
    if variant == "partial":
        assert mf.mf_mesh_query(mesh.h)["partial_assembly"]
    for seed in (0, 1):
        x = p.x(seed)
        y = gpu_apply(mesh, x)
        ref = oracle_apply(p, x)
        assert rel2(y, ref) <= TOL64, (physics, variant, rel2(y, ref))
    y32 = mesh.apply(gpu(x).float())
    torch.cuda.synchronize()
    assert rel2(y32.double().cpu().numpy(), ref) < 2e-6


def test_partial_assembly_is_the_auto_choice_and_rejected_on_tensor_grids():
    p = inputs.elasticity_box(10, jitter=0.1, seed=32)
    mesh = mf.Mesh.from_problem(p)
    assert mesh.info["partial_assembly"]  # small mesh: the data fit, so the auto variant uses it
    x = p.x()
    ya = gpu_apply(mesh, x)
    mesh.set_variant(mf.MF_VARIANT_PARTIAL)
    assert np.array_equal(gpu_apply(mesh, x), ya)
    q = inputs.laplace_box(6, graded=0.3, seed=33)  # tensor-product grid: face-marching kernel only
    mq = mf.Mesh.from_problem(q)
    with pytest.raises(mf.MfError):
        mq.set_variant(mf.MF_VARIANT_PARTIAL)
