"""Batched persistent CG (one cooperative launch for many problems) against the oracle and the
single-problem solver."""
import math

import numpy as np
import pytest

from oracle import fem, solvers
from paper_2308_09839_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_2308_09839_gb300 import autotune, mf  # noqa: E402

SIZES = [1, 3, 8, 13, 20, 31, 5, 17]


def _problems(sizes, seed0=100):
    return [inputs.laplace_box(n, ny=max(1, n - 1), nz=n + 2, graded=0.3, sigma=1.0, seed=seed0 + i)
            for i, n in enumerate(sizes)]


def _setup(ps):
    meshes = [mf.Mesh.from_problem(p) for p in ps]
    bs = [torch.from_numpy(p.b()).cuda() for p in ps]
    xs = [torch.zeros_like(b) for b in bs]
    return meshes, bs, xs


def test_batched_matches_oracle_cg():
    ps = _problems(SIZES)
    meshes, bs, xs = _setup(ps)
    infos = mf.mf_cg_solve_batched(meshes, mf.mf_solve_opts_default(), bs, xs)
    torch.cuda.synchronize()
    for p, info, x in zip(ps, infos, xs):
        A = fem.assemble_csr(p.physics, p.coords, p.cell_array(), p.mat, p.dirichlet, p.n_nodes)
        b = p.b()
        _, it_o, _ = solvers.cg(lambda v: A @ v, b, rtol=1e-8)
        assert info.status == mf.MF_OK
        assert abs(info.iters - it_o) <= max(2, math.ceil(0.01 * it_o)), (p.nx, info.iters, it_o)
        assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 1.05e-8 * np.linalg.norm(b)


def test_batched_matches_single_solver_and_is_deterministic():
    ps = _problems([6, 11, 23])
    meshes, bs, xs = _setup(ps)
    o = mf.mf_solve_opts_default()
    batch = mf.mf_batch_create(meshes, o)
    i1 = mf.mf_batch_solve(batch, bs, xs)
    x1 = [x.clone() for x in xs]
    i2 = mf.mf_batch_solve(batch, bs, xs)
    mf.mf_batch_destroy(batch)
    for a, b_, x, y in zip(i1, i2, x1, xs):
        assert a.iters == b_.iters
        assert torch.equal(x, y)
    for m, b, x, info in zip(meshes, bs, x1, i1):
        xr, ir = m.cg(b)
        assert abs(ir.iters - info.iters) <= 2
        assert float(torch.linalg.norm(xr - x) / torch.linalg.norm(xr)) < 1e-6


def test_batched_segment_choice_does_not_change_results():
    ps = _problems([9, 19, 27])
    meshes, bs, xs = _setup(ps)
    o = mf.mf_solve_opts_default()
    outs = []
    for seg in (1, 4, 64):
        for m in meshes:
            mf.mf_set_tile_segment(m, seg)
        mf.mf_cg_solve_batched(meshes, o, bs, xs)
        outs.append([x.clone() for x in xs])
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)
    for a, b in zip(outs[0], outs[2]):
        assert torch.equal(a, b)


def test_autotuner_sets_segments(tmp_path, monkeypatch):
    monkeypatch.setenv("MF_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    ps = _problems([8, 24, 40])
    meshes, bs, xs = _setup(ps)
    choice = autotune.tune(meshes, [p.nz + 1 for p in ps], bs, xs, iters=5)
    assert set(choice.values()) <= set(autotune.CANDIDATES)
    again = autotune.tune(meshes, [p.nz + 1 for p in ps], bs, xs, iters=5)  # from the cache
    assert again == choice
    infos = mf.mf_cg_solve_batched(meshes, mf.mf_solve_opts_default(), bs, xs)
    assert all(i.status == mf.MF_OK for i in infos)


def test_batched_barrier_timeout_returns_error():
    """A barrier budget of a few cycles makes every wait run out: the kernel must return and the
    host must report MF_ERR_TIMEOUT, with the context still usable."""
    ps = _problems([10, 12])
    meshes, bs, xs = _setup(ps)
    o = mf.mf_solve_opts_default()
    o.timeout_s = 1e-9
    with pytest.raises(mf.MfError) as e:
        mf.mf_cg_solve_batched(meshes, o, bs, xs)
    assert e.value.status == mf.MF_ERR_TIMEOUT
    infos = mf.mf_cg_solve_batched(meshes, mf.mf_solve_opts_default(), bs, xs)
    assert all(i.status == mf.MF_OK for i in infos)


def test_batched_rejects_unsupported_meshes():
    p = inputs.laplace_box(4, jitter=0.2, seed=1)  # not a tensor-product grid
    m = mf.Mesh.from_problem(p)
    b = torch.from_numpy(p.b()).cuda()
    with pytest.raises(mf.MfError) as e:
        mf.mf_cg_solve_batched([m], mf.mf_solve_opts_default(), [b], [torch.zeros_like(b)])
    assert e.value.status == mf.MF_ERR_UNSUPPORTED
