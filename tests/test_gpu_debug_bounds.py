"""The bounds-checked build (-DMF_DEBUG_BOUNDS, libmf_debug.so) runs tiny, ragged, jittered,
renumbered, tetrahedral and Q2 meshes through every operator path (all apply variants, multi-RHS,
CSR fill and SpMV, operator diagonal, CG, the batched solver) without a failed index check, and its
results match the oracle.  Every check that fails records a bit and redirects the access in bounds,
so this test cannot fault the GPU even if an index were wrong."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
import numpy as np, torch
from oracle import fem
from paper_2308_09839_gb300 import inputs, mf

def rel2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

errs = {}
def run(tag, p, structured=True, variants=(mf.MF_VARIANT_AUTO, mf.MF_VARIANT_REFERENCE)):
    m = mf.Mesh.from_problem(p, structured=structured)
    x = p.x()
    ref = fem.apply(p.physics, p.coords, p.cell_array(), p.mat, p.dirichlet, x)
    for v in variants:
        m.set_variant(v)
        y = m.apply(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        errs[f"{tag}/variant{v}"] = rel2(y.cpu().numpy(), ref)
    m.set_variant(mf.MF_VARIANT_AUTO)
    A = m.assemble_csr()
    ys = A.spmv(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    errs[f"{tag}/csr"] = rel2(ys.cpu().numpy(), ref)
    d = torch.empty(p.n_dof, dtype=torch.float64, device="cuda")
    mf.mf_operator_diagonal(m, d)
    b = torch.from_numpy(p.b()).cuda()
    xs, info = m.cg(b, max_iter=30, ok=(mf.MF_OK, mf.MF_NOT_CONVERGED))
    xc, _ = m.cg(b, max_iter=30, csr=A, ok=(mf.MF_OK, mf.MF_NOT_CONVERGED))
    torch.cuda.synchronize()
    return m

for n, ny, nz in ((1, 1, 1), (2, 2, 2), (3, 3, 3), (5, 3, 2)):
    run(f"lap{n}x{ny}x{nz}", inputs.laplace_box(n, ny=ny, nz=nz, seed=1))
    run(f"el{n}x{ny}x{nz}", inputs.elasticity_box(n, ny=ny, nz=nz, seed=2))
    run(f"vl{n}x{ny}x{nz}", inputs.vector_laplace_box(n, ny=ny, nz=nz, seed=3))
run("lap_graded", inputs.laplace_box(9, ny=7, nz=11, graded=0.3, seed=4))
allv = (mf.MF_VARIANT_AUTO, mf.MF_VARIANT_REFERENCE, mf.MF_VARIANT_GENERAL, mf.MF_VARIANT_PARTIAL)
run("lap_jit", inputs.laplace_box(4, ny=3, nz=5, jitter=0.2, seed=5), variants=allv)
run("el_jit", inputs.elasticity_box(3, ny=4, nz=2, jitter=0.2, seed=6), variants=allv)
run("lap_explicit", inputs.laplace_box(3, jitter=0.2, seed=7), structured=False)
run("tet_lap", inputs.tet_box("laplace", 2, ny=3, nz=2, jitter=0.1, seed=8))
run("tet_el", inputs.tet_box("elasticity", 2, jitter=0.1, seed=9))
run("q2_lap", inputs.q2_box("laplace", 2, ny=1, nz=2, jitter=0.1, seed=10))
run("q2_el", inputs.q2_box("elasticity", 2, jitter=0.1, seed=11))
# multi-RHS block apply on a tensor-product mesh
p = inputs.elasticity_box(4, ny=3, nz=5, seed=12)
m = mf.Mesh.from_problem(p)
xs = np.stack([p.x(s) for s in range(3)], axis=1)  # [dof][rhs]
X = torch.from_numpy(np.ascontiguousarray(xs.reshape(p.n_nodes, p.ndpn, 3).transpose(0, 2, 1))).cuda().reshape(-1)
Y = torch.empty_like(X)
mf.mf_apply_multi(m.h, 3, X, Y)
torch.cuda.synchronize()
Yh = Y.cpu().numpy().reshape(p.n_nodes, 3, p.ndpn)
for r in range(3):
    ref = fem.apply(p.physics, p.coords, p.cell_array(), p.mat, p.dirichlet, xs[:, r])
    errs[f"multi/rhs{r}"] = rel2(Yh[:, r, :].reshape(-1), ref)
# batched persistent solver over uneven sizes
probs = [inputs.laplace_box(n, seed=20 + n) for n in (2, 3, 5)]
meshes = [mf.Mesh.from_problem(q) for q in probs]
o = mf.mf_solve_opts_default(); o.max_iter = 20; o.rtol = 1e-30
bs = [torch.from_numpy(q.b()).cuda() for q in probs]
xb = [torch.zeros_like(b) for b in bs]
batch = mf.mf_batch_create(meshes, o)
mf.mf_batch_solve(batch, bs, xb)
mf.mf_batch_destroy(batch)
bits, enabled = mf.mf_debug_status()
print(json.dumps({"bits": bits, "enabled": enabled, "max_err": max(errs.values()), "errs": errs}))
"""


def test_bounds_checked_build_runs_clean():
    subprocess.run([sys.executable, "-m", "paper_2308_09839_gb300.build", "--debug"], cwd=ROOT, check=True,
                   timeout=1200, capture_output=True)
    env = dict(os.environ, MF_LIB=os.path.join(ROOT, "paper_2308_09839_gb300", "libmf_debug.so"))
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-4000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["enabled"], "the debug library did not compile its checks in"
    assert out["bits"] == 0, out
    bad = {k: v for k, v in out["errs"].items() if not v <= 1e-12}
    assert not bad, bad
