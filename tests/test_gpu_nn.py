"""BF16 tensor-core network kernels and the network runtime against the oracle (oracle/conv.py,
oracle/net.py).  Inputs are BF16-representable; the oracle accumulates in float64, the kernels in
FP32, so FP32 outputs agree to ~1e-5 relative and BF16 outputs to a BF16 rounding."""
import numpy as np
import pytest

from oracle import conv, net as onet

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
from paper_2308_09839_gb300 import mf  # noqa: E402


def bf(a):
    return torch.from_numpy(conv.bf16_round(a)).to(torch.bfloat16).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


SMALL = [((5, 7, 9), 2, 16), ((4, 4, 8), 16, 16), ((9, 6, 11), 16, 32), ((5, 5, 5), 32, 64),
         ((3, 9, 10), 64, 64), ((6, 5, 7), 64, 32), ((7, 7, 7), 32, 16), ((9, 9, 9), 16, 1), ((4, 5, 3), 3, 5),
         ((7, 6, 5), 64, 48), ((5, 6, 7), 64, 40),
         # 64 inputs to at most 16 outputs (forward) and 16 to 64 (its input gradient reads 64 channels
         # into 16): the configuration whose accumulator sets must span two planes
         ((6, 7, 5), 64, 16), ((5, 5, 6), 64, 8), ((5, 6, 6), 16, 64)]
# Node grids of the network's levels at sizes where the convolution kernels' persistent CTAs each
# loop over several work items (more output tiles than CTAs resident on the GPU), so that resident
# weights, re-staged halos and the per-item barriers are compared with the oracle too.  64 -> 64 (and
# 64 -> 48, 64 -> 40) forward runs as two launches over halves of the output channels; its input
# gradient takes the path that stages the weights in groups of taps.
LARGE = [((65, 65, 65), 2, 16), ((65, 65, 65), 16, 16), ((65, 65, 65), 16, 1), ((33, 33, 33), 16, 32),
         ((33, 33, 33), 32, 64), ((41, 41, 41), 64, 64), ((33, 33, 33), 64, 32), ((49, 49, 49), 32, 16),
         ((33, 33, 33), 64, 16)]
SHAPES = SMALL + LARGE


@pytest.mark.parametrize("dims,cin,cout", SHAPES)
def test_conv_fwd_matches_oracle(dims, cin, cout):
    rng = np.random.default_rng(cin * 100 + cout)
    nz, ny, nx = dims
    x = conv.bf16_round(rng.normal(size=(nz, ny, nx, cin)))
    w = conv.bf16_round(rng.normal(size=(27, cin, cout)) / np.sqrt(27 * cin))
    b = rng.normal(size=cout).astype(np.float32)
    skip = conv.bf16_round(rng.normal(size=(nz, ny, nx, cout)))
    ref = conv.conv3d(x, w, b) + skip
    y = torch.empty(nz, ny, nx, cout, dtype=torch.float32, device="cuda")
    mf.mf_conv3d_fwd(bf(x), bf(w), torch.from_numpy(b).cuda(), cout, skip=bf(skip), y_f32=y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), ref) < 1e-5
    # BF16 output: the FP32 result of the same launch (checked against the oracle) rounded to the
    # nearest BF16, after the ReLU, bit for bit
    yb = torch.empty(nz, ny, nx, cout, dtype=torch.bfloat16, device="cuda")
    yf = torch.empty(nz, ny, nx, cout, dtype=torch.float32, device="cuda")
    mf.mf_conv3d_fwd(bf(x), bf(w), torch.from_numpy(b).cuda(), cout, relu=True, y_bf16=yb, y_f32=yf)
    torch.cuda.synchronize()
    refr = np.maximum(conv.conv3d(x, w, b), 0)
    f32 = yf.cpu().numpy()
    assert rel(f32, refr) < 1e-5
    np.testing.assert_array_equal(yb.float().cpu().numpy(), conv.bf16_round(f32))


@pytest.mark.parametrize("dims,cin,cout", SHAPES)
def test_conv_dgrad_matches_oracle(dims, cin, cout):
    rng = np.random.default_rng(7 + cin + cout)
    nz, ny, nx = dims
    dy = conv.bf16_round(rng.normal(size=(nz, ny, nx, cout)))
    w = conv.bf16_round(rng.normal(size=(27, cin, cout)) / np.sqrt(27 * cout))
    dx = torch.empty(nz, ny, nx, cin, dtype=torch.float32, device="cuda")
    mf.mf_conv3d_dgrad(bf(dy), bf(w), cin, dx_f32=dx)
    torch.cuda.synchronize()
    assert rel(dx.cpu().numpy(), conv.conv3d_dgrad(dy, w)) < 1e-5


@pytest.mark.parametrize("dims,cin,cout", SHAPES)
def test_conv_wgrad_matches_oracle(dims, cin, cout):
    rng = np.random.default_rng(11 + cin + cout)
    nz, ny, nx = dims
    x = conv.bf16_round(rng.normal(size=(nz, ny, nx, cin)))
    dy = conv.bf16_round(rng.normal(size=(nz, ny, nx, cout)))
    dw, db = mf.mf_conv3d_wgrad(bf(x), bf(dy))
    torch.cuda.synchronize()
    rdw, rdb = conv.conv3d_wgrad(x, dy)
    assert rel(dw.cpu().numpy(), rdw) < 1e-5
    assert rel(db.cpu().numpy(), rdb) < 1e-5


def test_grid_transfers_match_oracle():
    rng = np.random.default_rng(3)
    xf = conv.bf16_round(rng.normal(size=(9, 5, 7, 4)))
    xc = conv.bf16_round(rng.normal(size=(3, 5, 4, 4)))
    r = mf.mf_grid_restrict(bf(xf), scale=2.0)
    p = mf.mf_grid_prolong(bf(xc), scale=0.5)
    torch.cuda.synchronize()
    rr, pr = 2.0 * conv.restrict(xf), 0.5 * conv.prolong(xc)
    assert np.all(np.abs(r.float().cpu().numpy() - rr) <= 2 ** -8 * np.abs(rr) + 1e-6)
    assert np.all(np.abs(p.float().cpu().numpy() - pr) <= 2 ** -8 * np.abs(pr) + 1e-6)


def _net_case(dims=(9, 13, 17), seed=0):
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    inp = rng.normal(size=(nz, ny, nx, 2)).astype(np.float32)
    tgt = rng.normal(size=(nz, ny, nx)).astype(np.float32)
    return inp, tgt


def test_network_forward_and_gradient_match_oracle():
    dims = (9, 13, 17)
    nt = mf.Net(*dims, seed=5)
    p = nt.params()
    assert p.size == onet.num_params()
    inp, tgt = _net_case(dims)
    r = torch.from_numpy(np.ascontiguousarray(inp[..., 0]).reshape(-1)).cuda()
    k = torch.from_numpy(np.ascontiguousarray(inp[..., 1]).reshape(-1)).cuda()
    t = torch.from_numpy(tgt.reshape(-1)).cuda()
    out = nt.forward(r, k)
    loss, g = nt.gradients(r, k, t)
    torch.cuda.synchronize()
    rloss, rg, rout = onet.loss_and_grad(p.astype(np.float64), inp, tgt, bf16=True)
    assert rel(out.cpu().numpy().reshape(rout.shape), rout) < 2e-2
    assert abs(loss - rloss) <= 2e-2 * abs(rloss)
    # per-layer gradient agreement (BF16 activations and gradients on both sides)
    off = 0
    for (_, ci, co, _) in onet.LAYERS:
        n = 27 * ci * co + co
        assert rel(g[off:off + n], rg[off:off + n]) < 5e-2, (ci, co)
        off += n


def test_network_training_reduces_loss_and_is_deterministic():
    dims = (9, 9, 9)
    inp, tgt = _net_case(dims, seed=1)
    r = torch.from_numpy(np.ascontiguousarray(inp[..., 0]).reshape(-1)).cuda()
    k = torch.from_numpy(np.ascontiguousarray(inp[..., 1]).reshape(-1)).cuda()
    # a learnable target: a smoothed copy of the input residual
    t = torch.from_numpy(conv.conv3d(inp[..., :1], np.full((27, 1, 1), 1.0 / 27))[..., 0].astype(np.float32).reshape(-1)).cuda()
    losses = []
    for rep in range(2):
        nt = mf.Net(*dims, seed=3)
        ls = [nt.train_step(r, k, t, 3e-3) for _ in range(60)]
        losses.append(ls)
        params = nt.params()
        if rep == 0:
            p0 = params
    assert losses[0][-1] < 0.5 * losses[0][0]
    assert losses[0] == losses[1]
    assert np.array_equal(p0, params)


def test_training_step_is_adam_on_the_clipped_gradient():
    """mf_net_train_step against oracle/optim.py, one step at a time: with the gradient g_t that
    mf_net_gradients returns at the current weights (the same forward and backward), the new FP32
    weights equal the oracle's FP64 Adam step on scale_t g_t, scale_t from the oracle's clip rule on
    ||g_t||.  The second step's target is scaled by 1e-3, which makes its gradient far larger than
    5x the first one's, so that step is clipped; the third is not.  Tolerance: 1e-4 lr plus 2.5e-7 of
    the weight, from the FP32 bias corrections 1 - b^t (their relative error reaches 3e-5 at t = 2)
    and the rounding of the weight (an FP32 emulation of the step stays below 0.15 of it)."""
    from oracle import optim
    dims = (9, 9, 9)
    inp, tgt = _net_case(dims, seed=2)
    r = torch.from_numpy(np.ascontiguousarray(inp[..., 0]).reshape(-1)).cuda()
    k = torch.from_numpy(np.ascontiguousarray(inp[..., 1]).reshape(-1)).cuda()
    t1 = torch.from_numpy(tgt.reshape(-1)).cuda()
    t2 = t1 * 1e-3
    nt = mf.Net(*dims, seed=4)
    p = nt.params().astype(np.float64)
    m, v, ema, lr, scales = np.zeros_like(p), np.zeros_like(p), 0.0, 1e-3, []
    for step, t in enumerate((t1, t2, t1), start=1):
        _, g = nt.gradients(r, k, t)
        g = g.astype(np.float64)
        assert np.all(np.isfinite(g)) and np.any(g != 0)
        scale, ema = optim.clip_scale(float(np.linalg.norm(g)), ema)
        scales.append(scale)
        p_exp, m, v = optim.adam_step(p, scale * g, m, v, step, lr)
        nt.train_step(r, k, t, lr)
        p_gpu = nt.params().astype(np.float64)
        err = np.abs(p_gpu - p_exp)
        tol = 1e-4 * lr + 2.5e-7 * np.abs(p_exp)
        assert np.all(err <= tol), (step, float((err / tol).max()))
        p = p_gpu
    nt.close()
    assert scales[0] == 1.0 and scales[1] < 0.1 and scales[2] == 1.0, scales


def test_learned_preconditioner_gains_over_jacobi_pcg():
    """Train on CG-generated pairs of a 32^3-cell GRF Laplace problem and use the network in
    flexible CG: it must reach the FP64 tolerance (true residual) and take fewer iterations than
    Jacobi-PCG (and so than plain CG).  (The wall-time comparison is reported by the benchmark.)"""
    from paper_2308_09839_gb300 import inputs, learned
    p = inputs.grf_laplace_128(seed=0, n=32)
    mesh = mf.Mesh.from_problem(p)
    nzyx = (p.nz + 1, p.ny + 1, p.nx + 1)
    R, E, c = learned.generate_pairs(mesh, p, 64, seed=1, k_range=(2, 60))
    lk = learned.node_logk(mesh)
    params, hist, secs = learned.train(R, E, lk, nzyx, crop=33, steps=1500, lr=2e-4)
    assert np.mean(hist[-50:]) < 0.7 * np.mean(hist[:20])
    net = learned.make_inference_net(params, nzyx, c)
    b = torch.from_numpy(p.b()).cuda()
    x_cg, i_cg = mesh.cg(b)
    x_j, i_j = mesh.cg(b, precond=mf.MF_PC_JACOBI)
    x_nn, i_nn = mesh.cg(b, net=net)
    torch.cuda.synchronize()
    assert i_nn.status == mf.MF_OK and i_nn.rel_res_true <= 1.05e-8
    print(f"plain CG {i_cg.iters} it, Jacobi-PCG {i_j.iters} it, learned FCG {i_nn.iters} it "
          f"(switched off at {i_nn.outer_iters})")
    assert i_nn.iters < i_j.iters < i_cg.iters


def test_fcg_with_zero_network_matches_oracle_fcg_m():
    """With every network parameter zero the correction vanishes (theta = 0) and the learned
    preconditioner is two damped-Jacobi sweeps (omega = 2/3), a fixed linear map; the GPU's
    truncated flexible CG (8 stored directions) must then follow the oracle's FCG(8) with that
    preconditioner: same iteration count (+-1) and the same solution."""
    from oracle import fem, solvers
    from paper_2308_09839_gb300 import inputs
    p = inputs.laplace_box(12, jitter=0.0, sigma=1.0, seed=4)
    mesh = mf.Mesh.from_problem(p)
    net = mf.Net(p.nx + 1, p.ny + 1, p.nz + 1, seed=0)
    net.set_params(np.zeros(net.n_params, np.float32))
    net.set_output_scale(1.0)
    b = p.b()
    x, info = mesh.cg(torch.from_numpy(b).cuda(), net=net, rtol=1e-8)
    torch.cuda.synchronize()
    A = fem.assemble_csr("laplace", p.coords, p.cell_array(), p.mat, p.dirichlet, p.n_nodes)
    d = A.diagonal()
    w = 2.0 / 3.0

    def two_sweeps(r):
        z1 = w * r / d
        return z1 + w * (r - A @ z1) / d

    xo, it_o, h_o = solvers.fcg_m(lambda v: A @ v, b, two_sweeps, m=8, rtol=1e-8)
    assert info.status == mf.MF_OK and info.outer_iters == -1
    assert abs(info.iters - it_o) <= 1, (info.iters, it_o)
    assert info.rel_res_true <= 1.05e-8 and h_o[-1] <= 1e-8
    assert rel(x.cpu().numpy(), xo) <= 1e-6
    net.close()


def test_training_pairs_match_oracle():
    """The training pairs of the learned preconditioner against the oracle: in FP64 before any
    scaling the pair satisfies A e = r with the oracle's A; r~ = D^-1/2 (b - A x_k) and
    e~ = D^1/2 (x* - x_k) with the oracle's diagonal; the FP32 pairs the workflow stores are r~/s and
    c e~/s with s = RMS(r~) and c the median ratio RMS(r~)/RMS(e~), to FP32 rounding."""
    from oracle import fem
    from paper_2308_09839_gb300 import inputs, learned
    p = inputs.laplace_box(16, ny=12, nz=9, sigma=1.0, layered=True, seed=2)
    mesh = mf.Mesh.from_problem(p)
    R, T, c, states = learned.generate_pairs(mesh, p, 5, seed=3, k_range=(2, 40), keep_states=True)
    torch.cuda.synchronize()
    A = fem.assemble_csr(p.physics, p.coords, p.cell_array(), p.mat, p.dirichlet, p.n_nodes)
    D = fem.diagonal(p.physics, p.coords, p.cell_array(), p.mat, p.dirichlet, p.n_nodes)
    free = p.dirichlet == 0
    ratios = []
    for i, (xs_d, xk_d) in enumerate(states):
        xs, xk = xs_d.cpu().numpy(), xk_d.cpu().numpy()
        b_d = mesh.apply(xs_d)
        r64 = torch.empty_like(xs_d)
        e64 = torch.empty_like(xs_d)
        r32 = torch.empty(p.n_dof, dtype=torch.float32, device="cuda")
        e32 = torch.empty_like(r32)
        sr, se = mf.mf_training_pair(mesh, b_d, xs_d, xk_d, r32, e32, r64=r64, e64=e64)
        r64, e64 = r64.cpu().numpy(), e64.cpu().numpy()
        # the defining identity, unscaled: A e = r on the free DoFs.  r = b - A x_k comes from two
        # FP64 applies, each within 1e-12 of the oracle relative to its own norm, so the bound is
        # relative to ||b|| + ||A x_k||, not to the (smaller) ||r||
        r_un, e_un = r64 * np.sqrt(D), e64 / np.sqrt(D)
        scale = np.linalg.norm((A @ xs)[free]) + np.linalg.norm((A @ xk)[free])
        assert np.linalg.norm(r_un[free] - (A @ e_un)[free]) <= 1e-12 * scale
        r_ref = np.where(free, (A @ xs - A @ xk) / np.sqrt(D), 0.0)
        e_ref = np.where(free, (xs - xk) * np.sqrt(D), 0.0)
        assert np.linalg.norm(r64 - r_ref) <= 1e-12 * scale / np.sqrt(D.min())
        assert rel(e64, e_ref) <= 1e-14
        assert abs(sr - (r64 ** 2).sum()) <= 1e-12 * sr and abs(se - (e_ref ** 2).sum()) <= 1e-12 * se
        # the stored FP32 pair: the FP64 pair (r64, e64: checked above) over s, rounded once
        s = np.sqrt(np.mean(r64 ** 2))
        ratios.append(s / np.sqrt(np.mean(e64 ** 2)))
        tol = lambda v: 2.0 ** -23 * np.abs(v) + 1e-30
        assert np.all(np.abs(r32.cpu().numpy() - r64 / s) <= tol(r64 / s))
        assert np.all(np.abs(R[i].cpu().numpy() - r64 / s) <= tol(r64 / s))
        ti = e64 / s
        assert np.all(np.abs(T[i].cpu().numpy() / c - ti) <= 2 * tol(ti))
    assert abs(c - float(np.median(ratios))) <= 1e-10 * c


def test_training_checkpoint_resume_is_bitwise(tmp_path):
    """A training run stopped at step 17, written to a .pt file, read back and resumed takes the same
    steps as the uninterrupted run: equal loss history and parameters, bit for bit (the network's whole
    training state: parameters, Adam moments and step, clip history, plus the crop generator)."""
    from paper_2308_09839_gb300 import learned
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    nzyx = (17, 17, 17)
    R = torch.randn(4, 17 ** 3, device="cuda", generator=g)
    E = torch.randn(4, 17 ** 3, device="cuda", generator=g)
    lk = torch.randn(17 ** 3, device="cuda", generator=g)
    kw = dict(crop=9, steps=40, lr=3e-3, seed=5, warmup=5)
    pa, ha, _ = learned.train(R, E, lk, nzyx, **kw)
    ck = learned.train(R, E, lk, nzyx, stop_at=17, **kw)
    assert ck["step"] == 17 and len(ck["hist"]) == 17
    path = str(tmp_path / "train.pt")
    learned.save_checkpoint(path, ck)
    pb, hb, _ = learned.train(R, E, lk, nzyx, resume=learned.load_checkpoint(path), **kw)
    assert ha == hb
    assert np.array_equal(pa, pb)
    # a buffer that is not a state, or a truncated one, is refused
    net = mf.Net(9, 9, 9, seed=0)
    blob = net.state()
    bad = blob.copy()
    bad[0] ^= 0xFF
    with pytest.raises(mf.MfError):
        net.load_state(bad)
    with pytest.raises(mf.MfError):
        net.load_state(blob[:-4])
    # header fields out of range (header: magic, n_params, step as 8-byte integers, two clip
    # floats, the output scale): a negative step, a zero output scale, a NaN clip average
    for off, val in ((16, np.int64(-1)), (32, np.float32(0.0)), (24, np.float32(np.nan))):
        bad = blob.copy()
        raw = np.array([val]).view(np.uint8)
        bad[off:off + raw.size] = raw
        with pytest.raises(mf.MfError):
            net.load_state(bad)
    assert np.array_equal(net.state(), blob)  # refused loads left the network as it was
    net.load_state(blob)
    net.close()


def test_node_logk_is_the_mean_over_adjacent_cells():
    """The network's second input channel (mf_node_logk): log kappa averaged over the cells that touch
    each node, checked by brute force on a small ragged box (corner nodes touch 1 cell, interior 8)."""
    from paper_2308_09839_gb300 import inputs
    p = inputs.laplace_box(4, ny=3, nz=2, sigma=1.0, seed=4)
    mesh = mf.Mesh.from_problem(p)
    got = mf.mf_node_logk(mesh).cpu().numpy()
    lk = np.log(p.mat).reshape(p.nz, p.ny, p.nx)
    for k in range(p.nz + 1):
        for j in range(p.ny + 1):
            for i in range(p.nx + 1):
                vals = [lk[ez, ey, ex] for ez in (k - 1, k) for ey in (j - 1, j) for ex in (i - 1, i)
                        if 0 <= ez < p.nz and 0 <= ey < p.ny and 0 <= ex < p.nx]
                n = inputs.node_id(i, j, k, p.nx, p.ny)
                assert abs(got[n] - np.mean(vals)) <= 1e-6 * max(1.0, abs(np.mean(vals)))
    # a mesh it does not serve is refused
    pe = inputs.elasticity_box(2, seed=1)
    with pytest.raises(mf.MfError):
        mf.mf_node_logk(mf.Mesh.from_problem(pe), out=torch.empty(pe.n_nodes, device="cuda"))
