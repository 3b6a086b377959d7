"""Pins of the network oracle (oracle/conv.py) against definitions it does not use itself."""
import numpy as np

from oracle import conv


def _rand(*s, seed=0):
    return np.random.default_rng(seed).normal(size=s)


def test_conv_brute_force_tiny():
    x = _rand(3, 4, 5, 2, seed=1)
    w = _rand(27, 2, 3, seed=2)
    b = _rand(3, seed=3)
    y = conv.conv3d(x, w, b)
    nz, ny, nx, _ = x.shape
    ref = np.zeros((nz, ny, nx, 3))
    for z in range(nz):
        for yy in range(ny):
            for xx in range(nx):
                acc = b.copy()
                for t in range(27):
                    dx, dy, dz = t % 3 - 1, (t // 3) % 3 - 1, t // 9 - 1
                    zz, yj, xi = z + dz, yy + dy, xx + dx
                    if 0 <= zz < nz and 0 <= yj < ny and 0 <= xi < nx:
                        acc += x[zz, yj, xi] @ w[t]
                ref[z, yy, xx] = acc
    assert np.allclose(y, ref, atol=1e-12)


def test_center_tap_is_a_matmul():
    x = _rand(4, 3, 5, 6, seed=4)
    w = np.zeros((27, 6, 7))
    w[13] = _rand(6, 7, seed=5)
    assert np.allclose(conv.conv3d(x, w), x @ w[13], atol=1e-12)


def test_dgrad_is_the_adjoint():
    x = _rand(5, 4, 6, 3, seed=6)
    y = _rand(5, 4, 6, 4, seed=7)
    w = _rand(27, 3, 4, seed=8)
    lhs = np.sum(conv.conv3d(x, w) * y)
    rhs = np.sum(x * conv.conv3d_dgrad(y, w))
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_wgrad_matches_directional_derivative():
    x = _rand(4, 5, 3, 3, seed=9)
    y = _rand(4, 5, 3, 2, seed=10)
    w = _rand(27, 3, 2, seed=11)
    d = _rand(27, 3, 2, seed=12)
    b = _rand(2, seed=13)
    db_dir = _rand(2, seed=14)
    f = lambda ww, bb: np.sum(conv.conv3d(x, ww, bb) * y)
    dw, dbias = conv.conv3d_wgrad(x, y)
    # the loss is linear in (w, b): the directional difference is exact
    assert abs((f(w + d, b + db_dir) - f(w, b)) - (np.sum(d * dw) + db_dir @ dbias)) < 1e-9


def test_restriction_prolongation_pair():
    rng = np.random.default_rng(15)
    xc = rng.normal(size=(3, 5, 4, 2))
    xf = rng.normal(size=(5, 9, 7, 2))
    # prolongation is 8 x the adjoint of full weighting
    assert abs(np.sum(conv.restrict(xf) * xc) * 8 - np.sum(xf * conv.prolong(xc))) < 1e-10
    # trilinear interpolation reproduces linear fields exactly
    zc, yc, xcc = np.meshgrid(np.arange(3), np.arange(5), np.arange(4), indexing="ij")
    lin = (0.3 * zc - 1.2 * yc + 0.7 * xcc + 2.0)[..., None]
    zf, yf, xf_ = np.meshgrid(np.arange(5) / 2, np.arange(9) / 2, np.arange(7) / 2, indexing="ij")
    assert np.allclose(conv.prolong(lin)[..., 0], 0.3 * zf - 1.2 * yf + 0.7 * xf_ + 2.0)
    # full weighting keeps constants at interior coarse nodes
    r = conv.restrict(np.ones((9, 9, 9, 1)))
    assert np.allclose(r[1:-1, 1:-1, 1:-1], 1.0)


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 3.14159265, -2.5e-3], dtype=np.float32)
    r = conv.bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7  # ties to even
    assert abs(r[3] - 3.140625) < 1e-7
    assert np.all(np.abs(r - v) <= np.abs(v) * 2 ** -8)


def test_network_oracle_gradient_matches_finite_differences():
    """The exact (no rounding) network oracle's backward equals central differences of its forward."""
    from oracle import net
    rng = np.random.default_rng(20)
    p = rng.normal(size=net.num_params()) * 0.2
    inp = rng.normal(size=(5, 5, 9, 2))
    tgt = rng.normal(size=(5, 5, 9))
    loss, g, _ = net.loss_and_grad(p, inp, tgt, bf16=False)
    idx = rng.choice(p.size, 40, replace=False)
    # include weights of every layer and the biases of the output layer
    idx = np.concatenate([idx, [p.size - 1, 5, 27 * 32 + 3]])
    eps = 1e-6
    for i in idx:
        dp = np.zeros_like(p)
        dp[i] = eps
        lp = net.loss_and_grad(p + dp, inp, tgt, bf16=False)[0]
        lm = net.loss_and_grad(p - dp, inp, tgt, bf16=False)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])
