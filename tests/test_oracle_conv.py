"""Pins of the network oracle (oracle/conv.py, oracle/net.py, oracle/optim.py) against definitions it does not use itself."""
import numpy as np
import pytest

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


def test_adam_closed_forms():
    """Adam (oracle/optim.py) against what its definition fixes: the first step from zero moments
    moves every parameter by lr g / (|g| + eps) (the bias corrections make m_hat = g, v_hat = g^2);
    a constant gradient keeps that step size at every later step; a zero gradient component never
    moves; and the moments follow their geometric sums."""
    from oracle import optim
    rng = np.random.default_rng(3)
    p0 = rng.standard_normal(50)
    g = rng.standard_normal(50) * np.logspace(-6, 2, 50)
    g[7] = 0.0
    lr, eps = 1e-3, 1e-8
    p1, m1, v1 = optim.adam_step(p0, g, np.zeros(50), np.zeros(50), 1, lr)
    np.testing.assert_allclose(p0 - p1, lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-18)
    p, m, v = p0, np.zeros(50), np.zeros(50)
    for t in range(1, 13):
        p, m, v = optim.adam_step(p, g, m, v, t, lr)
    np.testing.assert_allclose(p0 - p, 12 * lr * g / (np.abs(g) + eps), rtol=1e-10, atol=1e-16)
    assert p[7] == p0[7]
    np.testing.assert_allclose(m, (1 - 0.9 ** 12) * g, rtol=1e-12)
    np.testing.assert_allclose(v, (1 - 0.999 ** 12) * g * g, rtol=1e-12)
    # a gradient that flips sign at the second step: m = 0.9 (0.1 g) - 0.1 g and
    # v = (0.999 * 0.001 + 0.001) g^2, corrected by 1 - 0.9^2 and 1 - 0.999^2 (the difference of two
    # parameters of size up to 3 is exact to a few of their ulps, hence the absolute tolerance)
    p2, _, _ = optim.adam_step(p1, -g, m1, v1, 2, lr)
    m_hat = (0.9 * 0.1 * g - 0.1 * g) / (1 - 0.81)
    v_hat = (0.999 * 0.001 + 0.001) * g * g / (1 - 0.999 ** 2)
    np.testing.assert_allclose(p1 - p2, lr * m_hat / (np.sqrt(v_hat) + eps), rtol=1e-12, atol=4e-15)


def test_gradient_clip_special_cases():
    """The clip rule (oracle/optim.py): the first step keeps its gradient and sets the average; a
    norm up to 5x the average is kept; 10x is halved and the average moves by a tenth of the clipped
    norm; a non-finite norm skips the step and keeps the average."""
    from oracle import optim
    assert optim.clip_scale(3.0, 0.0) == (1.0, 3.0)
    s, e = optim.clip_scale(10.0, 2.0)
    assert s == 1.0 and e == pytest.approx(0.9 * 2.0 + 0.1 * 10.0)
    s, e = optim.clip_scale(20.0, 2.0)
    assert s == pytest.approx(0.5) and e == pytest.approx(0.9 * 2.0 + 0.1 * 10.0)
    assert optim.clip_scale(float("nan"), 2.0) == (0.0, 2.0)
    assert optim.clip_scale(float("inf"), 2.0) == (0.0, 2.0)
