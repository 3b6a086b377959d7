"""Plant plausible slips in the oracle (on the CPU, via monkeypatch) and check that a pin catches each.

This guards the pins themselves: a pin that cannot fail would not pin anything."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import fem
from paper_2308_09839_gb300 import inputs
from tests import _exact


def _affine_laplace_error():
    Jq = [[Fraction(2), Fraction(1, 8), Fraction(-3, 8)],
          [Fraction(-1, 4), Fraction(17, 8), Fraction(1, 4)],
          [Fraction(3, 8), Fraction(-1, 8), Fraction(15, 8)]]
    exact = np.array(_exact.affine_laplace_exact(Jq, Fraction(1)), dtype=float)
    J = np.array(Jq, dtype=float)
    X = fem.corner_signs() @ J.T
    A = fem.laplace_element_matrices(X[None], np.array([1.0]))[0]
    return np.max(np.abs(A - exact)) / np.max(np.abs(exact))


def _affine_elasticity_error():
    Jq = [[Fraction(2), Fraction(1, 8), Fraction(-3, 8)],
          [Fraction(-1, 4), Fraction(17, 8), Fraction(1, 4)],
          [Fraction(3, 8), Fraction(-1, 8), Fraction(15, 8)]]
    exact = np.array(_exact.affine_elasticity_exact(Jq, Fraction(7, 5), Fraction(3, 4)), dtype=float)
    X = fem.corner_signs() @ np.array(Jq, dtype=float).T
    A = fem.elasticity_element_matrices(X[None], np.array([1.4]), np.array([0.75]))[0]
    return np.max(np.abs(A - exact)) / np.max(np.abs(exact))


def test_unmutated_baseline():
    assert _affine_laplace_error() < 1e-13
    assert _affine_elasticity_error() < 1e-13


def test_catches_transposed_inverse_jacobian(monkeypatch):
    """grad phi = J^{-1} grad_ref phi (instead of J^{-T}) changes A^e on a non-symmetric J."""
    def wrong(J, dN):
        det = np.linalg.det(J)
        return np.einsum("eqij,qaj->eqai", np.linalg.inv(J), dN), det
    monkeypatch.setattr(fem, "physical_grads", wrong)
    assert _affine_laplace_error() > 1e-3


def test_catches_transposed_jacobian(monkeypatch):
    monkeypatch.setattr(fem, "jacobians", lambda X, dN: np.einsum("eai,qaj->eqji", X, dN))
    assert _affine_laplace_error() > 1e-3


def test_catches_dropped_stress_term(monkeypatch):
    """Dropping the mu (d_l phi_a d_k phi_b) term (i.e. sigma from grad u instead of sym grad u)."""
    orig = fem.elasticity_element_matrices

    def wrong(X, lam, mu):
        pts, w = fem.gauss_points()
        dN = fem.shape_ref_grads(pts)
        g, det = fem.physical_grads(fem.jacobians(X, dN), dN)
        wd = det * w[None, :]
        A = np.einsum("e,eq,eqak,eqbl->eakbl", lam, wd, g, g)
        dot = np.einsum("e,eq,eqai,eqbi->eab", 2 * mu, wd, g, g)
        for k in range(3):
            A[:, :, k, :, k] += dot
        return A.reshape(X.shape[0], 24, 24)
    monkeypatch.setattr(fem, "elasticity_element_matrices", wrong)
    assert _affine_elasticity_error() > 1e-3
    monkeypatch.setattr(fem, "elasticity_element_matrices", orig)


def test_catches_wrong_gauss_point(monkeypatch):
    """Gauss points at +-1/2 instead of +-1/sqrt(3): the cube closed form still holds for Laplace on
    a cube? No - the diagonal changes; the exact-rational pin fails."""
    monkeypatch.setattr(fem, "G", 0.5)
    assert _affine_laplace_error() > 1e-3


def test_catches_shape_function_sign_slip(monkeypatch):
    orig = fem.corner_signs

    def wrong():
        s = orig().copy()
        s[3, 0] *= -1
        return s
    monkeypatch.setattr(fem, "corner_signs", wrong)
    coords = inputs.box_coords(3, 3, 3, 0.2, 3)
    cells = inputs.box_cells(3, 3, 3)
    y = fem.apply("laplace", coords, cells, np.ones(cells.shape[0]), np.zeros(coords.shape[0], np.uint8),
                  np.ones(coords.shape[0]))
    assert np.max(np.abs(y)) > 1e-6  # A 1 = 0 pin fails


def test_catches_missing_dirichlet_column_drop(monkeypatch):
    """Applying A to x without zeroing Dirichlet columns breaks symmetry of the operator."""
    p = inputs.laplace_box(3, jitter=0.2, seed=4)
    cells = p.cell_array()
    d = p.dirichlet.astype(bool)

    def wrong_apply(x):
        y = fem.apply("laplace", p.coords, cells, p.mat, np.zeros_like(p.dirichlet), x)
        y[d] = x[d]
        return y
    x = inputs.uniform_vector(p.n_dof, 1)
    z = inputs.uniform_vector(p.n_dof, 2)
    assert abs(x @ wrong_apply(z) - z @ wrong_apply(x)) > 1e-6


# ---- the training step (oracle/optim.py): each slip must trip a pin in tests/test_oracle_conv.py

def _adam(correct_m=True, correct_v=True, eps_inside=False, swap=False, t_shift=0):
    def step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
        if swap:
            b1, b2 = b2, b1
        p, g, m, v = (np.asarray(a, dtype=np.float64) for a in (p, g, m, v))
        m1 = b1 * m + (1.0 - b1) * g
        v1 = b2 * v + (1.0 - b2) * g * g
        m_hat = m1 / (1.0 - b1 ** (t + t_shift)) if correct_m else m1
        v_hat = v1 / (1.0 - b2 ** (t + t_shift)) if correct_v else v1
        den = np.sqrt(v_hat + eps) if eps_inside else np.sqrt(v_hat) + eps
        return p - lr * m_hat / den, m1, v1
    return step


@pytest.mark.parametrize("slip", [dict(correct_m=False), dict(correct_v=False), dict(eps_inside=True),
                                  dict(swap=True), dict(t_shift=1)],
                         ids=["no-m-correction", "no-v-correction", "eps-inside-sqrt", "swapped-betas",
                              "step-off-by-one"])
def test_adam_pins_catch(monkeypatch, slip):
    from oracle import optim
    from tests import test_oracle_conv
    monkeypatch.setattr(optim, "adam_step", _adam(**slip))
    with pytest.raises(AssertionError):
        test_oracle_conv.test_adam_closed_forms()


def test_adam_pins_pass_unmutated(monkeypatch):
    from oracle import optim
    from tests import test_oracle_conv
    monkeypatch.setattr(optim, "adam_step", _adam())
    test_oracle_conv.test_adam_closed_forms()


@pytest.mark.parametrize("slip", ["weights-swapped", "threshold-absolute", "nan-resets"])
def test_clip_pins_catch(monkeypatch, slip):
    from oracle import optim
    from tests import test_oracle_conv

    def clip(norm, ema, ratio=5.0):
        if not np.isfinite(norm):
            return (0.0, 0.0) if slip == "nan-resets" else (0.0, ema)
        limit = ratio if slip == "threshold-absolute" else ratio * ema
        scale = limit / norm if (ema > 0.0 and norm > limit) else 1.0
        used = norm * scale
        if ema <= 0.0:
            return scale, used
        return scale, (0.1 * ema + 0.9 * used if slip == "weights-swapped" else 0.9 * ema + 0.1 * used)
    monkeypatch.setattr(optim, "clip_scale", clip)
    with pytest.raises(AssertionError):
        test_oracle_conv.test_gradient_clip_special_cases()


# ---- the Krylov solvers (oracle/solvers.py): each slip must trip a pin in tests/test_oracle_pins.py

def _cg(slip):
    def cg(apply, b, rtol=1e-8, max_iter=2000, x0=None, dot=None):
        dot = dot or (lambda u, v: float(np.dot(u, v)))
        x = np.zeros_like(b)
        r = b.copy()
        p = r.copy()
        bn = np.sqrt(dot(b, b))
        rr = dot(r, r)
        hist, k = [np.sqrt(rr) / bn], 0
        while k < max_iter and np.isfinite(rr) and np.sqrt(rr) > rtol * bn:
            Ap = apply(p)
            alpha = rr / (dot(p, p) if slip == "alpha-without-A" else dot(p, Ap))
            x += alpha * p
            r_old = r.copy()
            r -= alpha * Ap
            rr_new = dot(r, r)
            beta = rr / rr_new if slip == "beta-inverted" else rr_new / rr
            p = (r_old if slip == "p-from-old-r" else r) + beta * p
            rr = rr_new
            k += 1
            hist.append(np.sqrt(rr) / bn)
        return x, k, hist
    return cg


@pytest.mark.parametrize("slip", ["alpha-without-A", "beta-inverted", "p-from-old-r"])
def test_cg_pins_catch(monkeypatch, slip):
    from oracle import solvers
    from tests import test_oracle_pins
    monkeypatch.setattr(solvers, "cg", _cg(slip))
    with pytest.raises(AssertionError):
        test_oracle_pins.test_cg_finite_termination_small_spd()
    with pytest.raises(AssertionError):
        test_oracle_pins.test_cg_matches_direct_solve_and_residual()


def test_cg_pins_pass_unmutated(monkeypatch):
    from oracle import solvers
    from tests import test_oracle_pins
    monkeypatch.setattr(solvers, "cg", _cg(None))
    test_oracle_pins.test_cg_finite_termination_small_spd()
    test_oracle_pins.test_cg_matches_direct_solve_and_residual()


def _fcg_m(slip):
    def fcg_m(apply, b, precond, m=8, rtol=1e-8, max_iter=2000, keep_directions=False):
        x = np.zeros_like(b)
        r = b.copy()
        bn = float(np.linalg.norm(b))
        stored, allpairs, hist, k = [], [], [1.0], 0
        while k < max_iter and np.linalg.norm(r) > rtol * bn:
            z = precond(r)
            p = z.copy()
            window = stored[-1:] if slip == "last-direction-only" else stored
            for pj, apj, dj in window:
                c = float(np.dot(z, apj)) / dj
                p = p + c * pj if slip == "sign" else p - c * pj
            Ap = apply(p)
            pAp = float(np.dot(p, Ap))
            alpha = float(np.dot(p, r)) / pAp
            x += alpha * p
            r -= alpha * Ap
            stored.append((p, Ap, pAp))
            if len(stored) > m:
                stored.pop(0)
            if keep_directions:
                allpairs.append((p, Ap))
            k += 1
            hist.append(float(np.linalg.norm(r)) / bn)
        return (x, k, hist, allpairs) if keep_directions else (x, k, hist)
    return fcg_m


@pytest.mark.parametrize("slip", ["last-direction-only", "sign"])
def test_fcg_m_pins_catch(monkeypatch, slip):
    from oracle import solvers
    from tests import test_oracle_pins
    monkeypatch.setattr(solvers, "fcg_m", _fcg_m(slip))
    with pytest.raises(AssertionError):
        test_oracle_pins.test_fcg_m_special_cases_and_orthogonality()


def test_pcg_with_r_dot_r_is_caught(monkeypatch):
    """PCG whose beta uses r.r instead of r.z: FCG(1) with the same fixed preconditioner no longer
    reproduces it."""
    from oracle import solvers
    from tests import test_oracle_pins

    def pcg(apply, b, precond, rtol=1e-8, max_iter=2000):
        x, r = np.zeros_like(b), b.copy()
        z = precond(r)
        p, bn, rz, rr = z.copy(), float(np.linalg.norm(b)), float(np.dot(r, z)), float(np.dot(r, r))
        hist, k = [1.0], 0
        while k < max_iter and np.linalg.norm(r) > rtol * bn:
            Ap = apply(p)
            alpha = rz / float(np.dot(p, Ap))
            x += alpha * p
            r -= alpha * Ap
            z = precond(r)
            rr_new = float(np.dot(r, r))
            p = z + (rr_new / rr) * p
            rz, rr = float(np.dot(r, z)), rr_new
            k += 1
            hist.append(float(np.linalg.norm(r)) / bn)
        return x, k, hist
    monkeypatch.setattr(solvers, "pcg", pcg)
    with pytest.raises(AssertionError):
        test_oracle_pins.test_fcg_m_special_cases_and_orthogonality()


def test_single_sync_without_alpha_correction_is_caught(monkeypatch):
    """Chronopoulos-Gear with alpha = gamma / delta at every step (the beta term of the denominator
    dropped)."""
    from oracle import solvers
    from tests import test_oracle_pins

    def css(apply, b, precond=None, rtol=1e-8, max_iter=2000):
        M = precond or (lambda v: v.copy())
        x, r = np.zeros_like(b), b.copy()
        p, s = np.zeros_like(b), np.zeros_like(b)
        bn = float(np.linalg.norm(b))
        u, gamma_prev, hist, k = M(r), None, [1.0], 0
        while k < max_iter and np.isfinite(np.linalg.norm(r)) and np.linalg.norm(r) > rtol * bn:
            w = apply(u)
            gamma, delta = float(np.dot(r, u)), float(np.dot(w, u))
            beta = 0.0 if k == 0 else gamma / gamma_prev
            alpha = gamma / delta
            p = u + beta * p
            s = w + beta * s
            x += alpha * p
            r -= alpha * s
            u = M(r)
            gamma_prev = gamma
            k += 1
            hist.append(float(np.linalg.norm(r)) / bn)
        return x, k, hist
    monkeypatch.setattr(solvers, "cg_single_sync", css)
    with pytest.raises(AssertionError):
        test_oracle_pins.test_single_sync_cg_pins()


# ---- the network's operations (oracle/conv.py): each slip must trip a pin in tests/test_oracle_conv.py

def _conv_flipped(x, w, b=None):
    """conv3d with the tap offsets mirrored (correlation with the flipped kernel)."""
    nz, ny, nx, _ = x.shape
    xp = np.pad(np.asarray(x, dtype=np.float64), ((1, 1), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((nz, ny, nx, w.shape[2]))
    for t in range(27):
        ox, oy, oz = 2 - t % 3, 2 - (t // 3) % 3, 2 - t // 9
        y += xp[oz:oz + nz, oy:oy + ny, ox:ox + nx, :] @ np.asarray(w[t], dtype=np.float64)
    return y + b if b is not None else y


def _dgrad_unflipped(dy, w):
    """dgrad taking dy at v + off instead of v - off."""
    nz, ny, nx, _ = dy.shape
    dyp = np.pad(np.asarray(dy, dtype=np.float64), ((1, 1), (1, 1), (1, 1), (0, 0)))
    dx = np.zeros((nz, ny, nx, w.shape[1]))
    for t in range(27):
        ox, oy, oz = t % 3, (t // 3) % 3, t // 9
        dx += dyp[oz:oz + nz, oy:oy + ny, ox:ox + nx, :] @ np.asarray(w[t], dtype=np.float64).T
    return dx


def _wgrad_flipped(x, dy):
    """wgrad with x taken at v - off."""
    nz, ny, nx, ci = x.shape
    xp = np.pad(np.asarray(x, dtype=np.float64), ((1, 1), (1, 1), (1, 1), (0, 0)))
    d = np.asarray(dy, dtype=np.float64).reshape(-1, dy.shape[3])
    dw = np.zeros((27, ci, dy.shape[3]))
    for t in range(27):
        ox, oy, oz = 2 - t % 3, 2 - (t // 3) % 3, 2 - t // 9
        dw[t] = xp[oz:oz + nz, oy:oy + ny, ox:ox + nx, :].reshape(-1, ci).T @ d
    return dw, d.sum(axis=0)


def _restrict_injection(x):
    return np.asarray(x, dtype=np.float64)[::2, ::2, ::2]


def _bf16_truncate(a):
    f = np.asarray(a, dtype=np.float32)
    return (f.view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32)


@pytest.mark.parametrize("name,fn,pin", [
    ("conv3d", _conv_flipped, "test_conv_brute_force_tiny"),
    ("conv3d_dgrad", _dgrad_unflipped, "test_dgrad_is_the_adjoint"),
    ("conv3d_wgrad", _wgrad_flipped, "test_wgrad_matches_directional_derivative"),
    ("restrict", _restrict_injection, "test_restriction_prolongation_pair"),
    ("bf16_round", _bf16_truncate, "test_bf16_rounding"),
], ids=["conv-taps-mirrored", "dgrad-not-mirrored", "wgrad-mirrored", "restrict-by-injection",
        "bf16-truncation"])
def test_conv_pins_catch(monkeypatch, name, fn, pin):
    from oracle import conv
    from tests import test_oracle_conv
    monkeypatch.setattr(conv, name, fn)
    with pytest.raises(AssertionError):
        getattr(test_oracle_conv, pin)()


def test_prolongation_weight_slip_is_caught(monkeypatch):
    """Trilinear interpolation without the factor 2 (plain transpose of full weighting)."""
    from oracle import conv
    from tests import test_oracle_conv
    orig = conv.prolong
    monkeypatch.setattr(conv, "prolong", lambda x: 0.5 * orig(x))
    with pytest.raises(AssertionError):
        test_oracle_conv.test_restriction_prolongation_pair()


# ---- the Q2 hexahedron (oracle/fem.py): each slip must trip a pin in tests/test_oracle_q2.py

def _gauss2_tensor():
    g = np.array([-1.0, 1.0]) / np.sqrt(3.0)
    q = np.arange(8)
    idx = np.stack([q % 2, (q // 2) % 2, q // 4], axis=1)
    return g[idx], np.ones(8)


def _gauss3_weights_misplaced():
    g1 = np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)])
    w1 = np.array([8.0, 5.0, 5.0]) / 9.0
    q = np.arange(27)
    idx = np.stack([q % 3, (q // 3) % 3, q // 9], axis=1)
    return g1[idx], w1[idx[:, 0]] * w1[idx[:, 1]] * w1[idx[:, 2]]


def _lagrange2_derivative_sign(t):
    L = np.stack([0.5 * t * (t - 1.0), 1.0 - t * t, 0.5 * t * (t + 1.0)], axis=-1)
    dL = np.stack([t + 0.5, -2.0 * t, t + 0.5], axis=-1)
    return L, dL


@pytest.mark.parametrize("name,fn,pin", [
    ("gauss3_points", _gauss2_tensor, "test_q2_box_element_is_kronecker_sum"),
    ("gauss3_points", _gauss3_weights_misplaced, "test_q2_box_element_is_kronecker_sum"),
    ("_lagrange2", _lagrange2_derivative_sign, "test_q2_shape_functions")],
    ids=["two-point-rule", "weights-misplaced", "derivative-sign"])
def test_q2_pins_catch(monkeypatch, name, fn, pin):
    from tests import test_oracle_q2
    monkeypatch.setattr(fem, name, fn)
    with pytest.raises(AssertionError):
        getattr(test_oracle_q2, pin)()
