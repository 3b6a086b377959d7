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
