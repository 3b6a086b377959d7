"""Plain numpy optimiser step of the learned preconditioner's training (TEST INFRASTRUCTURE).

Only the tests, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may use this module.

- ``adam_step``: Adam with bias correction, as Kingma & Ba (2015, Algorithm 1) state it, in float64.
- ``clip_scale``: the gradient-norm clip of ``mf_net_train_step`` as its documentation states it:
  the gradient is scaled down to at most ``ratio`` times an exponential moving average (weight 0.9)
  of the norms that earlier steps applied; the first step sets the average; a non-finite norm skips
  the step (scale 0) and leaves the average alone.  This rule is the library's own, not the paper's;
  its pins are special cases (below the threshold, at a multiple of it, the first step, a NaN).
"""
from __future__ import annotations

import math

import numpy as np


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step at step number t >= 1 on gradient g: returns (p', m', v').

    m' = b1 m + (1 - b1) g and v' = b2 v + (1 - b2) g^2 (elementwise), bias-corrected by
    1 - b1^t and 1 - b2^t, then p' = p - lr m_hat / (sqrt(v_hat) + eps)."""
    p, g, m, v = (np.asarray(a, dtype=np.float64) for a in (p, g, m, v))
    m1 = b1 * m + (1.0 - b1) * g
    v1 = b2 * v + (1.0 - b2) * g * g
    m_hat = m1 / (1.0 - b1 ** t)
    v_hat = v1 / (1.0 - b2 ** t)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m1, v1


def clip_scale(norm, ema, ratio=5.0):
    """The scale applied to a gradient of 2-norm `norm`, and the new moving average: returns
    (scale, ema').  `ema` = 0 means no earlier step."""
    if not math.isfinite(norm):
        return 0.0, ema
    scale = 1.0
    if ema > 0.0 and norm > ratio * ema:
        scale = ratio * ema / norm
    used = norm * scale
    return scale, (0.9 * ema + 0.1 * used if ema > 0.0 else used)
