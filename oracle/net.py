"""Plain numpy forward and backward of the learned preconditioner's network (TEST INFRASTRUCTURE).

The same architecture as the library's network, composed from the textbook operations of
``oracle/conv.py`` in float64.  With ``bf16=True`` the weights and every stored activation and
gradient are rounded to bfloat16 where the GPU stores them in bfloat16, so the two can be compared
closely; with ``bf16=False`` it is the exact real-arithmetic network (used for finite differences).

Flat parameter layout: for each layer in order (e0, e1, e2, m2, d1, q1, d0, out) the weights
[27][Cin][Cout] followed by the bias [Cout].
"""
from __future__ import annotations

import numpy as np

from . import conv

# (level, cin, cout, relu): e0, e1, e2, m2, d1, q1, d0, out
LAYERS = [(0, 2, 16, 1), (1, 16, 32, 1), (2, 32, 64, 1), (2, 64, 64, 1),
          (1, 64, 32, 1), (1, 32, 16, 1), (0, 16, 16, 1), (0, 16, 1, 0)]


def num_params() -> int:
    return sum(27 * ci * co + co for _, ci, co, _ in LAYERS)


def unpack(p):
    out, off = [], 0
    for _, ci, co, _ in LAYERS:
        w = p[off:off + 27 * ci * co].reshape(27, ci, co)
        off += 27 * ci * co
        b = p[off:off + co]
        off += co
        out.append((w, b))
    return out


def _r(a, on):
    return conv.bf16_round(a).astype(np.float64) if on else np.asarray(a, dtype=np.float64)


def forward(p, inp, bf16=True):
    """inp: [z][y][x][2] (residual, log kappa).  Returns (output [z][y][x], cache)."""
    P = unpack(np.asarray(p, dtype=np.float64))
    Wb = [(_r(w, bf16), np.asarray(b, dtype=np.float64)) for w, b in P]
    c = {}
    c["in0"] = _r(inp, bf16)
    relu = lambda a: np.maximum(a, 0.0)
    c["e0"] = _r(relu(conv.conv3d(c["in0"], *Wb[0])), bf16)
    c["r0"] = _r(conv.restrict(c["e0"]), bf16)
    c["e1"] = _r(relu(conv.conv3d(c["r0"], *Wb[1])), bf16)
    c["r1"] = _r(conv.restrict(c["e1"]), bf16)
    c["e2"] = _r(relu(conv.conv3d(c["r1"], *Wb[2])), bf16)
    c["m2"] = _r(relu(conv.conv3d(c["e2"], *Wb[3])), bf16)
    c["p1"] = _r(conv.prolong(c["m2"]), bf16)
    c["d1"] = _r(relu(conv.conv3d(c["p1"], *Wb[4]) + c["e1"]), bf16)
    c["q1"] = _r(relu(conv.conv3d(c["d1"], *Wb[5])), bf16)
    c["p0"] = _r(conv.prolong(c["q1"]), bf16)
    c["d0"] = _r(relu(conv.conv3d(c["p0"], *Wb[6]) + c["e0"]), bf16)
    out = conv.conv3d(c["d0"], *Wb[7])[..., 0]
    c["W"] = Wb
    return out, c


def loss_and_grad(p, inp, target, bf16=True):
    """Relative squared error and its gradient with respect to the flat parameters."""
    out, c = forward(p, inp, bf16)
    den = float(np.sum(target * target))
    loss = float(np.sum((out - target) ** 2)) / den
    g_out = _r((2.0 * (out - target) / den)[..., None], bf16)
    Wb = c["W"]
    grads = [None] * len(LAYERS)

    def back(l, x_in, gpre, need_in=True):
        dw, db = conv.conv3d_wgrad(x_in, gpre)
        grads[l] = (dw, db)
        return conv.conv3d_dgrad(gpre, Wb[l][0]) if need_in else None

    mask = lambda g, a: np.where(a > 0, g, 0.0)
    g = _r(back(7, c["d0"], g_out), bf16)
    gpre6 = mask(g, c["d0"])
    g_e0 = gpre6
    g = _r(back(6, c["p0"], gpre6), bf16)
    g = _r(8.0 * conv.restrict(g), bf16)
    gpre5 = mask(g, c["q1"])
    g = _r(back(5, c["d1"], gpre5), bf16)
    gpre4 = mask(g, c["d1"])
    g_e1 = gpre4
    g = _r(back(4, c["p1"], gpre4), bf16)
    g = _r(8.0 * conv.restrict(g), bf16)
    gpre3 = mask(g, c["m2"])
    g = _r(back(3, c["e2"], gpre3), bf16)
    gpre2 = mask(g, c["e2"])
    g = _r(back(2, c["r1"], gpre2), bf16)
    g_e1 = _r(g_e1 + _r(conv.prolong(g) / 8.0, bf16), bf16)
    gpre1 = mask(g_e1, c["e1"])
    g = _r(back(1, c["r0"], gpre1), bf16)
    g_e0 = _r(g_e0 + _r(conv.prolong(g) / 8.0, bf16), bf16)
    gpre0 = mask(g_e0, c["e0"])
    back(0, c["in0"], gpre0, need_in=False)
    flat = np.concatenate([np.concatenate([dw.reshape(-1), db]) for dw, db in grads])
    return loss, flat, out
