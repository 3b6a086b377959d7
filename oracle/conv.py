"""Plain CPU reference of the learned preconditioner's network operations (TEST INFRASTRUCTURE).

The paper names matrix-free preconditioners as future work (Sec. 7) and has no network; these are
the textbook definitions of the operations the library's network uses, written out in numpy
(float64 unless stated), against which the BF16 tensor-core kernels are checked:

* 3x3x3 convolution, zero padding, stride 1, channels-last [z][y][x][C], weights [27][Cin][Cout]
  with tap t = dx + 3 dy + 9 dz for offsets (dx-1, dy-1, dz-1);
* its input gradient (the adjoint: correlation with the mirrored, transposed kernel) and its weight
  and bias gradients;
* full-weighting restriction from a (2m+1)^3 node grid to (m+1)^3 and its adjoint, trilinear
  prolongation (each coarse node i maps to fine node 2i).
"""
from __future__ import annotations

import numpy as np


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (round to nearest even) and return them as float32."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _pad(x):
    return np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))


def conv3d(x, w, b=None):
    """y[v, co] = b[co] + sum_t sum_ci w[t, ci, co] x[v + off_t, ci]."""
    nz, ny, nx, _ = x.shape
    xp = _pad(np.asarray(x, dtype=np.float64))
    y = np.zeros((nz, ny, nx, w.shape[2]))
    for t in range(27):
        dx, dy, dz = t % 3, (t // 3) % 3, t // 9
        y += xp[dz:dz + nz, dy:dy + ny, dx:dx + nx, :] @ np.asarray(w[t], dtype=np.float64)
    if b is not None:
        y += b
    return y


def conv3d_dgrad(dy, w):
    """dx[v, ci] = sum_t sum_co w[t, ci, co] dy[v - off_t, co]  (adjoint of conv3d in x)."""
    nz, ny, nx, _ = dy.shape
    dyp = _pad(np.asarray(dy, dtype=np.float64))
    dx = np.zeros((nz, ny, nx, w.shape[1]))
    for t in range(27):
        ox, oy, oz = t % 3, (t // 3) % 3, t // 9
        # v - off_t with off = (ox-1, oy-1, oz-1) -> slice start 2 - o in the padded array
        dx += dyp[2 - oz:2 - oz + nz, 2 - oy:2 - oy + ny, 2 - ox:2 - ox + nx, :] @ np.asarray(w[t], dtype=np.float64).T
    return dx


def conv3d_wgrad(x, dy):
    """dw[t, ci, co] = sum_v x[v + off_t, ci] dy[v, co];  db[co] = sum_v dy[v, co]."""
    nz, ny, nx, ci = x.shape
    xp = _pad(np.asarray(x, dtype=np.float64))
    d = np.asarray(dy, dtype=np.float64).reshape(-1, dy.shape[3])
    dw = np.zeros((27, ci, dy.shape[3]))
    for t in range(27):
        ox, oy, oz = t % 3, (t // 3) % 3, t // 9
        xs = xp[oz:oz + nz, oy:oy + ny, ox:ox + nx, :].reshape(-1, ci)
        dw[t] = xs.T @ d
    return dw, d.sum(axis=0)


def _fw_1d(n_fine):
    """1-D full-weighting restriction matrix (m+1) x (2m+1): weights 1/4, 1/2, 1/4."""
    m = (n_fine - 1) // 2
    R = np.zeros((m + 1, n_fine))
    for i in range(m + 1):
        for d, wgt in ((-1, 0.25), (0, 0.5), (1, 0.25)):
            j = 2 * i + d
            if 0 <= j < n_fine:
                R[i, j] += wgt
    return R


def restrict(x):
    """Full weighting in each direction on a (2m+1)^3 node grid, channels-last."""
    Rz, Ry, Rx = (_fw_1d(s) for s in x.shape[:3])
    return np.einsum("az,by,cx,zyxk->abck", Rz, Ry, Rx, np.asarray(x, dtype=np.float64))


def prolong(x):
    """Trilinear interpolation (m+1)^3 -> (2m+1)^3: the transpose of full weighting times 2 per axis."""
    Pz, Py, Px = (2.0 * _fw_1d(2 * s - 1).T for s in x.shape[:3])
    return np.einsum("za,yb,xc,abck->zyxk", Pz, Py, Px, np.asarray(x, dtype=np.float64))
