"""Learned preconditioner workflow: training pairs from the FP64 CG solver, training of the network
on the GPU with the library's own kernels, and flexible CG with the trained network.

Training pairs (residual, error): for a seeded random exact solution x*, the right-hand side is
b = A x*; the FP64 (Jacobi-preconditioned) CG solver is run for k iterations (k drawn per pair),
and the pair is the residual r_k = b - A x_k and the error e_k = x* - x_k, which satisfy A e_k = r_k
exactly.  The network learns D^{-1/2} r -> D^{1/2} e in the symmetrically scaled variables (see
generate_pairs); the solver uses it as the smooth-error correction between damped-Jacobi
smoothing steps of a two-level preconditioner inside flexible CG.

The network is trained on random crops of (4m+1)^3 nodes (cheaper per step; the convolutions are
local) and its parameters are then copied into a network created for the full node grid.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import mf


def node_logk(mesh: mf.Mesh) -> torch.Tensor:
    """The network's second input channel: the node mean of log kappa (mf_node_logk, on the device;
    the flexible CG forms the same field)."""
    return mf.mf_node_logk(mesh)


def generate_pairs(mesh: mf.Mesh, p, n_pairs: int, seed: int = 0, k_range=(2, 150), smooth: int = 2,
                   keep_states: bool = False):
    """Training pairs on the device (float32 [n_pairs][n_nodes] each) and the output scale c.

    For a seeded random exact solution x* (white noise from a seeded device generator, smoothed 0 to
    `smooth` times by a periodic 7-point average: a random input field, not part of the method),
    b = A x* and the FP64 Jacobi-preconditioned CG solver runs k iterations (k log-uniform in
    k_range).  The library then forms (mf_training_pair) r = b - A x_k and e = x* - x_k in FP64 and,
    with D = diag(A), the pair D^-1/2 r / s -> D^1/2 e / s, s = RMS(D^-1/2 r) (the symmetrically
    scaled system's residual and error).  The targets are finally multiplied by c, the median of
    RMS(D^-1/2 r) / RMS(D^1/2 e) over the pairs, which makes them O(1).  keep_states: also return the
    (x*, x_k) of every pair (for tests)."""
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    n = p.n_dof
    dmask = torch.from_numpy(p.dirichlet.astype(bool)).cuda()
    R = torch.empty(n_pairs, n, dtype=torch.float32, device="cuda")
    T = torch.empty(n_pairs, n, dtype=torch.float32, device="cuda")
    ratios, states = [], []
    nzyx = (p.nz + 1, p.ny + 1, p.nx + 1)
    for i in range(n_pairs):
        xs = torch.randn(nzyx, dtype=torch.float64, device="cuda", generator=gen)
        for _ in range(int(rng.integers(0, smooth + 1))):
            xs = (xs + torch.roll(xs, 1, 0) + torch.roll(xs, -1, 0) + torch.roll(xs, 1, 1) + torch.roll(xs, -1, 1)
                  + torch.roll(xs, 1, 2) + torch.roll(xs, -1, 2)) / 7.0
        xs = xs.reshape(-1).contiguous()
        xs[dmask] = 0.0
        b = mesh.apply(xs)
        k = int(math.exp(rng.uniform(math.log(k_range[0]), math.log(k_range[1]))))
        # a fixed graph block of 16 iterations (the device-side iteration limit stops at k), so one
        # captured graph serves every pair
        xk, _ = mesh.cg(b, max_iter=k, rtol=1e-14, check_every=16, precond=mf.MF_PC_JACOBI)
        rr, ee = mf.mf_training_pair(mesh, b, xs, xk, R[i], T[i])
        ratios.append(math.sqrt(rr) / max(math.sqrt(ee), 1e-300))
        if keep_states:
            states.append((xs.clone(), xk.clone()))
    c = float(np.median(ratios))
    T *= c
    if keep_states:
        return R, T, c, states
    return R, T, c


def _crop(t, nzyx, origin, size):
    z0, y0, x0 = origin
    return t.view(*nzyx)[z0:z0 + size, y0:y0 + size, x0:x0 + size].contiguous().view(-1)


def train(R, E, logk, nzyx, crop: int = 33, steps: int = 2000, lr: float = 2e-4, seed: int = 0, log_every: int = 0,
          warmup: int = 100, stop_at: int | None = None, resume: dict | None = None):
    """Train a network on random crops of `crop`^3 nodes (the full grid when `crop` equals its size)
    with Adam, linear warm-up over `warmup` steps and cosine decay; returns (params, loss history,
    seconds).

    Checkpoints: with `stop_at` the run stops after that many steps and returns a checkpoint dict
    instead (the network's training state from mf_net_state_save, the crop generator's state, the
    step and the loss history so far; save_checkpoint / load_checkpoint write and read it as a .pt
    file).  `resume` continues such a checkpoint; the resumed run takes the same steps, bitwise, as a
    run that was never stopped."""
    assert (crop - 1) % 4 == 0
    rng = np.random.default_rng(seed)
    net = mf.Net(crop, crop, crop, seed=seed)
    start, hist = 0, []
    if resume is not None:
        assert resume["crop"] == crop and resume["steps"] == steps, "checkpoint of another run"
        net.load_state(resume["net_state"])
        rng.bit_generator.state = resume["rng"]
        start, hist = int(resume["step"]), list(resume["hist"])
    lk = torch.from_numpy(logk).cuda() if isinstance(logk, np.ndarray) else logk
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(start, steps):
        if stop_at is not None and s == stop_at:
            ckpt = {"net_state": net.state(), "rng": rng.bit_generator.state, "step": s, "hist": hist,
                    "crop": crop, "steps": steps}
            net.close()
            return ckpt
        i = int(rng.integers(0, R.shape[0]))
        origin = [int(rng.integers(0, (d - crop) // 4 + 1)) * 4 for d in nzyx]
        r = _crop(R[i], nzyx, origin, crop)
        k = _crop(lk, nzyx, origin, crop)
        e = _crop(E[i], nzyx, origin, crop)
        step_lr = lr * min(1.0, (s + 1) / max(warmup, 1)) * (0.5 * (1 + math.cos(math.pi * s / steps)))
        loss = net.train_step(r, k, e, step_lr)
        hist.append(loss)
        if log_every and s % log_every == 0:
            print(f"step {s} loss {loss:.4f}")
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    params = net.params()
    net.close()
    return params, hist, secs


def save_checkpoint(path: str, ckpt: dict) -> None:
    """Write a training checkpoint (train(..., stop_at=...)) to a .pt file."""
    torch.save({k: (torch.from_numpy(v) if isinstance(v, np.ndarray) else v) for k, v in ckpt.items()}, path)


def load_checkpoint(path: str) -> dict:
    """Read a checkpoint written by save_checkpoint.  It holds tensors and plain values only, so it is
    read with torch's weights-only loader: a file holding any other object is refused, not unpickled."""
    d = torch.load(path, weights_only=True)
    return {k: (v.numpy() if isinstance(v, torch.Tensor) else v) for k, v in d.items()}


def make_inference_net(params, nzyx, out_scale: float) -> mf.Net:
    nz, ny, nx = nzyx
    net = mf.Net(nx, ny, nz, seed=0)
    net.set_params(params)
    net.set_output_scale(out_scale)
    return net
