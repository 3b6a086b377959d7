"""Textbook Krylov loops on top of the oracle's operators (TEST INFRASTRUCTURE).

* ``cg``   unpreconditioned conjugate gradient (Hestenes-Stiefel) with exactly the vector operations
           the paper lists per iteration in Table 4: one operator apply, the dot p^T A p, the updates
           of x and r, the dot r^T r, and the update of p.
* ``pcg``  the same with a fixed preconditioner z = M(r) (Jacobi when M = diag(A)^-1).
* ``fcg``  flexible CG for a preconditioner that may change between iterations (a network):
           beta_k = z_{k+1}^T (r_{k+1} - r_k) / (z_k^T r_k)  (Polak-Ribiere form, Notay 2000).
* ``fcg_m``  truncated flexible CG, FCG(m) (Notay 2000): each new direction is the preconditioned
           residual A-orthogonalised against the last m directions.
* ``iterative_refinement``  x += solve_inner(b - A x) until the FP64 residual meets the tolerance.
* ``cg_single_sync``  the single-synchronisation CG of Chronopoulos and Gear (1989): both inner
           products of an iteration, gamma = r^T u and delta = w^T u with u = M r and w = A u, are
           taken together, and s = A p is carried by a recurrence.  In exact arithmetic it produces
           the iterates of ``pcg``.

Readings: x0 = 0; stop when ||r_k||_2 <= rtol ||b||_2 (the paper gives no stopping norm); the
iteration count is the number of operator applies inside the loop.
"""
from __future__ import annotations

import math

import numpy as np


def cg(apply, b, rtol=1e-8, max_iter=100000, x0=None, dot=None):
    """Returns (x, iterations, residual history ||r_k||/||b||)."""
    dot = dot or (lambda u, v: float(np.dot(u, v)))
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply(x) if x0 is not None else b.copy()
    p = r.copy()
    bn = math.sqrt(dot(b, b))
    if bn == 0.0:
        return x, 0, [0.0]
    rr = dot(r, r)
    hist = [math.sqrt(rr) / bn]
    k = 0
    while k < max_iter and math.sqrt(rr) > rtol * bn:
        Ap = apply(p)
        pAp = dot(p, Ap)
        if not pAp > 0.0:
            raise FloatingPointError("CG breakdown: p^T A p <= 0")
        alpha = rr / pAp
        x += alpha * p
        r -= alpha * Ap
        rr_new = dot(r, r)
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        k += 1
        hist.append(math.sqrt(rr) / bn)
    return x, k, hist


def pcg(apply, b, precond, rtol=1e-8, max_iter=100000):
    """Preconditioned CG with a fixed symmetric preconditioner z = precond(r)."""
    x = np.zeros_like(b)
    r = b.copy()
    z = precond(r)
    p = z.copy()
    bn = float(np.linalg.norm(b))
    rz = float(np.dot(r, z))
    k = 0
    hist = [1.0]
    while k < max_iter and np.linalg.norm(r) > rtol * bn:
        Ap = apply(p)
        alpha = rz / float(np.dot(p, Ap))
        x += alpha * p
        r -= alpha * Ap
        z = precond(r)
        rz_new = float(np.dot(r, z))
        p = z + (rz_new / rz) * p
        rz = rz_new
        k += 1
        hist.append(float(np.linalg.norm(r)) / bn)
    return x, k, hist


def fcg(apply, b, precond, rtol=1e-8, max_iter=100000):
    """Flexible CG (Polak-Ribiere beta).  With precond = identity the iterates are CG's up to rounding."""
    x = np.zeros_like(b)
    r = b.copy()
    z = precond(r)
    p = z.copy()
    bn = float(np.linalg.norm(b))
    rz = float(np.dot(r, z))
    k = 0
    hist = [1.0]
    while k < max_iter and np.linalg.norm(r) > rtol * bn:
        Ap = apply(p)
        alpha = rz / float(np.dot(p, Ap))
        x += alpha * p
        r_old = r.copy()
        r -= alpha * Ap
        z = precond(r)
        beta = float(np.dot(z, r - r_old)) / rz
        rz = float(np.dot(r, z))
        p = z + beta * p
        k += 1
        hist.append(float(np.linalg.norm(r)) / bn)
    return x, k, hist


def fcg_m(apply, b, precond, m=8, rtol=1e-8, max_iter=100000, keep_directions=False):
    """Truncated flexible CG, FCG(m): z_k = M(r_k); p_k = z_k - sum over the last m directions j of
    (z_k . A p_j) / (p_j . A p_j) p_j; alpha_k = (p_k . r_k) / (p_k . A p_k); x += alpha_k p_k and
    r -= alpha_k A p_k.  Returns (x, iterations, residual history[, all (p, Ap) pairs])."""
    x = np.zeros_like(b)
    r = b.copy()
    bn = float(np.linalg.norm(b))
    stored = []  # (p_j, A p_j, p_j . A p_j), oldest first
    allpairs = []
    k = 0
    hist = [1.0]
    while k < max_iter and np.linalg.norm(r) > rtol * bn:
        z = precond(r)
        p = z.copy()
        for pj, apj, dj in stored:
            p -= float(np.dot(z, apj)) / dj * pj
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


def iterative_refinement(apply64, inner_solve, b, rtol=1e-10, max_outer=50):
    """x_{m+1} = x_m + d_m with d_m ~ A^{-1} (b - A x_m) from a lower-precision inner solve.
    Returns (x, outer iterations, history of the FP64 relative residual)."""
    x = np.zeros_like(b)
    bn = float(np.linalg.norm(b))
    r = b.copy()
    hist = [1.0]
    m = 0
    while m < max_outer and np.linalg.norm(r) > rtol * bn:
        x = x + inner_solve(r)
        r = b - apply64(x)
        m += 1
        hist.append(float(np.linalg.norm(r)) / bn)
    return x, m, hist


def cg_single_sync(apply, b, precond=None, rtol=1e-8, max_iter=100000):
    """Chronopoulos-Gear CG, x0 = 0; precond(r) = M r (None: identity).  Returns (x, iterations,
    residual history).  Iteration k: u_k = M r_k, w_k = A u_k, gamma_k = r_k.u_k, delta_k = w_k.u_k;
    beta_k = gamma_k / gamma_{k-1} (beta_0 = 0), alpha_k = gamma_k / (delta_k - beta_k gamma_k /
    alpha_{k-1}) (alpha_0 = gamma_0 / delta_0); p_k = u_k + beta_k p_{k-1}, s_k = w_k + beta_k
    s_{k-1}; x_{k+1} = x_k + alpha_k p_k, r_{k+1} = r_k - alpha_k s_k."""
    M = precond or (lambda v: v.copy())
    x = np.zeros_like(b)
    r = b.copy()
    p = np.zeros_like(b)
    s = np.zeros_like(b)
    bn = float(np.linalg.norm(b))
    if bn == 0.0:
        return x, 0, [0.0]
    u = M(r)
    gamma_prev = alpha_prev = None
    k = 0
    hist = [1.0]
    while k < max_iter and np.linalg.norm(r) > rtol * bn:
        w = apply(u)
        gamma = float(np.dot(r, u))
        delta = float(np.dot(w, u))
        if k == 0:
            beta, alpha = 0.0, gamma / delta
        else:
            beta = gamma / gamma_prev
            alpha = gamma / (delta - beta * gamma / alpha_prev)
        if not alpha > 0.0:
            raise FloatingPointError("single-synchronisation CG breakdown")
        p = u + beta * p
        s = w + beta * s
        x += alpha * p
        r -= alpha * s
        u = M(r)
        gamma_prev, alpha_prev = gamma, alpha
        k += 1
        hist.append(float(np.linalg.norm(r)) / bn)
    return x, k, hist

