"""Exact rational integration of polynomials on the reference cube (test helper, independent of the
oracle): used to pin the oracle's element matrices on parallelepipeds, where the integrand is a
polynomial and the exact integral is a rational number."""
from fractions import Fraction
from itertools import product


def pmul(p, q):
    out = {}
    for (a, b), (c, d) in product(p.items(), q.items()):
        k = (a[0] + c[0], a[1] + c[1], a[2] + c[2])
        out[k] = out.get(k, 0) + b * d
    return out


def padd(p, q, s=1):
    out = dict(p)
    for k, v in q.items():
        out[k] = out.get(k, 0) + s * v
    return out


def pscale(p, s):
    return {k: v * s for k, v in p.items()}


def integrate(p):
    """Integral over [-1, 1]^3 of sum c x^i y^j z^k."""
    tot = Fraction(0)
    for (i, j, k), c in p.items():
        if i % 2 or j % 2 or k % 2:
            continue
        tot += c * Fraction(2, i + 1) * Fraction(2, j + 1) * Fraction(2, k + 1)
    return tot


def corner(a):
    return ((a & 1) * 2 - 1, ((a >> 1) & 1) * 2 - 1, ((a >> 2) & 1) * 2 - 1)


def ref_grad_poly(a, d):
    """d phi_a / d xi_d as a polynomial, phi_a = 1/8 prod (1 + s_i x_i)."""
    s = corner(a)
    p = {(0, 0, 0): Fraction(s[d], 8)}
    for i in range(3):
        if i == d:
            continue
        e = [0, 0, 0]
        e[i] = 1
        p = pmul(p, {(0, 0, 0): Fraction(1), tuple(e): Fraction(s[i])})
    return p


def ref_moments():
    """M[j][k][a][b] = int grad_ref_j phi_a grad_ref_k phi_b over [-1,1]^3 (exact)."""
    g = [[ref_grad_poly(a, d) for d in range(3)] for a in range(8)]
    return [[[[integrate(pmul(g[a][j], g[b][k])) for b in range(8)] for a in range(8)] for k in range(3)] for j in range(3)]


def inv3(J):
    a, b, c = J[0]
    d, e, f = J[1]
    g, h, i = J[2]
    det = a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g)
    adj = [[e * i - f * h, c * h - b * i, b * f - c * e],
           [f * g - d * i, a * i - c * g, c * d - a * f],
           [d * h - e * g, b * g - a * h, a * e - b * d]]
    return [[adj[r][s] / det for s in range(3)] for r in range(3)], det


def affine_laplace_exact(J, kappa):
    """Exact element matrix of kappa * int grad phi_a . grad phi_b over the image of [-1,1]^3 under
    x = x0 + J xi (J rational 3x3)."""
    M = ref_moments()
    Ji, det = inv3(J)
    # grad phi = J^{-T} grad_ref phi  ->  (grad phi)_i = sum_j Ji[j][i] gref_j
    A = [[Fraction(0)] * 8 for _ in range(8)]
    for a in range(8):
        for b in range(8):
            s = Fraction(0)
            for i in range(3):
                for j in range(3):
                    for k in range(3):
                        s += Ji[j][i] * Ji[k][i] * M[j][k][a][b]
            A[a][b] = kappa * abs(det) * s
    return A


def affine_elasticity_exact(J, lam, mu):
    """Exact 24x24 element matrix of isotropic elasticity on the parallelepiped x = x0 + J xi."""
    M = ref_moments()
    Ji, det = inv3(J)

    def phys(a, b, p, q):  # int d_p phi_a d_q phi_b
        s = Fraction(0)
        for j in range(3):
            for k in range(3):
                s += Ji[j][p] * Ji[k][q] * M[j][k][a][b]
        return s

    A = [[Fraction(0)] * 24 for _ in range(24)]
    for a in range(8):
        for b in range(8):
            gg = sum(phys(a, b, i, i) for i in range(3))
            for k in range(3):
                for l in range(3):
                    v = lam * phys(a, b, k, l) + mu * phys(a, b, l, k)
                    if k == l:
                        v += mu * gg
                    A[3 * a + k][3 * b + l] = abs(det) * v
    return A
