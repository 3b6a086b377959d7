// Linear tetrahedra (P1), the simplex elements that Sec. 7 names as future work: the element
// integrals of Eqs. 1-3 (Laplace, vector Laplace, isotropic elasticity) on the reference
// tetrahedron {xi_k >= 0, xi + eta + zeta <= 1} with phi_0 = 1 - xi - eta - zeta, phi_k = xi_k.
//
// The gradients are constant over the element, so the one-point rule with weight 1/6 (the
// reference volume) is exact.  With edges e_k = x_k - x_0 (k = 1..3), D = det[e1 e2 e3] = 6 |T| and
// the scaled gradients n_a = D grad phi_a:
//   n_1 = e2 x e3,  n_2 = e3 x e1,  n_3 = e1 x e2,  n_0 = -(n_1 + n_2 + n_3).
// Laplace (Eq. 1):     A_ab = kappa |T| grad phi_a . grad phi_b = kappa n_a . n_b / (6 D).
// Elasticity (Eq. 3):  A_{3a+k,3b+l} = [lam n_ak n_bl + mu (n_al n_bk + delta_kl n_a . n_b)] / (6 D).
// Matrix-free, with H = sum_b u_b (x) n_b (= D grad u) and S = lam tr(H) I + mu (H + H^T) (= D sigma):
//   v_a = kappa n_a . (sum_b u_b n_b) / (6 D)   and   v_a = S n_a / (6 D).
// sum_b u_b n_b is formed as sum_{k=1..3} (u_k - u_0) n_k, which is the same sum (n_0 = -sum n_k).
#pragma once

#include "mf_internal.cuh"

namespace p1 {

template <typename R>
__device__ __forceinline__ void cross(const R a[3], const R b[3], R c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// Scaled gradients n[4][3] and D = 6 |T| of the tetrahedron with vertices X[4][3].
template <typename R>
__device__ __forceinline__ R geometry(const R X[4][3], R n[4][3]) {
  R e[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) e[k][i] = X[k + 1][i] - X[0][i];
  cross(e[1], e[2], n[1]);
  cross(e[2], e[0], n[2]);
  cross(e[0], e[1], n[3]);
#pragma unroll
  for (int i = 0; i < 3; ++i) n[0][i] = -(n[1][i] + n[2][i] + n[3][i]);
  return e[0][0] * n[1][0] + e[0][1] * n[1][1] + e[0][2] * n[1][2];
}

// v = A^e u, scalar Laplace (one component of the vector Laplacian).
template <typename R>
__device__ __forceinline__ void laplace(const R n[4][3], R D, R kappa, const R u[4], R v[4]) {
  R t[3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
    t[i] = (u[1] - u[0]) * n[1][i] + (u[2] - u[0]) * n[2][i] + (u[3] - u[0]) * n[3][i];
  const R c = kappa / (R(6) * D);
#pragma unroll
  for (int a = 0; a < 4; ++a) v[a] = c * (n[a][0] * t[0] + n[a][1] * t[1] + n[a][2] * t[2]);
}

// v = A^e u, isotropic elasticity (u, v xyz-interleaved per node).
template <typename R>
__device__ __forceinline__ void elasticity(const R n[4][3], R D, R lam, R mu, const R u[4][3], R v[4][3]) {
  R H[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      H[k][j] = (u[1][k] - u[0][k]) * n[1][j] + (u[2][k] - u[0][k]) * n[2][j] + (u[3][k] - u[0][k]) * n[3][j];
  const R tr = H[0][0] + H[1][1] + H[2][2];
  R S[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int l = 0; l < 3; ++l) S[k][l] = mu * (H[k][l] + H[l][k]) + (k == l ? lam * tr : R(0));
  const R c = R(1) / (R(6) * D);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k) v[a][k] = c * (S[k][0] * n[a][0] + S[k][1] * n[a][1] + S[k][2] * n[a][2]);
}

// Row block of node a of A^e: out[k][b][l] = A^e_{ND a + k, ND b + l} (Laplace: out[0][b][0]).
template <int PHYS>
__device__ __forceinline__ void element_rows(const double n[4][3], double D, int a, double c0, double c1,
                                             double out[][4][3]) {
  const double c = 1.0 / (6.0 * D);
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const double nn = n[a][0] * n[b][0] + n[a][1] * n[b][1] + n[a][2] * n[b][2];
    if (PHYS == MF_LAPLACE) {
      out[0][b][0] = c0 * nn * c;
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l)
          out[k][b][l] = c * (c0 * n[a][k] * n[b][l] + c1 * (n[a][l] * n[b][k] + (k == l ? nn : 0.0)));
    }
  }
}

// Node ids of tetrahedron e (connectivity [E][4]).
__device__ __forceinline__ void nodes_of(const int32_t *__restrict__ cells, int64_t e, int64_t nodes[4]) {
  const int4 c = __ldg(reinterpret_cast<const int4 *>(cells) + e);
  nodes[0] = c.x;
  nodes[1] = c.y;
  nodes[2] = c.z;
  nodes[3] = c.w;
}

}  // namespace p1
