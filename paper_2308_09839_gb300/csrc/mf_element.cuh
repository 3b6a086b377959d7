// Q1 reference element and the per-element arithmetic of Algorithm 1 (reference variant).
//
// Reference cube [-1, 1]^3; corner a has signs s_a = (+-1, +-1, +-1) with bit 0 -> xi, bit 1 -> eta,
// bit 2 -> zeta.  phi_a = 1/8 prod_d (1 + s_a,d xi_d); 2x2x2 Gauss points xi_q = s_q / sqrt(3),
// weights 1 (Sec. 2).  All loops are fully unrolled so every reference gradient below folds into
// an immediate constant (the "compile-time data-free element class" of Sec. 5).
#pragma once

#include <stdint.h>

namespace q1 {

constexpr double kG = 0.57735026918962576451;  // 1/sqrt(3)

__host__ __device__ constexpr double sgn(int a, int d) { return ((a >> d) & 1) ? 1.0 : -1.0; }

// d phi_a / d xi_j evaluated at Gauss point q.
__host__ __device__ constexpr double dN(int q, int a, int j) {
  return sgn(a, j) * 0.125 * (j == 0 ? 1.0 : 1.0 + sgn(a, 0) * sgn(q, 0) * kG) *
         (j == 1 ? 1.0 : 1.0 + sgn(a, 1) * sgn(q, 1) * kG) * (j == 2 ? 1.0 : 1.0 + sgn(a, 2) * sgn(q, 2) * kG);
}

// d phi_a / d xi_j at an arbitrary reference point.
__host__ __device__ inline double dN_at(const double xi[3], int a, int j) {
  double r = sgn(a, j) * 0.125;
  for (int d = 0; d < 3; ++d)
    if (d != j) r *= 1.0 + sgn(a, d) * xi[d];
  return r;
}

// Adjugate C = adj(J) (so J^{-1} = C / det J) and the determinant.
template <typename R>
__host__ __device__ __forceinline__ R adjugate(const R J[3][3], R C[3][3]) {
  C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  C[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  C[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  C[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  C[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  C[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  C[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  return J[0][0] * C[0][0] + J[0][1] * C[1][0] + J[0][2] * C[2][0];
}

// J_ij = sum_a X_a,i dphi_a/dxi_j at Gauss point q (Algorithm 1: J = sum_j x_j (x) grad_ref phi_j).
template <typename R, int Q>
__device__ __forceinline__ void jacobian(const R X[8][3], R J[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      R s = 0;
#pragma unroll
      for (int a = 0; a < 8; ++a) s += X[a][i] * (R)dN(Q, a, j);
      J[i][j] = s;
    }
}

// Scalar Laplace, Eq. 7 at one quadrature point:
//   v_a += grad_ref phi_a . J^{-1} (J^{-T} sum_b grad_ref phi_b u_b) w |J| kappa
// with J^{-1} = C/det:  flux = (kappa w / det) C C^T g.
template <typename R, int Q>
__device__ __forceinline__ void laplace_qp(const R X[8][3], const R u[8], R kappa, R v[8]) {
  R J[3][3], C[3][3];
  jacobian<R, Q>(X, J);
  const R det = adjugate(J, C);
  R g[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    R s = 0;
#pragma unroll
    for (int a = 0; a < 8; ++a) s += u[a] * (R)dN(Q, a, j);
    g[j] = s;
  }
  R t[3];  // C^T g
#pragma unroll
  for (int k = 0; k < 3; ++k) t[k] = C[0][k] * g[0] + C[1][k] * g[1] + C[2][k] * g[2];
  const R scale = kappa / det;  // w_q = 1
  R f[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) f[j] = scale * (C[j][0] * t[0] + C[j][1] * t[1] + C[j][2] * t[2]);
#pragma unroll
  for (int a = 0; a < 8; ++a) v[a] += (R)dN(Q, a, 0) * f[0] + (R)dN(Q, a, 1) * f[1] + (R)dN(Q, a, 2) * f[2];
}

template <typename R>
__device__ __forceinline__ void laplace_element(const R X[8][3], const R u[8], R kappa, R v[8]) {
#pragma unroll
  for (int a = 0; a < 8; ++a) v[a] = 0;
  laplace_qp<R, 0>(X, u, kappa, v);
  laplace_qp<R, 1>(X, u, kappa, v);
  laplace_qp<R, 2>(X, u, kappa, v);
  laplace_qp<R, 3>(X, u, kappa, v);
  laplace_qp<R, 4>(X, u, kappa, v);
  laplace_qp<R, 5>(X, u, kappa, v);
  laplace_qp<R, 6>(X, u, kappa, v);
  laplace_qp<R, 7>(X, u, kappa, v);
}

// Vector Laplace (Eq. 5) at one quadrature point: the flux of Eq. 7 for each of the three
// components, with the geometry (J, adj J, det J) shared between them.
template <typename R, int Q>
__device__ __forceinline__ void vector_laplace_qp(const R X[8][3], const R u[8][3], R kappa, R v[8][3]) {
  R J[3][3], C[3][3];
  jacobian<R, Q>(X, J);
  const R det = adjugate(J, C);
  const R scale = kappa / det;  // w_q = 1
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    R g[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      R s = 0;
#pragma unroll
      for (int a = 0; a < 8; ++a) s += u[a][k] * (R)dN(Q, a, j);
      g[j] = s;
    }
    R t[3], f[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) t[i] = C[0][i] * g[0] + C[1][i] * g[1] + C[2][i] * g[2];
#pragma unroll
    for (int j = 0; j < 3; ++j) f[j] = scale * (C[j][0] * t[0] + C[j][1] * t[1] + C[j][2] * t[2]);
#pragma unroll
    for (int a = 0; a < 8; ++a) v[a][k] += (R)dN(Q, a, 0) * f[0] + (R)dN(Q, a, 1) * f[1] + (R)dN(Q, a, 2) * f[2];
  }
}

template <typename R>
__device__ __forceinline__ void vector_laplace_element(const R X[8][3], const R u[8][3], R kappa, R v[8][3]) {
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k) v[a][k] = 0;
  vector_laplace_qp<R, 0>(X, u, kappa, v);
  vector_laplace_qp<R, 1>(X, u, kappa, v);
  vector_laplace_qp<R, 2>(X, u, kappa, v);
  vector_laplace_qp<R, 3>(X, u, kappa, v);
  vector_laplace_qp<R, 4>(X, u, kappa, v);
  vector_laplace_qp<R, 5>(X, u, kappa, v);
  vector_laplace_qp<R, 6>(X, u, kappa, v);
  vector_laplace_qp<R, 7>(X, u, kappa, v);
}

// Isotropic elasticity, Algorithm 1 at one quadrature point:
//   grad u = (sum_a u_a (x) grad_ref phi_a) J^{-1};  sigma = lam tr(eps) I + 2 mu eps, eps = sym grad u;
//   sigma *= w |J|;  P = sigma J^{-T};  v_a += P grad_ref phi_a.
// With J^{-1} = C/det:  grad u = H C / det and P = w sigma C^T (the det cancels).
template <typename R, int Q>
__device__ __forceinline__ void elasticity_qp(const R X[8][3], const R u[8][3], R lam, R mu, R v[8][3]) {
  R J[3][3], C[3][3];
  jacobian<R, Q>(X, J);
  const R det = adjugate(J, C);
  const R idet = (R)1 / det;
  R H[3][3];  // H_kj = sum_a u_a,k dphi_a/dxi_j
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      R s = 0;
#pragma unroll
      for (int a = 0; a < 8; ++a) s += u[a][k] * (R)dN(Q, a, j);
      H[k][j] = s;
    }
  R Gu[3][3];  // grad u = H C / det
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int l = 0; l < 3; ++l) Gu[k][l] = (H[k][0] * C[0][l] + H[k][1] * C[1][l] + H[k][2] * C[2][l]) * idet;
  const R tr = Gu[0][0] + Gu[1][1] + Gu[2][2];
  R S[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int l = 0; l < 3; ++l) S[k][l] = mu * (Gu[k][l] + Gu[l][k]) + (k == l ? lam * tr : (R)0);
  R P[3][3];  // w sigma C^T
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int j = 0; j < 3; ++j) P[k][j] = S[k][0] * C[j][0] + S[k][1] * C[j][1] + S[k][2] * C[j][2];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k) v[a][k] += P[k][0] * (R)dN(Q, a, 0) + P[k][1] * (R)dN(Q, a, 1) + P[k][2] * (R)dN(Q, a, 2);
}

template <typename R>
__device__ __forceinline__ void elasticity_element(const R X[8][3], const R u[8][3], R lam, R mu, R v[8][3]) {
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k) v[a][k] = 0;
  elasticity_qp<R, 0>(X, u, lam, mu, v);
  elasticity_qp<R, 1>(X, u, lam, mu, v);
  elasticity_qp<R, 2>(X, u, lam, mu, v);
  elasticity_qp<R, 3>(X, u, lam, mu, v);
  elasticity_qp<R, 4>(X, u, lam, mu, v);
  elasticity_qp<R, 5>(X, u, lam, mu, v);
  elasticity_qp<R, 6>(X, u, lam, mu, v);
  elasticity_qp<R, 7>(X, u, lam, mu, v);
}

}  // namespace q1
