// Triquadratic hexahedra (Q2, 27 nodes), the higher-order elements that Sec. 7 names as future
// work: the element integrals of Eqs. 4-6 with the isoparametric Q2 map and the 3x3x3 Gauss rule.
//
// Node a = i + 3 j + 9 k (i, j, k in {0, 1, 2}) sits at reference coordinates (i - 1, j - 1, k - 1);
// phi_a = L_i(xi) L_j(eta) L_k(zeta) with L_0(t) = t (t - 1) / 2, L_1(t) = 1 - t^2,
// L_2(t) = t (t + 1) / 2.  Gauss points 0 and +-sqrt(3/5) with weights 8/9 and 5/9 per direction;
// point q = i + 3 j + 9 k likewise.  Per quadrature point the arithmetic is that of Algorithm 1
// (J, adj J, det J; the flux or the stress), here over 27 nodes: one thread per element, the
// quadrature loop kept rolled (the 27 x 27 reference gradients are formed from the 1D tables).
#pragma once

#include "mf_element.cuh"
#include "mf_internal.cuh"

namespace q2 {

constexpr double kG3 = 0.77459666924148337704;  // sqrt(3/5)

__host__ __device__ __forceinline__ double gauss_point(int i) { return i == 0 ? -kG3 : (i == 1 ? 0.0 : kG3); }
__host__ __device__ __forceinline__ double gauss_weight(int i) { return i == 1 ? 8.0 / 9.0 : 5.0 / 9.0; }

// 1D quadratic Lagrange values and derivatives at t, per direction.
template <typename R>
struct Tab {
  R L[3][3], dL[3][3];  // [direction][node index]
};

template <typename R>
__device__ __forceinline__ void tables_at(const double xi[3], Tab<R> &t) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double s = xi[d];
    t.L[d][0] = (R)(0.5 * s * (s - 1.0));
    t.L[d][1] = (R)(1.0 - s * s);
    t.L[d][2] = (R)(0.5 * s * (s + 1.0));
    t.dL[d][0] = (R)(s - 0.5);
    t.dL[d][1] = (R)(-2.0 * s);
    t.dL[d][2] = (R)(s + 0.5);
  }
}

// Reference gradient of node a from the tables.
template <typename R>
__device__ __forceinline__ void ref_grad(const Tab<R> &t, int a, R g[3]) {
  const int i = a % 3, j = (a / 3) % 3, k = a / 9;
  g[0] = t.dL[0][i] * t.L[1][j] * t.L[2][k];
  g[1] = t.L[0][i] * t.dL[1][j] * t.L[2][k];
  g[2] = t.L[0][i] * t.L[1][j] * t.dL[2][k];
}

// J_rc = sum_a X_a,r dphi_a/dxi_c at the point of the tables.
template <typename R>
__device__ __forceinline__ void jacobian(const R X[27][3], const Tab<R> &t, R J[3][3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) J[r][c] = 0;
#pragma unroll
  for (int a = 0; a < 27; ++a) {
    R g[3];
    ref_grad(t, a, g);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) J[r][c] += X[a][r] * g[c];
  }
}

__device__ __forceinline__ void point_q(int q, double xi[3]) {
  xi[0] = gauss_point(q % 3);
  xi[1] = gauss_point((q / 3) % 3);
  xi[2] = gauss_point(q / 9);
}

__device__ __forceinline__ double weight_q(int q) {
  return gauss_weight(q % 3) * gauss_weight((q / 3) % 3) * gauss_weight(q / 9);
}

// v = A^e u for NC components: the scalar Laplace flux per component (Eq. 4 / Eq. 5), or
// elasticity (Eq. 6, Algorithm 1) when ELAST.
template <typename R, int NC, bool ELAST>
__device__ void element_apply(const R X[27][3], const R u[27][NC], R c0, R c1, R v[27][NC]) {
#pragma unroll
  for (int a = 0; a < 27; ++a)
#pragma unroll
    for (int k = 0; k < NC; ++k) v[a][k] = 0;
#pragma unroll 1
  for (int q = 0; q < 27; ++q) {
    double xi[3];
    point_q(q, xi);
    Tab<R> t;
    tables_at<R>(xi, t);
    R J[3][3], C[3][3];
    jacobian(X, t, J);
    const R det = q1::adjugate(J, C);
    const R w = (R)weight_q(q);
    R H[NC][3];  // H_kj = sum_a u_a,k dphi_a/dxi_j
#pragma unroll
    for (int k = 0; k < NC; ++k)
#pragma unroll
      for (int j = 0; j < 3; ++j) H[k][j] = 0;
#pragma unroll
    for (int a = 0; a < 27; ++a) {
      R g[3];
      ref_grad(t, a, g);
#pragma unroll
      for (int k = 0; k < NC; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) H[k][j] += u[a][k] * g[j];
    }
    R P[NC][3];  // v_a,k += sum_j P_kj dphi_a/dxi_j
    if constexpr (ELAST) {
      const R idet = (R)1 / det;
      R G[3][3];  // grad u = H C / det
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) G[k][l] = (H[k][0] * C[0][l] + H[k][1] * C[1][l] + H[k][2] * C[2][l]) * idet;
      const R tr = G[0][0] + G[1][1] + G[2][2];
      R S[3][3];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) S[k][l] = w * (c1 * (G[k][l] + G[l][k]) + (k == l ? c0 * tr : (R)0));
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) P[k % NC][j] = S[k][0] * C[j][0] + S[k][1] * C[j][1] + S[k][2] * C[j][2];
    } else {
      const R scale = w * c0 / det;  // flux = (w kappa / det) C C^T g
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        R tt[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) tt[i] = C[0][i] * H[k][0] + C[1][i] * H[k][1] + C[2][i] * H[k][2];
#pragma unroll
        for (int j = 0; j < 3; ++j) P[k][j] = scale * (C[j][0] * tt[0] + C[j][1] * tt[1] + C[j][2] * tt[2]);
      }
    }
#pragma unroll
    for (int a = 0; a < 27; ++a) {
      R g[3];
      ref_grad(t, a, g);
#pragma unroll
      for (int k = 0; k < NC; ++k) v[a][k] += P[k][0] * g[0] + P[k][1] * g[1] + P[k][2] * g[2];
    }
  }
}

// Row block of node a of A^e (FP64): out[k][b][l] = A^e_{NE a + k, NE b + l}.
template <int PHYS>
__device__ void element_rows(const double X[27][3], int a, double c0, double c1, double out[][27][3]) {
  constexpr int NE = PHYS == MF_ELASTICITY ? 3 : 1;
  for (int k = 0; k < NE; ++k)
    for (int b = 0; b < 27; ++b)
      for (int l = 0; l < 3; ++l) out[k][b][l] = 0.0;
  for (int q = 0; q < 27; ++q) {
    double xi[3];
    point_q(q, xi);
    Tab<double> t;
    tables_at<double>(xi, t);
    double J[3][3], C[3][3];
    jacobian(X, t, J);
    const double det = q1::adjugate(J, C);
    const double wd = weight_q(q) * det;
    double ga[3], r[3];
    ref_grad(t, a, r);
    for (int i = 0; i < 3; ++i) ga[i] = (C[0][i] * r[0] + C[1][i] * r[1] + C[2][i] * r[2]) / det;
    for (int b = 0; b < 27; ++b) {
      double gb[3];
      ref_grad(t, b, r);
      for (int i = 0; i < 3; ++i) gb[i] = (C[0][i] * r[0] + C[1][i] * r[1] + C[2][i] * r[2]) / det;
      const double gg = ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2];
      if (PHYS != MF_ELASTICITY) {
        out[0][b][0] += c0 * gg * wd;
      } else {
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l)
            out[k][b][l] += wd * (c0 * ga[k] * gb[l] + c1 * (ga[l] * gb[k] + (k == l ? gg : 0.0)));
      }
    }
  }
}

// Diagonal of A^e for all nodes: out[a][k] (FP64).
template <int PHYS>
__device__ void element_diag(const double X[27][3], double c0, double c1, double out[27][3]) {
  for (int a = 0; a < 27; ++a)
    for (int k = 0; k < 3; ++k) out[a][k] = 0.0;
  for (int q = 0; q < 27; ++q) {
    double xi[3];
    point_q(q, xi);
    Tab<double> t;
    tables_at<double>(xi, t);
    double J[3][3], C[3][3];
    jacobian(X, t, J);
    const double det = q1::adjugate(J, C);
    const double wd = weight_q(q) * det;
    for (int a = 0; a < 27; ++a) {
      double r[3], ga[3];
      ref_grad(t, a, r);
      for (int i = 0; i < 3; ++i) ga[i] = (C[0][i] * r[0] + C[1][i] * r[1] + C[2][i] * r[2]) / det;
      const double gg = ga[0] * ga[0] + ga[1] * ga[1] + ga[2] * ga[2];
      if (PHYS != MF_ELASTICITY) out[a][0] += c0 * gg * wd;
      else
        for (int k = 0; k < 3; ++k) out[a][k] += wd * (c0 * ga[k] * ga[k] + c1 * (ga[k] * ga[k] + gg));
    }
  }
}

// det J > 0 and finite at the 27 Gauss points and the 8 vertices.
__device__ inline bool dets_positive(const double X[27][3]) {
  bool ok = true;
  for (int p = 0; p < 35; ++p) {
    double xi[3];
    if (p < 27) {
      point_q(p, xi);
    } else {
      const int c = p - 27;
      xi[0] = (c & 1) ? 1.0 : -1.0;
      xi[1] = (c & 2) ? 1.0 : -1.0;
      xi[2] = (c & 4) ? 1.0 : -1.0;
    }
    Tab<double> t;
    tables_at<double>(xi, t);
    double J[3][3], C[3][3];
    jacobian(X, t, J);
    const double det = q1::adjugate(J, C);
    if (!(det > 0.0) || !isfinite(det)) ok = false;
  }
  return ok;
}


// ------------------------------------------------------------------------------------------------
// Partial assembly with sum factorisation (Laplace and vector Laplace on Q2 meshes).  Per element and
// Gauss point the symmetric flux matrix D_q = (w_q kappa / det J) adj(J) adj(J)^T (6 values) is
// computed once in FP64 and stored ([q][6][element], element fastest).  The apply then needs no
// geometry: with the 1D tables B_qi = L_i(x_q) and G_qi = L_i'(x_q), the reference gradient at all
// 27 points is (G x B x B) u, (B x G x B) u, (B x B x G) u, formed by one-dimensional contractions
// (8 passes of 27 x 3 multiply-adds instead of 27 x 27 x 3); the transposed contractions scatter
// D_q g_q back to the nodes.  Arrays are indexed [z][y][x] = 9 z + 3 y + x for nodes and points.
// ------------------------------------------------------------------------------------------------
struct SF {
  double B[3][3], G[3][3];  // [point][node]
};

__device__ __forceinline__ SF sf_tables() {
  SF t;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const double s = gauss_point(q);
    t.B[q][0] = 0.5 * s * (s - 1.0);
    t.B[q][1] = 1.0 - s * s;
    t.B[q][2] = 0.5 * s * (s + 1.0);
    t.G[q][0] = s - 0.5;
    t.G[q][1] = -2.0 * s;
    t.G[q][2] = s + 0.5;
  }
  return t;
}

// out = M along axis AX (0 x, 1 y, 2 z) applied to in: out[.., q, ..] = sum_i M[q][i] in[.., i, ..].
template <int AX, bool TRANS, bool ACC>
__device__ __forceinline__ void contract(const double M[3][3], const double in[27], double out[27]) {
  constexpr int st = AX == 0 ? 1 : AX == 1 ? 3 : 9;
#pragma unroll
  for (int o = 0; o < 27; ++o) {
    const int q = (o / st) % 3, base = o - q * st;
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) s += (TRANS ? M[i][q] : M[q][i]) * in[base + i * st];
    out[o] = ACC ? out[o] + s : s;
  }
}

// v = A^e u for one component with the partially assembled D (pointer to D[0][0][e], stride E).
__device__ __forceinline__ void pa_laplace(const SF &t, const double *__restrict__ D, int64_t E, const double u[27],
                                           double v[27]) {
  double a[27], b[27], gx[27], gy[27], gz[27];
  contract<2, false, false>(t.B, u, a);   // Bz u
  contract<1, false, false>(t.B, a, b);   // By Bz u
  contract<0, false, false>(t.G, b, gx);  // Gx By Bz u
  contract<1, false, false>(t.G, a, b);   // Gy Bz u
  contract<0, false, false>(t.B, b, gy);  // Bx Gy Bz u
  contract<2, false, false>(t.G, u, a);   // Gz u
  contract<1, false, false>(t.B, a, b);   // By Gz u
  contract<0, false, false>(t.B, b, gz);  // Bx By Gz u
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    const double *d = D + (int64_t)q * 6 * E;
    const double d00 = __ldg(d), d01 = __ldg(d + E), d02 = __ldg(d + 2 * E);
    const double d11 = __ldg(d + 3 * E), d12 = __ldg(d + 4 * E), d22 = __ldg(d + 5 * E);
    const double x = gx[q], y = gy[q], z = gz[q];
    gx[q] = d00 * x + d01 * y + d02 * z;
    gy[q] = d01 * x + d11 * y + d12 * z;
    gz[q] = d02 * x + d12 * y + d22 * z;
  }
  // v = Bz^T (By^T Gx^T fx + Gy^T Bx^T fy) + Gz^T By^T Bx^T fz
  contract<0, true, false>(t.G, gx, a);   // Gx^T fx
  contract<1, true, false>(t.B, a, b);    // By^T Gx^T fx
  contract<0, true, false>(t.B, gy, a);   // Bx^T fy
  contract<1, true, true>(t.G, a, b);     // + Gy^T Bx^T fy
  contract<2, true, false>(t.B, b, v);    // Bz^T (...)
  contract<0, true, false>(t.B, gz, a);   // Bx^T fz
  contract<1, true, false>(t.B, a, b);    // By^T Bx^T fz
  contract<2, true, true>(t.G, b, v);     // + Gz^T By^T Bx^T fz
}

}  // namespace q2
