// Matrix-free operator apply, reference variant: Algorithm 1 with one thread per element (Q1
// hexahedra; the same scheme runs the P1 tetrahedra of mf_tet.cuh).
//
// Each thread gathers its element's 8 support points and input values (Alg. 1, gather step),
// evaluates the Jacobian, its inverse and determinant at every Gauss point, applies the flux /
// stress, and adds v^e into y (Alg. 1, final step).  The paper does not say how the final
// additions avoid races; here the elements are split into colours whose elements share no node
// (2x2x2 parity classes on a structured box, a greedy colouring otherwise), one launch per colour,
// so every addition is a plain read-modify-write in a fixed order: no atomics, bitwise
// reproducible.
#include <vector>

#include "mf_element.cuh"
#include "mf_internal.cuh"
#include "mf_q2.cuh"
#include "mf_tet.cuh"

namespace {

// Element index of thread t in colour c of a structured box (parity class (c&1, c>>1&1, c>>2&1)).
__device__ __forceinline__ int64_t parity_element(int64_t t, int c, int nx, int ny, int nz) {
  const int px = c & 1, py = (c >> 1) & 1, pz = (c >> 2) & 1;
  const int64_t cnx = (nx - px + 1) / 2, cny = (ny - py + 1) / 2;
  const int64_t ix = t % cnx, r = t / cnx, iy = r % cny, iz = r / cny;
  return (2 * ix + px) + (int64_t)nx * ((2 * iy + py) + (int64_t)ny * (2 * iz + pz));
}

template <int PHYS, typename R>
__global__ void __launch_bounds__(128) apply_ref_colour(MeshView m, const R *__restrict__ x, R *__restrict__ y,
                                                        int colour, int64_t count, const int32_t *__restrict__ celems,
                                                        const int *__restrict__ skip) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count || (skip && *skip)) return;
  const int64_t e = celems ? (int64_t)celems[t] : parity_element(t, colour, m.nx, m.ny, m.nz);
  int64_t nodes[8];
  element_nodes(m, e, nodes);
  const R *Xc = coords_of<R>(m);
  const R *mat = mat_of<R>(m);
  R X[8][3];
  bool dir[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    X[a][0] = Xc[3 * nodes[a]];
    X[a][1] = Xc[3 * nodes[a] + 1];
    X[a][2] = Xc[3 * nodes[a] + 2];
    dir[a] = m.dmask[nodes[a]] != 0;
  }
  if (PHYS == MF_LAPLACE) {
    R u[8], v[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) u[a] = dir[a] ? (R)0 : x[nodes[a]];
    q1::laplace_element<R>(X, u, mat[e], v);
#pragma unroll
    for (int a = 0; a < 8; ++a)
      if (!dir[a]) y[nodes[a]] += v[a];
  } else {
    R u[8][3], v[8][3];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) u[a][k] = dir[a] ? (R)0 : x[3 * nodes[a] + k];
    if (PHYS == MF_VECTOR_LAPLACE) q1::vector_laplace_element<R>(X, u, mat[e], v);
    else q1::elasticity_element<R>(X, u, mat[2 * e], mat[2 * e + 1], v);
#pragma unroll
    for (int a = 0; a < 8; ++a)
      if (!dir[a]) {
        y[3 * nodes[a]] += v[a][0];
        y[3 * nodes[a] + 1] += v[a][1];
        y[3 * nodes[a] + 2] += v[a][2];
      }
  }
}

// Multi right-hand-side reference apply: the geometry (adjugate and determinant at every Gauss
// point) is computed once per element and reused for each right-hand side.  Layout [node][rhs][k].
template <int PHYS>
__global__ void __launch_bounds__(128) apply_multi_colour(MeshView m, const double *__restrict__ x,
                                                          double *__restrict__ y, int nrhs, int colour, int64_t count,
                                                          const int32_t *__restrict__ celems) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t e = celems ? (int64_t)celems[t] : parity_element(t, colour, m.nx, m.ny, m.nz);
  int64_t nodes[8];
  element_nodes(m, e, nodes);
  double X[8][3];
  bool dir[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
#pragma unroll
    for (int i = 0; i < 3; ++i) X[a][i] = m.X[3 * nodes[a] + i];
    dir[a] = m.dmask[nodes[a]] != 0;
  }
  constexpr int ND = phys_ndpn(PHYS);
  double Cq[8][3][3], idet[8];
#define MF_GEOM(Q)                                        \
  {                                                       \
    double J[3][3];                                       \
    q1::jacobian<double, Q>(X, J);                        \
    idet[Q] = 1.0 / q1::adjugate(J, Cq[Q]);               \
  }
  MF_GEOM(0) MF_GEOM(1) MF_GEOM(2) MF_GEOM(3) MF_GEOM(4) MF_GEOM(5) MF_GEOM(6) MF_GEOM(7)
#undef MF_GEOM
  const double c0 = phys_is_laplace(PHYS) ? m.mat[e] : m.mat[2 * e];
  const double c1 = phys_is_laplace(PHYS) ? 0.0 : m.mat[2 * e + 1];
  for (int r = 0; r < nrhs; ++r) {
    double u[8][ND], v[8][ND];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int k = 0; k < ND; ++k) {
        u[a][k] = dir[a] ? 0.0 : x[((int64_t)nodes[a] * nrhs + r) * ND + k];
        v[a][k] = 0.0;
      }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double(&C)[3][3] = Cq[q];
      if (phys_is_laplace(PHYS)) {
#pragma unroll
        for (int kc = 0; kc < ND; ++kc) {  // the scalar flux for each component (Eq. 5)
          double g[3];
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            double s = 0;
#pragma unroll
            for (int a = 0; a < 8; ++a) s += u[a][kc] * q1::dN(q, a, j);
            g[j] = s;
          }
          double tt[3], f[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) tt[k] = C[0][k] * g[0] + C[1][k] * g[1] + C[2][k] * g[2];
          const double sc = c0 * idet[q];
#pragma unroll
          for (int j = 0; j < 3; ++j) f[j] = sc * (C[j][0] * tt[0] + C[j][1] * tt[1] + C[j][2] * tt[2]);
#pragma unroll
          for (int a = 0; a < 8; ++a)
            v[a][kc] += q1::dN(q, a, 0) * f[0] + q1::dN(q, a, 1) * f[1] + q1::dN(q, a, 2) * f[2];
        }
      } else {
        double H[3][3], G[3][3], S[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            double s = 0;
#pragma unroll
            for (int a = 0; a < 8; ++a) s += u[a][k % ND] * q1::dN(q, a, j);
            H[k][j] = s;
          }
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int l = 0; l < 3; ++l) G[k][l] = (H[k][0] * C[0][l] + H[k][1] * C[1][l] + H[k][2] * C[2][l]) * idet[q];
        const double tr = G[0][0] + G[1][1] + G[2][2];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int l = 0; l < 3; ++l) S[k][l] = c1 * (G[k][l] + G[l][k]) + (k == l ? c0 * tr : 0.0);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          double P[3];
#pragma unroll
          for (int j = 0; j < 3; ++j) P[j] = S[k][0] * C[j][0] + S[k][1] * C[j][1] + S[k][2] * C[j][2];
#pragma unroll
          for (int a = 0; a < 8; ++a) v[a][k % ND] += P[0] * q1::dN(q, a, 0) + P[1] * q1::dN(q, a, 1) + P[2] * q1::dN(q, a, 2);
        }
      }
    }
#pragma unroll
    for (int a = 0; a < 8; ++a)
      if (!dir[a])
#pragma unroll
        for (int k = 0; k < ND; ++k) y[((int64_t)nodes[a] * nrhs + r) * ND + k] += v[a][k];
  }
}

// P1 tetrahedra, one thread per element of a colour: gather the 4 vertices and values, apply the
// element operator of mf_tet.cuh, add into y.  Layout [node][rhs][comp] with `nrhs` right-hand
// sides per node (the geometry is computed once per element for all of them).
template <int PHYS, typename R>
__global__ void __launch_bounds__(128) tet_apply_colour(MeshView m, const R *__restrict__ x, R *__restrict__ y,
                                                        int nrhs, int64_t count, const int32_t *__restrict__ celems,
                                                        const int *__restrict__ skip) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count || (skip && *skip)) return;
  constexpr int ND = phys_ndpn(PHYS);
  const int64_t e = celems[t];
  int64_t nodes[4];
  p1::nodes_of(m.cells, e, nodes);
  const R *Xc = coords_of<R>(m);
  const R *mat = mat_of<R>(m);
  R X[4][3], n[4][3];
  bool dir[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int i = 0; i < 3; ++i) X[a][i] = Xc[3 * nodes[a] + i];
    dir[a] = m.dmask[nodes[a]] != 0;
  }
  const R D = p1::geometry<R>(X, n);
  for (int r = 0; r < nrhs; ++r) {
    if (PHYS == MF_ELASTICITY) {
      R u[4][3], v[4][3];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) u[a][k] = dir[a] ? (R)0 : x[(nodes[a] * nrhs + r) * 3 + k];
      p1::elasticity<R>(n, D, mat[2 * e], mat[2 * e + 1], u, v);
#pragma unroll
      for (int a = 0; a < 4; ++a)
        if (!dir[a])
#pragma unroll
          for (int k = 0; k < 3; ++k) y[(nodes[a] * nrhs + r) * 3 + k] += v[a][k];
    } else {
#pragma unroll
      for (int k = 0; k < ND; ++k) {  // the scalar operator on each component (Eq. 5)
        R u[4], v[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) u[a] = dir[a] ? (R)0 : x[(nodes[a] * nrhs + r) * ND + k];
        p1::laplace<R>(n, D, mat[e], u, v);
#pragma unroll
        for (int a = 0; a < 4; ++a)
          if (!dir[a]) y[(nodes[a] * nrhs + r) * ND + k] += v[a];
      }
    }
  }
}

// Q2 hexahedra, one thread per element of a colour (mf_q2.cuh); `nrhs` right-hand sides per node,
// [node][rhs][comp], one after the other (the geometry is recomputed for each).
template <int PHYS, typename R>
__global__ void __launch_bounds__(64) q2_apply_colour(MeshView m, const R *__restrict__ x, R *__restrict__ y, int nrhs,
                                                      int64_t count, const int32_t *__restrict__ celems,
                                                      const int *__restrict__ skip) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count || (skip && *skip)) return;
  constexpr int ND = phys_ndpn(PHYS);
  const int64_t e = celems[t];
  const R *Xc = coords_of<R>(m);
  const R *mat = mat_of<R>(m);
  int64_t nodes[27];
  R X[27][3];
  bool dir[27];
  for (int a = 0; a < 27; ++a) {
    nodes[a] = m.cells[27 * e + a];
    for (int i = 0; i < 3; ++i) X[a][i] = Xc[3 * nodes[a] + i];
    dir[a] = m.dmask[nodes[a]] != 0;
  }
  const R c0 = phys_is_laplace(PHYS) ? mat[e] : mat[2 * e];
  const R c1 = phys_is_laplace(PHYS) ? (R)0 : mat[2 * e + 1];
  for (int r = 0; r < nrhs; ++r) {
    R u[27][ND], v[27][ND];
    for (int a = 0; a < 27; ++a)
      for (int k = 0; k < ND; ++k) u[a][k] = dir[a] ? (R)0 : x[(nodes[a] * nrhs + r) * ND + k];
    q2::element_apply<R, ND, PHYS == MF_ELASTICITY>(X, u, c0, c1, v);
    for (int a = 0; a < 27; ++a)
      if (!dir[a])
        for (int k = 0; k < ND; ++k) y[(nodes[a] * nrhs + r) * ND + k] += v[a][k];
  }
}

// Q2 partial assembly: D_q = (w_q kappa / det J) adj J adj J^T at the 27 Gauss points, [q][6][e].
__global__ void __launch_bounds__(64) q2pa_build(MeshView m, double *__restrict__ D) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.n_cells) return;
  const int64_t E = m.n_cells;
  double X[27][3];
  for (int a = 0; a < 27; ++a) {
    const int64_t n = m.cells[27 * e + a];
    for (int i = 0; i < 3; ++i) X[a][i] = m.X[3 * n + i];
  }
  const double kappa = m.mat[e];
  for (int q = 0; q < 27; ++q) {
    double xi[3];
    q2::point_q(q, xi);
    q2::Tab<double> t;
    q2::tables_at<double>(xi, t);
    double J[3][3], C[3][3];
    q2::jacobian(X, t, J);
    const double det = q1::adjugate(J, C);
    const double s = q2::weight_q(q) * kappa / det;
    double d[6];
    int k = 0;
    for (int r = 0; r < 3; ++r)
      for (int c = r; c < 3; ++c) d[k++] = s * (C[r][0] * C[c][0] + C[r][1] * C[c][1] + C[r][2] * C[c][2]);
    for (int j = 0; j < 6; ++j) D[((int64_t)q * 6 + j) * E + e] = d[j];
  }
}

// Q2 elasticity partial assembly (Eq. 6 with the Q2 map): per Gauss point K = J^-1 (9 values, K[c][l] =
// dxi_c/dx_l) and w det J lambda, w det J mu, stored [element][11][32] (points q < 27 used) so that the
// apply's warp reads each value of its element's 27 points with one coalesced load.
constexpr int kQ2ElVals = 11;
__global__ void __launch_bounds__(64) q2pa_el_build(MeshView m, double *__restrict__ D) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.n_cells) return;
  double X[27][3];
  for (int a = 0; a < 27; ++a) {
    const int64_t n = m.cells[27 * e + a];
    for (int i = 0; i < 3; ++i) X[a][i] = m.X[3 * n + i];
  }
  const double lam = m.mat[2 * e], mu = m.mat[2 * e + 1];
  double *De = D + e * kQ2ElVals * 32;
  for (int q = 0; q < 27; ++q) {
    double xi[3];
    q2::point_q(q, xi);
    q2::Tab<double> t;
    q2::tables_at<double>(xi, t);
    double J[3][3], C[3][3];
    q2::jacobian(X, t, J);
    const double det = q1::adjugate(J, C);
    for (int c = 0; c < 3; ++c)
      for (int l = 0; l < 3; ++l) De[(3 * c + l) * 32 + q] = C[c][l] / det;
    const double wd = q2::weight_q(q) * det;
    De[9 * 32 + q] = wd * lam;
    De[10 * 32 + q] = wd * mu;
  }
}

namespace q2w {

// One-dimensional contraction of a warp's element array along axis AX (0 x, 1 y, 2 z) for the three
// components: out[k] at this lane's index o = sum_i M[q][i] in[k][base + i st] (TRANS: M[i][q]), q the
// index of o along AX.  M is a 3 x 3 table in shared memory, in[k] a 32-entry row (27 used).
template <int AX, bool TRANS>
__device__ __forceinline__ void contract3(const double (*M)[3], const double (*in)[32], int o, double out[3]) {
  constexpr int st = AX == 0 ? 1 : AX == 1 ? 3 : 9;
  const int q = (o / st) % 3, base = o - q * st;
  const double m0 = TRANS ? M[0][q] : M[q][0], m1 = TRANS ? M[1][q] : M[q][1], m2 = TRANS ? M[2][q] : M[q][2];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    out[k] = __fma_rn(m2, in[k][base + 2 * st], __fma_rn(m1, in[k][base + st], m0 * in[k][base]));
}

__device__ __forceinline__ void put3(double (*dst)[32], int o, const double v[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) dst[k][o] = v[k];
}

}  // namespace q2w

// Q2 elasticity apply from the partial assembly: one warp per element, lane o < 27 is node o for the
// gather and the results and Gauss point o for the stress.  The reference gradients of the three
// components at the 27 points are formed by one-dimensional contractions with the 1D value and
// derivative tables B and G (the sum factorisation of the Q2 Laplace kernel: 8 passes of 3 multiply-adds
// per entry instead of 27 x 3), the stress P = S K^T with S = w det J (mu (grad u + grad u^T) + lambda
// tr(grad u) I), grad u = H K per point, and the transposed contractions take P back to the nodes.  The
// element's 27 x 3 results go to its own slots (as q2pa_elements); q2pa_gather sums them per node.
__global__ void __launch_bounds__(128) q2pa_el_elements(MeshView m, const double *__restrict__ D,
                                                       const double *__restrict__ x, int nrhs, int r,
                                                       double *__restrict__ buf, const int *__restrict__ skip) {
  constexpr int W = 4;  // elements (warps) per block
  __shared__ double tB[3][3], tG[3][3];
  __shared__ double sU[W][3][32], sA[W][3][32], sB[W][3][32];
  if (skip && *skip) return;
  if (threadIdx.x < 9) {
    const q2::SF t = q2::sf_tables();
    tB[threadIdx.x / 3][threadIdx.x % 3] = t.B[threadIdx.x / 3][threadIdx.x % 3];
    tG[threadIdx.x / 3][threadIdx.x % 3] = t.G[threadIdx.x / 3][threadIdx.x % 3];
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, o = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * W + w;
  if (e >= m.n_cells) return;  // whole warps; no block barrier follows
  const bool lv = o < 27;
  double (*U)[32] = sU[w], (*A)[32] = sA[w], (*B)[32] = sB[w];
  if (lv) {
    const int64_t node = __ldg(m.cells + 27 * e + o);
    const bool dir = m.dmask[node] != 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) U[k][o] = dir ? 0.0 : x[(node * nrhs + r) * 3 + k];
  }
  __syncwarp();
  double t[3], gx[3], gy[3], gz[3];
  // reference gradients: gx = Gx By Bz u, gy = Bx Gy Bz u, gz = Bx By Gz u
  if (lv) { q2w::contract3<2, false>(tB, U, o, t); q2w::put3(A, o, t); }
  __syncwarp();
  if (lv) { q2w::contract3<1, false>(tB, A, o, t); q2w::put3(B, o, t); }
  __syncwarp();
  if (lv) q2w::contract3<0, false>(tG, B, o, gx);
  __syncwarp();
  if (lv) { q2w::contract3<1, false>(tG, A, o, t); q2w::put3(B, o, t); }
  __syncwarp();
  if (lv) {
    q2w::contract3<0, false>(tB, B, o, gy);
    q2w::contract3<2, false>(tG, U, o, t);
    q2w::put3(A, o, t);
  }
  __syncwarp();
  if (lv) { q2w::contract3<1, false>(tB, A, o, t); q2w::put3(B, o, t); }
  __syncwarp();
  double fx[3], fy[3], fz[3];
  if (lv) {
    q2w::contract3<0, false>(tB, B, o, gz);
    const double *De = D + e * kQ2ElVals * 32 + o;
    double K[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int l = 0; l < 3; ++l) K[c][l] = __ldg(De + (3 * c + l) * 32);
    const double slam = __ldg(De + 9 * 32), smu = __ldg(De + 10 * 32);
    double G[3][3];  // grad u: G[k][l] = sum_c H[k][c] K[c][l], H[k] = (gx, gy, gz)[k]
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = 0; l < 3; ++l) G[k][l] = gx[k] * K[0][l] + gy[k] * K[1][l] + gz[k] * K[2][l];
    const double tr = slam * (G[0][0] + G[1][1] + G[2][2]);
    double S[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = 0; l < 3; ++l) S[k][l] = smu * (G[k][l] + G[l][k]) + (k == l ? tr : 0.0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {  // P[k][c] = sum_l S[k][l] K[c][l]
      fx[k] = S[k][0] * K[0][0] + S[k][1] * K[0][1] + S[k][2] * K[0][2];
      fy[k] = S[k][0] * K[1][0] + S[k][1] * K[1][1] + S[k][2] * K[1][2];
      fz[k] = S[k][0] * K[2][0] + S[k][1] * K[2][1] + S[k][2] * K[2][2];
    }
    q2w::put3(A, o, fx);
  }
  __syncwarp();
  // v = Bz^T (By^T Gx^T fx + Gy^T Bx^T fy) + Gz^T By^T Bx^T fz
  double bb[3], v[3];
  if (lv) { q2w::contract3<0, true>(tG, A, o, t); q2w::put3(B, o, t); }
  __syncwarp();
  if (lv) { q2w::contract3<1, true>(tB, B, o, bb); q2w::put3(A, o, fy); }
  __syncwarp();
  if (lv) { q2w::contract3<0, true>(tB, A, o, t); q2w::put3(B, o, t); }
  __syncwarp();
  if (lv) {
    q2w::contract3<1, true>(tG, B, o, t);
#pragma unroll
    for (int k = 0; k < 3; ++k) bb[k] += t[k];
    q2w::put3(A, o, bb);
  }
  __syncwarp();
  if (lv) { q2w::contract3<2, true>(tB, A, o, v); q2w::put3(B, o, fz); }
  __syncwarp();
  if (lv) { q2w::contract3<0, true>(tB, B, o, t); q2w::put3(A, o, t); }
  __syncwarp();
  if (lv) { q2w::contract3<1, true>(tB, A, o, t); q2w::put3(B, o, t); }
  __syncwarp();
  if (lv) {
    q2w::contract3<2, true>(tG, B, o, t);
#pragma unroll
    for (int k = 0; k < 3; ++k) buf[(e * 27 + o) * 3 + k] = v[k] + t[k];
  }
}

// Q2 Laplace / vector Laplace apply from the partial assembly in two launches, without colours: every
// element at once writes its 27 x ND results to its own slots of `buf` ([element][node][comp]); then
// every DoF sums its slots in a fixed order (the node's slot list, sorted by element) and the
// Dirichlet rows take y_d = x_d.  Deterministic, and all elements run in one launch (a colour of a
// Q2 box mesh holds only 1/8 of them).
template <int ND>
__global__ void __launch_bounds__(64) q2pa_elements(MeshView m, const double *__restrict__ D,
                                                    const double *__restrict__ x, int nrhs, int r,
                                                    double *__restrict__ buf, const int *__restrict__ skip) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.n_cells || (skip && *skip)) return;
  const q2::SF tab = q2::sf_tables();
  int32_t nodes[27];
  bool dir[27];
#pragma unroll
  for (int a = 0; a < 27; ++a) {
    nodes[a] = __ldg(m.cells + 27 * e + a);
    dir[a] = m.dmask[nodes[a]] != 0;
  }
  for (int k = 0; k < ND; ++k) {
    double u[27], v[27];
#pragma unroll
    for (int a = 0; a < 27; ++a) u[a] = dir[a] ? 0.0 : x[((int64_t)nodes[a] * nrhs + r) * ND + k];
    q2::pa_laplace(tab, D + e, m.n_cells, u, v);
#pragma unroll
    for (int a = 0; a < 27; ++a) buf[(e * 27 + a) * ND + k] = v[a];
  }
}

template <int ND>
__global__ void q2pa_gather(int64_t n_nodes, const int64_t *__restrict__ off, const int32_t *__restrict__ slots,
                            const uint8_t *__restrict__ dmask, const double *__restrict__ buf,
                            const double *__restrict__ x, double *__restrict__ y, int nrhs, int r,
                            const int *__restrict__ skip) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_nodes * ND || (skip && *skip)) return;
  const int64_t n = i / ND;
  const int k = (int)(i % ND);
  const int64_t o = (n * nrhs + r) * ND + k;
  if (dmask[n]) {
    y[o] = x[o];
    return;
  }
  double s = 0.0;
  for (int64_t t = off[n]; t < off[n + 1]; ++t) s += buf[(int64_t)slots[t] * ND + k];
  y[o] = s;
}

// Dirichlet rows: y_d = x_d.
template <typename R>
__global__ void dirichlet_rows(const int32_t *__restrict__ dn, int64_t n, int ndw, const R *__restrict__ x,
                               R *__restrict__ y, const int *__restrict__ skip) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n * ndw || (skip && *skip)) return;
  const int64_t node = dn[i / ndw];
  const int64_t k = i % ndw;
  y[node * ndw + k] = x[node * ndw + k];
}

// Apply for the elements other than Q1 (P1 tetrahedra, Q2 hexahedra): colour by colour, then the
// Dirichlet rows.
// Q2 Laplace / vector Laplace from the partial assembly: element launch and node gather per
// right-hand side.
mf_status q2pa_apply(const mf_mesh *m, const double *x, double *y, int nrhs, cudaStream_t s, const int *skip) {
  const MeshView v = m->view();
  const int nd = m->ndpn;
  for (int r = 0; r < nrhs; ++r) {
    mf_count_launches(2);
    if (nd == 1) {
      q2pa_elements<1><<<blocks_for(m->n_cells, 64), 64, 0, s>>>(v, m->q2pa, x, nrhs, r, m->q2buf, skip);
      q2pa_gather<1><<<blocks_for(m->n_nodes), kThreads, 0, s>>>(m->n_nodes, m->q2off, m->q2slots, m->dmask,
                                                                   m->q2buf, x, y, nrhs, r, skip);
    } else if (m->physics == MF_ELASTICITY) {
      q2pa_el_elements<<<(unsigned)((m->n_cells + 3) / 4), 128, 0, s>>>(v, m->q2pa, x, nrhs, r, m->q2buf, skip);
      q2pa_gather<3><<<blocks_for(m->n_nodes * 3), kThreads, 0, s>>>(m->n_nodes, m->q2off, m->q2slots, m->dmask,
                                                                       m->q2buf, x, y, nrhs, r, skip);
    } else {
      q2pa_elements<3><<<blocks_for(m->n_cells, 64), 64, 0, s>>>(v, m->q2pa, x, nrhs, r, m->q2buf, skip);
      q2pa_gather<3><<<blocks_for(m->n_nodes * 3), kThreads, 0, s>>>(m->n_nodes, m->q2off, m->q2slots, m->dmask,
                                                                       m->q2buf, x, y, nrhs, r, skip);
    }
  }
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

template <typename R>
mf_status explicit_apply(const mf_mesh *m, const R *x, R *y, int nrhs, cudaStream_t s, const int *skip) {
  if constexpr (sizeof(R) == 8) {
    if (m->npe == 27 && m->q2pa && m->variant != MF_VARIANT_REFERENCE) return q2pa_apply(m, x, y, nrhs, s, skip);
  }
  MF_CUDA(cudaMemsetAsync(y, 0, m->n_dof * nrhs * sizeof(R), s));
  const MeshView v = m->view();
  for (int c = 0; c < m->n_colours; ++c) {
    const int64_t cnt = colour_count(m, c);
    if (cnt == 0) continue;
    const int32_t *ce = m->colour_elems + m->colour_off[c];
    mf_count_launches(1);
    if (m->npe == 27) {
      if (m->physics == MF_LAPLACE)
        q2_apply_colour<MF_LAPLACE, R><<<blocks_for(cnt, 64), 64, 0, s>>>(v, x, y, nrhs, cnt, ce, skip);
      else if (m->physics == MF_VECTOR_LAPLACE)
        q2_apply_colour<MF_VECTOR_LAPLACE, R><<<blocks_for(cnt, 64), 64, 0, s>>>(v, x, y, nrhs, cnt, ce, skip);
      else
        q2_apply_colour<MF_ELASTICITY, R><<<blocks_for(cnt, 64), 64, 0, s>>>(v, x, y, nrhs, cnt, ce, skip);
    } else if (m->physics == MF_LAPLACE)
      tet_apply_colour<MF_LAPLACE, R><<<blocks_for(cnt, 128), 128, 0, s>>>(v, x, y, nrhs, cnt, ce, skip);
    else if (m->physics == MF_VECTOR_LAPLACE)
      tet_apply_colour<MF_VECTOR_LAPLACE, R><<<blocks_for(cnt, 128), 128, 0, s>>>(v, x, y, nrhs, cnt, ce, skip);
    else
      tet_apply_colour<MF_ELASTICITY, R><<<blocks_for(cnt, 128), 128, 0, s>>>(v, x, y, nrhs, cnt, ce, skip);
  }
  if (m->n_dnodes) mf_count_launches(1);
  if (m->n_dnodes)
    dirichlet_rows<R><<<blocks_for(m->n_dnodes * m->ndpn * nrhs), kThreads, 0, s>>>(m->dnodes, m->n_dnodes,
                                                                                  m->ndpn * nrhs, x, y, skip);
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

template <typename R>
mf_status apply_reference(const mf_mesh *m, const R *x, R *y, cudaStream_t s, const int *skip) {
  if (m->npe != 8) return explicit_apply<R>(m, x, y, 1, s, skip);  // P1 tetrahedra, Q2 hexahedra
  MF_CUDA(cudaMemsetAsync(y, 0, m->n_dof * sizeof(R), s));
  const MeshView v = m->view();
  for (int c = 0; c < m->n_colours; ++c) {
    const int64_t cnt = colour_count(m, c);
    if (cnt == 0) continue;
    const int32_t *ce = m->structured ? nullptr : m->colour_elems + m->colour_off[c];
    mf_count_launches(1);
    if (m->physics == MF_LAPLACE)
      apply_ref_colour<MF_LAPLACE, R><<<blocks_for(cnt, 128), 128, 0, s>>>(v, x, y, c, cnt, ce, skip);
    else if (m->physics == MF_VECTOR_LAPLACE)
      apply_ref_colour<MF_VECTOR_LAPLACE, R><<<blocks_for(cnt, 128), 128, 0, s>>>(v, x, y, c, cnt, ce, skip);
    else
      apply_ref_colour<MF_ELASTICITY, R><<<blocks_for(cnt, 128), 128, 0, s>>>(v, x, y, c, cnt, ce, skip);
  }
  if (m->n_dnodes) mf_count_launches(1);
  if (m->n_dnodes)
    dirichlet_rows<R><<<blocks_for(m->n_dnodes * m->ndpn), kThreads, 0, s>>>(m->dnodes, m->n_dnodes, m->ndpn, x, y, skip);
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

}  // namespace

size_t q2_pa_bytes(int physics, int64_t n_cells) {
  return physics == MF_ELASTICITY ? (size_t)n_cells * kQ2ElVals * 32 * sizeof(double)
                                  : (size_t)n_cells * 27 * 6 * sizeof(double);
}

mf_status q2_pa_setup(mf_mesh *m, cudaStream_t s) {
  if (m->q2pa) return MF_OK;
  if (m->npe != 27) {
    mf_set_error("the sum-factorised partial assembly is built for Q2 meshes");
    return MF_ERR_UNSUPPORTED;
  }
  const size_t bytes = q2_pa_bytes(m->physics, m->n_cells);
  cudaError_t e = cudaMalloc(&m->q2pa, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    m->q2pa = nullptr;
    mf_set_error("Q2 partial assembly: allocation of %zu bytes failed", bytes);
    return MF_ERR_OOM;
  }
  // node -> slot lists (slot = 27 e + a), each sorted by element: the order of the gather's sum
  const int64_t N = m->n_nodes, E = m->n_cells;
  std::vector<int64_t> off(N + 1, 0);
  for (int64_t t = 0; t < 27 * E; ++t) off[m->h_cells[t] + 1]++;
  for (int64_t n = 0; n < N; ++n) off[n + 1] += off[n];
  std::vector<int64_t> pos(off.begin(), off.end() - 1);
  std::vector<int32_t> slots(27 * E);
  for (int64_t t = 0; t < 27 * E; ++t) slots[pos[m->h_cells[t]]++] = (int32_t)t;
  const size_t buf_bytes = (size_t)E * 27 * m->ndpn * sizeof(double);
  if ((e = cudaMalloc(&m->q2off, (N + 1) * sizeof(int64_t))) != cudaSuccess ||
      (e = cudaMalloc(&m->q2slots, 27 * E * sizeof(int32_t))) != cudaSuccess ||
      (e = cudaMalloc(&m->q2buf, buf_bytes)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(m->q2pa); cudaFree(m->q2off); cudaFree(m->q2slots); cudaFree(m->q2buf);
    m->q2pa = nullptr; m->q2off = nullptr; m->q2slots = nullptr; m->q2buf = nullptr;
    mf_set_error("Q2 partial assembly: allocation failed");
    return MF_ERR_OOM;
  }
  MF_CUDA(cudaMemcpyAsync(m->q2off, off.data(), (N + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  MF_CUDA(cudaMemcpyAsync(m->q2slots, slots.data(), 27 * E * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  mf_count_launches(1);
  if (m->physics == MF_ELASTICITY) {
    MF_CUDA(cudaMemsetAsync(m->q2pa, 0, bytes, s));  // the unused point slots 27..31
    q2pa_el_build<<<blocks_for(m->n_cells, 64), 64, 0, s>>>(m->view(), m->q2pa);
  } else {
    q2pa_build<<<blocks_for(m->n_cells, 64), 64, 0, s>>>(m->view(), m->q2pa);
  }
  MF_CUDA(cudaGetLastError());
  MF_CUDA(cudaStreamSynchronize(s));
  return MF_OK;
}

mf_status apply_fp64(const mf_mesh *m, const double *x, double *y, cudaStream_t s, const int *skip) {
  if (m->variant == MF_VARIANT_AUTO && m->tp) return tile_apply_fp64(m, x, y, s, skip);
  if (m->variant != MF_VARIANT_REFERENCE && m->gen) return gen_apply_fp64(m, x, y, s, skip);
  return apply_reference<double>(m, x, y, s, skip);
}

mf_status apply_fp32(const mf_mesh *m, const float *x, float *y, cudaStream_t s, const int *skip) {
  if (m->variant == MF_VARIANT_AUTO && m->tp) return tile_apply_fp32(m, x, y, s, skip);
  if (m->variant != MF_VARIANT_REFERENCE && m->gen) return gen_apply_fp32(m, x, y, s, skip);
  return apply_reference<float>(m, x, y, s, skip);
}

mf_status apply_multi_fp64(const mf_mesh *m, int nrhs, const double *x, double *y, cudaStream_t s) {
  if (m->variant == MF_VARIANT_AUTO && m->tp) return tile_apply_multi_fp64(m, nrhs, x, y, s);
  if (m->npe != 8) return explicit_apply<double>(m, x, y, nrhs, s, nullptr);
  MF_CUDA(cudaMemsetAsync(y, 0, m->n_dof * nrhs * sizeof(double), s));
  const MeshView v = m->view();
  for (int c = 0; c < m->n_colours; ++c) {
    const int64_t cnt = colour_count(m, c);
    if (cnt == 0) continue;
    const int32_t *ce = m->structured ? nullptr : m->colour_elems + m->colour_off[c];
    mf_count_launches(1);
    if (m->physics == MF_LAPLACE)
      apply_multi_colour<MF_LAPLACE><<<blocks_for(cnt, 128), 128, 0, s>>>(v, x, y, nrhs, c, cnt, ce);
    else if (m->physics == MF_VECTOR_LAPLACE)
      apply_multi_colour<MF_VECTOR_LAPLACE><<<blocks_for(cnt, 128), 128, 0, s>>>(v, x, y, nrhs, c, cnt, ce);
    else
      apply_multi_colour<MF_ELASTICITY><<<blocks_for(cnt, 128), 128, 0, s>>>(v, x, y, nrhs, c, cnt, ce);
  }
  if (m->n_dnodes) mf_count_launches(1);
  if (m->n_dnodes)
    dirichlet_rows<double><<<blocks_for(m->n_dnodes * m->ndpn * nrhs), kThreads, 0, s>>>(
        m->dnodes, m->n_dnodes, m->ndpn * nrhs, x, y, nullptr);
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

// ----------------------------------------------------------------------------- entry points ----
static mf_status check_apply_args(const mf_mesh *m, const void *x, void *y, size_t bytes) {
  MF_ARG(m && x && y, "apply: null argument");
  const char *xb = (const char *)x, *yb = (const char *)y;
  MF_ARG(xb + bytes <= yb || yb + bytes <= xb, "apply: x and y overlap");
  return MF_OK;
}

extern "C" mf_status mf_apply_laplace(const mf_mesh *m, const double *x, double *y, mf_stream stream) {
  MF_RANGE("mf_apply_laplace");
  mf_clear_error();
  MF_TRY(check_apply_args(m, x, y, m ? m->n_dof * sizeof(double) : 0));
  MF_ARG(m->physics == MF_LAPLACE, "mf_apply_laplace: mesh was set up for another physics");
  return apply_fp64(m, x, y, (cudaStream_t)stream);
}

extern "C" mf_status mf_apply_vector_laplace(const mf_mesh *m, const double *x, double *y, mf_stream stream) {
  MF_RANGE("mf_apply_vector_laplace");
  mf_clear_error();
  MF_TRY(check_apply_args(m, x, y, m ? m->n_dof * sizeof(double) : 0));
  MF_ARG(m->physics == MF_VECTOR_LAPLACE, "mf_apply_vector_laplace: mesh was set up for another physics");
  return apply_fp64(m, x, y, (cudaStream_t)stream);
}

extern "C" mf_status mf_apply_elasticity(const mf_mesh *m, const double *x, double *y, mf_stream stream) {
  MF_RANGE("mf_apply_elasticity");
  mf_clear_error();
  MF_TRY(check_apply_args(m, x, y, m ? m->n_dof * sizeof(double) : 0));
  MF_ARG(m->physics == MF_ELASTICITY, "mf_apply_elasticity: mesh was set up for another physics");
  return apply_fp64(m, x, y, (cudaStream_t)stream);
}

extern "C" mf_status mf_apply_f32(const mf_mesh *m, const float *x, float *y, mf_stream stream) {
  MF_RANGE("mf_apply_f32");
  mf_clear_error();
  MF_TRY(check_apply_args(m, x, y, m ? m->n_dof * sizeof(float) : 0));
  return apply_fp32(m, x, y, (cudaStream_t)stream);
}

extern "C" mf_status mf_apply_multi(const mf_mesh *m, int32_t nrhs, const double *X, double *Y, mf_stream stream) {
  MF_RANGE("mf_apply_multi");
  mf_clear_error();
  MF_ARG(nrhs >= 1 && nrhs <= 16, "mf_apply_multi: nrhs must be in [1, 16]");
  MF_TRY(check_apply_args(m, X, Y, m ? m->n_dof * nrhs * sizeof(double) : 0));
  return apply_multi_fp64(m, nrhs, X, Y, (cudaStream_t)stream);
}
