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

#include "mf_dw.cuh"
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
  const int64_t e = mf_dbg_index(celems ? (int64_t)celems[t] : parity_element(t, colour, m.nx, m.ny, m.nz), m.n_cells,
                                 MF_DBG_CELL);
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
  const int64_t e = mf_dbg_index(celems ? (int64_t)celems[t] : parity_element(t, colour, m.nx, m.ny, m.nz), m.n_cells,
                                 MF_DBG_CELL);
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
  const int64_t e = mf_dbg_index((int64_t)celems[t], m.n_cells, MF_DBG_CELL);
  int64_t nodes[4];
  p1::nodes_of(m.cells, e, nodes);
#pragma unroll
  for (int a = 0; a < 4; ++a) nodes[a] = mf_dbg_index(nodes[a], m.n_nodes, MF_DBG_NODE);
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
  const int64_t e = mf_dbg_index((int64_t)celems[t], m.n_cells, MF_DBG_CELL);
  const R *Xc = coords_of<R>(m);
  const R *mat = mat_of<R>(m);
  int64_t nodes[27];
  R X[27][3];
  bool dir[27];
  for (int a = 0; a < 27; ++a) {
    nodes[a] = cell_node(m, 27, e, a);
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
    const int64_t n = cell_node(m, 27, e, a);
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
    const int64_t n = cell_node(m, 27, e, a);
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
    const int64_t node = cell_node(m, 27, e, o);
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

// Largest and smallest non-zero magnitudes (biased FP64 exponent fields) of the elasticity partial
// assembly, for J^-1 (ext[0], ext[1]) and for w det J lambda / mu (ext[2], ext[3]); ext starts at
// {0, ~0, 0, ~0}.  Order-independent (maxima and minima), so deterministic.
__global__ void q2pa_el_extent(const double *__restrict__ D, int64_t n_cells, unsigned *ext) {
  unsigned kmax = 0, kmin = ~0u, smax = 0, smin = ~0u;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_cells * kQ2ElVals * 32;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(i % 32), j = (int)((i / 32) % kQ2ElVals);
    if (q >= 27) continue;
    const unsigned e = (unsigned)((__double_as_longlong(D[i]) >> 52) & 0x7ff);
    if (e == 0) continue;  // zeros (and subnormals: flushed below)
    if (j < 9) { kmax = max(kmax, e); kmin = min(kmin, e); }
    else { smax = max(smax, e); smin = min(smin, e); }
  }
  atomicMax(ext, kmax);
  atomicMin(ext + 1, kmin);
  atomicMax(ext + 2, smax);
  atomicMin(ext + 3, smin);
}

// In place: every value of the elasticity partial assembly as a float pair of itself times 2^-sk
// (J^-1) or 2^-ss (w det J lambda, mu), exactly scaled; values below 2^-74 after the scaling (2^-74
// of the largest) become 0.
__global__ void q2pa_el_to_dw(double *__restrict__ D, int64_t n_cells, int sk, int ss) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_cells * kQ2ElVals * 32;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)((i / 32) % kQ2ElVals);
    const dwa::dw v = dwa::split_scaled(D[i], j < 9 ? sk : ss);
    reinterpret_cast<float2 *>(D)[i] = make_float2(v.h, v.l);
  }
}

namespace q2w {

// contract3 on double-word values (pairs in shared memory, the 1D tables as pairs), NC components.
template <int AX, bool TRANS, int NC>
__device__ __forceinline__ void contract3_dw(const float2 (*M)[3], const float2 (*in)[32], int o, dwa::dw out[NC]) {
  constexpr int st = AX == 0 ? 1 : AX == 1 ? 3 : 9;
  const int q = (o / st) % 3, base = o - q * st;
  const float2 f0 = TRANS ? M[0][q] : M[q][0], f1 = TRANS ? M[1][q] : M[q][1], f2 = TRANS ? M[2][q] : M[q][2];
  const dwa::dw m0{f0.x, f0.y}, m1{f1.x, f1.y}, m2{f2.x, f2.y};
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    const float2 a = in[k][base], b = in[k][base + st], c = in[k][base + 2 * st];
    out[k] = dwa::add(dwa::add(dwa::mul(m0, dwa::dw{a.x, a.y}), dwa::mul(m1, dwa::dw{b.x, b.y})),
                      dwa::mul(m2, dwa::dw{c.x, c.y}));
  }
}

template <int NC>
__device__ __forceinline__ void put3_dw(float2 (*dst)[32], int o, const dwa::dw v[NC]) {
#pragma unroll
  for (int k = 0; k < NC; ++k) dst[k][o] = make_float2(v[k].h, v[k].l);
}

}  // namespace q2w

// The elasticity apply of q2pa_el_elements in double-word FP32 arithmetic (FP64 accuracy on the FP32
// pipe), from the pair form of the partial assembly (q2pa_el_to_dw).  Each element scales its inputs
// by the power of two that brings its largest |x| to [1, 2) (exact; inputs below 2^-74 of it become 0)
// and its results back by 2^(s + ss + 2 sk), so every finite input keeps FP64-level accuracy
// relative to its element; the results go to the element's own slots as in the FP64 kernel.
__global__ void __launch_bounds__(128) q2pa_el_elements_dw(MeshView m, const float2 *__restrict__ D,
                                                          const double *__restrict__ x, int nrhs, int r,
                                                          double *__restrict__ buf, int sk, int ss,
                                                          const int *__restrict__ skip) {
  constexpr int W = 4;  // elements (warps) per block
  __shared__ float2 tB[3][3], tG[3][3];
  __shared__ float2 sU[W][3][32], sA[W][3][32], sB[W][3][32];
  if (skip && *skip) return;
  if (threadIdx.x < 9) {
    const q2::SF t = q2::sf_tables();
    const dwa::dw b = dwa::split(t.B[threadIdx.x / 3][threadIdx.x % 3]);
    const dwa::dw g = dwa::split(t.G[threadIdx.x / 3][threadIdx.x % 3]);
    tB[threadIdx.x / 3][threadIdx.x % 3] = make_float2(b.h, b.l);
    tG[threadIdx.x / 3][threadIdx.x % 3] = make_float2(g.h, g.l);
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, o = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * W + w;
  if (e >= m.n_cells) return;  // whole warps; no block barrier follows
  const bool lv = o < 27;
  float2 (*U)[32] = sU[w], (*A)[32] = sA[w], (*B)[32] = sB[w];
  double xv[3] = {0.0, 0.0, 0.0};
  dwa::MagRec mag;
  if (lv) {
    const int64_t node = cell_node(m, 27, e, o);
    const bool dir = m.dmask[node] != 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      xv[k] = dir ? 0.0 : x[(node * nrhs + r) * 3 + k];
      mag.add(xv[k]);
    }
  }
  int se = 0;
  dwa::mag_exponent(__reduce_max_sync(0xffffffffu, mag.key), se);  // all zero or not finite: se = 0
  if (lv) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const dwa::dw u = dwa::split_scaled(xv[k], se);
      U[k][o] = make_float2(u.h, u.l);
    }
  }
  __syncwarp();
  dwa::dw t[3], gx[3], gy[3], gz[3];
  if (lv) { q2w::contract3_dw<2, false, 3>(tB, U, o, t); q2w::put3_dw<3>(A, o, t); }
  __syncwarp();
  if (lv) { q2w::contract3_dw<1, false, 3>(tB, A, o, t); q2w::put3_dw<3>(B, o, t); }
  __syncwarp();
  if (lv) q2w::contract3_dw<0, false, 3>(tG, B, o, gx);
  __syncwarp();
  if (lv) { q2w::contract3_dw<1, false, 3>(tG, A, o, t); q2w::put3_dw<3>(B, o, t); }
  __syncwarp();
  if (lv) {
    q2w::contract3_dw<0, false, 3>(tB, B, o, gy);
    q2w::contract3_dw<2, false, 3>(tG, U, o, t);
    q2w::put3_dw<3>(A, o, t);
  }
  __syncwarp();
  if (lv) { q2w::contract3_dw<1, false, 3>(tB, A, o, t); q2w::put3_dw<3>(B, o, t); }
  __syncwarp();
  dwa::dw fx[3], fy[3], fz[3];
  if (lv) {
    q2w::contract3_dw<0, false, 3>(tB, B, o, gz);
    const float2 *De = D + e * kQ2ElVals * 32 + o;
    dwa::dw K[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        const float2 v = __ldg(De + (3 * c + l) * 32);
        K[c][l] = dwa::dw{v.x, v.y};
      }
    const float2 vl = __ldg(De + 9 * 32), vm = __ldg(De + 10 * 32);
    const dwa::dw slam{vl.x, vl.y}, smu{vm.x, vm.y};
    dwa::dw G[3][3];  // grad u: G[k][l] = sum_c H[k][c] K[c][l]
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = 0; l < 3; ++l)
        G[k][l] = dwa::add(dwa::add(dwa::mul(gx[k], K[0][l]), dwa::mul(gy[k], K[1][l])), dwa::mul(gz[k], K[2][l]));
    const dwa::dw tr = dwa::mul(slam, dwa::add(dwa::add(G[0][0], G[1][1]), G[2][2]));
    dwa::dw S[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        const dwa::dw sym = dwa::mul(smu, dwa::add(G[k][l], G[l][k]));
        S[k][l] = k == l ? dwa::add(sym, tr) : sym;
      }
#pragma unroll
    for (int k = 0; k < 3; ++k) {  // P[k][c] = sum_l S[k][l] K[c][l]
      fx[k] = dwa::add(dwa::add(dwa::mul(S[k][0], K[0][0]), dwa::mul(S[k][1], K[0][1])), dwa::mul(S[k][2], K[0][2]));
      fy[k] = dwa::add(dwa::add(dwa::mul(S[k][0], K[1][0]), dwa::mul(S[k][1], K[1][1])), dwa::mul(S[k][2], K[1][2]));
      fz[k] = dwa::add(dwa::add(dwa::mul(S[k][0], K[2][0]), dwa::mul(S[k][1], K[2][1])), dwa::mul(S[k][2], K[2][2]));
    }
    q2w::put3_dw<3>(A, o, fx);
  }
  __syncwarp();
  dwa::dw bb[3], v[3];
  if (lv) { q2w::contract3_dw<0, true, 3>(tG, A, o, t); q2w::put3_dw<3>(B, o, t); }
  __syncwarp();
  if (lv) { q2w::contract3_dw<1, true, 3>(tB, B, o, bb); q2w::put3_dw<3>(A, o, fy); }
  __syncwarp();
  if (lv) { q2w::contract3_dw<0, true, 3>(tB, A, o, t); q2w::put3_dw<3>(B, o, t); }
  __syncwarp();
  if (lv) {
    q2w::contract3_dw<1, true, 3>(tG, B, o, t);
#pragma unroll
    for (int k = 0; k < 3; ++k) bb[k] = dwa::add(bb[k], t[k]);
    q2w::put3_dw<3>(A, o, bb);
  }
  __syncwarp();
  if (lv) { q2w::contract3_dw<2, true, 3>(tB, A, o, v); q2w::put3_dw<3>(B, o, fz); }
  __syncwarp();
  if (lv) { q2w::contract3_dw<0, true, 3>(tB, B, o, t); q2w::put3_dw<3>(A, o, t); }
  __syncwarp();
  if (lv) { q2w::contract3_dw<1, true, 3>(tB, A, o, t); q2w::put3_dw<3>(B, o, t); }
  __syncwarp();
  if (lv) {
    q2w::contract3_dw<2, true, 3>(tG, B, o, t);
    const int so = se + ss + 2 * sk;
#pragma unroll
    for (int k = 0; k < 3; ++k) buf[(e * 27 + o) * 3 + k] = dwa::ldexp_exact(dwa::to_double(dwa::add(v[k], t[k])), so);
  }
}

// Q2 Laplace / vector Laplace partial assembly for the double-word warp kernel: the flux matrix D_q
// (6 values) per Gauss point, [element][6][32] (points q < 27 used), FP64 (converted to pairs in place
// afterwards).
__global__ void __launch_bounds__(64) q2pa_lap_build_w(MeshView m, double *__restrict__ D) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.n_cells) return;
  double X[27][3];
  for (int a = 0; a < 27; ++a) {
    const int64_t n = cell_node(m, 27, e, a);
    for (int i = 0; i < 3; ++i) X[a][i] = m.X[3 * n + i];
  }
  const double kappa = m.mat[e];
  double *De = D + e * 6 * 32;
  for (int q = 0; q < 27; ++q) {
    double xi[3];
    q2::point_q(q, xi);
    q2::Tab<double> t;
    q2::tables_at<double>(xi, t);
    double J[3][3], C[3][3];
    q2::jacobian(X, t, J);
    const double det = q1::adjugate(J, C);
    const double sc = q2::weight_q(q) * kappa / det;
    int k = 0;
    for (int r = 0; r < 3; ++r)
      for (int c = r; c < 3; ++c) De[(k++) * 32 + q] = sc * (C[r][0] * C[c][0] + C[r][1] * C[c][1] + C[r][2] * C[c][2]);
  }
}

// Extent of [element][NV][32] data: largest non-zero magnitude over all values (ext[0]) and smallest
// over the values j with bit j of `minmask` set (ext[1]) (biased FP64 exponent fields).
__global__ void q2pa_extent(const double *__restrict__ D, int64_t n_cells, int nv, unsigned minmask, unsigned *ext) {
  unsigned vmax = 0, vmin = ~0u;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_cells * nv * 32;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(i % 32), j = (int)((i / 32) % nv);
    if (q >= 27) continue;
    const unsigned e = (unsigned)((__double_as_longlong(D[i]) >> 52) & 0x7ff);
    if (e == 0) continue;
    vmax = max(vmax, e);
    if (minmask >> j & 1u) vmin = min(vmin, e);
  }
  atomicMax(ext, vmax);
  atomicMin(ext + 1, vmin);
}

// In place: the [element][NV][32] data as float pairs times 2^-sd (values below 2^-74 after it: 0).
__global__ void q2pa_to_dw(double *__restrict__ D, int64_t n_vals, int sd) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_vals; i += (int64_t)gridDim.x * blockDim.x) {
    const dwa::dw v = dwa::split_scaled(D[i], sd);
    reinterpret_cast<float2 *>(D)[i] = make_float2(v.h, v.l);
  }
}

// Q2 Laplace (NC = 1) and vector Laplace (NC = 3) apply in double-word arithmetic, one warp per
// element, as q2pa_el_elements_dw: per-element power-of-two scaling of the inputs, the 16
// contractions of every component in shared memory, per Gauss point f = D_q g for each component, the
// element's results (scaled back by 2^(s + sd)) to its own slots.
template <int NC>
__global__ void __launch_bounds__(128) q2pa_lap_elements_dw(MeshView m, const float2 *__restrict__ D,
                                                           const double *__restrict__ x, int nrhs, int r,
                                                           double *__restrict__ buf, int sd,
                                                           const int *__restrict__ skip) {
  constexpr int W = 4;
  __shared__ float2 tB[3][3], tG[3][3];
  __shared__ float2 sU[W][NC][32], sA[W][NC][32], sB[W][NC][32];
  if (skip && *skip) return;
  if (threadIdx.x < 9) {
    const q2::SF t = q2::sf_tables();
    const dwa::dw b = dwa::split(t.B[threadIdx.x / 3][threadIdx.x % 3]);
    const dwa::dw g = dwa::split(t.G[threadIdx.x / 3][threadIdx.x % 3]);
    tB[threadIdx.x / 3][threadIdx.x % 3] = make_float2(b.h, b.l);
    tG[threadIdx.x / 3][threadIdx.x % 3] = make_float2(g.h, g.l);
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, o = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * W + w;
  if (e >= m.n_cells) return;
  const bool lv = o < 27;
  float2 (*U)[32] = sU[w], (*A)[32] = sA[w], (*B)[32] = sB[w];
  double xv[NC];
  dwa::MagRec mag;
#pragma unroll
  for (int k = 0; k < NC; ++k) xv[k] = 0.0;
  if (lv) {
    const int64_t node = cell_node(m, 27, e, o);
    const bool dir = m.dmask[node] != 0;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      xv[k] = dir ? 0.0 : x[(node * nrhs + r) * NC + k];
      mag.add(xv[k]);
    }
  }
  int se = 0;
  dwa::mag_exponent(__reduce_max_sync(0xffffffffu, mag.key), se);
  if (lv) {
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const dwa::dw u = dwa::split_scaled(xv[k], se);
      U[k][o] = make_float2(u.h, u.l);
    }
  }
  __syncwarp();
  dwa::dw t[NC], gx[NC], gy[NC], gz[NC];
  if (lv) { q2w::contract3_dw<2, false, NC>(tB, U, o, t); q2w::put3_dw<NC>(A, o, t); }
  __syncwarp();
  if (lv) { q2w::contract3_dw<1, false, NC>(tB, A, o, t); q2w::put3_dw<NC>(B, o, t); }
  __syncwarp();
  if (lv) q2w::contract3_dw<0, false, NC>(tG, B, o, gx);
  __syncwarp();
  if (lv) { q2w::contract3_dw<1, false, NC>(tG, A, o, t); q2w::put3_dw<NC>(B, o, t); }
  __syncwarp();
  if (lv) {
    q2w::contract3_dw<0, false, NC>(tB, B, o, gy);
    q2w::contract3_dw<2, false, NC>(tG, U, o, t);
    q2w::put3_dw<NC>(A, o, t);
  }
  __syncwarp();
  if (lv) { q2w::contract3_dw<1, false, NC>(tB, A, o, t); q2w::put3_dw<NC>(B, o, t); }
  __syncwarp();
  dwa::dw fx[NC], fy[NC], fz[NC];
  if (lv) {
    q2w::contract3_dw<0, false, NC>(tB, B, o, gz);
    const float2 *De = D + e * 6 * 32 + o;
    dwa::dw d[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const float2 v = __ldg(De + j * 32);
      d[j] = dwa::dw{v.x, v.y};
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {  // f = D g, D symmetric: (d0 d1 d2; d1 d3 d4; d2 d4 d5)
      fx[k] = dwa::add(dwa::add(dwa::mul(d[0], gx[k]), dwa::mul(d[1], gy[k])), dwa::mul(d[2], gz[k]));
      fy[k] = dwa::add(dwa::add(dwa::mul(d[1], gx[k]), dwa::mul(d[3], gy[k])), dwa::mul(d[4], gz[k]));
      fz[k] = dwa::add(dwa::add(dwa::mul(d[2], gx[k]), dwa::mul(d[4], gy[k])), dwa::mul(d[5], gz[k]));
    }
    q2w::put3_dw<NC>(A, o, fx);
  }
  __syncwarp();
  dwa::dw bb[NC], v[NC];
  if (lv) { q2w::contract3_dw<0, true, NC>(tG, A, o, t); q2w::put3_dw<NC>(B, o, t); }
  __syncwarp();
  if (lv) { q2w::contract3_dw<1, true, NC>(tB, B, o, bb); q2w::put3_dw<NC>(A, o, fy); }
  __syncwarp();
  if (lv) { q2w::contract3_dw<0, true, NC>(tB, A, o, t); q2w::put3_dw<NC>(B, o, t); }
  __syncwarp();
  if (lv) {
    q2w::contract3_dw<1, true, NC>(tG, B, o, t);
#pragma unroll
    for (int k = 0; k < NC; ++k) bb[k] = dwa::add(bb[k], t[k]);
    q2w::put3_dw<NC>(A, o, bb);
  }
  __syncwarp();
  if (lv) { q2w::contract3_dw<2, true, NC>(tB, A, o, v); q2w::put3_dw<NC>(B, o, fz); }
  __syncwarp();
  if (lv) { q2w::contract3_dw<0, true, NC>(tB, B, o, t); q2w::put3_dw<NC>(A, o, t); }
  __syncwarp();
  if (lv) { q2w::contract3_dw<1, true, NC>(tB, A, o, t); q2w::put3_dw<NC>(B, o, t); }
  __syncwarp();
  if (lv) {
    q2w::contract3_dw<2, true, NC>(tG, B, o, t);
    const int so = se + sd;
#pragma unroll
    for (int k = 0; k < NC; ++k)
      buf[(e * 27 + o) * NC + k] = dwa::ldexp_exact(dwa::to_double(dwa::add(v[k], t[k])), so);
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
    nodes[a] = cell_node(m, 27, e, a);
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
      if (m->q2dw)
        q2pa_lap_elements_dw<1><<<(unsigned)((m->n_cells + 3) / 4), 128, 0, s>>>(
            v, reinterpret_cast<const float2 *>(m->q2pa), x, nrhs, r, m->q2buf, m->q2ss, skip);
      else
        q2pa_elements<1><<<blocks_for(m->n_cells, 64), 64, 0, s>>>(v, m->q2pa, x, nrhs, r, m->q2buf, skip);
      q2pa_gather<1><<<blocks_for(m->n_nodes), kThreads, 0, s>>>(m->n_nodes, m->q2off, m->q2slots, m->dmask,
                                                                   m->q2buf, x, y, nrhs, r, skip);
    } else if (m->physics == MF_ELASTICITY) {
      if (m->q2dw)
        q2pa_el_elements_dw<<<(unsigned)((m->n_cells + 3) / 4), 128, 0, s>>>(
            v, reinterpret_cast<const float2 *>(m->q2pa), x, nrhs, r, m->q2buf, m->q2sk, m->q2ss, skip);
      else
        q2pa_el_elements<<<(unsigned)((m->n_cells + 3) / 4), 128, 0, s>>>(v, m->q2pa, x, nrhs, r, m->q2buf, skip);
      q2pa_gather<3><<<blocks_for(m->n_nodes * 3), kThreads, 0, s>>>(m->n_nodes, m->q2off, m->q2slots, m->dmask,
                                                                       m->q2buf, x, y, nrhs, r, skip);
    } else {
      if (m->q2dw)
        q2pa_lap_elements_dw<3><<<(unsigned)((m->n_cells + 3) / 4), 128, 0, s>>>(
            v, reinterpret_cast<const float2 *>(m->q2pa), x, nrhs, r, m->q2buf, m->q2ss, skip);
      else
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
                                  : (size_t)n_cells * 6 * 32 * sizeof(double);
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
    // double-word form: J^-1 and w det J (lambda, mu) normalised by powers of two so that their largest
    // magnitudes lie in [1, 2); kept in FP64 when w det J lambda / mu span more than 2^60 (flushing the
    // smallest to 0 would change the operator)
    unsigned *ext = nullptr;
    MF_CUDA(cudaMalloc(&ext, 4 * sizeof(unsigned)));
    const unsigned init[4] = {0u, ~0u, 0u, ~0u};
    MF_CUDA(cudaMemcpyAsync(ext, init, sizeof init, cudaMemcpyHostToDevice, s));
    mf_count_launches(1);
    q2pa_el_extent<<<device_sm_count() * 4, 256, 0, s>>>(m->q2pa, m->n_cells, ext);
    unsigned h[4];
    cudaError_t ce = cudaMemcpyAsync(h, ext, sizeof h, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    cudaFree(ext);
    MF_CUDA(ce);
    const bool any_s = h[2] != 0u;
    m->q2dw = h[0] != 0u && h[0] < 0x7ffu && h[2] < 0x7ffu && (!any_s || h[2] - h[3] <= 60u);
    if (m->q2dw) {
      m->q2sk = (int)h[0] - 1023;
      m->q2ss = any_s ? (int)h[2] - 1023 : 0;
      mf_count_launches(1);
      q2pa_el_to_dw<<<device_sm_count() * 4, 256, 0, s>>>(m->q2pa, m->n_cells, m->q2sk, m->q2ss);
    }
  } else {
    // double-word form for the warp kernel ([element][6][32], normalised by the power of two that
    // brings the largest |D| to [1, 2)); the FP64 kernel's [q][6][element] layout when the diagonal
    // entries (kappa w |adj J col|^2 / det J) span more than 2^60
    MF_CUDA(cudaMemsetAsync(m->q2pa, 0, bytes, s));
    q2pa_lap_build_w<<<blocks_for(m->n_cells, 64), 64, 0, s>>>(m->view(), m->q2pa);
    unsigned *ext = nullptr;
    MF_CUDA(cudaMalloc(&ext, 2 * sizeof(unsigned)));
    const unsigned init[2] = {0u, ~0u};
    MF_CUDA(cudaMemcpyAsync(ext, init, sizeof init, cudaMemcpyHostToDevice, s));
    mf_count_launches(2);
    q2pa_extent<<<device_sm_count() * 4, 256, 0, s>>>(m->q2pa, m->n_cells, 6, 0x29u, ext);  // diagonal: j = 0, 3, 5
    unsigned h[2];
    cudaError_t ce = cudaMemcpyAsync(h, ext, sizeof h, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    cudaFree(ext);
    MF_CUDA(ce);
    m->q2dw = h[0] != 0u && h[0] < 0x7ffu && h[1] != ~0u && h[0] - h[1] <= 60u;
    if (m->q2dw) {
      m->q2ss = (int)h[0] - 1023;
      m->q2sk = 0;
      q2pa_to_dw<<<device_sm_count() * 4, 256, 0, s>>>(m->q2pa, m->n_cells * 6 * 32, m->q2ss);
    } else {
      q2pa_build<<<blocks_for(m->n_cells, 64), 64, 0, s>>>(m->view(), m->q2pa);
    }
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

MF_DBG_TU(apply)
