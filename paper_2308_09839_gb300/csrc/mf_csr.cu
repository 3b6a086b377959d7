// Matrix-based operator (Sec. 3 and Table 1): CSR assembly of the element matrices of Eqs. 4/5/6
// and the SpMV used as the baseline of the matrix-free kernels.  The vector Laplacian is stored
// block-diagonally (27 entries per row: its components do not couple).
//
// Fill: the paper describes an element loop that searches each global column and adds with an
// atomic.  Here the search is a binary search in the sorted row, and the add is a plain
// read-modify-write: elements are processed colour by colour (elements of one colour share no
// node, hence no row), which keeps the fill deterministic.
#include <algorithm>
#include <atomic>
#include <vector>

#include "mf_element.cuh"
#include "mf_internal.cuh"
#include "mf_q2.cuh"
#include "mf_tet.cuh"

namespace {

__device__ __forceinline__ int64_t parity_element_c(int64_t t, int c, int nx, int ny, int nz) {
  const int px = c & 1, py = (c >> 1) & 1, pz = (c >> 2) & 1;
  const int64_t cnx = (nx - px + 1) / 2, cny = (ny - py + 1) / 2;
  const int64_t ix = t % cnx, r = t / cnx, iy = r % cny, iz = r / cny;
  return (2 * ix + px) + (int64_t)nx * ((2 * iy + py) + (int64_t)ny * (2 * iz + pz));
}

// Rows of A^e belonging to corner a: out[k][b][l] = A^e_{ND a + k, ND b + l} (Eqs. 4 and 6).
template <int PHYS>
__device__ void element_rows(const double X[8][3], int a, double c0, double c1, double out[][8][3]) {
  constexpr int ND = phys_ndpn(PHYS);
  for (int k = 0; k < ND; ++k)
    for (int b = 0; b < 8; ++b)
      for (int l = 0; l < 3; ++l) out[k][b][l] = 0.0;
  for (int q = 0; q < 8; ++q) {
    double xi[3];
    for (int d = 0; d < 3; ++d) xi[d] = q1::sgn(q, d) * q1::kG;
    double J[3][3], C[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0;
        for (int c = 0; c < 8; ++c) s += X[c][i] * q1::dN_at(xi, c, j);
        J[i][j] = s;
      }
    const double det = q1::adjugate(J, C);
    // physical gradients g_b = J^{-T} grad_ref phi_b = C^T grad_ref phi_b / det
    double g[8][3];
    for (int b = 0; b < 8; ++b) {
      double r[3] = {q1::dN_at(xi, b, 0), q1::dN_at(xi, b, 1), q1::dN_at(xi, b, 2)};
      for (int i = 0; i < 3; ++i) g[b][i] = (C[0][i] * r[0] + C[1][i] * r[1] + C[2][i] * r[2]) / det;
    }
    const double wd = det;  // w_q = 1
    for (int b = 0; b < 8; ++b) {
      const double gg = g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2];
      if (PHYS == MF_LAPLACE) {
        out[0][b][0] += c0 * gg * wd;
      } else {
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l)
            out[k][b][l] += wd * (c0 * g[a][k] * g[b][l] + c1 * (g[a][l] * g[b][k] + (k == l ? gg : 0.0)));
      }
    }
  }
}

// Diagonal of A^e for all corners: out[a][k] = A^e_{ND a + k, ND a + k}, summed over the Gauss
// points in the same order and with the same expressions as element_rows.
template <int PHYS>
__device__ void element_diag(const double X[8][3], double c0, double c1, double out[8][3]) {
  for (int a = 0; a < 8; ++a)
    for (int k = 0; k < 3; ++k) out[a][k] = 0.0;
  for (int q = 0; q < 8; ++q) {
    double xi[3];
    for (int d = 0; d < 3; ++d) xi[d] = q1::sgn(q, d) * q1::kG;
    double J[3][3], C[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0;
        for (int c = 0; c < 8; ++c) s += X[c][i] * q1::dN_at(xi, c, j);
        J[i][j] = s;
      }
    const double det = q1::adjugate(J, C);
    const double wd = det;
    for (int a = 0; a < 8; ++a) {
      const double r[3] = {q1::dN_at(xi, a, 0), q1::dN_at(xi, a, 1), q1::dN_at(xi, a, 2)};
      double ga[3];
      for (int i = 0; i < 3; ++i) ga[i] = (C[0][i] * r[0] + C[1][i] * r[1] + C[2][i] * r[2]) / det;
      const double gg = ga[0] * ga[0] + ga[1] * ga[1] + ga[2] * ga[2];
      if (PHYS == MF_LAPLACE) {
        out[a][0] += c0 * gg * wd;
      } else {
        for (int k = 0; k < 3; ++k) out[a][k] += wd * (c0 * ga[k] * ga[k] + c1 * (ga[k] * ga[k] + gg));
      }
    }
  }
}

template <int PHYS>
__global__ void csr_fill_colour(MeshView m, int colour, int64_t count, const int32_t *__restrict__ celems,
                                const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col, double *val) {
  constexpr int ND = phys_ndpn(PHYS);
  constexpr int EP = PHYS == MF_VECTOR_LAPLACE ? MF_LAPLACE : PHYS;  // element matrix computed
  constexpr int NE = phys_ndpn(EP);
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= count * 8) return;
  const int64_t t = gid >> 3;
  const int a = (int)(gid & 7);
  const int64_t e =
      mf_dbg_index(celems ? (int64_t)celems[t] : parity_element_c(t, colour, m.nx, m.ny, m.nz), m.n_cells, MF_DBG_CELL);
  int64_t nodes[8];
  element_nodes(m, e, nodes);
  if (m.dmask[nodes[a]]) return;  // Dirichlet row: identity, set separately
  double X[8][3];
  for (int c = 0; c < 8; ++c)
    for (int i = 0; i < 3; ++i) X[c][i] = m.X[3 * nodes[c] + i];
  const double c0 = phys_is_laplace(PHYS) ? m.mat[e] : m.mat[2 * e];
  const double c1 = phys_is_laplace(PHYS) ? 0.0 : m.mat[2 * e + 1];
  double A[NE][8][3];
  element_rows<EP>(X, a, c0, c1, A);
  if constexpr (PHYS == MF_VECTOR_LAPLACE) {
    // block-diagonal: row 3 n + k couples only to columns 3 m + k, with the scalar entries
    for (int k = 0; k < 3; ++k) {
      const int64_t row = nodes[a] * 3 + k;
      for (int b = 0; b < 8; ++b) {
        if (m.dmask[nodes[b]]) continue;
        const int32_t target = (int32_t)(nodes[b] * 3 + k);
        int64_t lo = rowptr[row], hi = rowptr[row + 1];
        while (lo < hi) {
          const int64_t mid = (lo + hi) >> 1;
          if (col[mid] < target) lo = mid + 1; else hi = mid;
        }
        val[lo] += A[0][b][0];
      }
    }
    return;
  }
  const int64_t row0 = nodes[a] * ND;
  const int64_t lo0 = rowptr[row0], hi0 = rowptr[row0 + 1];
  for (int b = 0; b < 8; ++b) {
    if (m.dmask[nodes[b]]) continue;  // Dirichlet column dropped
    const int32_t target = (int32_t)(nodes[b] * ND);
    int64_t lo = lo0, hi = hi0;  // binary search for the first column of node b
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (col[mid] < target) lo = mid + 1; else hi = mid;
    }
    const int64_t rel = lo - lo0;
    for (int k = 0; k < ND; ++k) {
      const int64_t base = rowptr[row0 + k] + rel;
      for (int l = 0; l < ND; ++l) val[base + l] += A[k][b][l];
    }
  }
}

template <int PHYS>
__global__ void diag_colour(MeshView m, int colour, int64_t count, const int32_t *__restrict__ celems, double *diag) {
  constexpr int ND = phys_ndpn(PHYS);
  constexpr int EP = PHYS == MF_VECTOR_LAPLACE ? MF_LAPLACE : PHYS;
  constexpr int NE = phys_ndpn(EP);
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // one element per thread
  if (t >= count) return;
  const int64_t e =
      mf_dbg_index(celems ? (int64_t)celems[t] : parity_element_c(t, colour, m.nx, m.ny, m.nz), m.n_cells, MF_DBG_CELL);
  int64_t nodes[8];
  element_nodes(m, e, nodes);
  double X[8][3];
  for (int c = 0; c < 8; ++c)
    for (int i = 0; i < 3; ++i) X[c][i] = m.X[3 * nodes[c] + i];
  const double c0 = phys_is_laplace(PHYS) ? m.mat[e] : m.mat[2 * e];
  const double c1 = phys_is_laplace(PHYS) ? 0.0 : m.mat[2 * e + 1];
  double D[8][3];
  element_diag<EP>(X, c0, c1, D);
  // elements of one colour share no node: plain adds
  for (int a = 0; a < 8; ++a) {
    if (m.dmask[nodes[a]]) continue;
    for (int k = 0; k < ND; ++k) diag[nodes[a] * ND + k] += NE == 1 ? D[a][0] : D[a][k];
  }
}

// P1 tetrahedra: rows of node a of A^e (mf_tet.cuh) added into the CSR values, one thread per
// (element, node) of a colour.  Same search as csr_fill_colour: the three rows of a node share
// their column pattern, so the offset found in the first row serves all three.
template <int PHYS>
__global__ void tet_fill_colour(MeshView m, int64_t count, const int32_t *__restrict__ celems,
                                const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col, double *val) {
  constexpr int ND = phys_ndpn(PHYS);
  constexpr int EP = PHYS == MF_VECTOR_LAPLACE ? MF_LAPLACE : PHYS;
  constexpr int NE = phys_ndpn(EP);
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= count * 4) return;
  const int64_t e = mf_dbg_index((int64_t)celems[gid >> 2], m.n_cells, MF_DBG_CELL);
  const int a = (int)(gid & 3);
  int64_t nodes[4];
  p1::nodes_of(m.cells, e, nodes);
#pragma unroll
  for (int a = 0; a < 4; ++a) nodes[a] = mf_dbg_index(nodes[a], m.n_nodes, MF_DBG_NODE);
  if (m.dmask[nodes[a]]) return;  // Dirichlet row: identity, set separately
  double X[4][3], n[4][3];
  for (int c = 0; c < 4; ++c)
    for (int i = 0; i < 3; ++i) X[c][i] = m.X[3 * nodes[c] + i];
  const double D = p1::geometry<double>(X, n);
  const double c0 = phys_is_laplace(PHYS) ? m.mat[e] : m.mat[2 * e];
  const double c1 = phys_is_laplace(PHYS) ? 0.0 : m.mat[2 * e + 1];
  double A[NE][4][3];
  p1::element_rows<EP>(n, D, a, c0, c1, A);
  for (int b = 0; b < 4; ++b) {
    if (m.dmask[nodes[b]]) continue;  // Dirichlet column dropped
    for (int k = 0; k < (PHYS == MF_VECTOR_LAPLACE ? 3 : 1); ++k) {
      // vector Laplace: row 3 n + k holds only the columns 3 m + k (block-diagonal pattern)
      const int64_t row = nodes[a] * ND + k;
      const int32_t target = (int32_t)(nodes[b] * ND + (PHYS == MF_VECTOR_LAPLACE ? k : 0));
      int64_t lo = rowptr[row], hi = rowptr[row + 1];
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < target) lo = mid + 1; else hi = mid;
      }
      if (PHYS == MF_VECTOR_LAPLACE) {
        val[lo] += A[0][b][0];
      } else {
        const int64_t rel = lo - rowptr[row];
        for (int kk = 0; kk < ND; ++kk) {
          const int64_t base = rowptr[nodes[a] * ND + kk] + rel;
          for (int l = 0; l < ND; ++l) val[base + l] += NE == 1 ? A[0][b][0] : A[kk][b][l];
        }
      }
    }
  }
}

// Q2 hexahedra: rows of node a of A^e (mf_q2.cuh), one thread per (element, node) of a colour.
template <int PHYS>
__global__ void __launch_bounds__(64) q2_fill_colour(MeshView m, int64_t count, const int32_t *__restrict__ celems,
                                                     const int64_t *__restrict__ rowptr,
                                                     const int32_t *__restrict__ col, double *val) {
  constexpr int ND = phys_ndpn(PHYS);
  constexpr int EP = PHYS == MF_VECTOR_LAPLACE ? MF_LAPLACE : PHYS;
  constexpr int NE = phys_ndpn(EP);
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= count * 27) return;
  const int64_t e = mf_dbg_index((int64_t)celems[gid / 27], m.n_cells, MF_DBG_CELL);
  const int a = (int)(gid % 27);
  int64_t nodes[27];
  for (int c = 0; c < 27; ++c) nodes[c] = cell_node(m, 27, e, c);
  if (m.dmask[nodes[a]]) return;  // Dirichlet row: identity, set separately
  double X[27][3];
  for (int c = 0; c < 27; ++c)
    for (int i = 0; i < 3; ++i) X[c][i] = m.X[3 * nodes[c] + i];
  const double c0 = phys_is_laplace(PHYS) ? m.mat[e] : m.mat[2 * e];
  const double c1 = phys_is_laplace(PHYS) ? 0.0 : m.mat[2 * e + 1];
  double A[NE][27][3];
  q2::element_rows<EP>(X, a, c0, c1, A);
  for (int b = 0; b < 27; ++b) {
    if (m.dmask[nodes[b]]) continue;  // Dirichlet column dropped
    for (int k = 0; k < (PHYS == MF_VECTOR_LAPLACE ? 3 : 1); ++k) {
      const int64_t row = nodes[a] * ND + k;
      const int32_t target = (int32_t)(nodes[b] * ND + (PHYS == MF_VECTOR_LAPLACE ? k : 0));
      int64_t lo = rowptr[row], hi = rowptr[row + 1];
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < target) lo = mid + 1; else hi = mid;
      }
      if (PHYS == MF_VECTOR_LAPLACE) {
        val[lo] += A[0][b][0];
      } else {
        const int64_t rel = lo - rowptr[row];
        for (int kk = 0; kk < ND; ++kk) {
          const int64_t base = rowptr[nodes[a] * ND + kk] + rel;
          for (int l = 0; l < ND; ++l) val[base + l] += NE == 1 ? A[0][b][0] : A[kk][b][l];
        }
      }
    }
  }
}

// diag(A) of Q2 hexahedra, one thread per element of a colour.
template <int PHYS>
__global__ void __launch_bounds__(64) q2_diag_colour(MeshView m, int64_t count, const int32_t *__restrict__ celems,
                                                     double *diag) {
  constexpr int ND = phys_ndpn(PHYS);
  constexpr int EP = PHYS == MF_VECTOR_LAPLACE ? MF_LAPLACE : PHYS;
  constexpr int NE = phys_ndpn(EP);
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t e = mf_dbg_index((int64_t)celems[t], m.n_cells, MF_DBG_CELL);
  int64_t nodes[27];
  double X[27][3];
  for (int c = 0; c < 27; ++c) {
    nodes[c] = cell_node(m, 27, e, c);
    for (int i = 0; i < 3; ++i) X[c][i] = m.X[3 * nodes[c] + i];
  }
  const double c0 = phys_is_laplace(PHYS) ? m.mat[e] : m.mat[2 * e];
  const double c1 = phys_is_laplace(PHYS) ? 0.0 : m.mat[2 * e + 1];
  double D[27][3];
  q2::element_diag<EP>(X, c0, c1, D);
  for (int a = 0; a < 27; ++a) {
    if (m.dmask[nodes[a]]) continue;
    for (int k = 0; k < ND; ++k) diag[nodes[a] * ND + k] += NE == 1 ? D[a][0] : D[a][k];
  }
}

// diag(A) of P1 tetrahedra, one thread per element of a colour.
template <int PHYS>
__global__ void tet_diag_colour(MeshView m, int64_t count, const int32_t *__restrict__ celems, double *diag) {
  constexpr int ND = phys_ndpn(PHYS);
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t e = mf_dbg_index((int64_t)celems[t], m.n_cells, MF_DBG_CELL);
  int64_t nodes[4];
  p1::nodes_of(m.cells, e, nodes);
#pragma unroll
  for (int a = 0; a < 4; ++a) nodes[a] = mf_dbg_index(nodes[a], m.n_nodes, MF_DBG_NODE);
  double X[4][3], n[4][3];
  for (int c = 0; c < 4; ++c)
    for (int i = 0; i < 3; ++i) X[c][i] = m.X[3 * nodes[c] + i];
  const double D = p1::geometry<double>(X, n);
  const double c0 = phys_is_laplace(PHYS) ? m.mat[e] : m.mat[2 * e];
  const double c1 = phys_is_laplace(PHYS) ? 0.0 : m.mat[2 * e + 1];
  const double c = 1.0 / (6.0 * D);
  for (int a = 0; a < 4; ++a) {
    if (m.dmask[nodes[a]]) continue;
    const double nn = n[a][0] * n[a][0] + n[a][1] * n[a][1] + n[a][2] * n[a][2];
    for (int k = 0; k < ND; ++k)
      diag[nodes[a] * ND + k] +=
          phys_is_laplace(PHYS) ? c0 * nn * c : c * (c0 * n[a][k] * n[a][k] + c1 * (n[a][k] * n[a][k] + nn));
  }
}

__global__ void dirichlet_unit(const int32_t *dn, int64_t n, int nd, const int64_t *rowptr, double *val) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n * nd) return;
  const int64_t row = (int64_t)dn[i / nd] * nd + i % nd;
  val[rowptr[row]] = 1.0;
}

__global__ void dirichlet_diag(const int32_t *dn, int64_t n, int nd, double *diag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n * nd) return;
  diag[(int64_t)dn[i / nd] * nd + i % nd] = 1.0;
}

// Expand the node-level neighbour lists to DoF-level columns: row ND*n + k holds ND*m + l for every
// neighbour m of n (l = 0..ND-1), or only its own diagonal when n is constrained.
__global__ void expand_columns(int64_t n_nodes, int nd, bool blockdiag, const int64_t *__restrict__ noff,
                               const int32_t *__restrict__ nbr, const uint8_t *__restrict__ dmask,
                               const int64_t *__restrict__ rowptr, int32_t *col) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_nodes * nd) return;
  const int64_t n = i / nd, k = i % nd;
  int64_t p = rowptr[i];
  if (dmask[n]) {
    col[p] = (int32_t)i;
    return;
  }
  for (int64_t t = noff[n]; t < noff[n + 1]; ++t) {
    if (blockdiag) {
      col[p++] = (int32_t)(nbr[t] * nd + k);  // component k couples to component k only
    } else {
      for (int l = 0; l < nd; ++l) col[p++] = nbr[t] * nd + l;
    }
  }
}

// y = A x in FP64 with L lanes per row and 16-byte loads.  On GB300 the FP64 pipe runs about 0.6 T
// fused multiply-adds per second, about as fast as HBM delivers the 12-byte entries, so the kernel is
// shaped to spend as few FP64 instructions as possible beside the one multiply-add per entry: few lanes
// per row (2 for up to 27 entries, 4 for up to 87), so that the shuffle tree that combines them is
// short.  Lane l of a row reads the value pairs (and column pairs) a0 + 2 (l + L u), u < U, from the even
// index a0 at or just below the row start, so that every load is aligned; entries outside the row are
// skipped.  The arrays carry padding entries past nnz so that the pair at the end of the last row stays
// in bounds.  Rows longer than 2 L U - 1 continue in a tail loop.  Each lane sums its entries in
// order; the lane sums are combined by a fixed shuffle tree (deterministic).
// lanes per row for rows of up to 31 entries (27-point stencils, tetrahedra)
constexpr int kShortRowLanes = 4;

template <int L, int U>
__global__ void __launch_bounds__(256) spmv_pairs(int64_t n_rows, const int64_t *__restrict__ rowptr,
                                                  const int32_t *__restrict__ col, const double *__restrict__ val,
                                                  const double *__restrict__ x, double *__restrict__ y,
                                                  const int *__restrict__ skip) {
  if (skip && *skip) return;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t row = gid / L;
  const int lane = (int)(gid % L);
  double acc = 0.0;
  if (row < n_rows) {
    const int64_t beg = __ldg(rowptr + row), end = __ldg(rowptr + row + 1);
    const int64_t a0 = beg & ~(int64_t)1;
    double2 v[U];
    int2 c[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t p = a0 + 2 * (lane + (int64_t)L * u);
      if (p < end) {
        v[u] = __ldcs(reinterpret_cast<const double2 *>(val + p));
        c[u] = __ldcs(reinterpret_cast<const int2 *>(col + p));
      } else {
        v[u] = make_double2(0.0, 0.0);
        c[u] = make_int2(0, 0);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t p = a0 + 2 * (lane + (int64_t)L * u);
      if (p >= beg && p < end) acc = __fma_rn(v[u].x, __ldg(x + mf_dbg_index(c[u].x, (int)n_rows, MF_DBG_COLUMN)), acc);
      if (p + 1 < end) acc = __fma_rn(v[u].y, __ldg(x + mf_dbg_index(c[u].y, (int)n_rows, MF_DBG_COLUMN)), acc);
    }
    for (int64_t p = a0 + 2 * (lane + (int64_t)L * U); p < end; p += 2 * L) {
      const double2 vv = __ldcs(reinterpret_cast<const double2 *>(val + p));
      const int2 cc = __ldcs(reinterpret_cast<const int2 *>(col + p));
      acc = __fma_rn(vv.x, __ldg(x + mf_dbg_index(cc.x, (int)n_rows, MF_DBG_COLUMN)), acc);
      if (p + 1 < end) acc = __fma_rn(vv.y, __ldg(x + mf_dbg_index(cc.y, (int)n_rows, MF_DBG_COLUMN)), acc);
    }
  }
#pragma unroll
  for (int off = L / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (row < n_rows && lane == 0) y[row] = acc;
}

template <int PHYS>
void launch_fill(const mf_mesh *m, const MeshView &v, const mf_csr *A, cudaStream_t s) {
  for (int c = 0; c < m->n_colours; ++c) {
    const int64_t cnt = colour_count(m, c);
    if (!cnt) continue;
    const int32_t *ce = m->structured ? nullptr : m->colour_elems + m->colour_off[c];
    if (m->npe == 4)
      tet_fill_colour<PHYS><<<blocks_for(cnt * 4, 128), 128, 0, s>>>(v, cnt, ce, A->rowptr, A->col, A->val);
    else if (m->npe == 27)
      q2_fill_colour<PHYS><<<blocks_for(cnt * 27, 64), 64, 0, s>>>(v, cnt, ce, A->rowptr, A->col, A->val);
    else
      csr_fill_colour<PHYS><<<blocks_for(cnt * 8, 128), 128, 0, s>>>(v, c, cnt, ce, A->rowptr, A->col, A->val);
  }
}

template <int PHYS>
void launch_diag(const mf_mesh *m, const MeshView &v, double *diag, cudaStream_t s) {
  for (int c = 0; c < m->n_colours; ++c) {
    const int64_t cnt = colour_count(m, c);
    if (!cnt) continue;
    const int32_t *ce = m->structured ? nullptr : m->colour_elems + m->colour_off[c];
    if (m->npe == 4) tet_diag_colour<PHYS><<<blocks_for(cnt, 128), 128, 0, s>>>(v, cnt, ce, diag);
    else if (m->npe == 27) q2_diag_colour<PHYS><<<blocks_for(cnt, 64), 64, 0, s>>>(v, cnt, ce, diag);
    else diag_colour<PHYS><<<blocks_for(cnt, 128), 128, 0, s>>>(v, c, cnt, ce, diag);
  }
}

// Node-level neighbour lists (sorted, Dirichlet neighbours removed) on the host.
void node_neighbours(const mf_mesh *m, const std::vector<uint8_t> &dmask, std::vector<int64_t> &off,
                     std::vector<int32_t> &nbr) {
  const int64_t N = m->n_nodes;
  off.assign(N + 1, 0);
  if (m->structured) {
    const int nx = m->nx, ny = m->ny, nz = m->nz;
    // count
    for (int k = 0; k <= nz; ++k)
      for (int j = 0; j <= ny; ++j)
        for (int i = 0; i <= nx; ++i) {
          const int64_t n = i + (int64_t)(nx + 1) * (j + (int64_t)(ny + 1) * k);
          int64_t c = 0;
          if (!dmask[n])
            for (int dk = -1; dk <= 1; ++dk)
              for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di) {
                  const int ii = i + di, jj = j + dj, kk = k + dk;
                  if (ii < 0 || jj < 0 || kk < 0 || ii > nx || jj > ny || kk > nz) continue;
                  if (dmask[ii + (int64_t)(nx + 1) * (jj + (int64_t)(ny + 1) * kk)]) continue;
                  ++c;
                }
          off[n + 1] = c;
        }
    for (int64_t n = 0; n < N; ++n) off[n + 1] += off[n];
    nbr.resize(off[N]);
    for (int k = 0; k <= nz; ++k)
      for (int j = 0; j <= ny; ++j)
        for (int i = 0; i <= nx; ++i) {
          const int64_t n = i + (int64_t)(nx + 1) * (j + (int64_t)(ny + 1) * k);
          if (dmask[n]) continue;
          int64_t p = off[n];
          for (int dk = -1; dk <= 1; ++dk)
            for (int dj = -1; dj <= 1; ++dj)
              for (int di = -1; di <= 1; ++di) {
                const int ii = i + di, jj = j + dj, kk = k + dk;
                if (ii < 0 || jj < 0 || kk < 0 || ii > nx || jj > ny || kk > nz) continue;
                const int64_t mm = ii + (int64_t)(nx + 1) * (jj + (int64_t)(ny + 1) * kk);
                if (dmask[mm]) continue;
                nbr[p++] = (int32_t)mm;
              }
        }
    return;
  }
  const std::vector<int32_t> &cells = m->h_cells;
  const int64_t E = m->n_cells;
  const int npe = m->npe;
  std::vector<int64_t> eoff(N + 1, 0);
  for (int64_t i = 0; i < npe * E; ++i) eoff[cells[i] + 1]++;
  for (int64_t n = 0; n < N; ++n) eoff[n + 1] += eoff[n];
  std::vector<int64_t> fill(eoff.begin(), eoff.end() - 1);
  std::vector<int32_t> adj(npe * E);
  for (int64_t e = 0; e < E; ++e)
    for (int a = 0; a < npe; ++a) adj[fill[cells[npe * e + a]]++] = (int32_t)e;
  std::vector<std::vector<int32_t>> lists(N);
  std::vector<int32_t> tmp;
  for (int64_t n = 0; n < N; ++n) {
    if (dmask[n]) continue;
    tmp.clear();
    for (int64_t t = eoff[n]; t < eoff[n + 1]; ++t)
      for (int a = 0; a < npe; ++a) {
        const int32_t mm = cells[npe * (int64_t)adj[t] + a];
        if (!dmask[mm]) tmp.push_back(mm);
      }
    std::sort(tmp.begin(), tmp.end());
    tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
    lists[n] = tmp;
    off[n + 1] = (int64_t)tmp.size();
  }
  for (int64_t n = 0; n < N; ++n) off[n + 1] += off[n];
  nbr.resize(off[N]);
  for (int64_t n = 0; n < N; ++n) std::copy(lists[n].begin(), lists[n].end(), nbr.begin() + off[n]);
}

}  // namespace

mf_status spmv(const mf_csr *A, const double *x, double *y, cudaStream_t s, const int *skip) {
  mf_count_launches(1);
  // 2 L U value slots per row: 32 for rows of up to 31 entries, 88 for up to 87, 128 (and the tail
  // loop) beyond
  const int64_t maxrow = A->max_row;
  if (maxrow <= 31) {
    constexpr int L = kShortRowLanes, U = 32 / (2 * kShortRowLanes);
    spmv_pairs<L, U><<<blocks_for(A->n_rows * L), kThreads, 0, s>>>(A->n_rows, A->rowptr, A->col, A->val, x, y, skip);
  } else if (maxrow <= 87) {
    spmv_pairs<4, 11><<<blocks_for(A->n_rows * 4), kThreads, 0, s>>>(A->n_rows, A->rowptr, A->col, A->val, x, y, skip);
  } else {
    spmv_pairs<8, 8><<<blocks_for(A->n_rows * 8), kThreads, 0, s>>>(A->n_rows, A->rowptr, A->col, A->val, x, y, skip);
  }
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

mf_status operator_diagonal(const mf_mesh *m, double *diag, cudaStream_t s) {
  MF_CUDA(cudaMemsetAsync(diag, 0, m->n_dof * sizeof(double), s));
  const MeshView v = m->view();
  if (m->physics == MF_LAPLACE) launch_diag<MF_LAPLACE>(m, v, diag, s);
  else if (m->physics == MF_VECTOR_LAPLACE) launch_diag<MF_VECTOR_LAPLACE>(m, v, diag, s);
  else launch_diag<MF_ELASTICITY>(m, v, diag, s);
  if (m->n_dnodes) dirichlet_diag<<<blocks_for(m->n_dnodes * m->ndpn), kThreads, 0, s>>>(m->dnodes, m->n_dnodes, m->ndpn, diag);
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

extern "C" mf_status mf_assemble_csr(const mf_mesh *m, mf_stream stream, mf_csr **out) {
  MF_RANGE("mf_assemble_csr");
  mf_clear_error();
  MF_ARG(m && out, "mf_assemble_csr: null argument");
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  const int nd = m->ndpn;
  const bool blockdiag = m->physics == MF_VECTOR_LAPLACE;  // components do not couple
  std::vector<uint8_t> hmask(m->n_nodes);
  MF_CUDA(cudaMemcpyAsync(hmask.data(), m->dmask, m->n_nodes, cudaMemcpyDeviceToHost, s));
  MF_CUDA(cudaStreamSynchronize(s));
  std::vector<int64_t> noff;
  std::vector<int32_t> nbr;
  node_neighbours(m, hmask, noff, nbr);
  // DoF-level row pointers
  const int64_t n_rows = m->n_nodes * nd;
  std::vector<int64_t> rowptr(n_rows + 1, 0);
  for (int64_t n = 0; n < m->n_nodes; ++n)
    for (int k = 0; k < nd; ++k) rowptr[n * nd + k + 1] = hmask[n] ? 1 : (noff[n + 1] - noff[n]) * (blockdiag ? 1 : nd);
  for (int64_t r = 0; r < n_rows; ++r) rowptr[r + 1] += rowptr[r];
  const int64_t nnz = rowptr[n_rows];
  MF_ARG(nnz < (int64_t)INT32_MAX * 4, "mf_assemble_csr: matrix too large");

  mf_csr *A = new mf_csr();
  static std::atomic<uint64_t> next_id{1};
  A->id = next_id.fetch_add(1);
  A->n_rows = n_rows;
  A->nnz = nnz;
  int64_t maxrow = 0;
  for (int64_t r = 0; r < n_rows; ++r) maxrow = std::max(maxrow, rowptr[r + 1] - rowptr[r]);
  A->max_row = maxrow;
  int64_t *d_noff = nullptr;
  int32_t *d_nbr = nullptr;
  auto cleanup = [&]() {
    cudaFree(d_noff);
    cudaFree(d_nbr);
  };
  cudaError_t e = cudaSuccess;
  if ((e = cudaMalloc(&A->rowptr, (n_rows + 1) * sizeof(int64_t))) != cudaSuccess ||
      (e = cudaMalloc(&A->col, (nnz + 2) * sizeof(int32_t))) != cudaSuccess ||  // + 2: pair loads (spmv_pairs)
      (e = cudaMalloc(&A->val, (nnz + 2) * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&d_noff, noff.size() * sizeof(int64_t))) != cudaSuccess ||
      (e = cudaMalloc(&d_nbr, std::max<size_t>(nbr.size(), 1) * sizeof(int32_t))) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    mf_destroy_csr(A);
    mf_set_error("mf_assemble_csr: allocation of %lld non-zeros failed: %s", (long long)nnz, cudaGetErrorString(e));
    return MF_ERR_OOM;
  }
  MF_CUDA(cudaMemcpyAsync(A->rowptr, rowptr.data(), rowptr.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  MF_CUDA(cudaMemcpyAsync(d_noff, noff.data(), noff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  if (!nbr.empty()) MF_CUDA(cudaMemcpyAsync(d_nbr, nbr.data(), nbr.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  expand_columns<<<blocks_for(n_rows), kThreads, 0, s>>>(m->n_nodes, nd, blockdiag, d_noff, d_nbr, m->dmask, A->rowptr,
                                                          A->col);
  MF_CUDA(cudaMemsetAsync(A->val, 0, (nnz + 2) * sizeof(double), s));
  MF_CUDA(cudaMemsetAsync(A->col + nnz, 0, 2 * sizeof(int32_t), s));
  const MeshView v = m->view();
  if (m->physics == MF_LAPLACE) launch_fill<MF_LAPLACE>(m, v, A, s);
  else if (m->physics == MF_VECTOR_LAPLACE) launch_fill<MF_VECTOR_LAPLACE>(m, v, A, s);
  else launch_fill<MF_ELASTICITY>(m, v, A, s);
  if (m->n_dnodes) dirichlet_unit<<<blocks_for(m->n_dnodes * nd), kThreads, 0, s>>>(m->dnodes, m->n_dnodes, nd, A->rowptr, A->val);
  MF_CUDA(cudaGetLastError());
  MF_CUDA(cudaStreamSynchronize(s));
  cleanup();
  *out = A;
  return MF_OK;
}

extern "C" mf_status mf_csr_query(const mf_csr *A, int64_t *n_rows, int64_t *nnz, const int64_t **rowptr,
                                  const int32_t **col, const double **val) {
  MF_ARG(A != nullptr, "mf_csr_query: csr is NULL");
  if (n_rows) *n_rows = A->n_rows;
  if (nnz) *nnz = A->nnz;
  if (rowptr) *rowptr = A->rowptr;
  if (col) *col = A->col;
  if (val) *val = A->val;
  return MF_OK;
}

extern "C" mf_status mf_csr_export(const mf_csr *A, int64_t *rowptr, int32_t *col, double *val, mf_stream stream) {
  mf_clear_error();
  MF_ARG(A && rowptr && col && val, "mf_csr_export: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  MF_CUDA(cudaMemcpyAsync(rowptr, A->rowptr, (A->n_rows + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  MF_CUDA(cudaMemcpyAsync(col, A->col, A->nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  MF_CUDA(cudaMemcpyAsync(val, A->val, A->nnz * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return MF_OK;
}

extern "C" mf_status mf_spmv_csr(const mf_csr *A, const double *x, double *y, mf_stream stream) {
  MF_RANGE("mf_spmv_csr");
  mf_clear_error();
  MF_ARG(A && x && y, "mf_spmv_csr: null argument");
  const size_t bytes = A->n_rows * sizeof(double);
  MF_ARG((const char *)x + bytes <= (const char *)y || (const char *)y + bytes <= (const char *)x,
         "mf_spmv_csr: x and y overlap");
  return spmv(A, x, y, (cudaStream_t)stream);
}

extern "C" mf_status mf_destroy_csr(mf_csr *A) {
  if (!A) return MF_OK;
  cudaDeviceSynchronize();
  cudaFree(A->rowptr);
  cudaFree(A->col);
  cudaFree(A->val);
  delete A;
  return MF_OK;
}

MF_DBG_TU(csr)
