// Matrix-free apply for structured boxes with arbitrary (e.g. jittered) node coordinates,
// FP64-accurate on the FP32 pipes: Algorithm 1 with the Jacobian, its adjugate and determinant at
// every Gauss point, in double-word arithmetic, with the owner-computes z-marching tiles of
// mf_tile.cuh.
//
// Coordinates: the cell differences that build J must keep FP64 accuracy, which a float pair of the
// absolute coordinate (48 bits) would lose to cancellation on fine meshes.  So the node coordinate
// is stored as a tensor-product base grid (per-axis values from the mesh's x-, y- and z-axis node
// lines, as spacings) plus the node's offset from it, delta = X - X_base, as a float pair.  Then
// J = diag(h)/2 + sum_a delta_a (x) grad_ref phi_a, where the offsets are small, so their pair
// representation is accurate to ~2^-48 |delta|.
//
// Element arithmetic in the monomial (Walsh-Hadamard) basis: with c = H u / 8 (and likewise for
// the three offset components), the reference gradient at Gauss point q is, for direction j with
// the other axes k < l,
//   d_j u(q) = c_{j} + s_k g c_{jk} + s_l g c_{jl} + s_k s_l g^2 c_{jkl},   g = 1/sqrt(3),
// and the transposed map accumulates the flux back into the same modes; v = H^T w.
// Laplace: flux f = kappa adj(J) adj(J)^T grad_ref u / det J (Eq. 7).  Elasticity: grad u =
// H adj(J) / det J, sigma = lam tr(eps) I + 2 mu eps, P = sigma adj(J)^T (Algorithm 1).
#include <algorithm>
#include <type_traits>

#include "mf_element.cuh"
#include "mf_tile.cuh"

using namespace tile;
using dwa::dw;

namespace {

// g = 1/sqrt(3) and g^2 = 1/3 as (hi, lo) pairs
#define C_G 0x1.279a74p-1f, 0x1.640cc8p-27f
#define C_G2 0x1.555556p-2f, -0x1.555556p-27f

struct GenArgs {
  int nx, ny, nz;
  int tiles_x, tiles_y, seg;
  const float2 *hh;     // half spacings of the base grid: [hx/2 (nx) | hy/2 (ny) | hz/2 (nz)]
  const float2 *delta;  // [N][3] offsets from the base grid
  const float2 *mat;    // kappa[E] or (lam, mu)[E]
  const uint8_t *dmask;
  const void *pa;       // partial-assembly data (float2 or float, see PaView), or null
  int64_t n_cells;
  int oscale;           // y = 2^oscale (operator of the normalised cell constants and coordinates) x
};

// v or -v (negation of a float pair is exact: both parts change sign)
template <class N>
__device__ __forceinline__ typename N::T sgn(typename N::T v, int s) {
  return s > 0 ? v : N::neg(v);
}

// Hadamard coefficients of 8 nodal values, scaled by 1/8, bilinear modes times g, trilinear
// mode times g^2 (so a Gauss-point derivative is a signed sum of four coefficients).
template <class N>
__device__ __forceinline__ void modes(typename N::T c[8]) {
  fwht_fwd<N>(c);
#pragma unroll
  for (int m = 0; m < 8; ++m) c[m] = N::scale(c[m], 0.125f);
  c[3] = N::mul(c[3], N::c(C_G));
  c[5] = N::mul(c[5], N::c(C_G));
  c[6] = N::mul(c[6], N::c(C_G));
  c[7] = N::mul(c[7], N::c(C_G2));
}

// derivative along axis j at the Gauss point with signs s[] from its mode coefficients
template <class N>
__device__ __forceinline__ typename N::T dref(const typename N::T c[8], int j, const int s[3]) {
  const int k = j == 0 ? 1 : 0, l = j == 2 ? 1 : 2;
  const int mj = 1 << j, mk = mj | (1 << k), ml = mj | (1 << l);
  typename N::T v = N::add(c[mj], sgn<N>(c[mk], s[k]));
  v = N::add(v, sgn<N>(c[ml], s[l]));
  return N::add(v, sgn<N>(c[7], s[k] * s[l]));
}

// accumulate flux component f along axis j into slot accumulators A[4] (linear, k, l, kl)
template <class N>
__device__ __forceinline__ void accum(typename N::T A[4], typename N::T f, int j, const int s[3]) {
  const int k = j == 0 ? 1 : 0, l = j == 2 ? 1 : 2;
  A[0] = N::add(A[0], f);
  A[1] = N::add(A[1], sgn<N>(f, s[k]));
  A[2] = N::add(A[2], sgn<N>(f, s[l]));
  A[3] = N::add(A[3], sgn<N>(f, s[k] * s[l]));
}

// slot accumulators of the three directions -> mode vector w (times 1/8), then v = H^T w
template <class N>
__device__ __forceinline__ void unmodes(const typename N::T A[3][4], typename N::T v[8]) {
  v[0] = N::zero();
  v[1] = A[0][0];
  v[2] = A[1][0];
  v[4] = A[2][0];
  v[3] = N::mul(N::add(A[0][1], A[1][1]), N::c(C_G));  // xi eta: dir 0 slot k=1, dir 1 slot k=0
  v[5] = N::mul(N::add(A[0][2], A[2][1]), N::c(C_G));  // xi zeta: dir 0 slot l=2, dir 2 slot k=0
  v[6] = N::mul(N::add(A[1][2], A[2][2]), N::c(C_G));  // eta zeta: dir 1 slot l=2, dir 2 slot l=1
  v[7] = N::mul(N::add(N::add(A[0][3], A[1][3]), A[2][3]), N::c(C_G2));
#pragma unroll
  for (int m = 1; m < 8; ++m) v[m] = N::scale(v[m], 0.125f);
  fwht_inv<N>(v);
}

// J at the Gauss point: J_ij = hh_i delta_ij + d_j delta_i
template <class N>
__device__ __forceinline__ void jac(const typename N::T cd[3][8], const typename N::T hh[3], const int s[3],
                                    typename N::T J[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      J[i][j] = dref<N>(cd[i], j, s);
      if (i == j) J[i][j] = N::add(J[i][j], hh[i]);
    }
}

template <class N>
__device__ __forceinline__ typename N::T adj(const typename N::T J[3][3], typename N::T C[3][3]) {
#define M2(a, b, c, d) N::sub(N::mul(J a, J b), N::mul(J c, J d))
  C[0][0] = M2([1][1], [2][2], [1][2], [2][1]);
  C[0][1] = M2([0][2], [2][1], [0][1], [2][2]);
  C[0][2] = M2([0][1], [1][2], [0][2], [1][1]);
  C[1][0] = M2([1][2], [2][0], [1][0], [2][2]);
  C[1][1] = M2([0][0], [2][2], [0][2], [2][0]);
  C[1][2] = M2([0][2], [1][0], [0][0], [1][2]);
  C[2][0] = M2([1][0], [2][1], [1][1], [2][0]);
  C[2][1] = M2([0][1], [2][0], [0][0], [2][1]);
  C[2][2] = M2([0][0], [1][1], [0][1], [1][0]);
#undef M2
  return N::add(N::add(N::mul(J[0][0], C[0][0]), N::mul(J[0][1], C[1][0])), N::mul(J[0][2], C[2][0]));
}

template <class N>
__device__ __forceinline__ typename N::T ndiv(typename N::T a, typename N::T b);
template <>
__device__ __forceinline__ dw ndiv<NumDW>(dw a, dw b) { return dwa::div(a, b); }
template <>
__device__ __forceinline__ float ndiv<NumF32>(float a, float b) { return a / b; }

// Stored quadrature-point data of partial assembly (Table 3), as pairs (DW) or floats (FP32):
// pa[(q * K + k) * n_cells + e].  Laplace and vector Laplace: K = 6, the symmetric flux matrix
// D_q = kappa w adj(J) adj(J)^T / det J (entries 00 01 02 11 12 22); elasticity: K = 10, adj(J)
// row-major and 1/det J.
// With pairs (DW) the data of the next Gauss point are copied asynchronously (cp.async, no
// registers) into this thread's two shared-memory slot sets while the current point is computed.
struct PaView {
  const void *pa;
  int64_t n_cells;
  int64_t e;
  void *buf;   // per-thread slots in shared memory: buf[(b * K + k) * stride], b = q & 1 (DW only)
  int stride;
};

template <class N>
__device__ __forceinline__ typename N::T pa_load(const PaView &P, int q, int K, int k) {
  const typename N::S *p = static_cast<const typename N::S *>(P.pa);
  if constexpr (std::is_same<N, NumDW>::value) {
    const float2 *b = static_cast<const float2 *>(P.buf);
    return N::ld(b[((q & 1) * K + k) * P.stride]);
  } else {
    return N::ld(p[((int64_t)q * K + k) * P.n_cells + P.e]);
  }
}

// issue the asynchronous copies of Gauss point q's K pairs (DW) into slot set q & 1
template <class N>
__device__ __forceinline__ void pa_issue(const PaView &P, int q, int K) {
  if constexpr (std::is_same<N, NumDW>::value) {
    const float2 *p = static_cast<const float2 *>(P.pa);
    float2 *b = static_cast<float2 *>(P.buf);
    for (int k = 0; k < K; ++k) {
      const unsigned s = (unsigned)__cvta_generic_to_shared(b + ((q & 1) * K + k) * P.stride);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(p + ((int64_t)q * K + k) * P.n_cells + P.e));
    }
    asm volatile("cp.async.commit_group;\n" ::);
  }
}

// before reading point q: point q's copies are complete (point q + 1's may still be in flight)
template <class N>
__device__ __forceinline__ void pa_wait(int q) {
  if constexpr (std::is_same<N, NumDW>::value) {
    if (q < 7) asm volatile("cp.async.wait_group 1;\n" ::);
    else asm volatile("cp.async.wait_group 0;\n" ::);
  }
}

// Laplace element (Eq. 7), in place on u; with PA the flux matrix is loaded instead of computed.
template <class N, bool PA = false>
__device__ void laplace_general(typename N::T u[8], const typename N::T del[8][3], const typename N::T hh[3],
                                typename N::T kappa, const PaView &P = PaView{}) {
  using T = typename N::T;
  T cd[3][8];
  if constexpr (!PA) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int a = 0; a < 8; ++a) cd[i][a] = del[a][i];
      modes<N>(cd[i]);
    }
  }
  modes<N>(u);
  T A[3][4];
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int t = 0; t < 4; ++t) A[j][t] = N::zero();
  if constexpr (PA) pa_issue<N>(P, 0, 6);
#pragma unroll ((PA && std::is_same<N, NumF32>::value) ? 8 : 1)
  for (int q = 0; q < 8; ++q) {
    const int s[3] = {(q & 1) ? 1 : -1, (q & 2) ? 1 : -1, (q & 4) ? 1 : -1};
    T gu[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) gu[j] = dref<N>(u, j, s);
    if constexpr (PA) {
      if (q < 7) pa_issue<N>(P, q + 1, 6);
      pa_wait<N>(q);
      T D[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) D[k] = pa_load<N>(P, q, 6, k);
      const T f0 = N::add(N::add(N::mul(D[0], gu[0]), N::mul(D[1], gu[1])), N::mul(D[2], gu[2]));
      const T f1 = N::add(N::add(N::mul(D[1], gu[0]), N::mul(D[3], gu[1])), N::mul(D[4], gu[2]));
      const T f2 = N::add(N::add(N::mul(D[2], gu[0]), N::mul(D[4], gu[1])), N::mul(D[5], gu[2]));
      accum<N>(A[0], f0, 0, s);
      accum<N>(A[1], f1, 1, s);
      accum<N>(A[2], f2, 2, s);
    } else {
      T J[3][3], C[3][3];
      jac<N>(cd, hh, s, J);
      const T det = adj<N>(J, C);
      const T sc = ndiv<N>(kappa, det);
      T t[3];
#pragma unroll
      for (int k = 0; k < 3; ++k)
        t[k] = N::add(N::add(N::mul(C[0][k], gu[0]), N::mul(C[1][k], gu[1])), N::mul(C[2][k], gu[2]));
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const T f = N::mul(sc, N::add(N::add(N::mul(C[j][0], t[0]), N::mul(C[j][1], t[1])), N::mul(C[j][2], t[2])));
        accum<N>(A[j], f, j, s);
      }
    }
  }
  unmodes<N>(A, u);
}

// Vector Laplace element (Eq. 5: the flux of Eq. 7 for each component, geometry shared), in place
// on u[component][corner]; slot accumulators in shared memory as for elasticity.
template <class N, bool PA = false>
__device__ void vector_laplace_general(typename N::T u[3][8], const typename N::T del[8][3], const typename N::T hh[3],
                                       typename N::T kappa, typename N::S *Ash, int stride, const PaView &P = PaView{}) {
  using T = typename N::T;
  T cd[3][8];
  if constexpr (!PA) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int a = 0; a < 8; ++a) cd[i][a] = del[a][i];
      modes<N>(cd[i]);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) modes<N>(u[c]);
  for (int t = 0; t < 36; ++t) N::st(Ash[t * stride], N::zero());
  if constexpr (PA) pa_issue<N>(P, 0, 6);
#pragma unroll ((PA && std::is_same<N, NumF32>::value) ? 8 : 1)
  for (int q = 0; q < 8; ++q) {
    const int s[3] = {(q & 1) ? 1 : -1, (q & 2) ? 1 : -1, (q & 4) ? 1 : -1};
    // flux matrix D = kappa adj(J) adj(J)^T / det (stored, or formed from J)
    T D[6];
    if constexpr (PA) {
      if (q < 7) pa_issue<N>(P, q + 1, 6);
      pa_wait<N>(q);
#pragma unroll
      for (int k = 0; k < 6; ++k) D[k] = pa_load<N>(P, q, 6, k);
    } else {
      T J[3][3], C[3][3];
      jac<N>(cd, hh, s, J);
      const T det = adj<N>(J, C);
      const T sc = ndiv<N>(kappa, det);
      const int r[6] = {0, 0, 0, 1, 1, 2}, cc[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int k = 0; k < 6; ++k)
        D[k] = N::mul(sc, N::add(N::add(N::mul(C[r[k]][0], C[cc[k]][0]), N::mul(C[r[k]][1], C[cc[k]][1])),
                                 N::mul(C[r[k]][2], C[cc[k]][2])));
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T gu[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) gu[j] = dref<N>(u[c], j, s);
      const T fv[3] = {N::add(N::add(N::mul(D[0], gu[0]), N::mul(D[1], gu[1])), N::mul(D[2], gu[2])),
                       N::add(N::add(N::mul(D[1], gu[0]), N::mul(D[3], gu[1])), N::mul(D[4], gu[2])),
                       N::add(N::add(N::mul(D[2], gu[0]), N::mul(D[4], gu[1])), N::mul(D[5], gu[2]))};
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const T f = fv[j];
        T A4[4];
#pragma unroll
        for (int tt = 0; tt < 4; ++tt) A4[tt] = N::ld(Ash[((c * 3 + j) * 4 + tt) * stride]);
        accum<N>(A4, f, j, s);
#pragma unroll
        for (int tt = 0; tt < 4; ++tt) N::st(Ash[((c * 3 + j) * 4 + tt) * stride], A4[tt]);
      }
    }
  }
#pragma unroll 1
  for (int c = 0; c < 3; ++c) {
    T A[3][4];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int t = 0; t < 4; ++t) A[j][t] = N::ld(Ash[((c * 3 + j) * 4 + t) * stride]);
    unmodes<N>(A, u[c]);
  }
}

// Elasticity element (Algorithm 1), in place on u[component][corner].  The slot accumulators of
// the three output components live in shared memory (per-thread slice `Ash`) to bound registers.
template <class N, bool PA = false>
__device__ void elasticity_general(typename N::T u[3][8], const typename N::T del[8][3], const typename N::T hh[3],
                                   typename N::T lam, typename N::T mu, typename N::S *Ash, int stride,
                                   const PaView &P = PaView{}) {
  using T = typename N::T;
  T cd[3][8];
  if constexpr (!PA) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int a = 0; a < 8; ++a) cd[i][a] = del[a][i];
      modes<N>(cd[i]);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) modes<N>(u[c]);
  for (int t = 0; t < 36; ++t) N::st(Ash[t * stride], N::zero());
  if constexpr (PA) pa_issue<N>(P, 0, 10);
#pragma unroll ((PA && std::is_same<N, NumF32>::value) ? 8 : 1)
  for (int q = 0; q < 8; ++q) {
    const int s[3] = {(q & 1) ? 1 : -1, (q & 2) ? 1 : -1, (q & 4) ? 1 : -1};
    T C[3][3], idet;
    if constexpr (PA) {
      if (q < 7) pa_issue<N>(P, q + 1, 10);
      pa_wait<N>(q);
#pragma unroll
      for (int k = 0; k < 9; ++k) C[k / 3][k % 3] = pa_load<N>(P, q, 10, k);
      idet = pa_load<N>(P, q, 10, 9);
    } else {
      T J[3][3];
      jac<N>(cd, hh, s, J);
      const T det = adj<N>(J, C);
      idet = ndiv<N>(N::c(1.0f, 0.0f), det);
    }
    T G[3][3];  // grad u = H C / det, H_cj = d_j u_c
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T Hr[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) Hr[j] = dref<N>(u[c], j, s);
#pragma unroll
      for (int l = 0; l < 3; ++l)
        G[c][l] = N::mul(idet, N::add(N::add(N::mul(Hr[0], C[0][l]), N::mul(Hr[1], C[1][l])), N::mul(Hr[2], C[2][l])));
    }
    const T tr = N::add(N::add(G[0][0], G[1][1]), G[2][2]);
    const T ltr = N::mul(lam, tr);
    T S[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        S[c][l] = N::mul(mu, N::add(G[c][l], G[l][c]));
        if (c == l) S[c][l] = N::add(S[c][l], ltr);
      }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        // P_cj = (sigma C^T)_cj = sum_l S_cl C_jl
        const T P = N::add(N::add(N::mul(S[c][0], C[j][0]), N::mul(S[c][1], C[j][1])), N::mul(S[c][2], C[j][2]));
        T A4[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) A4[t] = N::ld(Ash[((c * 3 + j) * 4 + t) * stride]);
        accum<N>(A4, P, j, s);
#pragma unroll
        for (int t = 0; t < 4; ++t) N::st(Ash[((c * 3 + j) * 4 + t) * stride], A4[t]);
      }
  }
#pragma unroll 1
  for (int c = 0; c < 3; ++c) {
    T A[3][4];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int t = 0; t < 4; ++t) A[j][t] = N::ld(Ash[((c * 3 + j) * 4 + t) * stride]);
    unmodes<N>(A, u[c]);
  }
}

template <int PHYS, class N, int EX, int EY>
struct GenSmem {
  static constexpr int ND = phys_ndpn(PHYS);
  static constexpr int NP = (EX + 1) * (EY + 1), NACC = (EX - 1) * (EY - 1) * ND;
  typename N::S up[2][NP * ND];
  typename N::S dp[2][NP * 3];
  typename N::S acc[2][NACC];
  typename N::S ash[PHYS == MF_LAPLACE ? 1 : 36 * EX * EY];
  typename N::S pbuf[std::is_same<N, NumDW>::value ? 20 * EX * EY : 1];  // partial-assembly prefetch slots
  unsigned red[32];  // per-warp input magnitude records
};

// Owner-computes tile traversal marching up in z (output-plane accumulators in shared memory,
// summed in a fixed order), with the node offsets staged next to the input values.  One pass over
// this CTA's work item; SC: x * 2^-sc in and y * 2^so out (normalised meshes and the rescaled pass
// for inputs outside the double-word range).  Double-word passes record the magnitude of the inputs
// read in `mag` (Dirichlet entries excluded).
template <int PHYS, class N, int EX, int EY, bool PA, bool SC>
__device__ __forceinline__ void gen_pass(const GenArgs &g, const typename N::IO *__restrict__ x,
                                         typename N::IO *__restrict__ y, GenSmem<PHYS, N, EX, EY> &sm, int sc, int so,
                                         dwa::MagRec &mag) {
  using T = typename N::T;
  using S = typename N::S;
  using IO = typename N::IO;
  constexpr bool IS_DW = std::is_same<N, NumDW>::value;
  constexpr int ND = phys_ndpn(PHYS);
  constexpr int NT = EX * EY, TX = EX - 1, TY = EY - 1, PX = EX + 1, PY = EY + 1, NP = PX * PY;
  constexpr int LOADS = (NP + NT - 1) / NT;
  constexpr int NACC = TX * TY * ND;
  (void)PY;
  auto conv_in = [&](IO v) -> T {
    if constexpr (IS_DW && SC) return dwa::split_scaled(v, sc);
    else return N::in(v);
  };
  auto conv_out = [&](T v) -> IO {
    if constexpr (!SC) return N::out(v);
    else if constexpr (IS_DW) return dwa::ldexp_exact(N::out(v), so);
    else return dwa::ldexpf_exact(N::out(v), so);
  };
  (void)sc;
  (void)so;
  __syncthreads();  // a previous pass over the item may still be reading sm
  const int tid = threadIdx.x;
  const int bx = blockIdx.x % g.tiles_x;
  const int by = (blockIdx.x / g.tiles_x) % g.tiles_y;
  const int bz = blockIdx.x / (g.tiles_x * g.tiles_y);
  const int i0 = bx * TX, j0 = by * TY;
  const int NXP = g.nx + 1, NYP = g.ny + 1;
  const int k0 = bz * g.seg, k1 = min(k0 + g.seg, g.nz + 1);
  const int tx = tid % EX, ty = tid / EX;
  const int ex = i0 - 1 + tx, ey = j0 - 1 + ty;
  const bool ein = ex >= 0 && ex < g.nx && ey >= 0 && ey < g.ny;
  const int ownx = min(TX, NXP - i0), owny = min(TY, NYP - j0);
  T hxh = N::zero(), hyh = N::zero();
  if (ein) {
    hxh = N::from2(__ldg(g.hh + ex));
    hyh = N::from2(__ldg(g.hh + g.nx + ey));
  }
  for (int t = tid; t < 2 * NACC; t += NT) N::st(sm.acc[t / NACC][t % NACC], N::zero());

  IO xr[LOADS][ND];
  float2 dl[LOADS][3];
  bool dr[LOADS];
  auto fetch = [&](int k) {
#pragma unroll
    for (int l = 0; l < LOADS; ++l) {
      const int p = tid + l * NT;
      const int ix = i0 - 1 + p % PX, iy = j0 - 1 + p / PX;
      const bool ok = p < NP && ix >= 0 && ix < NXP && iy >= 0 && iy < NYP;
      const int64_t node =
          ok ? mf_dbg_index(ix + (int64_t)NXP * (iy + (int64_t)NYP * k), (int64_t)NXP * NYP * (g.nz + 1), MF_DBG_NODE) : 0;
      dr[l] = ok ? __ldg(g.dmask + node) != 0 : true;
#pragma unroll
      for (int c = 0; c < ND; ++c) xr[l][c] = ok ? __ldg(x + node * ND + c) : (IO)0;
      if constexpr (!PA) {
#pragma unroll
        for (int c = 0; c < 3; ++c) dl[l][c] = ok ? __ldg(g.delta + node * 3 + c) : make_float2(0.f, 0.f);
      }
    }
  };
  auto stage = [&](int k) {
#pragma unroll
    for (int l = 0; l < LOADS; ++l) {
      const int p = tid + l * NT;
      if (p < NP) {
#pragma unroll
        for (int c = 0; c < ND; ++c) {
          N::st(sm.up[k & 1][p * ND + c], dr[l] ? N::zero() : conv_in(xr[l][c]));
          if constexpr (IS_DW)
            if (!dr[l]) mag.add(xr[l][c]);
        }
        if constexpr (!PA) {
#pragma unroll
          for (int c = 0; c < 3; ++c) N::st(sm.dp[k & 1][p * 3 + c], N::from2(dl[l][c]));
        }
      }
    }
  };
  auto write_plane = [&](int k) {
    S *a = sm.acc[k & 1];
    for (int t = tid; t < NACC; t += NT) {
      const int idx = t / ND, c = t % ND;
      const int lx = idx % TX, ly = idx / TX;
      if (lx < ownx && ly < owny) {
        const int64_t node = mf_dbg_index((i0 + lx) + (int64_t)NXP * ((j0 + ly) + (int64_t)NYP * k),
                                          (int64_t)NXP * NYP * (g.nz + 1), MF_DBG_NODE);
        y[node * ND + c] = __ldg(g.dmask + node) ? x[node * ND + c] : conv_out(N::ld(a[t]));
      }
      N::st(a[t], N::zero());
    }
  };

  const int s_lo = max(k0 - 1, 0), s_hi = min(k1 - 1, g.nz - 1);
  fetch(s_lo);
  stage(s_lo);
  fetch(s_lo + 1);
  for (int ez = s_lo; ez <= s_hi; ++ez) {
    stage(ez + 1);
    __syncthreads();
    if (ez + 2 <= g.nz) fetch(ez + 2);
    T v[ND][8];
    if (ein) {
      T del[8][3];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int p = (tx + (a & 1)) + PX * (ty + ((a >> 1) & 1));
        const int pl = (a & 4) ? ((ez + 1) & 1) : (ez & 1);
#pragma unroll
        for (int c = 0; c < ND; ++c) v[c][a] = N::ld(sm.up[pl][p * ND + c]);
#pragma unroll
        for (int c = 0; c < 3; ++c) del[a][c] = PA ? N::zero() : N::ld(sm.dp[pl][p * 3 + c]);
      }
      const int64_t e = ex + (int64_t)g.nx * (ey + (int64_t)g.ny * ez);
      const T hh[3] = {hxh, hyh, N::from2(__ldg(g.hh + g.nx + g.ny + ez))};
      const PaView P{g.pa, g.n_cells, e, sm.pbuf + tid, NT};
      if constexpr (PHYS == MF_LAPLACE) {
        laplace_general<N, PA>(v[0], del, hh, N::from2(__ldg(g.mat + e)), P);
      } else if constexpr (PHYS == MF_VECTOR_LAPLACE) {
        vector_laplace_general<N, PA>(v, del, hh, N::from2(__ldg(g.mat + e)), sm.ash + tid, NT, P);
      } else {
        elasticity_general<N, PA>(v, del, hh, N::from2(__ldg(g.mat + 2 * e)), N::from2(__ldg(g.mat + 2 * e + 1)),
                                  sm.ash + tid, NT, P);
      }
    }
    const bool bot = ez >= k0, top = ez + 1 < k1;
#pragma unroll
    for (int ay = 0; ay < 2; ++ay) {
#pragma unroll
      for (int ax = 0; ax < 2; ++ax) {
        const int lx = tx - 1 + ax, ly = ty - 1 + ay;
        if (ein && lx >= 0 && lx < ownx && ly >= 0 && ly < owny) {
          const int idx = (lx + TX * ly) * ND;
          const int a = ax + 2 * ay;
#pragma unroll
          for (int c = 0; c < ND; ++c) {
            if (bot) N::st(sm.acc[ez & 1][idx + c], N::add(N::ld(sm.acc[ez & 1][idx + c]), v[c][a]));
            if (top) N::st(sm.acc[(ez + 1) & 1][idx + c], N::add(N::ld(sm.acc[(ez + 1) & 1][idx + c]), v[c][a + 4]));
          }
        }
        __syncwarp();
      }
      __syncthreads();
    }
    if (ez >= k0) write_plane(ez);
  }
  if (s_hi + 1 == g.nz && g.nz >= k0 && g.nz < k1) write_plane(g.nz);
}

// One CTA per work item.  Double-word arithmetic: if the largest input the CTA read lies outside
// [2^kMagLo, 2^kMagHi], the item is computed again with x scaled by the power of two that brings
// that input to [1, 2) and y scaled back (FP64 accuracy over FP64's whole range; the decision
// depends on the item's own inputs only, and the second pass rewrites every value of the first).
template <int PHYS, class N, int EX, int EY, bool PA>
__global__ void __launch_bounds__(EX *EY, (PA && std::is_same<N, NumF32>::value) ? 2 : 1)
    gen_apply(GenArgs g, const typename N::IO *__restrict__ x, typename N::IO *__restrict__ y,
              const int *__restrict__ skip) {
  extern __shared__ __align__(16) unsigned char gen_smem_raw[];
  auto &sm = *reinterpret_cast<GenSmem<PHYS, N, EX, EY> *>(gen_smem_raw);
  if (skip && *skip) return;
  dwa::MagRec mag;
  if (g.oscale == 0) gen_pass<PHYS, N, EX, EY, PA, false>(g, x, y, sm, 0, 0, mag);
  else gen_pass<PHYS, N, EX, EY, PA, true>(g, x, y, sm, 0, g.oscale, mag);
  if constexpr (std::is_same<N, NumDW>::value) {
    const unsigned t = __reduce_max_sync(0xffffffffu, mag.key);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sm.red[threadIdx.x >> 5] = t;
    __syncthreads();
    unsigned T = 0u;
#pragma unroll
    for (int i = 0; i < EX * EY / 32; ++i) T = max(T, sm.red[i]);
    int s = 0;
    if (dwa::mag_exponent(T, s) && (s < dwa::kMagLo || s > dwa::kMagHi))
      gen_pass<PHYS, N, EX, EY, PA, true>(g, x, y, sm, s, g.oscale + s, mag);
  }
}

// ------------------------------------------------------------------------------------ setup ----
// Half spacings of the base grid from the axis node lines, and node offsets from the base grid.
__global__ void gen_axes(const double *X, int nx, int ny, int nz, double geo, float2 *hh) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nx + ny + nz) return;
  double a, b;
  if (t < nx) {
    a = X[3 * (int64_t)t];
    b = X[3 * (int64_t)(t + 1)];
  } else if (t < nx + ny) {
    const int j = t - nx;
    a = X[3 * (int64_t)(nx + 1) * j + 1];
    b = X[3 * (int64_t)(nx + 1) * (j + 1) + 1];
  } else {
    const int k = t - nx - ny;
    a = X[3 * (int64_t)(nx + 1) * (ny + 1) * k + 2];
    b = X[3 * (int64_t)(nx + 1) * (ny + 1) * (k + 1) + 2];
  }
  const dw v = dwa::from_double_slow(0.5 * (b - a) * geo);  // normalised (geo: power of two)
  hh[t] = make_float2(v.h, v.l);
}

__global__ void gen_delta(const double *X, int nx, int ny, int nz, double geo, float2 *delta) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t Nn = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  if (n >= Nn) return;
  const int i = (int)(n % (nx + 1)), j = (int)((n / (nx + 1)) % (ny + 1)), k = (int)(n / ((int64_t)(nx + 1) * (ny + 1)));
  const double base[3] = {X[3 * (int64_t)i], X[3 * (int64_t)(nx + 1) * j + 1],
                          X[3 * (int64_t)(nx + 1) * (ny + 1) * k + 2]};
  for (int c = 0; c < 3; ++c) {
    const dw v = dwa::from_double_slow((X[3 * n + c] - base[c]) * geo);
    delta[3 * n + c] = make_float2(v.h, v.l);
  }
}

__global__ void gen_mat_pairs(const double *m, int64_t n, double scale, float2 *out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const dw v = dwa::from_double_slow(m[i] * scale);
  out[i] = make_float2(v.h, v.l);
}

template <int PHYS, class N> struct GenShape;
template <class N> struct GenShape<MF_LAPLACE, N> { static constexpr int EX = 32, EY = 8; };
template <class N> struct GenShape<MF_ELASTICITY, N> { static constexpr int EX = 32, EY = 8; };
template <class N> struct GenShape<MF_VECTOR_LAPLACE, N> { static constexpr int EX = 32, EY = 8; };

template <int PHYS, class N, bool PA>
mf_status gen_launch(const mf_mesh *m, const typename N::IO *x, typename N::IO *y, cudaStream_t s, const int *skip) {
  constexpr int EX = GenShape<PHYS, N>::EX, EY = GenShape<PHYS, N>::EY;
  GenArgs g;
  g.nx = m->nx;
  g.ny = m->ny;
  g.nz = m->nz;
  g.tiles_x = (m->nx + 1 + EX - 2) / (EX - 1);
  g.tiles_y = (m->ny + 1 + EY - 2) / (EY - 1);
  const int cols = g.tiles_x * g.tiles_y;
  const int nseg = std::max(1, std::min(m->nz + 1, (device_sm_count() * 4 + cols - 1) / cols));
  g.seg = (m->nz + 1 + nseg - 1) / nseg;
  g.hh = m->gen_axis;
  g.delta = m->gen_delta;
  g.mat = m->mat_pairs;
  g.dmask = m->dmask;
  g.pa = std::is_same<N, NumDW>::value ? (const void *)m->pa : (const void *)m->pa32;
  g.n_cells = m->n_cells;
  g.oscale = m->dw_oscale;
  const int smem = (int)sizeof(GenSmem<PHYS, N, EX, EY>);
  auto kern = gen_apply<PHYS, N, EX, EY, PA>;
  static bool set = false;
  if (!set) {
    MF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    set = true;
  }
  const int items = cols * ((m->nz + 1 + g.seg - 1) / g.seg);
  mf_count_launches(1);
  kern<<<items, EX * EY, smem, s>>>(g, x, y, skip);
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

}  // namespace

// values stored by partial assembly: 8 Gauss points x (10 elasticity, 6 Laplace) per cell
static int64_t pa_values(const mf_mesh *m) { return 8LL * (m->physics == MF_ELASTICITY ? 10 : 6) * m->n_cells; }

mf_status gen_setup(mf_mesh *m, cudaStream_t s) {
  if (!m->structured || m->tp) return MF_OK;
  const int n = m->nx + m->ny + m->nz;
  MF_CUDA(cudaMalloc(&m->gen_axis, n * sizeof(float2)));
  MF_CUDA(cudaMalloc(&m->gen_delta, 3 * m->n_nodes * sizeof(float2)));
  gen_axes<<<blocks_for(n), kThreads, 0, s>>>(m->X, m->nx, m->ny, m->nz, m->dw_geo, m->gen_axis);
  gen_delta<<<blocks_for(m->n_nodes), kThreads, 0, s>>>(m->X, m->nx, m->ny, m->nz, m->dw_geo, m->gen_delta);
  if (!m->mat_pairs) {
    const int64_t nm = m->n_cells * phys_nmat(m->physics);
    MF_CUDA(cudaMalloc(&m->mat_pairs, nm * sizeof(float2)));
    gen_mat_pairs<<<blocks_for(nm), kThreads, 0, s>>>(m->mat, nm, m->dw_mat, m->mat_pairs);
  }
  MF_CUDA(cudaGetLastError());
  MF_CUDA(cudaStreamSynchronize(s));
  m->gen = true;
  // The auto variant uses partial assembly when its data take at most a quarter of the device's
  // total memory: a function of the mesh and the device model, not of what else is allocated.  If
  // the allocation fails all the same, the mesh keeps the general kernel (flag bit 3 of
  // mf_mesh_query reports which one the auto variant runs).
  size_t free_b = 0, total_b = 0;
  MF_CUDA(cudaMemGetInfo(&free_b, &total_b));
  if ((double)pa_values(m) * (sizeof(float2) + sizeof(float)) <= 0.25 * (double)total_b) {
    const mf_status st = pa_setup(m, s);
    if (st != MF_OK && st != MF_ERR_OOM) return st;
    mf_clear_error();
  }
  return MF_OK;
}

namespace {

// Quadrature-point data of partial assembly, computed in FP64 from the node coordinates (J, adj J,
// det J at the 2x2x2 Gauss points, Algorithm 1) and stored as pairs and floats: one thread per cell.
template <int PHYS>
__global__ void pa_build(const double *__restrict__ X, int nx, int ny, int nz, const double *__restrict__ mat,
                         double geo, double matscale, float2 *__restrict__ pa, float *__restrict__ pa32) {
  constexpr int K = PHYS == MF_ELASTICITY ? 10 : 6;
  const int64_t E = (int64_t)nx * ny * nz;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((int64_t)nx * ny));
  double Xe[8][3];
  for (int a = 0; a < 8; ++a) {
    const int64_t node = (i + (a & 1)) + (int64_t)(nx + 1) * ((j + ((a >> 1) & 1)) + (int64_t)(ny + 1) * (k + (a >> 2)));
    for (int c = 0; c < 3; ++c) Xe[a][c] = X[3 * node + c] * geo;  // normalised coordinates
  }
  for (int q = 0; q < 8; ++q) {
    double xi[3];
    for (int d = 0; d < 3; ++d) xi[d] = q1::sgn(q, d) * q1::kG;
    double J[3][3], C[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        double sum = 0.0;
        for (int a = 0; a < 8; ++a) sum += Xe[a][r] * q1::dN_at(xi, a, c);
        J[r][c] = sum;
      }
    const double det = q1::adjugate(J, C);
    double v[K];
    if (PHYS == MF_ELASTICITY) {
      for (int t = 0; t < 9; ++t) v[t] = C[t / 3][t % 3];
      v[9] = 1.0 / det;
    } else {
      const int r[6] = {0, 0, 0, 1, 1, 2}, c[6] = {0, 1, 2, 1, 2, 2};
      for (int t = 0; t < 6; ++t)
        v[t] = mat[e] * matscale * (C[r[t]][0] * C[c[t]][0] + C[r[t]][1] * C[c[t]][1] + C[r[t]][2] * C[c[t]][2]) / det;
    }
    for (int t = 0; t < K; ++t) {
      const dw d = dwa::from_double_slow(v[t]);
      const int64_t idx = ((int64_t)q * K + t) * E + e;
      pa[idx] = make_float2(d.h, d.l);
      pa32[idx] = (float)v[t];
    }
  }
}

template <class N>
mf_status gen_dispatch(const mf_mesh *m, const typename N::IO *x, typename N::IO *y, cudaStream_t s,
                       const int *skip) {
  const bool pa = m->pa && m->variant != MF_VARIANT_GENERAL;
  if (m->physics == MF_LAPLACE)
    return pa ? gen_launch<MF_LAPLACE, N, true>(m, x, y, s, skip) : gen_launch<MF_LAPLACE, N, false>(m, x, y, s, skip);
  if (m->physics == MF_VECTOR_LAPLACE)
    return pa ? gen_launch<MF_VECTOR_LAPLACE, N, true>(m, x, y, s, skip)
              : gen_launch<MF_VECTOR_LAPLACE, N, false>(m, x, y, s, skip);
  return pa ? gen_launch<MF_ELASTICITY, N, true>(m, x, y, s, skip)
            : gen_launch<MF_ELASTICITY, N, false>(m, x, y, s, skip);
}

}  // namespace

mf_status pa_setup(mf_mesh *m, cudaStream_t s) {
  if (m->pa) return MF_OK;
  if (!m->gen) {
    mf_set_error("partial assembly needs a structured mesh that is not a tensor-product grid");
    return MF_ERR_UNSUPPORTED;
  }
  const int64_t n = pa_values(m);
  cudaError_t e = cudaMalloc(&m->pa, n * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&m->pa32, n * sizeof(float));
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(m->pa);
    cudaFree(m->pa32);
    m->pa = nullptr;
    m->pa32 = nullptr;
    mf_set_error("partial assembly: no room for %lld quadrature-point values", (long long)n);
    return MF_ERR_OOM;
  }
  if (m->physics == MF_ELASTICITY)
    pa_build<MF_ELASTICITY><<<blocks_for(m->n_cells), kThreads, 0, s>>>(m->X, m->nx, m->ny, m->nz, m->mat, m->dw_geo,
                                                                          m->dw_mat, m->pa, m->pa32);
  else
    pa_build<MF_LAPLACE><<<blocks_for(m->n_cells), kThreads, 0, s>>>(m->X, m->nx, m->ny, m->nz, m->mat, m->dw_geo,
                                                                       m->dw_mat, m->pa, m->pa32);
  MF_CUDA(cudaGetLastError());
  MF_CUDA(cudaStreamSynchronize(s));
  return MF_OK;
}

mf_status gen_apply_fp64(const mf_mesh *m, const double *x, double *y, cudaStream_t s, const int *skip) {
  return gen_dispatch<NumDW>(m, x, y, s, skip);
}

mf_status gen_apply_fp32(const mf_mesh *m, const float *x, float *y, cudaStream_t s, const int *skip) {
  return gen_dispatch<NumF32>(m, x, y, s, skip);
}

MF_DBG_TU(general)
