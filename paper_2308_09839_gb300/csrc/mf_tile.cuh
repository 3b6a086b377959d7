// Tensor-product element arithmetic shared by the face-marching kernels (mf_march.cuh, which also
// serve the batched persistent solver): number types, Walsh-Hadamard transforms, the Laplace and
// elasticity coefficients, the work decomposition.
#pragma once
//
// What it computes is Eq. 7 (Laplace) / Eq. 9 and Algorithm 1 (elasticity) with 2x2x2 Gauss on
// structured boxes whose cells are axis-aligned (tensor-product geometry):
//
// 1. Geometry from per-axis spacings.  A cell of a tensor-product grid is the box
//    [x_i, x_i+1] x [y_j, y_j+1] x [z_k, z_k+1], so J = diag(hx, hy, hz)/2 is constant on the cell
//    and is computed per element from three spacings (kept, with their inverses, in tiny per-axis
//    arrays built at setup from the coordinates).  Coordinates are not re-read per apply.
//
// 2. Exact rewriting of the quadrature in the monomial (Walsh-Hadamard) basis.  Writing the
//    element field as u = sum_m c_m M_m(xi) with M in {1, xi, eta, zeta, xi eta, xi zeta,
//    eta zeta, xi eta zeta}, the coefficients are c = H u / 8 with H the 8x8 Hadamard matrix, and
//    with J constant the 2-point Gauss sums of Eqs. 4/6 are the exact integrals of products of
//    those monomials (degree <= 2 per variable).  They are diagonal or nearly so in this basis:
//    scalar Laplace:   v = H^T D H u,  D = diag(0, g1, g2, (g1+g2)/3, g3, (g1+g3)/3, (g2+g3)/3,
//                      (g1+g2+g3)/9) / 16 with g1 = kappa hy hz / hx (cyclic);
//    elasticity: the same per component plus 24 couplings between components through lam and mu
//                (see elasticity_modes below).
//
// 3. Double-word arithmetic (mf_dw.cuh) for FP64 accuracy; the GB300 FP64 pipe is ~60x slower
//    than FP32.  x is split into float pairs with integer operations; y leaves through one FP64 add.
#include <algorithm>
#include <type_traits>

#include "mf_dw.cuh"
#include "mf_internal.cuh"

namespace tile {

using dwa::dw;

// ------------------------------------------------------------------ number types (traits) ----
struct NumDW {  // FP64-accurate double-word
  using T = dw;
  using S = float2;
  using IO = double;
  static __device__ __forceinline__ T zero() { return dw{0.f, 0.f}; }
  static __device__ __forceinline__ T add(T a, T b) { return dwa::add(a, b); }
  static __device__ __forceinline__ T sub(T a, T b) { return dwa::sub(a, b); }
  static __device__ __forceinline__ T neg(T a) { return dwa::neg(a); }  // exact
  static __device__ __forceinline__ T mul(T a, T b) { return dwa::mul(a, b); }
  static __device__ __forceinline__ T scale(T a, float p) { return dwa::scale(a, p); }
  static __device__ __forceinline__ T from2(float2 v) { return dw{v.x, v.y}; }
  static __device__ __forceinline__ T ld(const S &s) { return dw{s.x, s.y}; }
  static __device__ __forceinline__ void st(S &s, T v) { s = make_float2(v.h, v.l); }
  static __device__ __forceinline__ T in(IO v) { return dwa::split(v); }
  static __device__ __forceinline__ IO out(T v) { return dwa::to_double(v); }
  static __device__ __forceinline__ T c(float h, float l) { return dw{h, l}; }
};

struct NumF32 {  // plain FP32 (mixed-precision inner solves)
  using T = float;
  using S = float;
  using IO = float;
  static __device__ __forceinline__ T zero() { return 0.f; }
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
  static __device__ __forceinline__ T neg(T a) { return -a; }
  static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
  static __device__ __forceinline__ T scale(T a, float p) { return a * p; }
  static __device__ __forceinline__ T from2(float2 v) { return v.x; }
  static __device__ __forceinline__ T ld(const S &s) { return s; }
  static __device__ __forceinline__ void st(S &s, T v) { s = v; }
  static __device__ __forceinline__ T in(IO v) { return v; }
  static __device__ __forceinline__ IO out(T v) { return v; }
  static __device__ __forceinline__ T c(float h, float) { return h; }
};

// 1/3, 1/9, 1/48, 1/144 as (hi, lo) pairs: hi = nearest float, lo = nearest float to the rest.
#define C_THIRD 0x1.555556p-2f, -0x1.555556p-27f
#define C_NINTH 0x1.c71c72p-4f, -0x1.c71c72p-31f
#define C_48TH 0x1.555556p-6f, -0x1.555556p-31f
#define C_144TH 0x1.c71c72p-8f, -0x1.c71c72p-35f

// Forward transform c = H u in place: butterflies (lo, hi) -> (lo + hi, hi - lo) along each bit.
template <class N>
__device__ __forceinline__ void fwht_fwd(typename N::T u[8]) {
#pragma unroll
  for (int d = 1; d < 8; d <<= 1)
#pragma unroll
    for (int a = 0; a < 8; ++a)
      if (!(a & d)) {
        const typename N::T lo = u[a], hi = u[a | d];
        u[a] = N::add(lo, hi);
        u[a | d] = N::sub(hi, lo);
      }
}

// Transposed transform y = H^T v in place: (lo, hi) -> (lo - hi, lo + hi).
template <class N>
__device__ __forceinline__ void fwht_inv(typename N::T v[8]) {
#pragma unroll
  for (int d = 1; d < 8; d <<= 1)
#pragma unroll
    for (int a = 0; a < 8; ++a)
      if (!(a & d)) {
        const typename N::T lo = v[a], hi = v[a | d];
        v[a] = N::sub(lo, hi);
        v[a | d] = N::add(lo, hi);
      }
}

// Scalar Laplace on an axis-aligned box.  The per-element coefficients (depending on geometry and
// kappa only) are computed once and applied to every right-hand side.
// Modes are indexed by the bit set of the monomial: 1 xi, 2 eta, 4 zeta, 3 xi eta, 5 xi zeta,
// 6 eta zeta, 7 xi eta zeta.  hy_ihx = hy/hx, hx_ihy = hx/hy and hxhy = hx hy are per-thread
// invariants of the z-march.
template <class N>
struct LapCoef {
  typename N::T s1, s2, s3, s12, s13, s23, s123;
};

template <class N>
__device__ __forceinline__ LapCoef<N> laplace_coef(typename N::T k, typename N::T hy_ihx, typename N::T hx_ihy,
                                                   typename N::T hxhy, typename N::T hz, typename N::T ihz) {
  using T = typename N::T;
  const T kz = N::mul(k, hz);
  const T g1 = N::mul(kz, hy_ihx);              // kappa hy hz / hx
  const T g2 = N::mul(kz, hx_ihy);              // kappa hx hz / hy
  const T g3 = N::mul(N::mul(k, ihz), hxhy);    // kappa hx hy / hz
  const T g12 = N::add(g1, g2);
  LapCoef<N> c;
  c.s1 = N::scale(g1, 0.0625f);
  c.s2 = N::scale(g2, 0.0625f);
  c.s3 = N::scale(g3, 0.0625f);
  c.s12 = N::mul(g12, N::c(C_48TH));
  c.s13 = N::mul(N::add(g1, g3), N::c(C_48TH));
  c.s23 = N::mul(N::add(g2, g3), N::c(C_48TH));
  c.s123 = N::mul(N::add(g12, g3), N::c(C_144TH));
  return c;
}

// Isotropic elasticity on an axis-aligned box.  With r_k = h_{k+1} h_{k+2} / h_k and the mode
// coefficients c^k = H u^k:
//   same-component terms:  W^l_k = (k == l ? lam + 2 mu : mu) r_k / 16 weighted like the Laplace D;
//   cross-component terms: lam h_m / 16 and mu h_m / 16 (m the third axis) between the linear and
//   bilinear modes of components k != l, as derived from Eq. 6 with J diagonal.
template <class N>
struct ElCoef {
  typename N::T lr[3], mr[3], L[3], M[3], L3[3], M3[3];
};

template <class N>
__device__ __forceinline__ ElCoef<N> elasticity_coef(typename N::T lam, typename N::T mu, const typename N::T h[3],
                                                     const typename N::T ih[3]) {
  using T = typename N::T;
  const T h01 = N::mul(h[0], h[1]), h02 = N::mul(h[0], h[2]), h12 = N::mul(h[1], h[2]);
  const T r[3] = {N::mul(h12, ih[0]), N::mul(h02, ih[1]), N::mul(h01, ih[2])};
  const T l2m = N::add(lam, N::scale(mu, 2.0f));
  ElCoef<N> e;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    e.mr[k] = N::scale(N::mul(mu, r[k]), 0.0625f);
    e.lr[k] = N::scale(N::mul(l2m, r[k]), 0.0625f);
    e.L[k] = N::scale(N::mul(lam, h[k]), 0.0625f);
    e.M[k] = N::scale(N::mul(mu, h[k]), 0.0625f);
    e.L3[k] = N::mul(e.L[k], N::c(C_THIRD));
    e.M3[k] = N::mul(e.M[k], N::c(C_THIRD));
  }
  return e;
}

// Mode coefficients c[k][m] = (H u^k)_m -> o[l][m] = (D c)_l,m (modes 1..6 are coupled between
// components; modes 0 and 7 of c are not read, o[l][0] = 0).
template <class N>
__device__ __forceinline__ void elasticity_modes(const ElCoef<N> &e, const typename N::T c[3][8], typename N::T o[3][8]) {
  using T = typename N::T;
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const T W1 = l == 0 ? e.lr[0] : e.mr[0];
    const T W2 = l == 1 ? e.lr[1] : e.mr[1];
    const T W3 = l == 2 ? e.lr[2] : e.mr[2];
    const T W12 = N::add(W1, W2), W13 = N::add(W1, W3), W23 = N::add(W2, W3);
    o[l][0] = N::zero();
    o[l][1] = N::mul(W1, c[l][1]);
    o[l][2] = N::mul(W2, c[l][2]);
    o[l][4] = N::mul(W3, c[l][4]);
    o[l][3] = N::mul(N::mul(W12, N::c(C_THIRD)), c[l][3]);
    o[l][5] = N::mul(N::mul(W13, N::c(C_THIRD)), c[l][5]);
    o[l][6] = N::mul(N::mul(W23, N::c(C_THIRD)), c[l][6]);
    o[l][7] = N::mul(N::mul(N::add(W12, W3), N::c(C_NINTH)), c[l][7]);
  }
#define ACC(l, m, coef, k, mm) o[l][m] = N::add(o[l][m], N::mul(e.coef, c[k][mm]))
  // components 0 <-> 1 (third axis 2)
  ACC(1, 2, L[2], 0, 1); ACC(1, 6, L3[2], 0, 5); ACC(1, 1, M[2], 0, 2); ACC(1, 5, M3[2], 0, 6);
  ACC(0, 1, L[2], 1, 2); ACC(0, 5, L3[2], 1, 6); ACC(0, 2, M[2], 1, 1); ACC(0, 6, M3[2], 1, 5);
  // components 0 <-> 2 (third axis 1)
  ACC(2, 4, L[1], 0, 1); ACC(2, 6, L3[1], 0, 3); ACC(2, 1, M[1], 0, 4); ACC(2, 3, M3[1], 0, 6);
  ACC(0, 1, L[1], 2, 4); ACC(0, 3, L3[1], 2, 6); ACC(0, 4, M[1], 2, 1); ACC(0, 6, M3[1], 2, 3);
  // components 1 <-> 2 (third axis 0)
  ACC(2, 4, L[0], 1, 2); ACC(2, 5, L3[0], 1, 3); ACC(2, 2, M[0], 1, 4); ACC(2, 3, M3[0], 1, 5);
  ACC(1, 2, L[0], 2, 4); ACC(1, 3, L3[0], 2, 5); ACC(1, 4, M[0], 2, 2); ACC(1, 5, M3[0], 2, 3);
#undef ACC
}

struct TileArgs {
  int nx, ny, nz;
  int tiles_x, tiles_y, seg;
  int nrhs, r0;  // vectors hold nrhs right-hand sides per node ([node][rhs][comp]); first one of the launch
  const float2 *hx, *hy, *hz, *ihx, *ihy, *ihz;  // per-axis spacings and inverses (pairs)
  const float2 *mat;                             // kappa[E] or (lam, mu)[E] as pairs
  const uint8_t *dmask;
  int oscale;  // y = 2^oscale x (operator of the normalised cell constants and spacings) x
  // range check of the stand-alone launches (march_apply / march_apply_dot and their fix-up kernel):
  // per-CTA flag words, and this launch's bit in them
  unsigned *flags;
  unsigned bit;
};

// Segment length from a wave model: with R CTAs resident at a time, nseg segments of seg = ceil((nz
// + 1) / nseg) planes take about ceil(cols * nseg / R) waves of (seg + 1) element layers each (the
// +1 is the recomputed layer below a segment); the smallest estimate wins, ties to fewer segments.
inline int wave_segment(int cols, int nzp1, int resident_total) {
  int best_seg = nzp1;
  long long best = -1;
  for (int nseg = 1; nseg <= nzp1; ++nseg) {
    const int seg = (nzp1 + nseg - 1) / nseg;
    if (nseg > 1 && seg == (nzp1 + nseg - 2) / (nseg - 1)) continue;  // same segment length as before
    const long long waves = ((long long)cols * nseg + resident_total - 1) / resident_total;
    const long long cost = waves * (seg + 1);
    if (best < 0 || cost < best) {
      best = cost;
      best_seg = seg;
    }
  }
  return best_seg;
}

// Grid decomposition of a structured mesh into tile columns and z-segments of `seg` node planes
// (seg <= 0: by the wave model for `resident` CTAs per SM on the device's SMs and `batch` launches' worth
// of columns (right-hand sides), or, without an occupancy figure, enough segments for about four
// CTAs per SM).
inline TileArgs make_tile_args(const mf_mesh *m, int EX, int EY, int seg, int resident = 0, int batch = 1) {
  TileArgs g;
  g.nx = m->nx;
  g.ny = m->ny;
  g.nz = m->nz;
  const int TX = EX - 1, TY = EY - 1;
  g.tiles_x = (m->nx + 1 + TX - 1) / TX;
  g.tiles_y = (m->ny + 1 + TY - 1) / TY;
  if (seg <= 0) {
    const int cols = g.tiles_x * g.tiles_y;
    if (resident > 0) {
      seg = wave_segment(cols * batch, m->nz + 1, device_sm_count() * resident);
    } else {
      const int target = device_sm_count() * 4;
      const int nseg = std::max(1, std::min(m->nz + 1, (target + cols - 1) / cols));
      seg = (m->nz + 1 + nseg - 1) / nseg;
    }
  }
  g.seg = std::max(1, std::min(seg, m->nz + 1));
  const int n = m->nx + m->ny + m->nz;
  g.hx = m->tp_axis;
  g.hy = m->tp_axis + m->nx;
  g.hz = m->tp_axis + m->nx + m->ny;
  g.ihx = m->tp_axis + n;
  g.ihy = m->tp_axis + n + m->nx;
  g.ihz = m->tp_axis + n + m->nx + m->ny;
  g.mat = m->mat_pairs;
  g.dmask = m->dmask;
  g.oscale = m->dw_oscale;
  g.flags = m->tp_flags;
  g.bit = 0u;
  g.nrhs = 1;
  g.r0 = 0;
  return g;
}

inline int tile_items(const TileArgs &g) {
  const int nseg = (g.nz + 1 + g.seg - 1) / g.seg;
  return g.tiles_x * g.tiles_y * nseg;
}


}  // namespace tile
