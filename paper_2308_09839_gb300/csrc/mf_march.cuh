// Face-marching apply on tensor-product boxes (auto variant): scalar Laplace,
// vector Laplace (the scalar element operator on each component, Eq. 5) and isotropic elasticity.
//
// The arithmetic is that of the Walsh-Hadamard form in mf_tile.cuh (Eqs. 7 and 9 with 2x2x2
// Gauss, rewritten exactly in the Walsh-Hadamard monomial basis: A^e = H^T D_e H with D_e diagonal
// for Laplace and diagonal plus 24 couplings between components for elasticity), in double-word
// FP32 for FP64 accuracy or in plain FP32.  What changes is the organisation, which shares work
// between neighbouring elements:
//
//  * H = Hz (Hy Hx): the 8-point transform of an element is the 2D transform of its bottom and of
//    its top face of 4 nodes, followed by one butterfly along z.  The face transform of node plane
//    k is shared by the elements below and above it: a thread owns a column of elements, marches
//    up in z and carries the top-face transform of one element over as the bottom-face transform
//    of the next.  Forward cost per element: 8 + 8 adds instead of 24.
//  * H^T = (Hy Hx)^T Hz^T likewise: after the z butterfly the bottom-face part of an element and
//    the top-face part of the element below belong to the same face, so they are added first and
//    transposed once (4 + 8 adds), then the element's top-face part is carried up.
//  * The four faces around a node are summed in the plane: along x by a warp shuffle (a warp is a
//    row of 32 element columns), along y by one shared-memory exchange per plane.  Every owned
//    node is then complete and written once (coalesced along x), without atomics, memset or
//    read-modify-write; the summation order is fixed, so the result is bitwise reproducible.
//
// A CTA covers EX x EY element columns = an (EX-1) x (EY-1) block of owned nodes plus one halo
// ring of elements on the low sides (recomputed by the neighbouring CTA), over a z-segment of
// node planes [k0, k1) (plus the element layer below k0), for one right-hand side (blockIdx.y; the
// vectors of a multi-RHS apply are [node][rhs][comp]).  One __syncthreads per plane.
#pragma once

#include "mf_tile.cuh"

namespace march {

using tile::TileArgs;

template <class N>
__device__ __forceinline__ typename N::T shfl_up1(typename N::T v);
template <>
__device__ __forceinline__ tile::NumDW::T shfl_up1<tile::NumDW>(tile::NumDW::T v) {
  return dwa::dw{__shfl_up_sync(0xffffffffu, v.h, 1), __shfl_up_sync(0xffffffffu, v.l, 1)};
}
template <>
__device__ __forceinline__ tile::NumF32::T shfl_up1<tile::NumF32>(tile::NumF32::T v) {
  return __shfl_up_sync(0xffffffffu, v, 1);
}

template <int NC, class N, int EX, int EY>
struct MarchSmem {
  typename N::S up[2][(EX + 1) * (EY + 1) * NC];  // staged node planes (double buffered)
  typename N::S xrow[2][NC * EX * EY];            // partial sums of the top node row of each face
  unsigned mag;                                   // largest input magnitude record of the item
};

// PHYS = MF_LAPLACE (Eq. 7), MF_VECTOR_LAPLACE (Eq. 5) or MF_ELASTICITY (Eq. 9, Algorithm 1);
// vectors hold NC values per node (x, y, z components interleaved for the vector operators).
// One work item (tile column x z-segment `item`, right-hand side `rr`); must be called by all
// EX*EY/RY threads of the CTA.  A thread owns RY consecutive element rows of its x column: the
// x-butterflies of the node rows its faces share are formed once, and the y-sums of the node rows
// between them stay in registers (only the top row's go through shared memory).
// COHERENT: read x through L2 only (x was written by other CTAs earlier in the same persistent
// kernel, so the read-only and L1 paths may hold stale lines).
// DOT: also return this thread's part of x . y over the nodes it writes (the dot product a CG
// iteration needs next, p . Ap, formed while the result is written; FP64 products and sums).
// SC: power-of-two scaling, x * 2^-sc in and y * 2^so out (the cell constants and spacings of a
// normalised mesh, and the rescaled pass for inputs outside the double-word range); without SC
// neither is applied (so must be 0).  Double-word passes record the magnitude of the inputs read in
// `mag` (Dirichlet entries excluded) and publish the item's largest in sm.mag.
template <int PHYS, class N, int EX, int EY, bool COHERENT, bool DOT, bool SC, int RY = 1>
__device__ __forceinline__ double march_pass(const TileArgs &g, int item, int64_t rr,
                                             const typename N::IO *__restrict__ x, typename N::IO *__restrict__ y,
                                             MarchSmem<phys_ndpn(PHYS), N, EX, EY> &sm, int sc, int so,
                                             dwa::MagRec &mag) {
  constexpr bool IS_DW = std::is_same<N, tile::NumDW>::value;
  auto conv_in = [&](typename N::IO v) -> typename N::T {
    if constexpr (IS_DW && SC) return dwa::split_scaled(v, sc);
    else return N::in(v);
  };
  auto conv_out = [&](typename N::T v) -> typename N::IO {
    if constexpr (!SC) return N::out(v);
    else if constexpr (IS_DW) return dwa::ldexp_exact(N::out(v), so);
    else return dwa::ldexpf_exact(N::out(v), so);
  };
  (void)sc;
  (void)so;
  double dacc = 0.0;
  static_assert(EX == 32, "a warp is one row of element columns");
  static_assert(EY % RY == 0, "whole row groups per thread");
  using T = typename N::T;
  using IO = typename N::IO;
  constexpr int NC = phys_ndpn(PHYS);
  constexpr int NT = EX * EY / RY, PX = EX + 1, NP = (EX + 1) * (EY + 1);
  constexpr int LOADS = (NP + NT - 1) / NT;
  auto ldx = [](const IO *p) -> IO { return COHERENT ? __ldcg(p) : __ldg(p); };
  __syncthreads();  // the previous item of a persistent CTA may still be reading sm
  if (threadIdx.x == 0) sm.mag = 0u;

  const int tid = threadIdx.x;
  const int bx = item % g.tiles_x;
  const int by = (item / g.tiles_x) % g.tiles_y;
  const int bz = item / (g.tiles_x * g.tiles_y);
  const int i0 = bx * (EX - 1), j0 = by * (EY - 1);
  const int NXP = g.nx + 1, NYP = g.ny + 1;
  const int k0 = bz * g.seg, k1 = min(k0 + g.seg, g.nz + 1);
  const int tx = tid % EX, tw = tid / EX;
  const int ex = i0 - 1 + tx, ey0 = j0 - 1 + tw * RY;  // element rows ey0 .. ey0 + RY - 1
  const bool xin = ex >= 0 && ex < g.nx;
  bool ein[RY], own[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    const int ey = ey0 + r;
    ein[r] = xin && ey >= 0 && ey < g.ny;
    // this thread's lower-left node (ex, ey) of row r is owned by the CTA
    own[r] = tx >= 1 && tw * RY + r >= 1 && ex < NXP && ey < NYP;
  }

  // per-column geometry invariants
  T hx = N::zero(), ihx = N::zero();
  if (xin) {
    hx = N::from2(__ldg(g.hx + ex));
    ihx = N::from2(__ldg(g.ihx + ex));
  }
  T hy[RY], ihy[RY], hy_ihx[RY], hx_ihy[RY], hxhy[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    hy[r] = ihy[r] = N::zero();
    if (ein[r]) {
      hy[r] = N::from2(__ldg(g.hy + ey0 + r));
      ihy[r] = N::from2(__ldg(g.ihy + ey0 + r));
    }
    hy_ihx[r] = hx_ihy[r] = hxhy[r] = N::zero();
    if constexpr (phys_is_laplace(PHYS)) {
      hy_ihx[r] = N::mul(hy[r], ihx);
      hx_ihy[r] = N::mul(hx, ihy[r]);
      hxhy[r] = N::mul(hx, hy[r]);
    }
  }

  // plane staging: global -> registers (one plane ahead) -> shared memory
  IO xr[LOADS][NC];
  bool dr[LOADS];
  // in-plane node index of each load slot (-1: outside the mesh or the tile's plane)
  const int64_t NPL = (int64_t)NXP * NYP;
  int nib[LOADS];
#pragma unroll
  for (int l = 0; l < LOADS; ++l) {
    const int p = tid + l * NT;
    const int ix = i0 - 1 + p % PX, iy = j0 - 1 + p / PX;
    nib[l] = (p < NP && ix >= 0 && ix < NXP && iy >= 0 && iy < NYP) ? ix + NXP * iy : -1;
  }
  auto fetch = [&](int k) {
#pragma unroll
    for (int l = 0; l < LOADS; ++l) {
      const bool ok = nib[l] >= 0;
      const int64_t node = nib[l] + (int64_t)k * NPL;
      dr[l] = ok ? __ldg(g.dmask + node) != 0 : true;
#pragma unroll
      for (int c = 0; c < NC; ++c) xr[l][c] = ok ? ldx(x + (node * g.nrhs + rr) * NC + c) : (IO)0;
    }
  };
  auto stage = [&](int k) {
    auto *u = sm.up[k & 1];
#pragma unroll
    for (int l = 0; l < LOADS; ++l) {
      const int p = tid + l * NT;
      if (p < NP) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          N::st(u[p * NC + c], dr[l] ? N::zero() : conv_in(xr[l][c]));
          if constexpr (IS_DW)
            if (!dr[l]) mag.add(xr[l][c]);
        }
      }
    }
  };
  // 2D forward transforms of this thread's RY faces in plane k (modes: bit 0 x, bit 1 y): the
  // x-butterflies of the RY + 1 node rows, then the y-butterflies of each face
  auto face_fwd = [&](int k, T F[RY][NC][4]) {
    const auto *u = sm.up[k & 1];
    const int p = tx + PX * (tw * RY);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T a[RY + 1][2];
#pragma unroll
      for (int j = 0; j <= RY; ++j) {
        const T u0 = N::ld(u[(p + j * PX) * NC + c]), u1 = N::ld(u[(p + j * PX + 1) * NC + c]);
        a[j][0] = N::add(u0, u1);
        a[j][1] = N::sub(u1, u0);
      }
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        F[r][c][0] = N::add(a[r][0], a[r + 1][0]);
        F[r][c][1] = N::add(a[r][1], a[r + 1][1]);
        F[r][c][2] = N::sub(a[r + 1][0], a[r][0]);
        F[r][c][3] = N::sub(a[r + 1][1], a[r][1]);
      }
    }
  };

  const int s_lo = max(k0 - 1, 0);      // first element layer (the one below the segment)
  const int s_hi = min(k1 - 1, g.nz);   // last step; step nz only completes the top plane
  const int plim = min(k1, g.nz);       // highest node plane read
  fetch(s_lo);
  stage(s_lo);
  if (s_lo + 1 <= plim) {
    fetch(s_lo + 1);
    stage(s_lo + 1);
  }
  if (s_lo + 2 <= plim) fetch(s_lo + 2);
  __syncthreads();
  T Fb[RY][NC][4], Gc[RY][NC][4];  // bottom-face transforms of the current elements; top parts from below
  face_fwd(s_lo, Fb);
#pragma unroll
  for (int r = 0; r < RY; ++r)
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int m = 0; m < 4; ++m) Gc[r][c][m] = N::zero();
  __syncthreads();  // everyone has read plane s_lo before its buffer is reused

  // material of the elements: loaded one step ahead for elasticity; for the Laplace operators at
  // the top of the step, ahead of the face transform
  constexpr int NM = phys_nmat(PHYS);
  constexpr bool PREFETCH = PHYS != MF_LAPLACE;
  const int e_step = g.nx * g.ny * NM;
  const float2 *matp = g.mat + NM * (ex + (int64_t)g.nx * (ey0 + (int64_t)g.ny * s_lo));
  float2 mat_next[RY][NM];
#pragma unroll
  for (int r = 0; r < RY; ++r)
#pragma unroll
    for (int q = 0; q < NM; ++q)
      mat_next[r][q] = (PREFETCH && ein[r] && s_lo < g.nz) ? __ldg(matp + r * g.nx * NM + q) : make_float2(0.f, 0.f);

  for (int ez = s_lo; ez <= s_hi; ++ez) {
    float2 mat_cur[RY][NM];
    if constexpr (PREFETCH) {
      matp += e_step;
#pragma unroll
      for (int r = 0; r < RY; ++r)
#pragma unroll
        for (int q = 0; q < NM; ++q) {
          mat_cur[r][q] = mat_next[r][q];
          mat_next[r][q] = (ein[r] && ez + 1 < g.nz) ? __ldg(matp + r * g.nx * NM + q) : make_float2(0.f, 0.f);
        }
    } else {
#pragma unroll
      for (int r = 0; r < RY; ++r)
#pragma unroll
        for (int q = 0; q < NM; ++q)
          mat_cur[r][q] = (ein[r] && ez < g.nz) ? __ldg(matp + r * g.nx * NM + q) : make_float2(0.f, 0.f);
      matp += e_step;
    }
    T Ft[RY][NC][4];
    if (ez < g.nz) face_fwd(ez + 1, Ft);
    else {
#pragma unroll
      for (int r = 0; r < RY; ++r)
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
          for (int m = 0; m < 4; ++m) Ft[r][c][m] = N::zero();
    }
    T hz = N::zero(), ihz = N::zero();
    if (ez < g.nz) {
      hz = N::from2(__ldg(g.hz + ez));
      ihz = N::from2(__ldg(g.ihz + ez));
    }
    T rb[RY][NC], tp[RY][NC];  // contributions to each face's bottom and top node rows (x-summed)
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      T S[NC][4];
      if (ein[r] && ez < g.nz) {
        // o[l][m]: D times the 8 modes; the z butterfly gives mode m (m < 4) as Fb + Ft and mode
        // m + 4 as Ft - Fb; mode 0 has D = 0
        T o[NC][8];
        if constexpr (phys_is_laplace(PHYS)) {  // Laplace; vector Laplace: the same D per component
          const tile::LapCoef<N> cf =
              tile::laplace_coef<N>(N::from2(mat_cur[r][0]), hy_ihx[r], hx_ihy[r], hxhy[r], hz, ihz);
#pragma unroll
          for (int l = 0; l < NC; ++l) {
            o[l][1] = N::mul(cf.s1, N::add(Fb[r][l][1], Ft[r][l][1]));
            o[l][2] = N::mul(cf.s2, N::add(Fb[r][l][2], Ft[r][l][2]));
            o[l][3] = N::mul(cf.s12, N::add(Fb[r][l][3], Ft[r][l][3]));
            o[l][4] = N::mul(cf.s3, N::sub(Ft[r][l][0], Fb[r][l][0]));
            o[l][5] = N::mul(cf.s13, N::sub(Ft[r][l][1], Fb[r][l][1]));
            o[l][6] = N::mul(cf.s23, N::sub(Ft[r][l][2], Fb[r][l][2]));
            o[l][7] = N::mul(cf.s123, N::sub(Ft[r][l][3], Fb[r][l][3]));
          }
        } else {
          const T h[3] = {hx, hy[r], hz}, ih[3] = {ihx, ihy[r], ihz};
          const tile::ElCoef<N> cf =
              tile::elasticity_coef<N>(N::from2(mat_cur[r][0]), N::from2(mat_cur[r][NM - 1]), h, ih);
          T c[3][8];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            c[k][0] = N::zero();
#pragma unroll
            for (int m = 1; m < 4; ++m) c[k][m] = N::add(Fb[r][k][m], Ft[r][k][m]);
#pragma unroll
            for (int m = 0; m < 4; ++m) c[k][m + 4] = N::sub(Ft[r][k][m], Fb[r][k][m]);
          }
          tile::elasticity_modes<N>(cf, c, o);
        }
        // transposed z butterfly: bottom part o[m] - o[m+4] (summed with the carried top part of
        // the element below), top part o[m] + o[m+4] (carried up)
#pragma unroll
        for (int l = 0; l < NC; ++l) {
          S[l][0] = N::sub(Gc[r][l][0], o[l][4]);
          Gc[r][l][0] = o[l][4];
#pragma unroll
          for (int m = 1; m < 4; ++m) {
            S[l][m] = N::add(Gc[r][l][m], N::sub(o[l][m], o[l][m + 4]));
            Gc[r][l][m] = N::add(o[l][m], o[l][m + 4]);
          }
        }
      } else {
#pragma unroll
        for (int l = 0; l < NC; ++l)
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            S[l][m] = Gc[r][l][m];
            Gc[r][l][m] = N::zero();
          }
      }
      // transposed 2D transform of the face sums -> contributions to the face's 4 corner nodes;
      // along x node (ex, .) gets this face's left corners and the left neighbour face's right ones
#pragma unroll
      for (int l = 0; l < NC; ++l) {
        const T t0 = N::sub(S[l][0], S[l][1]), t1 = N::add(S[l][0], S[l][1]);
        const T t2 = N::sub(S[l][2], S[l][3]), t3 = N::add(S[l][2], S[l][3]);
        const T v00 = N::sub(t0, t2), v01 = N::add(t0, t2), v10 = N::sub(t1, t3), v11 = N::add(t1, t3);
        rb[r][l] = N::add(v00, shfl_up1<N>(v10));
        tp[r][l] = N::add(v01, shfl_up1<N>(v11));
      }
    }
    // the top node row of the thread's last face goes to the thread above through shared memory
#pragma unroll
    for (int l = 0; l < NC; ++l) N::st(sm.xrow[ez & 1][l * NT + tid], tp[RY - 1][l]);
    bool wr[RY], dir[RY];
    int64_t node[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      wr[r] = own[r] && ez >= k0;
      node[r] = (ex + NXP * (ey0 + r)) + (int64_t)ez * NPL;
      dir[r] = wr[r] && __ldg(g.dmask + node[r]) != 0;  // issued before the barrier
    }
    if (ez + 2 <= plim) {
      stage(ez + 2);  // plane ez's buffer: its last reader finished before the previous barrier
      if (ez + 3 <= plim) fetch(ez + 3);
    }
    if constexpr (IS_DW) {
      // every plane has been staged by now: publish the item's largest input record, which the
      // barrier below makes visible to the whole CTA after the march
      if (ez == s_hi) {
        const unsigned w = __reduce_max_sync(0xffffffffu, mag.key);
        if ((threadIdx.x & 31) == 0) atomicMax(&sm.mag, w);
      }
    }
    __syncthreads();
    // y: node (ex, ey) gets the bottom row of the faces at ey and the top row of the faces at ey - 1
    // (this thread's previous row, or the thread below for the first row)
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      if (wr[r]) {
#pragma unroll
        for (int l = 0; l < NC; ++l) {
          const T below = r == 0 ? N::ld(sm.xrow[ez & 1][l * NT + tid - EX]) : tp[r > 0 ? r - 1 : 0][l];
          const T tot = N::add(rb[r][l], below);
          const int64_t vi = (node[r] * g.nrhs + rr) * NC + l;
          if constexpr (DOT) {
            const IO xv = ldx(x + vi);
            const IO yv = dir[r] ? xv : conv_out(tot);
            y[vi] = yv;
            dacc += (double)xv * (double)yv;
          } else {
            y[vi] = dir[r] ? ldx(x + vi) : conv_out(tot);
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RY; ++r)
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int m = 0; m < 4; ++m) Fb[r][c][m] = Ft[r][c][m];
  }
  return dacc;
}

// The scaled pass as a separate (not inlined) function: it runs for normalised meshes and for the
// rare work items whose inputs lie outside the double-word range, and keeping its code out of the
// unscaled pass leaves that pass its registers.
template <int PHYS, class N, int EX, int EY, bool COHERENT, bool DOT, int RY>
__device__ __noinline__ double march_pass_scaled(const TileArgs &g, int item, int64_t rr,
                                                 const typename N::IO *__restrict__ x, typename N::IO *__restrict__ y,
                                                 MarchSmem<phys_ndpn(PHYS), N, EX, EY> &sm, int sc, int so,
                                                 dwa::MagRec &mag) {
  return march_pass<PHYS, N, EX, EY, COHERENT, DOT, true, RY>(g, item, rr, x, y, sm, sc, so, mag);
}

// One work item with the output scaling of the mesh; for double-word arithmetic, if the largest input
// the CTA read lies outside [2^kMagLo, 2^kMagHi] the item is computed again with x scaled by the power
// of two that brings that input to [1, 2) (and y scaled back), so results keep FP64 accuracy over
// FP64's whole range.  The decision depends on the item's own inputs only (deterministic); the
// second pass overwrites every value the first one wrote.
template <int PHYS, class N, int EX, int EY, bool COHERENT, bool DOT = false, int RY = 1>
__device__ __forceinline__ double march_item(const TileArgs &g, int item, int64_t rr,
                                             const typename N::IO *__restrict__ x, typename N::IO *__restrict__ y,
                                             MarchSmem<phys_ndpn(PHYS), N, EX, EY> &sm) {
  dwa::MagRec mag;
  double d = g.oscale == 0
                 ? march_pass<PHYS, N, EX, EY, COHERENT, DOT, false, RY>(g, item, rr, x, y, sm, 0, 0, mag)
                 : march_pass_scaled<PHYS, N, EX, EY, COHERENT, DOT, RY>(g, item, rr, x, y, sm, 0, g.oscale, mag);
  if constexpr (std::is_same<N, tile::NumDW>::value) {
    int s = 0;
    if (dwa::mag_exponent(sm.mag, s) && (s < dwa::kMagLo || s > dwa::kMagHi))
      d = march_pass_scaled<PHYS, N, EX, EY, COHERENT, DOT, RY>(g, item, rr, x, y, sm, s, g.oscale + s, mag);
  }
  return d;
}

template <int PHYS, class N, int EX, int EY, int RY, int MINB>
__global__ void __launch_bounds__(EX *EY / RY, MINB) march_apply(TileArgs g, const typename N::IO *__restrict__ x,
                                                                 typename N::IO *__restrict__ y,
                                                                 const int *__restrict__ skip) {
  __shared__ MarchSmem<phys_ndpn(PHYS), N, EX, EY> sm;
  if (skip && *skip) return;
  // right-hand side fastest: CTAs that run together read the same x lines ([node][rhs][comp])
  march_item<PHYS, N, EX, EY, false, false, RY>(g, blockIdx.x / g.nrhs, g.r0 + blockIdx.x % g.nrhs, x, y, sm);
}

// Apply with the dot product x . y fused in (one right-hand side): each CTA stores its part, the
// last CTA to finish (ticket) sums the parts in CTA order into *out and resets the ticket, so the
// result does not depend on scheduling.  partials: one slot per CTA.
template <int PHYS, class N, int EX, int EY, int RY, int MINB>
__global__ void __launch_bounds__(EX *EY / RY, MINB)
    march_apply_dot(TileArgs g, const typename N::IO *__restrict__ x, typename N::IO *__restrict__ y,
                    const int *__restrict__ skip, double *__restrict__ partials, unsigned int *ticket,
                    double *out) {
  constexpr int NT = EX * EY / RY, NW = NT / 32;
  __shared__ MarchSmem<phys_ndpn(PHYS), N, EX, EY> sm;
  __shared__ double red[NW];
  __shared__ bool last;
  if (skip && *skip) return;
  double d = march_item<PHYS, N, EX, EY, false, true, RY>(g, blockIdx.x, g.r0, x, y, sm);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
  if (lane == 0) red[w] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < NW; ++i) s += red[i];
    partials[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += NT) s += __ldcg(partials + i);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  __syncthreads();
  if (lane == 0) red[w] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < NW; ++i) t += red[i];
    *out = t;
    *ticket = 0u;
  }
}

// Launch shapes: EX = 32 element columns per warp row, EY element rows, RY rows per thread (threads
// EX EY / RY), MINB resident CTAs per SM.
// Double-word elasticity takes 12 rows at 168 registers (12 warps per SM, halo factor 1.13): at 8
// rows it needed 241 registers and ran 8 warps per SM, 17 % slower at 160^3.  FP32 elasticity keeps
// 8 rows, where it is fastest.
#ifndef MF_LAP_EY
#define MF_LAP_EY 16
#endif
#ifndef MF_LAP_RY
#define MF_LAP_RY 2
#endif
#ifndef MF_LAP_MINB
#define MF_LAP_MINB 2
#endif
template <int PHYS, class N> struct MarchShape { static constexpr int EX = 32, EY = 8, RY = 1, MINB = 4; };
template <> struct MarchShape<MF_LAPLACE, tile::NumDW> {
  static constexpr int EX = 32, EY = MF_LAP_EY, RY = MF_LAP_RY, MINB = MF_LAP_MINB;
};
template <class N> struct MarchShape<MF_ELASTICITY, N> { static constexpr int EX = 32, EY = 8, RY = 1, MINB = 1; };
template <> struct MarchShape<MF_ELASTICITY, tile::NumDW> { static constexpr int EX = 32, EY = 12, RY = 1, MINB = 1; };
template <class N> struct MarchShape<MF_VECTOR_LAPLACE, N> { static constexpr int EX = 32, EY = 8, RY = 1, MINB = 2; };

}  // namespace march
