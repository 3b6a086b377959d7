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

// Operands of the CG iteration fused into the apply (classic Hestenes-Stiefel recurrence, FP64
// vectors, one right-hand side).  The apply of iteration k forms its input
//   p_k = z_k + beta_{k-1} p_{k-1},   z_k = r_k (or D^-1 r_k with Jacobi),
// node by node while it stages the node planes (every CTA recomputes its halo nodes), stores p_k
// and the deferred solution update x_k = x_{k-1} + alpha_{k-1} p_{k-1} for the nodes it owns, and
// returns A p_k and p_k . A p_k.  p_{k-1} and p_k live in two buffers: neighbouring CTAs still read
// p_{k-1} at their halo nodes while this one writes p_k.  The FP64 formulas are those of the
// separate vector kernels (same operations, same rounding), so the iterates are bitwise the same.
struct CgFuse {
  const double *r, *pold;  // r_k, p_{k-1}
  const double *invd;      // 1 / diag(A) (Jacobi) or null
  double *pnew, *x;        // p_k (written), x (updated in place)
  const double *ab;        // alpha_{k-1}, beta_{k-1} (device scalars)
};

// 8-byte asynchronous copy global -> shared (zero-filled when !valid: nothing is read)
__device__ __forceinline__ void cpa8(void *dst, const void *src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(valid ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cpa_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// PHYS = MF_LAPLACE (Eq. 7), MF_VECTOR_LAPLACE (Eq. 5) or MF_ELASTICITY (Eq. 9, Algorithm 1);
// vectors hold NC values per node (x, y, z components interleaved for the vector operators).
// One work item (tile column x z-segment `item`, right-hand side `rr`); must be called by all EX*EY
// threads of the CTA.  COHERENT: read x through L2 only (x was written by other CTAs earlier in the
// same persistent kernel, so the read-only and L1 paths may hold stale lines).
// DOT: also return this thread's part of x . y over the nodes it writes (the dot product a CG
// iteration needs next, p . Ap, formed while the result is written; FP64 products and sums).
// SC: power-of-two scaling, x * 2^-sc in and y * 2^so out (the cell constants and spacings of a
// normalised mesh, and the rescaled pass for inputs outside the double-word range); without SC
// neither is applied.  Double-word passes record in `mag` the magnitude of the inputs this thread
// staged (Dirichlet entries excluded).
// CGU (with DOT, FP64 vectors): the CG iteration of CgFuse fused in; x is then p_k's buffer (cg.pnew),
// the staged values are formed from cg's vectors copied asynchronously into `raw` (two buffers of
// 3 or 4 arrays of the plane's NP x NC values, then a ring of 4 planes of the owned nodes' p_k in FP64
// for the write phase), and sab holds alpha_{k-1}, beta_{k-1}.
template <int PHYS, class N, int EX, int EY, bool COHERENT, bool DOT, bool SC, bool CGU = false>
__device__ __forceinline__ double march_pass(const TileArgs &g, int item, int64_t rr,
                                             const typename N::IO *__restrict__ x, typename N::IO *__restrict__ y,
                                             MarchSmem<phys_ndpn(PHYS), N, EX, EY> &sm, int sc, int so,
                                             dwa::MagRec &mag, const CgFuse *cg = nullptr, double *raw = nullptr,
                                             const double *sab = nullptr) {
  static_assert(!CGU || (DOT && std::is_same<typename N::IO, double>::value), "CG fusion: FP64 vectors with the dot");
  (void)cg;
  (void)raw;
  (void)sab;
  constexpr bool IS_DW = std::is_same<N, tile::NumDW>::value;
  // Unscaled double-word passes split without split()'s path for magnitudes outside [2^-74, 2^127):
  // such inputs lie outside the range window, so the magnitude record sends their work item to the
  // scaled pass, which overwrites everything this pass wrote.
  auto conv_in = [&](typename N::IO v) -> typename N::T {
    if constexpr (IS_DW && SC) {
      return dwa::split_shift(v, sc);
    } else if constexpr (IS_DW) {
      unsigned e;
      return dwa::split_fast(v, e);
    } else {
      return N::in(v);
    }
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
  using T = typename N::T;
  using IO = typename N::IO;
  constexpr int NC = phys_ndpn(PHYS);
  constexpr int NT = EX * EY, PX = EX + 1, NP = (EX + 1) * (EY + 1), TX = EX - 1, TY = EY - 1;
  constexpr int LOADS = (NP + NT - 1) / NT;
  (void)TX;
  (void)TY;
  auto ldx = [](const IO *p) -> IO { return COHERENT ? __ldcg(p) : __ldg(p); };
  __syncthreads();  // the previous item of a persistent CTA may still be reading sm

  const int tid = threadIdx.x;
  const int bx = item % g.tiles_x;
  const int by = (item / g.tiles_x) % g.tiles_y;
  const int bz = item / (g.tiles_x * g.tiles_y);
  const int i0 = bx * (EX - 1), j0 = by * (EY - 1);
  const int NXP = g.nx + 1, NYP = g.ny + 1;
  const int k0 = bz * g.seg, k1 = min(k0 + g.seg, g.nz + 1);
  const int tx = tid % EX, ty = tid / EX;
  const int ex = i0 - 1 + tx, ey = j0 - 1 + ty;
  const bool ein = ex >= 0 && ex < g.nx && ey >= 0 && ey < g.ny;
  // this thread's lower-left node (ex, ey) is owned by the CTA
  const bool own = tx >= 1 && ty >= 1 && ex < NXP && ey < NYP;

  // per-column geometry invariants
  T hx = N::zero(), hy = N::zero(), ihx = N::zero(), ihy = N::zero();
  if (ein) {
    hx = N::from2(__ldg(g.hx + ex));
    ihx = N::from2(__ldg(g.ihx + ex));
    hy = N::from2(__ldg(g.hy + ey));
    ihy = N::from2(__ldg(g.ihy + ey));
  }
  T hy_ihx = N::zero(), hx_ihy = N::zero(), hxhy = N::zero();
  if constexpr (phys_is_laplace(PHYS)) {
    hy_ihx = N::mul(hy, ihx);
    hx_ihy = N::mul(hx, ihy);
    hxhy = N::mul(hx, hy);
  }

  // plane staging: global -> registers (one plane ahead) -> shared memory
  IO xr[LOADS][NC];
  bool dr[LOADS];
  // in-plane node index of each load slot (-1: outside the mesh or the tile's plane)
  const int64_t NPL = (int64_t)NXP * NYP, NN = NPL * (g.nz + 1);
  (void)NN;
  int nib[LOADS];
#pragma unroll
  for (int l = 0; l < LOADS; ++l) {
    const int p = tid + l * NT;
    const int ix = i0 - 1 + p % PX, iy = j0 - 1 + p / PX;
    nib[l] = (p < NP && ix >= 0 && ix < NXP && iy >= 0 && iy < NYP) ? ix + NXP * iy : -1;
  }
  // CGU: slots whose node this CTA owns (written once: p_k and x), and the raw array layout
  unsigned own_slot = 0u;
  const int na = CGU && cg->invd ? 4 : 3;  // r, p_{k-1}, x [, 1/diag]
  if constexpr (CGU) {
#pragma unroll
    for (int l = 0; l < LOADS; ++l) {
      const int p = tid + l * NT, px = p % PX, py = p / PX;
      if (nib[l] >= 0 && px >= 1 && px <= EX - 1 && py >= 1 && py <= EY - 1) own_slot |= 1u << l;
    }
  }
  auto rawp = [&](int k, int a, int idx) -> double * { return raw + ((k & 1) * na + a) * (NP * NC) + idx; };
  // p_k of the owned nodes by owner thread, planes k mod 4: written at staging, read two steps later in
  // the write phase; the next write to the same plane slot comes two barriers after that read
  auto pown = [&](int k, int idx) -> double * { return raw + 2 * na * (NP * NC) + (k & 3) * (NT * NC) + idx; };
  auto fetch = [&](int k) {
#pragma unroll
    for (int l = 0; l < LOADS; ++l) {
      const bool ok = nib[l] >= 0;
      const int64_t node = ok ? mf_dbg_index(nib[l] + (int64_t)k * NPL, NN, MF_DBG_NODE) : 0;
      dr[l] = ok ? __ldg(g.dmask + node) != 0 : true;
      if constexpr (CGU) {
        const int p = tid + l * NT;
        const bool ownk = (own_slot >> l & 1u) && k >= k0 && k < k1;
        if (p < NP)
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const int64_t gi = node * NC + c;
            cpa8(rawp(k, 0, p * NC + c), cg->r + (ok ? gi : 0), ok);
            cpa8(rawp(k, 1, p * NC + c), cg->pold + (ok ? gi : 0), ok);
            cpa8(rawp(k, 2, p * NC + c), cg->x + (ownk ? gi : 0), ownk);
            if (na == 4) cpa8(rawp(k, 3, p * NC + c), cg->invd + (ok ? gi : 0), ok);
          }
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) xr[l][c] = ok ? ldx(x + (node * g.nrhs + rr) * NC + c) : (IO)0;
      }
    }
    if constexpr (CGU) cpa_commit();
  };
  auto stage = [&](int k) {
    auto *u = sm.up[k & 1];
    if constexpr (CGU) cpa_wait_all();  // this thread's copies of plane k (issued one step earlier)
#pragma unroll
    for (int l = 0; l < LOADS; ++l) {
      const int p = tid + l * NT;
      if (p < NP)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          IO v;
          if constexpr (CGU) {
            const int i = p * NC + c;
            const double rv = *rawp(k, 0, i), po = *rawp(k, 1, i);
            const double z = na == 4 ? __dmul_rn(rv, *rawp(k, 3, i)) : rv;
            v = __fma_rn(sab[1], po, z);  // p_k
            if ((own_slot >> l & 1u) && k >= k0 && k < k1) {
              const int64_t gi = mf_dbg_index(nib[l] + (int64_t)k * NPL, NN, MF_DBG_NODE) * NC + c;
              cg->pnew[gi] = v;
              cg->x[gi] = __fma_rn(sab[0], po, *rawp(k, 2, i));
              *pown(k, ((p % PX) + EX * (p / PX)) * NC + c) = v;  // owner thread (p % PX, p / PX)
            }
          } else {
            v = xr[l][c];
          }
          N::st(u[p * NC + c], dr[l] ? N::zero() : conv_in(v));
          if constexpr (IS_DW)
            if (!dr[l]) mag.add(v);
        }
    }
  };
  // 2D forward transform of this thread's face in plane k (modes: bit 0 x, bit 1 y)
  auto face_fwd = [&](int k, T F[NC][4]) {
    const auto *u = sm.up[k & 1];
    const int p = tx + PX * ty;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const T u0 = N::ld(u[p * NC + c]), u1 = N::ld(u[(p + 1) * NC + c]);
      const T u2 = N::ld(u[(p + PX) * NC + c]), u3 = N::ld(u[(p + PX + 1) * NC + c]);
      const T a0 = N::add(u0, u1), a1 = N::sub(u1, u0), a2 = N::add(u2, u3), a3 = N::sub(u3, u2);
      F[c][0] = N::add(a0, a2);
      F[c][1] = N::add(a1, a3);
      F[c][2] = N::sub(a2, a0);
      F[c][3] = N::sub(a3, a1);
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
  T Fb[NC][4], Gc[NC][4];  // bottom-face transform of the current element; top-face part from below
  face_fwd(s_lo, Fb);
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int m = 0; m < 4; ++m) Gc[c][m] = N::zero();
  __syncthreads();  // everyone has read plane s_lo before its buffer is reused

  // material of the element: loaded one step ahead for elasticity; for Laplace (64 registers at
  // two 512-thread CTAs per SM) at the top of the step, ahead of the face transform
  constexpr int NM = phys_nmat(PHYS);
  constexpr bool PREFETCH = PHYS != MF_LAPLACE;
  const int e_step = g.nx * g.ny * NM;
  const float2 *matp = g.mat + NM * (ex + (int64_t)g.nx * (ey + (int64_t)g.ny * s_lo));
  const int64_t NMC = (int64_t)NM * g.nx * g.ny * g.nz;  // cell constants of the mesh
  (void)NMC;
  float2 mat_next[NM];
#pragma unroll
  for (int q = 0; q < NM; ++q)
    mat_next[q] = (PREFETCH && ein && s_lo < g.nz) ? __ldg(MF_DBG_PTR(matp + q, g.mat, NMC, MF_DBG_CELL))
                                                   : make_float2(0.f, 0.f);

  for (int ez = s_lo; ez <= s_hi; ++ez) {
    const bool elem = ein && ez < g.nz;
    float2 mat_cur[NM];
    if constexpr (PREFETCH) {
      matp += e_step;
#pragma unroll
      for (int q = 0; q < NM; ++q) {
        mat_cur[q] = mat_next[q];
        mat_next[q] = (ein && ez + 1 < g.nz) ? __ldg(MF_DBG_PTR(matp + q, g.mat, NMC, MF_DBG_CELL))
                                             : make_float2(0.f, 0.f);
      }
    } else {
#pragma unroll
      for (int q = 0; q < NM; ++q)
        mat_cur[q] = elem ? __ldg(MF_DBG_PTR(matp + q, g.mat, NMC, MF_DBG_CELL)) : make_float2(0.f, 0.f);
      matp += e_step;
    }
    T Ft[NC][4], S[NC][4];
    if (ez < g.nz) face_fwd(ez + 1, Ft);
    else {
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int m = 0; m < 4; ++m) Ft[c][m] = N::zero();
    }
    if (elem) {
      const T hz = N::from2(__ldg(g.hz + ez)), ihz = N::from2(__ldg(g.ihz + ez));
      // o[l][m]: D times the 8 modes; the z butterfly gives mode m (m < 4) as Fb + Ft and mode
      // m + 4 as Ft - Fb; mode 0 has D = 0
      T o[NC][8];
      if constexpr (phys_is_laplace(PHYS)) {  // Laplace; vector Laplace: the same D per component
        const tile::LapCoef<N> cf = tile::laplace_coef<N>(N::from2(mat_cur[0]), hy_ihx, hx_ihy, hxhy, hz, ihz);
#pragma unroll
        for (int l = 0; l < NC; ++l) {
          o[l][1] = N::mul(cf.s1, N::add(Fb[l][1], Ft[l][1]));
          o[l][2] = N::mul(cf.s2, N::add(Fb[l][2], Ft[l][2]));
          o[l][3] = N::mul(cf.s12, N::add(Fb[l][3], Ft[l][3]));
          o[l][4] = N::mul(cf.s3, N::sub(Ft[l][0], Fb[l][0]));
          o[l][5] = N::mul(cf.s13, N::sub(Ft[l][1], Fb[l][1]));
          o[l][6] = N::mul(cf.s23, N::sub(Ft[l][2], Fb[l][2]));
          o[l][7] = N::mul(cf.s123, N::sub(Ft[l][3], Fb[l][3]));
        }
      } else {
        const T h[3] = {hx, hy, hz}, ih[3] = {ihx, ihy, ihz};
        const tile::ElCoef<N> cf =
            tile::elasticity_coef<N>(N::from2(mat_cur[0]), N::from2(mat_cur[NM - 1]), h, ih);
        T c[3][8];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          c[k][0] = N::zero();
#pragma unroll
          for (int m = 1; m < 4; ++m) c[k][m] = N::add(Fb[k][m], Ft[k][m]);
#pragma unroll
          for (int m = 0; m < 4; ++m) c[k][m + 4] = N::sub(Ft[k][m], Fb[k][m]);
        }
        tile::elasticity_modes<N>(cf, c, o);
      }
      // transposed z butterfly: bottom part o[m] - o[m+4] (summed with the carried top part of the
      // element below), top part o[m] + o[m+4] (carried up)
#pragma unroll
      for (int l = 0; l < NC; ++l) {
        S[l][0] = N::sub(Gc[l][0], o[l][4]);
        Gc[l][0] = o[l][4];
#pragma unroll
        for (int m = 1; m < 4; ++m) {
          S[l][m] = N::add(Gc[l][m], N::sub(o[l][m], o[l][m + 4]));
          Gc[l][m] = N::add(o[l][m], o[l][m + 4]);
        }
      }
    } else {
#pragma unroll
      for (int l = 0; l < NC; ++l)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          S[l][m] = Gc[l][m];
          Gc[l][m] = N::zero();
        }
    }
    // transposed 2D transform of the face sums -> contributions to the face's 4 corner nodes; along
    // x node (ex, .) gets this face's left corners and the left neighbour face's right corners
    T rb[NC];
#pragma unroll
    for (int l = 0; l < NC; ++l) {
      const T t0 = N::sub(S[l][0], S[l][1]), t1 = N::add(S[l][0], S[l][1]);
      const T t2 = N::sub(S[l][2], S[l][3]), t3 = N::add(S[l][2], S[l][3]);
      const T v00 = N::sub(t0, t2), v01 = N::add(t0, t2), v10 = N::sub(t1, t3), v11 = N::add(t1, t3);
      rb[l] = N::add(v00, shfl_up1<N>(v10));
      N::st(sm.xrow[ez & 1][l * NT + tid], N::add(v01, shfl_up1<N>(v11)));
    }
    const bool wr = own && ez >= k0;
    const int64_t node = wr ? mf_dbg_index((ex + NXP * ey) + (int64_t)ez * NPL, NN, MF_DBG_NODE) : 0;
    const bool dir = wr && __ldg(g.dmask + node) != 0;  // issued before the barrier
    if (ez + 2 <= plim) {
      stage(ez + 2);  // plane ez's buffer: its last reader finished before the previous barrier
      if (ez + 3 <= plim) fetch(ez + 3);
    }
    __syncthreads();
    // y: node (ex, ey) gets the bottom row of this thread's faces and the top row of the row below
    if (wr) {
#pragma unroll
      for (int l = 0; l < NC; ++l) {
        const T tot = N::add(rb[l], N::ld(sm.xrow[ez & 1][l * NT + tid - EX]));
        const int64_t vi = (node * g.nrhs + rr) * NC + l;
        if constexpr (DOT) {
          IO xv;
          if constexpr (CGU) xv = *pown(ez, tid * NC + l);  // p_k, staged two steps earlier
          else xv = ldx(x + vi);
          const IO yv = dir ? xv : conv_out(tot);
          y[vi] = yv;
          dacc += (double)xv * (double)yv;
        } else {
          y[vi] = dir ? ldx(x + vi) : conv_out(tot);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int m = 0; m < 4; ++m) Fb[c][m] = Ft[c][m];
  }
  return dacc;
}

// The scaled pass as a separate (not inlined) function: it runs for normalised meshes and for the
// rare work items whose inputs lie outside the double-word range, and keeping its code out of the
// unscaled pass leaves that pass its registers.
template <int PHYS, class N, int EX, int EY, bool COHERENT, bool DOT>
__device__ __noinline__ double march_pass_scaled(const TileArgs &g, int item, int64_t rr,
                                                 const typename N::IO *__restrict__ x, typename N::IO *__restrict__ y,
                                                 MarchSmem<phys_ndpn(PHYS), N, EX, EY> &sm, int sc, int so,
                                                 dwa::MagRec &mag) {
  return march_pass<PHYS, N, EX, EY, COHERENT, DOT, true>(g, item, rr, x, y, sm, sc, so, mag);
}

// One work item with the output scaling of the mesh; for double-word arithmetic, if the largest input
// the CTA read lies outside [2^kMagLo, 2^kMagHi] the item is computed again with x scaled by the power
// of two that brings that input to [1, 2) (and y scaled back), so results keep FP64 accuracy over
// FP64's whole range.  The decision depends on the item's own inputs only (deterministic); the
// second pass overwrites every value the first one wrote.
template <int PHYS, class N, int EX, int EY, bool COHERENT, bool DOT = false>
__device__ __forceinline__ double march_item(const TileArgs &g, int item, int64_t rr,
                                             const typename N::IO *__restrict__ x, typename N::IO *__restrict__ y,
                                             MarchSmem<phys_ndpn(PHYS), N, EX, EY> &sm) {
  dwa::MagRec mag;
  double d = g.oscale == 0
                 ? march_pass<PHYS, N, EX, EY, COHERENT, DOT, false>(g, item, rr, x, y, sm, 0, 0, mag)
                 : march_pass_scaled<PHYS, N, EX, EY, COHERENT, DOT>(g, item, rr, x, y, sm, 0, g.oscale, mag);
  if constexpr (std::is_same<N, tile::NumDW>::value) {
    const unsigned w = __reduce_max_sync(0xffffffffu, mag.key);
    __syncthreads();
    if (threadIdx.x == 0) sm.mag = 0u;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicMax(&sm.mag, w);
    __syncthreads();
    int s = 0;
    if (dwa::mag_exponent(sm.mag, s) && (s < dwa::kMagLo || s > dwa::kMagHi))
      d = march_pass_scaled<PHYS, N, EX, EY, COHERENT, DOT>(g, item, rr, x, y, sm, s, g.oscale + s, mag);
  }
  return d;
}

// Stand-alone launches: one pass per work item, without the range check's second pass, so that the
// check adds no code (and no registers) to them.  A thread whose staged inputs' largest magnitude lies
// outside [2^kMagLo, 2^kMagHi] sets this launch's bit in the CTA's flag word; march_fixup, launched
// right after on the same stream, redoes those work items with the scaled pass.  SCALED: the
// instantiation for normalised meshes (y scaled by 2^oscale; the host picks it by the mesh).
template <int PHYS, class N, int EX, int EY, int MINB, bool SCALED = false>
__global__ void __launch_bounds__(EX *EY, MINB) march_apply(TileArgs g, const typename N::IO *__restrict__ x,
                                                                 typename N::IO *__restrict__ y,
                                                                 const int *__restrict__ skip) {
  __shared__ MarchSmem<phys_ndpn(PHYS), N, EX, EY> sm;
  if (skip && *skip) return;
  dwa::MagRec mag;
  // right-hand side fastest: CTAs that run together read the same x lines ([node][rhs][comp])
  march_pass<PHYS, N, EX, EY, false, false, SCALED>(g, blockIdx.x / g.nrhs, g.r0 + blockIdx.x % g.nrhs, x, y, sm, 0,
                                                        SCALED ? g.oscale : 0, mag);
  if constexpr (std::is_same<N, tile::NumDW>::value)
    if (dwa::mag_outside(mag.key)) atomicOr(g.flags + blockIdx.x, g.bit);
}

// Sum of the per-CTA parts in CTA order into *out (the last CTA of the launch to arrive does it and
// resets the ticket), so that the result does not depend on scheduling.
template <int NT>
__device__ __forceinline__ void ordered_dot_sum(double d, double *__restrict__ partials, int slot, int nslots,
                                                unsigned int *ticket, double *out, bool store) {
  constexpr int NW = NT / 32;
  __shared__ double red[NW];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
  if (lane == 0) red[w] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    if (store) {
      double s = 0.0;
      for (int i = 0; i < NW; ++i) s += red[i];
      partials[slot] = s;
    }
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (int i = threadIdx.x; i < nslots; i += NT) s += __ldcg(partials + i);
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

// Apply with the dot product x . y fused in (one right-hand side): each CTA stores its part, the
// last CTA to finish sums the parts in CTA order into *out.  partials: one slot per CTA.  SCALED as
// for march_apply.
template <int PHYS, class N, int EX, int EY, int MINB, bool SCALED = false>
__global__ void __launch_bounds__(EX *EY, MINB)
    march_apply_dot(TileArgs g, const typename N::IO *__restrict__ x, typename N::IO *__restrict__ y,
                    const int *__restrict__ skip, double *__restrict__ partials, unsigned int *ticket,
                    double *out) {
  __shared__ MarchSmem<phys_ndpn(PHYS), N, EX, EY> sm;
  if (skip && *skip) return;
  dwa::MagRec mag;
  const double d = march_pass<PHYS, N, EX, EY, false, true, SCALED>(g, blockIdx.x, g.r0, x, y, sm, 0,
                                                                     SCALED ? g.oscale : 0, mag);
  if constexpr (std::is_same<N, tile::NumDW>::value)
    if (dwa::mag_outside(mag.key)) atomicOr(g.flags + blockIdx.x, g.bit);
  ordered_dot_sum<EX * EY>(d, partials, blockIdx.x, gridDim.x, ticket, out, true);
}

// One CG iteration's apply with the vector updates of CgFuse fused in: stores p_k and x for the owned
// nodes, y = A p_k, and p_k . A p_k summed in CTA order into *out (as march_apply_dot).  Dynamic shared
// memory: cg_raw_bytes.  Unscaled meshes only (the caller keeps the separate kernels on a normalised
// mesh); inputs outside the double-word window flag the CTA for march_fixup, which reads p_k back
// from cg.pnew.
template <int PHYS, class N, int EX, int EY, int MINB>
__global__ void __launch_bounds__(EX *EY, MINB)
    march_apply_cg(TileArgs g, CgFuse cg, typename N::IO *__restrict__ y, const int *__restrict__ skip,
                   double *__restrict__ partials, unsigned int *ticket, double *out) {
  __shared__ MarchSmem<phys_ndpn(PHYS), N, EX, EY> sm;
  __shared__ double sab[2];
  extern __shared__ __align__(16) double cg_raw[];
  if (skip && *skip) return;
  if (threadIdx.x < 2) sab[threadIdx.x] = cg.ab[threadIdx.x];  // visible after march_pass's first barrier
  dwa::MagRec mag;
  const double d = march_pass<PHYS, N, EX, EY, true, true, false, true>(g, blockIdx.x, 0, cg.pnew, y, sm, 0, 0, mag,
                                                                         &cg, cg_raw, sab);
  if (dwa::mag_outside(mag.key)) atomicOr(g.flags + blockIdx.x, g.bit);
  ordered_dot_sum<EX * EY>(d, partials, blockIdx.x, gridDim.x, ticket, out, true);
}

// Dynamic shared memory of march_apply_cg: two buffers of (3 or 4) arrays of a plane's values, and
// the ring of 4 planes of owned p_k.
template <int PHYS, int EX, int EY>
constexpr size_t cg_raw_bytes(bool jacobi) {
  return sizeof(double) * (2 * (jacobi ? 4 : 3) * (EX + 1) * (EY + 1) + 4 * EX * EY) * phys_ndpn(PHYS);
}

// Largest input magnitude record of a work item (the inputs its CTA stages, Dirichlet entries
// excluded), over the whole CTA (all threads call it and receive it).
template <int PHYS, class N, int EX, int EY>
__device__ unsigned march_prescan(const TileArgs &g, int item, int64_t rr, const typename N::IO *__restrict__ x,
                                  unsigned *slot) {
  constexpr int NC = phys_ndpn(PHYS), NT = EX * EY, PX = EX + 1, NP = (EX + 1) * (EY + 1);
  const int bx = item % g.tiles_x, by = (item / g.tiles_x) % g.tiles_y, bz = item / (g.tiles_x * g.tiles_y);
  const int i0 = bx * (EX - 1), j0 = by * (EY - 1), NXP = g.nx + 1, NYP = g.ny + 1;
  const int k0 = bz * g.seg, k1 = min(k0 + g.seg, g.nz + 1);
  const int plo = max(k0 - 1, 0), phi = min(k1, g.nz);
  const int64_t NPL = (int64_t)NXP * NYP;
  dwa::MagRec mag;
  for (int p = threadIdx.x; p < NP; p += NT) {
    const int ix = i0 - 1 + p % PX, iy = j0 - 1 + p / PX;
    if (ix < 0 || ix >= NXP || iy < 0 || iy >= NYP) continue;
    for (int k = plo; k <= phi; ++k) {
      const int64_t node = ix + NXP * iy + (int64_t)k * NPL;
      if (__ldg(g.dmask + node)) continue;
#pragma unroll
      for (int c = 0; c < NC; ++c) mag.add(__ldg(x + (node * g.nrhs + rr) * NC + c));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *slot = 0u;
  __syncthreads();
  const unsigned w = __reduce_max_sync(0xffffffffu, mag.key);
  if ((threadIdx.x & 31) == 0) atomicMax(slot, w);
  __syncthreads();
  return *slot;
}

// Fix-up after march_apply / march_apply_dot (n_cta CTAs, the flags of this launch's bit): every
// flagged work item whose CTA-wide largest input lies outside the double-word window is computed
// again with its inputs scaled into [1, 2) and y scaled back (with the mesh's output scaling on a
// normalised mesh).  Each flag bit is cleared as it is read.  With DOT
// the recomputed items' parts are stored and, if any changed, the dot product is summed again in CTA
// order by the last CTA of this launch.  Persistent: CTAs loop over the items.
// ctl: two words of the mesh (ctl[0]: some part changed, ctl[1]: ticket of this kernel), zero between
// launches.
template <int PHYS, class N, int EX, int EY, bool DOT>
__global__ void __launch_bounds__(EX *EY) march_fixup(TileArgs g, const typename N::IO *__restrict__ x,
                                                          typename N::IO *__restrict__ y, const int *__restrict__ skip,
                                                          int n_cta, double *__restrict__ partials, unsigned int *ctl,
                                                          double *out) {
  __shared__ MarchSmem<phys_ndpn(PHYS), N, EX, EY> sm;
  __shared__ unsigned todo, mslot;
  __shared__ int changed;
  constexpr bool IS_DW = std::is_same<N, tile::NumDW>::value;
  if (skip && *skip) return;
  if (threadIdx.x == 0) changed = 0;
  // quick exit: one plain load per thread over this CTA's items (the usual case: nothing flagged)
  bool mine = false;
  for (int c = blockIdx.x + (int)threadIdx.x * (int)gridDim.x; c < n_cta; c += EX * EY * (int)gridDim.x)
    mine |= IS_DW && (__ldcg(g.flags + c) & g.bit) != 0u;
  const bool some = __syncthreads_or(mine) != 0;
  for (int c = blockIdx.x; some && c < n_cta; c += gridDim.x) {
    __syncthreads();
    if (threadIdx.x == 0) todo = IS_DW ? (atomicAnd(g.flags + c, ~g.bit) & g.bit) : 0u;
    __syncthreads();
    if (!todo) continue;
    const int item = DOT ? c : c / g.nrhs;
    const int64_t rr = DOT ? g.r0 : g.r0 + c % g.nrhs;
    int sc = 0;
    if constexpr (IS_DW) {
      int s = 0;
      if (dwa::mag_exponent(march_prescan<PHYS, N, EX, EY>(g, item, rr, x, &mslot), s) &&
          (s < dwa::kMagLo || s > dwa::kMagHi))
        sc = s;
      else
        continue;  // the first pass was within the window after all
    }
    dwa::MagRec mag;
    const double d = march_pass<PHYS, N, EX, EY, false, DOT, true>(g, item, rr, x, y, sm, sc, g.oscale + sc, mag);
    if constexpr (DOT) {
      double t = d;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
      __shared__ double red[EX * EY / 32];
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
      __syncthreads();
      if (threadIdx.x == 0) {
        double u = 0.0;
        for (int i = 0; i < EX * EY / 32; ++i) u += red[i];
        partials[c] = u;
        changed = 1;
      }
    }
  }
  if constexpr (DOT) {
    __syncthreads();
    __shared__ int last;
    // every CTA reports whether it changed a part; the last one to arrive sums again if any did
    if (threadIdx.x == 0) {
      if (changed) atomicOr(ctl, 1u);
      __threadfence();
      last = atomicAdd(ctl + 1, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const bool any = __ldcg(ctl) != 0u;
    if (any) {
      constexpr int NT = EX * EY, NW = NT / 32;
      __shared__ double red2[NW];
      double s = 0.0;
      for (int i = threadIdx.x; i < n_cta; i += NT) s += __ldcg(partials + i);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if ((threadIdx.x & 31) == 0) red2[threadIdx.x >> 5] = s;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < NW; ++i) t += red2[i];
        *out = t;
      }
    }
    if (threadIdx.x == 0) {
      ctl[0] = 0u;
      ctl[1] = 0u;
    }
  }
}

// Launch shapes: EX = 32 element columns per warp row, EY rows, MINB resident CTAs per SM.
// Double-word elasticity takes 12 rows at 168 registers (12 warps per SM, halo factor 1.13): at 8
// rows it needed 241 registers and ran 8 warps per SM, 17 % slower at 160^3.  FP32 elasticity keeps
// 8 rows, where it is fastest.  Two element rows per thread (x-butterflies of shared node rows
// formed once, y-sums between them in registers) were measured slower for the double-word Laplace
// apply at 256^3: 0.52-0.58 ms on 32x8, 32x12 and 32x16 tiles against 0.50 ms with one row per
// thread on 32x8 tiles at 4 CTAs per SM (half the warps hide less latency).
template <int PHYS, class N> struct MarchShape { static constexpr int EX = 32, EY = 8, MINB = 4; };
template <class N> struct MarchShape<MF_ELASTICITY, N> { static constexpr int EX = 32, EY = 8, MINB = 1; };
template <> struct MarchShape<MF_ELASTICITY, tile::NumDW> { static constexpr int EX = 32, EY = 12, MINB = 1; };
template <class N> struct MarchShape<MF_VECTOR_LAPLACE, N> { static constexpr int EX = 32, EY = 8, MINB = 2; };

}  // namespace march
