// Setup of the tensor-product geometry and launch of the face-marching apply (single and
// multi-RHS; the kernels live in mf_march.cuh and mf_tile.cuh).
#include <algorithm>
#include <atomic>

#include "mf_march.cuh"
#include "mf_tile.cuh"

using namespace tile;
using dwa::dw;

namespace {

// ------------------------------------------------------------------------------------ setup ----
// Tensor-product check: every node's x depends on i only, y on j only, z on k only.
__global__ void tp_check(const double *X, int nx, int ny, int nz, int *not_tp) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t N = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  if (n >= N) return;
  const int i = (int)(n % (nx + 1));
  const int j = (int)((n / (nx + 1)) % (ny + 1));
  const int k = (int)(n / ((int64_t)(nx + 1) * (ny + 1)));
  const double xr = X[3 * (int64_t)i];
  const double yr = X[3 * (int64_t)(nx + 1) * j + 1];
  const double zr = X[3 * (int64_t)(nx + 1) * (ny + 1) * k + 2];
  if (X[3 * n] != xr || X[3 * n + 1] != yr || X[3 * n + 2] != zr) atomicOr(not_tp, 1);
}

// Spacing h and 1/h of every cell along each axis, as (hi, lo) pairs.
__global__ void tp_axes(const double *X, int nx, int ny, int nz, double geo, float2 *out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = nx + ny + nz;
  if (t >= n) return;
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
  const double h = (b - a) * geo;  // normalised spacing (geo is a power of two)
  const dw hh = dwa::from_double_slow(h), ih = dwa::from_double_slow(1.0 / h);
  out[t] = make_float2(hh.h, hh.l);
  out[n + t] = make_float2(ih.h, ih.l);
}

__global__ void mat_pairs(const double *m, int64_t n, double scale, float2 *out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const dw v = dwa::from_double_slow(m[i] * scale);  // normalised cell constant (scale: power of two)
  out[i] = make_float2(v.h, v.l);
}

}  // namespace

mf_status tile_setup(mf_mesh *m, cudaStream_t s) {
  m->tp = false;
  if (!m->structured) return MF_OK;
  int *flag = nullptr;
  MF_CUDA(cudaMalloc(&flag, sizeof(int)));
  MF_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
  tp_check<<<blocks_for(m->n_nodes), kThreads, 0, s>>>(m->X, m->nx, m->ny, m->nz, flag);
  int h = 1;
  MF_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  MF_CUDA(cudaStreamSynchronize(s));
  cudaFree(flag);
  if (h) return MF_OK;
  const int n = m->nx + m->ny + m->nz;
  MF_CUDA(cudaMalloc(&m->tp_axis, 2 * n * sizeof(float2)));
  tp_axes<<<blocks_for(n), kThreads, 0, s>>>(m->X, m->nx, m->ny, m->nz, m->dw_geo, m->tp_axis);
  const int64_t nm = m->n_cells * phys_nmat(m->physics);
  MF_CUDA(cudaMalloc(&m->mat_pairs, nm * sizeof(float2)));
  mat_pairs<<<blocks_for(nm), kThreads, 0, s>>>(m->mat, nm, m->dw_mat, m->mat_pairs);
  // range flags: 2 control words + one word per CTA of the largest launch (z-segments of one
  // plane, 16 right-hand sides)
  const int64_t nflags = 2 + 16 * tile_dot_slots(m);
  MF_CUDA(cudaMalloc(&m->tp_flags, nflags * sizeof(unsigned)));
  MF_CUDA(cudaMemsetAsync(m->tp_flags, 0, nflags * sizeof(unsigned), s));
  MF_CUDA(cudaGetLastError());
  MF_CUDA(cudaStreamSynchronize(s));
  m->tp = true;
  return MF_OK;
}

// The fix-up kernel of the range check (mf_march.cuh), right after a double-word face-marching
// launch of n_cta CTAs (it reads the flags and returns quickly when none is set; FP32 launches have no
// range check).  Persistent grid.
template <int PHYS, class N, bool DOT>
static mf_status fixup_launch(const mf_mesh *m, const TileArgs &g, const typename N::IO *x, typename N::IO *y,
                              cudaStream_t s, const int *skip, int n_cta, double *partials, double *out) {
  if (!std::is_same<N, NumDW>::value) return MF_OK;
  using MS = march::MarchShape<PHYS, N>;
  constexpr int NT = MS::EX * MS::EY;
  auto kern = march::march_fixup<PHYS, N, MS::EX, MS::EY, DOT>;
  // one CTA per SM: enough for the rare items to redo, and a short scan of the flags otherwise
  const int grid = std::max(1, std::min(n_cta, device_sm_count()));
  mf_count_launches(1);
  kern<<<grid, NT, 0, s>>>(g, x, y, skip, n_cta, partials, m->tp_flags, out);
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

// The face-marching kernels (mf_march.cuh): one launch for `nrhs` right-hand sides of
// [node][rhs][comp] vectors (CTA = work item x nrhs + right-hand side).
template <int PHYS, class N>
static mf_status march_launch(const mf_mesh *m, const typename N::IO *x, typename N::IO *y, cudaStream_t s,
                              const int *skip, int nrhs = 1) {
  using MS = march::MarchShape<PHYS, N>;
  constexpr int NT = MS::EX * MS::EY;
  auto kern0 = march::march_apply<PHYS, N, MS::EX, MS::EY, MS::MINB, false>;
  auto kern = m->dw_oscale != 0 ? march::march_apply<PHYS, N, MS::EX, MS::EY, MS::MINB, true> : kern0;
  static std::atomic<int> resident{0};  // CTAs per SM: a property of the kernel, same for every caller
  if (resident.load() == 0) {
    int r = 0;
    MF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, kern0, NT, 0));
    resident.store(std::max(r, 1));
  }
  TileArgs g = make_tile_args(m, MS::EX, MS::EY, m->tile_seg, resident.load(), nrhs);
  g.nrhs = nrhs;
  g.r0 = 0;
  g.flags = m->tp_flags + 2;
  g.bit = 1u << (m->tp_epoch.fetch_add(1u) & 31u);
  const int n_cta = tile_items(g) * nrhs;
  kern<<<n_cta, NT, 0, s>>>(g, x, y, skip);
  MF_TRY((fixup_launch<PHYS, N, false>(m, g, x, y, s, skip, n_cta, nullptr, nullptr)));
  return MF_OK;
}

template <class N>
static mf_status tile_launch(const mf_mesh *m, const typename N::IO *x, typename N::IO *y, cudaStream_t s,
                             const int *skip) {
  mf_count_launches(1);
  if (m->physics == MF_LAPLACE) MF_TRY((march_launch<MF_LAPLACE, N>(m, x, y, s, skip)));
  else if (m->physics == MF_VECTOR_LAPLACE) MF_TRY((march_launch<MF_VECTOR_LAPLACE, N>(m, x, y, s, skip)));
  else MF_TRY((march_launch<MF_ELASTICITY, N>(m, x, y, s, skip)));
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

// Resident CTAs per SM of the fused-dot apply.  Its work decomposition (z-segments from the wave
// model) is also that of the fused CG apply, so that both sum p . Ap over the same CTAs in the same
// order.
template <int PHYS, class N>
static mf_status dot_resident(int *out) {
  using MS = march::MarchShape<PHYS, N>;
  static std::atomic<int> resident{0};
  if (resident.load() == 0) {
    int r = 0;
    MF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &r, march::march_apply_dot<PHYS, N, MS::EX, MS::EY, MS::MINB>, MS::EX * MS::EY, 0));
    resident.store(std::max(r, 1));
  }
  *out = resident.load();
  return MF_OK;
}

// Apply with x . y fused (CG: p . Ap); partials needs one slot per CTA (tile_dot_slots).
template <int PHYS, class N>
static mf_status march_dot_launch(const mf_mesh *m, const typename N::IO *x, typename N::IO *y, cudaStream_t s,
                                  const int *skip, double *partials, unsigned int *ticket, double *out) {
  using MS = march::MarchShape<PHYS, N>;
  constexpr int NT = MS::EX * MS::EY;
  auto kern = m->dw_oscale != 0 ? march::march_apply_dot<PHYS, N, MS::EX, MS::EY, MS::MINB, true>
                                 : march::march_apply_dot<PHYS, N, MS::EX, MS::EY, MS::MINB, false>;
  int resident = 0;
  MF_TRY((dot_resident<PHYS, N>(&resident)));
  TileArgs g = make_tile_args(m, MS::EX, MS::EY, m->tile_seg, resident);
  g.flags = m->tp_flags + 2;
  g.bit = 1u << (m->tp_epoch.fetch_add(1u) & 31u);
  const int n_cta = tile_items(g);
  mf_count_launches(1);
  kern<<<n_cta, NT, 0, s>>>(g, x, y, skip, partials, ticket, out);
  MF_CUDA(cudaGetLastError());
  MF_TRY((fixup_launch<PHYS, N, true>(m, g, x, y, s, skip, n_cta, partials, out)));
  return MF_OK;
}

// At most one CTA per tile column and node plane (z-segments of one plane), for the FP64 and the
// FP32 launch shapes of the mesh's physics.
template <int PHYS>
static int64_t dot_slots(const mf_mesh *m) {
  auto tiles = [m](int EX, int EY) {
    return (int64_t)((m->nx + EX - 1) / (EX - 1)) * ((m->ny + EY - 1) / (EY - 1)) * (m->nz + 1);
  };
  using S64 = march::MarchShape<PHYS, NumDW>;
  using S32 = march::MarchShape<PHYS, NumF32>;
  return std::max(tiles(S64::EX, S64::EY), tiles(S32::EX, S32::EY));
}

int64_t tile_dot_slots(const mf_mesh *m) {
  if (m->physics == MF_LAPLACE) return dot_slots<MF_LAPLACE>(m);
  if (m->physics == MF_VECTOR_LAPLACE) return dot_slots<MF_VECTOR_LAPLACE>(m);
  return dot_slots<MF_ELASTICITY>(m);
}

template <class N>
static mf_status tile_apply_dot(const mf_mesh *m, const typename N::IO *x, typename N::IO *y, cudaStream_t s,
                                const int *skip, double *partials, unsigned int *ticket, double *out) {
  if (m->physics == MF_LAPLACE) return march_dot_launch<MF_LAPLACE, N>(m, x, y, s, skip, partials, ticket, out);
  if (m->physics == MF_VECTOR_LAPLACE)
    return march_dot_launch<MF_VECTOR_LAPLACE, N>(m, x, y, s, skip, partials, ticket, out);
  return march_dot_launch<MF_ELASTICITY, N>(m, x, y, s, skip, partials, ticket, out);
}

mf_status tile_apply_dot_fp64(const mf_mesh *m, const double *x, double *y, cudaStream_t s, const int *skip,
                              double *partials, unsigned int *ticket, double *out) {
  return tile_apply_dot<NumDW>(m, x, y, s, skip, partials, ticket, out);
}

mf_status tile_apply_dot_fp32(const mf_mesh *m, const float *x, float *y, cudaStream_t s, const int *skip,
                              double *partials, unsigned int *ticket, double *out) {
  return tile_apply_dot<NumF32>(m, x, y, s, skip, partials, ticket, out);
}

// One classic CG iteration's apply with the p and x updates fused in (march_apply_cg), then the
// fix-up kernel of the range check on p_k's buffer.
template <int PHYS>
static mf_status march_cg_launch(const mf_mesh *m, const march::CgFuse &cg, double *y, cudaStream_t s, const int *skip,
                                 double *partials, unsigned int *ticket, double *out) {
  using MS = march::MarchShape<PHYS, NumDW>;
  constexpr int NT = MS::EX * MS::EY;
  auto kern = march::march_apply_cg<PHYS, NumDW, MS::EX, MS::EY, MS::MINB>;
  const size_t dyn = march::cg_raw_bytes<PHYS, MS::EX, MS::EY>(cg.invd != nullptr);
  static std::atomic<bool> ready{false};
  if (!ready.load()) {
    MF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)march::cg_raw_bytes<PHYS, MS::EX, MS::EY>(true)));
    ready.store(true);  // the shared-memory carveout is left to the driver: L1 keeps the rest
  }
  int resident = 0;
  MF_TRY((dot_resident<PHYS, NumDW>(&resident)));
  TileArgs g = make_tile_args(m, MS::EX, MS::EY, m->tile_seg, resident);
  g.flags = m->tp_flags + 2;
  g.bit = 1u << (m->tp_epoch.fetch_add(1u) & 31u);
  const int n_cta = tile_items(g);
  mf_count_launches(1);
  kern<<<n_cta, NT, dyn, s>>>(g, cg, y, skip, partials, ticket, out);
  MF_CUDA(cudaGetLastError());
  MF_TRY((fixup_launch<PHYS, NumDW, true>(m, g, cg.pnew, y, s, skip, n_cta, partials, out)));
  return MF_OK;
}

mf_status tile_apply_cg_fp64(const mf_mesh *m, const double *r, const double *pold, const double *invd, double *pnew,
                             double *x, double *y, const double *alpha_beta, cudaStream_t s, const int *skip,
                             double *partials, unsigned int *ticket, double *out) {
  if (m->dw_oscale != 0) {
    mf_set_error("internal: the fused CG apply needs an unscaled mesh");
    return MF_ERR_UNSUPPORTED;
  }
  const march::CgFuse cg{r, pold, invd, pnew, x, alpha_beta};
  if (m->physics == MF_LAPLACE) return march_cg_launch<MF_LAPLACE>(m, cg, y, s, skip, partials, ticket, out);
  if (m->physics == MF_VECTOR_LAPLACE)
    return march_cg_launch<MF_VECTOR_LAPLACE>(m, cg, y, s, skip, partials, ticket, out);
  return march_cg_launch<MF_ELASTICITY>(m, cg, y, s, skip, partials, ticket, out);
}

// Multi right-hand-side apply on [node][rhs][comp] vectors: one face-marching launch over all
// right-hand sides; every column is computed exactly as by the single apply.
mf_status tile_apply_multi_fp64(const mf_mesh *m, int nrhs, const double *x, double *y, cudaStream_t s) {
  mf_count_launches(1);
  if (m->physics == MF_LAPLACE) MF_TRY((march_launch<MF_LAPLACE, NumDW>(m, x, y, s, nullptr, nrhs)));
  else if (m->physics == MF_VECTOR_LAPLACE) MF_TRY((march_launch<MF_VECTOR_LAPLACE, NumDW>(m, x, y, s, nullptr, nrhs)));
  else MF_TRY((march_launch<MF_ELASTICITY, NumDW>(m, x, y, s, nullptr, nrhs)));
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

mf_status tile_apply_fp64(const mf_mesh *m, const double *x, double *y, cudaStream_t s, const int *skip) {
  return tile_launch<NumDW>(m, x, y, s, skip);
}

mf_status tile_apply_fp32(const mf_mesh *m, const float *x, float *y, cudaStream_t s, const int *skip) {
  return tile_launch<NumF32>(m, x, y, s, skip);
}

MF_DBG_TU(tile)
