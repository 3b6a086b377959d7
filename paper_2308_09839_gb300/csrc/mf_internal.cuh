// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "mf.h"

// NVTX range around a library call: Nsight tools show the C-ABI calls (setup, apply, CSR, CG and its
// graph blocks, network calls) on the timeline.  Without a tool attached a push or pop is a check of
// a null function pointer.
struct MfRange {
  explicit MfRange(const char *name) { nvtxRangePushA(name); }
  ~MfRange() { nvtxRangePop(); }
  MfRange(const MfRange &) = delete;
  MfRange &operator=(const MfRange &) = delete;
};
#define MF_RANGE(name) MfRange mf_range_scope_(name)

// Physics traits: DoFs per node, cell constants per cell, and whether the element arithmetic is the
// scalar Laplace one (applied to each component for the vector Laplacian of Eq. 5).
__host__ __device__ constexpr int phys_ndpn(int p) { return p == MF_LAPLACE ? 1 : 3; }
__host__ __device__ constexpr int phys_nmat(int p) { return p == MF_ELASTICITY ? 2 : 1; }
__host__ __device__ constexpr bool phys_is_laplace(int p) { return p != MF_ELASTICITY; }

// ------------------------------------------------------------------------------------ errors ----
void mf_set_error(const char *fmt, ...);
void mf_clear_error();

#define MF_CUDA(call)                                                                            \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) {                                                                     \
      mf_set_error("%s:%d: %s failed: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_));   \
      return e_ == cudaErrorMemoryAllocation ? MF_ERR_OOM : MF_ERR_CUDA;                         \
    }                                                                                            \
  } while (0)

#define MF_TRY(expr)                  \
  do {                                \
    mf_status s_ = (expr);            \
    if (s_ != MF_OK) return s_;       \
  } while (0)

#define MF_ARG(cond, ...)             \
  do {                                \
    if (!(cond)) {                    \
      mf_set_error(__VA_ARGS__);      \
      return MF_ERR_ARG;              \
    }                                 \
  } while (0)

// Kernel-launch accounting (mf_kernel_launches): every host function that launches kernels adds
// the number it launched.
void mf_count_launches(int64_t n);
int64_t mf_launches_now();

// ------------------------------------------------------------------- bounds-checked builds ----
// Built with -DMF_DEBUG_BOUNDS (`python -m paper_2308_09839_gb300.build --debug` makes libmf_debug.so)
// the index checks of the kernels are compiled in: mf_dbg_index(i, n, bit) returns i when
// 0 <= i < n and otherwise sets `bit` in this translation unit's status word and returns 0, an index
// inside every buffer it is used on, so the kernel finishes without touching memory outside its
// buffers (its results are then meaningless and the status says so).  mf_debug_status gathers and
// clears the words of all translation units.  Release builds compile the checks to nothing.
enum : unsigned { MF_DBG_NODE = 1u, MF_DBG_CELL = 2u, MF_DBG_COLUMN = 4u };
#ifdef MF_DEBUG_BOUNDS
static __device__ unsigned mf_dbg_word;
template <typename I>
__device__ __forceinline__ I mf_dbg_index(I i, I n, unsigned bit) {
  if (i >= 0 && i < n) return i;
  atomicOr(&mf_dbg_word, bit);
  return (I)0;
}
#define MF_DBG_TU(name)                                                   \
  unsigned mf_dbg_take_##name() {                                         \
    unsigned h = 0u;                                                      \
    const unsigned z = 0u;                                                \
    if (cudaMemcpyFromSymbol(&h, mf_dbg_word, sizeof h) != cudaSuccess) h = ~0u; \
    cudaMemcpyToSymbol(mf_dbg_word, &z, sizeof z);                        \
    return h;                                                             \
  }
#else
template <typename I>
__device__ __forceinline__ I mf_dbg_index(I i, I, unsigned) {
  return i;
}
#define MF_DBG_TU(name) \
  unsigned mf_dbg_take_##name() { return 0u; }
#endif
// pointer p into the buffer [base, base + n), checked like mf_dbg_index (release builds: p itself)
#ifdef MF_DEBUG_BOUNDS
#define MF_DBG_PTR(p, base, n, bit) ((base) + mf_dbg_index((int64_t)((p) - (base)), (int64_t)(n), (bit)))
#else
#define MF_DBG_PTR(p, base, n, bit) (p)
#endif
unsigned mf_dbg_take_apply();
unsigned mf_dbg_take_tile();
unsigned mf_dbg_take_cg();
unsigned mf_dbg_take_batched();
unsigned mf_dbg_take_general();
unsigned mf_dbg_take_csr();

// ------------------------------------------------------------------------- device geometry ----
// Plain view of a mesh, passed by value to kernels.
struct MeshView {
  const double *X;     // [N][3] node coordinates
  const float *X32;    // [N][3] FP32 copy
  const int32_t *cells;  // [E][8] ([E][4] for tetrahedra), null for structured boxes
  const double *mat;   // Laplace: kappa[E]; elasticity: (lam, mu)[E][2]
  const float *mat32;  // FP32 copy of mat
  const uint8_t *dmask;  // [N] Dirichlet mask (never null: zero-filled when unconstrained)
  int32_t nx, ny, nz;
  int64_t n_nodes, n_cells;
};

// Template accessors for the real type.
template <typename Real> __device__ __forceinline__ const Real *coords_of(const MeshView &m);
template <> __device__ __forceinline__ const double *coords_of<double>(const MeshView &m) { return m.X; }
template <> __device__ __forceinline__ const float *coords_of<float>(const MeshView &m) { return m.X32; }
template <typename Real> __device__ __forceinline__ const Real *mat_of(const MeshView &m);
template <> __device__ __forceinline__ const double *mat_of<double>(const MeshView &m) { return m.mat; }
template <> __device__ __forceinline__ const float *mat_of<float>(const MeshView &m) { return m.mat32; }

// Structured box: node id of element e's corner a.
__host__ __device__ __forceinline__ int64_t box_corner_node(int64_t e, int a, int nx, int ny) {
  int64_t ex = e % nx;
  int64_t t = e / nx;
  int64_t ey = t % ny;
  int64_t ez = t / ny;
  return (ex + (a & 1)) + (int64_t)(nx + 1) * ((ey + ((a >> 1) & 1)) + (int64_t)(ny + 1) * (ez + ((a >> 2) & 1)));
}

__device__ __forceinline__ void element_nodes(const MeshView &m, int64_t e, int64_t nodes[8]) {
  if (m.cells) {
    const int4 *c4 = reinterpret_cast<const int4 *>(m.cells + 8 * e);
    int4 lo = __ldg(c4), hi = __ldg(c4 + 1);
    nodes[0] = lo.x; nodes[1] = lo.y; nodes[2] = lo.z; nodes[3] = lo.w;
    nodes[4] = hi.x; nodes[5] = hi.y; nodes[6] = hi.z; nodes[7] = hi.w;
  } else {
    int64_t base = box_corner_node(e, 0, m.nx, m.ny);
    const int64_t sx = 1, sy = m.nx + 1, sz = (int64_t)(m.nx + 1) * (m.ny + 1);
#pragma unroll
    for (int a = 0; a < 8; ++a) nodes[a] = base + (a & 1) * sx + ((a >> 1) & 1) * sy + ((a >> 2) & 1) * sz;
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) nodes[a] = mf_dbg_index(nodes[a], m.n_nodes, MF_DBG_NODE);
}

// node a of element e of an explicit connectivity with npe nodes per element (checked in
// bounds-checked builds)
__device__ __forceinline__ int64_t cell_node(const MeshView &m, int npe, int64_t e, int a) {
  return mf_dbg_index((int64_t)__ldg(m.cells + (int64_t)npe * e + a), m.n_nodes, MF_DBG_NODE);
}

// -------------------------------------------------------------------------------- the mesh ----
struct CgWorkspace;

struct mf_mesh {
  int physics = 0;
  int ndpn = 1;
  int device = 0;
  int variant = MF_VARIANT_AUTO;
  int64_t n_nodes = 0, n_cells = 0, n_dof = 0, n_free = 0;
  int npe = 8;  // nodes per element: 8 (Q1 hexahedron) or 4 (P1 tetrahedron, explicit cells only)
  bool structured = false;
  bool all_affine = false;
  int32_t nx = 0, ny = 0, nz = 0;
  // owned device buffers
  double *X = nullptr;
  float *X32 = nullptr;
  int32_t *cells = nullptr;
  double *mat = nullptr;   // kappa or (lam, mu)
  float *mat32 = nullptr;
  uint8_t *dmask = nullptr;
  int32_t *dnodes = nullptr;  // Dirichlet node list
  int64_t n_dnodes = 0;
  // element colouring (unstructured): colour c holds colour_elems[colour_off[c] .. colour_off[c+1])
  int n_colours = 0;
  std::vector<int64_t> colour_off;
  int32_t *colour_elems = nullptr;
  // solver workspace (created lazily by mf_cg_solve)
  CgWorkspace *cg = nullptr;
  // host copy of the connectivity used by CSR assembly (empty for structured meshes)
  std::vector<int32_t> h_cells;
  // tensor-product geometry (structured boxes of axis-aligned cells): per-axis spacings and their
  // inverses as (hi, lo) float pairs [hx | hy | hz | 1/hx | 1/hy | 1/hz], and the cell constants
  // as pairs; enables the FP64-accurate tile kernels of mf_tile.cu
  bool tp = false;
  // Range of the double-word kernels (tensor-product, general and partial-assembly).  At setup the
  // cell constants are scaled by dw_mat = 2^-s_k and the coordinates by dw_geo = 2^-s_h (powers of
  // two, exact) when their magnitudes lie outside the window the double-word arithmetic covers; the
  // kernels then evaluate 2^-(s_k + s_h) A and scale y by 2^dw_oscale.  dw_ok is false when the
  // constants or the cell sizes span more than that arithmetic covers: the double-word data are not
  // built and every apply runs the FP64 reference kernel.
  bool dw_ok = true;
  int dw_oscale = 0;
  // per-CTA range flags of the face-marching launches (tile_flag_words entries; see mf_march.cuh) and
  // the launch counter whose low 5 bits pick each launch's flag bit
  unsigned *tp_flags = nullptr;
  mutable std::atomic<unsigned> tp_epoch{0};
  double dw_mat = 1.0, dw_geo = 1.0;
  int tile_seg = 0;  // z-segment length of the tile kernels (0: heuristic; set by the autotuner)
  // general structured geometry (structured boxes that are not tensor-product grids): half
  // spacings of the base grid [hx/2 | hy/2 | hz/2] and node offsets from it, as float pairs;
  // enables the FP64-accurate general tile kernels of mf_general.cu
  bool gen = false;
  float2 *gen_axis = nullptr;
  float2 *gen_delta = nullptr;
  float2 *tp_axis = nullptr;
  float2 *mat_pairs = nullptr;
  // partial assembly of the general structured geometry (Table 3): per quadrature point the flux
  // matrix (Laplace, 6 values) or adj(J) and 1/det J (elasticity, 10 values), as float pairs and as
  // floats, [q][k][cell]; built when it fits the device (auto variant) or on request
  float2 *pa = nullptr;
  float *pa32 = nullptr;
  // partial assembly of Q2 meshes, per Gauss point: Laplace the flux matrix (6 values, FP64,
  // [q][k][cell]); elasticity J^-1 and w det J (lambda, mu) (11 values, [cell][k][32]), FP64 or, when
  // q2dw, as float pairs normalised by 2^-q2sk (J^-1) and 2^-q2ss (the rest), in place
  double *q2pa = nullptr;
  bool q2dw = false;
  int q2sk = 0, q2ss = 0;
  int64_t *q2off = nullptr;   // node -> slot lists of the element outputs (CSR form, N + 1)
  int32_t *q2slots = nullptr; // slots 27 e + a, per node sorted by element
  double *q2buf = nullptr;    // element outputs [E][27][ndpn]

  MeshView view() const {
    MeshView v;
    v.X = X; v.X32 = X32; v.cells = cells; v.mat = mat; v.mat32 = mat32; v.dmask = dmask;
    v.nx = nx; v.ny = ny; v.nz = nz; v.n_nodes = n_nodes; v.n_cells = n_cells;
    return v;
  }
};

struct mf_csr {
  uint64_t id = 0;  // unique per assembled matrix in the process (never reused): keys cached solver graphs
  int64_t n_rows = 0, nnz = 0;
  int64_t *rowptr = nullptr;
  int32_t *col = nullptr;
  double *val = nullptr;
  int64_t max_row = 0;  // longest row (entries): chooses the SpMV kernel shape
};

// --------------------------------------------------------------------- internal entry points ----
// Operator apply on `stream` (FP64).  Picks the variant; x and y are DoF vectors.
// `skip` (device int, may be null): when it holds a nonzero value at run time every kernel of the
// apply returns immediately (used by solver loops captured in CUDA graphs after convergence).
mf_status apply_fp64(const mf_mesh *m, const double *x, double *y, cudaStream_t s, const int *skip = nullptr);
mf_status apply_fp32(const mf_mesh *m, const float *x, float *y, cudaStream_t s, const int *skip = nullptr);
mf_status apply_multi_fp64(const mf_mesh *m, int nrhs, const double *x, double *y, cudaStream_t s);
mf_status spmv(const mf_csr *A, const double *x, double *y, cudaStream_t s, const int *skip = nullptr);
// tensor-product tile kernels (mf_tile.cu)
mf_status tile_setup(mf_mesh *m, cudaStream_t s);
mf_status tile_apply_fp64(const mf_mesh *m, const double *x, double *y, cudaStream_t s, const int *skip);
mf_status tile_apply_fp32(const mf_mesh *m, const float *x, float *y, cudaStream_t s, const int *skip);
// tensor-product apply with x . y fused into its write phase (*out, deterministic); partials needs
// tile_dot_slots(m) entries, ticket a zeroed counter
int64_t tile_dot_slots(const mf_mesh *m);
mf_status tile_apply_dot_fp64(const mf_mesh *m, const double *x, double *y, cudaStream_t s, const int *skip,
                              double *partials, unsigned int *ticket, double *out);
mf_status tile_apply_dot_fp32(const mf_mesh *m, const float *x, float *y, cudaStream_t s, const int *skip,
                              double *partials, unsigned int *ticket, double *out);
// One classic CG iteration's apply with the updates of p (from r and p_{k-1}) and x fused in; y = A p_k
// and p_k . A p_k in *out (tensor-product meshes with the auto variant, unscaled).
mf_status tile_apply_cg_fp64(const mf_mesh *m, const double *r, const double *pold, const double *invd, double *pnew,
                             double *x, double *y, const double *alpha_beta, cudaStream_t s, const int *skip,
                             double *partials, unsigned int *ticket, double *out);
mf_status tile_apply_multi_fp64(const mf_mesh *m, int nrhs, const double *x, double *y, cudaStream_t s);
// general structured kernels (mf_general.cu)
mf_status gen_setup(mf_mesh *m, cudaStream_t s);
mf_status pa_setup(mf_mesh *m, cudaStream_t s);
mf_status q2_pa_setup(mf_mesh *m, cudaStream_t s);  // mf_apply.cu
size_t q2_pa_bytes(int physics, int64_t n_cells);  // mf_apply.cu: bytes of the Q2 partial assembly
mf_status gen_apply_fp64(const mf_mesh *m, const double *x, double *y, cudaStream_t s, const int *skip);
mf_status gen_apply_fp32(const mf_mesh *m, const float *x, float *y, cudaStream_t s, const int *skip);
// diag(A) of the matrix-free operator (Jacobi), FP64, Dirichlet rows 1.
mf_status operator_diagonal(const mf_mesh *m, double *diag, cudaStream_t s);
void cg_workspace_free(CgWorkspace *w);

// Number of SMs of the current device (cached per device; 152 on GB300).  Sizes persistent grids
// and the wave model of the tile kernels; the reductions whose order must not depend on the GPU use
// fixed grids instead.
int device_sm_count();

// Forward 3x3x3 convolution of a channels-last BF16 input stored with cin_stride >= cin channels per
// voxel, on the tensor-core path (mf_nn.cu); MF_ERR_UNSUPPORTED when that path cannot run it.
mf_status conv3d_fwd_strided(const void *x, int nx, int ny, int nz, int cin, int cin_stride, const void *w,
                             const float *bias, int cout, const void *skip, int relu, void *y_bf16, float *y_f32,
                             cudaStream_t stream);

// number of element colours and the launch grid for one colour
int64_t colour_count(const mf_mesh *m, int c);

constexpr int kThreads = 256;
inline unsigned blocks_for(int64_t n, int threads = kThreads) {
  int64_t b = (n + threads - 1) / threads;
  return (unsigned)(b < 1 ? 1 : b);
}
