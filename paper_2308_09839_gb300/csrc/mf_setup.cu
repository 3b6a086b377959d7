// Mesh setup (inputs of Algorithm 1 and the cell constants of Table 2): validation, material
// conversion, Dirichlet list, element colouring for the atomic-free scatter, error reporting.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <numeric>

#include "mf_element.cuh"
#include "mf_internal.cuh"
#include "mf_q2.cuh"
#include "mf_tet.cuh"

// ------------------------------------------------------------------------------------ errors ----
static thread_local char g_err[1024] = "";

void mf_set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
void mf_clear_error() { g_err[0] = 0; }

extern "C" const char *mf_last_error(void) { return g_err; }
extern "C" const char *mf_version(void) { return "mf-gb300 0.1 (sm_103a)"; }

static std::atomic<int64_t> g_launches{0};
void mf_count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t mf_launches_now() { return g_launches.load(std::memory_order_relaxed); }
extern "C" int64_t mf_kernel_launches(void) { return mf_launches_now(); }

int device_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  int n = cache[dev].load();
  if (n == 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    cache[dev].store(n);
  }
  return n;
}

// ------------------------------------------------------------------------- setup kernels ----
enum : int { BAD_DET = 1, BAD_NODE = 2, BAD_COORD = 4, BAD_MAT = 8 };

struct ValidateOut {
  int flags;
  int not_affine;     // set if any cell is not a parallelepiped
  long long first_bad;  // smallest element index with a problem
  unsigned long long det_max, det_min;  // bit patterns of the largest and smallest det J (positive)
};

// det J at the 8 Gauss points and the 8 corners must be positive and finite; node ids in range;
// material finite and admissible.  Also records whether every cell is affine (x(xi) has no
// bilinear or trilinear terms), in which case J is constant over the cell.
__global__ void validate_kernel(MeshView m, int physics, ValidateOut *out) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.n_cells) return;
  int flags = 0;
  int64_t nodes[8];
  if (m.cells) {
    for (int a = 0; a < 8; ++a) {
      int32_t n = m.cells[8 * e + a];
      if (n < 0 || n >= m.n_nodes) flags |= BAD_NODE;
      nodes[a] = n;
    }
  } else {
    element_nodes(m, e, nodes);
  }
  if (!(flags & BAD_NODE)) {
    double X[8][3];
    for (int a = 0; a < 8; ++a)
      for (int i = 0; i < 3; ++i) {
        X[a][i] = m.X[3 * nodes[a] + i];
        if (!isfinite(X[a][i])) flags |= BAD_COORD;
      }
    if (!(flags & BAD_COORD)) {
      for (int p = 0; p < 16; ++p) {
        double xi[3];
        for (int d = 0; d < 3; ++d) xi[d] = q1::sgn(p & 7, d) * (p < 8 ? q1::kG : 1.0);
        double J[3][3], C[3][3];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int a = 0; a < 8; ++a) s += X[a][i] * q1::dN_at(xi, a, j);
            J[i][j] = s;
          }
        double det = q1::adjugate(J, C);
        if (!(det > 0.0) || !isfinite(det)) flags |= BAD_DET;
        if (p < 8 && det > 0.0 && isfinite(det)) {
          const unsigned long long bits = (unsigned long long)__double_as_longlong(det);
          atomicMax(&out->det_max, bits);
          atomicMin(&out->det_min, bits);
        }
      }
      // monomial coefficients of xi*eta, eta*zeta, xi*zeta, xi*eta*zeta in x(xi)
      double scale = 0;
      for (int i = 0; i < 3; ++i) scale = fmax(scale, fabs(X[7][i] - X[0][i]));
      bool affine = true;
      for (int mono = 3; mono < 7; ++mono) {
        int mask = (mono == 3) ? 3 : (mono == 4) ? 6 : (mono == 5) ? 5 : 7;
        for (int i = 0; i < 3; ++i) {
          double c = 0;
          for (int a = 0; a < 8; ++a) {
            double sgnp = 1;
            for (int d = 0; d < 3; ++d)
              if (mask >> d & 1) sgnp *= q1::sgn(a, d);
            c += sgnp * X[a][i];
          }
          if (fabs(c) > 1e-14 * scale) affine = false;
        }
      }
      if (!affine) atomicOr(&out->not_affine, 1);
    }
  }
  if (phys_is_laplace(physics)) {
    double k = m.mat[e];
    if (!(k > 0.0) || !isfinite(k)) flags |= BAD_MAT;
  } else {
    double E = m.mat[2 * e], nu = m.mat[2 * e + 1];
    if (!(E > 0.0) || !isfinite(E) || !(nu > -1.0 && nu < 0.5)) flags |= BAD_MAT;
  }
  if (flags) {
    atomicOr(&out->flags, flags);
    atomicMin(&out->first_bad, (long long)e);
  }
}

// Tetrahedra: node ids in range, finite coordinates, positive orientation (D = 6 |T| > 0), material
// admissible.
__global__ void validate_tet_kernel(MeshView m, int physics, ValidateOut *out) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.n_cells) return;
  int flags = 0;
  int64_t nodes[4];
  for (int a = 0; a < 4; ++a) {
    const int32_t n = m.cells[4 * e + a];
    if (n < 0 || n >= m.n_nodes) flags |= BAD_NODE;
    nodes[a] = n;
  }
  if (!(flags & BAD_NODE)) {
    double X[4][3], n[4][3];
    for (int a = 0; a < 4; ++a)
      for (int i = 0; i < 3; ++i) {
        X[a][i] = m.X[3 * nodes[a] + i];
        if (!isfinite(X[a][i])) flags |= BAD_COORD;
      }
    if (!(flags & BAD_COORD)) {
      const double D = p1::geometry<double>(X, n);
      if (!(D > 0.0) || !isfinite(D)) flags |= BAD_DET;
    }
  }
  if (phys_is_laplace(physics)) {
    double k = m.mat[e];
    if (!(k > 0.0) || !isfinite(k)) flags |= BAD_MAT;
  } else {
    double E = m.mat[2 * e], nu = m.mat[2 * e + 1];
    if (!(E > 0.0) || !isfinite(E) || !(nu > -1.0 && nu < 0.5)) flags |= BAD_MAT;
  }
  if (flags) {
    atomicOr(&out->flags, flags);
    atomicMin(&out->first_bad, (long long)e);
  }
}

// Q2 hexahedra: node ids in range, finite coordinates, det J > 0 at the 27 Gauss points and the 8
// vertices, material admissible.
__global__ void validate_q2_kernel(MeshView m, int physics, ValidateOut *out) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.n_cells) return;
  int flags = 0;
  int64_t nodes[27];
  for (int a = 0; a < 27; ++a) {
    const int32_t n = m.cells[27 * e + a];
    if (n < 0 || n >= m.n_nodes) flags |= BAD_NODE;
    nodes[a] = n;
  }
  if (!(flags & BAD_NODE)) {
    double X[27][3];
    for (int a = 0; a < 27; ++a)
      for (int i = 0; i < 3; ++i) {
        X[a][i] = m.X[3 * nodes[a] + i];
        if (!isfinite(X[a][i])) flags |= BAD_COORD;
      }
    if (!(flags & BAD_COORD) && !q2::dets_positive(X)) flags |= BAD_DET;
  }
  if (phys_is_laplace(physics)) {
    double k = m.mat[e];
    if (!(k > 0.0) || !isfinite(k)) flags |= BAD_MAT;
  } else {
    double E = m.mat[2 * e], nu = m.mat[2 * e + 1];
    if (!(E > 0.0) || !isfinite(E) || !(nu > -1.0 && nu < 0.5)) flags |= BAD_MAT;
  }
  if (flags) {
    atomicOr(&out->flags, flags);
    atomicMin(&out->first_bad, (long long)e);
  }
}

// (E, nu) -> (lam, mu) per cell, plus the FP32 copies.
__global__ void material_kernel(const double *in, double *out, float *out32, int64_t n_cells, int physics) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n_cells) return;
  if (phys_is_laplace(physics)) {
    out[e] = in[e];
    out32[e] = (float)in[e];
  } else {
    double E = in[2 * e], nu = in[2 * e + 1];
    double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    double mu = E / (2.0 * (1.0 + nu));
    out[2 * e] = lam;
    out[2 * e + 1] = mu;
    out32[2 * e] = (float)lam;
    out32[2 * e + 1] = (float)mu;
  }
}

// Largest |cell constant| and smallest positive one (kappa, or mu of (lam, mu)), as bit patterns
// of positive doubles (their integer order is their numeric order).
__global__ void mat_range_kernel(const double *mat, int64_t n_cells, int physics, unsigned long long *out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n_cells) return;
  double big, small;
  if (phys_is_laplace(physics)) {
    big = small = fabs(mat[e]);
  } else {
    small = fabs(mat[2 * e + 1]);
    big = fmax(fabs(mat[2 * e]), small);
  }
  atomicMax(out, (unsigned long long)__double_as_longlong(big));
  if (small > 0.0) atomicMin(out + 1, (unsigned long long)__double_as_longlong(small));
}

__global__ void to_f32_kernel(const double *in, float *out, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}

// --------------------------------------------------------------------------- host helpers ----
template <typename T>
static mf_status dmalloc(T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    mf_set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
    return MF_ERR_OOM;
  }
  return MF_OK;
}

static void free_mesh(mf_mesh *m) {
  if (!m) return;
  if (m->cg) cg_workspace_free(m->cg);
  cudaFree(m->X);
  cudaFree(m->X32);
  cudaFree(m->cells);
  cudaFree(m->mat);
  cudaFree(m->mat32);
  cudaFree(m->dmask);
  cudaFree(m->dnodes);
  cudaFree(m->colour_elems);
  cudaFree(m->tp_axis);
  cudaFree(m->tp_flags);
  cudaFree(m->mat_pairs);
  cudaFree(m->gen_axis);
  cudaFree(m->gen_delta);
  cudaFree(m->pa);
  cudaFree(m->pa32);
  cudaFree(m->q2pa);
  cudaFree(m->q2off);
  cudaFree(m->q2slots);
  cudaFree(m->q2buf);
  delete m;
}

// Greedy element colouring: elements of one colour share no node, so the scatter of one colour
// needs no atomics.  Deterministic (elements visited in index order, smallest free colour).
static mf_status colour_elements(mf_mesh *m, cudaStream_t s) {
  const int64_t E = m->n_cells, N = m->n_nodes;
  const int npe = m->npe;
  const std::vector<int32_t> &cells = m->h_cells;
  std::vector<int64_t> off(N + 1, 0);
  for (int64_t i = 0; i < npe * E; ++i) off[cells[i] + 1]++;
  for (int64_t n = 0; n < N; ++n) off[n + 1] += off[n];
  std::vector<int64_t> fill(off.begin(), off.end() - 1);
  std::vector<int32_t> adj(npe * E);
  for (int64_t e = 0; e < E; ++e)
    for (int a = 0; a < npe; ++a) adj[fill[cells[npe * e + a]]++] = (int32_t)e;
  std::vector<int8_t> colour(E, -1);
  int ncol = 0;
  for (int64_t e = 0; e < E; ++e) {
    uint64_t used = 0;
    for (int a = 0; a < npe; ++a) {
      int32_t n = cells[npe * e + a];
      for (int64_t t = off[n]; t < off[n + 1]; ++t) {
        int8_t c = colour[adj[t]];
        if (c >= 0) used |= 1ull << c;
      }
    }
    int c = 0;
    while (c < 64 && (used >> c & 1)) ++c;
    if (c >= 64) {
      mf_set_error("element colouring needs more than 64 colours (element %lld)", (long long)e);
      return MF_ERR_MESH;
    }
    colour[e] = (int8_t)c;
    ncol = std::max(ncol, c + 1);
  }
  m->n_colours = ncol;
  m->colour_off.assign(ncol + 1, 0);
  for (int64_t e = 0; e < E; ++e) m->colour_off[colour[e] + 1]++;
  for (int c = 0; c < ncol; ++c) m->colour_off[c + 1] += m->colour_off[c];
  std::vector<int64_t> pos(m->colour_off.begin(), m->colour_off.end() - 1);
  std::vector<int32_t> order(E);
  for (int64_t e = 0; e < E; ++e) order[pos[colour[e]]++] = (int32_t)e;
  MF_TRY(dmalloc(&m->colour_elems, E));
  MF_CUDA(cudaMemcpyAsync(m->colour_elems, order.data(), E * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  MF_CUDA(cudaStreamSynchronize(s));
  return MF_OK;
}

int64_t colour_count(const mf_mesh *m, int c) {
  if (!m->structured) return m->colour_off[c + 1] - m->colour_off[c];
  int px = c & 1, py = (c >> 1) & 1, pz = (c >> 2) & 1;
  return (int64_t)((m->nx - px + 1) / 2) * ((m->ny - py + 1) / 2) * ((m->nz - pz + 1) / 2);
}

// Window of the double-word kernels.  A structured mesh's cell constants (kappa, or lam and mu) and
// cell sizes (det J at the Gauss points ~ (h/2)^3) are checked here: when the largest of them lies
// outside the window, the double-word data are built from values scaled by a power of two (exact)
// and the kernels scale y back; when they span more than the double-word arithmetic covers (cell
// constants over a ratio of 2^80, det J over 2^60, i.e. cell sizes over 2^20), the double-word
// kernels are switched off and the mesh runs the FP64 reference kernel.
static mf_status dw_range_setup(mf_mesh *m, unsigned long long det_max_bits, unsigned long long det_min_bits,
                                cudaStream_t s) {
  unsigned long long *d = nullptr;
  MF_TRY(dmalloc(&d, 2));
  unsigned long long h[2] = {0ull, ~0ull};
  MF_CUDA(cudaMemcpyAsync(d, h, sizeof(h), cudaMemcpyHostToDevice, s));
  mat_range_kernel<<<blocks_for(m->n_cells), kThreads, 0, s>>>(m->mat, m->n_cells, m->physics, d);
  MF_CUDA(cudaGetLastError());
  MF_CUDA(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
  MF_CUDA(cudaStreamSynchronize(s));
  cudaFree(d);
  double mat_max, mat_min, det_max, det_min;
  memcpy(&mat_max, &h[0], 8);
  memcpy(&mat_min, &h[1], 8);
  memcpy(&det_max, &det_max_bits, 8);
  memcpy(&det_min, &det_min_bits, 8);
  m->dw_ok = mat_max > 0.0 && mat_min > 0.0 && det_max > 0.0 && det_min > 0.0 && std::isfinite(mat_max) &&
             std::isfinite(det_max) && std::ilogb(mat_max) - std::ilogb(mat_min) <= 80 &&
             std::ilogb(det_max) - std::ilogb(det_min) <= 60;
  m->dw_oscale = 0;
  m->dw_mat = m->dw_geo = 1.0;
  if (!m->dw_ok) return MF_OK;
  const int ek = std::ilogb(mat_max), ed = std::ilogb(det_max);
  const int sk = (ek < -8 || ek > 8) ? ek : 0;
  // det J = (h/2)^3 on a box cell: the length scale is 2^(ed/3)
  const int sh = (ed < -40 || ed > 24) ? (ed >= 0 ? ed / 3 : -((-ed + 2) / 3)) : 0;
  m->dw_mat = std::ldexp(1.0, -sk);
  m->dw_geo = std::ldexp(1.0, -sh);
  m->dw_oscale = sk + sh;
  return MF_OK;
}

// ----------------------------------------------------------------------------- entry points ----
static mf_status setup_mesh(int npe, int physics, int64_t n_nodes, int64_t n_cells, const double *coords,
                            const int32_t *cells, int32_t nx, int32_t ny, int32_t nz, const double *mat,
                            const uint8_t *dirichlet, mf_stream stream, mf_mesh **out) {
  mf_clear_error();
  MF_ARG(out != nullptr, "mf_setup_mesh: out is NULL");
  *out = nullptr;
  MF_ARG(physics == MF_LAPLACE || physics == MF_ELASTICITY || physics == MF_VECTOR_LAPLACE,
         "mf_setup_mesh: unknown physics %d", physics);
  MF_ARG(coords && mat, "mf_setup_mesh: coords and mat are required");
  MF_ARG(npe == 8 || cells != nullptr, "mf_setup_mesh: tetrahedral and Q2 meshes need an explicit connectivity");
  MF_ARG(n_nodes >= npe && n_cells >= 1, "mf_setup_mesh: need n_nodes >= %d and n_cells >= 1", npe);
  // the kernels index coordinates and DoFs (3 per node) and the connectivity (npe per cell) with
  // 32-bit integers: larger meshes are refused here rather than indexed past 2^31 - 1
  MF_ARG(3 * n_nodes <= (int64_t)INT32_MAX, "mf_setup_mesh: %lld nodes: 3 n_nodes must fit int32",
         (long long)n_nodes);
  MF_ARG((int64_t)npe * n_cells <= (int64_t)INT32_MAX,
         "mf_setup_mesh: %lld cells of %d nodes: the connectivity's size must fit int32", (long long)n_cells, npe);
  if (!cells) {
    MF_ARG(nx > 0 && ny > 0 && nz > 0, "mf_setup_mesh: structured mesh needs nx, ny, nz > 0");
    MF_ARG((int64_t)nx * ny * nz == n_cells, "mf_setup_mesh: n_cells != nx*ny*nz");
    MF_ARG((int64_t)(nx + 1) * (ny + 1) * (nz + 1) == n_nodes, "mf_setup_mesh: n_nodes != (nx+1)(ny+1)(nz+1)");
  }
  cudaStream_t s = (cudaStream_t)stream;
  mf_mesh *m = new mf_mesh();
  MF_CUDA(cudaGetDevice(&m->device));
  m->physics = physics;
  m->ndpn = phys_ndpn(physics);
  m->n_nodes = n_nodes;
  m->n_cells = n_cells;
  m->npe = npe;
  m->n_dof = n_nodes * m->ndpn;
  m->structured = cells == nullptr;
  m->nx = cells ? 0 : nx;
  m->ny = cells ? 0 : ny;
  m->nz = cells ? 0 : nz;
  const int nmat = phys_nmat(physics);
  mf_status st = MF_OK;
#define SETUP_TRY(expr)               \
  do {                                \
    st = (expr);                      \
    if (st != MF_OK) goto fail;       \
  } while (0)
#define SETUP_CUDA(call)                                                                         \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) {                                                                     \
      mf_set_error("mf_setup_mesh: %s failed: %s", #call, cudaGetErrorString(e_));               \
      st = e_ == cudaErrorMemoryAllocation ? MF_ERR_OOM : MF_ERR_CUDA;                           \
      goto fail;                                                                                 \
    }                                                                                            \
  } while (0)
  {
    SETUP_TRY(dmalloc(&m->X, 3 * n_nodes));
    SETUP_TRY(dmalloc(&m->X32, 3 * n_nodes));
    SETUP_TRY(dmalloc(&m->mat, nmat * n_cells));
    SETUP_TRY(dmalloc(&m->mat32, nmat * n_cells));
    SETUP_TRY(dmalloc(&m->dmask, n_nodes));
    SETUP_CUDA(cudaMemcpyAsync(m->X, coords, 3 * n_nodes * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (cells) {
      SETUP_TRY(dmalloc(&m->cells, npe * n_cells));
      SETUP_CUDA(cudaMemcpyAsync(m->cells, cells, npe * n_cells * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
    if (dirichlet)
      SETUP_CUDA(cudaMemcpyAsync(m->dmask, dirichlet, n_nodes, cudaMemcpyDeviceToDevice, s));
    else
      SETUP_CUDA(cudaMemsetAsync(m->dmask, 0, n_nodes, s));
    to_f32_kernel<<<blocks_for(3 * n_nodes), kThreads, 0, s>>>(m->X, m->X32, 3 * n_nodes);
    SETUP_CUDA(cudaGetLastError());

    // validation (uses the caller's material array before conversion)
    ValidateOut *dv = nullptr;
    SETUP_TRY(dmalloc(&dv, 1));
    ValidateOut hv = {0, 0, (long long)n_cells, 0ull, ~0ull};
    SETUP_CUDA(cudaMemcpyAsync(dv, &hv, sizeof(hv), cudaMemcpyHostToDevice, s));
    MeshView v = m->view();
    v.mat = mat;
    if (npe == 4) validate_tet_kernel<<<blocks_for(n_cells), kThreads, 0, s>>>(v, physics, dv);
    else if (npe == 27) validate_q2_kernel<<<blocks_for(n_cells, 64), 64, 0, s>>>(v, physics, dv);
    else validate_kernel<<<blocks_for(n_cells), kThreads, 0, s>>>(v, physics, dv);
    SETUP_CUDA(cudaGetLastError());
    SETUP_CUDA(cudaMemcpyAsync(&hv, dv, sizeof(hv), cudaMemcpyDeviceToHost, s));
    SETUP_CUDA(cudaStreamSynchronize(s));
    cudaFree(dv);
    if (hv.flags) {
      mf_set_error("mf_setup_mesh: invalid mesh (element %lld:%s%s%s%s)", hv.first_bad,
                   hv.flags & BAD_DET ? " det J <= 0" : "", hv.flags & BAD_NODE ? " node id out of range" : "",
                   hv.flags & BAD_COORD ? " non-finite coordinate" : "", hv.flags & BAD_MAT ? " bad material" : "");
      st = MF_ERR_MESH;
      goto fail;
    }
    m->all_affine = hv.not_affine == 0 && npe != 27;  // Q2 cells are not checked for affinity
    material_kernel<<<blocks_for(n_cells), kThreads, 0, s>>>(mat, m->mat, m->mat32, n_cells, physics);
    SETUP_CUDA(cudaGetLastError());

    // Dirichlet node list
    std::vector<uint8_t> hmask(n_nodes);
    SETUP_CUDA(cudaMemcpyAsync(hmask.data(), m->dmask, n_nodes, cudaMemcpyDeviceToHost, s));
    SETUP_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> dn;
    for (int64_t i = 0; i < n_nodes; ++i)
      if (hmask[i]) dn.push_back((int32_t)i);
    m->n_dnodes = (int64_t)dn.size();
    m->n_free = (n_nodes - m->n_dnodes) * m->ndpn;
    SETUP_TRY(dmalloc(&m->dnodes, dn.size()));
    if (!dn.empty())
      SETUP_CUDA(cudaMemcpyAsync(m->dnodes, dn.data(), dn.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));

    if (cells) {
      m->h_cells.resize(npe * n_cells);
      SETUP_CUDA(cudaMemcpyAsync(m->h_cells.data(), cells, npe * n_cells * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      SETUP_CUDA(cudaStreamSynchronize(s));
      SETUP_TRY(colour_elements(m, s));
      if (npe == 27) {
        // the auto variant uses the Q2 partial assembly when it takes at most a quarter of the
        // device's total memory (a function of the mesh and the device model); if the allocation
        // fails all the same, the mesh keeps the reference kernel (flag bit 3 reports it)
        size_t free_b = 0, total_b = 0;
        SETUP_CUDA(cudaMemGetInfo(&free_b, &total_b));
        if ((double)q2_pa_bytes(physics, n_cells) <= 0.25 * (double)total_b) {
          st = q2_pa_setup(m, s);
          if (st != MF_OK && st != MF_ERR_OOM) goto fail;
          st = MF_OK;
          mf_clear_error();
        }
      }
    } else {
      m->n_colours = 8;  // parity colouring of the box
      SETUP_TRY(dw_range_setup(m, hv.det_max, hv.det_min, s));
      if (m->dw_ok) {
        SETUP_TRY(tile_setup(m, s));
        SETUP_TRY(gen_setup(m, s));
      }
    }
    SETUP_CUDA(cudaStreamSynchronize(s));
  }
  *out = m;
  return MF_OK;
fail:
  cudaStreamSynchronize(s);
  free_mesh(m);
  return st;
#undef SETUP_TRY
#undef SETUP_CUDA
}

extern "C" mf_status mf_setup_mesh(int physics, int64_t n_nodes, int64_t n_cells, const double *coords,
                                   const int32_t *cells, int32_t nx, int32_t ny, int32_t nz, const double *mat,
                                   const uint8_t *dirichlet, mf_stream stream, mf_mesh **out) {
  MF_RANGE("mf_setup_mesh");
  return setup_mesh(8, physics, n_nodes, n_cells, coords, cells, nx, ny, nz, mat, dirichlet, stream, out);
}

extern "C" mf_status mf_setup_mesh_elem(int element, int physics, int64_t n_nodes, int64_t n_cells,
                                        const double *coords, const int32_t *cells, const double *mat,
                                        const uint8_t *dirichlet, mf_stream stream, mf_mesh **out) {
  MF_RANGE("mf_setup_mesh_elem");
  mf_clear_error();
  MF_ARG(element == MF_ELEM_HEX8 || element == MF_ELEM_TET4 || element == MF_ELEM_HEX27,
         "mf_setup_mesh_elem: unknown element %d", element);
  MF_ARG(cells != nullptr, "mf_setup_mesh_elem: cells is required");
  const int npe = element == MF_ELEM_TET4 ? 4 : element == MF_ELEM_HEX27 ? 27 : 8;
  return setup_mesh(npe, physics, n_nodes, n_cells, coords, cells, 0, 0, 0, mat, dirichlet, stream, out);
}

extern "C" mf_status mf_destroy_mesh(mf_mesh *mesh) {
  MF_RANGE("mf_destroy_mesh");
  mf_clear_error();
  if (!mesh) return MF_OK;
  MF_CUDA(cudaDeviceSynchronize());
  free_mesh(mesh);
  return MF_OK;
}

extern "C" mf_status mf_mesh_query(const mf_mesh *m, int64_t *n_nodes, int64_t *n_cells, int64_t *n_dof,
                                   int64_t *n_free, int32_t *n_colours, int32_t *flags) {
  MF_ARG(m != nullptr, "mf_mesh_query: mesh is NULL");
  if (n_nodes) *n_nodes = m->n_nodes;
  if (n_cells) *n_cells = m->n_cells;
  if (n_dof) *n_dof = m->n_dof;
  if (n_free) *n_free = m->n_free;
  if (n_colours) *n_colours = m->n_colours;
  if (flags)
    *flags = (m->structured ? 1 : 0) | (m->all_affine ? 2 : 0) | (m->tp ? 4 : 0) | (m->pa || m->q2pa ? 8 : 0) |
             (m->npe == 4 ? 16 : 0) | (m->npe == 27 ? 32 : 0) | (m->structured && !m->dw_ok ? 64 : 0) |
             (m->dw_ok && m->dw_oscale != 0 ? 128 : 0);
  return MF_OK;
}

extern "C" mf_status mf_set_apply_variant(mf_mesh *m, int variant) {
  MF_ARG(m != nullptr, "mf_set_apply_variant: mesh is NULL");
  MF_ARG(variant == MF_VARIANT_AUTO || variant == MF_VARIANT_REFERENCE || variant == MF_VARIANT_GENERAL ||
             variant == MF_VARIANT_PARTIAL,
         "mf_set_apply_variant: unknown variant %d", variant);
  if (variant == MF_VARIANT_PARTIAL && m->npe == 27) {  // Q2 Laplace: sum-factorised partial assembly
    MF_TRY(q2_pa_setup(m, 0));
    m->variant = variant;
    return MF_OK;
  }
  if (variant == MF_VARIANT_GENERAL || variant == MF_VARIANT_PARTIAL) {
    if (!m->gen) {
      mf_set_error("mf_set_apply_variant: the general and partial-assembly variants need a structured mesh that is "
                   "not a tensor-product grid, with cell constants and cell sizes within the double-word range "
                   "(flag bit 6 of mf_mesh_query set means they are not)");
      return MF_ERR_UNSUPPORTED;
    }
  }
  if (variant == MF_VARIANT_PARTIAL && !m->pa) MF_TRY(pa_setup(m, 0));
  m->variant = variant;
  return MF_OK;
}

extern "C" mf_status mf_debug_status(uint32_t *bits, int32_t *enabled) {
  mf_clear_error();
  MF_ARG(bits != nullptr, "mf_debug_status: bits is NULL");
#ifdef MF_DEBUG_BOUNDS
  if (enabled) *enabled = 1;
  MF_CUDA(cudaDeviceSynchronize());
  *bits = mf_dbg_take_apply() | mf_dbg_take_tile() | mf_dbg_take_cg() | mf_dbg_take_batched() |
          mf_dbg_take_general() | mf_dbg_take_csr();
#else
  if (enabled) *enabled = 0;
  *bits = 0u;
#endif
  return MF_OK;
}
