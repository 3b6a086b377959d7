// Conjugate gradient on the device (the per-iteration operations of Table 4), with the scalars
// alpha, beta and the residual norms kept in device memory.
//
// The paper observes that the dot-product implementation decides CG performance (Sec. 6, the
// "dot" figure) and leaves kernel fusion undone.  Here each dot is fused into the vector update
// that produces its operand, and reduced with a fixed two-level tree (per-block partials in a
// fixed grid-stride partition, summed in index order by the last block to finish): results are
// bitwise reproducible and no host round trip is needed per iteration.  `check_every` iterations
// are captured in one CUDA graph; every kernel first reads a device "done" flag, so iterations
// after convergence cost only their launch.
//
// Per iteration (FP64, no preconditioner), in DoF-vector passes:
//   apply A p -> Ap                     (operator)
//   pAp = p.Ap; alpha = rho/pAp          read p, Ap
//   x += alpha p; r -= alpha Ap; rho' = r.r   read x, p, r, Ap; write x, r
//   p = r + beta p                       read r, p; write p
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>

#include "mf_internal.cuh"

namespace {

// Reduction grids: a fixed number of blocks (4 per SM of a 152-SM GB300), so that the reduction
// tree, and with it every dot product's rounding, is the same on every run and every GPU.
constexpr int kRedBlocksPerSm = 4;
constexpr int kRedBlocks = 152 * kRedBlocksPerSm;
constexpr int kRedThreads = 256;
// The per-iteration vector kernels take kVecUnroll strided elements per step of their grid-stride
// loop and issue all of the step's loads before its arithmetic, so that each thread has kVecUnroll
// times the loads of a plain grid-stride loop in flight (HBM needs far more bytes in flight per SM
// than 32 warps with one 8-byte load each).  A thread still visits i, i + S, i + 2S, ... in that
// order, so every sum is formed in the order of the plain loop.  Their launch bounds keep all
// kRedBlocks blocks resident at once (at most 64 registers a thread).
constexpr int kVecUnroll = 4;

struct CgScalars {
  double bb, rr, rz, pAp, alpha, beta, tol2, res2;
  int iter, max_iter, done, status;
  unsigned int ticket;
  int xpend;  // the last x/r update ran: alpha p of that iteration is still owed to x (fused CG)
};

// Sum NV per-thread values over the whole grid.  Returns true in the last block to arrive, whose
// thread 0 then holds the totals in `out`.  Every block of the launch must call it.
template <int NV>
__device__ __forceinline__ bool grid_reduce(double (&v)[NV], double *partials, unsigned int *ticket, double (&out)[NV]) {
  __shared__ double sh[NV][kRedThreads / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    if (lane == 0) sh[k][w] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int i = 0; i < kRedThreads / 32; ++i) s += sh[k][i];
      partials[k * gridDim.x + blockIdx.x] = s;
    }
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  const volatile double *vp = partials;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += vp[k * gridDim.x + i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    __syncthreads();
    if (lane == 0) sh[k][w] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int i = 0; i < kRedThreads / 32; ++i) s += sh[k][i];
      out[k] = s;
    }
    *ticket = 0;
  }
  return true;
}

#define GRID_STRIDE(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// x = 0, r = b, p = z = M r; rho = r.z, ||b||^2.
template <typename R>
__global__ void __launch_bounds__(kRedThreads) cg_init(int64_t n, const R *__restrict__ b, R *__restrict__ x,
                                                       R *__restrict__ r, R *__restrict__ p,
                                                       const double *__restrict__ invdiag, double *partials,
                                                       CgScalars *sc, double rtol, int max_iter) {
  double v[2] = {0.0, 0.0};
  GRID_STRIDE(i, n) {
    const R bi = b[i];
    x[i] = (R)0;
    r[i] = bi;
    const double z = invdiag ? (double)bi * invdiag[i] : (double)bi;
    p[i] = (R)z;
    v[0] += (double)bi * (double)bi;
    v[1] += (double)bi * z;
  }
  double out[2];
  if (grid_reduce<2>(v, partials, &sc->ticket, out) && threadIdx.x == 0) {
    sc->bb = out[0];
    sc->rr = out[0];
    sc->rz = out[1];
    sc->alpha = 0.0;  // the fused iteration's first apply: p_0 = z_0 + 0 p and x += 0 p
    sc->beta = 0.0;
    sc->xpend = 0;
    sc->tol2 = rtol * rtol * out[0];
    sc->iter = 0;
    sc->max_iter = max_iter;
    sc->status = 0;
    sc->done = (out[0] <= sc->tol2) ? 1 : 0;
    if (!isfinite(out[0])) {
      sc->status = MF_ERR_BREAKDOWN;
      sc->done = 1;
    }
  }
}

// pAp = p.Ap (when the operator does not fuse it into its own write phase).
template <typename R>
__global__ void __launch_bounds__(kRedThreads, kRedBlocksPerSm) cg_pap(int64_t n, const R *__restrict__ p, const R *__restrict__ Ap,
                                                      double *partials, CgScalars *sc) {
  if (sc->done) return;
  double v[1] = {0.0};
  const int64_t S = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + (kVecUnroll - 1) * S < n; i += kVecUnroll * S) {
    R pu[kVecUnroll], au[kVecUnroll];
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u) {
      pu[u] = p[i + u * S];
      au[u] = Ap[i + u * S];
    }
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u) v[0] += (double)pu[u] * (double)au[u];
  }
  for (; i < n; i += S) v[0] += (double)p[i] * (double)Ap[i];
  double out[1];
  if (grid_reduce<1>(v, partials, &sc->ticket, out) && threadIdx.x == 0) sc->pAp = out[0];
}

// x += alpha p; r -= alpha Ap; rho' = r.z (z = M r), ||r||^2; beta = rho'/rho; convergence test.
// X false: r only, x and p are not read (the fused iteration adds alpha p to x in the next apply, or
// cg_flush_x at the end).  A step takes kVecUnroll elements for r alone and half as many for x and r,
// about eight loads in flight per thread either way.
template <typename R, bool X>
__global__ void __launch_bounds__(kRedThreads, kRedBlocksPerSm) cg_update_xr(int64_t n, R *__restrict__ x, R *__restrict__ r,
                                                            const R *__restrict__ p, const R *__restrict__ Ap,
                                                            const double *__restrict__ invdiag, double *partials,
                                                            CgScalars *sc) {
  if (sc->done) return;
  // alpha = rho / pAp (every block forms it from the same scalars; block 0 records it)
  const double pap = sc->pAp;
  if (!(pap > 0.0) || !isfinite(pap)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      sc->status = MF_ERR_BREAKDOWN;
      sc->done = 1;
      sc->xpend = 0;
    }
    return;
  }
  const double alpha = sc->rz / pap;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->alpha = alpha;
    sc->xpend = 1;
  }
  double v[2] = {0.0, 0.0};
  // one element: x_j and r_j updated from the loaded values, then the two sums
  auto elem = [&](int64_t j, R pj, R xj, R aj, R rj, double dj) {
    if constexpr (X) x[j] = (R)__fma_rn(alpha, (double)pj, (double)xj);
    const R ri = (R)__fma_rn(-alpha, (double)aj, (double)rj);
    r[j] = ri;
    const double rd = (double)ri;
    v[0] += rd * rd;
    v[1] += invdiag ? rd * rd * dj : rd * rd;
  };
  const int64_t S = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  constexpr int U = X ? kVecUnroll / 2 : kVecUnroll;
  for (; i + (U - 1) * S < n; i += U * S) {
    R pu[U], xu[U], au[U], ru[U];
    double du[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t j = i + u * S;
      pu[u] = X ? p[j] : (R)0;
      xu[u] = X ? x[j] : (R)0;
      au[u] = Ap[j];
      ru[u] = r[j];
      du[u] = invdiag ? invdiag[j] : 1.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) elem(i + u * S, pu[u], xu[u], au[u], ru[u], du[u]);
  }
  for (; i < n; i += S)
    elem(i, X ? p[i] : (R)0, X ? x[i] : (R)0, Ap[i], r[i], invdiag ? invdiag[i] : 1.0);
  double out[2];
  if (grid_reduce<2>(v, partials, &sc->ticket, out) && threadIdx.x == 0) {
    const double rr = out[0], rz = out[1];
    sc->beta = rz / sc->rz;
    sc->rr = rr;
    sc->rz = rz;
    sc->iter += 1;
    if (!isfinite(rr) || !isfinite(rz)) {
      sc->status = MF_ERR_BREAKDOWN;
      sc->done = 1;
    } else if (rr <= sc->tol2) {
      sc->done = 1;
    } else if (sc->iter >= sc->max_iter) {
      sc->status = MF_NOT_CONVERGED;
      sc->done = 1;
    }
  }
}

// p = z + beta p.
template <typename R>
__global__ void __launch_bounds__(kRedThreads, kRedBlocksPerSm) cg_update_p(int64_t n, const R *__restrict__ r, R *__restrict__ p,
                                                           const double *__restrict__ invdiag, const CgScalars *sc) {
  if (sc->done) return;
  const double beta = sc->beta;
  auto elem = [&](int64_t j, R rj, R pj, double dj) {
    const double z = invdiag ? __dmul_rn((double)rj, dj) : (double)rj;
    p[j] = (R)__fma_rn(beta, (double)pj, z);
  };
  const int64_t S = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + (kVecUnroll - 1) * S < n; i += kVecUnroll * S) {
    R ru[kVecUnroll], pu[kVecUnroll];
    double du[kVecUnroll];
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u) {
      const int64_t j = i + u * S;
      ru[u] = r[j];
      pu[u] = p[j];
      du[u] = invdiag ? invdiag[j] : 1.0;
    }
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u) elem(i + u * S, ru[u], pu[u], du[u]);
  }
  for (; i < n; i += S) elem(i, r[i], p[i], invdiag ? invdiag[i] : 1.0);
}

// End of a fused CG solve that started at iteration iter0: the last iteration's x += alpha p, if its
// x/r update ran (p_k is in p0 when k - iter0 is even, in p1 when it is odd; k = iter - 1).
__global__ void __launch_bounds__(kRedThreads) cg_flush_x(int64_t n, double *__restrict__ x,
                                                          const double *__restrict__ p0,
                                                          const double *__restrict__ p1, const CgScalars *sc,
                                                          int iter0) {
  if (!sc->xpend) return;
  const double alpha = sc->alpha;
  const double *p = ((sc->iter - 1 - iter0) & 1) ? p1 : p0;
  GRID_STRIDE(i, n) x[i] = __fma_rn(alpha, p[i], x[i]);
}

// ---- single-synchronisation CG (Chronopoulos and Gear 1989), the pipelined recurrence.  With
// u = M^-1 r and w = A u, both dot products of an iteration, gamma = r.u and delta = u.w, are
// formed where their operands are produced (gamma in the update, delta in the apply), and
//   beta_i = gamma_i / gamma_{i-1},  alpha_i = gamma_i / (delta_i - beta_i gamma_i / alpha_{i-1}),
//   p = u + beta p,  s = w + beta s (= A p),  x += alpha p,  r -= alpha s,  u = M^-1 r
// run in one pass: per iteration the apply and one update kernel (the classic recurrence needs a
// second vector kernel, because its p update waits for the reduced r.r).

// x = 0, r = b, u = M^-1 b (u is r without a preconditioner), p = s = 0; gamma = r.u, ||b||^2,
// beta = 0, alpha = 1 (so that the first alpha is gamma / delta).
template <typename R>
__global__ void __launch_bounds__(kRedThreads) cgp_init(int64_t n, const R *__restrict__ b, R *__restrict__ x,
                                                        R *__restrict__ r, R *__restrict__ u, R *__restrict__ p,
                                                        R *__restrict__ s, const double *__restrict__ invdiag,
                                                        double *partials, CgScalars *sc, double rtol, int max_iter) {
  double v[2] = {0.0, 0.0};
  GRID_STRIDE(i, n) {
    const R bi = b[i];
    x[i] = (R)0;
    r[i] = bi;
    p[i] = (R)0;
    s[i] = (R)0;
    const double z = invdiag ? (double)bi * invdiag[i] : (double)bi;
    if (u) u[i] = (R)z;
    v[0] += (double)bi * (double)bi;
    v[1] += (double)bi * z;
  }
  double out[2];
  if (grid_reduce<2>(v, partials, &sc->ticket, out) && threadIdx.x == 0) {
    sc->bb = out[0];
    sc->rr = out[0];
    sc->rz = out[1];
    sc->beta = 0.0;
    sc->alpha = 1.0;
    sc->tol2 = rtol * rtol * out[0];
    sc->iter = 0;
    sc->max_iter = max_iter;
    sc->status = 0;
    sc->done = (out[0] <= sc->tol2) ? 1 : 0;
    if (!isfinite(out[0])) {
      sc->status = MF_ERR_BREAKDOWN;
      sc->done = 1;
    }
  }
}

// The update pass of an iteration: alpha from gamma (sc->rz), delta (sc->pAp), beta and the previous
// alpha; p, s, x, r and u; then gamma' = r.u and ||r||^2, beta' = gamma'/gamma, convergence test.
template <typename R>
__global__ void __launch_bounds__(kRedThreads) cgp_update(int64_t n, R *__restrict__ x, R *__restrict__ r,
                                                          R *__restrict__ u, R *__restrict__ p, R *__restrict__ s,
                                                          const R *__restrict__ w, const double *__restrict__ invdiag,
                                                          double *partials, CgScalars *sc) {
  if (sc->done) return;
  const double gamma = sc->rz, beta = sc->beta;
  const double denom = sc->pAp - beta * gamma / sc->alpha;
  if (!(denom > 0.0) || !isfinite(denom)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      sc->status = MF_ERR_BREAKDOWN;
      sc->done = 1;
    }
    return;
  }
  const double alpha = gamma / denom;
  const R *uu = u ? u : r;
  double v[2] = {0.0, 0.0};
  GRID_STRIDE(i, n) {
    const double pi = (double)uu[i] + beta * (double)p[i];
    const double si = (double)w[i] + beta * (double)s[i];
    p[i] = (R)pi;
    s[i] = (R)si;
    x[i] = (R)((double)x[i] + alpha * pi);
    const R ri = (R)((double)r[i] - alpha * si);
    r[i] = ri;
    const double rd = (double)ri;
    const double z = invdiag ? rd * invdiag[i] : rd;
    if (u) u[i] = (R)z;
    v[0] += rd * rd;
    v[1] += rd * z;
  }
  double out[2];
  if (grid_reduce<2>(v, partials, &sc->ticket, out) && threadIdx.x == 0) {
    const double rr = out[0], rz = out[1];
    sc->beta = rz / gamma;
    sc->alpha = alpha;
    sc->rr = rr;
    sc->rz = rz;
    sc->iter += 1;
    if (!isfinite(rr) || !isfinite(rz)) {
      sc->status = MF_ERR_BREAKDOWN;
      sc->done = 1;
    } else if (rr <= sc->tol2) {
      sc->done = 1;
    } else if (sc->iter >= sc->max_iter) {
      sc->status = MF_NOT_CONVERGED;
      sc->done = 1;
    }
  }
}

// res = b - Ax (stored when `res` is not null); res2 = ||b - Ax||^2.
__global__ void __launch_bounds__(kRedThreads) residual_kernel(int64_t n, const double *__restrict__ b,
                                                               const double *__restrict__ Ax, double *__restrict__ res,
                                                               double *partials, CgScalars *sc) {
  double v[1] = {0.0};
  GRID_STRIDE(i, n) {
    const double ri = b[i] - Ax[i];
    if (res) res[i] = ri;
    v[0] += ri * ri;
  }
  double out[1];
  if (grid_reduce<1>(v, partials, &sc->ticket, out) && threadIdx.x == 0) sc->res2 = out[0];
}

__global__ void invert_kernel(int64_t n, double *d) {
  GRID_STRIDE(i, n) d[i] = 1.0 / d[i];
}

__global__ void to_f32(int64_t n, const double *__restrict__ a, float *__restrict__ b) {
  GRID_STRIDE(i, n) b[i] = (float)a[i];
}

__global__ void add_f32(int64_t n, double *__restrict__ x, const float *__restrict__ d) {
  GRID_STRIDE(i, n) x[i] += (double)d[i];
}

// Training pair of the learned preconditioner: r~ = D^-1/2 (b - A x_k), e~ = D^1/2 (x* - x_k) with
// D = diag(A) (invdiag holds 1/D), Dirichlet entries 0; sums of r~^2 and e~^2 into sc->res2, sc->bb.
__global__ void __launch_bounds__(kRedThreads)
    pair_kernel(int64_t n, int ndpn, const double *__restrict__ b, const double *__restrict__ Axk,
                const double *__restrict__ xs, const double *__restrict__ xk, const double *__restrict__ invdiag,
                const uint8_t *__restrict__ dmask, double *__restrict__ r, double *__restrict__ e, double *partials,
                CgScalars *sc) {
  double v[2] = {0.0, 0.0};
  GRID_STRIDE(i, n) {
    const bool dir = dmask[i / ndpn] != 0;
    const double sq = sqrt(invdiag[i]);  // D^-1/2
    const double ri = dir ? 0.0 : (b[i] - Axk[i]) * sq;
    const double ei = dir ? 0.0 : (xs[i] - xk[i]) / sq;
    r[i] = ri;
    e[i] = ei;
    v[0] += ri * ri;
    v[1] += ei * ei;
  }
  double out[2];
  if (grid_reduce<2>(v, partials, &sc->ticket, out) && threadIdx.x == 0) {
    sc->res2 = out[0];
    sc->bb = out[1];
  }
}

// r32 = r~ / s, e32 = e~ / s with s = RMS(r~) = sqrt(sc->res2 / n) (1 when r~ = 0).
__global__ void pair_scale(int64_t n, const double *__restrict__ r, const double *__restrict__ e,
                           const CgScalars *__restrict__ sc, float *__restrict__ r32, float *__restrict__ e32) {
  const double ss = sc->res2 > 0.0 ? sqrt(sc->res2 / (double)n) : 1.0;
  GRID_STRIDE(i, n) {
    r32[i] = (float)(r[i] / ss);
    e32[i] = (float)(e[i] / ss);
  }
}

using OpFn = std::function<mf_status(const void *in, void *out, cudaStream_t s, const int *skip)>;
// operator with in . out fused: writes the dot product to *dot (null function when not available)
using OpDotFn = std::function<mf_status(const void *in, void *out, cudaStream_t s, const int *skip, double *dot)>;

}  // namespace

struct CgWorkspace {
  int64_t n = 0;
  double *x = nullptr, *r = nullptr, *p = nullptr, *Ap = nullptr, *invdiag = nullptr, *bb = nullptr;
  double *s = nullptr, *u = nullptr;  // pipelined recurrence: s = A p, u = M^-1 r (Jacobi only)
  double *p2 = nullptr;               // fused classic iteration: p of odd iterations (p: even)
  float *x32 = nullptr, *r32 = nullptr, *p32 = nullptr, *Ap32 = nullptr;
  double *partials = nullptr;
  double *dotp = nullptr;       // per-CTA parts of the dot product fused into the apply
  unsigned int *dticket = nullptr;
  CgScalars *sc = nullptr, *sc32 = nullptr;
  CgScalars *h_sc = nullptr;
  cudaStream_t cap = nullptr;
  // What a captured graph depends on besides the workspace: the operator (matrix-free, or which
  // assembled matrix: its device arrays and sizes are baked into the graph), the mesh's apply
  // variant, the preconditioner, the recurrence and the iterations per launch.  A CSR matrix is
  // identified by its process-unique id, so a matrix assembled after another was destroyed never
  // matches a graph captured for the old one, even at the same host address.
  struct Key {
    int op = -1, precond = -1, variant = -1, check_every = -1, recurrence = -1, precision = -1;
    uint64_t csr_id = 0;
    bool operator==(const Key &o) const {
      return op == o.op && precond == o.precond && variant == o.variant && check_every == o.check_every &&
             recurrence == o.recurrence && precision == o.precision && csr_id == o.csr_id;
    }
  };
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    Key key;
    int64_t kernels = 0;  // kernel nodes per replay
  } g[2];
  bool invdiag_ready = false;  // invdiag holds 1 / diag(A) of this mesh
  // What the last classic FP64 solve left for mf_cg_state_save: fused (1) or split (0) iteration, -1
  // for no state; its status and preconditioner; where its last search direction is and whether the
  // split kernels had already formed p_k from it.
  int last_fused = -1, last_status = 0, last_precond = 0;
  const double *last_p = nullptr;
  bool last_p_new = false;
};

void cg_workspace_free(CgWorkspace *w) {
  if (!w) return;
  for (auto &g : w->g)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  cudaFree(w->x); cudaFree(w->r); cudaFree(w->p); cudaFree(w->Ap); cudaFree(w->invdiag); cudaFree(w->bb);
  cudaFree(w->s); cudaFree(w->u); cudaFree(w->p2);
  cudaFree(w->x32); cudaFree(w->r32); cudaFree(w->p32); cudaFree(w->Ap32);
  cudaFree(w->partials); cudaFree(w->sc); cudaFree(w->sc32); cudaFree(w->dotp); cudaFree(w->dticket);
  if (w->h_sc) cudaFreeHost(w->h_sc);
  if (w->cap) cudaStreamDestroy(w->cap);
  delete w;
}

namespace {

mf_status ensure_workspace(mf_mesh *m, bool need32, bool needdiag) {
  if (!m->cg) {
    CgWorkspace *w = new CgWorkspace();
    m->cg = w;
    w->n = m->n_dof;
    const size_t nb = w->n * sizeof(double);
    MF_CUDA(cudaMalloc(&w->x, nb));
    MF_CUDA(cudaMalloc(&w->r, nb));
    MF_CUDA(cudaMalloc(&w->p, nb));
    MF_CUDA(cudaMalloc(&w->Ap, nb));
    MF_CUDA(cudaMalloc(&w->partials, 4 * kRedBlocks * sizeof(double)));
    MF_CUDA(cudaMalloc(&w->sc, sizeof(CgScalars)));
    MF_CUDA(cudaMalloc(&w->sc32, sizeof(CgScalars)));
    MF_CUDA(cudaMemset(w->sc, 0, sizeof(CgScalars)));
    MF_CUDA(cudaMemset(w->sc32, 0, sizeof(CgScalars)));
    MF_CUDA(cudaMallocHost(&w->h_sc, 2 * sizeof(CgScalars)));
    MF_CUDA(cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking));
    if (m->tp) {
      MF_CUDA(cudaMalloc(&w->dotp, tile_dot_slots(m) * sizeof(double)));
      MF_CUDA(cudaMalloc(&w->dticket, sizeof(unsigned int)));
      MF_CUDA(cudaMemset(w->dticket, 0, sizeof(unsigned int)));
    }
  }
  CgWorkspace *w = m->cg;
  if (need32 && !w->x32) {
    const size_t nf = w->n * sizeof(float);
    MF_CUDA(cudaMalloc(&w->x32, nf));
    MF_CUDA(cudaMalloc(&w->r32, nf));
    MF_CUDA(cudaMalloc(&w->p32, nf));
    MF_CUDA(cudaMalloc(&w->Ap32, nf));
  }
  if (needdiag && !w->invdiag) MF_CUDA(cudaMalloc(&w->invdiag, w->n * sizeof(double)));
  return MF_OK;
}

// 1 / diag(A) in the workspace.  The diagonal depends on the mesh alone, so it is computed by the
// first solve that needs it and kept for the later ones.
mf_status ensure_invdiag(mf_mesh *m, cudaStream_t s) {
  MF_TRY(ensure_workspace(m, false, true));
  CgWorkspace *w = m->cg;
  if (w->invdiag_ready) return MF_OK;
  MF_TRY(operator_diagonal(m, w->invdiag, s));
  mf_count_launches(1);
  invert_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(w->n, w->invdiag);
  MF_CUDA(cudaGetLastError());
  w->invdiag_ready = true;
  return MF_OK;
}

// One CG iteration (Table 4) for vectors of type R.
template <typename R>
mf_status cg_iteration(const OpFn &op, const OpDotFn &opdot, int64_t n, R *x, R *r, R *p, R *Ap,
                       const double *invdiag, double *partials, CgScalars *sc, cudaStream_t s) {
  if (opdot) {
    MF_TRY(opdot(p, Ap, s, &sc->done, &sc->pAp));  // Ap = A p and pAp in one kernel
    mf_count_launches(2);
  } else {
    MF_TRY(op(p, Ap, s, &sc->done));
    mf_count_launches(3);
    cg_pap<R><<<kRedBlocks, kRedThreads, 0, s>>>(n, p, Ap, partials, sc);
  }
  cg_update_xr<R, true><<<kRedBlocks, kRedThreads, 0, s>>>(n, x, r, p, Ap, invdiag, partials, sc);
  cg_update_p<R><<<kRedBlocks, kRedThreads, 0, s>>>(n, r, p, invdiag, sc);
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

// One iteration of the single-synchronisation recurrence: w = A u with delta = u.w, then the update.
mf_status cgp_iteration(const OpFn &op, const OpDotFn &opdot, int64_t n, double *x, double *r, double *u, double *p,
                        double *sv, double *wv, const double *invdiag, double *partials, CgScalars *sc,
                        cudaStream_t s) {
  double *in = u ? u : r;
  if (opdot) {
    MF_TRY(opdot(in, wv, s, &sc->done, &sc->pAp));  // w = A u and u.w in one kernel
    mf_count_launches(1);
  } else {
    MF_TRY(op(in, wv, s, &sc->done));
    mf_count_launches(2);
    cg_pap<double><<<kRedBlocks, kRedThreads, 0, s>>>(n, in, wv, partials, sc);
  }
  cgp_update<double><<<kRedBlocks, kRedThreads, 0, s>>>(n, x, r, u, p, sv, wv, invdiag, partials, sc);
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

// Run the CG loop that cg_init prepared: blocks of `k` iterations (graph or plain launches),
// host reads the done flag after each block.
using IterFn = std::function<mf_status(cudaStream_t)>;

template <typename R>
mf_status cg_loop(CgWorkspace *w, int slot, const CgWorkspace::Key &key, const OpFn &op, const OpDotFn &opdot, int64_t n, R *x,
                  R *r, R *p, R *Ap,
                  const double *invdiag, CgScalars *sc, int k, bool use_graph, double deadline_s,
                  std::chrono::steady_clock::time_point t0, cudaStream_t s, CgScalars *host,
                  const IterFn &iter = IterFn()) {
  auto body = [&](cudaStream_t st) -> mf_status {
    for (int it = 0; it < k; ++it) {
      if (iter) MF_TRY(iter(st));
      else MF_TRY(cg_iteration<R>(op, opdot, n, x, r, p, Ap, invdiag, w->partials, sc, st));
    }
    return MF_OK;
  };
  CgWorkspace::Graph &g = w->g[slot];
  if (use_graph && (g.exec == nullptr || !(g.key == key))) {
    if (g.exec) {
      cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
    }
    cudaGraph_t graph;
    MF_CUDA(cudaStreamBeginCapture(w->cap, cudaStreamCaptureModeThreadLocal));
    const int64_t before = mf_launches_now();
    mf_status st = body(w->cap);
    g.kernels = mf_launches_now() - before;
    mf_count_launches(-g.kernels);  // captured, not launched: counted per replay below
    cudaError_t ce = cudaStreamEndCapture(w->cap, &graph);
    if (st != MF_OK) return st;
    if (ce != cudaSuccess) {
      mf_set_error("CG graph capture failed: %s", cudaGetErrorString(ce));
      return MF_ERR_CUDA;
    }
    ce = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      g.exec = nullptr;
      mf_set_error("CG graph instantiation failed: %s", cudaGetErrorString(ce));
      return MF_ERR_CUDA;
    }
    g.key = key;
  }
  for (;;) {
    MF_RANGE("mf_cg_block");
    if (use_graph) {
      MF_CUDA(cudaGraphLaunch(g.exec, s));
      mf_count_launches(g.kernels);
    }
    else MF_TRY(body(s));
    MF_CUDA(cudaMemcpyAsync(host, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    MF_CUDA(cudaStreamSynchronize(s));
    if (host->done) return MF_OK;
    if (deadline_s > 0) {
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el > deadline_s) {
        mf_set_error("mf_cg_solve: timeout after %.3f s (%d iterations)", el, host->iter);
        return MF_ERR_TIMEOUT;
      }
    }
  }
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// Flexible CG with the learned preconditioner (MF_PC_LEARNED).  The preconditioner z = M(r) changes
// with r (a network), so beta uses the Polak-Ribiere form z_{k+1}.(r_{k+1} - r_k) / (z_k.r_k)
// (Notay, SIAM J. Sci. Comput. 22, 2000).  If the residual stops improving (no new best over 500
// iterations) or a breakdown appears, the network is switched off and the solve restarts as
// Jacobi-preconditioned CG from the current iterate.  M is a two-level preconditioner with the network as the
// correction of smooth errors between damped-Jacobi smoothing steps (omega = 2/3, D = diag(A)):
//   z1 = omega D^-1 r;  r1 = r - A z1;  cn = D^-1/2 (s/c) NN(D^-1/2 r1 / s, log kappa), s = RMS(D^-1/2 r1);
//   z2 = z1 + theta cn with the energy-norm step theta = max(0, cn.r1 / cn.A cn) (a useless or harmful
//   correction gets theta ~ 0);  z = z2 + omega D^-1 (r - A z2).
// c is the network's output scale; z = 0 on Dirichlet DoFs.  The FP64 CG stays the fallback and
// what decides convergence (the true residual is recomputed at the end).
// ------------------------------------------------------------------------------------------------
extern "C" mf_status mf_net_forward(mf_net *N, const float *r, const float *logk, float *out, mf_stream stream);
int64_t net_nodes(const mf_net *N);
const int *net_dims(const mf_net *N);
float net_out_scale(const mf_net *N);

namespace {

__global__ void __launch_bounds__(kRedThreads) dot2_kernel(int64_t n, const double *a, const double *b, const double *c,
                                                           const double *d, double *partials, CgScalars *sc, double *out) {
  double v[2] = {0.0, 0.0};
  GRID_STRIDE(i, n) {
    v[0] += a[i] * b[i];
    if (c) v[1] += c[i] * d[i];
  }
  double o[2];
  if (grid_reduce<2>(v, partials, &sc->ticket, o) && threadIdx.x == 0) {
    out[0] = o[0];
    if (c) out[1] = o[1];  // single dots write one scalar only
  }
}

// ||D^{-1/2} r||^2 into *out (isd = D^{-1/2})
__global__ void __launch_bounds__(kRedThreads) scaled_norm2(int64_t n, const double *r, const double *isd,
                                                            double *partials, CgScalars *sc, double *out) {
  double v[1] = {0.0};
  GRID_STRIDE(i, n) {
    const double t = r[i] * isd[i];
    v[0] += t * t;
  }
  double o[1];
  if (grid_reduce<1>(v, partials, &sc->ticket, o) && threadIdx.x == 0) out[0] = o[0];
}

// rhat = D^{-1/2} r / s (FP32), s = RMS of D^{-1/2} r from ss = ||D^{-1/2} r||^2
__global__ void scale_to_f32(int64_t n, const double *r, const double *isd, const double *ss, float *out) {
  // one FP64 division per thread, not per node: GB300's FP64 divide is a long sequence on its narrow
  // FP64 pipe (the output is rounded to FP32, far coarser than the reciprocal's rounding)
  const double is = 1.0 / sqrt(fmax(*ss, 1e-300) / (double)n);
  GRID_STRIDE(i, n) out[i] = (float)(r[i] * isd[i] * is);
}

// z = beta z + omega D^{-1} r (damped Jacobi step; beta = 0 starts z), zero on Dirichlet nodes
__global__ void jacobi_step(int64_t n, const double *r, const double *isd, double omega, double beta,
                            const uint8_t *dmask, double *z) {
  GRID_STRIDE(i, n) {
    const double d = omega * isd[i] * isd[i] * r[i];
    z[i] = dmask[i] ? 0.0 : (beta == 0.0 ? d : z[i] + d);
  }
}

// out = r - t
__global__ void sub_to(int64_t n, const double *r, const double *t, double *out) {
  GRID_STRIDE(i, n) out[i] = r[i] - t[i];
}

// c = D^{-1/2} (s / c_out) zf (network correction), zero on Dirichlet nodes
__global__ void net_correction(int64_t n, const float *zf, const double *isd, const double *ss, double c_out,
                               const uint8_t *dmask, double *c) {
  const double s = sqrt(fmax(*ss, 1e-300) / (double)n) / c_out;
  GRID_STRIDE(i, n) c[i] = dmask[i] ? 0.0 : isd[i] * s * (double)zf[i];
}

// energy-norm step for the correction: theta = max(0, c.r1 / c.Ac); z += theta c; r1 -= theta Ac
__global__ void theta_update(int64_t n, const double *num_den, const double *c, const double *Ac, double *z,
                             double *r1) {
  const double den = num_den[1];
  const double th = den > 0.0 ? fmax(0.0, num_den[0] / den) : 0.0;
  GRID_STRIDE(i, n) {
    z[i] += th * c[i];
    r1[i] -= th * Ac[i];
  }
}

__global__ void sqrt_to(int64_t n, const double *__restrict__ a, double *__restrict__ b) {
  GRID_STRIDE(i, n) b[i] = sqrt(a[i]);
}

// Truncated flexible CG keeps the last kFcgM search directions and their images under A.
constexpr int kFcgM = 8;

struct DirSet {
  const double *v[kFcgM];  // the stored directions (or their images) taking part, cnt of them
  int idx[kFcgM];          // their ring slots (for the stored p.Ap)
  int cnt;
};

// out[j] = z . v_j for the cnt vectors of `vs` (one pass over z)
__global__ void __launch_bounds__(kRedThreads) multi_dot(int64_t n, const double *z, DirSet vs, double *partials,
                                                         CgScalars *sc, double *out) {
  double v[kFcgM];
#pragma unroll
  for (int j = 0; j < kFcgM; ++j) v[j] = 0.0;
  GRID_STRIDE(i, n) {
    const double zi = z[i];
#pragma unroll
    for (int j = 0; j < kFcgM; ++j)
      if (j < vs.cnt) v[j] += zi * vs.v[j][i];
  }
  double o[kFcgM];
  if (grid_reduce<kFcgM>(v, partials, &sc->ticket, o) && threadIdx.x == 0)
    for (int j = 0; j < vs.cnt; ++j) out[j] = o[j];
}

// p = z - sum_j (zAp_j / pAp_j) p_j   (A-orthogonalisation against the stored directions)
__global__ void orthogonalise(int64_t n, const double *z, DirSet ps, const double *zAp, const double *pAp, double *p) {
  double c[kFcgM];
#pragma unroll
  for (int j = 0; j < kFcgM; ++j) c[j] = j < ps.cnt ? zAp[j] / pAp[ps.idx[j]] : 0.0;
  GRID_STRIDE(i, n) {
    double s = z[i];
#pragma unroll
    for (int j = 0; j < kFcgM; ++j)
      if (j < ps.cnt) s -= c[j] * ps.v[j][i];
    p[i] = s;
  }
}

// alpha = (p.r) / (p.Ap); x += alpha p; r -= alpha Ap; pAp is kept for later orthogonalisations
__global__ void fcg_update_xr(int64_t n, double *x, double *r, const double *p, const double *Ap,
                              const double *pAp_pr, double *pAp_keep) {
  const double alpha = pAp_pr[1] / pAp_pr[0];
  if (blockIdx.x == 0 && threadIdx.x == 0) *pAp_keep = pAp_pr[0];
  GRID_STRIDE(i, n) {
    x[i] += alpha * p[i];
    r[i] -= alpha * Ap[i];
  }
}

// node field of log(kappa): mean of log kappa over the cells touching each node (structured box)
__global__ void node_logk(const double *kappa, int nx, int ny, int nz, float *out) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t N = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  if (n >= N) return;
  const int i = (int)(n % (nx + 1)), j = (int)((n / (nx + 1)) % (ny + 1)), k = (int)(n / ((int64_t)(nx + 1) * (ny + 1)));
  double s = 0.0;
  int c = 0;
  for (int dk = -1; dk <= 0; ++dk)
    for (int dj = -1; dj <= 0; ++dj)
      for (int di = -1; di <= 0; ++di) {
        const int ex = i + di, ey = j + dj, ez = k + dk;
        if (ex < 0 || ey < 0 || ez < 0 || ex >= nx || ey >= ny || ez >= nz) continue;
        s += log(kappa[ex + (int64_t)nx * (ey + (int64_t)ny * ez)]);
        ++c;
      }
  out[n] = (float)(s / c);
}

struct FcgBufs {
  double *z, *dev, *isd, *t, *r1, *cn, *P, *AP, *pAp, *part;  // P, AP: kFcgM stored directions and images
  float *rf, *zf, *logk;
};

mf_status fcg_solve(mf_mesh *m, const mf_solve_opts *o, const double *b, double *x, mf_solve_info *info,
                    cudaStream_t s, std::chrono::steady_clock::time_point t0) {
  const mf_net *net = o->net;
  MF_ARG(net != nullptr, "mf_cg_solve: MF_PC_LEARNED needs opts->net");
  MF_ARG(m->physics == MF_LAPLACE && m->structured, "mf_cg_solve: MF_PC_LEARNED needs a structured Laplace mesh");
  const int *nd = net_dims(net);
  MF_ARG(nd[0] == m->nx + 1 && nd[1] == m->ny + 1 && nd[2] == m->nz + 1,
         "mf_cg_solve: the network was created for a different node grid");
  MF_TRY(ensure_invdiag(m, s));
  CgWorkspace *w = m->cg;
  const int64_t n = m->n_dof;
  FcgBufs f{};
  auto release = [&]() {
    cudaFree(f.z); cudaFree(f.dev); cudaFree(f.rf); cudaFree(f.zf); cudaFree(f.logk); cudaFree(f.isd);
    cudaFree(f.t); cudaFree(f.r1); cudaFree(f.cn); cudaFree(f.P); cudaFree(f.AP); cudaFree(f.pAp); cudaFree(f.part);
  };
  {
    cudaError_t e = cudaSuccess;
    auto alloc = [&](auto **ptr, size_t bytes) {
      if (e == cudaSuccess) e = cudaMalloc((void **)ptr, bytes);
    };
    alloc(&f.z, n * sizeof(double));
    alloc(&f.dev, 32 * sizeof(double));
    alloc(&f.rf, n * sizeof(float));
    alloc(&f.zf, n * sizeof(float));
    alloc(&f.logk, n * sizeof(float));
    alloc(&f.isd, n * sizeof(double));
    alloc(&f.t, n * sizeof(double));
    alloc(&f.r1, n * sizeof(double));
    alloc(&f.cn, n * sizeof(double));
    alloc(&f.P, (size_t)kFcgM * n * sizeof(double));
    alloc(&f.AP, (size_t)kFcgM * n * sizeof(double));
    alloc(&f.pAp, kFcgM * sizeof(double));
    alloc(&f.part, (size_t)kFcgM * kRedBlocks * sizeof(double));
    if (e != cudaSuccess) {
      release();
      cudaGetLastError();
      mf_set_error("mf_cg_solve: out of device memory for the flexible CG workspace");
      return MF_ERR_OOM;
    }
  }
  mf_count_launches(2);
  node_logk<<<blocks_for(n), kThreads, 0, s>>>(m->mat, m->nx, m->ny, m->nz, f.logk);
  sqrt_to<<<kRedBlocks, kRedThreads, 0, s>>>(n, w->invdiag, f.isd);  // D^-1/2
  const double c_out = (double)net_out_scale(net);
  bool learned = true;
  int fallback_at = -1;
  // dev: [0] r.r  [2] p.Ap  [3] p.r  [5] |D^-1/2 r1|^2  [6] cn.r1  [7] cn.A cn  [8..8+kFcgM) z.Ap_j
  auto dot2 = [&](const double *a, const double *bb, const double *c, const double *d, double *out) {
    mf_count_launches(1);
    dot2_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(n, a, bb, c, d, w->partials, w->sc, out);
  };
  auto precond = [&](const double *r, double *z) -> mf_status {
    const double omega = 2.0 / 3.0;
    if (!learned) {  // after the switch-off: Jacobi (z = D^-1 r)
      mf_count_launches(1);
      jacobi_step<<<kRedBlocks, kRedThreads, 0, s>>>(n, r, f.isd, 1.0, 0.0, m->dmask, z);
      return MF_OK;
    }
    // two-level form: damped-Jacobi pre-smoothing, network correction of the smoothed residual,
    // damped-Jacobi post-smoothing
    mf_count_launches(2);
    jacobi_step<<<kRedBlocks, kRedThreads, 0, s>>>(n, r, f.isd, omega, 0.0, m->dmask, z);
    MF_TRY(apply_fp64(m, z, f.t, s));
    sub_to<<<kRedBlocks, kRedThreads, 0, s>>>(n, r, f.t, f.r1);
    mf_count_launches(3);
    scaled_norm2<<<kRedBlocks, kRedThreads, 0, s>>>(n, f.r1, f.isd, w->partials, w->sc, f.dev + 5);
    scale_to_f32<<<kRedBlocks, kRedThreads, 0, s>>>(n, f.r1, f.isd, f.dev + 5, f.rf);
    MF_TRY(mf_net_forward(const_cast<mf_net *>(net), f.rf, f.logk, f.zf, (mf_stream)s));
    mf_count_launches(1);
    net_correction<<<kRedBlocks, kRedThreads, 0, s>>>(n, f.zf, f.isd, f.dev + 5, c_out, m->dmask, f.cn);
    MF_TRY(apply_fp64(m, f.cn, f.t, s));
    dot2(f.cn, f.r1, f.cn, f.t, f.dev + 6);  // dev[6] = c.r1, dev[7] = c.Ac
    mf_count_launches(2);
    theta_update<<<kRedBlocks, kRedThreads, 0, s>>>(n, f.dev + 6, f.cn, f.t, z, f.r1);
    jacobi_step<<<kRedBlocks, kRedThreads, 0, s>>>(n, f.r1, f.isd, omega, 1.0, m->dmask, z);
    return MF_OK;
  };
  double h[4];
  mf_status st = MF_OK;
  // x = 0, r = b
  MF_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  MF_CUDA(cudaMemcpyAsync(w->r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  dot2(w->r, w->r, nullptr, nullptr, f.dev + 0);
  MF_CUDA(cudaMemcpyAsync(h, f.dev, sizeof(double), cudaMemcpyDeviceToHost, s));
  MF_CUDA(cudaStreamSynchronize(s));
  const double bb = h[0];
  const double tol2 = o->rtol * o->rtol * bb;
  double rr = bb, best = bb, window_start = bb;
  int it = 0, since = 0, cnt = 0, slot = 0;  // cnt stored directions, the next goes to `slot`
  const int window = 500;  // the residual norm of CG is not monotone: judge stalls over long windows
  if (!(bb > 0.0)) {
    release();
    if (info) { info->iters = 0; info->status = bb == 0.0 ? MF_OK : MF_ERR_BREAKDOWN; info->rel_res = 0; info->rel_res_true = 0; }
    return bb == 0.0 ? MF_OK : MF_ERR_BREAKDOWN;
  }
  auto Pv = [&](int j) { return f.P + (size_t)j * n; };
  auto APv = [&](int j) { return f.AP + (size_t)j * n; };
  // switch the network off and restart as Jacobi-preconditioned CG from the current iterate (from
  // x = 0 when the iterate is no longer finite): r = b - A x, no stored directions
  auto restart_jacobi = [&]() -> mf_status {
    learned = false;
    fallback_at = it;
    cnt = 0;
    MF_TRY(apply_fp64(m, x, w->Ap, s));
    mf_count_launches(1);
    residual_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(n, b, w->Ap, w->r, w->partials, w->sc);
    CgScalars hs;
    MF_CUDA(cudaMemcpyAsync(&hs, w->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    MF_CUDA(cudaStreamSynchronize(s));
    if (!std::isfinite(hs.res2)) {
      MF_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
      MF_CUDA(cudaMemcpyAsync(w->r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      rr = bb;
    } else {
      rr = hs.res2;
    }
    return MF_OK;
  };
  while (!(rr <= tol2) && it < o->max_iter) {
    st = precond(w->r, f.z);
    if (st != MF_OK) break;
    // new direction: z A-orthogonalised against the last cnt directions
    double *p = Pv(slot), *Ap = APv(slot);
    if (cnt == 0) {
      MF_CUDA(cudaMemcpyAsync(p, f.z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else {
      DirSet aps{}, ps{};
      for (int j = 0; j < cnt; ++j) {
        const int sj = (slot - 1 - j + kFcgM) % kFcgM;
        aps.v[j] = APv(sj);
        ps.v[j] = Pv(sj);
        aps.idx[j] = ps.idx[j] = sj;
      }
      aps.cnt = ps.cnt = cnt;
      mf_count_launches(2);
      multi_dot<<<kRedBlocks, kRedThreads, 0, s>>>(n, f.z, aps, f.part, w->sc, f.dev + 8);
      orthogonalise<<<kRedBlocks, kRedThreads, 0, s>>>(n, f.z, ps, f.dev + 8, f.pAp, p);
    }
    MF_TRY(apply_fp64(m, p, Ap, s));
    dot2(p, Ap, p, w->r, f.dev + 2);  // dev[2] = p.Ap, dev[3] = p.r
    mf_count_launches(1);
    fcg_update_xr<<<kRedBlocks, kRedThreads, 0, s>>>(n, x, w->r, p, Ap, f.dev + 2, f.pAp + slot);
    dot2(w->r, w->r, nullptr, nullptr, f.dev + 0);
    ++it;
    MF_CUDA(cudaMemcpyAsync(h, f.dev, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    MF_CUDA(cudaStreamSynchronize(s));
    rr = h[0];
    if (!std::isfinite(rr) || !(h[2] > 0.0)) {
      if (!learned) { st = MF_ERR_BREAKDOWN; break; }
      MF_TRY(restart_jacobi());  // breakdown with the network: Jacobi-PCG from here
      continue;
    }
    slot = (slot + 1) % kFcgM;
    cnt = cnt < kFcgM ? cnt + 1 : kFcgM;
    if (rr <= tol2) break;
    if (o->timeout_s > 0 && std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > o->timeout_s) {
      st = MF_ERR_TIMEOUT;
      break;
    }
    if (learned) {
      if (rr < best) best = rr;
      if (++since >= window) {
        if (best >= 0.98 * window_start) {  // no new best residual over the whole window
          MF_TRY(restart_jacobi());
          continue;
        }
        window_start = best;
        since = 0;
      }
    }
  }
  if (st == MF_OK && !(rr <= tol2)) st = std::isfinite(rr) ? MF_NOT_CONVERGED : MF_ERR_BREAKDOWN;
  // true residual
  MF_TRY(apply_fp64(m, x, w->Ap, s));
  mf_count_launches(1);
  residual_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(n, b, w->Ap, nullptr, w->partials, w->sc);
  CgScalars hs;
  MF_CUDA(cudaMemcpyAsync(&hs, w->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
  MF_CUDA(cudaStreamSynchronize(s));
  release();
  if (info) {
    info->iters = it;
    info->outer_iters = fallback_at;  // iteration at which the network was switched off, -1 if never
    info->status = st;
    info->rel_res = std::sqrt(rr / bb);
    info->rel_res_true = std::sqrt(hs.res2 / bb);
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (st == MF_NOT_CONVERGED) mf_set_error("mf_cg_solve: not converged within the iteration limit");
  if (st == MF_ERR_BREAKDOWN) mf_set_error("mf_cg_solve: breakdown");
  return st;
}

}  // namespace

extern "C" void mf_solve_opts_default(mf_solve_opts *o) {
  if (!o) return;
  o->op = MF_OP_MATFREE;
  o->precision = MF_PREC_FP64;
  o->precond = MF_PC_NONE;
  o->max_iter = 100000;
  o->rtol = 1e-8;
  o->check_every = 32;
  o->use_graph = 1;
  o->timeout_s = 0.0;
  o->inner_rtol = 1e-4;
  o->max_outer = 50;
  o->csr = nullptr;
  o->net = nullptr;
  o->recurrence = MF_CG_CLASSIC;
}

namespace {

// Host layout of a CG checkpoint: this header, then x, r and the search direction (n doubles each).
struct CgStateHeader {
  uint64_t magic;
  int64_t n;
  int32_t fused;     // 1: fused classic iteration (direction p_{k-1}); 0: split kernels
  int32_t precond;   // MF_PC_NONE or MF_PC_JACOBI
  int32_t iter;      // k
  int32_t p_is_new;  // split kernels: the direction is already p_k
  double rz, rr, bb, beta;
};
constexpr uint64_t kStateMagic = 0x3174537447436d66ull;  // "mfCGtSt1"

// Puts a checkpoint's vectors and scalars into the workspace in place of cg_init: x, r, the direction
// (into `p`), and the device scalars (alpha = 0: the state's x already holds every update).
mf_status restore_state(CgWorkspace *w, const CgStateHeader &h, const double *vecs, double *p, double rtol,
                        int max_iter, cudaStream_t s) {
  const size_t nb = (size_t)h.n * sizeof(double);
  MF_CUDA(cudaMemcpyAsync(w->x, vecs, nb, cudaMemcpyHostToDevice, s));
  MF_CUDA(cudaMemcpyAsync(w->r, vecs + h.n, nb, cudaMemcpyHostToDevice, s));
  MF_CUDA(cudaMemcpyAsync(p, vecs + 2 * h.n, nb, cudaMemcpyHostToDevice, s));
  CgScalars c{};
  c.bb = h.bb;
  c.rr = h.rr;
  c.rz = h.rz;
  c.beta = h.beta;
  c.tol2 = rtol * rtol * h.bb;  // as cg_init forms it
  c.iter = h.iter;
  c.max_iter = max_iter;
  c.done = h.iter >= max_iter ? 1 : 0;
  c.status = c.done ? MF_NOT_CONVERGED : 0;
  MF_CUDA(cudaStreamSynchronize(s));  // h_sc may still be read by an earlier copy on this stream
  w->h_sc[0] = c;
  MF_CUDA(cudaMemcpyAsync(w->sc, w->h_sc, sizeof(CgScalars), cudaMemcpyHostToDevice, s));
  return MF_OK;
}

// rs: a checkpoint's header to resume from (null: a new solve), rv: its vectors x, r, direction.
mf_status cg_solve_impl(mf_mesh *m, const mf_solve_opts *o, const double *b, double *x, mf_solve_info *info,
                        cudaStream_t stream, const CgStateHeader *rs, const double *rv);

}  // namespace

extern "C" mf_status mf_cg_solve(mf_mesh *m, const mf_solve_opts *o, const double *b, double *x, mf_solve_info *info,
                                 mf_stream stream) {
  MF_RANGE("mf_cg_solve");
  mf_clear_error();
  return cg_solve_impl(m, o, b, x, info, (cudaStream_t)stream, nullptr, nullptr);
}

extern "C" size_t mf_cg_state_bytes(const mf_mesh *m) {
  return m ? sizeof(CgStateHeader) + 3 * (size_t)m->n_dof * sizeof(double) : 0;
}

extern "C" mf_status mf_cg_state_save(mf_mesh *m, void *host_state, size_t bytes, mf_stream stream) {
  MF_RANGE("mf_cg_state_save");
  mf_clear_error();
  MF_ARG(m && host_state, "mf_cg_state_save: null argument");
  MF_ARG(bytes >= mf_cg_state_bytes(m), "mf_cg_state_save: %zu bytes given, %zu needed", bytes, mf_cg_state_bytes(m));
  CgWorkspace *w = m->cg;
  MF_ARG(w && w->last_fused >= 0 && (w->last_status == MF_NOT_CONVERGED || w->last_status == MF_ERR_TIMEOUT),
         "mf_cg_state_save: no stopped classic FP64 CG solve on this mesh to save");
  cudaStream_t s = (cudaStream_t)stream;
  CgScalars c;
  MF_CUDA(cudaMemcpyAsync(w->h_sc, w->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
  MF_CUDA(cudaStreamSynchronize(s));
  c = w->h_sc[0];
  CgStateHeader h{};
  h.magic = kStateMagic;
  h.n = m->n_dof;
  h.fused = w->last_fused;
  h.precond = w->last_precond;
  h.iter = c.iter;
  h.p_is_new = w->last_p_new ? 1 : 0;
  h.rz = c.rz;
  h.rr = c.rr;
  h.bb = c.bb;
  h.beta = c.beta;
  std::memcpy(host_state, &h, sizeof h);
  double *v = reinterpret_cast<double *>(static_cast<char *>(host_state) + sizeof h);
  const size_t nb = (size_t)m->n_dof * sizeof(double);
  MF_CUDA(cudaMemcpyAsync(v, w->x, nb, cudaMemcpyDeviceToHost, s));
  MF_CUDA(cudaMemcpyAsync(v + m->n_dof, w->r, nb, cudaMemcpyDeviceToHost, s));
  MF_CUDA(cudaMemcpyAsync(v + 2 * m->n_dof, w->last_p, nb, cudaMemcpyDeviceToHost, s));
  MF_CUDA(cudaStreamSynchronize(s));
  return MF_OK;
}

extern "C" mf_status mf_cg_resume(mf_mesh *m, const mf_solve_opts *o, const void *host_state, size_t bytes,
                                  const double *b, double *x, mf_solve_info *info, mf_stream stream) {
  MF_RANGE("mf_cg_resume");
  mf_clear_error();
  MF_ARG(m && o && host_state && b && x, "mf_cg_resume: null argument");
  MF_ARG(bytes >= sizeof(CgStateHeader), "mf_cg_resume: state too small");
  CgStateHeader h;
  std::memcpy(&h, host_state, sizeof h);
  MF_ARG(h.magic == kStateMagic && h.n == m->n_dof && bytes >= mf_cg_state_bytes(m) && h.iter >= 0 &&
             (h.fused == 0 || h.fused == 1),
         "mf_cg_resume: the state does not belong to this mesh (or is corrupt)");
  MF_ARG(o->precision == MF_PREC_FP64, "mf_cg_resume: FP64 solves only");
  MF_ARG(o->precond == h.precond, "mf_cg_resume: the state was written with preconditioner %d", h.precond);
  MF_ARG(o->recurrence == MF_CG_CLASSIC || o->recurrence == MF_CG_CLASSIC_SPLIT,
         "mf_cg_resume: the classic recurrence only");
  const double *vecs = reinterpret_cast<const double *>(static_cast<const char *>(host_state) + sizeof h);
  return cg_solve_impl(m, o, b, x, info, (cudaStream_t)stream, &h, vecs);
}

namespace {

mf_status cg_solve_impl(mf_mesh *m, const mf_solve_opts *o, const double *b, double *x, mf_solve_info *info,
                        cudaStream_t stream, const CgStateHeader *rs, const double *rv) {
  const auto t0 = std::chrono::steady_clock::now();
  MF_ARG(m && o && b && x, "mf_cg_solve: null argument");
  MF_ARG(o->op == MF_OP_MATFREE || o->op == MF_OP_CSR, "mf_cg_solve: unknown op %d", o->op);
  MF_ARG(o->op == MF_OP_MATFREE || o->csr != nullptr, "mf_cg_solve: op CSR needs opts->csr");
  MF_ARG(o->op == MF_OP_MATFREE || o->csr->n_rows == m->n_dof, "mf_cg_solve: CSR size does not match the mesh");
  MF_ARG(o->precision == MF_PREC_FP64 || o->precision == MF_PREC_MIXED_IR, "mf_cg_solve: unknown precision");
  MF_ARG(o->precond == MF_PC_NONE || o->precond == MF_PC_JACOBI || o->precond == MF_PC_LEARNED,
         "mf_cg_solve: unknown preconditioner");
  if (o->precond == MF_PC_LEARNED) {
    MF_ARG(o->precision == MF_PREC_FP64 && o->op == MF_OP_MATFREE, "mf_cg_solve: MF_PC_LEARNED is FP64 matrix-free");
    MF_ARG(o->recurrence == MF_CG_CLASSIC, "mf_cg_solve: MF_PC_LEARNED runs flexible CG (classic recurrence only)");
    return fcg_solve(m, o, b, x, info, (cudaStream_t)stream, t0);
  }
  MF_ARG(o->recurrence == MF_CG_CLASSIC || o->recurrence == MF_CG_PIPELINED || o->recurrence == MF_CG_CLASSIC_SPLIT,
         "mf_cg_solve: unknown recurrence %d", o->recurrence);
  MF_ARG(o->recurrence == MF_CG_CLASSIC || o->precision == MF_PREC_FP64,
         "mf_cg_solve: the pipelined and split recurrences are FP64 (MIXED_IR uses the classic one)");
  MF_ARG(o->precision == MF_PREC_FP64 || o->precond == MF_PC_NONE, "mf_cg_solve: MIXED_IR takes no preconditioner");
  MF_ARG(o->precision == MF_PREC_FP64 || o->op == MF_OP_MATFREE, "mf_cg_solve: MIXED_IR needs the matrix-free operator");
  MF_ARG(o->max_iter > 0 && o->rtol > 0 && o->check_every > 0, "mf_cg_solve: bad max_iter/rtol/check_every");
  cudaStream_t s = (cudaStream_t)stream;
  const bool mixed = o->precision == MF_PREC_MIXED_IR;
  const bool jac = o->precond == MF_PC_JACOBI;
  MF_TRY(ensure_workspace(m, mixed, jac));
  CgWorkspace *w = m->cg;
  w->last_fused = -1;  // until this solve stops with a state to save
  const int64_t n = m->n_dof;
  if (jac) MF_TRY(ensure_invdiag(m, s));
  const mf_csr *A = o->csr;
  OpFn op64 = [m, A, o](const void *in, void *out, cudaStream_t st, const int *skip) -> mf_status {
    if (o->op == MF_OP_CSR) return spmv(A, (const double *)in, (double *)out, st, skip);
    return apply_fp64(m, (const double *)in, (double *)out, st, skip);
  };
  OpFn op32 = [m](const void *in, void *out, cudaStream_t st, const int *skip) -> mf_status {
    return apply_fp32(m, (const float *)in, (float *)out, st, skip);
  };
  // tensor-product meshes with the auto variant: p . Ap fused into the face-marching apply
  const bool fuse = m->tp && m->variant == MF_VARIANT_AUTO && w->dotp != nullptr;
  OpDotFn opdot64, opdot32;
  if (fuse && o->op == MF_OP_MATFREE)
    opdot64 = [m, w](const void *in, void *out, cudaStream_t st, const int *skip, double *dot) -> mf_status {
      return tile_apply_dot_fp64(m, (const double *)in, (double *)out, st, skip, w->dotp, w->dticket, dot);
    };
  if (fuse)
    opdot32 = [m, w](const void *in, void *out, cudaStream_t st, const int *skip, double *dot) -> mf_status {
      return tile_apply_dot_fp32(m, (const float *)in, (float *)out, st, skip, w->dotp, w->dticket, dot);
    };
  CgWorkspace::Key key64;
  key64.op = o->op;
  key64.precond = o->precond;
  key64.variant = m->variant;
  key64.check_every = o->check_every;
  key64.recurrence = o->recurrence;
  key64.precision = MF_PREC_FP64;
  key64.csr_id = o->op == MF_OP_CSR ? A->id : 0;
  CgWorkspace::Key key32;
  key32.op = MF_OP_MATFREE;
  key32.precond = MF_PC_NONE;
  key32.variant = m->variant;
  key32.check_every = o->check_every;
  key32.recurrence = MF_CG_CLASSIC;
  key32.precision = MF_PREC_MIXED_IR;
  mf_status st = MF_OK;
  int iters = 0, outer = 0;
  double rel_rec = 0.0;
  CgScalars *h = w->h_sc;
  if (!mixed && o->recurrence == MF_CG_PIPELINED) {
    if (!w->s) MF_CUDA(cudaMalloc(&w->s, n * sizeof(double)));
    if (jac && !w->u) MF_CUDA(cudaMalloc(&w->u, n * sizeof(double)));
    double *u = jac ? w->u : nullptr;
    const double *idg = jac ? w->invdiag : nullptr;
    mf_count_launches(1);
    cgp_init<double><<<kRedBlocks, kRedThreads, 0, s>>>(n, b, w->x, w->r, u, w->p, w->s, idg, w->partials, w->sc,
                                                       o->rtol, o->max_iter);
    MF_CUDA(cudaGetLastError());
    IterFn iter = [&](cudaStream_t st) {
      return cgp_iteration(op64, opdot64, n, w->x, w->r, u, w->p, w->s, w->Ap, idg, w->partials, w->sc, st);
    };
    st = cg_loop<double>(w, 0, key64, op64, opdot64, n, w->x, w->r, w->p, w->Ap, idg, w->sc, o->check_every,
                         o->use_graph != 0, o->timeout_s, t0, s, h, iter);
    if (st != MF_OK && st != MF_ERR_TIMEOUT) return st;
    if (st == MF_OK) st = (mf_status)h->status;
    iters = h->iter;
    rel_rec = h->bb > 0 ? std::sqrt(h->rr / h->bb) : 0.0;
  } else if (!mixed && o->recurrence == MF_CG_CLASSIC && fuse && o->op == MF_OP_MATFREE && m->dw_oscale == 0 &&
             m->physics == MF_LAPLACE) {
    // scalar Laplace only: with three components per node (elasticity, vector Laplace) the fused
    // kernel's extra staging cost more than the vector kernels it saves (elasticity 160^3: 0.652
    // against 0.635 ms per iteration, with Jacobi 0.719 against 0.666 ms)
    MF_ARG(!rs || rs->fused == 1, "mf_cg_resume: the state was written by the split kernels (MF_CG_CLASSIC_SPLIT)");
    // classic recurrence with the p and x updates in the apply: per iteration the fused apply (and its
    // range fix-up) and the r update.  p_k alternates between w->p (even k) and w->p2 (odd k); a graph
    // holds an even number of iterations, so that each replay starts on an even k.
    if (!w->p2) MF_CUDA(cudaMalloc(&w->p2, n * sizeof(double)));
    const double *idg = jac ? w->invdiag : nullptr;
    if (rs) {
      // the state's p_{k-1} and beta_{k-1} with alpha = 0 (x_k is complete): the first apply forms p_k
      MF_TRY(restore_state(w, *rs, rv, w->p2, o->rtol, o->max_iter, s));
    } else {
      mf_count_launches(1);
      // p_{-1} = z_0 with beta_{-1} = 0 and alpha_{-1} = 0: the first apply forms p_0 = z_0, leaves x = 0
      cg_init<double><<<kRedBlocks, kRedThreads, 0, s>>>(n, b, w->x, w->r, w->p2, idg, w->partials, w->sc, o->rtol,
                                                        o->max_iter);
      MF_CUDA(cudaGetLastError());
    }
    const int iter0 = rs ? rs->iter : 0;
    int pos = 0;
    IterFn iter = [&](cudaStream_t st) -> mf_status {
      double *pn = (pos & 1) ? w->p2 : w->p, *po = (pos & 1) ? w->p : w->p2;
      ++pos;
      MF_TRY(tile_apply_cg_fp64(m, w->r, po, idg, pn, w->x, w->Ap, &w->sc->alpha, st, &w->sc->done, w->dotp,
                                w->dticket, &w->sc->pAp));
      mf_count_launches(1);
      cg_update_xr<double, false><<<kRedBlocks, kRedThreads, 0, st>>>(n, nullptr, w->r, nullptr, w->Ap, idg, w->partials,
                                                               w->sc);
      MF_CUDA(cudaGetLastError());
      return MF_OK;
    };
    const int kb = o->check_every % 2 ? 2 * o->check_every : o->check_every;
    st = cg_loop<double>(w, 0, key64, op64, opdot64, n, w->x, w->r, w->p, w->Ap, idg, w->sc, kb, o->use_graph != 0,
                         o->timeout_s, t0, s, h, iter);
    if (st != MF_OK && st != MF_ERR_TIMEOUT) return st;
    mf_count_launches(1);
    cg_flush_x<<<kRedBlocks, kRedThreads, 0, s>>>(n, w->x, w->p, w->p2, w->sc, iter0);
    MF_CUDA(cudaGetLastError());
    if (st == MF_OK) st = (mf_status)h->status;
    iters = h->iter;
    rel_rec = h->bb > 0 ? std::sqrt(h->rr / h->bb) : 0.0;
    // the last direction: written by the apply of position iters - iter0 - 1 (the old buffer of
    // position 0 when no iteration ran)
    const int npos = iters - iter0;
    w->last_p = npos <= 0 ? w->p2 : (((npos - 1) & 1) ? w->p2 : w->p);
    w->last_p_new = false;
    w->last_fused = 1;
    w->last_status = st;
    w->last_precond = o->precond;
  } else if (!mixed) {
    MF_ARG(!rs || rs->fused == 0, "mf_cg_resume: the state was written by the fused iteration (MF_CG_CLASSIC)");
    if (rs) {
      MF_TRY(restore_state(w, *rs, rv, w->p, o->rtol, o->max_iter, s));
      if (!rs->p_is_new) {  // the solve stopped before its p update: p_k = z_k + beta_{k-1} p_{k-1}
        mf_count_launches(1);
        cg_update_p<double><<<kRedBlocks, kRedThreads, 0, s>>>(n, w->r, w->p, jac ? w->invdiag : nullptr, w->sc);
        MF_CUDA(cudaGetLastError());
      }
    } else {
      mf_count_launches(1);
      cg_init<double><<<kRedBlocks, kRedThreads, 0, s>>>(n, b, w->x, w->r, w->p, jac ? w->invdiag : nullptr,
                                                        w->partials, w->sc, o->rtol, o->max_iter);
      MF_CUDA(cudaGetLastError());
    }
    st = cg_loop<double>(w, 0, key64, op64, opdot64, n, w->x, w->r, w->p, w->Ap, jac ? w->invdiag : nullptr, w->sc,
                         o->check_every, o->use_graph != 0, o->timeout_s, t0, s, h);
    if (st != MF_OK && st != MF_ERR_TIMEOUT) return st;
    if (st == MF_OK) st = (mf_status)h->status;
    iters = h->iter;
    rel_rec = h->bb > 0 ? std::sqrt(h->rr / h->bb) : 0.0;
    // a solve stopped by its iteration limit skipped its last p update (done was set); one stopped by
    // the wall clock ended a whole graph block, p update included
    w->last_p = w->p;
    w->last_p_new = !h->done;
    w->last_fused = 0;
    w->last_status = st;
    w->last_precond = o->precond;
  } else {
    // FP64 iterative refinement around an FP32 inner CG: x_{m+1} = x_m + A32^{-1}(b - A64 x_m).
    MF_CUDA(cudaMemsetAsync(w->x, 0, n * sizeof(double), s));
    MF_CUDA(cudaMemcpyAsync(w->r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    mf_count_launches(1);
    residual_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(n, b, w->x, nullptr, w->partials, w->sc);  // ||b||^2 (x = 0)
    MF_CUDA(cudaMemcpyAsync(h, w->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    MF_CUDA(cudaStreamSynchronize(s));
    const double bb = h->res2;
    double rr = bb;
    const double tol2 = o->rtol * o->rtol * bb;
    st = MF_NOT_CONVERGED;
    while (outer < o->max_outer && iters < o->max_iter) {
      if (rr <= tol2) {
        st = MF_OK;
        break;
      }
      mf_count_launches(1);
      to_f32<<<kRedBlocks, kRedThreads, 0, s>>>(n, w->r, w->r32);
      // inner solve A32 d = r32 (b of the inner CG lives in Ap32 so r32 can be the inner residual)
      MF_CUDA(cudaMemcpyAsync(w->Ap32, w->r32, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
      mf_count_launches(1);
      cg_init<float><<<kRedBlocks, kRedThreads, 0, s>>>(n, w->Ap32, w->x32, w->r32, w->p32, nullptr, w->partials,
                                                       w->sc32, o->inner_rtol, o->max_iter - iters);
      MF_CUDA(cudaGetLastError());
      mf_status si = cg_loop<float>(w, 1, key32, op32, opdot32, n, w->x32, w->r32, w->p32, w->Ap32, nullptr, w->sc32,
                                    o->check_every, o->use_graph != 0, o->timeout_s, t0, s, h + 1);
      if (si != MF_OK) {
        st = si;
        break;
      }
      iters += h[1].iter;
      if (h[1].status == MF_ERR_BREAKDOWN) {
        st = MF_ERR_BREAKDOWN;
        break;
      }
      mf_count_launches(1);
      add_f32<<<kRedBlocks, kRedThreads, 0, s>>>(n, w->x, w->x32);
      MF_TRY(apply_fp64(m, w->x, w->Ap, s));
      mf_count_launches(1);
      residual_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(n, b, w->Ap, w->r, w->partials, w->sc);
      MF_CUDA(cudaMemcpyAsync(h, w->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
      MF_CUDA(cudaStreamSynchronize(s));
      rr = h->res2;
      ++outer;
      if (!std::isfinite(rr)) {
        st = MF_ERR_BREAKDOWN;
        break;
      }
    }
    if (st == MF_NOT_CONVERGED && rr <= tol2) st = MF_OK;
    rel_rec = bb > 0 ? std::sqrt(rr / bb) : 0.0;
  }
  // true residual with the FP64 operator of the solve
  MF_CUDA(cudaMemcpyAsync(x, w->x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  MF_TRY(op64(w->x, w->Ap, s, nullptr));
  mf_count_launches(1);
  residual_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(n, b, w->Ap, nullptr, w->partials, w->sc);
  MF_CUDA(cudaGetLastError());
  MF_CUDA(cudaMemcpyAsync(h, w->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
  MF_CUDA(cudaStreamSynchronize(s));
  const double res2 = h->res2;
  double bb = h->bb;
  if (mixed || bb == 0.0) {
    // ||b||^2 = ||b - 0||^2 (the FP64 scalars of a mixed solve live in the refinement loop)
    MF_CUDA(cudaMemsetAsync(w->Ap, 0, n * sizeof(double), s));
    mf_count_launches(1);
    residual_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(n, b, w->Ap, nullptr, w->partials, w->sc);
    MF_CUDA(cudaMemcpyAsync(h, w->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    MF_CUDA(cudaStreamSynchronize(s));
    bb = h->res2;
  }
  if (info) {
    info->iters = iters;
    info->outer_iters = outer;
    info->status = st;
    info->rel_res = rel_rec;
    info->rel_res_true = bb > 0 ? std::sqrt(res2 / bb) : 0.0;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (st == MF_ERR_BREAKDOWN) mf_set_error("mf_cg_solve: breakdown (p^T A p <= 0 or non-finite scalar)");
  if (st == MF_NOT_CONVERGED) mf_set_error("mf_cg_solve: not converged within the iteration limit");
  return st;
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// Allocation-free CG (mf_cg_solve_noalloc).
//
// Some callers cannot allocate device memory once they are running: applications that reserve the
// whole device for their own memory pool at start-up, or that run under a memory budget enforced
// outside CUDA, and code paths where a cudaMalloc would stall or be forbidden.  For them the
// solver's scratch (three DoF vectors, the block partials of the reductions and the device
// scalars) lives in one fixed-size array with static storage inside this library.  Every GPU that
// loads the library holds the array until the process exits.
// ------------------------------------------------------------------------------------------------
namespace {

constexpr int64_t kNoAllocMaxDof = MF_NOALLOC_MAX_DOF;
constexpr int64_t kNoAllocScalarsDoubles = (sizeof(CgScalars) + sizeof(double) - 1) / sizeof(double);
constexpr int64_t kNoAllocDoubles = 3 * kNoAllocMaxDof + 4 * kRedBlocks + kNoAllocScalarsDoubles;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

constexpr int kMaxDevices = 64;
static double *g_noalloc_ptr[kMaxDevices] = {nullptr};
static std::mutex g_noalloc_mutex;

// Device address of the scratch array on the current device, looked up once per device.  In host
// code the array's name is only a host-side stand-in, so kernels get this address instead.
mf_status noalloc_scratch(double **out) {
  int dev = 0;
  MF_CUDA(cudaGetDevice(&dev));
  MF_ARG(dev >= 0 && dev < kMaxDevices, "mf_cg_solve_noalloc: device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      mf_set_error("mf_cg_solve_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return MF_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = (double *)p;
  }
  *out = g_noalloc_ptr[dev];
  return MF_OK;
}

}  // namespace

extern "C" mf_status mf_cg_solve_noalloc(const mf_mesh *m, const mf_solve_opts *o, const double *b, double *x,
                                         mf_solve_info *info, mf_stream stream) {
  MF_RANGE("mf_cg_solve_noalloc");
  mf_clear_error();
  const auto t0 = std::chrono::steady_clock::now();
  MF_ARG(m && o && b && x, "mf_cg_solve_noalloc: null argument");
  MF_ARG(m->n_dof <= kNoAllocMaxDof, "mf_cg_solve_noalloc: %lld DoFs exceed the fixed scratch limit of %lld DoFs",
         (long long)m->n_dof, (long long)kNoAllocMaxDof);
  MF_ARG(o->op == MF_OP_MATFREE || (o->op == MF_OP_CSR && o->csr != nullptr && o->csr->n_rows == m->n_dof),
         "mf_cg_solve_noalloc: op must be MATFREE, or CSR with a matching opts->csr");
  MF_ARG(o->precision == MF_PREC_FP64 && o->precond == MF_PC_NONE,
         "mf_cg_solve_noalloc: only FP64 without preconditioner is available");
  MF_ARG(o->max_iter > 0 && o->rtol > 0 && o->check_every > 0, "mf_cg_solve_noalloc: bad max_iter/rtol/check_every");
  MF_ARG(o->recurrence == MF_CG_CLASSIC, "mf_cg_solve_noalloc: only the classic recurrence");
  cudaStream_t s = (cudaStream_t)stream;
  double *base = nullptr;
  MF_TRY(noalloc_scratch(&base));
  const int64_t n = m->n_dof;
  double *r = base, *p = base + kNoAllocMaxDof, *Ap = base + 2 * kNoAllocMaxDof;
  double *partials = base + 3 * kNoAllocMaxDof;
  CgScalars *sc = reinterpret_cast<CgScalars *>(partials + 4 * kRedBlocks);
  // the array keeps the previous call's contents: the reduction ticket must start at zero
  MF_CUDA(cudaMemsetAsync(sc, 0, sizeof(CgScalars), s));
  const mf_csr *A = o->csr;
  const bool use_csr = o->op == MF_OP_CSR;
  OpFn op = [m, A, use_csr](const void *in, void *out, cudaStream_t st, const int *skip) -> mf_status {
    if (use_csr) return spmv(A, (const double *)in, (double *)out, st, skip);
    return apply_fp64(m, (const double *)in, (double *)out, st, skip);
  };
  mf_count_launches(1);
  cg_init<double><<<kRedBlocks, kRedThreads, 0, s>>>(n, b, x, r, p, nullptr, partials, sc, o->rtol, o->max_iter);
  MF_CUDA(cudaGetLastError());
  CgScalars h{};
  mf_status st = MF_OK;
  for (;;) {
    for (int it = 0; it < o->check_every; ++it)
      MF_TRY(cg_iteration<double>(op, OpDotFn(), n, x, r, p, Ap, nullptr, partials, sc, s));
    MF_CUDA(cudaMemcpyAsync(&h, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    MF_CUDA(cudaStreamSynchronize(s));
    if (h.done) break;
    if (o->timeout_s > 0 &&
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > o->timeout_s) {
      mf_set_error("mf_cg_solve_noalloc: timeout (%d iterations)", h.iter);
      st = MF_ERR_TIMEOUT;
      break;
    }
  }
  if (st == MF_OK) st = (mf_status)h.status;
  const int iters = h.iter;
  const double bb = h.bb, rr = h.rr;
  // true residual ||b - A x|| with the same operator (Ap is free scratch now)
  MF_TRY(op(x, Ap, s, nullptr));
  mf_count_launches(1);
  residual_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(n, b, Ap, nullptr, partials, sc);
  MF_CUDA(cudaGetLastError());
  MF_CUDA(cudaMemcpyAsync(&h, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
  MF_CUDA(cudaStreamSynchronize(s));
  if (info) {
    info->iters = iters;
    info->outer_iters = 0;
    info->status = st;
    info->rel_res = bb > 0 ? std::sqrt(rr / bb) : 0.0;
    info->rel_res_true = bb > 0 ? std::sqrt(h.res2 / bb) : 0.0;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (st == MF_ERR_BREAKDOWN) mf_set_error("mf_cg_solve_noalloc: breakdown (p^T A p <= 0 or non-finite scalar)");
  if (st == MF_NOT_CONVERGED) mf_set_error("mf_cg_solve_noalloc: not converged within the iteration limit");
  return st;
}

extern "C" mf_status mf_training_pair(mf_mesh *m, const double *b, const double *xs, const double *xk, double *r64,
                                      double *e64, float *r32, float *e32, double *sums, mf_stream stream) {
  MF_RANGE("mf_training_pair");
  mf_clear_error();
  MF_ARG(m && b && xs && xk && r32 && e32, "mf_training_pair: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  MF_TRY(ensure_invdiag(m, s));
  CgWorkspace *w = m->cg;
  const int64_t n = m->n_dof;
  double *r = r64 ? r64 : w->r, *e = e64 ? e64 : w->p;
  MF_TRY(apply_fp64(m, xk, w->Ap, s));
  mf_count_launches(2);
  pair_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(n, m->ndpn, b, w->Ap, xs, xk, w->invdiag, m->dmask, r, e, w->partials,
                                                 w->sc);
  pair_scale<<<kRedBlocks, kRedThreads, 0, s>>>(n, r, e, w->sc, r32, e32);
  MF_CUDA(cudaGetLastError());
  CgScalars h;
  MF_CUDA(cudaMemcpyAsync(&h, w->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
  MF_CUDA(cudaStreamSynchronize(s));
  if (sums) {
    sums[0] = h.res2;
    sums[1] = h.bb;
  }
  return MF_OK;
}

extern "C" mf_status mf_operator_diagonal(const mf_mesh *m, double *diag, mf_stream stream) {
  MF_RANGE("mf_operator_diagonal");
  mf_clear_error();
  MF_ARG(m && diag, "mf_operator_diagonal: null argument");
  return operator_diagonal(m, diag, (cudaStream_t)stream);
}

extern "C" mf_status mf_node_logk(const mf_mesh *m, float *out, mf_stream stream) {
  MF_RANGE("mf_node_logk");
  mf_clear_error();
  MF_ARG(m && out, "mf_node_logk: null argument");
  if (!m->structured || m->physics != MF_LAPLACE || m->npe != 8) {
    mf_set_error("mf_node_logk: scalar Laplace on a structured box only");
    return MF_ERR_UNSUPPORTED;
  }
  mf_count_launches(1);
  node_logk<<<blocks_for(m->n_nodes), kThreads, 0, (cudaStream_t)stream>>>(m->mat, m->nx, m->ny, m->nz, out);
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

MF_DBG_TU(cg)
