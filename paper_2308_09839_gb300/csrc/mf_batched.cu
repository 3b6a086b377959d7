// Batched CG: many independent problems (one mesh each) solved by conjugate gradient in ONE
// persistent, cooperative kernel launch, captured once in a CUDA graph.
//
// The paper solves one problem at a time and leaves kernel fusion of CG undone (Sec. 6).  For a
// batch of small-to-medium problems the per-kernel launch latency and the host round trips of a
// one-at-a-time solve dominate, so here every CTA of a grid sized to be co-resident loops over the
// whole solve: each CG phase (operator apply, p.Ap with alpha, x/r update with r.r, beta and the
// convergence test, p update) is a list of work items over all still-active problems, and phases
// are separated by a grid-wide barrier.  Every problem keeps its own scalars, iteration count and
// convergence flag; a converged problem drops out of the work lists.
//
// Work items: the operator is the face-marching kernel of mf_march.cuh, one item per (tile column,
// z-segment) of each problem; the z-segment length per problem is a tunable (set by
// mf_set_tile_segment, e.g. from an autotuner).  Vector phases use chunks of kChunk DoFs.
// Reductions: each chunk writes a partial, the last chunk of a problem to finish (per-problem
// ticket) sums the partials in chunk order, so results do not depend on scheduling.
//
// Barrier waits are bounded: a CTA that waits longer than the budget sets the error flag and
// every CTA leaves the kernel; the host reports MF_ERR_TIMEOUT.
#include <chrono>
#include <cmath>
#include <vector>

#include "mf_march.cuh"
#include "mf_tile.cuh"

using namespace tile;

namespace {

constexpr int kChunk = 4096;
using Shape = march::MarchShape<MF_LAPLACE, NumDW>;
constexpr int kEX = Shape::EX, kEY = Shape::EY, kThreadsB = kEX * kEY;

struct BScalars {
  double bb, rr, pAp, alpha, beta, tol2;
  int iter, done, status, pad0;
  unsigned int ticket;
  int pad1;
};

struct BProblem {
  TileArgs g;
  int item0, n_items;
  int chunk0, n_chunks;
  int64_t n;
  const double *b;
  double *x, *r, *p, *Ap;
  double *partials;  // [n_chunks]
  BScalars *sc;
};

struct BControl {
  unsigned int count;
  unsigned int gen;
  int err;
  int active;
};

struct BArgs {
  BProblem *probs;
  int n_probs;
  int total_items, total_chunks;
  const int *item_prob, *chunk_prob;
  BControl *ctl;
  long long budget;  // clock cycles a barrier wait may take
  int max_iter;
  double rtol2;      // stop when ||r||^2 <= rtol^2 ||b||^2
};

// Grid-wide barrier with a bounded wait.  Returns false (in every thread) once any CTA has timed out.
__device__ bool grid_barrier(BControl *ctl, long long budget) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int *gen = &ctl->gen;
    volatile int *err = &ctl->err;
    const unsigned int my = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&ctl->count, 1u);
    if (arrived == gridDim.x - 1) {
      ctl->count = 0;
      __threadfence();
      atomicAdd(&ctl->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == my && *err == 0) {
        if (clock64() - t0 > budget) {
          atomicExch(&ctl->err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok = (*err == 0);
  }
  __syncthreads();
  return ok != 0;
}

// Sum over the CTA (fixed shuffle tree, then warps in order); result valid in thread 0.
__device__ double block_sum(double v, double *sh) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
  return s;
}

// Store this chunk's partial; if it is the problem's last chunk to arrive, sum all partials in
// chunk order and return true (total in *out, valid in thread 0 of this CTA).
__device__ bool chunk_reduce(BProblem &P, int lc, double part, double *sh, double *out) {
  __shared__ int last;
  if (threadIdx.x == 0) {
    P.partials[lc] = part;
    __threadfence();
    last = atomicAdd(&P.sc->ticket, 1u) == (unsigned)(P.n_chunks - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double s = 0.0;
  for (int i = threadIdx.x; i < P.n_chunks; i += blockDim.x) s += __ldcg(P.partials + i);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    *out = s;
    P.sc->ticket = 0;
  }
  return true;
}

__global__ void __launch_bounds__(kThreadsB, 4) batched_cg(BArgs A) {
  __shared__ march::MarchSmem<1, NumDW, kEX, kEY> sm;
  __shared__ double sh[kThreadsB / 32];
  const int G = gridDim.x;
  const int tid = threadIdx.x;

  // ---- init: x = 0, r = p = b, ||b||^2
  for (int c = blockIdx.x; c < A.total_chunks; c += G) {
    BProblem P = A.probs[A.chunk_prob[c]];
    const int lc = c - P.chunk0;
    const int64_t i0 = (int64_t)lc * kChunk, i1 = min(i0 + kChunk, P.n);
    double s = 0.0;
    for (int64_t i = i0 + tid; i < i1; i += blockDim.x) {
      const double bi = P.b[i];
      P.x[i] = 0.0;
      P.r[i] = bi;
      P.p[i] = bi;
      s += bi * bi;
    }
    s = block_sum(s, sh);
    double tot;
    if (chunk_reduce(P, lc, s, sh, &tot) && tid == 0) {
      BScalars *sc = P.sc;
      sc->bb = tot;
      sc->rr = tot;
      sc->tol2 = A.rtol2 * tot;
      sc->iter = 0;
      sc->status = isfinite(tot) ? 0 : MF_ERR_BREAKDOWN;
      sc->done = (!isfinite(tot) || tot <= sc->tol2) ? 1 : 0;
      if (sc->done) atomicSub(&A.ctl->active, 1);
    }
  }
  if (!grid_barrier(A.ctl, A.budget)) return;
  for (int it = 0; it < A.max_iter; ++it) {
    if (__ldcg(&A.ctl->active) <= 0) break;
    // ---- A: Ap = A p
    for (int w = blockIdx.x; w < A.total_items; w += G) {
      const BProblem *P = A.probs + A.item_prob[w];
      if (__ldcg(&P->sc->done)) continue;
      const TileArgs g = P->g;
      march::march_item<MF_LAPLACE, NumDW, kEX, kEY, true>(g, w - P->item0, 0, P->p, P->Ap, sm);
    }
    if (!grid_barrier(A.ctl, A.budget)) return;
    // ---- B: pAp, alpha
    for (int c = blockIdx.x; c < A.total_chunks; c += G) {
      BProblem P = A.probs[A.chunk_prob[c]];
      if (__ldcg(&P.sc->done)) continue;
      const int lc = c - P.chunk0;
      const int64_t i0 = (int64_t)lc * kChunk, i1 = min(i0 + kChunk, P.n);
      double s = 0.0;
      for (int64_t i = i0 + tid; i < i1; i += blockDim.x) s += __ldcg(P.p + i) * __ldcg(P.Ap + i);
      s = block_sum(s, sh);
      double pap;
      if (chunk_reduce(P, lc, s, sh, &pap) && tid == 0) {
        BScalars *sc = P.sc;
        sc->pAp = pap;
        if (!(pap > 0.0) || !isfinite(pap)) {
          sc->status = MF_ERR_BREAKDOWN;
          sc->done = 1;
          atomicSub(&A.ctl->active, 1);
        } else {
          sc->alpha = sc->rr / pap;
        }
      }
    }
    if (!grid_barrier(A.ctl, A.budget)) return;
    // ---- C: x += alpha p, r -= alpha Ap, rr, beta, convergence
    for (int c = blockIdx.x; c < A.total_chunks; c += G) {
      BProblem P = A.probs[A.chunk_prob[c]];
      if (__ldcg(&P.sc->done)) continue;
      const double alpha = __ldcg(&P.sc->alpha);
      const int lc = c - P.chunk0;
      const int64_t i0 = (int64_t)lc * kChunk, i1 = min(i0 + kChunk, P.n);
      double s = 0.0;
      for (int64_t i = i0 + tid; i < i1; i += blockDim.x) {
        P.x[i] = __ldcg(P.x + i) + alpha * __ldcg(P.p + i);
        const double ri = __ldcg(P.r + i) - alpha * __ldcg(P.Ap + i);
        P.r[i] = ri;
        s += ri * ri;
      }
      s = block_sum(s, sh);
      double rr;
      if (chunk_reduce(P, lc, s, sh, &rr) && tid == 0) {
        BScalars *sc = P.sc;
        sc->beta = rr / sc->rr;
        sc->rr = rr;
        sc->iter += 1;
        if (!isfinite(rr)) {
          sc->status = MF_ERR_BREAKDOWN;
          sc->done = 1;
        } else if (rr <= sc->tol2) {
          sc->done = 1;
        } else if (sc->iter >= A.max_iter) {
          sc->status = MF_NOT_CONVERGED;
          sc->done = 1;
        }
        if (sc->done) atomicSub(&A.ctl->active, 1);
      }
    }
    if (!grid_barrier(A.ctl, A.budget)) return;
    // ---- D: p = r + beta p
    for (int c = blockIdx.x; c < A.total_chunks; c += G) {
      BProblem P = A.probs[A.chunk_prob[c]];
      if (__ldcg(&P.sc->done)) continue;
      const double beta = __ldcg(&P.sc->beta);
      const int lc = c - P.chunk0;
      const int64_t i0 = (int64_t)lc * kChunk, i1 = min(i0 + kChunk, P.n);
      for (int64_t i = i0 + tid; i < i1; i += blockDim.x) P.p[i] = __ldcg(P.r + i) + beta * __ldcg(P.p + i);
    }
    if (!grid_barrier(A.ctl, A.budget)) return;
  }
}

}  // namespace

struct mf_batch {
  int n = 0;
  int grid = 0;
  std::vector<mf_mesh *> meshes;
  std::vector<BProblem> hprobs;
  BProblem *probs = nullptr;
  BScalars *sc = nullptr;
  BControl *ctl = nullptr;
  double *work = nullptr;
  int *maps = nullptr;
  BArgs args{};
  double rtol = 1e-8;
  int max_iter = 100000;
  double timeout_s = 0.0;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  std::vector<BScalars> hsc;
  int64_t kernels = 0;
};

namespace {

void batch_free(mf_batch *B) {
  if (!B) return;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->cap) cudaStreamDestroy(B->cap);
  cudaFree(B->probs);
  cudaFree(B->sc);
  cudaFree(B->ctl);
  cudaFree(B->work);
  cudaFree(B->maps);
  delete B;
}

}  // namespace

extern "C" mf_status mf_set_tile_segment(mf_mesh *m, int32_t seg) {
  MF_ARG(m != nullptr && seg >= 0, "mf_set_tile_segment: bad argument");
  m->tile_seg = seg;
  return MF_OK;
}

extern "C" mf_status mf_batch_create(mf_mesh *const *meshes, int32_t n, const mf_solve_opts *o, mf_batch **out) {
  MF_RANGE("mf_batch_create");
  mf_clear_error();
  MF_ARG(meshes && o && out && n > 0, "mf_batch_create: bad argument");
  *out = nullptr;
  MF_ARG(o->precision == MF_PREC_FP64 && o->precond == MF_PC_NONE && o->op == MF_OP_MATFREE,
         "mf_batch_create: the batched solver is matrix-free FP64 CG without preconditioner");
  MF_ARG(o->max_iter > 0 && o->rtol > 0, "mf_batch_create: bad max_iter/rtol");
  MF_ARG(o->recurrence == MF_CG_CLASSIC, "mf_batch_create: the batched solver uses the classic recurrence");
  for (int i = 0; i < n; ++i) {
    MF_ARG(meshes[i] != nullptr, "mf_batch_create: mesh %d is NULL", i);
    if (meshes[i]->physics != MF_LAPLACE || !meshes[i]->tp) {
      mf_set_error("mf_batch_create: mesh %d: the batched solver needs Laplace meshes on tensor-product grids", i);
      return MF_ERR_UNSUPPORTED;
    }
  }
  mf_batch *B = new mf_batch();
  B->n = n;
  B->rtol = o->rtol;
  B->max_iter = o->max_iter;
  B->timeout_s = o->timeout_s;
  B->meshes.assign(meshes, meshes + n);
  // work lists
  std::vector<int> item_prob, chunk_prob;
  int64_t total_dof = 0;
  B->hprobs.resize(n);
  for (int i = 0; i < n; ++i) {
    const mf_mesh *m = meshes[i];
    BProblem &P = B->hprobs[i];
    P.g = make_tile_args(m, kEX, kEY, m->tile_seg > 0 ? m->tile_seg : 16);
    P.item0 = (int)item_prob.size();
    P.n_items = tile_items(P.g);
    item_prob.insert(item_prob.end(), P.n_items, i);
    P.n = m->n_dof;
    P.chunk0 = (int)chunk_prob.size();
    P.n_chunks = (int)((P.n + kChunk - 1) / kChunk);
    chunk_prob.insert(chunk_prob.end(), P.n_chunks, i);
    total_dof += P.n;
  }
  const int total_chunks = (int)chunk_prob.size();
  auto fail = [&](cudaError_t e, const char *what) {
    cudaGetLastError();
    mf_set_error("mf_batch_create: %s: %s", what, cudaGetErrorString(e));
    batch_free(B);
    return e == cudaErrorMemoryAllocation ? MF_ERR_OOM : MF_ERR_CUDA;
  };
  cudaError_t e;
  if ((e = cudaMalloc(&B->probs, n * sizeof(BProblem))) != cudaSuccess) return fail(e, "cudaMalloc");
  if ((e = cudaMalloc(&B->sc, n * sizeof(BScalars))) != cudaSuccess) return fail(e, "cudaMalloc");
  if ((e = cudaMalloc(&B->ctl, sizeof(BControl))) != cudaSuccess) return fail(e, "cudaMalloc");
  if ((e = cudaMalloc(&B->work, (3 * total_dof + total_chunks) * sizeof(double))) != cudaSuccess)
    return fail(e, "cudaMalloc");
  if ((e = cudaMalloc(&B->maps, (item_prob.size() + chunk_prob.size()) * sizeof(int))) != cudaSuccess)
    return fail(e, "cudaMalloc");
  double *w = B->work;
  for (int i = 0; i < n; ++i) {
    BProblem &P = B->hprobs[i];
    P.r = w;
    P.p = w + P.n;
    P.Ap = w + 2 * P.n;
    w += 3 * P.n;
  }
  for (int i = 0; i < n; ++i) {
    B->hprobs[i].partials = w;
    w += B->hprobs[i].n_chunks;
    B->hprobs[i].sc = B->sc + i;
    B->hprobs[i].b = nullptr;
    B->hprobs[i].x = nullptr;
  }
  if ((e = cudaMemcpy(B->maps, item_prob.data(), item_prob.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail(e, "cudaMemcpy");
  if ((e = cudaMemcpy(B->maps + item_prob.size(), chunk_prob.data(), chunk_prob.size() * sizeof(int),
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail(e, "cudaMemcpy");
  // co-resident grid
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_cg, kThreadsB, 0)) != cudaSuccess)
    return fail(e, "occupancy query");
  if (per_sm < 1) {
    batch_free(B);
    mf_set_error("mf_batch_create: the batched kernel cannot be resident");
    return MF_ERR_CUDA;
  }
  B->grid = sms * per_sm;
  BArgs &A = B->args;
  A.probs = B->probs;
  A.n_probs = n;
  A.total_items = (int)item_prob.size();
  A.total_chunks = total_chunks;
  A.item_prob = B->maps;
  A.chunk_prob = B->maps + item_prob.size();
  A.ctl = B->ctl;
  // bound on one barrier wait, in SM clock cycles (~2 GHz): opts->timeout_s when given, else ~2 s
  A.budget = o->timeout_s > 0 ? (long long)(o->timeout_s * 2.0e9) : 4000000000ll;
  A.max_iter = o->max_iter;
  A.rtol2 = o->rtol * o->rtol;
  B->hsc.resize(n);
  if ((e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking)) != cudaSuccess) return fail(e, "stream");
  // capture the one persistent cooperative launch
  cudaGraph_t graph;
  if ((e = cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return fail(e, "capture");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(B->grid);
  cfg.blockDim = dim3(kThreadsB);
  cfg.stream = B->cap;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t le = cudaLaunchKernelEx(&cfg, batched_cg, A);
  e = cudaStreamEndCapture(B->cap, &graph);
  if (le != cudaSuccess) return fail(le, "cooperative launch capture");
  if (e != cudaSuccess) return fail(e, "end capture");
  e = cudaGraphInstantiate(&B->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    B->exec = nullptr;
    return fail(e, "graph instantiate");
  }
  B->kernels = 1;
  *out = B;
  return MF_OK;
}

extern "C" mf_status mf_batch_solve(mf_batch *B, const double *const *b, double *const *x, mf_solve_info *infos,
                                    mf_stream stream) {
  MF_RANGE("mf_batch_solve");
  mf_clear_error();
  MF_ARG(B && b && x, "mf_batch_solve: null argument");
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  for (int i = 0; i < B->n; ++i) {
    MF_ARG(b[i] && x[i], "mf_batch_solve: problem %d has a null vector", i);
    B->hprobs[i].b = b[i];
    B->hprobs[i].x = x[i];
  }
  MF_CUDA(cudaMemcpyAsync(B->probs, B->hprobs.data(), B->n * sizeof(BProblem), cudaMemcpyHostToDevice, s));
  MF_CUDA(cudaMemsetAsync(B->sc, 0, B->n * sizeof(BScalars), s));
  BControl c0 = {0u, 0u, 0, B->n};
  MF_CUDA(cudaMemcpyAsync(B->ctl, &c0, sizeof(c0), cudaMemcpyHostToDevice, s));
  MF_CUDA(cudaGraphLaunch(B->exec, s));
  mf_count_launches(B->kernels);
  BControl c1;
  MF_CUDA(cudaMemcpyAsync(B->hsc.data(), B->sc, B->n * sizeof(BScalars), cudaMemcpyDeviceToHost, s));
  MF_CUDA(cudaMemcpyAsync(&c1, B->ctl, sizeof(c1), cudaMemcpyDeviceToHost, s));
  MF_CUDA(cudaStreamSynchronize(s));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  mf_status st = MF_OK;
  if (c1.err) {
    mf_set_error("mf_batch_solve: a grid barrier timed out");
    st = MF_ERR_TIMEOUT;
  }
  for (int i = 0; i < B->n; ++i) {
    const BScalars &sc = B->hsc[i];
    mf_status si = (mf_status)sc.status;
    if (si == MF_OK && !sc.done) si = MF_NOT_CONVERGED;
    if (st == MF_OK && si != MF_OK) st = si;
    if (infos) {
      infos[i].iters = sc.iter;
      infos[i].outer_iters = 0;
      infos[i].status = c1.err ? MF_ERR_TIMEOUT : si;
      infos[i].rel_res = sc.bb > 0 ? std::sqrt(sc.rr / sc.bb) : 0.0;
      infos[i].rel_res_true = -1.0;  // not recomputed by the batched solver
      infos[i].seconds = secs;
    }
  }
  return st;
}

extern "C" mf_status mf_batch_destroy(mf_batch *B) {
  if (!B) return MF_OK;
  cudaDeviceSynchronize();
  batch_free(B);
  return MF_OK;
}

extern "C" mf_status mf_cg_solve_batched(mf_mesh *const *meshes, int32_t n, const mf_solve_opts *o,
                                         const double *const *b, double *const *x, mf_solve_info *infos,
                                         mf_stream stream) {
  mf_batch *B = nullptr;
  MF_TRY(mf_batch_create(meshes, n, o, &B));
  const mf_status st = mf_batch_solve(B, b, x, infos, stream);
  mf_batch_destroy(B);
  return st;
}

MF_DBG_TU(batched)
