// Network runtime of the learned preconditioner (architecture in mf_nn.cu): parameters, forward,
// backward, Adam, and the flexible CG that applies the network as a preconditioner.
//
// Everything runs on the device through the library's own kernels; the host only sequences them.
#include <cuda_bf16.h>

#include <chrono>
#include <cmath>
#include <random>
#include <cstring>
#include <vector>

#include "mf_internal.cuh"

typedef __nv_bfloat16 bf16;

extern "C" mf_status mf_conv3d_fwd(const void *x, int32_t nx, int32_t ny, int32_t nz, int32_t cin, const void *w,
                                   const float *bias, int32_t cout, const void *skip, int32_t relu, void *y_bf16,
                                   float *y_f32, mf_stream stream);
extern "C" mf_status mf_conv3d_dgrad(const void *dy, int32_t nx, int32_t ny, int32_t nz, int32_t cin, const void *w,
                                     int32_t cout, void *dx_bf16, float *dx_f32, mf_stream stream);
extern "C" int64_t mf_conv3d_wgrad_workspace(int32_t nx, int32_t ny, int32_t nz, int32_t cin, int32_t cout);
extern "C" mf_status mf_conv3d_wgrad(const void *x, const void *dy, int32_t nx, int32_t ny, int32_t nz, int32_t cin,
                                     int32_t cout, float *dw, float *db, float *workspace, int64_t ws_bytes,
                                     mf_stream stream);
extern "C" mf_status mf_grid_restrict(const void *in, int32_t nfx, int32_t nfy, int32_t nfz, int32_t c, void *out,
                                      float scale, mf_stream stream);
extern "C" mf_status mf_grid_prolong(const void *in, int32_t ncx, int32_t ncy, int32_t ncz, int32_t c, void *out,
                                     float scale, mf_stream stream);
mf_status nn_relu_mask(const void *d, const void *act, int64_t n, void *out, cudaStream_t s);
mf_status nn_add(void *a, const void *b, int64_t n, cudaStream_t s);
mf_status nn_f32_to_bf16(const float *a, void *b, int64_t n, cudaStream_t s);

namespace {

struct Layer {
  int level, cin, cout, relu;
  int64_t w_off, b_off;  // offsets in the flat parameter array (floats)
};

// e0, e1, e2, m2, d1, q1, d0, out
const int kLayers[8][4] = {{0, 2, 16, 1}, {1, 16, 32, 1}, {2, 32, 64, 1}, {2, 64, 64, 1},
                           {1, 64, 32, 1}, {1, 32, 16, 1}, {0, 16, 16, 1}, {0, 16, 1, 0}};

// The network input: 2 channels per voxel (residual, log kappa), and the same padded to 16 channels
// (zeros) for the tensor-core convolution, whose TMA loads move 16-byte channel chunks.
__global__ void make_input(const float *__restrict__ r, const float *__restrict__ logk, int64_t n, bf16 *__restrict__ in,
                           bf16 *__restrict__ in16) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bf16 a = __float2bfloat16(r[i]), b = __float2bfloat16(logk[i]);
  in[2 * i] = a;
  in[2 * i + 1] = b;
  __align__(16) bf16 v[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __float2bfloat16(0.0f);
  v[0] = a;
  v[1] = b;
  uint4 *o = reinterpret_cast<uint4 *>(in16 + 16 * i);
  o[0] = reinterpret_cast<const uint4 *>(v)[0];
  o[1] = reinterpret_cast<const uint4 *>(v)[1];
}

// Relative squared error L = sum (o - t)^2 / sum t^2 and its gradient 2 (o - t) / sum t^2 (bf16).
// Relative squared error: per-block partials of sum (o - t)^2 and sum t^2 over a grid-stride range
// (kLossBlocks blocks), then one block sums the partials in order (deterministic).
constexpr int kLossBlocks = 256;

__global__ void __launch_bounds__(256) loss_part(const float *__restrict__ o, const float *__restrict__ t, int64_t n,
                                                 float *__restrict__ part) {
  __shared__ float s1[256], s2[256];
  float a = 0.f, b = 0.f;
  for (int64_t i = blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    const float d = o[i] - t[i];
    a += d * d;
    b += t[i] * t[i];
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) {
      s1[threadIdx.x] += s1[threadIdx.x + off];
      s2[threadIdx.x] += s2[threadIdx.x + off];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s1[0];
    part[2 * blockIdx.x + 1] = s2[0];
  }
}

__global__ void loss_final(const float *__restrict__ part, int nparts, float *__restrict__ out2) {
  if (threadIdx.x > 1) return;
  float s = 0.f;
  for (int p = 0; p < nparts; ++p) s += part[2 * p + threadIdx.x];
  out2[threadIdx.x] = s;
}

__global__ void loss_grad(const float *__restrict__ o, const float *__restrict__ t, int64_t n,
                          const float *__restrict__ sums, bf16 *__restrict__ g) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float den = fmaxf(sums[1], 1e-30f);
  g[i] = __float2bfloat16(2.0f * (o[i] - t[i]) / den);
}

// Gradient-norm clipping against loss spikes: partial sums of g^2 (fixed grid, fixed order), then
// one thread forms ||g|| and the scale min(1, kClipRatio * ema / ||g||) against an exponential
// moving average of the (clipped) norms of earlier steps; state = {ema, scale}.
constexpr int kClipBlocks = 256;
constexpr float kClipRatio = 5.0f;

__global__ void __launch_bounds__(256) grad_sq_part(const float *__restrict__ g, int64_t n, float *__restrict__ part) {
  __shared__ float sh[256];
  float s = 0.f;
  for (int64_t i = blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) s += g[i] * g[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void clip_scale(const float *__restrict__ part, int nparts, float *__restrict__ state) {
  if (threadIdx.x != 0) return;
  float s = 0.f;
  for (int p = 0; p < nparts; ++p) s += part[p];
  const float norm = sqrtf(s), ema = state[0];
  float scale = 1.0f;
  if (ema > 0.f && norm > kClipRatio * ema) scale = kClipRatio * ema / norm;
  if (!isfinite(norm)) scale = 0.0f;  // skip a non-finite step
  const float used = isfinite(norm) ? norm * scale : ema;
  state[0] = ema > 0.f ? 0.9f * ema + 0.1f * used : used;
  state[1] = scale;
}

// Adam (Kingma & Ba 2015) with bias correction on the clipped gradient gscale[0] * g; writes the
// BF16 copy of the weights.
__global__ void adam_k(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2, bf16 *__restrict__ pb,
                       const float *__restrict__ gscale) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i] * gscale[0];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  pb[i] = __float2bfloat16(pi);
}

}  // namespace

struct mf_net {
  int n[3][3];       // node dims per level [level][x,y,z]
  int64_t V[3];      // voxels per level
  std::vector<Layer> layers;
  int64_t n_params = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // flat FP32
  bf16 *pb = nullptr;                                           // BF16 copy (weights used by kernels)
  int64_t step = 0;
  // activations (bf16) and gradients
  bf16 *in16 = nullptr;  // the input padded to 16 channels (tensor-core path of layer 0)
  bf16 *in0 = nullptr, *e0 = nullptr, *r0 = nullptr, *e1 = nullptr, *r1 = nullptr, *e2 = nullptr, *m2 = nullptr,
       *p1 = nullptr, *d1 = nullptr, *q1 = nullptr, *p0 = nullptr, *d0 = nullptr;
  float *out = nullptr;
  bf16 *g_out = nullptr, *g_a = nullptr, *g_b = nullptr, *g_c = nullptr, *g_e1 = nullptr, *g_e0 = nullptr;
  float *ws = nullptr;
  int64_t ws_bytes = 0;
  float *sums = nullptr;
  float *lpart = nullptr;  // loss partials [kLossBlocks][2]
  float *cpart = nullptr;  // squared-gradient partials [kClipBlocks]
  float *clip = nullptr;   // {moving average of the gradient norm, scale of this step}
  float out_scale = 1.0f;
  std::vector<void *> allocs;
};

namespace {

template <typename T>
mf_status nalloc(mf_net *N, T **p, int64_t count) {
  cudaError_t e = cudaMalloc((void **)p, std::max<int64_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    mf_set_error("mf_net: cudaMalloc failed: %s", cudaGetErrorString(e));
    return MF_ERR_OOM;
  }
  N->allocs.push_back(*p);
  return MF_OK;
}

void net_free(mf_net *N) {
  if (!N) return;
  for (void *q : N->allocs) cudaFree(q);
  delete N;
}

const bf16 *W(const mf_net *N, int l) { return N->pb + N->layers[l].w_off; }
const float *B(const mf_net *N, int l) { return N->p + N->layers[l].b_off; }

mf_status conv(const mf_net *N, int l, const bf16 *in, const bf16 *skip, bf16 *out_b, float *out_f, cudaStream_t s) {
  const Layer &L = N->layers[l];
  const int *d = N->n[L.level];
  return mf_conv3d_fwd(in, d[0], d[1], d[2], L.cin, W(N, l), B(N, l), L.cout, skip, L.relu, out_b, out_f, (mf_stream)s);
}

mf_status forward(mf_net *N, cudaStream_t s) {
  const int *n0 = N->n[0], *n1 = N->n[1];
  {  // layer 0 on the tensor cores from the padded input, else from the 2-channel one
    const Layer &L = N->layers[0];
    const int *d = N->n[0];
    const mf_status st = conv3d_fwd_strided(N->in16, d[0], d[1], d[2], L.cin, 16, W(N, 0), B(N, 0), L.cout, nullptr,
                                            L.relu, N->e0, nullptr, s);
    if (st == MF_ERR_UNSUPPORTED) MF_TRY(conv(N, 0, N->in0, nullptr, N->e0, nullptr, s));
    else MF_TRY(st);
  }
  MF_TRY(mf_grid_restrict(N->e0, n0[0], n0[1], n0[2], 16, N->r0, 1.0f, (mf_stream)s));
  MF_TRY(conv(N, 1, N->r0, nullptr, N->e1, nullptr, s));
  MF_TRY(mf_grid_restrict(N->e1, n1[0], n1[1], n1[2], 32, N->r1, 1.0f, (mf_stream)s));
  MF_TRY(conv(N, 2, N->r1, nullptr, N->e2, nullptr, s));
  MF_TRY(conv(N, 3, N->e2, nullptr, N->m2, nullptr, s));
  MF_TRY(mf_grid_prolong(N->m2, N->n[2][0], N->n[2][1], N->n[2][2], 64, N->p1, 1.0f, (mf_stream)s));
  MF_TRY(conv(N, 4, N->p1, N->e1, N->d1, nullptr, s));
  MF_TRY(conv(N, 5, N->d1, nullptr, N->q1, nullptr, s));
  MF_TRY(mf_grid_prolong(N->q1, n1[0], n1[1], n1[2], 16, N->p0, 1.0f, (mf_stream)s));
  MF_TRY(conv(N, 6, N->p0, N->e0, N->d0, nullptr, s));
  MF_TRY(conv(N, 7, N->d0, nullptr, nullptr, N->out, s));
  return MF_OK;
}

// gradient of one conv layer: given dL/d(pre-activation) `gpre` and its input `in`, accumulate
// weight/bias gradients and (optionally) the input gradient into `gin`.
mf_status conv_back(mf_net *N, int l, const bf16 *in, const bf16 *gpre, bf16 *gin, cudaStream_t s) {
  const Layer &L = N->layers[l];
  const int *d = N->n[L.level];
  MF_TRY(mf_conv3d_wgrad(in, gpre, d[0], d[1], d[2], L.cin, L.cout, N->g + L.w_off, N->g + L.b_off, N->ws, N->ws_bytes,
                         (mf_stream)s));
  if (gin) MF_TRY(mf_conv3d_dgrad(gpre, d[0], d[1], d[2], L.cin, W(N, l), L.cout, gin, nullptr, (mf_stream)s));
  return MF_OK;
}

mf_status backward(mf_net *N, const float *target, float *loss_host, cudaStream_t s) {
  const int64_t V0 = N->V[0], V1 = N->V[1], V2 = N->V[2];
  const int *n0 = N->n[0], *n1 = N->n[1], *n2 = N->n[2];
  mf_count_launches(3);
  loss_part<<<kLossBlocks, 256, 0, s>>>(N->out, target, V0, N->lpart);
  loss_final<<<1, 32, 0, s>>>(N->lpart, kLossBlocks, N->sums);
  loss_grad<<<blocks_for(V0), kThreads, 0, s>>>(N->out, target, V0, N->sums, N->g_out);
  MF_CUDA(cudaGetLastError());
  // out = conv7(d0), linear
  MF_TRY(conv_back(N, 7, N->d0, N->g_out, N->g_a, s));                 // g_a = dL/dd0
  // d0 = relu(conv6(p0) + e0)
  MF_TRY(nn_relu_mask(N->g_a, N->d0, V0 * 16, N->g_b, s));             // g_b = gpre6
  MF_TRY(cudaMemcpyAsync(N->g_e0, N->g_b, V0 * 16 * sizeof(bf16), cudaMemcpyDeviceToDevice, s) == cudaSuccess
             ? MF_OK : MF_ERR_CUDA);
  MF_TRY(conv_back(N, 6, N->p0, N->g_b, N->g_a, s));                   // g_a = dL/dp0
  // p0 = P q1  ->  dL/dq1 = P^T g = 8 R g
  MF_TRY(mf_grid_restrict(N->g_a, n0[0], n0[1], n0[2], 16, N->g_c, 8.0f, (mf_stream)s));  // g_c: [V1][16]
  // q1 = relu(conv5(d1))
  MF_TRY(nn_relu_mask(N->g_c, N->q1, V1 * 16, N->g_c, s));
  MF_TRY(conv_back(N, 5, N->d1, N->g_c, N->g_b, s));                   // g_b = dL/dd1 [V1][32]
  // d1 = relu(conv4(p1) + e1)
  MF_TRY(nn_relu_mask(N->g_b, N->d1, V1 * 32, N->g_b, s));             // gpre4
  MF_TRY(cudaMemcpyAsync(N->g_e1, N->g_b, V1 * 32 * sizeof(bf16), cudaMemcpyDeviceToDevice, s) == cudaSuccess
             ? MF_OK : MF_ERR_CUDA);
  MF_TRY(conv_back(N, 4, N->p1, N->g_b, N->g_a, s));                   // g_a = dL/dp1 [V1][64]
  // p1 = P m2
  MF_TRY(mf_grid_restrict(N->g_a, n1[0], n1[1], n1[2], 64, N->g_c, 8.0f, (mf_stream)s));  // g_c: [V2][64]
  // m2 = relu(conv3(e2))
  MF_TRY(nn_relu_mask(N->g_c, N->m2, V2 * 64, N->g_c, s));
  MF_TRY(conv_back(N, 3, N->e2, N->g_c, N->g_b, s));                   // g_b = dL/de2 [V2][64]
  // e2 = relu(conv2(r1))
  MF_TRY(nn_relu_mask(N->g_b, N->e2, V2 * 64, N->g_b, s));
  MF_TRY(conv_back(N, 2, N->r1, N->g_b, N->g_c, s));                   // g_c = dL/dr1 [V2][32]
  // r1 = R e1  ->  dL/de1 += R^T g = P g / 8
  MF_TRY(mf_grid_prolong(N->g_c, n2[0], n2[1], n2[2], 32, N->g_a, 0.125f, (mf_stream)s));  // g_a: [V1][32]
  MF_TRY(nn_add(N->g_e1, N->g_a, V1 * 32, s));
  // e1 = relu(conv1(r0))
  MF_TRY(nn_relu_mask(N->g_e1, N->e1, V1 * 32, N->g_e1, s));
  MF_TRY(conv_back(N, 1, N->r0, N->g_e1, N->g_c, s));                  // g_c = dL/dr0 [V1][16]
  // r0 = R e0
  MF_TRY(mf_grid_prolong(N->g_c, n1[0], n1[1], n1[2], 16, N->g_a, 0.125f, (mf_stream)s));  // g_a: [V0][16]
  MF_TRY(nn_add(N->g_e0, N->g_a, V0 * 16, s));
  // e0 = relu(conv0(in0))
  MF_TRY(nn_relu_mask(N->g_e0, N->e0, V0 * 16, N->g_e0, s));
  MF_TRY(conv_back(N, 0, N->in0, N->g_e0, nullptr, s));
  if (loss_host) {
    float h[2];
    MF_CUDA(cudaMemcpyAsync(h, N->sums, 2 * sizeof(float), cudaMemcpyDeviceToHost, s));
    MF_CUDA(cudaStreamSynchronize(s));
    *loss_host = h[0] / std::max(h[1], 1e-30f);
  }
  return MF_OK;
}

mf_status load_input(mf_net *N, const float *r, const float *logk, cudaStream_t s) {
  mf_count_launches(1);
  make_input<<<blocks_for(N->V[0]), kThreads, 0, s>>>(r, logk, N->V[0], N->in0, N->in16);
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

}  // namespace

extern "C" mf_status mf_net_create(int32_t nx, int32_t ny, int32_t nz, uint64_t seed, mf_net **out) {
  MF_RANGE("mf_net_create");
  mf_clear_error();
  MF_ARG(out != nullptr, "mf_net_create: out is NULL");
  *out = nullptr;
  MF_ARG(nx >= 5 && ny >= 5 && nz >= 5 && (nx - 1) % 4 == 0 && (ny - 1) % 4 == 0 && (nz - 1) % 4 == 0,
         "mf_net_create: node dims must be 4m+1 >= 5");
  mf_net *N = new mf_net();
  int d[3] = {nx, ny, nz};
  for (int l = 0; l < 3; ++l)
    for (int a = 0; a < 3; ++a) N->n[l][a] = l == 0 ? d[a] : (N->n[l - 1][a] + 1) / 2;
  for (int l = 0; l < 3; ++l) N->V[l] = (int64_t)N->n[l][0] * N->n[l][1] * N->n[l][2];
  int64_t off = 0;
  for (auto &L : kLayers) {
    Layer y{L[0], L[1], L[2], L[3], 0, 0};
    y.w_off = off;
    off += 27 * (int64_t)y.cin * y.cout;
    y.b_off = off;
    off += y.cout;
    N->layers.push_back(y);
  }
  N->n_params = off;
  const int64_t V0 = N->V[0], V1 = N->V[1], V2 = N->V[2];
  mf_status st = MF_OK;
#define NA(ptr, cnt)                      \
  if ((st = nalloc(N, &(ptr), (cnt))) != MF_OK) { \
    net_free(N);                          \
    return st;                            \
  }
  NA(N->p, off) NA(N->g, off) NA(N->m, off) NA(N->v, off) NA(N->pb, off)
  NA(N->in0, V0 * 2) NA(N->in16, V0 * 16) NA(N->e0, V0 * 16) NA(N->r0, V1 * 16) NA(N->e1, V1 * 32) NA(N->r1, V2 * 32) NA(N->e2, V2 * 64)
  NA(N->m2, V2 * 64) NA(N->p1, V1 * 64) NA(N->d1, V1 * 32) NA(N->q1, V1 * 16) NA(N->p0, V0 * 16) NA(N->d0, V0 * 16)
  NA(N->out, V0) NA(N->g_out, V0)
  const int64_t gmax = std::max(std::max(V0 * 16, V1 * 64), V2 * 64);
  NA(N->g_a, gmax) NA(N->g_b, gmax) NA(N->g_c, gmax) NA(N->g_e1, V1 * 32) NA(N->g_e0, V0 * 16) NA(N->sums, 2) NA(N->lpart, 2 * kLossBlocks) NA(N->cpart, kClipBlocks) NA(N->clip, 2)
  int64_t wsb = 0;
  for (auto &L : N->layers) {
    const int *dd = N->n[L.level];
    wsb = std::max(wsb, mf_conv3d_wgrad_workspace(dd[0], dd[1], dd[2], L.cin, L.cout));
  }
  N->ws_bytes = wsb;
  NA(N->ws, wsb / (int64_t)sizeof(float) + 1)
#undef NA
  // He-normal initialisation (seeded), zero biases, small output layer
  std::vector<float> h(off, 0.0f);
  std::mt19937_64 rng(seed);
  for (size_t li = 0; li < N->layers.size(); ++li) {
    const Layer &L = N->layers[li];
    std::normal_distribution<float> nd(0.0f, std::sqrt(2.0f / (27.0f * L.cin)) * (li + 1 == N->layers.size() ? 0.1f : 1.0f));
    for (int64_t i = 0; i < 27 * (int64_t)L.cin * L.cout; ++i) h[L.w_off + i] = nd(rng);
  }
  cudaError_t e = cudaMemcpy(N->p, h.data(), off * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(N->m, 0, off * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(N->v, 0, off * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(N->clip, 0, 2 * sizeof(float));  // no norm history yet
  if (e != cudaSuccess) {
    mf_set_error("mf_net_create: %s", cudaGetErrorString(e));
    net_free(N);
    return MF_ERR_CUDA;
  }
  st = nn_f32_to_bf16(N->p, N->pb, off, 0);
  if (st == MF_OK && cudaDeviceSynchronize() != cudaSuccess) st = MF_ERR_CUDA;
  if (st != MF_OK) {
    net_free(N);
    return st;
  }
  *out = N;
  return MF_OK;
}

extern "C" mf_status mf_net_destroy(mf_net *N) {
  if (!N) return MF_OK;
  cudaDeviceSynchronize();
  net_free(N);
  return MF_OK;
}

extern "C" int64_t mf_net_num_params(const mf_net *N) { return N ? N->n_params : 0; }

extern "C" mf_status mf_net_get_params(const mf_net *N, float *host) {
  MF_ARG(N && host, "mf_net_get_params: null argument");
  MF_CUDA(cudaMemcpy(host, N->p, N->n_params * sizeof(float), cudaMemcpyDeviceToHost));
  return MF_OK;
}

extern "C" mf_status mf_net_set_params(mf_net *N, const float *host) {
  MF_ARG(N && host, "mf_net_set_params: null argument");
  MF_CUDA(cudaMemcpy(N->p, host, N->n_params * sizeof(float), cudaMemcpyHostToDevice));
  MF_TRY(nn_f32_to_bf16(N->p, N->pb, N->n_params, 0));
  MF_CUDA(cudaDeviceSynchronize());
  return MF_OK;
}

// Training state: a header, then the FP32 parameters and Adam's first and second moments.
namespace {
constexpr uint64_t kNetStateMagic = 0x31303054454e464dull;  // the bytes "MFNET001"
struct NetStateHeader {
  uint64_t magic;
  int64_t n_params, step;
  float clip[2];  // moving average of the gradient norm, last step's scale
  float out_scale, pad;
};
}  // namespace

extern "C" int64_t mf_net_state_bytes(const mf_net *N) {
  return N ? (int64_t)sizeof(NetStateHeader) + 3 * N->n_params * (int64_t)sizeof(float) : 0;
}

extern "C" mf_status mf_net_state_save(const mf_net *N, void *host, int64_t bytes) {
  mf_clear_error();
  MF_ARG(N && host, "mf_net_state_save: null argument");
  MF_ARG(bytes >= mf_net_state_bytes(N), "mf_net_state_save: buffer of %lld bytes, %lld needed", (long long)bytes,
         (long long)mf_net_state_bytes(N));
  MF_CUDA(cudaDeviceSynchronize());
  NetStateHeader h{};
  h.magic = kNetStateMagic;
  h.n_params = N->n_params;
  h.step = N->step;
  MF_CUDA(cudaMemcpy(h.clip, N->clip, 2 * sizeof(float), cudaMemcpyDeviceToHost));
  h.out_scale = N->out_scale;
  char *o = static_cast<char *>(host);
  std::memcpy(o, &h, sizeof(h));
  o += sizeof(h);
  const size_t pb = N->n_params * sizeof(float);
  MF_CUDA(cudaMemcpy(o, N->p, pb, cudaMemcpyDeviceToHost));
  MF_CUDA(cudaMemcpy(o + pb, N->m, pb, cudaMemcpyDeviceToHost));
  MF_CUDA(cudaMemcpy(o + 2 * pb, N->v, pb, cudaMemcpyDeviceToHost));
  return MF_OK;
}

extern "C" mf_status mf_net_state_load(mf_net *N, const void *host, int64_t bytes) {
  mf_clear_error();
  MF_ARG(N && host, "mf_net_state_load: null argument");
  MF_ARG(bytes >= (int64_t)sizeof(NetStateHeader), "mf_net_state_load: %lld bytes is no network state", (long long)bytes);
  NetStateHeader h;
  std::memcpy(&h, host, sizeof(h));
  MF_ARG(h.magic == kNetStateMagic, "mf_net_state_load: not a network state");
  MF_ARG(h.n_params == N->n_params, "mf_net_state_load: state of %lld parameters, network has %lld",
         (long long)h.n_params, (long long)N->n_params);
  MF_ARG(bytes >= mf_net_state_bytes(N), "mf_net_state_load: truncated state (%lld bytes)", (long long)bytes);
  MF_ARG(h.step >= 0 && std::isfinite(h.out_scale) && h.out_scale > 0.0f && std::isfinite(h.clip[0]) &&
             h.clip[0] >= 0.0f && std::isfinite(h.clip[1]),
         "mf_net_state_load: corrupt header (step %lld, output scale %g)", (long long)h.step, (double)h.out_scale);
  MF_CUDA(cudaDeviceSynchronize());
  const char *o = static_cast<const char *>(host) + sizeof(h);
  const size_t pb = N->n_params * sizeof(float);
  MF_CUDA(cudaMemcpy(N->p, o, pb, cudaMemcpyHostToDevice));
  MF_CUDA(cudaMemcpy(N->m, o + pb, pb, cudaMemcpyHostToDevice));
  MF_CUDA(cudaMemcpy(N->v, o + 2 * pb, pb, cudaMemcpyHostToDevice));
  MF_CUDA(cudaMemcpy(N->clip, h.clip, 2 * sizeof(float), cudaMemcpyHostToDevice));
  N->step = h.step;
  N->out_scale = h.out_scale;
  MF_TRY(nn_f32_to_bf16(N->p, N->pb, N->n_params, 0));  // the same rounding as the Adam kernel's copy
  MF_CUDA(cudaDeviceSynchronize());
  return MF_OK;
}

extern "C" mf_status mf_net_set_output_scale(mf_net *N, float scale) {
  MF_ARG(N && scale > 0, "mf_net_set_output_scale: bad argument");
  N->out_scale = scale;
  return MF_OK;
}

extern "C" mf_status mf_net_forward(mf_net *N, const float *r, const float *logk, float *out, mf_stream stream) {
  MF_RANGE("mf_net_forward");
  mf_clear_error();
  MF_ARG(N && r && logk && out, "mf_net_forward: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  MF_TRY(load_input(N, r, logk, s));
  MF_TRY(forward(N, s));
  MF_CUDA(cudaMemcpyAsync(out, N->out, N->V[0] * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return MF_OK;
}

extern "C" mf_status mf_net_gradients(mf_net *N, const float *r, const float *logk, const float *target, float *grads_host,
                                      float *loss_host, mf_stream stream) {
  MF_RANGE("mf_net_gradients");
  mf_clear_error();
  MF_ARG(N && r && logk && target, "mf_net_gradients: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  MF_TRY(load_input(N, r, logk, s));
  MF_TRY(forward(N, s));
  MF_TRY(backward(N, target, loss_host, s));
  if (grads_host) {
    MF_CUDA(cudaMemcpyAsync(grads_host, N->g, N->n_params * sizeof(float), cudaMemcpyDeviceToHost, s));
    MF_CUDA(cudaStreamSynchronize(s));
  }
  return MF_OK;
}

extern "C" mf_status mf_net_train_step(mf_net *N, const float *r, const float *logk, const float *target, float lr,
                                       float *loss_host, mf_stream stream) {
  MF_RANGE("mf_net_train_step");
  mf_clear_error();
  MF_ARG(N && r && logk && target && lr > 0, "mf_net_train_step: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  MF_TRY(load_input(N, r, logk, s));
  MF_TRY(forward(N, s));
  MF_TRY(backward(N, target, loss_host, s));
  N->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, (float)N->step), c2 = 1.0f - std::pow(b2, (float)N->step);
  mf_count_launches(3);
  grad_sq_part<<<kClipBlocks, 256, 0, s>>>(N->g, N->n_params, N->cpart);
  clip_scale<<<1, 32, 0, s>>>(N->cpart, kClipBlocks, N->clip);
  adam_k<<<blocks_for(N->n_params), kThreads, 0, s>>>(N->p, N->g, N->m, N->v, N->n_params, lr, b1, b2, 1e-8f, c1, c2,
                                                      N->pb, N->clip + 1);
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

// accessors for the flexible CG (mf_cg.cu)
int64_t net_nodes(const mf_net *N) { return N->V[0]; }
const int *net_dims(const mf_net *N) { return N->n[0]; }
float net_out_scale(const mf_net *N) { return N->out_scale; }
