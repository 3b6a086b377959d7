// Learned preconditioner network: a 3-level convolutional encoder-decoder on the node grid, with
// BF16 operands and FP32 accumulation on the tensor cores.
//
// The paper names matrix-free preconditioners as future work (Sec. 7); this network is the
// project's own extension.  Architecture (node grids (4m+1)^3 -> (2m+1)^3 -> (m+1)^3):
//   e0 = relu(conv 2->16 (input))                          level 0
//   e1 = relu(conv 16->32 (R e0))                          level 1
//   e2 = relu(conv 32->64 (R e1)); m2 = relu(conv 64->64 e2)   level 2
//   d1 = relu(conv 64->32 (P m2) + e1); q1 = relu(conv 32->16 d1)  level 1
//   d0 = relu(conv 16->16 (P q1) + e0); out = conv 16->1 d0        level 0
// with R full-weighting restriction and P trilinear prolongation between node grids (fixed, as in
// geometric multigrid), all convolutions 3x3x3, zero padding, with bias.
//
// Kernels:
//  * conv_mma: implicit-GEMM convolution, M = 128 output voxels per CTA (an 8x4x4 block), N =
//    output channels, K = 27 taps x input channels.  The CTA stages its (10x6x6) input halo once in
//    shared memory (channels-last, padded rows against bank conflicts), then for each tap stages
//    that tap's weights and issues mma.sync m16n8k16 BF16 x BF16 -> FP32.  The same kernel computes
//    the input gradient (MODE 1) with the mirrored, transposed weights.
//  * conv_wgrad: weight and bias gradients, FP32 on the CUDA cores, split over voxel partitions
//    and reduced in fixed order (deterministic).
//  * restrict / prolong (and their adjoints as scaled prolong / restrict), relu masks, loss, Adam.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "mf_internal.cuh"

typedef __nv_bfloat16 bf16;

namespace {

constexpr int TXc = 8, TYc = 4, TZc = 4, HXc = TXc + 2, HYc = TYc + 2, HZc = TZc + 2, NHc = HXc * HYc * HZc;
constexpr int kConvThreads = 128;

struct ConvArgs {
  const bf16 *in;
  int nx, ny, nz, ck;     // input tensor: [nz][ny][nx][ck]
  const bf16 *w;          // MODE 0: [27][ck][cn]; MODE 1: [27][cn][ck]
  const float *bias;      // MODE 0 only, [cn] or null
  const bf16 *skip;       // MODE 0: [..][cn] added before relu, or null
  int relu;
  int cn;                 // output channels actually stored (<= CN)
  bf16 *out_bf;           // [..][cn] or null
  float *out_f;           // [..][cn] or null
  int tiles_x, tiles_y;
};

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// CKP: input channels padded to a multiple of 16; CN: output channels padded to a multiple of 8.
template <int CKP, int CN, int MODE>
__global__ void __launch_bounds__(kConvThreads) conv_mma(ConvArgs a) {
  constexpr int SK = CKP + 8;  // padded smem row (bf16 elements)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bf16 *in_s = reinterpret_cast<bf16 *>(smem_raw);
  bf16 *w_s = in_s + NHc * SK;
  const int tid = threadIdx.x;
  const int bx = blockIdx.x % a.tiles_x;
  const int by = (blockIdx.x / a.tiles_x) % a.tiles_y;
  const int bz = blockIdx.x / (a.tiles_x * a.tiles_y);
  const int x0 = bx * TXc, y0 = by * TYc, z0 = bz * TZc;

  // stage the input halo (zero outside the grid and for padded channels)
  for (int idx = tid; idx < NHc * CKP; idx += kConvThreads) {
    const int hv = idx / CKP, c = idx % CKP;
    const int hx = hv % HXc, hy = (hv / HXc) % HYc, hz = hv / (HXc * HYc);
    const int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = z0 - 1 + hz;
    bf16 v = __float2bfloat16(0.0f);
    if (c < a.ck && gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz)
      v = a.in[(((int64_t)gz * a.ny + gy) * a.nx + gx) * a.ck + c];
    in_s[hv * SK + c] = v;
  }

  const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  float acc[2][CN / 8][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < CN / 8; ++nt)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[mt][nt][j] = 0.0f;

  for (int tap = 0; tap < 27; ++tap) {
    __syncthreads();
    for (int idx = tid; idx < CN * CKP; idx += kConvThreads) {
      const int n = idx / CKP, k = idx % CKP;
      bf16 v = __float2bfloat16(0.0f);
      if (k < a.ck && n < a.cn) {
        if (MODE == 0) v = a.w[((int64_t)tap * a.ck + k) * a.cn + n];
        else v = a.w[((int64_t)(26 - tap) * a.cn + n) * a.ck + k];
      }
      w_s[n * SK + k] = v;
    }
    __syncthreads();
    const int dx = tap % 3, dy = (tap / 3) % 3, dz = tap / 9;
    int hv[2][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = 32 * warp + 16 * mt + g + 8 * h;
        const int tx = r & 7, ty = (r >> 3) & 3, tz = r >> 5;
        hv[mt][h] = (tz + dz) * (HXc * HYc) + (ty + dy) * HXc + (tx + dx);
      }
#pragma unroll
    for (int k0 = 0; k0 < CKP; k0 += 16) {
      uint32_t af[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        af[mt][0] = *reinterpret_cast<const uint32_t *>(in_s + hv[mt][0] * SK + k0 + 2 * t);
        af[mt][1] = *reinterpret_cast<const uint32_t *>(in_s + hv[mt][1] * SK + k0 + 2 * t);
        af[mt][2] = *reinterpret_cast<const uint32_t *>(in_s + hv[mt][0] * SK + k0 + 8 + 2 * t);
        af[mt][3] = *reinterpret_cast<const uint32_t *>(in_s + hv[mt][1] * SK + k0 + 8 + 2 * t);
      }
#pragma unroll
      for (int nt = 0; nt < CN / 8; ++nt) {
        const uint32_t b0 = *reinterpret_cast<const uint32_t *>(w_s + (nt * 8 + g) * SK + k0 + 2 * t);
        const uint32_t b1 = *reinterpret_cast<const uint32_t *>(w_s + (nt * 8 + g) * SK + k0 + 8 + 2 * t);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) mma_bf16(acc[mt][nt], af[mt][0], af[mt][1], af[mt][2], af[mt][3], b0, b1);
      }
    }
  }
  // epilogue
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = 32 * warp + 16 * mt + g + 8 * h;
      const int gx = x0 + (r & 7), gy = y0 + ((r >> 3) & 3), gz = z0 + (r >> 5);
      if (gx >= a.nx || gy >= a.ny || gz >= a.nz) continue;
      const int64_t vox = ((int64_t)gz * a.ny + gy) * a.nx + gx;
#pragma unroll
      for (int nt = 0; nt < CN / 8; ++nt)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int n = nt * 8 + 2 * t + j;
          if (n >= a.cn) continue;
          float v = acc[mt][nt][2 * h + j];
          if (MODE == 0) {
            if (a.bias) v += a.bias[n];
            if (a.skip) v += __bfloat162float(a.skip[vox * a.cn + n]);
            if (a.relu) v = fmaxf(v, 0.0f);
          }
          if (a.out_bf) a.out_bf[vox * a.cn + n] = __float2bfloat16(v);
          if (a.out_f) a.out_f[vox * a.cn + n] = v;
        }
    }
}

template <int CKP, int CN, int MODE>
mf_status launch_conv_t(const ConvArgs &a, cudaStream_t s) {
  const int smem = (NHc + CN) * (CKP + 8) * (int)sizeof(bf16);
  static bool attr_set = false;
  if (!attr_set) {
    MF_CUDA(cudaFuncSetAttribute(conv_mma<CKP, CN, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    attr_set = true;
  }
  const int tz = (a.nz + TZc - 1) / TZc;
  mf_count_launches(1);
  conv_mma<CKP, CN, MODE><<<a.tiles_x * a.tiles_y * tz, kConvThreads, smem, s>>>(a);
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

template <int MODE>
mf_status launch_conv(ConvArgs a, cudaStream_t s) {
  a.tiles_x = (a.nx + TXc - 1) / TXc;
  a.tiles_y = (a.ny + TYc - 1) / TYc;
  const int ckp = a.ck <= 16 ? 16 : a.ck <= 32 ? 32 : 64;
  const int cnp = a.cn <= 8 ? 8 : a.cn <= 16 ? 16 : a.cn <= 32 ? 32 : 64;
  MF_ARG(a.ck <= 64 && a.cn <= 64 && a.ck > 0 && a.cn > 0, "conv3d: channels must be in [1, 64]");
#define CASE(K, N) \
  if (ckp == K && cnp == N) return launch_conv_t<K, N, MODE>(a, s);
  CASE(16, 8) CASE(16, 16) CASE(16, 32) CASE(16, 64)
  CASE(32, 8) CASE(32, 16) CASE(32, 32) CASE(32, 64)
  CASE(64, 8) CASE(64, 16) CASE(64, 32) CASE(64, 64)
#undef CASE
  return MF_ERR_ARG;
}

// ------------------------------------------------------------------------ weight gradient ----
// dw[t][ci][co] = sum_v x[v + off_t][ci] dy[v][co]; partials over P voxel partitions, FP32.
constexpr int kWgThreads = 256, kWgChunk = 64;

__global__ void __launch_bounds__(kWgThreads) conv_wgrad_part(const bf16 *__restrict__ x, const bf16 *__restrict__ dy,
                                                              int nx, int ny, int nz, int ci, int co, int nparts,
                                                              float *__restrict__ part) {
  // blockIdx.x = tap + 27 * partition
  const int tap = blockIdx.x % 27, pidx = blockIdx.x / 27;
  const int ox = tap % 3 - 1, oy = (tap / 3) % 3 - 1, oz = tap / 9 - 1;
  const int64_t nvox = (int64_t)nx * ny * nz;
  const int64_t v0 = nvox * pidx / nparts, v1 = nvox * (pidx + 1) / nparts;
  __shared__ float xs[kWgChunk][65], ds[kWgChunk][65];
  const int npair = ci * co;
  float accv[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) accv[i] = 0.0f;
  for (int64_t base = v0; base < v1; base += kWgChunk) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < kWgChunk * 64; idx += kWgThreads) {
      const int j = idx / 64, c = idx % 64;
      const int64_t v = base + j;
      float xv = 0.0f, dv = 0.0f;
      if (v < v1) {
        const int gx = (int)(v % nx), gy = (int)((v / nx) % ny), gz = (int)(v / ((int64_t)nx * ny));
        const int sx = gx + ox, sy = gy + oy, sz = gz + oz;
        if (c < ci && sx >= 0 && sx < nx && sy >= 0 && sy < ny && sz >= 0 && sz < nz)
          xv = __bfloat162float(x[(((int64_t)sz * ny + sy) * nx + sx) * ci + c]);
        if (c < co) dv = __bfloat162float(dy[v * co + c]);
      }
      xs[j][c] = xv;
      ds[j][c] = dv;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int pair = threadIdx.x + i * kWgThreads;
      if (pair < npair) {
        const int a = pair / co, b = pair % co;
        float s = accv[i];
        for (int j = 0; j < kWgChunk; ++j) s = fmaf(xs[j][a], ds[j][b], s);
        accv[i] = s;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int pair = threadIdx.x + i * kWgThreads;
    if (pair < npair) part[((int64_t)pidx * 27 + tap) * npair + pair] = accv[i];
  }
}

__global__ void conv_wgrad_reduce(const float *__restrict__ part, int nparts, int n, float *__restrict__ dw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.0f;
  for (int p = 0; p < nparts; ++p) s += part[(int64_t)p * n + i];
  dw[i] = s;
}

// db[co] = sum_v dy[v][co] (fixed-order two-level sum)
__global__ void bias_grad(const bf16 *__restrict__ dy, int64_t nvox, int co, float *__restrict__ db) {
  const int c = blockIdx.x;
  __shared__ float sh[256];
  float s = 0.0f;
  for (int64_t v = threadIdx.x; v < nvox; v += blockDim.x) s += __bfloat162float(dy[v * co + c]);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[c] = sh[0];
}

// ------------------------------------------------------------------- grid transfer ops ----
// Full weighting (m+1)^3 <- (2m+1)^3, scaled by `scale`; weights 1/4, 1/2, 1/4 per axis.
__global__ void restrict_k(const bf16 *__restrict__ in, int nfx, int nfy, int nfz, int c, bf16 *__restrict__ out,
                           float scale) {
  const int ncx = (nfx + 1) / 2, ncy = (nfy + 1) / 2, ncz = (nfz + 1) / 2;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)ncx * ncy * ncz * c;
  if (i >= n) return;
  const int ch = (int)(i % c);
  const int64_t v = i / c;
  const int cx = (int)(v % ncx), cy = (int)((v / ncx) % ncy), cz = (int)(v / ((int64_t)ncx * ncy));
  float s = 0.0f;
  for (int dz = -1; dz <= 1; ++dz) {
    const int fz = 2 * cz + dz;
    if (fz < 0 || fz >= nfz) continue;
    const float wz = dz == 0 ? 0.5f : 0.25f;
    for (int dy = -1; dy <= 1; ++dy) {
      const int fy = 2 * cy + dy;
      if (fy < 0 || fy >= nfy) continue;
      const float wy = dy == 0 ? 0.5f : 0.25f;
      for (int dx = -1; dx <= 1; ++dx) {
        const int fx = 2 * cx + dx;
        if (fx < 0 || fx >= nfx) continue;
        const float wx = dx == 0 ? 0.5f : 0.25f;
        s += wx * wy * wz * __bfloat162float(in[(((int64_t)fz * nfy + fy) * nfx + fx) * c + ch]);
      }
    }
  }
  out[i] = __float2bfloat16(s * scale);
}

// Trilinear prolongation (2m+1)^3 <- (m+1)^3, scaled by `scale`.
__global__ void prolong_k(const bf16 *__restrict__ in, int ncx, int ncy, int ncz, int c, bf16 *__restrict__ out,
                          float scale) {
  const int nfx = 2 * ncx - 1, nfy = 2 * ncy - 1, nfz = 2 * ncz - 1;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)nfx * nfy * nfz * c;
  if (i >= n) return;
  const int ch = (int)(i % c);
  const int64_t v = i / c;
  const int fx = (int)(v % nfx), fy = (int)((v / nfx) % nfy), fz = (int)(v / ((int64_t)nfx * nfy));
  float s = 0.0f;
  const int xs[2] = {fx / 2, (fx + 1) / 2}, ys[2] = {fy / 2, (fy + 1) / 2}, zs[2] = {fz / 2, (fz + 1) / 2};
  const int nxp = (fx & 1) ? 2 : 1, nyp = (fy & 1) ? 2 : 1, nzp = (fz & 1) ? 2 : 1;
  const float w = 1.0f / (float)(nxp * nyp * nzp);
  for (int a = 0; a < nzp; ++a)
    for (int b = 0; b < nyp; ++b)
      for (int d = 0; d < nxp; ++d)
        s += __bfloat162float(in[(((int64_t)zs[a] * ncy + ys[b]) * ncx + xs[d]) * c + ch]);
  out[i] = __float2bfloat16(s * w * scale);
}

// d = d_out * (act > 0)
__global__ void relu_mask(const bf16 *__restrict__ d, const bf16 *__restrict__ act, int64_t n, bf16 *__restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = __bfloat162float(act[i]) > 0.0f ? d[i] : __float2bfloat16(0.0f);
}

// a += b (bf16, FP32 add)
__global__ void add_bf(bf16 *__restrict__ a, const bf16 *__restrict__ b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) a[i] = __float2bfloat16(__bfloat162float(a[i]) + __bfloat162float(b[i]));
}

__global__ void f32_to_bf16(const float *__restrict__ a, bf16 *__restrict__ b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16(a[i]);
}

}  // namespace

// ----------------------------------------------------------------------------- entry points ----
extern "C" mf_status mf_conv3d_fwd(const void *x, int32_t nx, int32_t ny, int32_t nz, int32_t cin, const void *w,
                                   const float *bias, int32_t cout, const void *skip, int32_t relu, void *y_bf16,
                                   float *y_f32, mf_stream stream) {
  mf_clear_error();
  MF_ARG(x && w && (y_bf16 || y_f32) && nx > 0 && ny > 0 && nz > 0, "mf_conv3d_fwd: bad argument");
  ConvArgs a{};
  a.in = (const bf16 *)x;
  a.nx = nx; a.ny = ny; a.nz = nz; a.ck = cin;
  a.w = (const bf16 *)w;
  a.bias = bias;
  a.skip = (const bf16 *)skip;
  a.relu = relu;
  a.cn = cout;
  a.out_bf = (bf16 *)y_bf16;
  a.out_f = y_f32;
  return launch_conv<0>(a, (cudaStream_t)stream);
}

extern "C" mf_status mf_conv3d_dgrad(const void *dy, int32_t nx, int32_t ny, int32_t nz, int32_t cin, const void *w,
                                     int32_t cout, void *dx_bf16, float *dx_f32, mf_stream stream) {
  mf_clear_error();
  MF_ARG(dy && w && (dx_bf16 || dx_f32) && nx > 0 && ny > 0 && nz > 0, "mf_conv3d_dgrad: bad argument");
  ConvArgs a{};
  a.in = (const bf16 *)dy;
  a.nx = nx; a.ny = ny; a.nz = nz; a.ck = cout;
  a.w = (const bf16 *)w;
  a.cn = cin;
  a.out_bf = (bf16 *)dx_bf16;
  a.out_f = dx_f32;
  return launch_conv<1>(a, (cudaStream_t)stream);
}

static int64_t wgrad_parts(int64_t nvox) {
  int64_t p = (nvox + 4095) / 4096;
  return p < 1 ? 1 : p > 64 ? 64 : p;
}

extern "C" int64_t mf_conv3d_wgrad_workspace(int32_t nx, int32_t ny, int32_t nz, int32_t cin, int32_t cout) {
  return wgrad_parts((int64_t)nx * ny * nz) * 27 * cin * cout * (int64_t)sizeof(float);
}

extern "C" mf_status mf_conv3d_wgrad(const void *x, const void *dy, int32_t nx, int32_t ny, int32_t nz, int32_t cin,
                                     int32_t cout, float *dw, float *db, float *workspace, int64_t ws_bytes,
                                     mf_stream stream) {
  mf_clear_error();
  MF_ARG(x && dy && dw && workspace && cin > 0 && cout > 0 && cin <= 64 && cout <= 64, "mf_conv3d_wgrad: bad argument");
  const int64_t nvox = (int64_t)nx * ny * nz;
  const int64_t parts = wgrad_parts(nvox);
  MF_ARG(ws_bytes >= mf_conv3d_wgrad_workspace(nx, ny, nz, cin, cout), "mf_conv3d_wgrad: workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  mf_count_launches(db ? 3 : 2);
  conv_wgrad_part<<<(unsigned)(27 * parts), kWgThreads, 0, s>>>((const bf16 *)x, (const bf16 *)dy, nx, ny, nz, cin,
                                                                cout, (int)parts, workspace);
  const int n = 27 * cin * cout;
  conv_wgrad_reduce<<<(n + 255) / 256, 256, 0, s>>>(workspace, (int)parts, n, dw);
  if (db) bias_grad<<<cout, 256, 0, s>>>((const bf16 *)dy, nvox, cout, db);
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

extern "C" mf_status mf_grid_restrict(const void *in, int32_t nfx, int32_t nfy, int32_t nfz, int32_t c, void *out,
                                      float scale, mf_stream stream) {
  mf_clear_error();
  MF_ARG(in && out && nfx % 2 == 1 && nfy % 2 == 1 && nfz % 2 == 1 && c > 0, "mf_grid_restrict: bad argument");
  const int64_t n = (int64_t)((nfx + 1) / 2) * ((nfy + 1) / 2) * ((nfz + 1) / 2) * c;
  mf_count_launches(1);
  restrict_k<<<blocks_for(n), kThreads, 0, (cudaStream_t)stream>>>((const bf16 *)in, nfx, nfy, nfz, c, (bf16 *)out, scale);
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

extern "C" mf_status mf_grid_prolong(const void *in, int32_t ncx, int32_t ncy, int32_t ncz, int32_t c, void *out,
                                     float scale, mf_stream stream) {
  mf_clear_error();
  MF_ARG(in && out && ncx > 0 && ncy > 0 && ncz > 0 && c > 0, "mf_grid_prolong: bad argument");
  const int64_t n = (int64_t)(2 * ncx - 1) * (2 * ncy - 1) * (2 * ncz - 1) * c;
  mf_count_launches(1);
  prolong_k<<<blocks_for(n), kThreads, 0, (cudaStream_t)stream>>>((const bf16 *)in, ncx, ncy, ncz, c, (bf16 *)out, scale);
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

// internal helpers used by the network runtime (mf_net.cu)
mf_status nn_relu_mask(const void *d, const void *act, int64_t n, void *out, cudaStream_t s) {
  mf_count_launches(1);
  relu_mask<<<blocks_for(n), kThreads, 0, s>>>((const bf16 *)d, (const bf16 *)act, n, (bf16 *)out);
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}
mf_status nn_add(void *a, const void *b, int64_t n, cudaStream_t s) {
  mf_count_launches(1);
  add_bf<<<blocks_for(n), kThreads, 0, s>>>((bf16 *)a, (const bf16 *)b, n);
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}
mf_status nn_f32_to_bf16(const float *a, void *b, int64_t n, cudaStream_t s) {
  mf_count_launches(1);
  f32_to_bf16<<<blocks_for(n), kThreads, 0, s>>>(a, (bf16 *)b, n);
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}
