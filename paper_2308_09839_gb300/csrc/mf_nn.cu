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
//  * conv_mma: implicit-GEMM convolution, persistent CTAs over work items of 16x4x4 output voxels
//    (M = 256 per item, N = output channels, K = 27 taps x input channels).  Each item's 18x6x6
//    input halo is staged in shared memory (channels-last, rows padded by 16 bytes); the weights of
//    all taps are staged once per CTA when they fit (else in groups of 9 taps); ldmatrix feeds
//    mma.sync m16n8k16 BF16 x BF16 -> FP32.  The same kernel computes the input gradient (MODE 1)
//    with the mirrored, transposed weights.
//  * conv_wgrad_mma: weight and bias gradients on the tensor cores (per tap a GEMM contracting over
//    voxels, ldmatrix.trans fragments, FP32 accumulation), partial sums per CTA reduced in fixed
//    order (deterministic).
//  * restrict / prolong (and their adjoints as scaled prolong / restrict), relu masks, loss, Adam.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "mf_internal.cuh"
#include "mf_umma.cuh"

typedef __nv_bfloat16 bf16;

namespace {

// Work item: 16 x 4 x 4 output voxels (8 warps; warp w computes the two x-rows of 16 voxels
// m16 = 2w, 2w+1 as m16n8k16 row tiles); input halo 18 x 6 x 6 voxels.
constexpr int TXc = 16, TYc = 4, TZc = 4, HXc = TXc + 2, HYc = TYc + 2, HZc = TZc + 2, NHc = HXc * HYc * HZc;
constexpr int kConvThreads = 256;

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
  int tiles_x, tiles_y, tiles;
  int cphys;              // channels per voxel of `in` in memory (>= ck; 0: ck), tensor-core path only
  // forward (MODE 0) on the pipelined tensor-core path only: this launch computes output channels
  // n0 .. n0 + cn - 1 of cs (weights [27][ck][cs], bias [cs], skip and outputs [..][cs]); 0, 0: all
  int n0, cs;
};

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// ldmatrix: four (two) 8x8 b16 matrices; lane L supplies the address of row L % 8 of matrix L / 8.
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const bf16 *p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(s));
}
__device__ __forceinline__ void ldsm_x2(uint32_t (&r)[2], const bf16 *p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(s));
}

// CKP: input channels padded to a multiple of 16; CN: output channels padded to a multiple of 8.
// SK: shared row length (16 bytes of padding keep the ldmatrix rows on distinct banks); G: taps whose
// weights are staged at once (all 27 when they fit, which then stay resident for the CTA's life).
template <int CKP, int CN>
struct ConvCfg {
  static constexpr int SK = CKP + 8;
  static constexpr int G = ((NHc + 27 * CN) * SK * 2 <= 220 * 1024) ? 27 : 9;
  static constexpr int SMEM = (NHc + G * CN) * SK * 2;
};

// Implicit-GEMM 3x3x3 convolution, persistent: each CTA loops over work items.  Per item the input
// halo is staged in shared memory (16-byte loads when the channel count is the padded one), then
// for each tap and 16-channel chunk the A fragments (rows = the tap-shifted halo rows) and B
// fragments (the tap's weights) are read with ldmatrix and issued as mma.sync m16n8k16 BF16 x BF16
// -> FP32.  MODE 1 computes the input gradient with the mirrored, transposed weights.
template <int CKP, int CN, int MODE>
__global__ void __launch_bounds__(kConvThreads) conv_mma(ConvArgs a) {
  using Cfg = ConvCfg<CKP, CN>;
  constexpr int SK = Cfg::SK, G = Cfg::G;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bf16 *in_s = reinterpret_cast<bf16 *>(smem_raw);
  bf16 *w_s = in_s + NHc * SK;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const bf16 zero = __float2bfloat16(0.0f);
  auto stage_w = [&](int t0) {  // weights of taps [t0, t0 + G) as w_s[tap - t0][n][k], zero padded
    for (int idx = tid; idx < G * CN * CKP; idx += kConvThreads) {
      const int k = idx % CKP, n = (idx / CKP) % CN, tl = idx / (CKP * CN), tap = t0 + tl;
      bf16 v = zero;
      if (k < a.ck && n < a.cn) {
        if (MODE == 0) v = a.w[((int64_t)tap * a.ck + k) * a.cn + n];
        else v = a.w[((int64_t)(26 - tap) * a.cn + n) * a.ck + k];
      }
      w_s[(tl * CN + n) * SK + k] = v;
    }
  };
  const bool vec = a.ck == CKP && ((uintptr_t)a.in & 15) == 0;
  if (G == 27) stage_w(0);  // published by the first barrier of the loop
  if (!vec)  // channels [ck, CKP) of the halo stay zero: only [0, ck) is rewritten per item
    for (int idx = tid; idx < NHc * SK; idx += kConvThreads) in_s[idx] = zero;

  for (int item = blockIdx.x; item < a.tiles; item += gridDim.x) {
    const int bx = item % a.tiles_x, by = (item / a.tiles_x) % a.tiles_y, bz = item / (a.tiles_x * a.tiles_y);
    const int x0 = bx * TXc, y0 = by * TYc, z0 = bz * TZc;
    __syncthreads();  // the previous item's reads of in_s are done
    if (vec) {
      constexpr int CH = CKP / 8;  // 16-byte chunks per voxel
      for (int idx = tid; idx < NHc * CH; idx += kConvThreads) {
        const int hv = idx / CH, ch = idx % CH;
        const int hx = hv % HXc, hy = (hv / HXc) % HYc, hz = hv / (HXc * HYc);
        const int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = z0 - 1 + hz;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz)
          v = __ldg(reinterpret_cast<const uint4 *>(a.in + (((int64_t)gz * a.ny + gy) * a.nx + gx) * CKP) + ch);
        *reinterpret_cast<uint4 *>(in_s + hv * SK + ch * 8) = v;
      }
    } else {
      for (int idx = tid; idx < NHc * a.ck; idx += kConvThreads) {
        const int hv = idx / a.ck, c = idx % a.ck;
        const int hx = hv % HXc, hy = (hv / HXc) % HYc, hz = hv / (HXc * HYc);
        const int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = z0 - 1 + hz;
        bf16 v = zero;
        if (gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz)
          v = a.in[(((int64_t)gz * a.ny + gy) * a.nx + gx) * a.ck + c];
        in_s[hv * SK + c] = v;
      }
    }
    float acc[2][CN / 8][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < CN / 8; ++nt)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[mt][nt][j] = 0.0f;
    for (int t0 = 0; t0 < 27; t0 += G) {
      if (G < 27) {
        __syncthreads();  // the previous group's weights are no longer read
        stage_w(t0);
      }
      __syncthreads();
#pragma unroll 1
      for (int tl = 0; tl < G; ++tl) {
        const int tap = t0 + tl, dx = tap % 3, dy = (tap / 3) % 3, dz = tap / 9;
        const bf16 *arow[2];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          const int m16 = 2 * warp + mt, ty = m16 & 3, tz = m16 >> 2;
          arow[mt] = in_s + ((tz + dz) * (HXc * HYc) + (ty + dy) * HXc + (lane & 15) + dx) * SK + 8 * (lane >> 4);
        }
        const bf16 *brow = w_s + (tl * CN + (lane & 7)) * SK + 8 * ((lane >> 3) & 1);
#pragma unroll
        for (int k0 = 0; k0 < CKP; k0 += 16) {
          uint32_t af[2][4];
          ldsm_x4(af[0], arow[0] + k0);
          ldsm_x4(af[1], arow[1] + k0);
#pragma unroll
          for (int nt = 0; nt < CN / 8; ++nt) {
            uint32_t bfr[2];
            ldsm_x2(bfr, brow + nt * 8 * SK + k0);
            mma_bf16(acc[0][nt], af[0][0], af[0][1], af[0][2], af[0][3], bfr[0], bfr[1]);
            mma_bf16(acc[1][nt], af[1][0], af[1][1], af[1][2], af[1][3], bfr[0], bfr[1]);
          }
        }
      }
    }
    // epilogue: rows g and g + 8 of each m16 tile are the voxels x0 + g (+8) of that x-row
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int m16 = 2 * warp + mt;
      const int gy = y0 + (m16 & 3), gz = z0 + (m16 >> 2);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int gx = x0 + g + 8 * h;
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
  }
}

// Resident CTAs per SM of a persistent kernel: the occupancy calculator's figure, or the bound from
// the device's shared-memory, register and thread limits if that is higher (the calculator can
// assume a smaller shared-memory carveout than the one the kernel requested), capped by the tensor
// memory: resident CTAs x `cols` columns must fit the 512 columns of an SM.  0 on a CUDA error.
static int persistent_resident(const void *kern, int threads, int dyn_smem, int cols) {
  int r = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, kern, threads, dyn_smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaFuncAttributes fa;
  int dev = 0, smem_sm = 0, resv = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaFuncGetAttributes(&fa, kern) == cudaSuccess &&
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess) {
    const int per_cta = dyn_smem + (int)fa.sharedSizeBytes + resv;
    const int warps = (threads + 31) / 32;
    const int regs_warp = ((std::max(fa.numRegs, 1) * 32 + 255) / 256) * 256;  // allocation unit: 256 per warp
    const int by_smem = smem_sm / std::max(per_cta, 1);
    const int by_regs = 65536 / (regs_warp * warps);
    const int by_warps = 64 / warps;
    r = std::max(r, std::min(std::min(by_smem, by_regs), std::min(by_warps, 32)));
  } else {
    cudaGetLastError();
  }
  return std::max(1, std::min(r, 512 / std::max(cols, 1)));
}

template <int CKP, int CN, int MODE>
mf_status launch_conv_t(ConvArgs a, cudaStream_t s) {
  constexpr int smem = ConvCfg<CKP, CN>::SMEM;
  static std::atomic<int> resident{0};  // CTAs per SM: a property of the kernel
  if (resident.load() == 0) {
    MF_CUDA(cudaFuncSetAttribute(conv_mma<CKP, CN, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int r = 0;
    MF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, conv_mma<CKP, CN, MODE>, kConvThreads, smem));
    resident.store(std::max(r, 1));
  }
  a.tiles = a.tiles_x * a.tiles_y * ((a.nz + TZc - 1) / TZc);
  const int grid = std::min(a.tiles, device_sm_count() * resident.load());
  mf_count_launches(1);
  conv_mma<CKP, CN, MODE><<<grid, kConvThreads, smem, s>>>(a);
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

// ------------------------------------------------------------ tcgen05 implicit-GEMM convolution ----
// The same convolution on the 5th-generation tensor cores, for 16, 32 or 64 input channels.
//
// Work item: 8 (x) x 16 (y) x TZ (z) output voxels.  The item's input halo of 10 x 18 x (TZ + 2)
// voxels arrives by one TMA tensor load, in the shared-memory order [z][channel chunk][y][x][8
// channels] (a 5-D tensor map over the channels-last input whose chunk dimension has a 16-byte
// stride), with zeros outside the grid.  In that order the 8 voxels of an x-row of the tile form a
// 128-byte core matrix of the no-swizzle K-major layout for every channel chunk, so the A operand of
// tap (dx, dy, dz) for output plane z is the halo itself at a byte offset: MMA row m = x + 8 y reads
// halo voxel (x + dx, y + dy, z + dz), with rows grouped in eights 160 bytes apart (one halo y-row)
// and channel chunks 2880 bytes apart.  No im2col copy is made.  The weights of all taps (or of 9 at a
// time when they do not fit) are stored by the threads in the same canonical layout ([tap][channel
// chunk][output channel][8]).  One thread issues tcgen05.mma M = 128, N = output channels, K = 16
// for every (plane, tap, channel pair), accumulating in tensor memory (one 128 x N FP32 accumulator
// per output plane); tcgen05.commit signals an mbarrier, and the four warps read the accumulators
// back (warp w: tile rows 32 w .. 32 w + 31) and apply bias, skip, ReLU and the BF16/FP32 stores.
// Waits are bounded: on a timeout the kernel records an error in tc_status and stops.
constexpr int kTcThreads = 128;

// The tcgen05 path is the default; MF_CONV_MMA_SYNC=1 in the environment selects the mma.sync
// kernel instead (for comparisons).
static bool conv_tc_enabled() {
  static const bool on = [] {
    const char *e = getenv("MF_CONV_MMA_SYNC");
    return !(e && e[0] == '1');
  }();
  return on;
}
constexpr int TXt = 8, TYt = 16, HXt = TXt + 2, HYt = TYt + 2;
constexpr int kTcYS = HXt * 16, kTcKCS = HYt * kTcYS;  // halo byte strides: y-row, channel chunk
constexpr long long kTcBudget = 1ll << 31;             // clock cycles per wait (about one second)

__device__ int tc_status;  // nonzero after a timed-out wait (read by the network's synchronous calls)

template <int CKP, int CN>
struct TcCfg {
  static constexpr int KC = CKP / 8;                 // channel chunks
  static constexpr int TZ = CKP == 64 ? 2 : 4;        // output planes per item
  static constexpr int HZ = TZ + 2;
  static constexpr int ZS = KC * kTcKCS;              // halo byte stride of a z-plane
  static constexpr int HALO = HZ * ZS;                // halo bytes
  static constexpr int TAPB = CKP * CN * 2;           // weight bytes per tap
  static constexpr int G = (HALO + 27 * TAPB <= 200 * 1024) ? 27 : 9;  // taps staged at once
  static constexpr int SMEM = 1024 + HALO + G * TAPB; // + alignment slack
  static constexpr int COLS = TZ * CN <= 32 ? 32 : TZ * CN <= 64 ? 64 : TZ * CN <= 128 ? 128 : 256;
};

struct TcArgs {
  int nx, ny, nz, ck, cn, relu;
  const bf16 *w;
  const float *bias;
  const bf16 *skip;
  bf16 *out_bf;
  float *out_f;
  int tiles_x, tiles_y, tiles;
  int vec_out;  // cn == CN and 16-byte aligned output / skip: vector epilogue
  int n0, cs;   // conv_tcp, MODE 0: output channels n0 .. n0 + cn - 1 of cs per voxel (else 0 and cn)
};

template <int CKP, int CN, int MODE>
__global__ void __launch_bounds__(kTcThreads) conv_tc(TcArgs a, const __grid_constant__ CUtensorMap tmap) {
  using Cfg = TcCfg<CKP, CN>;
  constexpr int KC = Cfg::KC, TZ = Cfg::TZ, G = Cfg::G, NG = 27 / G, KS = CKP / 16;
  constexpr uint32_t IDESC = umma::idesc_bf16(128, CN);
  extern __shared__ __align__(16) unsigned char tc_smem_raw[];
  __shared__ __align__(8) uint64_t halo_bar, mma_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  // 1024-byte aligned halo, weights after it
  unsigned char *base = tc_smem_raw + ((1024 - (umma::smem_u32(tc_smem_raw) & 1023)) & 1023);
  unsigned char *halo = base;
  unsigned char *wsm = base + Cfg::HALO;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    umma::mbar_init(&halo_bar, 1);
    umma::mbar_init(&mma_bar, 1);
    umma::mbar_init_fence();
    abort_flag = 0;
  }
  if (warp == 0) umma::tmem_alloc(&tmem_slot, Cfg::COLS);
  // weights of taps [t0, t0 + G) in the canonical K-major layout: 16 bytes = 8 input channels of one
  // output channel; zero beyond the real channel counts
  auto stage_w = [&](int t0) {
    for (int idx = tid; idx < G * KC * CN; idx += kTcThreads) {
      const int n = idx % CN, kc = (idx / CN) % KC, tl = idx / (CN * KC), tap = t0 + tl;
      __align__(16) bf16 v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k = kc * 8 + j;
        bf16 e = __float2bfloat16(0.0f);
        if (k < a.ck && n < a.cn) {
          if (MODE == 0) e = a.w[((int64_t)tap * a.ck + k) * a.cn + n];
          else e = a.w[((int64_t)(26 - tap) * a.cn + n) * a.ck + k];
        }
        v[j] = e;
      }
      *reinterpret_cast<uint4 *>(wsm + (size_t)tl * Cfg::TAPB + ((size_t)kc * CN + n) * 16) =
          *reinterpret_cast<const uint4 *>(v);
    }
  };
  if (G == 27) stage_w(0);
  umma::fence_proxy_async_smem();
  umma::tc_fence_before_sync();
  __syncthreads();
  umma::tc_fence_after_sync();
  const uint32_t tmem = tmem_slot;
  const uint32_t halo_a = umma::smem_u32(halo), w_a = umma::smem_u32(wsm);
  uint32_t halo_phase = 0, mma_phase = 0;

  auto wait_all = [&](uint64_t *bar, uint32_t &phase) {  // every thread waits; a timeout aborts the CTA
    if (!umma::mbar_wait(bar, phase, kTcBudget)) {
      abort_flag = 1;
      atomicExch(&tc_status, 1);
    }
    phase ^= 1u;
  };

  for (int item = blockIdx.x; item < a.tiles; item += gridDim.x) {
    const int bx = item % a.tiles_x, by = (item / a.tiles_x) % a.tiles_y, bz = item / (a.tiles_x * a.tiles_y);
    const int x0 = bx * TXt, y0 = by * TYt, z0 = bz * TZ;
    if (tid == 0) {
      umma::mbar_arrive_expect_tx(&halo_bar, Cfg::HALO);
      umma::tma_load_5d(halo, &tmap, &halo_bar, 0, x0 - 1, y0 - 1, 0, z0 - 1);
    }
    for (int gi = 0; gi < NG; ++gi) {
      if (NG > 1) {
        if (gi > 0) wait_all(&mma_bar, mma_phase);  // the previous group's MMAs no longer read wsm
        __syncthreads();
        if (abort_flag) break;
        stage_w(gi * G);
        umma::fence_proxy_async_smem();
        __syncthreads();
      }
      if (gi == 0) wait_all(&halo_bar, halo_phase);
      __syncthreads();
      if (abort_flag) break;
      if (tid == 0) {
        umma::tc_fence_after_sync();
        const uint64_t ad0 = umma::sdesc(halo_a, kTcKCS, kTcYS), bd0 = umma::sdesc(w_a, CN * 16, 128);
#pragma unroll 1
        for (int tl = 0; tl < G; ++tl) {
          const int tap = gi * G + tl, dx = tap % 3, dy = (tap / 3) % 3, dz = tap / 9;
          const uint32_t ta = (uint32_t)(dz * Cfg::ZS + dy * kTcYS + dx * 16), tb = (uint32_t)(tl * Cfg::TAPB);
#pragma unroll
          for (int zi = 0; zi < TZ; ++zi)
#pragma unroll
            for (int ks = 0; ks < KS; ++ks)
              umma::mma_bf16(tmem + (uint32_t)(zi * CN),
                             umma::sdesc_add(ad0, ta + (uint32_t)(zi * Cfg::ZS + 2 * ks * kTcKCS)),
                             umma::sdesc_add(bd0, tb + (uint32_t)(2 * ks * CN * 16)), IDESC,
                             (tap > 0 || ks > 0) ? 1u : 0u);
        }
        umma::mma_commit(&mma_bar);
      }
    }
    if (abort_flag) break;
    wait_all(&mma_bar, mma_phase);  // every MMA of the item is complete
    __syncthreads();
    if (abort_flag) break;
    umma::tc_fence_after_sync();
    // epilogue: warp w holds tile rows m = 32 w + lane, i.e. x = m % 8, y = m / 8
    const int m = 32 * warp + lane, gx = x0 + (m & 7), gy = y0 + (m >> 3);
#pragma unroll 1
    for (int zi = 0; zi < TZ; ++zi) {
      const int gz = z0 + zi;
      const bool in = gx < a.nx && gy < a.ny && gz < a.nz;
      const int64_t vox = ((int64_t)gz * a.ny + gy) * a.nx + gx;
#pragma unroll
      for (int c0 = 0; c0 < CN; c0 += 16) {
        float v[16];
        umma::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(zi * CN + c0), v);
        if (!in) continue;
        if (MODE == 0) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = c0 + j;
            if (n < a.cn) {
              if (a.bias) v[j] += __ldg(a.bias + n);
              if (a.skip && !a.vec_out) v[j] += __bfloat162float(a.skip[vox * a.cn + n]);
            }
          }
          if (a.skip && a.vec_out) {
            const uint4 *sp = reinterpret_cast<const uint4 *>(a.skip + vox * CN + c0);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const uint4 u = __ldg(sp + h);
              const __nv_bfloat162 *q = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const float2 f = __bfloat1622float2(q[j]);
                v[8 * h + 2 * j] += f.x;
                v[8 * h + 2 * j + 1] += f.y;
              }
            }
          }
          if (a.relu)
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j], 0.0f);
        }
        if (a.vec_out) {
          if (a.out_bf) {
            __align__(16) __nv_bfloat162 q[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) q[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
            uint4 *op = reinterpret_cast<uint4 *>(a.out_bf + vox * CN + c0);
            op[0] = reinterpret_cast<const uint4 *>(q)[0];
            op[1] = reinterpret_cast<const uint4 *>(q)[1];
          }
          if (a.out_f) {
            float4 *op = reinterpret_cast<float4 *>(a.out_f + vox * CN + c0);
#pragma unroll
            for (int j = 0; j < 4; ++j) op[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = c0 + j;
            if (n < a.cn) {
              if (a.out_bf) a.out_bf[vox * a.cn + n] = __float2bfloat16(v[j]);
              if (a.out_f) a.out_f[vox * a.cn + n] = v[j];
            }
          }
        }
      }
    }
    umma::tc_fence_before_sync();
    __syncthreads();  // accumulators read before the next item's MMAs overwrite them
  }
  // a CTA that gave up still owns the copies and MMAs it issued: wait for them (bounded) so that
  // nothing writes this CTA's shared or tensor memory after it exits
  if (abort_flag && tid == 0) {
    umma::mbar_wait(&halo_bar, halo_phase, kTcBudget);
    umma::mbar_wait(&mma_bar, mma_phase, kTcBudget);
  }
  umma::tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, Cfg::COLS);
}

// Pipelined form of conv_tc for the shapes whose 27 taps of weights fit in shared memory next to one
// or two halo buffers.  Warp-specialised: warp 0 loads the halos of the CTA's items by TMA into a
// ring of NS buffers; warp 1 issues the MMAs of an item into one of two accumulator sets in tensor
// memory, as soon as its halo has arrived and the epilogue has released that set, and commits to
// the halo's "empty" and the set's "full" barrier; warps 2-5 drain the accumulators (warp w: tile
// rows 32 (w % 4) .. + 31, its tensor-memory lane quarter) while the next item's loads and MMAs run.
// Per item the planes TZ and the stages NS are the largest that fit.
constexpr int kTcpThreads = 192;

template <int CKP, int CN>
struct TcpCfg {
  static constexpr int KC = CKP / 8;
  static constexpr int TAPB = CKP * CN * 2;
  static constexpr int W = 27 * TAPB;
  static constexpr int LIMIT = 220 * 1024;
  static constexpr int halo(int tz) { return (tz + 2) * KC * kTcKCS; }
  // one plane per item only when an accumulator set still spans 32 columns (the epilogue reads the
  // sets in blocks of 32): with 16 output channels the single-buffered two-plane form is taken instead
  static constexpr int TZ = (2 * halo(4) + W <= LIMIT)               ? 4
                            : (2 * halo(2) + W <= LIMIT)             ? 2
                            : (2 * halo(1) + W <= LIMIT && CN >= 32) ? 1
                            : (halo(2) + W <= LIMIT)                 ? 2
                                                                     : 1;
  static constexpr int NS = (2 * halo(TZ) + W <= LIMIT) ? 2 : 1;
  static constexpr int HALO = halo(TZ);
  static constexpr bool FITS = NS * HALO + W <= LIMIT;
  static constexpr int ZS = KC * kTcKCS;
  static constexpr int SMEM = 1024 + NS * HALO + W;
  static constexpr int ACC = TZ * CN;  // columns of one accumulator set
  static constexpr int COLS = 2 * ACC <= 32 ? 32 : 2 * ACC <= 64 ? 64 : 2 * ACC <= 128 ? 128 : 2 * ACC <= 256 ? 256 : 512;
};

// All 27 taps of weights in the canonical K-major layout, the three taps of an (x, y) shift side by
// side along N: w_s[shift][k / 8][dz CN + n][k % 8] with tap = 9 dz + shift (zero beyond the real
// channel counts), so that one MMA can take the taps dz = d0..d1 of a shift as a B operand of
// (d1 - d0 + 1) CN columns.  The global weights are read in 16-byte runs along their contiguous
// index (output channels n in the forward layout [tap][k][n], input channels k in the transposed one
// of the input gradient) and scattered into shared memory as 2-byte stores.
template <int CKP, int CN, int MODE>
__device__ __forceinline__ void stage_weights(const TcArgs &a, unsigned char *wsm, int tid, int nthreads) {
  constexpr int KC = CKP / 8;
  bf16 *w_s = reinterpret_cast<bf16 *>(wsm);
  auto put = [&](int tap, int k, int n, bf16 v) {
    w_s[((size_t)((tap % 9) * KC + (k >> 3)) * (3 * CN) + (tap / 9) * CN + n) * 8 + (k & 7)] = v;
  };
  const bf16 zero = __float2bfloat16(0.0f);
  // contiguous dimension: n (MODE 0, length cn) or k (MODE 1, length ck); the other one is strided
  const int cl = MODE == 0 ? a.cn : a.ck, ol = MODE == 0 ? CKP : CN, cpad = MODE == 0 ? CN : CKP;
  const bool vec = cl % 8 == 0 && a.cs % 8 == 0 && a.n0 % 8 == 0 && ((uintptr_t)a.w & 15) == 0;
  const int runs = cpad / 8;  // 8-element runs along the contiguous dimension
  for (int idx = tid; idx < 27 * ol * runs; idx += nthreads) {
    const int o = idx % ol, run = (idx / ol) % runs, tap = idx / (runs * ol);  // o fastest: fewer bank conflicts
    const int c0 = run * 8;
    __align__(16) bf16 v[8];
    const bool inside = MODE == 0 ? (o < a.ck && c0 < a.cn) : (o < a.cn && c0 < a.ck);
    const int64_t base = MODE == 0 ? ((int64_t)tap * a.ck + o) * a.cs + a.n0 + c0
                                   : ((int64_t)(26 - tap) * a.cn + o) * a.ck + c0;
    if (inside && vec) {
      *reinterpret_cast<uint4 *>(v) = __ldg(reinterpret_cast<const uint4 *>(a.w + base));
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = (inside && c0 + j < cl) ? a.w[base + j] : zero;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (MODE == 0) put(tap, o, c0 + j, v[j]);   // o = k, contiguous n
      else put(tap, c0 + j, o, v[j]);             // o = n, contiguous k
    }
  }
}

template <int CKP, int CN, int MODE>
__global__ void __launch_bounds__(kTcpThreads) conv_tcp(TcArgs a, const __grid_constant__ CUtensorMap tmap) {
  using Cfg = TcpCfg<CKP, CN>;
  constexpr int KC = Cfg::KC, TZ = Cfg::TZ, NS = Cfg::NS, KS = CKP / 16, ACC = Cfg::ACC;
  static_assert(ACC % 32 == 0, "the epilogue reads an accumulator set in blocks of 32 columns");
  extern __shared__ __align__(16) unsigned char tcp_smem_raw[];
  __shared__ __align__(8) uint64_t full[NS], empty[NS], accf[2], acce[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  unsigned char *base = tcp_smem_raw + ((1024 - (umma::smem_u32(tcp_smem_raw) & 1023)) & 1023);
  unsigned char *wsm = base + NS * Cfg::HALO;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  volatile int *abort_v = &abort_flag;

  if (tid == 0) {
    for (int i = 0; i < NS; ++i) {
      umma::mbar_init(&full[i], 1);
      umma::mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      umma::mbar_init(&accf[i], 1);
      umma::mbar_init(&acce[i], 4);
    }
    umma::mbar_init_fence();
    abort_flag = 0;
  }
  __shared__ float bias_s[CN];
  if (warp == 1) umma::tmem_alloc(&tmem_slot, Cfg::COLS);
  stage_weights<CKP, CN, MODE>(a, wsm, tid, kTcpThreads);
  for (int n = tid; n < CN; n += kTcpThreads) bias_s[n] = (MODE == 0 && a.bias && n < a.cn) ? a.bias[a.n0 + n] : 0.0f;
  umma::fence_proxy_async_smem();
  umma::tc_fence_before_sync();
  __syncthreads();
  umma::tc_fence_after_sync();
  const uint32_t tmem = tmem_slot;
  const int nloc = (int)blockIdx.x < a.tiles ? (a.tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  auto fail = [&]() {
    *abort_v = 1;
    atomicExch(&tc_status, 1);
  };
  auto coords = [&](int i, int &x0, int &y0, int &z0) {
    const int item = blockIdx.x + i * gridDim.x;
    const int bx = item % a.tiles_x, by = (item / a.tiles_x) % a.tiles_y, bz = item / (a.tiles_x * a.tiles_y);
    x0 = bx * TXt;
    y0 = by * TYt;
    z0 = bz * TZ;
  };

  if (warp == 0) {  // ------------------------------------------------------------- TMA producer
    if (lane == 0) {
      int issued = 0;
      for (int i = 0; i < nloc && !*abort_v; ++i) {
        const int s = i % NS;
        if (i >= NS && !umma::mbar_wait(&empty[s], (uint32_t)((i / NS - 1) & 1), kTcBudget)) {
          fail();
          break;
        }
        int x0, y0, z0;
        coords(i, x0, y0, z0);
        umma::mbar_arrive_expect_tx(&full[s], Cfg::HALO);
        umma::tma_load_5d(base + s * Cfg::HALO, &tmap, &full[s], 0, x0 - 1, y0 - 1, 0, z0 - 1);
        ++issued;
      }
      if (*abort_v)  // bounded drain of the copies this CTA still has in flight
        for (int j = issued - 1; j >= 0 && j >= issued - NS; --j)
          umma::mbar_wait(&full[j % NS], (uint32_t)((j / NS) & 1), kTcBudget);
    }
  } else if (warp == 1) {  // --------------------------------------------------------- MMA issue
    if (lane == 0) {
      const uint64_t bd0 = umma::sdesc(umma::smem_u32(wsm), 3 * CN * 16, 128);
      int done = 0;
      for (int i = 0; i < nloc && !*abort_v; ++i) {
        const int s = i % NS, ac = i & 1;
        if (!umma::mbar_wait(&full[s], (uint32_t)((i / NS) & 1), kTcBudget)) {
          fail();
          break;
        }
        if (i >= 2 && !umma::mbar_wait(&acce[ac], (uint32_t)(((i >> 1) - 1) & 1), kTcBudget)) {
          fail();
          break;
        }
        umma::tc_fence_after_sync();
        // Output plane zi accumulates in columns (TZ - 1 - zi) CN of the set (planes in reverse), so
        // that the taps dz = d0..d1 of an (x, y) shift reading halo plane hp (output planes hp - dz)
        // fill adjacent columns: one MMA with N = (d1 - d0 + 1) CN and the shift's weights d0..d1
        // side by side reads its A operand (the halo view) once for up to three taps.  The (0, 0)
        // shift first writes every plane with its dz = 0 tap alone (accumulate off).  All MMAs are
        // unrolled: descriptors are the item's base descriptors plus compile-time offsets.
        const uint64_t ad0 = umma::sdesc(umma::smem_u32(base + s * Cfg::HALO), kTcKCS, kTcYS);
        const uint32_t dcol = tmem + (uint32_t)(ac * ACC);
        auto issue = [&](int shift, int hp, int ks, int dlo, int dhi, uint32_t acc) {
          const int dx = shift % 3, dy = shift / 3;
          const int n = (dhi - dlo + 1) * CN;
          const uint32_t idesc = n == CN ? umma::idesc_bf16(128, CN)
                                 : n == 2 * CN ? umma::idesc_bf16(128, 2 * CN) : umma::idesc_bf16(128, 3 * CN);
          umma::mma_bf16(dcol + (uint32_t)((TZ - 1 - hp + dlo) * CN),
                         umma::sdesc_add(ad0, (uint32_t)(hp * Cfg::ZS + 2 * ks * kTcKCS + dy * kTcYS + dx * 16)),
                         umma::sdesc_add(bd0, (uint32_t)(((shift * KC + 2 * ks) * 3 * CN + dlo * CN) * 16)), idesc,
                         acc);
        };
#pragma unroll
        for (int zi = 0; zi < TZ; ++zi) issue(0, zi, 0, 0, 0, 0u);
#pragma unroll
        for (int shift = 0; shift < 9; ++shift)
#pragma unroll
          for (int ks = 0; ks < KS; ++ks)
#pragma unroll
            for (int hp = 0; hp < TZ + 2; ++hp) {
              const int lo = (shift == 0 && ks == 0) ? max(1, hp - TZ + 1) : max(0, hp - TZ + 1);
              const int hi = min(2, hp);
              if (lo <= hi) issue(shift, hp, ks, lo, hi, 1u);
            }
        umma::mma_commit(&empty[s]);
        umma::mma_commit(&accf[ac]);
        done = i + 1;
      }
      if (*abort_v && done > 0)  // bounded drain of the MMAs still in flight
        umma::mbar_wait(&accf[(done - 1) & 1], (uint32_t)(((done - 1) >> 1) & 1), kTcBudget);
    }
  } else {  // ----------------------------------------------------------------------- epilogue
    const int q = warp & 3, m = 32 * q + lane;
    const bool vskip = MODE == 0 && a.skip && a.vec_out;
    for (int i = 0; i < nloc; ++i) {
      const int ac = i & 1;
      int x0, y0, z0;
      coords(i, x0, y0, z0);
      const int gx = x0 + (m & 7), gy = y0 + (m >> 3);
      // the skip values of the item's voxels are loaded before the wait, so that their latency
      // overlaps the item's MMAs
      uint4 sk[TZ][CN / 8];
      if (vskip) {
#pragma unroll
        for (int zi = 0; zi < TZ; ++zi) {
          const bool in = gx < a.nx && gy < a.ny && z0 + zi < a.nz;
          const uint4 *sp =
              reinterpret_cast<const uint4 *>(a.skip + (((int64_t)(z0 + zi) * a.ny + gy) * a.nx + gx) * a.cs + a.n0);
#pragma unroll
          for (int h = 0; h < CN / 8; ++h) sk[zi][h] = in ? __ldg(sp + h) : make_uint4(0u, 0u, 0u, 0u);
        }
      }
      const bool ok = umma::mbar_wait(&accf[ac], (uint32_t)((i >> 1) & 1), kTcBudget);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) fail();
        break;
      }
      if (*abort_v) break;
      umma::tc_fence_after_sync();
      // the accumulator set (TZ planes x CN columns) in blocks of LW columns, one tensor-memory load
      // and one wait per block, then 16-column groups (plane zi, channels c0 .. c0 + 15)
      constexpr int LW = ACC % 64 == 0 && CN <= 16 ? 64 : 32;
#pragma unroll
      for (int cb = 0; cb < ACC; cb += LW) {
        float vb[LW];
        if constexpr (LW == 64) umma::tmem_ld64(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(ac * ACC + cb), vb);
        else umma::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(ac * ACC + cb), vb);
#pragma unroll
        for (int g = 0; g < LW / 16; ++g) {
          const int zi = TZ - 1 - (cb + 16 * g) / CN, c0 = (cb + 16 * g) % CN;  // planes in reverse
          const int gz = z0 + zi;
          const bool in = gx < a.nx && gy < a.ny && gz < a.nz;
          const int64_t vox = ((int64_t)gz * a.ny + gy) * a.nx + gx;
          float *v = vb + 16 * g;
          if (!in) continue;
          if (MODE == 0) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int n = c0 + j;
              v[j] += bias_s[n];
              if (a.skip && !a.vec_out && n < a.cn) v[j] += __bfloat162float(a.skip[vox * a.cs + a.n0 + n]);
            }
            if (vskip) {
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const uint4 u = sk[zi][c0 / 8 + h];
                const __nv_bfloat162 *qq = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                  const float2 f = __bfloat1622float2(qq[j]);
                  v[8 * h + 2 * j] += f.x;
                  v[8 * h + 2 * j + 1] += f.y;
                }
              }
            }
            if (a.relu)
#pragma unroll
              for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j], 0.0f);
          }
          if (a.vec_out) {
            if (a.out_bf) {
              __align__(16) __nv_bfloat162 qq[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) qq[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
              uint4 *op = reinterpret_cast<uint4 *>(a.out_bf + vox * a.cs + a.n0 + c0);
              op[0] = reinterpret_cast<const uint4 *>(qq)[0];
              op[1] = reinterpret_cast<const uint4 *>(qq)[1];
            }
            if (a.out_f) {
              float4 *op = reinterpret_cast<float4 *>(a.out_f + vox * a.cs + a.n0 + c0);
#pragma unroll
              for (int j = 0; j < 4; ++j) op[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            }
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int n = c0 + j;
              if (n < a.cn) {
                if (a.out_bf) a.out_bf[vox * a.cs + a.n0 + n] = __float2bfloat16(v[j]);
                if (a.out_f) a.out_f[vox * a.cs + a.n0 + n] = v[j];
              }
            }
          }
        }
      }
      umma::tc_fence_before_sync();
      __syncwarp();
      if (lane == 0) umma::mbar_arrive(&acce[ac]);  // this warp's lanes of the set are free again
    }
  }
  umma::tc_fence_before_sync();
  __syncthreads();
  umma::tc_fence_after_sync();
  if (warp == 1) umma::tmem_dealloc(tmem, Cfg::COLS);
}

// 5-D tensor map of a channels-last BF16 tensor [nz][ny][nx][C] (C = 16, 32 or 64) for conv_tc:
// dims (innermost first) 8 channels, x, y, channel chunk, z; strides 2C, 2C nx, 16, 2C nx ny bytes; box
// 8 x 10 x 18 x C/8 x (TZ + 2); zeros outside.  False if the driver rejects it.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

static bool make_halo_map(CUtensorMap *map, const bf16 *in, int nx, int ny, int nz, int C, int hz) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || ((uintptr_t)in & 15) != 0) return false;
  const cuuint64_t dims[5] = {8, (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)(C / 8), (cuuint64_t)nz};
  const cuuint64_t strides[4] = {(cuuint64_t)C * 2, (cuuint64_t)C * 2 * nx, 16, (cuuint64_t)C * 2 * nx * ny};
  const cuuint32_t box[5] = {8, (cuuint32_t)HXt, (cuuint32_t)HYt, (cuuint32_t)(C / 8), (cuuint32_t)hz};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16 *>(in), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Launch the tcgen05 convolution; false (nothing launched) when the tensor map cannot be made.
template <int CKP, int CN, int MODE>
static bool launch_conv_tcp_t(const ConvArgs &c, cudaStream_t s, mf_status *st) {
  using Cfg = TcpCfg<CKP, CN>;
  CUtensorMap map;
  if (!make_halo_map(&map, c.in, c.nx, c.ny, c.nz, CKP, Cfg::TZ + 2)) return false;
  static std::atomic<int> resident{0};
  auto kern = conv_tcp<CKP, CN, MODE>;
  if (resident.load() == 0) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
            cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    const int r = persistent_resident((const void *)kern, kTcpThreads, Cfg::SMEM, Cfg::COLS);
    if (r < 1) return false;
    resident.store(r);
  }
  TcArgs a;
  a.nx = c.nx; a.ny = c.ny; a.nz = c.nz; a.ck = c.ck; a.cn = c.cn; a.relu = c.relu;
  a.w = c.w; a.bias = c.bias; a.skip = c.skip; a.out_bf = c.out_bf; a.out_f = c.out_f;
  a.n0 = MODE == 0 ? c.n0 : 0;
  a.cs = MODE == 0 && c.cs ? c.cs : c.cn;
  a.tiles_x = (c.nx + TXt - 1) / TXt;
  a.tiles_y = (c.ny + TYt - 1) / TYt;
  a.tiles = a.tiles_x * a.tiles_y * ((c.nz + Cfg::TZ - 1) / Cfg::TZ);
  auto al = [](const void *p) { return p == nullptr || ((uintptr_t)p & 15) == 0; };
  a.vec_out = c.cn == CN && a.cs % 8 == 0 && a.n0 % 8 == 0 && al(c.out_bf) && al(c.out_f) && al(c.skip);
  const int grid = std::min(a.tiles, device_sm_count() * resident.load());
  mf_count_launches(1);
  kern<<<grid, kTcpThreads, Cfg::SMEM, s>>>(a, map);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    mf_set_error("conv_tcp launch failed: %s", cudaGetErrorString(e));
    *st = MF_ERR_CUDA;
  } else {
    *st = MF_OK;
  }
  return true;
}

template <int CKP, int CN, int MODE>
static bool launch_conv_tc_t(const ConvArgs &c, cudaStream_t s, mf_status *st) {
  if constexpr (TcpCfg<CKP, CN>::FITS) return launch_conv_tcp_t<CKP, CN, MODE>(c, s, st);
  using Cfg = TcCfg<CKP, CN>;
  CUtensorMap map;
  if (!make_halo_map(&map, c.in, c.nx, c.ny, c.nz, CKP, Cfg::HZ)) return false;
  static std::atomic<int> resident{0};
  auto kern = conv_tc<CKP, CN, MODE>;
  if (resident.load() == 0) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
            cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    const int r = persistent_resident((const void *)kern, kTcThreads, Cfg::SMEM, Cfg::COLS);
    if (r < 1) return false;
    resident.store(r);
  }
  TcArgs a;
  a.nx = c.nx; a.ny = c.ny; a.nz = c.nz; a.ck = c.ck; a.cn = c.cn; a.relu = c.relu;
  a.w = c.w; a.bias = c.bias; a.skip = c.skip; a.out_bf = c.out_bf; a.out_f = c.out_f;
  a.n0 = 0;
  a.cs = c.cn;
  a.tiles_x = (c.nx + TXt - 1) / TXt;
  a.tiles_y = (c.ny + TYt - 1) / TYt;
  a.tiles = a.tiles_x * a.tiles_y * ((c.nz + Cfg::TZ - 1) / Cfg::TZ);
  auto al = [](const void *p) { return p == nullptr || ((uintptr_t)p & 15) == 0; };
  a.vec_out = c.cn == CN && al(c.out_bf) && al(c.out_f) && al(c.skip);
  const int grid = std::min(a.tiles, device_sm_count() * resident.load());
  mf_count_launches(1);
  kern<<<grid, kTcThreads, Cfg::SMEM, s>>>(a, map);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    mf_set_error("conv_tc launch failed: %s", cudaGetErrorString(e));
    *st = MF_ERR_CUDA;
  } else {
    *st = MF_OK;
  }
  return true;
}

// The tcgen05 path when the input has 16, 32 or 64 channels (the tensor map's 16-byte chunks) and
// at most 64 outputs; false otherwise (the caller then runs conv_mma).
template <int MODE>
static bool launch_conv_tc(const ConvArgs &c, cudaStream_t s, mf_status *st) {
  const int ph = c.cphys ? c.cphys : c.ck;  // stored channels: the tensor map's 16-byte chunks
  if (!(ph == 16 || ph == 32 || ph == 64) || c.ck > ph || c.cn < 1 || c.cn > 64) return false;
  const int cnp = c.cn <= 16 ? 16 : c.cn <= 32 ? 32 : 64;
  if constexpr (MODE == 0) {
    // 64 input x more than 32 output channels: the 27 taps of weights (up to 221 KB) do not fit beside
    // a halo, so the output channels are computed in two launches of the pipelined kernel (32 + rest),
    // each with its half of the weights resident, instead of restaging tap groups for every item
    if (ph == 64 && cnp == 64 && c.n0 == 0 && (c.cs == 0 || c.cs == c.cn)) {
      ConvArgs h = c;
      h.cs = c.cn;
      h.cn = 32;
      if (!launch_conv_tcp_t<64, 32, 0>(h, s, st)) return false;
      if (*st != MF_OK) return true;
      h.n0 = 32;
      h.cn = c.cn - 32;
      return launch_conv_tcp_t<64, 32, 0>(h, s, st);
    }
  }
#define TCCASE(K, N) \
  if (ph == K && cnp == N) return launch_conv_tc_t<K, N, MODE>(c, s, st);
  TCCASE(16, 16) TCCASE(16, 32) TCCASE(16, 64)
  TCCASE(32, 16) TCCASE(32, 32) TCCASE(32, 64)
  TCCASE(64, 16) TCCASE(64, 32) TCCASE(64, 64)
#undef TCCASE
  return false;
}

template <int MODE>
mf_status launch_conv(ConvArgs a, cudaStream_t s) {
  if (conv_tc_enabled()) {
    mf_status st = MF_OK;
    if (launch_conv_tc<MODE>(a, s, &st)) return st;
    if (getenv("MF_DEBUG")) fprintf(stderr, "conv: mma.sync path (mode %d, cin %d, cout %d)\n", MODE, a.ck, a.cn);
  }
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
// dw[t][ci][co] = sum_v x[v + off_t][ci] dy[v][co] and db[co] = sum_v dy[v][co] on the tensor
// cores: for each tap a GEMM with M = input channels, N = output channels and K = voxels.  A CTA
// takes 8 taps (one per warp; blockIdx.y picks the group) and loops over the same 16x4x4-voxel
// work items as the convolution: it stages the item's input halo and output gradient in shared
// memory, and each warp accumulates its tap's Cin x Cout block over the item's 256 voxels with
// ldmatrix.trans fragments (the voxel index is the contraction index) and mma.sync m16n8k16 BF16 ->
// FP32.  Every CTA writes its partial sums; a fixed-order reduction over the CTAs gives dw and db
// (deterministic: the partition does not depend on the GPU).
constexpr int kWgParts = 256;  // CTAs along the voxel items (the partition of the partial sums)

__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const bf16 *p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(s));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t (&r)[2], const bf16 *p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(s));
}

template <int CKP, int CNP>
struct WgCfg {
  static constexpr int SKX = CKP + 8, SKD = CNP + 8;
  static constexpr int NV = TXc * TYc * TZc;  // voxels per item
  static constexpr int SMEM = (NHc * SKX + NV * SKD) * 2;
};

template <int CKP, int CNP>
__global__ void __launch_bounds__(kConvThreads) conv_wgrad_mma(const bf16 *__restrict__ x, const bf16 *__restrict__ dy,
                                                               int nx, int ny, int nz, int ci, int co, int tiles_x,
                                                               int tiles_y, int tiles, float *__restrict__ part) {
  using Cfg = WgCfg<CKP, CNP>;
  constexpr int SKX = Cfg::SKX, SKD = Cfg::SKD, NV = Cfg::NV;
  extern __shared__ __align__(16) unsigned char wg_smem_raw[];
  bf16 *x_s = reinterpret_cast<bf16 *>(wg_smem_raw);
  bf16 *d_s = x_s + NHc * SKX;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const int tap = 8 * blockIdx.y + warp;
  const bool active = tap < 27;
  const int dx = tap % 3, dyo = (tap / 3) % 3, dz = tap / 9;
  const bf16 zero = __float2bfloat16(0.0f);
  const bool vx = ci == CKP && ((uintptr_t)x & 15) == 0, vd = co == CNP && ((uintptr_t)dy & 15) == 0;
  (void)t;
  // padded channels stay zero from this initial clear; only the real ones are rewritten per item
  for (int idx = tid; idx < NHc * SKX + NV * SKD; idx += kConvThreads) x_s[idx] = zero;
  float acc[CKP / 16][CNP / 8][4];
#pragma unroll
  for (int mi = 0; mi < CKP / 16; ++mi)
#pragma unroll
    for (int nj = 0; nj < CNP / 8; ++nj)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[mi][nj][j] = 0.0f;

  for (int item = blockIdx.x; item < tiles; item += gridDim.x) {
    const int bx = item % tiles_x, by = (item / tiles_x) % tiles_y, bz = item / (tiles_x * tiles_y);
    const int x0 = bx * TXc, y0 = by * TYc, z0 = bz * TZc;
    __syncthreads();  // the previous item's reads are done
    if (vx) {
      constexpr int CH = CKP / 8;
      for (int idx = tid; idx < NHc * CH; idx += kConvThreads) {
        const int hv = idx / CH, ch = idx % CH;
        const int gx = x0 - 1 + hv % HXc, gy = y0 - 1 + (hv / HXc) % HYc, gz = z0 - 1 + hv / (HXc * HYc);
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz)
          v = __ldg(reinterpret_cast<const uint4 *>(x + (((int64_t)gz * ny + gy) * nx + gx) * CKP) + ch);
        *reinterpret_cast<uint4 *>(x_s + hv * SKX + ch * 8) = v;
      }
    } else {
      for (int idx = tid; idx < NHc * ci; idx += kConvThreads) {
        const int hv = idx / ci, c = idx % ci;
        const int gx = x0 - 1 + hv % HXc, gy = y0 - 1 + (hv / HXc) % HYc, gz = z0 - 1 + hv / (HXc * HYc);
        bf16 v = zero;
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz)
          v = x[(((int64_t)gz * ny + gy) * nx + gx) * ci + c];
        x_s[hv * SKX + c] = v;
      }
    }
    // output gradient of the item's voxels; row r = x offset + 16 (y offset + 4 z offset)
    if (vd) {
      constexpr int CH = CNP / 8;
      for (int idx = tid; idx < NV * CH; idx += kConvThreads) {
        const int r = idx / CH, ch = idx % CH;
        const int gx = x0 + (r & 15), gy = y0 + ((r >> 4) & 3), gz = z0 + (r >> 6);
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (gx < nx && gy < ny && gz < nz)
          v = __ldg(reinterpret_cast<const uint4 *>(dy + (((int64_t)gz * ny + gy) * nx + gx) * CNP) + ch);
        *reinterpret_cast<uint4 *>(d_s + r * SKD + ch * 8) = v;
      }
    } else {
      for (int idx = tid; idx < NV * co; idx += kConvThreads) {
        const int r = idx / co, c = idx % co;
        const int gx = x0 + (r & 15), gy = y0 + ((r >> 4) & 3), gz = z0 + (r >> 6);
        bf16 v = zero;
        if (gx < nx && gy < ny && gz < nz) v = dy[(((int64_t)gz * ny + gy) * nx + gx) * co + c];
        d_s[r * SKD + c] = v;
      }
    }
    __syncthreads();
    if (active) {
#pragma unroll 1
      for (int kc = 0; kc < NV / 16; ++kc) {  // 16 voxels: one x-row of the item
        const int ty = kc & 3, tz = kc >> 2;
        const int v = (lane & 7) + 8 * (lane >> 4);  // voxel of the row addressed by this lane
        const bf16 *arow = x_s + ((tz + dz) * (HXc * HYc) + (ty + dyo) * HXc + v + dx) * SKX + 8 * ((lane >> 3) & 1);
        const bf16 *brow = d_s + (kc * 16 + (lane & 15)) * SKD;
        uint32_t bfr[CNP / 8][2];
#pragma unroll
        for (int nj = 0; nj < CNP / 8; ++nj) ldsm_x2_t(bfr[nj], brow + 8 * nj);
#pragma unroll
        for (int mi = 0; mi < CKP / 16; ++mi) {
          uint32_t af[4];
          ldsm_x4_t(af, arow + 16 * mi);
#pragma unroll
          for (int nj = 0; nj < CNP / 8; ++nj)
            mma_bf16(acc[mi][nj], af[0], af[1], af[2], af[3], bfr[nj][0], bfr[nj][1]);
        }
      }
    }
  }
  // partial sums of this CTA: part[p][27 ci co] with p = blockIdx.x
  float *pp = part + (int64_t)blockIdx.x * (27 * (int64_t)ci * co);
  if (active) {
#pragma unroll
    for (int mi = 0; mi < CKP / 16; ++mi)
#pragma unroll
      for (int nj = 0; nj < CNP / 8; ++nj)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int a = 16 * mi + g + 8 * (j >> 1), b = 8 * nj + 2 * t + (j & 1);
          if (a < ci && b < co) pp[((int64_t)tap * ci + a) * co + b] = acc[mi][nj][j];
        }
  }
}

// Bias gradient partials: block b sums voxels [nvox b / parts, nvox (b + 1) / parts) of every
// channel (thread = channel + co * lane, coalesced), lanes combined in fixed order.
__global__ void __launch_bounds__(256) bias_grad_part(const bf16 *__restrict__ dy, int64_t nvox, int co, int parts,
                                                      float *__restrict__ part) {
  __shared__ float sh[256];
  const int lanes = 256 / co, c = threadIdx.x % co, l = threadIdx.x / co;
  const int64_t v0 = nvox * blockIdx.x / parts, v1 = nvox * (blockIdx.x + 1) / parts;
  float s = 0.0f;
  if (l < lanes)
    for (int64_t v = v0 + l; v < v1; v += lanes) s += __bfloat162float(dy[v * co + c]);
  sh[threadIdx.x] = s;
  __syncthreads();
  if ((int)threadIdx.x < co) {
    float tot = 0.0f;
    for (int q = 0; q < lanes; ++q) tot += sh[q * co + threadIdx.x];
    part[(int64_t)blockIdx.x * co + threadIdx.x] = tot;
  }
}

// out[i] = sum_p part[p][i], p in order (deterministic); i < n
__global__ void conv_wgrad_reduce(const float *__restrict__ part, int nparts, int64_t n, float *__restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.0f;
  for (int p = 0; p < nparts; ++p) s += part[(int64_t)p * n + i];
  out[i] = s;
}

// ------------------------------------------------------------------- grid transfer ops ----
// Grid transfers on channels-last BF16 tensors: one thread per output voxel and group of 8
// channels (16-byte loads and stores when the channel count is a multiple of 8, else per channel),
// FP32 sums.
template <int V>
__device__ __forceinline__ void ld_ch(const bf16 *p, float (&f)[V]) {
  if constexpr (V == 8) {
    const uint4 u = __ldg(reinterpret_cast<const uint4 *>(p));
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 t = __bfloat1622float2(h[i]);
      f[2 * i] = t.x;
      f[2 * i + 1] = t.y;
    }
  } else {
    f[0] = __bfloat162float(*p);
  }
}
template <int V>
__device__ __forceinline__ void st_ch(bf16 *p, const float (&f)[V]) {
  if constexpr (V == 8) {
    uint4 u;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
    *reinterpret_cast<uint4 *>(p) = u;
  } else {
    *p = __float2bfloat16(f[0]);
  }
}

// Full weighting (m+1)^3 <- (2m+1)^3, scaled by `scale`; weights 1/4, 1/2, 1/4 per axis.
template <int V>
__global__ void restrict_k(const bf16 *__restrict__ in, int nfx, int nfy, int nfz, int c, bf16 *__restrict__ out,
                           float scale) {
  // grid: x over the (coarse y, coarse x, channel group) items of one plane, y over the planes
  // (32-bit index arithmetic)
  const int ncx = (nfx + 1) / 2, ncy = (nfy + 1) / 2;
  const int cg = c / V, row = ncx * cg;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ncy * row) return;
  const int cy = i / row, r = i - cy * row;
  const int cx = r / cg, ch = (r - cx * cg) * V;
  const int cz = blockIdx.y;
  const int64_t v = ((int64_t)cz * ncy + cy) * ncx + cx;
  float s[V], t[V];
#pragma unroll
  for (int q = 0; q < V; ++q) s[q] = 0.0f;
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
        const float w = (dx == 0 ? 0.5f : 0.25f) * wy * wz;
        ld_ch<V>(in + (((int64_t)fz * nfy + fy) * nfx + fx) * c + ch, t);
#pragma unroll
        for (int q = 0; q < V; ++q) s[q] += w * t[q];
      }
    }
  }
#pragma unroll
  for (int q = 0; q < V; ++q) s[q] *= scale;
  st_ch<V>(out + v * c + ch, s);
}

// Trilinear prolongation (2m+1)^3 <- (m+1)^3, scaled by `scale`.
template <int V>
__global__ void prolong_k(const bf16 *__restrict__ in, int ncx, int ncy, int ncz, int c, bf16 *__restrict__ out,
                          float scale) {
  // grid: x over the (fine y, fine x, channel group) items of one plane, y over the planes
  const int nfx = 2 * ncx - 1, nfy = 2 * ncy - 1;
  const int cg = c / V, row = nfx * cg;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nfy * row) return;
  const int fy = i / row, r = i - fy * row;
  const int fx = r / cg, ch = (r - fx * cg) * V;
  const int fz = blockIdx.y;
  const int64_t v = ((int64_t)fz * nfy + fy) * nfx + fx;
  const int xs[2] = {fx / 2, (fx + 1) / 2}, ys[2] = {fy / 2, (fy + 1) / 2}, zs[2] = {fz / 2, (fz + 1) / 2};
  const int nxp = (fx & 1) ? 2 : 1, nyp = (fy & 1) ? 2 : 1, nzp = (fz & 1) ? 2 : 1;
  const float w = scale / (float)(nxp * nyp * nzp);
  float s[V], t[V];
#pragma unroll
  for (int q = 0; q < V; ++q) s[q] = 0.0f;
  for (int a = 0; a < nzp; ++a)
    for (int b = 0; b < nyp; ++b)
      for (int d = 0; d < nxp; ++d) {
        ld_ch<V>(in + (((int64_t)zs[a] * ncy + ys[b]) * ncx + xs[d]) * c + ch, t);
#pragma unroll
        for (int q = 0; q < V; ++q) s[q] += t[q];
      }
#pragma unroll
  for (int q = 0; q < V; ++q) s[q] *= w;
  st_ch<V>(out + v * c + ch, s);
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
  MF_RANGE("mf_conv3d_fwd");
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

// Forward convolution of an input stored with `cin_stride` >= cin channels per voxel (the channels
// beyond cin are ignored), on the tensor-core path; MF_ERR_UNSUPPORTED when that path cannot take it.
mf_status conv3d_fwd_strided(const void *x, int nx, int ny, int nz, int cin, int cin_stride, const void *w,
                             const float *bias, int cout, const void *skip, int relu, void *y_bf16, float *y_f32,
                             cudaStream_t stream) {
  ConvArgs a{};
  a.in = (const bf16 *)x;
  a.nx = nx; a.ny = ny; a.nz = nz; a.ck = cin; a.cphys = cin_stride;
  a.w = (const bf16 *)w;
  a.bias = bias;
  a.skip = (const bf16 *)skip;
  a.relu = relu;
  a.cn = cout;
  a.out_bf = (bf16 *)y_bf16;
  a.out_f = y_f32;
  mf_status st = MF_OK;
  if (!conv_tc_enabled() || !launch_conv_tc<0>(a, stream, &st)) return MF_ERR_UNSUPPORTED;
  return st;
}

extern "C" mf_status mf_conv3d_dgrad(const void *dy, int32_t nx, int32_t ny, int32_t nz, int32_t cin, const void *w,
                                     int32_t cout, void *dx_bf16, float *dx_f32, mf_stream stream) {
  MF_RANGE("mf_conv3d_dgrad");
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

static int wgrad_tiles(int nx, int ny, int nz) {
  return ((nx + TXc - 1) / TXc) * ((ny + TYc - 1) / TYc) * ((nz + TZc - 1) / TZc);
}

// Number of partial sums (CTAs along the voxel items): at most one per item and kWgParts, and few
// enough that the partials (parts x 27 cin cout floats) stay near 2^22 values for the reduction.
static int wgrad_parts(int nx, int ny, int nz, int cin, int cout) {
  const int by_size = std::max(32, (int)((1 << 22) / (27 * (int64_t)cin * cout)));
  return std::min(std::min(wgrad_tiles(nx, ny, nz), kWgParts), by_size);
}

extern "C" int64_t mf_conv3d_wgrad_workspace(int32_t nx, int32_t ny, int32_t nz, int32_t cin, int32_t cout) {
  const int64_t parts = wgrad_parts(nx, ny, nz, cin, cout);
  return (parts * 27 * (int64_t)cin * cout + (int64_t)kWgParts * cout) * (int64_t)sizeof(float);
}

template <int CKP, int CNP>
static mf_status launch_wgrad_t(const bf16 *x, const bf16 *dy, int nx, int ny, int nz, int ci, int co, int parts,
                                float *ws, cudaStream_t s) {
  constexpr int smem = WgCfg<CKP, CNP>::SMEM;
  static std::atomic<int> attr{0};
  if (attr.load() == 0) {
    MF_CUDA(cudaFuncSetAttribute(conv_wgrad_mma<CKP, CNP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    attr.store(1);
  }
  const int tx = (nx + TXc - 1) / TXc, ty = (ny + TYc - 1) / TYc;
  conv_wgrad_mma<CKP, CNP><<<dim3(parts, 4), kConvThreads, smem, s>>>(x, dy, nx, ny, nz, ci, co, tx, ty,
                                                                      wgrad_tiles(nx, ny, nz), ws);
  return MF_OK;
}

extern "C" mf_status mf_conv3d_wgrad(const void *x, const void *dy, int32_t nx, int32_t ny, int32_t nz, int32_t cin,
                                     int32_t cout, float *dw, float *db, float *workspace, int64_t ws_bytes,
                                     mf_stream stream) {
  MF_RANGE("mf_conv3d_wgrad");
  mf_clear_error();
  MF_ARG(x && dy && dw && workspace && cin > 0 && cout > 0 && cin <= 64 && cout <= 64 && nx > 0 && ny > 0 && nz > 0,
         "mf_conv3d_wgrad: bad argument");
  MF_ARG(ws_bytes >= mf_conv3d_wgrad_workspace(nx, ny, nz, cin, cout), "mf_conv3d_wgrad: workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const int parts = wgrad_parts(nx, ny, nz, cin, cout);
  const int ckp = cin <= 16 ? 16 : cin <= 32 ? 32 : 64;
  const int cnp = cout <= 8 ? 8 : cout <= 16 ? 16 : cout <= 32 ? 32 : 64;
  const bf16 *xb = (const bf16 *)x, *db16 = (const bf16 *)dy;
  mf_count_launches(db ? 4 : 2);
#define WG(K, N) \
  if (ckp == K && cnp == N) MF_TRY((launch_wgrad_t<K, N>(xb, db16, nx, ny, nz, cin, cout, parts, workspace, s)));
  WG(16, 8) WG(16, 16) WG(16, 32) WG(16, 64)
  WG(32, 8) WG(32, 16) WG(32, 32) WG(32, 64)
  WG(64, 8) WG(64, 16) WG(64, 32) WG(64, 64)
#undef WG
  const int64_t nw = 27 * (int64_t)cin * cout;
  conv_wgrad_reduce<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(workspace, parts, nw, dw);
  if (db) {
    float *bp = workspace + parts * nw;
    bias_grad_part<<<kWgParts, 256, 0, s>>>((const bf16 *)dy, (int64_t)nx * ny * nz, cout, kWgParts, bp);
    conv_wgrad_reduce<<<1, 256, 0, s>>>(bp, kWgParts, cout, db);
  }
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

// 16-byte channel groups: channel count a multiple of 8 and both tensors 16-byte aligned
static bool vec8(const void *in, const void *out, int c) {
  return c % 8 == 0 && ((uintptr_t)in & 15) == 0 && ((uintptr_t)out & 15) == 0;
}

extern "C" mf_status mf_grid_restrict(const void *in, int32_t nfx, int32_t nfy, int32_t nfz, int32_t c, void *out,
                                      float scale, mf_stream stream) {
  MF_RANGE("mf_grid_restrict");
  mf_clear_error();
  MF_ARG(in && out && nfx % 2 == 1 && nfy % 2 == 1 && nfz % 2 == 1 && c > 0, "mf_grid_restrict: bad argument");
  const int ncx = (nfx + 1) / 2, ncy = (nfy + 1) / 2, ncz = (nfz + 1) / 2;
  MF_ARG(ncz <= 65535 && (int64_t)ncx * ncy * c < INT32_MAX, "mf_grid_restrict: grid too large");
  mf_count_launches(1);
  constexpr int T = 256;
  if (vec8(in, out, c))
    restrict_k<8><<<dim3((ncx * ncy * (c / 8) + T - 1) / T, ncz), T, 0, (cudaStream_t)stream>>>(
        (const bf16 *)in, nfx, nfy, nfz, c, (bf16 *)out, scale);
  else
    restrict_k<1><<<dim3((ncx * ncy * c + T - 1) / T, ncz), T, 0, (cudaStream_t)stream>>>(
        (const bf16 *)in, nfx, nfy, nfz, c, (bf16 *)out, scale);
  MF_CUDA(cudaGetLastError());
  return MF_OK;
}

extern "C" mf_status mf_grid_prolong(const void *in, int32_t ncx, int32_t ncy, int32_t ncz, int32_t c, void *out,
                                     float scale, mf_stream stream) {
  MF_RANGE("mf_grid_prolong");
  mf_clear_error();
  MF_ARG(in && out && ncx > 0 && ncy > 0 && ncz > 0 && c > 0, "mf_grid_prolong: bad argument");
  const int nfx = 2 * ncx - 1, nfy = 2 * ncy - 1, nfz = 2 * ncz - 1;
  MF_ARG(nfz <= 65535 && (int64_t)nfx * nfy * c < INT32_MAX, "mf_grid_prolong: grid too large");
  mf_count_launches(1);
  constexpr int T = 256;
  if (vec8(in, out, c))
    prolong_k<8><<<dim3((nfx * nfy * (c / 8) + T - 1) / T, nfz), T, 0, (cudaStream_t)stream>>>(
        (const bf16 *)in, ncx, ncy, ncz, c, (bf16 *)out, scale);
  else
    prolong_k<1><<<dim3((nfx * nfy * c + T - 1) / T, nfz), T, 0, (cudaStream_t)stream>>>(
        (const bf16 *)in, ncx, ncy, ncz, c, (bf16 *)out, scale);
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
