// Learned warm start for the solve of Eq. 1: a network of eight 3x3
// convolution layers maps the observation b to an image estimate u_hat, and
// FISTA (Sec. I-B, which starts from zero) starts from x_0 = W^dagger u_hat.
//
//   a_0 = b (1 channel);  a_l = relu(conv3x3(a_{l-1}; w_l, c_l)), l = 1..7, 32 channels;
//   u_hat = b + conv3x3(a_7; w_8, c_8)
//
// conv3x3 is the 'same' cross-correlation with zero padding.  Storage: hidden
// activations and their gradients channels-last bfloat16 (64 bytes a pixel),
// single-channel images float32 with a row pitch, master parameters float32
// (each layer's weights in (Cout, Cin, 3, 3) order, then its biases).
//
// Kernels:
//  * k_conv32_tc: the 32 -> 32 layers (forward, and the data gradient with
//    the flipped, transposed weights and the ReLU mask of the layer below) as
//    implicit GEMMs on tcgen05: per output row of a 4 x 128 pixel tile,
//    D[128 pixels][32 channels] += A_tap B_tap over 9 taps x 2 halves of 16
//    input channels (kind::f16, bf16 operands, f32 accumulators in tensor
//    memory).  The input window is held in shared memory with each
//    8-channel group of a row stored pixel-contiguous (16 bytes a pixel), so
//    the A operand of a tap is a descriptor at a 16-byte pixel offset of the
//    window: the canonical K-major layout needs no im2col copy.
//  * k_conv32_wgrad: the weight gradient of the 32 -> 32 layers, a reduction
//    over pixels (K), with the warp-level MMA (m16n8k16 bf16, fragments from
//    the same window layout by ldmatrix.trans); one warp per tap.
//  * k_conv_in / k_conv_out / k_conv_out_bwd / k_thin_wgrad: the 1 -> 32 and
//    32 -> 1 layers on the CUDA cores (9 or 288 multiply-adds a pixel).
//  * k_loss_grad, k_reduce_wgrad, k_adam, k_pack: loss and its gradient,
//    deterministic partial sums, the Adam update, the bf16 operand packing.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <initializer_list>
#include <string>

#include "adjwt_cnn.h"
#include "adjwt_internal.h"
#include "device_common.cuh"
#include "tma.cuh"
#include "umma.cuh"

namespace adjwt {
namespace {

constexpr int kC = 32;                        // hidden channels
constexpr int kTW = 128;                      // output pixels of a tile row (the MMA's M)
constexpr int kTH = 4;                        // output rows of a tile
constexpr int kHaloW = kTW + 2;               // input pixels of a window row
constexpr int kGroups = 4;                    // 8-channel groups (16 bytes)
constexpr int kPlane = kHaloW * 16;           // one channel group of one window row: 2080 bytes
constexpr int kInRow = kGroups * kPlane;      // 8320
constexpr int kInBytes = (kTH + 2) * kInRow;  // 49920
constexpr int kKSteps = 18;                   // 9 taps x 2 halves of 16 channels
constexpr int kLayerPack = kKSteps * 1024;    // packed B operand of one layer and direction: 18432 bytes
constexpr int kFwdThreads = 128;
constexpr int kFwdSmem = kInBytes + kLayerPack + 128;
constexpr uint32_t kFwdTmemCols = 128;        // kTH accumulators of 32 columns
constexpr int kDzPlane = kTW * 16;            // 2048
constexpr int kDzRow = kGroups * kDzPlane;    // 8192
constexpr int kDzBytes = kTH * kDzRow;        // 32768
constexpr int kWgThreads = 288;               // nine warps, one per tap
constexpr int kWgSmem = kInBytes + kDzBytes + 128;
constexpr int kWgStride = 9 * kC * kC + kC;   // floats of one CTA's partial
constexpr int kWgMaxGrid = 320;
constexpr int kThinStride = 9 * kC + kC + 1;  // 321
constexpr int kThinMaxGrid = 2432;
constexpr int kThinThreads = 256;             // 16 channel pairs x 16 row segments
constexpr int kLossBlocks = 1024;

// parameter offsets (floats)
constexpr int64_t kOffW0 = 0, kOffB0 = 288;
__host__ __device__ constexpr int64_t off_w(int l) { return 320 + (int64_t)(l - 1) * (9 * kC * kC + kC); }
__host__ __device__ constexpr int64_t off_b(int l) { return off_w(l) + 9 * kC * kC; }
constexpr int64_t kOffW7 = 320 + 6 * (9 * kC * kC + kC), kOffB7 = kOffW7 + 288, kParamCount = kOffB7 + 1;
static_assert(kParamCount == 56097, "parameter count");

// tcgen05 instruction descriptor: f32 accumulate, bf16 A and B, both K-major, M = 128, N = 32
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(kIdescBf16), "r"(accumulate));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void unpack8(const uint4& q, float* v) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = __bfloat1622float2(h[i]);
    v[2 * i] = f.x;
    v[2 * i + 1] = f.y;
  }
}

__device__ __forceinline__ void store_pixel(__nv_bfloat16* dst, const float (&v)[32]) {
  uint4* d = reinterpret_cast<uint4*>(dst);
#pragma unroll
  for (int q = 0; q < 4; ++q)
    d[q] = make_uint4(pack_bf16x2(v[8 * q], v[8 * q + 1]), pack_bf16x2(v[8 * q + 2], v[8 * q + 3]),
                      pack_bf16x2(v[8 * q + 4], v[8 * q + 5]), pack_bf16x2(v[8 * q + 6], v[8 * q + 7]));
}

__device__ __forceinline__ unsigned char* align128(unsigned char* p) {
  return p + ((128 - (smem_u32(p) & 127)) & 127);
}

// The (kTH + 2) x kHaloW x 32 input window of the tile at (n, y0, x0):
// byte (r, g, q) at r kInRow + g kPlane + 16 q holds channels 8g .. 8g + 7 of
// pixel (y0 - 1 + r, x0 - 1 + q); zero outside the image.  Consecutive
// threads copy consecutive 16-byte groups of one pixel (coalesced reads).
__device__ __forceinline__ void load_window(unsigned char* dst, const __nv_bfloat16* act, int H, int W, int n, int y0,
                                            int x0, int tid, int nthreads) {
  constexpr int total = (kTH + 2) * kHaloW * kGroups;
  for (int i = tid; i < total; i += nthreads) {
    const int g = i & 3, q = (i >> 2) % kHaloW, r = i / (4 * kHaloW);
    const int y = y0 - 1 + r, x = x0 - 1 + q;
    const bool in = y >= 0 && y < H && x >= 0 && x < W;
    const __nv_bfloat16* src = in ? act + ((((int64_t)n * H + y) * W + x) * kC + g * 8) : act;
    cp_async16(reinterpret_cast<float*>(dst + r * kInRow + g * kPlane + q * 16), reinterpret_cast<const float*>(src),
               in ? 16u : 0u);
  }
}

// --------------------------------------------------------------- tcgen05 conv
template <bool MASK>
__global__ void __launch_bounds__(kFwdThreads) k_conv32_tc(int H, int W, int tiles_x, int tiles_y,
                                                           const __nv_bfloat16* __restrict__ in,
                                                           const __nv_bfloat16* __restrict__ wpack,
                                                           const float* __restrict__ bias, int relu,
                                                           const __nv_bfloat16* __restrict__ mask,
                                                           __nv_bfloat16* __restrict__ out, int* status) {
  pdl_entry();
  extern __shared__ unsigned char dyn[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_holder;
  __shared__ float bias_s[kC];
  unsigned char* sm = align128(dyn);
  unsigned char* win = sm;
  unsigned char* wsm = sm + kInBytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tx = blockIdx.x % tiles_x, ty = (blockIdx.x / tiles_x) % tiles_y, n = blockIdx.x / (tiles_x * tiles_y);
  const int x0 = tx * kTW, y0 = ty * kTH;

  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                 "r"(kFwdTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid < kC) bias_s[tid] = bias ? bias[tid] : 0.0f;
  load_window(win, in, H, W, n, y0, x0, tid, kFwdThreads);
  for (int i = tid; i < kLayerPack / 16; i += kFwdThreads)
    cp_async16(reinterpret_cast<float*>(wsm + 16 * i), reinterpret_cast<const float*>(wpack + 8 * i), 16u);
  cp_async_commit();
  cp_async_wait_all();
  umma_operands_ready();
  const uint32_t tmem = tmem_holder;

  if (tid == 0) {
    // A: 128 pixels (8-row groups 128 bytes apart) x 16 channels (two groups kPlane apart);
    // B: 32 output channels (8-row groups 128 bytes apart) x 16 channels (two groups 512 apart).
    // Every operand address stays below 2^18 bytes, so the descriptor at byte offset o is the
    // base descriptor plus o / 16 (the 14-bit start field never carries): the 72 MMAs issue
    // with one add each.
    const uint64_t a0 = umma_desc(smem_u32(win), kPlane, 128), b0 = umma_desc(smem_u32(wsm), 512, 128);
#pragma unroll
    for (int r = 0; r < kTH; ++r) {
#pragma unroll
      for (int s = 0; s < kKSteps; ++s) {
        const int t = s >> 1, h = s & 1, dy = t / 3, dx = t - 3 * dy;
        umma_bf16(tmem + r * 32, a0 + (uint64_t)(((r + dy) * kInRow + 2 * h * kPlane + dx * 16) >> 4),
                  b0 + (uint64_t)(s * 64), s > 0);
      }
    }
    umma_commit(&bar);
  }
  bool ok = tid == 0 ? mbar_wait(&bar, 0) : true;
  if (tid == 0 && !ok) record_status(status, ADJWT_ERR_TIMEOUT);
  ok = __syncthreads_and(ok);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const uint32_t tmem_warp = tmem + ((uint32_t)(32 * warp) << 16);
    const int x = x0 + 32 * warp + lane;
#pragma unroll 1
    for (int r = 0; r < kTH; ++r) {
      float v[32];
      tmem_ld32(tmem_warp + r * 32, v);  // pixel x of row y0 + r, channels 0 .. 31
      const int y = y0 + r;
      if (y < H && x < W) {
        const int64_t pix = ((int64_t)n * H + y) * W + x;
#pragma unroll
        for (int c = 0; c < kC; ++c) {
          v[c] += bias_s[c];
          if (relu) v[c] = fmaxf(v[c], 0.0f);
        }
        if (MASK) {
          const uint4* mq = reinterpret_cast<const uint4*>(mask + pix * kC);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float m[8];
            unpack8(__ldg(mq + q), m);
#pragma unroll
            for (int e = 0; e < 8; ++e)
              if (!(m[e] > 0.0f)) v[8 * q + e] = 0.0f;
          }
        }
        store_pixel(out + pix * kC, v);
      }
    }
  } else if (tid == 0) {
    (void)mbar_wait(&bar, 0);  // one more bounded wait before the accumulators are released
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kFwdTmemCols));
}

// ---------------------------------------------------------- weight gradient
// part[cta][t * 1024 + co * 32 + ci] = sum over the CTA's pixels p of
// dz[p][co] x[p + offset_t][ci]; part[cta][9216 + co] = sum dz[p][co].
__global__ void __launch_bounds__(kWgThreads, 2) k_conv32_wgrad(int N, int H, int W, int tiles_x, int tiles_y,
                                                                const __nv_bfloat16* __restrict__ x,
                                                                const __nv_bfloat16* __restrict__ dz,
                                                                float* __restrict__ part) {
  pdl_entry();
  extern __shared__ unsigned char dyn[];
  __shared__ float dbred[128][8];
  unsigned char* sm = align128(dyn);
  unsigned char* win = sm;
  unsigned char* dzs = sm + kInBytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int dy = warp / 3, dx = warp - 3 * dy;  // this warp's tap
  const int li = lane >> 3, lj = lane & 7;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.0f;
  float dbacc[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  const int64_t tiles = (int64_t)N * tiles_y * tiles_x;
  const uint32_t wb = smem_u32(win), zb = smem_u32(dzs);
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int tx = static_cast<int>(tile % tiles_x), ty = static_cast<int>((tile / tiles_x) % tiles_y);
    const int n = static_cast<int>(tile / ((int64_t)tiles_x * tiles_y));
    const int x0 = tx * kTW, y0 = ty * kTH;
    load_window(win, x, H, W, n, y0, x0, tid, kWgThreads);
    for (int i = tid; i < kTH * kTW * kGroups; i += kWgThreads) {
      const int g = i & 3, q = (i >> 2) % kTW, r = i / (4 * kTW);
      const int y = y0 + r, xx = x0 + q;
      const bool in = y < H && xx < W;
      const __nv_bfloat16* src = in ? dz + ((((int64_t)n * H + y) * W + xx) * kC + g * 8) : dz;
      cp_async16(reinterpret_cast<float*>(dzs + r * kDzRow + g * kDzPlane + q * 16),
                 reinterpret_cast<const float*>(src), in ? 16u : 0u);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
#pragma unroll 1
    for (int r = 0; r < kTH; ++r) {
#pragma unroll 2
      for (int kb = 0; kb < kTW / 16; ++kb) {
        const int p0 = 16 * kb;
        uint32_t a[2][4], b[4][2];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)  // A[m = co][k = pixel] from the dz rows (stored pixel-major)
          ldsm_x4_t(zb + r * kDzRow + (2 * mt + (li & 1)) * kDzPlane + (p0 + 8 * (li >> 1) + lj) * 16, a[mt][0],
                    a[mt][1], a[mt][2], a[mt][3]);
#pragma unroll
        for (int np = 0; np < 2; ++np)  // B[k = pixel][n = ci] from the shifted window row
          ldsm_x4_t(wb + (r + dy) * kInRow + (2 * np + (li >> 1)) * kPlane + (p0 + dx + 8 * (li & 1) + lj) * 16,
                    b[2 * np][0], b[2 * np][1], b[2 * np + 1][0], b[2 * np + 1][1]);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) mma_bf16_16816(acc[mt][nt], a[mt], b[nt][0], b[nt][1]);
      }
    }
    if (tid < 128) {  // bias gradient: thread (row, channel group, pixel slice) adds 16-byte groups
      const int r = tid >> 5, g = (tid >> 3) & 3, qq = tid & 7;
      const uint4* grp = reinterpret_cast<const uint4*>(dzs + r * kDzRow + g * kDzPlane);
#pragma unroll 4
      for (int q = qq; q < kTW; q += 8) {
        float v[8];
        unpack8(grp[q], v);
#pragma unroll
        for (int e = 0; e < 8; ++e) dbacc[e] += v[e];
      }
    }
    __syncthreads();
  }
  float* base = part + (int64_t)blockIdx.x * kWgStride;
  const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int co = 16 * mt + g, ci = 8 * nt + 2 * t4;
      float* o = base + warp * kC * kC;
      o[co * kC + ci] = acc[mt][nt][0];
      o[co * kC + ci + 1] = acc[mt][nt][1];
      o[(co + 8) * kC + ci] = acc[mt][nt][2];
      o[(co + 8) * kC + ci + 1] = acc[mt][nt][3];
    }
  if (tid < 128)
#pragma unroll
    for (int e = 0; e < 8; ++e) dbred[tid][e] = dbacc[e];
  __syncthreads();
  if (tid < kC) {  // channel c = 8 g + e: rows r and slices qq of thread r 32 + g 8 + qq
    const int g = tid >> 3, e = tid & 7;
    float t = 0.0f;
    for (int r = 0; r < kTH; ++r)
      for (int qq = 0; qq < 8; ++qq) t += dbred[r * 32 + g * 8 + qq][e];
    base[9 * kC * kC + tid] = t;
  }
}

// Thin-layer weight gradient: part[cta][t * 32 + c] = sum over image pixels p
// of A[p][c] s[p + sigma offset_t] (sigma = +1, or -1 when flip: the tap is
// then stored as 8 - t), part[cta][288 + c] = sum A[p][c], part[cta][320] =
// sum s[p].  A: (N, H, W, 32) bf16; s: float32 image, row pitch sp, zero
// outside.  Thread (channel pair cp, slot) walks 32-pixel row segments with a
// sliding 3 x 3 window of s.
__global__ void __launch_bounds__(kThinThreads) k_thin_wgrad(int N, int H, int W, const __nv_bfloat16* __restrict__ A,
                                                             const float* __restrict__ s, int64_t sp, int flip,
                                                             float* __restrict__ part) {
  pdl_entry();
  __shared__ float red[16][16][21];
  const int cp = threadIdx.x & 15, slot = threadIdx.x >> 4;
  const int segs = (W + 31) / 32;
  const int64_t units = (int64_t)N * H * segs;
  float acc[18], sa0 = 0.0f, sa1 = 0.0f, ss = 0.0f;
#pragma unroll
  for (int i = 0; i < 18; ++i) acc[i] = 0.0f;
  for (int64_t u = (int64_t)blockIdx.x * 16 + slot; u < units; u += (int64_t)gridDim.x * 16) {
    const int seg = static_cast<int>(u % segs);
    const int64_t ny = u / segs;
    const int y = static_cast<int>(ny % H), n = static_cast<int>(ny / H);
    const int xs = seg * 32, xe = min(W, xs + 32);
    const float* srow[3];
    bool rin[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int yy = y + d - 1;
      rin[d] = yy >= 0 && yy < H;
      srow[d] = s + ((int64_t)n * H + (rin[d] ? yy : 0)) * sp;
    }
    float w[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      w[d][0] = (rin[d] && xs >= 1) ? __ldg(srow[d] + xs - 1) : 0.0f;
      w[d][1] = rin[d] ? __ldg(srow[d] + xs) : 0.0f;
    }
    const __nv_bfloat162* arow = reinterpret_cast<const __nv_bfloat162*>(A + ((int64_t)n * H + y) * W * kC) + cp;
    for (int x = xs; x < xe; ++x) {
#pragma unroll
      for (int d = 0; d < 3; ++d) w[d][2] = (rin[d] && x + 1 < W) ? __ldg(srow[d] + x + 1) : 0.0f;
      const float2 a = __bfloat1622float2(arow[(int64_t)x * (kC / 2)]);
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        acc[2 * t] = fmaf(a.x, w[t / 3][t % 3], acc[2 * t]);
        acc[2 * t + 1] = fmaf(a.y, w[t / 3][t % 3], acc[2 * t + 1]);
      }
      sa0 += a.x;
      sa1 += a.y;
      if (cp == 0) ss += w[1][1];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        w[d][0] = w[d][1];
        w[d][1] = w[d][2];
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 18; ++i) red[slot][cp][i] = acc[i];
  red[slot][cp][18] = sa0;
  red[slot][cp][19] = sa1;
  red[slot][cp][20] = ss;
  __syncthreads();
  float* base = part + (int64_t)blockIdx.x * kThinStride;
  for (int o = threadIdx.x; o < kThinStride; o += kThinThreads) {
    int pcp, j, tout = 0;
    if (o < 288) {
      const int t = o / 32, c = o % 32;
      pcp = c >> 1;
      j = 2 * t + (c & 1);
      tout = flip ? 8 - t : t;
    } else if (o < 320) {
      pcp = (o - 288) >> 1;
      j = 18 + ((o - 288) & 1);
    } else {
      pcp = 0;
      j = 20;
    }
    float v = 0.0f;
    for (int sl = 0; sl < 16; ++sl) v += red[sl][pcp][j];
    base[o < 288 ? tout * 32 + (o % 32) : o] = v;
  }
}

// out_w[c * 9 + t] = sum_g part[g][t * C + c]; out_b[j] = sum_g part[g][boff + j]
// (float64 sums in a fixed order).  A block takes 32 consecutive outputs;
// its eight warps sum the parts g = warp (mod 8), then warp 0 adds the eight.
__global__ void __launch_bounds__(256) k_reduce_wgrad(int nparts, int stride, const float* __restrict__ part, int C,
                                                      float* __restrict__ out_w, int boff, int nb,
                                                      float* __restrict__ out_b) {
  pdl_entry();
  __shared__ double red[8][32];
  const int j = threadIdx.x & 31, sl = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + j;
  const int nw = 9 * C;
  const bool valid = i < nw + nb;
  double acc = 0.0;
  if (valid) {
    const int src = i < nw ? i : boff + (i - nw);
    for (int g = sl; g < nparts; g += 8) acc += part[(int64_t)g * stride + src];
  }
  red[sl][j] = acc;
  __syncthreads();
  if (sl == 0 && valid) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += red[q][j];
    if (i < nw)
      out_w[(i % C) * 9 + i / C] = static_cast<float>(t);
    else
      out_b[i - nw] = static_cast<float>(t);
  }
}

// ------------------------------------------------------------- thin layers
// The thin layers keep their 32 x 9 weights in shared memory transposed to
// [tap][channel] and read them as float4 (broadcast: every thread of a warp
// reads the same address), four channels per load.
__global__ void __launch_bounds__(256) k_conv_in(int N, int H, int W, const float* __restrict__ img, int64_t pitch,
                                                 const float* __restrict__ p, __nv_bfloat16* __restrict__ out) {
  pdl_entry();
  __shared__ __align__(16) float wt[9 * kC + kC];  // wt[t][c] = w_1[c][t], then c_1
  for (int i = threadIdx.x; i < 9 * kC; i += blockDim.x) wt[(i % 9) * kC + i / 9] = p[i];
  if (threadIdx.x < kC) wt[9 * kC + threadIdx.x] = p[288 + threadIdx.x];
  __syncthreads();
  const float4* w4 = reinterpret_cast<const float4*>(wt);
  const int64_t total = (int64_t)N * H * W;
  for (int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pix < total; pix += (int64_t)gridDim.x * blockDim.x) {
    const int x = static_cast<int>(pix % W), y = static_cast<int>((pix / W) % H), n = static_cast<int>(pix / ((int64_t)W * H));
    float v[32];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 c4 = w4[9 * 8 + q];
      v[4 * q] = c4.x;
      v[4 * q + 1] = c4.y;
      v[4 * q + 2] = c4.z;
      v[4 * q + 3] = c4.w;
    }
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
      const float st = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? __ldg(img + ((int64_t)n * H + yy) * pitch + xx) : 0.0f;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 wv = w4[t * 8 + q];
        v[4 * q] = fmaf(wv.x, st, v[4 * q]);
        v[4 * q + 1] = fmaf(wv.y, st, v[4 * q + 1]);
        v[4 * q + 2] = fmaf(wv.z, st, v[4 * q + 2]);
        v[4 * q + 3] = fmaf(wv.w, st, v[4 * q + 3]);
      }
    }
#pragma unroll
    for (int c = 0; c < kC; ++c) v[c] = fmaxf(v[c], 0.0f);
    store_pixel(out + pix * kC, v);
  }
}

__global__ void __launch_bounds__(256) k_conv_out(int N, int H, int W, const __nv_bfloat16* __restrict__ a,
                                                  const float* __restrict__ p, const float* __restrict__ src,
                                                  int64_t pitch, float* __restrict__ out) {
  pdl_entry();
  __shared__ __align__(16) float wt[9 * kC];  // wt[t][ci] = w_8[ci][t]
  for (int i = threadIdx.x; i < 9 * kC; i += blockDim.x) wt[(i % 9) * kC + i / 9] = p[i];
  __syncthreads();
  const float bias = p[288];
  const float4* w4 = reinterpret_cast<const float4*>(wt);
  const int64_t total = (int64_t)N * H * W;
  for (int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pix < total; pix += (int64_t)gridDim.x * blockDim.x) {
    const int x = static_cast<int>(pix % W), y = static_cast<int>((pix / W) % H), n = static_cast<int>(pix / ((int64_t)W * H));
    float acc = bias;
#pragma unroll 3
    for (int t = 0; t < 9; ++t) {
      const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
      if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
      const uint4* q = reinterpret_cast<const uint4*>(a + (((int64_t)n * H + yy) * W + xx) * kC);
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        float v[8];
        unpack8(__ldg(q + g), v);
        const float4 wa = w4[t * 8 + 2 * g], wb = w4[t * 8 + 2 * g + 1];
        acc = fmaf(wa.x, v[0], acc);
        acc = fmaf(wa.y, v[1], acc);
        acc = fmaf(wa.z, v[2], acc);
        acc = fmaf(wa.w, v[3], acc);
        acc = fmaf(wb.x, v[4], acc);
        acc = fmaf(wb.y, v[5], acc);
        acc = fmaf(wb.z, v[6], acc);
        acc = fmaf(wb.w, v[7], acc);
      }
    }
    const int64_t o = ((int64_t)n * H + y) * pitch + x;
    out[o] = src[o] + acc;
  }
}

// dz[p][ci] = [a[p][ci] > 0] sum_t w_8[ci][t] dout[p - offset_t]
__global__ void __launch_bounds__(256) k_conv_out_bwd(int N, int H, int W, const float* __restrict__ dout,
                                                      const float* __restrict__ p, const __nv_bfloat16* __restrict__ a,
                                                      __nv_bfloat16* __restrict__ dz) {
  pdl_entry();
  __shared__ __align__(16) float wt[9 * kC];  // wt[t][ci] = w_8[ci][8 - t]: pairs with dout[p + offset_t]
  for (int i = threadIdx.x; i < 9 * kC; i += blockDim.x) wt[(8 - i % 9) * kC + i / 9] = p[i];
  __syncthreads();
  const float4* w4 = reinterpret_cast<const float4*>(wt);
  const int64_t total = (int64_t)N * H * W;
  for (int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pix < total; pix += (int64_t)gridDim.x * blockDim.x) {
    const int x = static_cast<int>(pix % W), y = static_cast<int>((pix / W) % H), n = static_cast<int>(pix / ((int64_t)W * H));
    float v[32];
#pragma unroll
    for (int c = 0; c < kC; ++c) v[c] = 0.0f;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
      const float st = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? __ldg(dout + ((int64_t)n * H + yy) * W + xx) : 0.0f;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 wv = w4[t * 8 + q];
        v[4 * q] = fmaf(wv.x, st, v[4 * q]);
        v[4 * q + 1] = fmaf(wv.y, st, v[4 * q + 1]);
        v[4 * q + 2] = fmaf(wv.z, st, v[4 * q + 2]);
        v[4 * q + 3] = fmaf(wv.w, st, v[4 * q + 3]);
      }
    }
    const uint4* mq = reinterpret_cast<const uint4*>(a + pix * kC);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      float m[8];
      unpack8(__ldg(mq + g), m);
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (!(m[e] > 0.0f)) v[8 * g + e] = 0.0f;
    }
    store_pixel(dz + pix * kC, v);
  }
}

// dout = (u_hat - u_ref) * inv (dense rows of W); part[block] = sum (u_hat - u_ref)^2
__global__ void __launch_bounds__(256) k_loss_grad(int N, int H, int W, const float* __restrict__ u,
                                                   const float* __restrict__ ref, int64_t pitch, float inv,
                                                   float* __restrict__ dout, double* __restrict__ part) {
  pdl_entry();
  __shared__ double scratch[8];
  const int64_t total = (int64_t)N * H * W;
  double acc = 0.0;
  for (int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pix < total; pix += (int64_t)gridDim.x * blockDim.x) {
    const int x = static_cast<int>(pix % W);
    const int64_t row = pix / W;
    const float d = u[row * pitch + x] - ref[row * pitch + x];
    dout[pix] = d * inv;
    acc += (double)d * d;
  }
  const double t = block_sum<256>(acc, scratch);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_adam(int64_t count, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float bc1, float bc2) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

// Packed bf16 B operands of the 32 -> 32 layers: for layer l (1..6) and
// direction d (0 forward, 1 data gradient), K-step s = 2 tap + half holds
// element (n, k) at byte s 1024 + (k / 8) 512 + (n / 8) 128 + (n % 8) 16 + (k % 8) 2:
// forward B[n = co][k] = w[co][16 half + k][tap]; data gradient
// B[n = ci][k] = w[16 half + k][ci][8 - tap] (flipped taps, channels swapped).
__global__ void k_pack(const float* __restrict__ params, __nv_bfloat16* __restrict__ packed) {
  pdl_entry();
  const int total = 6 * 2 * (kLayerPack / 2);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int l = e / kLayerPack + 1, dir = (e / (kLayerPack / 2)) & 1, rem = e % (kLayerPack / 2);
    const int s = rem / 512, within = rem % 512;
    const int kg = within / 256, ng = (within / 64) & 3, nr = (within / 8) & 7, kc = within & 7;
    const int nn = ng * 8 + nr, kk = 16 * (s & 1) + kg * 8 + kc, t = s >> 1;
    const float* w = params + off_w(l);
    const float val = dir == 0 ? w[(nn * kC + kk) * 9 + t] : w[(kk * kC + nn) * 9 + (8 - t)];
    packed[e] = __float2bfloat16_rn(val);
  }
}

// ------------------------------------------------------------------ host side
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int check_dims(int n, int rows, int cols, const char* who) {
  if (n < 0 || rows < 0 || cols < 0) return fail(ADJWT_ERR_SHAPE, std::string(who) + ": negative size");
  return ADJWT_OK;
}

int check_ptrs(std::initializer_list<const void*> ps, const char* who) {
  for (const void* p : ps) {
    if (!p) return fail(ADJWT_ERR_INVALID_ARG, std::string(who) + ": NULL pointer");
    if (!aligned16(p)) return fail(ADJWT_ERR_ALIGN, std::string(who) + ": pointer not 16-byte aligned");
  }
  return ADJWT_OK;
}

int64_t act_elems(int n, int rows, int cols) { return (int64_t)n * rows * cols * kC; }

int thin_grid(int64_t pixels) { return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(kThinMaxGrid, (pixels + 255) / 256))); }

int launch_conv32(int n, int H, int W, const __nv_bfloat16* in, const __nv_bfloat16* wpack, const float* bias,
                  int relu, const __nv_bfloat16* mask, __nv_bfloat16* out, cudaStream_t st) {
  const int tiles_x = (W + kTW - 1) / kTW, tiles_y = (H + kTH - 1) / kTH;
  const int64_t grid = (int64_t)n * tiles_x * tiles_y;
  if (grid == 0) return ADJWT_OK;
  if (grid > 0x7FFFFFFF) return fail(ADJWT_ERR_SHAPE, "cnn: image batch too large");
  int* status = device_status_ptr();
  if (mask) {
    ADJWT_CUDA_CHECK(set_smem(k_conv32_tc<true>, kFwdSmem));
    ADJWT_TRACED("cnn_conv32_tc_bwd", 0, st,
                 ADJWT_CUDA_CHECK(pdl_launch(k_conv32_tc<true>, dim3((unsigned)grid), dim3(kFwdThreads), kFwdSmem, st,
                                             H, W, tiles_x, tiles_y, in, wpack, bias, relu, mask, out, status)));
  } else {
    ADJWT_CUDA_CHECK(set_smem(k_conv32_tc<false>, kFwdSmem));
    ADJWT_TRACED("cnn_conv32_tc", 0, st,
                 ADJWT_CUDA_CHECK(pdl_launch(k_conv32_tc<false>, dim3((unsigned)grid), dim3(kFwdThreads), kFwdSmem, st,
                                             H, W, tiles_x, tiles_y, in, wpack, bias, relu, mask, out, status)));
  }
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return ADJWT_OK;
}

int wgrad_grid(int n, int H, int W) {
  const int64_t tiles = (int64_t)n * ((W + kTW - 1) / kTW) * ((H + kTH - 1) / kTH);
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(tiles, std::min(kWgMaxGrid, 2 * sm_count()))));
}

int launch_reduce(int nparts, int stride, const float* part, int C, float* out_w, int boff, int nb, float* out_b,
                  cudaStream_t st) {
  const int count = 9 * C + nb;
  ADJWT_TRACED("cnn_reduce_wgrad", 0, st,
               ADJWT_CUDA_CHECK(pdl_launch(k_reduce_wgrad, dim3((count + 31) / 32), dim3(256), 0, st, nparts, stride,
                                           part, C, out_w, boff, nb, out_b)));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return ADJWT_OK;
}

int launch_conv32_wgrad(int n, int H, int W, const __nv_bfloat16* x, const __nv_bfloat16* dz, float* grad_w,
                        float* grad_b, float* part, cudaStream_t st) {
  const int tiles_x = (W + kTW - 1) / kTW, tiles_y = (H + kTH - 1) / kTH;
  const int grid = wgrad_grid(n, H, W);
  ADJWT_CUDA_CHECK(set_smem(k_conv32_wgrad, kWgSmem));
  ADJWT_TRACED("cnn_conv32_wgrad", 0, st,
               ADJWT_CUDA_CHECK(pdl_launch(k_conv32_wgrad, dim3(grid), dim3(kWgThreads), kWgSmem, st, n, H, W, tiles_x,
                                           tiles_y, x, dz, part)));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return launch_reduce(grid, kWgStride, part, kC * kC, grad_w, 9 * kC * kC, kC, grad_b, st);
}

int launch_thin_wgrad(int n, int H, int W, const __nv_bfloat16* A, const float* s, int64_t sp, bool flip,
                      float* grad_w, float* grad_b, float* part, cudaStream_t st) {
  const int grid = thin_grid((int64_t)n * H * ((W + 31) / 32) * 16);
  ADJWT_TRACED("cnn_thin_wgrad", 0, st,
               ADJWT_CUDA_CHECK(pdl_launch(k_thin_wgrad, dim3(grid), dim3(kThinThreads), 0, st, n, H, W, A, s, sp,
                                           flip ? 1 : 0, part)));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  // bias: sum A (flip = false: the first layer's dz) or sum s (flip: the last layer's dout)
  return launch_reduce(grid, kThinStride, part, kC, grad_w, flip ? 320 : 288, flip ? 1 : kC, grad_b, st);
}

int pix_grid(int64_t pixels) {
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((pixels + 255) / 256, 16 * (int64_t)sm_count())));
}

struct BwdWs {
  float* dout;
  __nv_bfloat16 *za, *zb;
  float* part;
  double* lpart;
  size_t bytes;
};

BwdWs layout_bwd(int n, int H, int W, char* base) {
  BwdWs w{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += static_cast<size_t>(round_up(static_cast<int64_t>(bytes), 256));
    return p;
  };
  const int64_t px = (int64_t)n * H * W;
  w.dout = reinterpret_cast<float*>(take(px * 4));
  w.za = reinterpret_cast<__nv_bfloat16*>(take(px * kC * 2));
  w.zb = reinterpret_cast<__nv_bfloat16*>(take(px * kC * 2));
  w.part = reinterpret_cast<float*>(take(std::max<size_t>((size_t)kWgMaxGrid * kWgStride, (size_t)kThinMaxGrid * kThinStride) * 4));
  w.lpart = reinterpret_cast<double*>(take(kLossBlocks * 8));
  w.bytes = off;
  return w;
}

}  // namespace
}  // namespace adjwt

using namespace adjwt;

extern "C" size_t adjwt_cnn_param_count(void) { return static_cast<size_t>(kParamCount); }
extern "C" size_t adjwt_cnn_packed_bytes(void) { return static_cast<size_t>(6 * 2 * kLayerPack); }
extern "C" size_t adjwt_cnn_activation_bytes(int n, int rows, int cols) {
  if (n < 0 || rows < 0 || cols < 0) return 0;
  return static_cast<size_t>(7 * act_elems(n, rows, cols) * 2);
}
extern "C" size_t adjwt_cnn_workspace_size(int n, int rows, int cols) {
  if (n < 0 || rows < 0 || cols < 0) return 0;
  return layout_bwd(n, rows, cols, nullptr).bytes;
}
extern "C" size_t adjwt_cnn_wgrad_workspace_size(void) { return static_cast<size_t>(kWgMaxGrid) * kWgStride * 4; }

extern "C" int cnn_pack(const float* params, void* packed, adjwt_stream_t stream) {
  int rc = check_ptrs({params, packed}, "cnn_pack");
  if (rc) return rc;
  cudaStream_t st = stream;
  ADJWT_TRACED("cnn_pack", 0, st,
               ADJWT_CUDA_CHECK(pdl_launch(k_pack, dim3(216), dim3(256), 0, st, params,
                                           static_cast<__nv_bfloat16*>(packed))));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return ADJWT_OK;
}

extern "C" int cnn_conv32(int n, int rows, int cols, const void* in, const void* packed_layer, const float* bias,
                          int relu, const void* mask, void* out, adjwt_stream_t stream) {
  int rc = check_dims(n, rows, cols, "cnn_conv32");
  if (rc) return rc;
  if ((int64_t)n * rows * cols == 0) return ADJWT_OK;
  rc = check_ptrs({in, packed_layer, out}, "cnn_conv32");
  if (!rc && mask) rc = check_ptrs({mask}, "cnn_conv32");
  if (rc) return rc;
  const size_t bytes = static_cast<size_t>(act_elems(n, rows, cols)) * 2;
  const uintptr_t a = reinterpret_cast<uintptr_t>(in), o = reinterpret_cast<uintptr_t>(out);
  if (a < o + bytes && o < a + bytes) return fail(ADJWT_ERR_ALIAS, "cnn_conv32: output overlaps input");
  return launch_conv32(n, rows, cols, static_cast<const __nv_bfloat16*>(in),
                       static_cast<const __nv_bfloat16*>(packed_layer), bias, relu,
                       static_cast<const __nv_bfloat16*>(mask), static_cast<__nv_bfloat16*>(out), stream);
}

extern "C" int cnn_conv32_wgrad(int n, int rows, int cols, const void* x, const void* dz, float* grad_w, float* grad_b,
                                void* ws, size_t ws_bytes, adjwt_stream_t stream) {
  int rc = check_dims(n, rows, cols, "cnn_conv32_wgrad");
  if (!rc) rc = check_ptrs({x, dz, grad_w, grad_b}, "cnn_conv32_wgrad");
  if (rc) return rc;
  if (!ws || ws_bytes < adjwt_cnn_wgrad_workspace_size() || !aligned16(ws))
    return fail(ADJWT_ERR_WORKSPACE, "cnn_conv32_wgrad: workspace of adjwt_cnn_wgrad_workspace_size() bytes needed");
  return launch_conv32_wgrad(n, rows, cols, static_cast<const __nv_bfloat16*>(x), static_cast<const __nv_bfloat16*>(dz),
                             grad_w, grad_b, static_cast<float*>(ws), stream);
}

extern "C" int cnn_forward(int n, int rows, int cols, const float* b, int64_t pitch, const float* params,
                           const void* packed, void* act, float* u_hat, adjwt_stream_t stream) {
  int rc = check_dims(n, rows, cols, "cnn_forward");
  if (rc) return rc;
  if ((int64_t)n * rows * cols == 0) return ADJWT_OK;
  if (pitch < cols) return fail(ADJWT_ERR_SHAPE, "cnn_forward: pitch < cols");
  rc = check_ptrs({b, params, packed, act, u_hat}, "cnn_forward");
  if (rc) return rc;
  cudaStream_t st = stream;
  const int64_t px = (int64_t)n * rows * cols;
  auto* A = static_cast<__nv_bfloat16*>(act);
  const auto* P = static_cast<const __nv_bfloat16*>(packed);
  ADJWT_TRACED("cnn_conv_in", 0, st,
               ADJWT_CUDA_CHECK(pdl_launch(k_conv_in, dim3(pix_grid(px)), dim3(256), 0, st, n, rows, cols, b, pitch,
                                           params + kOffW0, A)));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  for (int l = 1; l <= 6; ++l) {
    rc = launch_conv32(n, rows, cols, A + (l - 1) * px * kC, P + (size_t)(l - 1) * 2 * (kLayerPack / 2),
                       params + off_b(l), 1, nullptr, A + l * px * kC, st);
    if (rc) return rc;
  }
  ADJWT_TRACED("cnn_conv_out", 0, st,
               ADJWT_CUDA_CHECK(pdl_launch(k_conv_out, dim3(pix_grid(px)), dim3(256), 0, st, n, rows, cols,
                                           A + 6 * px * kC, params + kOffW7, b, pitch, u_hat)));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return ADJWT_OK;
}

extern "C" int cnn_backward(int n, int rows, int cols, const float* b, const float* u_hat, const float* u_ref,
                            int64_t pitch, const float* params, const void* packed, const void* act, float* grad,
                            double* loss_dev, void* ws, size_t ws_bytes, adjwt_stream_t stream) {
  int rc = check_dims(n, rows, cols, "cnn_backward");
  if (rc) return rc;
  if (pitch < cols) return fail(ADJWT_ERR_SHAPE, "cnn_backward: pitch < cols");
  rc = check_ptrs({b, u_hat, u_ref, params, packed, act, grad, loss_dev}, "cnn_backward");
  if (rc) return rc;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < adjwt_cnn_workspace_size(n, rows, cols))
    return fail(ADJWT_ERR_WORKSPACE, "cnn_backward: workspace of adjwt_cnn_workspace_size bytes, 256-byte aligned, needed");
  cudaStream_t st = stream;
  const int64_t px = (int64_t)n * rows * cols;
  if (px == 0) {
    ADJWT_CUDA_CHECK(cudaMemsetAsync(grad, 0, kParamCount * sizeof(float), st));
    ADJWT_CUDA_CHECK(cudaMemsetAsync(loss_dev, 0, sizeof(double), st));
    return ADJWT_OK;
  }
  const BwdWs w = layout_bwd(n, rows, cols, static_cast<char*>(ws));
  const auto* A = static_cast<const __nv_bfloat16*>(act);
  const auto* P = static_cast<const __nv_bfloat16*>(packed);
  const int lb = static_cast<int>(std::min<int64_t>(kLossBlocks, (px + 255) / 256));
  ADJWT_TRACED("cnn_loss_grad", 0, st,
               ADJWT_CUDA_CHECK(pdl_launch(k_loss_grad, dim3(lb), dim3(256), 0, st, n, rows, cols, u_hat, u_ref, pitch,
                                           static_cast<float>(1.0 / (double)px), w.dout, w.lpart)));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  rc = launch_sum_partials(w.lpart, lb, 0.5 / (double)px, nullptr, 0, 0.0, loss_dev, st);
  if (rc) return rc;
  // last layer: weights from (a_7, dout), then dz_7 = [a_7 > 0] conv^T(dout)
  rc = launch_thin_wgrad(n, rows, cols, A + 6 * px * kC, w.dout, cols, true, grad + kOffW7, grad + kOffB7, w.part, st);
  if (rc) return rc;
  ADJWT_TRACED("cnn_conv_out_bwd", 0, st,
               ADJWT_CUDA_CHECK(pdl_launch(k_conv_out_bwd, dim3(pix_grid(px)), dim3(256), 0, st, n, rows, cols, w.dout,
                                           params + kOffW7, A + 6 * px * kC, w.za)));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  __nv_bfloat16 *cur = w.za, *nxt = w.zb;
  for (int l = 6; l >= 1; --l) {
    const __nv_bfloat16* x_in = A + (l - 1) * px * kC;  // a_l's input: the output of layer l - 1
    rc = launch_conv32_wgrad(n, rows, cols, x_in, cur, grad + off_w(l), grad + off_b(l), w.part, st);
    if (rc) return rc;
    rc = launch_conv32(n, rows, cols, cur, P + (size_t)((l - 1) * 2 + 1) * (kLayerPack / 2), nullptr, 0, x_in, nxt, st);
    if (rc) return rc;
    std::swap(cur, nxt);
  }
  return launch_thin_wgrad(n, rows, cols, cur, b, pitch, false, grad + kOffW0, grad + kOffB0, w.part, st);
}

extern "C" int cnn_adam(int64_t count, float* params, const float* grad, float* m, float* v, int64_t step, double lr,
                        double beta1, double beta2, double eps, adjwt_stream_t stream) {
  if (count < 0) return fail(ADJWT_ERR_SHAPE, "cnn_adam: count < 0");
  if (step < 1) return fail(ADJWT_ERR_INVALID_ARG, "cnn_adam: step must be >= 1");
  if (!(beta1 >= 0.0 && beta1 < 1.0 && beta2 >= 0.0 && beta2 < 1.0 && eps > 0.0 && lr >= 0.0))
    return fail(ADJWT_ERR_INVALID_ARG, "cnn_adam: need 0 <= beta < 1, eps > 0, lr >= 0");
  if (count == 0) return ADJWT_OK;
  int rc = check_ptrs({params, grad, m, v}, "cnn_adam");
  if (rc) return rc;
  cudaStream_t st = stream;
  const float bc1 = static_cast<float>(1.0 - std::pow(beta1, (double)step));
  const float bc2 = static_cast<float>(1.0 - std::pow(beta2, (double)step));
  ADJWT_TRACED("cnn_adam", 0, st,
               ADJWT_CUDA_CHECK(pdl_launch(k_adam, dim3(pix_grid(count)), dim3(256), 0, st, count, params, grad, m, v,
                                           static_cast<float>(lr), static_cast<float>(beta1), static_cast<float>(beta2),
                                           static_cast<float>(eps), bc1, bc2)));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return ADJWT_OK;
}
