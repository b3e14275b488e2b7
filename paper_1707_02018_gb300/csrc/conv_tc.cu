// Channel gradient (Sec. II, Eq. 5) for 49 <= k <= 64 (taps zero-padded to
// 64) on the 5th-generation tensor cores.
//
// The unit of work is a chunk of 4096 samples of one row, m0 .. m0 + 4095,
// seen as 128 blocks of 32 (block a, offset c: sample m0 + 32 a + c).  Two of
// the three sums of Eq. 5 are then M = 128 (blocks) x N = 32 x K = 96
// products:
//   r[32a + c]      = sum_{q<96} W[a][q] H1[q][c],  W[a][q] = s[m0 - 64 + 32a + q],  H1[q][c] = h[c + 64 - q]
//   grad_s[32a + c] = sum_{q<96} V[a][q] H2[q][c],  V[a][q] = r[m0 + 32a + q],       H2[q][c] = h[q - c]
// issued with tcgen05.mma (kind::tf32, accumulators in tensor memory), and
//   part[j] = sum_{a<128, c<32} s[m0 + 32a + c] r[m0 + 32a + c + j]      (j < k)
// runs on the warp-level m16n8k8 TF32 MMA while the tensor core computes
// grad_s: warp w takes blocks 16 w .. 16 w + 15 for the whole band of
// P[c][q] = sum_a s[32a + c] r[32a + q] (c < 32, q - c < 64) and folds each
// product straight into per-thread diagonal sums (j = q - c), which one
// deterministic pass over shared memory then adds up.
//
// Operands live in shared memory in the K-major no-swizzle layout as block
// matrices B[a'][j] = x[base + 32 a' + j] stored [j/4][a'][4]: each row of a
// 4-column slab is 16 bytes, so the K range [32 t, 32 t + 32) of W (or V) is
// the same matrix t rows down (descriptor start + 16 t bytes).  The Toeplitz
// factors are a band array G[rho][k'] (8 columns, rows 0 .. 119) of which
// K-step kk reads the 32 rows from 88 - 8 kk; the H2 band replaces the H1
// band once the first product is done.  The 64 residuals past the chunk (read
// by grad_s and grad_h of its last two blocks) come from the CUDA cores.
// Float32 accuracy: each operand is split into a TF32 high part and the float
// remainder (x = x_hi + x_lo), and a product is A_hi B_hi + A_hi B_lo +
// A_lo B_hi.  The band array stores the hi and lo halves of each 8-row group
// side by side, so one N = 64 MMA forms A_hi B_hi and A_hi B_lo (columns
// 16 (c/8) + c%8 and 16 (c/8) + 8 + c%8) and an N = 32 MMA over every other
// group forms A_lo B_hi: two MMAs and two reads of the A tile per K-step.
//
// CTAs are persistent (two per SM, about 110 KB of shared memory each) and
// walk the chunks in a grid-stride loop; cp.async brings the next chunk's raw
// s, x (or r) and h into shared memory while the current chunk is computed,
// so a chunk starts from on-chip data.  Every mbarrier wait is bounded.
#include <algorithm>

#include "adjwt_internal.h"
#include "tma.cuh"
#include "umma.cuh"

namespace adjwt {
namespace {

constexpr int kNT = 256;
constexpr int kLb = 32;                  // block length (N of the products)
constexpr int kBlocks = 128;             // blocks per chunk (M)
constexpr int kChunk = kBlocks * kLb;    // 4096 samples per chunk
constexpr int kKSteps = (kLb + 64) / 8;  // 12 K-steps of 8
constexpr int kSRows = kBlocks + 4;      // s rows: s[m0 - 64] .. s[m0 + 4159]
constexpr int kRNeed = kBlocks + 2;      // r rows read: r[m0] .. r[m0 + 4159]
constexpr int kRRows = kBlocks + 4;      // r slab pitch (rows); 132 = 4 mod 8 keeps the fragment reads conflict-free
constexpr int kGGroups = 15;             // band row groups of 8 (rows 0 .. 119)
constexpr int kGSlab = 2 * kGGroups * 32 + 16;  // floats per 4-column band slab: hi, lo groups side by side; +16 spreads the banks
constexpr int kGOff = 88;                // K-step kk reads band rows kGOff - 8 kk ..
constexpr int kRawPitch = kLb + 4;       // raw x / r rows: 16-byte reads of a column are conflict-free
constexpr int kOutPitch = kLb + 1;       // grad_s staging tile pitch (conflict-free column writes)

// float offsets in dynamic shared memory (each a multiple of 32 floats)
constexpr int kS_HI = 0;
constexpr int kS_LO = kS_HI + kSRows * kLb;
constexpr int kR_HI = kS_LO + kSRows * kLb;
constexpr int kR_LO = kR_HI + kRRows * kLb;
constexpr int kG_HI = kR_LO + kRRows * kLb;
constexpr int kSRaw = kG_HI + 2 * kGSlab;              // s[m0 - 64 .. m0 + 4160), linear
constexpr int kXRaw = kSRaw + kSRows * kLb;            // x (or r) rows of kRawPitch
constexpr int kH = kXRaw + (kRNeed * kRawPitch + 31) / 32 * 32;  // two tap buffers (current, next)
constexpr int kSLin = kH + 128;          // s[m0 + 4032] .. s[m0 + 4159] (taps of the 64 tail residuals)
constexpr int kTotal = kSLin + 128;
constexpr int kDiag = 18;                // diagonal sums per thread: d = 0 .. 8, two parities
constexpr size_t kSmemBytes = 128 + (size_t)kTotal * 4;
static_assert(kSmemBytes <= 113 * 1024, "two CTAs per SM");
static_assert(8 * kDiag * 36 + 4 * 64 <= kR_HI, "grad_h scratch fits in the s arrays");
static_assert(kBlocks * kOutPitch <= kRRows * kLb, "grad_s staging fits in the r array");
constexpr uint32_t kTmemCols = 256;  // per product: A_hi (B_hi|B_lo) in 64 columns, A_lo B_hi in 32

__host__ __device__ constexpr int blk_idx(int row, int j, int rows) { return ((j >> 2) * rows + row) * 4 + (j & 3); }

// v = hi + lo exactly: hi keeps the 10 explicit mantissa bits a TF32 operand
// carries (so it is exact whether the tensor core truncates or rounds), lo is
// the float remainder.
__device__ __forceinline__ void tf32_split(float v, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
  lo = v - hi;
}

// instruction descriptors: f32 accumulate, tf32 A and B, both K-major, M = 128, N = 64 or 32
__host__ __device__ constexpr uint32_t idesc_n(uint32_t n) { return (1u << 4) | (2u << 7) | (2u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24); }

__device__ __forceinline__ void umma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// The 16 product values of row a = 32 (warp % 4) + lane, columns c0 .. c0 + 15
// (c0 = 16 (warp / 4)), of the product accumulated at tensor memory column col.
__device__ __forceinline__ void product_row16(uint32_t tmem_warp, uint32_t col, int c0, float (&v)[16]) {
  float both[32], lo_hi[16];
  tmem_ld32(tmem_warp + col + 2 * c0, both);  // c in [c0, c0 + 16): columns 16 (c/8) + c%8 (+ 8 for A_hi B_lo)
  tmem_ld16(tmem_warp + col + 64 + c0, lo_hi);
#pragma unroll
  for (int e = 0; e < 16; ++e) v[e] = (both[16 * (e >> 3) + 8 + (e & 7)] + lo_hi[e]) + both[16 * (e >> 3) + (e & 7)];
}

// hi/lo split of four consecutive columns into one 16-byte slab row each
__device__ __forceinline__ void split_store4(float* hi, float* lo, int idx, float a, float b, float c, float d) {
  float4 h4, l4;
  tf32_split(a, h4.x, l4.x);
  tf32_split(b, h4.y, l4.y);
  tf32_split(c, h4.z, l4.z);
  tf32_split(d, h4.w, l4.w);
  *reinterpret_cast<float4*>(hi + idx) = h4;
  *reinterpret_cast<float4*>(lo + idx) = l4;
}


__device__ __forceinline__ void mma_m16n8k8(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One product (24 MMAs: 12 K-steps x A_hi (B_hi|B_lo), A_lo B_hi) into tensor
// memory columns tmem_d .. + 63 and tmem_d + 64 .. + 95.  X: block matrix with
// slab pitch `rows` (hi at xh, lo at xl); g: the interleaved band array.
__device__ __forceinline__ void issue_product(uint32_t tmem_d, uint32_t xh, uint32_t xl, int rows, uint32_t g) {
  const uint32_t lbo_x = rows * 16, lbo_g = kGSlab * 4;
#pragma unroll 1
  for (int kk = 0; kk < kKSteps; ++kk) {
    const uint32_t aoff = 2 * (kk & 3) * lbo_x + 16 * (kk >> 2);
    const uint32_t boff = (kGOff / 8 - kk) * 256;  // hi half of row group 11 - kk
    const uint64_t ah = umma_desc(xh + aoff, lbo_x, 128), al = umma_desc(xl + aoff, lbo_x, 128);
    const uint64_t b_both = umma_desc(g + boff, lbo_g, 128);  // groups hi, lo, hi, lo, ...: N = 64
    const uint64_t b_hi = umma_desc(g + boff, lbo_g, 256);    // hi groups only: N = 32
    umma_tf32(tmem_d, ah, b_both, idesc_n(64), kk > 0);
    umma_tf32(tmem_d + 64, al, b_hi, idesc_n(32), kk > 0);
  }
}

__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, int* status) {
  if (mbar_wait(bar, parity)) return true;
  record_status(status, ADJWT_ERR_TIMEOUT);
  return false;
}

// Block-wide wait for a product: thread 0 polls the barrier (bounded), the
// others wait at the block barrier; true for every thread if it completed.
__device__ __forceinline__ bool block_wait_product(uint64_t* bar, uint32_t parity, int* status) {
  const bool ok = threadIdx.x == 0 ? wait_bar(bar, parity, status) : true;
  const bool all = __syncthreads_and(ok);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return all;
}


// Raw s of one chunk: s_raw[u] = s[m0 - 64 + u] (zero off the row), u < 4224.
// vec: the row is 16-byte aligned and n a multiple of 4.
__device__ __forceinline__ void fetch_s(float* s_raw, const float* srow, int64_t n, int64_t m0, bool vec, int tid) {
  if (vec) {
    for (int u = 4 * tid; u < kSRows * kLb; u += 4 * kNT) {
      const int64_t q = m0 - 64 + u;
      const bool in = q >= 0 && q < n;
      cp_async16(s_raw + u, in ? srow + q : srow, in ? 16u : 0u);
    }
  } else {
    for (int u = tid; u < kSRows * kLb; u += kNT) {
      const int64_t q = m0 - 64 + u;
      const bool in = q >= 0 && q < n;
      cp_async4(s_raw + u, in ? srow + q : srow, in ? 4u : 0u);
    }
  }
}

// Raw x (fused: rows 0..127) or r (given: rows 0..129) of one chunk:
// x_raw[a * kRawPitch + c] = row[m0 + 32 a + c] (zero past len or if row is null).
__device__ __forceinline__ void fetch_rows(float* x_raw, const float* row, int64_t len, int64_t m0, int rows,
                                           bool vec, int tid) {
  if (!row) {
    for (int u = tid; u < rows * kLb; u += kNT) x_raw[(u / kLb) * kRawPitch + u % kLb] = 0.0f;
  } else if (vec) {
    for (int u = 4 * tid; u < rows * kLb; u += 4 * kNT) {
      const int64_t q = m0 + u;
      const bool in = q < len;
      cp_async16(x_raw + (u / kLb) * kRawPitch + u % kLb, in ? row + q : row, in ? 16u : 0u);
    }
  } else {
    for (int u = tid; u < rows * kLb; u += kNT) {
      const int64_t q = m0 + u;
      const bool in = q < len;
      cp_async4(x_raw + (u / kLb) * kRawPitch + u % kLb, in ? row + q : row, in ? 4u : 0u);
    }
  }
}

// Toeplitz band for product 1 (G[rho][k'] = h[rho - k' - 24]) or product 2
// (G[rho][k'] = h[k' - rho + 88]), split hi/lo: slab k'/4, row group rho/8
// with its hi half at 32-float slot 2 (rho/8) and its lo half at the next slot.
__device__ __forceinline__ void build_band(float* G, const float* h_sm, bool second, int tid) {
  for (int i = tid; i < kGGroups * 64; i += kNT) {
    const int rho = i >> 3, kq = i & 7;
    const int ti = second ? kq - rho + kGOff : rho - kq - (kGOff - 64);
    const float g = (ti >= 0 && ti < 64) ? h_sm[ti] : 0.0f;
    const int o = (kq >> 2) * kGSlab + (rho >> 3) * 64 + (rho & 7) * 4 + (kq & 3);
    tf32_split(g, G[o], G[o + 32]);
  }
}

__device__ __forceinline__ void operands_ready() {
  fence_proxy_async();  // generic-proxy writes of the operands -> tensor core
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

template <bool FUSED>
__global__ void __launch_bounds__(kNT, 2) k_conv_tc(int64_t n, int K, int batch, const float* __restrict__ s,
                                                    const float* __restrict__ h, const float* __restrict__ x,
                                                    const float* __restrict__ r_in, float* __restrict__ r_out,
                                                    float* __restrict__ grad_s, float* __restrict__ part_h, int nchunks,
                                                    int vec, int* status) {
  pdl_entry();
  extern __shared__ unsigned char dyn[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_holder;
  float* sm = reinterpret_cast<float*>(dyn + ((128 - (smem_u32(dyn) & 127)) & 127));
  float* S_hi = sm + kS_HI;
  float* S_lo = sm + kS_LO;
  float* R_hi = sm + kR_HI;
  float* R_lo = sm + kR_LO;
  float* G = sm + kG_HI;
  float* s_raw = sm + kSRaw;
  float* x_raw = sm + kXRaw;
  float* s_lin = sm + kSLin;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t nr = n + K - 1;
  const int64_t total = (int64_t)batch * nchunks;
  const bool vec_s = vec & 1, vec_x = vec & 2;
  const float* xs = FUSED ? x : r_in;  // the second input row array (row length nr)
  const int xrows = FUSED ? kBlocks : kRNeed;

  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // prologue: the first chunk's raw inputs
  if (blockIdx.x < total) {
    const int b = static_cast<int>(blockIdx.x / nchunks);
    const int64_t m0 = (int64_t)(blockIdx.x % nchunks) * kChunk;
    fetch_s(s_raw, s + (size_t)b * n, n, m0, vec_s, tid);
    fetch_rows(x_raw, xs ? xs + (size_t)b * nr : nullptr, nr, m0, xrows, vec_x, tid);
    if (tid < 64) cp_async4(sm + kH + tid, h + (size_t)b * K + (tid < K ? tid : 0), tid < K ? 4u : 0u);
    cp_async_commit();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_holder;
  const uint32_t base = smem_u32(sm);
  const uint32_t tmem_warp = tmem + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's 32 lanes
  uint32_t phase = 0;
  bool ok = true;
  int hb = 0;  // tap buffer of the current chunk

  for (int64_t cid = blockIdx.x; cid < total && ok; cid += gridDim.x) {
    const int b = static_cast<int>(cid / nchunks);
    const int cx = static_cast<int>(cid % nchunks);
    const int64_t m0 = (int64_t)cx * kChunk;
    const bool last = cx == nchunks - 1;
    const int64_t nxt = cid + gridDim.x;
    const bool has_next = nxt < total;
    const int nb = has_next ? static_cast<int>(nxt / nchunks) : 0;
    const int64_t nm0 = has_next ? (int64_t)(nxt % nchunks) * kChunk : 0;
    const float* h_sm = sm + kH + 64 * hb;

    cp_async_wait_all();
    __syncthreads();  // this chunk's raw inputs are in shared memory
    // ---- split s (and r, if given) into the hi/lo block matrices ----
    for (int u = 4 * tid; u < kSRows * kLb; u += 4 * kNT) {
      const float4 v = *reinterpret_cast<const float4*>(s_raw + u);
      split_store4(S_hi, S_lo, blk_idx(u / kLb, u % kLb, kSRows), v.x, v.y, v.z, v.w);
      if (u >= kChunk) *reinterpret_cast<float4*>(s_lin + u - kChunk) = v;
    }
    if (!FUSED) {
      for (int u = 4 * tid; u < kRNeed * kLb; u += 4 * kNT) {
        const float4 v = *reinterpret_cast<const float4*>(x_raw + (u / kLb) * kRawPitch + u % kLb);
        split_store4(R_hi, R_lo, blk_idx(u / kLb, u % kLb, kRRows), v.x, v.y, v.z, v.w);
      }
    }
    build_band(G, h_sm, !FUSED, tid);
    operands_ready();
    // the raw s (and raw r) buffers are free: fetch the next chunk's
    if (has_next) {
      fetch_s(s_raw, s + (size_t)nb * n, n, nm0, vec_s, tid);
      if (!FUSED) fetch_rows(x_raw, r_in + (size_t)nb * nr, nr, nm0, kRNeed, vec_x, tid);
      if (tid < 64) cp_async4(sm + kH + 64 * (hb ^ 1) + tid, h + (size_t)nb * K + (tid < K ? tid : 0), tid < K ? 4u : 0u);
    }
    cp_async_commit();

    if (FUSED) {
      // ---- r = h * s - x: product 1 into tmem columns [0, 96) ----
      if (tid == 0) {
        issue_product(tmem, base + kS_HI * 4, base + kS_LO * 4, kSRows, base + kG_HI * 4);
        umma_commit(&bar);
      }
      // meanwhile the CUDA cores form r on the 64 positions past the chunk
      // (r rows 128 and 129): four threads per position, taps i = quarter mod 4
      {
        const int e = tid >> 2, quarter = tid & 3;
        float acc = 0.0f;
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          const int i = 4 * t + quarter;
          acc = fmaf(h_sm[i], s_lin[e + 64 - i], acc);  // s[m0 + 4096 + e - i]
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (quarter == 0) {
          const int p = kChunk + e;
          const int64_t q = m0 + p;
          float rv = 0.0f;
          if (q < nr) rv = acc - (x ? __ldg(x + (size_t)b * nr + q) : 0.0f);
          const int i = blk_idx(p / kLb, p % kLb, kRRows);
          tf32_split(rv, R_hi[i], R_lo[i]);
          if (last && r_out && p < kChunk + K - 1 && q < nr) r_out[(size_t)b * nr + q] = rv;
        }
      }
      ok = block_wait_product(&bar, phase, status);
      phase ^= 1;
      if (!ok) break;
      {
        const int a = 32 * (warp & 3) + lane, c0 = 16 * (warp >> 2);
        float d[16];
        product_row16(tmem_warp, 0, c0, d);
#pragma unroll
        for (int g4 = 0; g4 < 16; g4 += 4) {
          const float4 xv = *reinterpret_cast<const float4*>(x_raw + a * kRawPitch + c0 + g4);
          const float xe[4] = {xv.x, xv.y, xv.z, xv.w};
          float rv[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int64_t q = m0 + kLb * a + c0 + g4 + e;
            rv[e] = q < nr ? d[g4 + e] - xe[e] : 0.0f;
          }
          split_store4(R_hi, R_lo, blk_idx(a, c0 + g4, kRRows), rv[0], rv[1], rv[2], rv[3]);
        }
      }
      build_band(G, h_sm, true, tid);  // product 1 has finished reading the first band
      operands_ready();
      if (has_next) fetch_rows(x_raw, x ? x + (size_t)nb * nr : nullptr, nr, nm0, kBlocks, vec_x, tid);
      cp_async_commit();
    }

    // ---- grad_s: product 2 into tmem columns [128, 224), overlapped with grad_h ----
    if (grad_s && tid == 0) {
      issue_product(tmem + 128, base + kR_HI * 4, base + kR_LO * 4, kRRows, base + kG_HI * 4);
      umma_commit(&bar);
    }
    if (FUSED && r_out) {
      // r = hi + lo exactly; a warp stores 128 consecutive samples
      float* rout = r_out + (size_t)b * nr;
      for (int v = 4 * tid; v < kChunk; v += 4 * kNT) {
        const int a = v / kLb, c = v % kLb;
        const int i = blk_idx(a, c, kRRows);
        const float4 hv = *reinterpret_cast<const float4*>(R_hi + i);
        const float4 lv = *reinterpret_cast<const float4*>(R_lo + i);
        const float rv[4] = {hv.x + lv.x, hv.y + lv.y, hv.z + lv.z, hv.w + lv.w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (m0 + v + e < nr) rout[m0 + v + e] = rv[e];
      }
    }

    // ---- grad_h partial (warp MMA; see the header) ----
    if (part_h) {
      const int g = lane >> 2, t = lane & 3;
      float diag[kDiag];  // diag[2 d + bit]: entries with q - c = 8 d + 2 t + bit - g (d < 0 or > 8: never a lag < 64)
#pragma unroll
      for (int i = 0; i < kDiag; ++i) diag[i] = 0.0f;
#pragma unroll 1
      for (int kk = 2 * warp; kk < 2 * warp + 2; ++kk) {
        const int a0 = 8 * kk + t, a1 = a0 + 4;  // blocks; s of block a is s row a + 2
        uint32_t ah[2][4], al[2][4];
#pragma unroll
        for (int mc = 0; mc < 2; ++mc) {
          const int c_a = 16 * mc + g, c_b = c_a + 8;
          const int i0 = blk_idx(a0 + 2, c_a, kSRows), i1 = blk_idx(a0 + 2, c_b, kSRows);
          const int i2 = blk_idx(a1 + 2, c_a, kSRows), i3 = blk_idx(a1 + 2, c_b, kSRows);
          ah[mc][0] = __float_as_uint(S_hi[i0]);
          ah[mc][1] = __float_as_uint(S_hi[i1]);
          ah[mc][2] = __float_as_uint(S_hi[i2]);
          ah[mc][3] = __float_as_uint(S_hi[i3]);
          al[mc][0] = __float_as_uint(S_lo[i0]);
          al[mc][1] = __float_as_uint(S_lo[i1]);
          al[mc][2] = __float_as_uint(S_lo[i2]);
          al[mc][3] = __float_as_uint(S_lo[i3]);
        }
#pragma unroll
        for (int nt = 0; nt < 12; ++nt) {
          const int q = 8 * nt + g;  // r[32a + q]: row a + q / 32, column q % 32
          const int j0 = blk_idx(a0 + q / kLb, q % kLb, kRRows), j1 = blk_idx(a1 + q / kLb, q % kLb, kRRows);
          const uint32_t bh0 = __float_as_uint(R_hi[j0]), bl0 = __float_as_uint(R_lo[j0]);
          const uint32_t bh1 = __float_as_uint(R_hi[j1]), bl1 = __float_as_uint(R_lo[j1]);
#pragma unroll
          for (int mc = 0; mc < 2; ++mc) {
            const int u = nt - 2 * mc;  // n tile relative to the m tile's band start
            if (u < 0 || u > 9) continue;
            float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            mma_m16n8k8(acc, al[mc], bh0, bh1);
            mma_m16n8k8(acc, ah[mc], bl0, bl1);
            mma_m16n8k8(acc, ah[mc], bh0, bh1);
            // element i: c = 16 mc + g + 8 (i >> 1), q = 8 nt + 2 t + (i & 1)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int d = u - (i >> 1);
              if (d >= 0 && d <= 8) diag[2 * d + (i & 1)] += acc[i];
            }
          }
        }
      }
      __syncthreads();  // the diagonal sums and their totals reuse the s arrays
      float* dg = S_hi;  // dg[(warp * kDiag + slot) * 36 + 8 t + g]: conflict-free both ways
#pragma unroll
      for (int i = 0; i < kDiag; ++i) dg[(warp * kDiag + i) * 36 + 8 * t + g] = diag[i];
      __syncthreads();
      float* red4 = dg + 8 * kDiag * 36;
      {
        // lag j collects, from each warp, the lanes (g, t) and parities with
        // 8 d + bit = j + g - 2 t: g = (bit - j + 2 t) mod 8
        const int j = tid & 63, part = tid >> 6;
        float tsum = 0.0f;
#pragma unroll
        for (int w = 2 * part; w < 2 * part + 2; ++w)
#pragma unroll
          for (int tt = 0; tt < 4; ++tt)
#pragma unroll
            for (int bit = 0; bit < 2; ++bit) {
              const int gg = (bit - j + 2 * tt) & 7;
              const int e = j + gg - 2 * tt;  // = 8 d + bit >= 0
              const int d = (e - bit) / 8;    // 0 .. 8 for j < 64
              tsum += dg[(w * kDiag + 2 * d + bit) * 36 + 8 * tt + gg];
            }
        red4[part * 64 + j] = tsum;
      }
      __syncthreads();
      float* dst = part_h + ((size_t)b * nchunks + cx) * K;
      for (int j = tid; j < K; j += kNT) dst[j] = (red4[j] + red4[64 + j]) + (red4[128 + j] + red4[192 + j]);
    }

    // ---- grad_s out of tensor memory, staged in the (now free) r array ----
    if (grad_s) {
      ok = block_wait_product(&bar, phase, status);  // the barrier also ends grad_h's and the r store's reads of r
      phase ^= 1;
      if (!ok) break;
      float* out_t = R_hi;
      {
        const int a = 32 * (warp & 3) + lane, c0 = 16 * (warp >> 2);
        float d[16];
        product_row16(tmem_warp, 128, c0, d);
#pragma unroll
        for (int e = 0; e < 16; ++e) out_t[a * kOutPitch + c0 + e] = d[e];
      }
      __syncthreads();
      float* out = grad_s + (size_t)b * n;
      for (int v = tid; v < kChunk; v += kNT) {
        const int64_t m = m0 + v;
        if (m < n) out[m] = out_t[(v / kLb) * kOutPitch + (v % kLb)];
      }
    }
    hb ^= 1;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // shared arrays and tensor memory are reused by the next chunk
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  cp_async_wait_all();  // no copy may land after the CTA has exited
  if (!ok && tid == 0) (void)mbar_wait(&bar, phase ^ 1);  // give a late product one more bounded wait
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace

bool conv_tc_supported(int k) { return k >= 49 && k <= 64; }
int64_t conv_tc_nchunks(int64_t n) { return (n + kChunk - 1) / kChunk; }

int launch_conv_tc(int batch, int64_t n, int k, const float* s, const float* h, const float* x, const float* r_in,
                   float* r_out, float* grad_h, float* grad_s, float* partials, cudaStream_t st) {
  if (batch == 0 || n == 0) return ADJWT_OK;
  const int64_t nch = conv_tc_nchunks(n);
  if (nch > 0x7fffffff) return fail(ADJWT_ERR_SHAPE, "conv: n too large");
  const int64_t total = (int64_t)batch * nch;
  const unsigned grid = static_cast<unsigned>(std::min<int64_t>(total, 2 * (int64_t)sm_count()));
  float* part = grad_h ? partials : nullptr;
  auto kern = r_in ? k_conv_tc<false> : k_conv_tc<true>;
  auto aligned = [](const void* p, int64_t len) { return reinterpret_cast<uintptr_t>(p) % 16 == 0 && len % 4 == 0; };
  const float* xs = r_in ? r_in : x;
  const int vec = (aligned(s, n) ? 1 : 0) | (xs && aligned(xs, n + k - 1) ? 2 : 0);
  ADJWT_CUDA_CHECK(set_smem(kern, kSmemBytes));
  ADJWT_TRACED(r_in ? "conv_adjoint" : "conv_gradient", 0, st,
               pdl_launch(kern, dim3(grid), kNT, kSmemBytes, st, n, k, batch, s, h, r_in ? nullptr : x, r_in,
                          r_in ? nullptr : r_out, grad_s, part, static_cast<int>(nch), vec, device_status_ptr()));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  if (grad_h) {
    const int64_t tot = (int64_t)batch * k;
    const unsigned nb = static_cast<unsigned>((tot + 255) / 256);
    ADJWT_TRACED("conv_reduce", 0, st, conv_reduce(nb, k, static_cast<int>(nch), partials, grad_h, tot, st));
    ADJWT_CUDA_CHECK(cudaGetLastError());
  }
  return ADJWT_OK;
}

}  // namespace adjwt
