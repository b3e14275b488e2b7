// Register-blocked channel gradient (Sec. II, Eq. 5) for k <= kFusedMaxK.
//
// The taps are zero-padded to kp = 16 * ceil(k / 16) (h[i] = 0 for i >= k),
// which leaves r = h * s - x, grad_s and the first k lags of grad_h unchanged
// and gives every window a 16-aligned start.  One CTA owns a chunk of CH
// samples of one row (CH = the largest multiple of 16 with CH + kp - 1 <= 4096).
// In shared memory it holds
//   s_loc[u] = s[m0 - (kp-1) + u]      u < 4096 + kp   (zero off-row)
//   r_loc[v] = r[m0 + v]               v < 4096 + kp + 32 (zero past n + k - 1)
// and either loads r (conv_adjoint) or computes it on chip for the 4096
// positions the chunk needs (conv_gradient; the kp - 1 overlap with the next
// chunk is recomputed there).  The per-thread grad_h partials reuse the
// s_loc space once the products are done.  Then
//   grad_s[m0 + m] = sum_i h[i] r_loc[m + i]                        (m < CH)
//   part[j]        = sum_{m < CH} s_loc[m + kp - 1] r_loc[m + j]     (j < k)
// Every product loop is a 16-output sliding window: a thread keeps 16
// accumulators, 16 taps and a 16-entry circular register buffer, so 16 taps
// cost 16 window loads, four vector tap loads and 256 FMAs.  Shared arrays
// carry one pad word per 16 (index p -> p + p/16): the 16-word lane stride of
// the windows then lands on 32 distinct banks, and with 16-aligned windows
// all load offsets inside a 16-tap step are compile-time constants.
#include <cstdlib>

#include "adjwt_internal.h"
#include "device_common.cuh"

namespace adjwt {

constexpr int kFusedMaxK = 1024;

namespace {

constexpr int kNT = 256;
constexpr int kW = 16;           // outputs per thread (window length)
constexpr int kSpan = kNT * kW;  // 4096 positions of r per chunk

__host__ __device__ __forceinline__ int padx(int p) { return p + (p >> 4); }
__host__ __device__ inline int pad16(int k) { return (k + 15) & ~15; }
__host__ __device__ inline int chunk_of(int k) { return ((kSpan - pad16(k) + 1) / 16) * 16; }

struct FusedGeo {
  int kp, ch, s_len, r_len, groups, tpg;
  __host__ __device__ explicit FusedGeo(int k) {
    kp = pad16(k);
    ch = chunk_of(k);
    s_len = kSpan + kp;
    r_len = kSpan + kp + 32;
    groups = kp / 16;
    tpg = kNT / groups;
  }
  __host__ __device__ int s_words() const { return padx(s_len) + 4; }
  __host__ __device__ int r_words() const { return padx(r_len) + 4; }
  __host__ __device__ int red_words() const { return kp * (tpg + 1); }
};

// 16 taps h[i0 .. i0+15] into registers (the tap array is 16-aligned)
__device__ __forceinline__ void load_taps16(const float* h_sm, int i0, float (&hv)[kW]) {
  const float4* p = reinterpret_cast<const float4*>(h_sm + i0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 v = p[q];
    hv[4 * q] = v.x;
    hv[4 * q + 1] = v.y;
    hv[4 * q + 2] = v.z;
    hv[4 * q + 3] = v.w;
  }
}

template <bool FUSED>
__global__ void __launch_bounds__(kNT, 4) k_conv_grad(int64_t n, int K, const float* __restrict__ s,
                                                    const float* __restrict__ h, const float* __restrict__ x,
                                                    const float* __restrict__ r_in, float* __restrict__ r_out,
                                                    float* __restrict__ grad_s, float* __restrict__ part_h,
                                                    int nchunks) {
  pdl_entry();
  extern __shared__ __align__(16) float sm[];
  const FusedGeo g(K);
  const int kp = g.kp;
  float* h_sm = sm;                      // kp floats (16-aligned)
  float* s_loc = h_sm + kp;
  float* r_loc = s_loc + g.s_words();
  float* red = s_loc;  // grad_h partials, written once every thread is done with s_loc
  const int b = blockIdx.y;
  const int64_t m0 = (int64_t)blockIdx.x * g.ch;
  const int64_t nr = n + K - 1;
  const int tid = threadIdx.x;
  const float* srow = s + (size_t)b * n;

  const int base = tid * kW;  // this thread's 16-aligned window start
  // x for this thread's 16 residuals, requested before the staging below so
  // that its latency overlaps the staging
  float xv[kW];
  if (FUSED) {
    const float* xrow = x ? x + (size_t)b * nr : nullptr;
#pragma unroll
    for (int o = 0; o < kW; ++o) {
      const int64_t q = m0 + base + o;
      xv[o] = (xrow && q < nr) ? __ldg(xrow + q) : 0.0f;
    }
  }

  // ---- stage h (zero-padded), s, and r (adjoint only); 16 loads in flight per thread
  for (int i = tid; i < kp; i += kNT) h_sm[i] = (h && i < K) ? __ldg(h + (size_t)b * K + i) : 0.0f;
  for (int u0 = tid; u0 < g.s_len; u0 += kW * kNT) {
    float v[kW];
#pragma unroll
    for (int j = 0; j < kW; ++j) {
      const int u = u0 + j * kNT;
      const int64_t q = m0 - (kp - 1) + u;
      v[j] = (u < g.s_len && q >= 0 && q < n) ? __ldg(srow + q) : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < kW; ++j) {
      const int u = u0 + j * kNT;
      if (u < g.s_len) s_loc[padx(u)] = v[j];
    }
  }
  if (!FUSED) {
    const float* rrow = r_in + (size_t)b * nr;
    for (int v0 = tid; v0 < g.r_len; v0 += kW * kNT) {
      float v[kW];
#pragma unroll
      for (int j = 0; j < kW; ++j) {
        const int vv = v0 + j * kNT;
        const int64_t q = m0 + vv;
        v[j] = (vv < g.r_len && vv < g.ch + kp - 1 && q < nr) ? __ldg(rrow + q) : 0.0f;
      }
#pragma unroll
      for (int j = 0; j < kW; ++j) {
        const int vv = v0 + j * kNT;
        if (vv < g.r_len) r_loc[padx(vv)] = v[j];
      }
    }
  } else {
    for (int v = kSpan + tid; v < g.r_len; v += kNT) r_loc[padx(v)] = 0.0f;
  }
  __syncthreads();

  // ---- r = h * s - x on [m0, m0 + 4096) ------------------------------------
  if (FUSED) {
    // S[z] = s_loc[z + kp - 1]; r_loc[base + o] = sum_i h[i] S[base + o - i]
    float acc[kW], buf[kW], hv[kW];
#pragma unroll
    for (int o = 0; o < kW; ++o) acc[o] = 0.0f;
    // slot z holds S[base + z - 16*t] for the current 16-tap step t; start: S[base + 0..15]
    // S[base + o] = s_loc[base + kp - 1 + o]: offset 15 of block (base+kp-16)/16, then the next block
    {
      const float* blk = s_loc + padx(base + kp - 16);  // 16 words of block (base+kp-16)/16, then a pad
      buf[0] = blk[15];
#pragma unroll
      for (int o = 1; o < kW; ++o) buf[o] = blk[17 + o - 1];
    }
    for (int i0 = 0; i0 < kp; i0 += kW) {
      load_taps16(h_sm, i0, hv);
      // S[base - i] for i = i0 + ii, ii >= 1 (or i0 > 0): s_loc index base + kp - 1 - i0 - ii
      const float* blk = s_loc + padx(base + kp - 16 - i0);  // block holding indices base+kp-16-i0 .. +15
#pragma unroll
      for (int ii = 0; ii < kW; ++ii) {
        if (ii > 0) {
          buf[(kW - ii) & (kW - 1)] = blk[15 - ii];
        } else if (i0 > 0) {
          buf[0] = blk[15];
        }
#pragma unroll
        for (int o = 0; o < kW; ++o) acc[o] = fmaf(hv[ii], buf[(o - ii) & (kW - 1)], acc[o]);
      }
    }
    float* rrow = r_out ? r_out + (size_t)b * nr : nullptr;
    const int own = g.ch + (blockIdx.x == nchunks - 1 ? K - 1 : 0);
#pragma unroll
    for (int o = 0; o < kW; ++o) {
      const int64_t q = m0 + base + o;
      float v = 0.0f;
      if (q < nr) {
        v = acc[o] - xv[o];
        if (rrow && base + o < own) rrow[q] = v;
      }
      r_loc[padx(base + o)] = v;
    }
    __syncthreads();
  }

  // ---- grad_s[m0 + m] = sum_i h[i] r_loc[m + i] ------------------------------
  if (grad_s && base < g.ch) {
    float acc[kW], buf[kW], hv[kW];
    {
      const float* blk = r_loc + padx(base);
#pragma unroll
      for (int o = 0; o < kW; ++o) {
        acc[o] = 0.0f;
        buf[o] = blk[o];  // slot z: r_loc[base + z]
      }
    }
    for (int i0 = 0; i0 < kp; i0 += kW) {
      load_taps16(h_sm, i0, hv);
      // new value at tap i = i0 + ii (ii >= 1 or i0 > 0): r_loc[base + i + 15]
      const float* nxt = r_loc + padx(base + i0 + 16);  // block (base+i0)/16 + 1
#pragma unroll
      for (int ii = 0; ii < kW; ++ii) {
        if (ii > 0) {
          buf[(ii + kW - 1) & (kW - 1)] = nxt[ii - 1];
        } else if (i0 > 0) {
          buf[kW - 1] = nxt[-2];  // r_loc[base + i0 + 15]: offset 15 of the previous block
        }
#pragma unroll
        for (int o = 0; o < kW; ++o) acc[o] = fmaf(hv[ii], buf[(o + ii) & (kW - 1)], acc[o]);
      }
    }
    float* out = grad_s + (size_t)b * n;
#pragma unroll
    for (int o = 0; o < kW; ++o) {
      const int64_t m = m0 + base + o;
      if (base + o < g.ch && m < n) out[m] = acc[o];
    }
  }

  // ---- partial grad_h over this chunk ------------------------------------
  if (part_h) {
    const int grp = tid / g.tpg, lane_in_grp = tid - grp * g.tpg;
    float acc[kW];
#pragma unroll
    for (int o = 0; o < kW; ++o) acc[o] = 0.0f;
    if (grp < g.groups) {
      const int j0 = grp * kW;
      const int nseg = g.ch / 16;
      for (int seg = lane_in_grp; seg < nseg; seg += g.tpg) {
        const int mb = seg * 16;
        float buf[kW];
        const float* r0 = r_loc + padx(mb + j0);       // r_loc[mb + j0 + z], z < 16
        const float* r1 = r_loc + padx(mb + j0 + 16);  // next block
        const float* sv = s_loc + padx(mb + kp - 16);  // s_loc[mb + kp - 1 + mm]: offset 15, then next block
#pragma unroll
        for (int o = 0; o < kW; ++o) buf[o] = r0[o];
#pragma unroll
        for (int mm = 0; mm < kW; ++mm) {
          if (mm > 0) buf[(mm + kW - 1) & (kW - 1)] = r1[mm - 1];
          const float sval = mm == 0 ? sv[15] : sv[17 + mm - 1];
#pragma unroll
          for (int o = 0; o < kW; ++o) acc[o] = fmaf(sval, buf[(o + mm) & (kW - 1)], acc[o]);
        }
      }
    }
    __syncthreads();  // red aliases s_loc
    if (grp < g.groups) {
      const int j0 = grp * kW;
#pragma unroll
      for (int o = 0; o < kW; ++o) red[(j0 + o) * (g.tpg + 1) + lane_in_grp] = acc[o];
    }
    __syncthreads();
    float* dst = part_h + ((size_t)b * nchunks + blockIdx.x) * K;
    for (int j = tid; j < K; j += kNT) {
      const float* rr = red + j * (g.tpg + 1);
      float t = 0.0f;
      for (int l = 0; l < g.tpg; ++l) t += rr[l];
      dst[j] = t;
    }
  }
}

size_t fused_smem(int k) {
  const FusedGeo g(k);
  return (size_t)(g.kp + g.s_words() + g.r_words()) * sizeof(float);  // red_words() <= s_words()
}

}  // namespace

int64_t conv_fused_nchunks(int64_t n, int k) {
  const int ch = chunk_of(k);
  return (n + ch - 1) / ch;
}

bool conv_fused_supported(int k) { return k >= 1 && k <= kFusedMaxK; }

// r_in != null: conv_adjoint (r given).  r_in == null: r = h * s - x computed
// in the kernel (x may be null), written to r_out if non-null.
int launch_conv_fused(int batch, int64_t n, int k, const float* s, const float* h, const float* x, const float* r_in,
                      float* r_out, float* grad_h, float* grad_s, float* partials, cudaStream_t st) {
  if (batch == 0) return ADJWT_OK;
  static const bool force_fp32 = [] {
    const char* e = std::getenv("ADJWT_CONV_FP32");
    return e && std::atoi(e) != 0;
  }();
  if (conv_tc_supported(k) && !force_fp32)
    return launch_conv_tc(batch, n, k, s, h, x, r_in, r_out, grad_h, grad_s, partials, st);
  const int64_t nch = conv_fused_nchunks(n, k);
  if (nch > 0x7fffffff) return fail(ADJWT_ERR_SHAPE, "conv: n too large");
  const size_t smem = fused_smem(k);
  dim3 grid(static_cast<unsigned>(nch), static_cast<unsigned>(batch));
  float* part = grad_h ? partials : nullptr;
  if (r_in) {
    ADJWT_CUDA_CHECK(set_smem(k_conv_grad<false>, smem));
    ADJWT_TRACED("conv_adjoint", 0, st,
                 pdl_launch(k_conv_grad<false>, grid, kNT, smem, st, n, k, s, h, nullptr, r_in, nullptr, grad_s, part,
                                                             static_cast<int>(nch)));
  } else {
    ADJWT_CUDA_CHECK(set_smem(k_conv_grad<true>, smem));
    ADJWT_TRACED("conv_gradient", 0, st,
                 pdl_launch(k_conv_grad<true>, grid, kNT, smem, st, n, k, s, h, x, nullptr, r_out, grad_s, part,
                                                            static_cast<int>(nch)));
  }
  ADJWT_CUDA_CHECK(cudaGetLastError());
  if (grad_h) {
    const int64_t total = (int64_t)batch * k;
    const unsigned nb = static_cast<unsigned>((total + 255) / 256);
    ADJWT_TRACED("conv_reduce", 0, st, conv_reduce(nb, k, static_cast<int>(nch), partials, grad_h, total, st));
    ADJWT_CUDA_CHECK(cudaGetLastError());
  }
  return ADJWT_OK;
}

}  // namespace adjwt
