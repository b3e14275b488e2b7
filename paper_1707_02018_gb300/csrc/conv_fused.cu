// Register-blocked channel gradient (Sec. II, Eq. 5) for k <= kFusedMaxK.
//
// One CTA owns a chunk of CH samples of one row (CH = the largest multiple of
// 32 with CH + k - 1 <= 4096).  In shared memory it holds
//   s_loc[u] = s[m0 - (k-1) + u]      u < CH + 2k - 2   (zero off-row)
//   r_loc[v] = r[m0 + v]              v < 4096 + slack  (zero past n + k - 1)
// and either loads r (conv_adjoint) or computes it, r = h * s - x, for the
// 4096 positions the chunk needs (conv_gradient; the k - 1 overlap with the
// next chunk is recomputed there).  Then
//   grad_s[m0 + m] = sum_i h[i] r_loc[m + i]                 (m < CH)
//   part[j]        = sum_{m < CH} s_loc[m + k - 1] r_loc[m + j]   (j < k)
// Every product loop is a 16-output sliding window: a thread keeps 16
// accumulators and a 16-entry circular register buffer, so each tap costs one
// window load, one broadcast operand load and 16 FMAs.  Shared arrays use one
// pad word per 16 (index p -> p + p/16), which puts the 16-word lane stride of
// every window on 32 distinct banks.
#include "adjwt_internal.h"
#include "device_common.cuh"

namespace adjwt {

constexpr int kFusedMaxK = 1024;

namespace {

constexpr int kNT = 256;
constexpr int kW = 16;      // outputs per thread (window length)
constexpr int kSpan = kNT * kW;  // 4096 positions of r per chunk
constexpr int kSeg = 16;    // samples per grad_h segment

__host__ __device__ __forceinline__ int padx(int p) { return p + (p >> 4); }

__host__ __device__ inline int chunk_of(int k) { return ((kSpan - k + 1) / kSeg) * kSeg; }

struct FusedGeo {
  int k, ch, s_len, r_len, groups, tpg;
  __host__ __device__ FusedGeo(int k_) : k(k_) {
    ch = chunk_of(k);
    s_len = kSpan + k;              // the r windows of the last threads reach s[m0 + 4095]
    r_len = kSpan + k + kW + kSeg;  // windows may run past the last real sample
    groups = (k + kW - 1) / kW;
    tpg = kNT / groups;
  }
  __host__ __device__ int s_words() const { return padx(s_len) + 1; }
  __host__ __device__ int r_words() const { return padx(r_len) + 1; }
  __host__ __device__ int red_words() const { return tpg * groups * kW; }
};

template <bool FUSED>
__global__ void __launch_bounds__(kNT) k_conv_grad(int64_t n, int K, const float* __restrict__ s,
                                                    const float* __restrict__ h, const float* __restrict__ x,
                                                    const float* __restrict__ r_in, float* __restrict__ r_out,
                                                    float* __restrict__ grad_s, float* __restrict__ part_h,
                                                    int nchunks) {
  extern __shared__ float sm[];
  const FusedGeo g(K);
  float* s_loc = sm;
  float* r_loc = s_loc + g.s_words();
  float* h_sm = r_loc + g.r_words();
  float* red = h_sm + K;
  const int b = blockIdx.y;
  const int64_t m0 = (int64_t)blockIdx.x * g.ch;
  const int64_t nr = n + K - 1;
  const int tid = threadIdx.x;
  const float* srow = s + (size_t)b * n;

  // ---- stage s (and h) ---------------------------------------------------
  for (int u = tid; u < g.s_len; u += kNT) {
    const int64_t q = m0 - (K - 1) + u;
    s_loc[padx(u)] = (q >= 0 && q < n) ? __ldg(srow + q) : 0.0f;
  }
  if (h)
    for (int i = tid; i < K; i += kNT) h_sm[i] = __ldg(h + (size_t)b * K + i);
  if (!FUSED) {
    const float* rrow = r_in + (size_t)b * nr;
    for (int v = tid; v < g.r_len; v += kNT) {
      const int64_t q = m0 + v;
      r_loc[padx(v)] = (v < g.ch + K - 1 && q < nr) ? __ldg(rrow + q) : 0.0f;
    }
  } else {
    for (int v = kSpan + tid; v < g.r_len; v += kNT) r_loc[padx(v)] = 0.0f;
  }
  __syncthreads();

  // ---- r = h * s - x on [m0, m0 + 4096) ------------------------------------
  if (FUSED) {
    const int base = tid * kW;        // local r index of this thread's first output
    const int sb = base + K - 1;      // s_loc index of s[m0 + base]
    float acc[kW], buf[kW];
#pragma unroll
    for (int o = 0; o < kW; ++o) {
      acc[o] = 0.0f;
      buf[o] = s_loc[padx(sb + o)];   // slot z holds S[base + z], S[z] = s_loc[z + K - 1]
    }
    for (int i0 = 0; i0 < K; i0 += kW) {
#pragma unroll
      for (int ii = 0; ii < kW; ++ii) {
        const int i = i0 + ii;
        if (i < K) {
          if (i > 0) buf[(kW - ii) & (kW - 1)] = s_loc[padx(sb - i)];
          const float hv = h_sm[i];
#pragma unroll
          for (int o = 0; o < kW; ++o) acc[o] = fmaf(hv, buf[(o - ii) & (kW - 1)], acc[o]);
        }
      }
    }
    const float* xrow = x ? x + (size_t)b * nr : nullptr;
#pragma unroll
    for (int o = 0; o < kW; ++o) {
      const int64_t q = m0 + base + o;
      float v = 0.0f;
      if (q < nr) {
        v = acc[o];
        if (xrow) v -= __ldg(xrow + q);
        if (r_out && base + o < g.ch + (blockIdx.x == nchunks - 1 ? K - 1 : 0)) r_out[(size_t)b * nr + q] = v;
      }
      r_loc[padx(base + o)] = v;
    }
    __syncthreads();
  }

  // ---- grad_s[m0 + m] = sum_i h[i] r_loc[m + i] ------------------------------
  if (grad_s) {
    const int base = tid * kW;
    if (base < g.ch) {
      float acc[kW], buf[kW];
#pragma unroll
      for (int o = 0; o < kW; ++o) {
        acc[o] = 0.0f;
        buf[o] = r_loc[padx(base + o)];  // slot z holds r_loc[base + z] (mod kW)
      }
      for (int i0 = 0; i0 < K; i0 += kW) {
#pragma unroll
        for (int ii = 0; ii < kW; ++ii) {
          const int i = i0 + ii;
          if (i < K) {
            if (i > 0) buf[(ii + kW - 1) & (kW - 1)] = r_loc[padx(base + i + kW - 1)];
            const float hv = h_sm[i];
#pragma unroll
            for (int o = 0; o < kW; ++o) acc[o] = fmaf(hv, buf[(o + ii) & (kW - 1)], acc[o]);
          }
        }
      }
      float* out = grad_s + (size_t)b * n;
#pragma unroll
      for (int o = 0; o < kW; ++o) {
        const int64_t m = m0 + base + o;
        if (base + o < g.ch && m < n) out[m] = acc[o];
      }
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
      const int nseg = g.ch / kSeg;
      for (int seg = lane_in_grp; seg < nseg; seg += g.tpg) {
        const int mb = seg * kSeg;
        float buf[kW];
#pragma unroll
        for (int o = 0; o < kW; ++o) buf[o] = r_loc[padx(mb + j0 + o)];  // slot z: r_loc[mb + j0 + z]
#pragma unroll
        for (int mm = 0; mm < kSeg; ++mm) {
          if (mm > 0) buf[(mm + kW - 1) & (kW - 1)] = r_loc[padx(mb + mm + j0 + kW - 1)];
          const float sv = s_loc[padx(mb + mm + K - 1)];
#pragma unroll
          for (int o = 0; o < kW; ++o) acc[o] = fmaf(sv, buf[(o + mm) & (kW - 1)], acc[o]);
        }
      }
    }
    if (grp < g.groups) {
#pragma unroll
      for (int o = 0; o < kW; ++o) red[lane_in_grp * (g.groups * kW) + grp * kW + o] = acc[o];
    }
    __syncthreads();
    float* dst = part_h + ((size_t)b * nchunks + blockIdx.x) * K;
    for (int j = tid; j < K; j += kNT) {
      float t = 0.0f;
      for (int l = 0; l < g.tpg; ++l) t += red[l * (g.groups * kW) + j];
      dst[j] = t;
    }
  }
}

size_t fused_smem(int k) {
  const FusedGeo g(k);
  return (size_t)(g.s_words() + g.r_words() + k + g.red_words()) * sizeof(float);
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
  const int64_t nch = conv_fused_nchunks(n, k);
  if (nch > 0x7fffffff) return fail(ADJWT_ERR_SHAPE, "conv: n too large");
  const size_t smem = fused_smem(k);
  dim3 grid(static_cast<unsigned>(nch), static_cast<unsigned>(batch));
  float* part = grad_h ? partials : nullptr;
  if (r_in) {
    ADJWT_CUDA_CHECK(cudaFuncSetAttribute(k_conv_grad<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ADJWT_TRACED("conv_adjoint", 0, st,
                 k_conv_grad<false><<<grid, kNT, smem, st>>>(n, k, s, h, nullptr, r_in, nullptr, grad_s, part,
                                                             static_cast<int>(nch)));
  } else {
    ADJWT_CUDA_CHECK(cudaFuncSetAttribute(k_conv_grad<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ADJWT_TRACED("conv_gradient", 0, st,
                 k_conv_grad<true><<<grid, kNT, smem, st>>>(n, k, s, h, x, nullptr, r_out, grad_s, part,
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
