// Multi-level 2D wavelet kernels: W (reconstruction), W^* (exact adjoint,
// Eq. 4) and W^dagger (analysis), one launch per level.
//
// Analysis direction (W^* and W^dagger), one level, per axis:
//     out[k] = sum_i f[i] z[2k+1-i],   z[e] = w(e) * y[src(e)]
// with e the coordinate of the length N + 2L' extended signal, src(e) the
// extension map of Sec. I-A (zero / half-point symmetric / periodic) and
// w = 1/c for W^* (the weighted extension (E^dagger)^*, Eq. 2) or 1 for
// W^dagger; f are the dual analysis filters (reversed synthesis filters,
// Eq. 3 / Eq. 4) for W^* and the analysis filters for W^dagger.  The
// extension is applied in the load path: each CTA gathers its extended tile
// once into shared memory, then runs the column pass and the row pass there.
//
// Reconstruction W = E^dagger S, per axis:
//     Ysyn(x) = sum_k a_lo[k] g_lo[x+2L'-2k-1] + a_hi[k] g_hi[x+2L'-2k-1]
//     out[t]  = (1/c[t]) * sum_{x : ext(x) = t} Ysyn(x),  x in [-L', N+L')
// (x is the extended coordinate shifted by L').  The fold E^dagger is a
// gather: a CTA computes Ysyn over its own rows plus, at the image border,
// the L' mirrored rows (symmetric case), so no atomics are needed.  The
// periodic extension's far copies and tiny images (N <= 2L') go through a
// per-pixel gather kernel.
#include <algorithm>
#include <type_traits>

#include "adjwt_internal.h"
#include "device_common.cuh"

namespace adjwt {
namespace {

constexpr int kTile = kSynthTile;
constexpr int kThreads = 256;

struct AnaArgs {
  const float* in;
  int in_pitch;
  int Nr, Nc, nr, nc, mode;
  const float* winv_r;
  const float* winv_c;
  float* dst[4];  // plain destinations (LL, LH, HL, HH)
  float* px[4];   // prox state buffers (non-null => prox band)
  float* py[4];
  int out_pitch;
  float step, thresh, beta;
  double* l1;     // per-CTA partials (null = skip)
  float flo[kMaxTaps], fhi[kMaxTaps];
};

template <int L>
__global__ void __launch_bounds__(kThreads) k_analysis(const AnaArgs a) {
  constexpr int Lp = L - 1;
  constexpr int E = 2 * kTile + L - 2;  // extended samples feeding one tile
  constexpr int EP = E + 1;
  __shared__ float T[E][EP];
  __shared__ float V[2][kTile][EP];
  __shared__ int s_src[2][E];
  __shared__ float s_w[2][E];
  __shared__ double red[kThreads / 32];

  const int k0 = blockIdx.y * kTile, l0 = blockIdx.x * kTile;
  const int tid = threadIdx.x;

  for (int i = tid; i < 2 * E; i += kThreads) {
    const int axis = i / E, el = i - axis * E;
    const int e = (axis == 0 ? 2 * k0 : 2 * l0) + 1 - Lp + el;
    const int N = axis == 0 ? a.Nr : a.Nc;
    int s;
    if (a.mode == 3) {
      s = pos_mod(e, N);
    } else {
      s = (e >= 0 && e < N + 2 * Lp) ? ext_src(e - Lp, N, a.mode) : -1;
    }
    const float* winv = axis == 0 ? a.winv_r : a.winv_c;
    s_src[axis][el] = s;
    s_w[axis][el] = (s >= 0 && winv) ? __ldg(winv + s) : 1.0f;
  }
  __syncthreads();

  for (int i = tid; i < E * E; i += kThreads) {
    const int er = i / E, ec = i - er * E;
    const int sr = s_src[0][er], sc = s_src[1][ec];
    float v = 0.0f;
    if (sr >= 0 && sc >= 0) v = s_w[0][er] * s_w[1][ec] * __ldg(a.in + (size_t)sr * a.in_pitch + sc);
    T[er][ec] = v;
  }
  __syncthreads();

  // column pass (filter along rows, keep odd samples)
  for (int i = tid; i < kTile * E; i += kThreads) {
    const int kk = i / E, ec = i - kk * E;
    float lo = 0.0f, hi = 0.0f;
#pragma unroll
    for (int t = 0; t < L; ++t) {
      const float v = T[2 * kk + Lp - t][ec];
      lo = fmaf(a.flo[t], v, lo);
      hi = fmaf(a.fhi[t], v, hi);
    }
    V[0][kk][ec] = lo;
    V[1][kk][ec] = hi;
  }
  __syncthreads();

  // row pass + store / prox epilogue
  double l1 = 0.0;
  for (int i = tid; i < kTile * kTile; i += kThreads) {
    const int kk = i / kTile, ll = i - kk * kTile;
    const int k = k0 + kk, l = l0 + ll;
    if (k >= a.nr || l >= a.out_pitch) continue;
    const bool inside = l < a.nc;
    float res[4];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      float lo = 0.0f, hi = 0.0f;
#pragma unroll
      for (int t = 0; t < L; ++t) {
        const float v = V[f][kk][2 * ll + Lp - t];
        lo = fmaf(a.flo[t], v, lo);
        hi = fmaf(a.fhi[t], v, hi);
      }
      res[f] = lo;      // band (f, lo): f = 0 -> LL, f = 1 -> LH
      res[2 + f] = hi;  // band (f, hi): f = 0 -> HL, f = 1 -> HH
    }
    const size_t idx = (size_t)k * a.out_pitch + l;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      if (a.px[b]) {
        float xn = 0.0f, yn = 0.0f;
        if (inside) {
          const float v = a.py[b][idx] - a.step * res[b];
          const float mag = fabsf(v) - a.thresh;
          xn = mag > 0.0f ? copysignf(mag, v) : 0.0f;
          const float xo = a.px[b][idx];
          yn = fmaf(a.beta, xn - xo, xn);
          l1 += fabs((double)xn);
        }
        a.px[b][idx] = xn;
        a.py[b][idx] = yn;
      } else if (a.dst[b]) {
        a.dst[b][idx] = inside ? res[b] : 0.0f;
      }
    }
  }
  if (a.l1) {
    const double tot = block_sum<kThreads>(l1, red);
    if (tid == 0) a.l1[blockIdx.y * gridDim.x + blockIdx.x] = tot;
  }
}

struct SynArgs {
  const float* band[4];  // LL, LH, HL, HH of level j
  int band_pitch;
  float* out;
  int out_pitch;
  int Nr, Nc, nr, nc, mode;
  const float* winv_r;
  const float* winv_c;
  float g[2][kMaxTaps];  // synthesis filters lo / hi
};

template <int L>
__global__ void __launch_bounds__(kThreads) k_synthesis(const SynArgs a) {
  constexpr int Lp = L - 1;
  constexpr int XM = kTile + 2 * Lp;       // virtual rows a tile may need
  constexpr int KM = (XM + L) / 2 + 2;     // coefficient rows feeding them
  constexpr int KP = KM + 1;
  __shared__ float C[4][KM][KP];
  __shared__ float H[2][XM][KP];           // reused as Y[kTile][XM + 1]
  __shared__ float G[2][kTile][KP];
  float(*Y)[XM + 1] = reinterpret_cast<float(*)[XM + 1]>(&H[0][0][0]);
  static_assert(kTile * (XM + 1) <= 2 * XM * KP, "Y must fit in H");

  const int tid = threadIdx.x;
  const int t0r = blockIdx.y * kTile, t0c = blockIdx.x * kTile;
  const bool sym = a.mode == 1;
  // filter index m = x + off - 2k - 1: the extended modes carry the L' shift of
  // the extension on top of the bank's delay L'; the circular mode has none
  const int off = a.mode == 3 ? Lp : 2 * Lp;
  int xa[2], xb[2], ka[2], nk[2];
  {
    const int t0[2] = {t0r, t0c};
    const int N[2] = {a.Nr, a.Nc};
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
      xa[ax] = (sym && t0[ax] < Lp) ? -Lp : t0[ax];
      xb[ax] = (sym && t0[ax] + kTile > N[ax] - Lp) ? N[ax] + Lp : t0[ax] + kTile;
      ka[ax] = floor_div(xa[ax] + off - Lp, 2);
      nk[ax] = floor_div(xb[ax] + off - 2, 2) - ka[ax] + 1;
    }
  }
  const int nx_r = xb[0] - xa[0], nx_c = xb[1] - xa[1];

  // coefficient tiles of the four bands (periodic wrap for PER, zeros outside otherwise)
  for (int i = tid; i < 4 * nk[0] * nk[1]; i += kThreads) {
    const int b = i / (nk[0] * nk[1]);
    const int rem = i - b * nk[0] * nk[1];
    const int kk = rem / nk[1], ll = rem - kk * nk[1];
    int k = ka[0] + kk, l = ka[1] + ll;
    float v = 0.0f;
    if (a.mode == 3) {
      k = pos_mod(k, a.nr);
      l = pos_mod(l, a.nc);
      v = __ldg(a.band[b] + (size_t)k * a.band_pitch + l);
    } else if (k >= 0 && k < a.nr && l >= 0 && l < a.nc) {
      v = __ldg(a.band[b] + (size_t)k * a.band_pitch + l);
    }
    C[b][kk][ll] = v;
  }
  __syncthreads();

  // column pass: H[hb][x][l] = sum_va sum_q C[va + 2 hb][k][l] g_va[m]
  for (int i = tid; i < 2 * nx_r * nk[1]; i += kThreads) {
    const int hb = i / (nx_r * nk[1]);
    const int rem = i - hb * nx_r * nk[1];
    const int xx = rem / nk[1], ll = rem - xx * nk[1];
    const int x = xa[0] + xx;
    const int m0 = (x + off - 1) & 1;
    float acc = 0.0f;
#pragma unroll
    for (int q = 0; q < L / 2; ++q) {
      const int m = m0 + 2 * q;
      const int kk = ((x + off - 1 - m) >> 1) - ka[0];
      acc = fmaf(C[2 * hb][kk][ll], a.g[0][m], acc);
      acc = fmaf(C[2 * hb + 1][kk][ll], a.g[1][m], acc);
    }
    H[hb][xx][ll] = acc;
  }
  __syncthreads();

  // fold rows (E^dagger along the vertical axis)
  for (int i = tid; i < 2 * kTile * nk[1]; i += kThreads) {
    const int hb = i / (kTile * nk[1]);
    const int rem = i - hb * kTile * nk[1];
    const int tt = rem / nk[1], ll = rem - tt * nk[1];
    const int t = t0r + tt;
    float v = 0.0f;
    if (t < a.Nr) {
      v = H[hb][t - xa[0]][ll];
      if (sym) {
        if (t < Lp) v += H[hb][-1 - t - xa[0]][ll];
        if (t >= a.Nr - Lp) v += H[hb][2 * a.Nr - 1 - t - xa[0]][ll];
      }
      if (a.winv_r) v *= __ldg(a.winv_r + t);
    }
    G[hb][tt][ll] = v;
  }
  __syncthreads();

  // row pass: Y[t][x] = sum_hb sum_q G[hb][t][l] g_hb[m]
  for (int i = tid; i < kTile * nx_c; i += kThreads) {
    const int tt = i / nx_c, xx = i - tt * nx_c;
    const int x = xa[1] + xx;
    const int m0 = (x + off - 1) & 1;
    float acc = 0.0f;
#pragma unroll
    for (int q = 0; q < L / 2; ++q) {
      const int m = m0 + 2 * q;
      const int ll = ((x + off - 1 - m) >> 1) - ka[1];
      acc = fmaf(G[0][tt][ll], a.g[0][m], acc);
      acc = fmaf(G[1][tt][ll], a.g[1][m], acc);
    }
    Y[tt][xx] = acc;
  }
  __syncthreads();

  // fold columns and store
  const bool ppd = a.mode == 2;
  for (int i = tid; i < kTile * kTile; i += kThreads) {
    const int tt = i / kTile, cc = i - tt * kTile;
    const int tr = t0r + tt, tc = t0c + cc;
    if (tr >= a.Nr || tc >= a.Nc) continue;
    float v = Y[tt][tc - xa[1]];
    if (sym) {
      if (tc < Lp) v += Y[tt][-1 - tc - xa[1]];
      if (tc >= a.Nc - Lp) v += Y[tt][2 * a.Nc - 1 - tc - xa[1]];
    }
    if (ppd) {  // pixels with periodic far copies belong to the border kernel
      if (tr < Lp || tr >= a.Nr - Lp || tc < Lp || tc >= a.Nc - Lp) continue;
    }
    if (a.winv_c) v *= __ldg(a.winv_c + tc);
    a.out[(size_t)tr * a.out_pitch + tc] = v;
  }
}

// Per-pixel gather of W = E^dagger S for pixels with copies anywhere in the
// extended domain (periodic-extension borders, tiny images).
template <int L>
__global__ void __launch_bounds__(kThreads) k_synthesis_gather(const SynArgs a, int border_only, int64_t count) {
  constexpr int Lp = L - 1;
  const int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (idx >= count) return;
  int tr, tc;
  if (!border_only) {
    tr = (int)(idx / a.Nc);
    tc = (int)(idx - (int64_t)tr * a.Nc);
  } else {
    const int64_t top = (int64_t)2 * Lp * a.Nc;
    if (idx < top) {
      const int row = (int)(idx / a.Nc);
      tr = row < Lp ? row : a.Nr - 2 * Lp + row;
      tc = (int)(idx - (int64_t)row * a.Nc);
    } else {
      const int64_t j = idx - top;
      tr = Lp + (int)(j / (2 * Lp));
      const int cc = (int)(j - (int64_t)(tr - Lp) * 2 * Lp);
      tc = cc < Lp ? cc : a.Nc - 2 * Lp + cc;
    }
  }
  // copies of t in [-L', N + L'): translation class (and mirror class for SYM)
  const int N[2] = {a.Nr, a.Nc};
  const int t[2] = {tr, tc};
  int xs[2][2 * kMaxTaps];
  int nx[2] = {0, 0};
#pragma unroll
  for (int ax = 0; ax < 2; ++ax) {
    const int P = a.mode == 1 ? 2 * N[ax] : (a.mode == 0 ? 0 : N[ax]);
    if (P == 0) {
      xs[ax][nx[ax]++] = t[ax];
      continue;
    }
    const int starts[2] = {t[ax], -1 - t[ax]};
    const int nclass = a.mode == 1 ? 2 : 1;
    for (int c = 0; c < nclass; ++c) {
      int x = starts[c] - P * floor_div(starts[c] + Lp, P);
      for (; x < N[ax] + Lp && nx[ax] < 2 * kMaxTaps; x += P) xs[ax][nx[ax]++] = x;
    }
  }
  float acc = 0.0f;
  for (int ir = 0; ir < nx[0]; ++ir) {
    const int xr = xs[0][ir];
    for (int ic = 0; ic < nx[1]; ++ic) {
      const int xc = xs[1][ic];
      for (int qr = 0; qr < L / 2; ++qr) {
        const int mr = ((xr + 1) & 1) + 2 * qr;
        const int k = (xr + 2 * Lp - 1 - mr) >> 1;
        if (k < 0 || k >= a.nr) continue;
        for (int qc = 0; qc < L / 2; ++qc) {
          const int mc = ((xc + 1) & 1) + 2 * qc;
          const int l = (xc + 2 * Lp - 1 - mc) >> 1;
          if (l < 0 || l >= a.nc) continue;
          const size_t o = (size_t)k * a.band_pitch + l;
#pragma unroll
          for (int va = 0; va < 2; ++va)
#pragma unroll
            for (int hb = 0; hb < 2; ++hb)
              acc = fmaf(__ldg(a.band[va + 2 * hb] + o), a.g[va][mr] * a.g[hb][mc], acc);
        }
      }
    }
  }
  if (a.winv_r) acc *= __ldg(a.winv_r + tr);
  if (a.winv_c) acc *= __ldg(a.winv_c + tc);
  a.out[(size_t)tr * a.out_pitch + tc] = acc;
}

template <typename Fn>
int dispatch_L(int L, Fn&& fn) {
  switch (L) {
    case 2: return fn(std::integral_constant<int, 2>());
    case 4: return fn(std::integral_constant<int, 4>());
    case 8: return fn(std::integral_constant<int, 8>());
    case 10: return fn(std::integral_constant<int, 10>());
    default: return fail(ADJWT_ERR_INVALID_ARG, "unsupported filter length");
  }
}

int analysis_grid(const Level& L, dim3* g) {
  *g = dim3((L.band_pitch + kTile - 1) / kTile, (L.ax[0].n + kTile - 1) / kTile);
  return static_cast<int>(g->x * g->y);
}

}  // namespace

int wt_l1_partial_slots(const adjwt_wt_plan* p) {
  int total = 0;
  for (const Level& L : p->lv) {
    dim3 g;
    total += analysis_grid(L, &g);
  }
  return total;
}

int launch_wt_analysis(const adjwt_wt_plan* p, const float* image, float* coeffs, bool adjoint,
                       const ProxArgs& prox, float* llbuf0, float* llbuf1, cudaStream_t s, int* l1_slots_used) {
  float* llbuf[2] = {llbuf0, llbuf1};
  const FilterBank& fb = p->fb;
  int slot = 0;
  for (int j = 1; j <= p->levels; ++j) {
    const Level& L = p->lv[j - 1];
    AnaArgs a{};
    a.in = (j == 1) ? image : llbuf[(j - 1) % 2];
    a.in_pitch = L.in_pitch;
    a.Nr = L.ax[0].N;
    a.Nc = L.ax[1].N;
    a.nr = L.ax[0].n;
    a.nc = L.ax[1].n;
    a.mode = p->bc;
    a.winv_r = adjoint ? L.ax[0].winv : nullptr;
    a.winv_c = adjoint ? L.ax[1].winv : nullptr;
    a.out_pitch = L.band_pitch;
    for (int b = 0; b < 4; ++b) {
      const bool final_band = (b > 0) || (j == p->levels);
      float* base = nullptr;
      if (final_band) {
        if (prox.x) {
          a.px[b] = prox.x + L.off_band[b];
          a.py[b] = prox.y + L.off_band[b];
        } else {
          base = coeffs + L.off_band[b];
        }
      } else {
        base = llbuf[j % 2];
      }
      a.dst[b] = base;
    }
    a.step = prox.step;
    a.thresh = prox.thresh;
    a.beta = prox.beta;
    for (int t = 0; t < fb.L; ++t) {
      if (adjoint) {  // dual analysis filters: synthesis filters reversed (Eq. 3, Eq. 4)
        a.flo[t] = static_cast<float>(fb.rec_lo[fb.L - 1 - t]);
        a.fhi[t] = static_cast<float>(fb.rec_hi[fb.L - 1 - t]);
      } else {
        a.flo[t] = static_cast<float>(fb.dec_lo[t]);
        a.fhi[t] = static_cast<float>(fb.dec_hi[t]);
      }
    }
    dim3 grid;
    const int ncta = analysis_grid(L, &grid);
    a.l1 = (prox.x && prox.l1_partials) ? prox.l1_partials + slot : nullptr;
    slot += ncta;
    const char* name = !adjoint ? "wt_analysis" : (prox.x ? "wt_adjoint_prox" : "wt_adjoint");
    int rc = dispatch_L(fb.L, [&](auto Lc) {
      ADJWT_TRACED(name, j, s, k_analysis<decltype(Lc)::value><<<grid, kThreads, 0, s>>>(a));
      return ADJWT_OK;
    });
    if (rc) return rc;
    ADJWT_CUDA_CHECK(cudaGetLastError());
  }
  if (l1_slots_used) *l1_slots_used = slot;
  return ADJWT_OK;
}

int launch_wt_synth(const adjwt_wt_plan* p, const float* coeffs, float* image, float* llbuf0, float* llbuf1,
                    cudaStream_t s) {
  float* llbuf[2] = {llbuf0, llbuf1};
  const FilterBank& fb = p->fb;
  const int Lp = fb.L - 1;
  for (int j = p->levels; j >= 1; --j) {
    const Level& L = p->lv[j - 1];
    SynArgs a{};
    for (int b = 0; b < 4; ++b)
      a.band[b] = (b == 0 && j < p->levels) ? llbuf[j % 2] : coeffs + L.off_band[b];
    a.band_pitch = L.band_pitch;
    a.out = (j == 1) ? image : llbuf[(j - 1) % 2];
    a.out_pitch = L.in_pitch;
    a.Nr = L.ax[0].N;
    a.Nc = L.ax[1].N;
    a.nr = L.ax[0].n;
    a.nc = L.ax[1].n;
    a.mode = p->bc;
    a.winv_r = L.ax[0].winv;
    a.winv_c = L.ax[1].winv;
    for (int t = 0; t < fb.L; ++t) {
      a.g[0][t] = static_cast<float>(fb.rec_lo[t]);
      a.g[1][t] = static_cast<float>(fb.rec_hi[t]);
    }
    int rc = dispatch_L(fb.L, [&](auto Lc) {
      constexpr int LL = decltype(Lc)::value;
      if (L.generic_synth) {
        const int64_t count = (int64_t)a.Nr * a.Nc;
        const unsigned nb = (unsigned)((count + kThreads - 1) / kThreads);
        ADJWT_TRACED("wt_synth_gather", j, s, k_synthesis_gather<LL><<<nb, kThreads, 0, s>>>(a, 0, count));
      } else {
        dim3 grid((a.Nc + kTile - 1) / kTile, (a.Nr + kTile - 1) / kTile);
        ADJWT_TRACED("wt_synth", j, s, k_synthesis<LL><<<grid, kThreads, 0, s>>>(a));
        if (p->bc == kPpd) {
          const int64_t count = (int64_t)2 * Lp * a.Nc + (int64_t)(a.Nr - 2 * Lp) * 2 * Lp;
          const unsigned nb = (unsigned)((count + kThreads - 1) / kThreads);
          ADJWT_TRACED("wt_synth_gather", j, s, k_synthesis_gather<LL><<<nb, kThreads, 0, s>>>(a, 1, count));
        }
      }
      return ADJWT_OK;
    });
    if (rc) return rc;
    ADJWT_CUDA_CHECK(cudaGetLastError());
  }
  return ADJWT_OK;
}

}  // namespace adjwt
