// Device helpers shared by the libadjwt kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace adjwt {

// Checked builds (-DADJWT_BOUNDS_CHECK): the index arithmetic of the tile
// bodies' global loads and stores is tested against the extents of their
// buffers; an access outside them is skipped (a load reads zero) and
// ADJWT_ERR_BOUNDS is recorded in the device status word (first writer
// wins).  Release builds compile the test away.
#ifdef ADJWT_BOUNDS_CHECK
__device__ __forceinline__ bool in_bounds(int* status, bool ok) {
  if (!ok && status) atomicCAS(status, 0, -9 /* ADJWT_ERR_BOUNDS */);
  return ok;
}
#else
__device__ __forceinline__ bool in_bounds(int*, bool) { return true; }
#endif

__device__ __forceinline__ int floor_div(int a, int b) {  // b > 0
  int q = a / b;
  return (a % b != 0 && a < 0) ? q - 1 : q;
}

__device__ __forceinline__ int pos_mod(int a, int b) {  // b > 0
  int m = a % b;
  return m < 0 ? m + b : m;
}

// Source index of virtual position x (image coordinates) under the extension
// `mode` (0 zero, 1 half-point symmetric, 2/3 periodic); -1 means a zero.
__device__ __forceinline__ int ext_src(int x, int N, int mode) {
  if (mode == 0) return (x >= 0 && x < N) ? x : -1;
  if (mode == 1) {
    int m = pos_mod(x, 2 * N);
    return m < N ? m : 2 * N - 1 - m;
  }
  return pos_mod(x, N);
}

// Tile t of an nty x ntx grid in "border first" order: the tiles outside the
// interior rectangle [ir0, ir1) x [ic0, ic1) come first (the rows above, the
// rows below, then the columns beside it), then the interior row by row.
// Persistent kernels whose border tiles cost more walk tiles in this order,
// so that each CTA takes at most one border tile and starts with it.  An
// empty rectangle (ir1 <= ir0 or ic1 <= ic0) must be passed as all zeros.
__device__ __forceinline__ void border_first_tile(int t, int ntx, int nty, int ir0, int ir1, int ic0, int ic1,
                                                  int* ty, int* tx) {
  const int iw = ic1 - ic0, nb = ntx * nty - iw * (ir1 - ir0);
  if (t >= nb) {
    const int u = t - nb, q = u / iw;
    *ty = ir0 + q;
    *tx = ic0 + (u - q * iw);
    return;
  }
  const int ntop = ir0 * ntx, nbot = (nty - ir1) * ntx;
  if (t < ntop) {
    *ty = t / ntx;
    *tx = t - *ty * ntx;
  } else if (t < ntop + nbot) {
    const int j = t - ntop, q = j / ntx;
    *ty = ir1 + q;
    *tx = j - q * ntx;
  } else {
    const int j = t - ntop - nbot, side = ic0 + (ntx - ic1), q = j / side, k = j - q * side;
    *ty = ir0 + q;
    *tx = k < ic0 ? k : ic1 + (k - ic0);
  }
}

// Block-wide float64 sum; every thread passes its value, thread 0 gets the total.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* scratch /* NT/32 doubles */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) t += scratch[w];
  }
  return t;
}

}  // namespace adjwt
