// Device kernels of the deflated Schur-complement solve (sm_103a).
//
// Vectors live in two layouts: node vectors (element-major, n*n nodes per
// element, x index fastest) and padded slot vectors (4n slots per element,
// faces W,E,S,N, face node t increasing along the face; slots on physical
// boundary faces are kept at zero).  Every per-element kernel runs one CTA per
// element (or per checkerboard block) and stages the element's small vectors
// in shared memory; the element matrices are streamed once from HBM/L2 with
// row-per-warp, lane-per-column coalesced loads.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace smpm {

struct DevGeo {
  int mx, my, n, M;
  long long nel, kp, r, d;
  double tau_x, tau_y, p_x, p_y, sx, sy;
};

__device__ __forceinline__ int dev_neighbour(const DevGeo& g, int e, int F) {
  int ix = e % g.mx, iy = e / g.mx;
  switch (F) {
    case 0: return ix > 0 ? e - 1 : -1;
    case 1: return ix < g.mx - 1 ? e + 1 : -1;
    case 2: return iy > 0 ? e - g.mx : -1;
    default: return iy < g.my - 1 ? e + g.mx : -1;
  }
}

__device__ __forceinline__ int dev_iface(const DevGeo& g, int e, int F) {
  int ix = e % g.mx, iy = e / g.mx, row = 2 * g.mx - 1;
  switch (F) {
    case 0: return ix > 0 ? iy * row + ix - 1 : -1;
    case 1: return ix < g.mx - 1 ? iy * row + ix : -1;
    case 2: return iy > 0 ? (iy - 1) * row + g.mx - 1 + ix : -1;
    default: return iy < g.my - 1 ? iy * row + g.mx - 1 + ix : -1;
  }
}

template <typename S>
__device__ __forceinline__ S warp_sum(S v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// y[row] = sum_col A[row*M + col] x[col] (A row-major in global memory, x and
// y in shared memory); one warp per row, lanes stride the columns.
template <typename S, typename Acc>
__device__ __forceinline__ void gemv_rows(const S* __restrict__ A, const S* x, Acc* y, int M) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int row = warp; row < M; row += nw) {
    const S* a = A + (size_t)row * M;
    Acc acc = 0;
    for (int c = lane; c < M; c += 32) acc += (Acc)__ldg(a + c) * (Acc)x[c];
    acc = warp_sum(acc);
    if (lane == 0) y[row] = acc;
  }
}

}  // namespace smpm
