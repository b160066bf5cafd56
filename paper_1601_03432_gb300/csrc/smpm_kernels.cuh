// Device geometry and small helpers shared by the kernels of the deflated
// Schur-complement solve (sm_103a): neighbour and interface lookups, warp
// sums and the element GEMVs.
//
// Vectors live in two layouts: node vectors (element-major, n*n nodes per
// element, x index fastest) and padded slot vectors (4n slots per element,
// faces W,E,S,N, face node t increasing along the face; slots on physical
// boundary faces are kept at zero).  Element matrices are stored
// column-major, so the threads (or lanes) that own consecutive rows read
// each column coalesced.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace smpm {

struct DevGeo {
  int mx, my, n, M;
  long long nel, kp, r, d;
  // [tau, p, 2/h] of the W/E faces of every element column (cgeo, 3 mx) and
  // of the S/N faces of every row (rgeo, 3 my); device memory
  const double* cgeo;
  const double* rgeo;
  // weight of face F of element e in the deflation vectors z_j (zw[4e + F]):
  // z_j is the restriction of B 1 to interface j's slots, scaled by the mean
  // of its two sides; null on uniform grids, where every weight is 1
  const double* zw;
  int graded;  // fast-diagonalisation factors per column / row (else per face-type class)
  int pad_;
};

__device__ __forceinline__ double dev_zw(const DevGeo& g, int e, int F) {
  return g.zw ? __ldg(g.zw + 4 * (size_t)e + F) : 1.0;
}

// [tau, p, 2/h] of face F of element e
__device__ __forceinline__ const double* face_geo(const DevGeo& g, int e, int F) {
  return F < 2 ? g.cgeo + 3 * (e % g.mx) : g.rgeo + 3 * (e / g.mx);
}

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

// y[r] = sum_c A[c*M + r] x[c] for r < M: A column-major (shared or global
// memory; consecutive threads read consecutive rows), x in shared memory.
// One thread per row with four independent partial sums: every FP64 product
// is a plain FMA (no warp-shuffle reduction adds on the scarce FP64 pipe).
template <typename S>
__device__ __forceinline__ void gemv_cm(const S* A, const S* x, S* y, int M) {
  for (int r = threadIdx.x; r < M; r += blockDim.x) {
    S s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    int c = 0;
    for (; c + 3 < M; c += 4) {
      s0 += A[(size_t)c * M + r] * x[c];
      s1 += A[(size_t)(c + 1) * M + r] * x[c + 1];
      s2 += A[(size_t)(c + 2) * M + r] * x[c + 2];
      s3 += A[(size_t)(c + 3) * M + r] * x[c + 3];
    }
    for (; c < M; ++c) s0 += A[(size_t)c * M + r] * x[c];
    y[r] = (s0 + s1) + (s2 + s3);
  }
}

// y[r] = sum_{c < cols} A[c*ld + r] x[c] for r < rows, A column-major with
// leading dimension ld.  The CTA splits the columns into P = blockDim / rows
// parts (P <= 8, a power of two): thread (part, r) with r fastest reads
// consecutive rows (conflict-free in shared memory, coalesced in global), and
// the P partial sums meet in the scratch buffer red (>= P*rows entries).  FP64
// work thus spreads over all warps of the CTA, with P-1 adds per row on top
// of the rows*cols FMAs.  Ends with __syncthreads.
template <typename S>
__device__ __forceinline__ void gemv_split(const S* A, int ld, const S* x, S* y, int rows, int cols, S* red,
                                           bool accumulate = false, S alpha = S(1)) {
  int P = 1;
  while (P * 2 * rows <= (int)blockDim.x && P < 8) P *= 2;
  const int t = threadIdx.x, r = t % rows, part = t / rows;
  if (part < P) {
    S s0 = 0, s1 = 0;
    int c = part;
    for (; c + P < cols; c += 2 * P) {
      s0 += A[(size_t)c * ld + r] * x[c];
      s1 += A[(size_t)(c + P) * ld + r] * x[c + P];
    }
    if (c < cols) s0 += A[(size_t)c * ld + r] * x[c];
    red[part * rows + r] = s0 + s1;
  }
  __syncthreads();
  for (int i = t; i < rows; i += blockDim.x) {
    S sum = red[i];
    for (int p = 1; p < P; ++p) sum += red[p * rows + i];
    y[i] = accumulate ? y[i] + alpha * sum : sum;
  }
  __syncthreads();
}

}  // namespace smpm
