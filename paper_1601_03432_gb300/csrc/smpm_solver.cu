// CUDA solve path and C ABI of the deflated Schur-complement method
// (Joshi & Diamessis, Algorithms 1-3).  See include/smpm.h for the contract.
//
// A solve (schur_solve) is three cooperative, persistent launches on the
// caller's stream; the host synchronises once, to read the report:
//   k_pre    b <- b - u_L u_L^T b (Eq. regularize_poisson), b_S = B A^-1 b
//            by fast-diagonalisation element solves and Robin flux pushes,
//            b_S <- b_S - u_S u_S^T b_S (Eq. regularize_schur), Z^T b_S and
//            the GMRES right-hand side P b_S (smpm_prepost.cuh);
//   k_gmres  the whole restarted GMRES on P S M^-1 (smpm_gmres.cuh): five
//            phases per Arnoldi step separated by grid barriers;
//   k_post   x_S = Q M^-1 x_1 + Z C^+ Z^T b_S (Eq. deflated_schur), the
//            recovery u = A^-1 (b - E x_S), the true Schur residual and the
//            zero GLL-weighted mean (smpm_prepost.cuh).
// Mixed precision replaces k_gmres by a fixed sequence of
// (k_gmres<float>, k_refine) pairs (smpm_refine.cuh); the adjoint solve runs
// the same kernels on the transposed factor set.
//
// Many grids and right-hand sides are solved in one launch by k_batch
// (smpm_batch.cuh): teams of CTAs run the same bodies with team barriers.
//
// The single-operator entry points use small one-pass kernels:
//   y = S v          k_schur_warpk (several warps per element, M <= 96),
//                    k_schur_stream (bulk-copy ring, larger M), k_schur
//                    (from global memory when one matrix exceeds the ring);
//                    batched: k_schur_warp_batch, k_schur_stream_batch;
//   S M^-1 and M^-1  k_black (block solves a = G (p - X q), b = q - T_e a),
//                    k_white (white elements' T_e products, c = Z^T y);
//   P and Q          k_zt (c = Z^T v), k_coarse (c_hat = C^+ c),
//                    k_defl_dots, k_sub, k_assemble;
//   b_S, recovery    k_schur_rhs, k_recover;
//   allocation-free  k_deflate_noalloc.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <mutex>
#include <new>
#include <type_traits>
#include <string>
#include <vector>

#include "smpm_internal.h"
#include "smpm_kernels.cuh"

using namespace smpm;

namespace {

thread_local std::string g_last_error;

constexpr int kSlotsPerBlock = 256;   // slots per CTA in the vector kernels
constexpr int kElemThreads = 256;     // threads per element CTA
constexpr int kTraceCap = 1 << 16;    // entries of the optional phase trace
constexpr int kGmresThreads = 256;    // threads per CTA of the persistent GMRES kernel
// per-solve control block (zeroed by one memset): 64 barrier counters |
// err, done, nref | 8 accumulators | 32 refinement residual norms
constexpr size_t kCtlBytes = 720;  // + 32 inner iteration counts
constexpr int kMaxRefine = 8;        // FP64 refinement steps of the mixed-precision path
constexpr int kMaxStreamBufs = 4;    // shared-memory buffers of the GMRES kernel's matrix stream
constexpr int kWarpElemsMin = 4;     // owned blocks per CTA from which each warp takes its own element
constexpr double kInnerTol = 1e-4;   // relative tolerance of each FP32 inner GMRES
// the coarse solve is fused into the white-element phase when the atomic adds
// it costs per Arnoldi step (d per CTA) stay below this
constexpr long long kFusedCoarseMaxAdds = 1LL << 17;

struct GState {
  double tolabs, beta0, beta, wnorm0sq, resid;
  int j, converged, breakdown, nan;
  double g[kMaxRestart + 1];
  double cs[kMaxRestart], sn[kMaxRestart];
  double R[(kMaxRestart + 1) * kMaxRestart];  // column j at R[j*(kMaxRestart+1)]
  double h1[kMaxRestart + 2], h2[kMaxRestart + 2];
  double y[kMaxRestart];
  double scal[8];
};


// ------------------------------------------------------------ reductions
__device__ bool last_block_done(unsigned* cnt) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(cnt, 1u);
    am_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

// out[l] = sum_b part[l*nblk + b] for l < nout, in a fixed order.
__device__ void finalize_partials(const double* part, int nblk, int nout, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int l = warp; l < nout; l += nw) {
    double acc = 0;
    for (int b = lane; b < nblk; b += 32) acc += __ldcg(part + (size_t)l * nblk + b);
    acc = warp_sum(acc);
    if (lane == 0) out[l] = acc;
  }
}

// part[l*nblk + blockIdx] = sum_{i<CH} V[l][base+i] * wsh[i] for l < nvec, and
// (with_norm) part[nvec*nblk + blockIdx] = sum wsh[i]^2.
template <typename S>
__device__ void block_multidot(const S* __restrict__ V, long long kp, int nvec, long long base, const double* wsh,
                               bool with_norm, double* part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int CH = blockDim.x;
  const int nout = nvec + (with_norm ? 1 : 0);
  for (int l = warp; l < nout; l += nw) {
    double acc = 0;
    if (l < nvec) {
      const S* v = V + (size_t)l * kp + base;
      for (int i = lane; i < CH && base + i < kp; i += 32) acc += (double)__ldg(v + i) * wsh[i];
    } else {
      for (int i = lane; i < CH; i += 32) acc += wsh[i] * wsh[i];
    }
    acc = warp_sum(acc);
    if (lane == 0) part[(size_t)l * gridDim.x + blockIdx.x] = acc;
  }
}

// ------------------------------------------------------- element solves
// U = A_e^-1 B by fast diagonalisation (the Kronecker-sum structure of A_e):
// U = Vy ((Vy^-1 B Vx^-T) ./ (lx_i + ly_j)) Vx^T.  B, U, t1: n*n in shared.
__device__ void elem_solve_dev(int n, const double* __restrict__ fx, const double* __restrict__ fy, const double* B,
                               double* U, double* t1) {
  const double *Vx = fx, *Vxi = fx + n * n, *lx = fx + 2 * n * n;
  const double *Vy = fy, *Vyi = fy + n * n, *ly = fy + 2 * n * n;
  const int nn = n * n;
  for (int q = threadIdx.x; q < nn; q += blockDim.x) {  // t1 = Vyi B
    int j = q / n, a = q % n;
    double s = 0;
    for (int b = 0; b < n; ++b) s += __ldg(Vyi + j * n + b) * B[b * n + a];
    t1[q] = s;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nn; q += blockDim.x) {  // U = t1 Vxi^T ./ (lx + ly)
    int j = q / n, i = q % n;
    double s = 0;
    for (int a = 0; a < n; ++a) s += t1[j * n + a] * __ldg(Vxi + i * n + a);
    U[q] = s / (__ldg(lx + i) + __ldg(ly + j));
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nn; q += blockDim.x) {  // t1 = U Vx^T
    int j = q / n, a = q % n;
    double s = 0;
    for (int i = 0; i < n; ++i) s += U[j * n + i] * __ldg(Vx + a * n + i);
    t1[q] = s;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nn; q += blockDim.x) {  // U = Vy t1
    int b = q / n, a = q % n;
    double s = 0;
    for (int j = 0; j < n; ++j) s += __ldg(Vy + b * n + j) * t1[j * n + a];
    U[q] = s;
  }
  __syncthreads();
}

__device__ __forceinline__ void face_node(int n, int F, int t, int* a, int* b) {
  switch (F) {
    case 0: *a = 0; *b = t; break;
    case 1: *a = n - 1; *b = t; break;
    case 2: *a = t; *b = 0; break;
    default: *a = t; *b = n - 1; break;
  }
}

// n_F . grad U at face node t (U in shared memory, D in global).
// n_F . grad U at face node t of face F (sc = 2/h of the element across F).
__device__ double normal_deriv(const DevGeo& g, const double* __restrict__ D, const double* U, int F, int t,
                               double sc) {
  const int n = g.n;
  double acc = 0;
  switch (F) {
    case 0: for (int c = 0; c < n; ++c) acc += __ldg(D + c) * U[t * n + c]; return -sc * acc;
    case 1: for (int c = 0; c < n; ++c) acc += __ldg(D + (n - 1) * n + c) * U[t * n + c]; return sc * acc;
    case 2: for (int c = 0; c < n; ++c) acc += __ldg(D + c) * U[c * n + t]; return -sc * acc;
    default: for (int c = 0; c < n; ++c) acc += __ldg(D + (n - 1) * n + c) * U[c * n + t]; return sc * acc;
  }
}

// fast-diagonalisation entry: face-type class, or the column / row on a graded grid
__device__ __forceinline__ const double* fd_x(const DevGeo& g, const double* fdx, int e) {
  int ix = e % g.mx;
  int cls = g.graded ? ix : ((ix > 0 ? 1 : 0) | (ix < g.mx - 1 ? 2 : 0));
  return fdx + (size_t)cls * (2 * g.n * g.n + g.n);
}
__device__ __forceinline__ const double* fd_y(const DevGeo& g, const double* fdy, int e) {
  int iy = e / g.mx;
  int cls = g.graded ? iy : ((iy > 0 ? 1 : 0) | (iy < g.my - 1 ? 2 : 0));
  return fdy + (size_t)cls * (2 * g.n * g.n + g.n);
}

// b_S = B A^-1 b (Eq. schur_complement_system): one CTA per element; the flux of
// w = A_e^-1 b_e into the slot (nbr, opp F, t) is -tau' (p' w - n_F.grad w),
// tau' and p' those of the neighbour's face opp F.
// Slots on boundary faces are not written (the caller zeroes b_S).
__global__ void k_schur_rhs(DevGeo g, const double* __restrict__ fdx, const double* __restrict__ fdy,
                            const double* __restrict__ D, const double* __restrict__ b, double* bS) {
  extern __shared__ double sh[];
  const int n = g.n, nn = n * n, e = blockIdx.x;
  double *B = sh, *U = sh + nn, *t1 = sh + 2 * nn;
  for (int q = threadIdx.x; q < nn; q += blockDim.x) B[q] = b[(size_t)e * nn + q];
  __syncthreads();
  elem_solve_dev(n, fd_x(g, fdx, e), fd_y(g, fdy, e), B, U, t1);
  for (int i = threadIdx.x; i < 4 * n; i += blockDim.x) {
    int F = i / n, t = i % n;
    int e2 = dev_neighbour(g, e, F);
    if (e2 < 0) continue;
    int a, bb;
    face_node(n, F, t, &a, &bb);
    const double* fn = face_geo(g, e2, F ^ 1);
    double val = fn[1] * U[bb * n + a] - normal_deriv(g, D, U, F, t, face_geo(g, e, F)[2]);
    bS[(size_t)e2 * g.M + (F ^ 1) * n + t] = -fn[0] * val;
  }
}

// u = A^-1 (b - E x): one CTA per element.
__global__ void k_recover(DevGeo g, const double* __restrict__ fdx, const double* __restrict__ fdy,
                          const double* __restrict__ b, const double* __restrict__ x, double* u) {
  extern __shared__ double sh[];
  const int n = g.n, nn = n * n, e = blockIdx.x;
  double *B = sh, *U = sh + nn, *t1 = sh + 2 * nn;
  for (int q = threadIdx.x; q < nn; q += blockDim.x) B[q] = b[(size_t)e * nn + q];
  __syncthreads();
  for (int F = 0; F < 4; ++F) {  // faces one after another: corner nodes get both slots
    if (dev_neighbour(g, e, F) >= 0)
      for (int t = threadIdx.x; t < n; t += blockDim.x) {
        int a, bb;
        face_node(n, F, t, &a, &bb);
        B[bb * n + a] -= x[(size_t)e * g.M + F * n + t];
      }
    __syncthreads();
  }
  elem_solve_dev(n, fd_x(g, fdx, e), fd_y(g, fdy, e), B, U, t1);
  for (int q = threadIdx.x; q < nn; q += blockDim.x) u[(size_t)e * nn + q] = U[q];
}

// ------------------------------------------------------- slot operators
// y = S v = v + scatter_e(T_e v_e) (Eq. schur_complement_system), push form:
// element e writes the neighbours' slots facing it (each slot has exactly one
// writer) and its own boundary-face slots.
template <typename S>
__global__ void k_schur(DevGeo g, const S* __restrict__ T, const S* __restrict__ v, S* y) {
  extern __shared__ unsigned char shraw[];
  S* ve = reinterpret_cast<S*>(shraw);
  S* z = ve + g.M;
  const int e = blockIdx.x, M = g.M, n = g.n;
  for (int i = threadIdx.x; i < M; i += blockDim.x) ve[i] = v[(size_t)e * M + i];
  __syncthreads();
  gemv_cm(T + (size_t)e * M * M, ve, z, M);
  __syncthreads();
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    int F = i / n, t = i % n;
    int e2 = dev_neighbour(g, e, F);
    if (e2 >= 0) {
      size_t s = (size_t)e2 * M + (F ^ 1) * n + t;
      y[s] = v[s] + z[i];
    } else {
      y[(size_t)e * M + i] = ve[i];
    }
  }
}

// Black step: t = M^-1 v on the block of black element e (own slots p,
// facing slots q): a = G (p - X q), b = q - T_e a.  Writes t on the whole
// block (every slot is in exactly one block).
template <typename S>
__global__ void k_black(DevGeo g, const int* __restrict__ black, const S* __restrict__ T, const S* __restrict__ G,
                        const S* __restrict__ X, const S* __restrict__ v, S* t) {
  extern __shared__ unsigned char shraw[];
  const int M = g.M, n = g.n, ib = blockIdx.x, e = black[ib];
  S* p = reinterpret_cast<S*>(shraw);
  S* q = p + M;
  S* r1 = q + M;
  S* a = r1 + M;
  S* z = a + M;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    int F = i / n, tt = i % n;
    int e2 = dev_neighbour(g, e, F);
    p[i] = v[(size_t)e * M + i];
    q[i] = e2 >= 0 ? v[(size_t)e2 * M + (F ^ 1) * n + tt] : S(0);
  }
  __syncthreads();
  const S* Xb = X + (size_t)ib * 4 * n * n;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    int F = i / n, tt = i % n;
    const S* xf = Xb + (size_t)F * n * n;  // X_F column-major
    S s = p[i];
    for (int s2 = 0; s2 < n; ++s2) s -= __ldg(xf + s2 * n + tt) * q[F * n + s2];
    r1[i] = s;
  }
  __syncthreads();
  gemv_cm(G + (size_t)ib * M * M, r1, a, M);
  __syncthreads();
  gemv_cm(T + (size_t)e * M * M, a, z, M);
  __syncthreads();
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    int F = i / n, tt = i % n;
    int e2 = dev_neighbour(g, e, F);
    t[(size_t)e * M + i] = a[i];
    if (e2 >= 0) t[(size_t)e2 * M + (F ^ 1) * n + tt] = q[i] - z[i];
  }
}

// White step: y = S t given t = M^-1 v: on white-owned slots y = v; on the
// black slots facing white element e, y = t + (T_e t_e).  Also c = Z^T y for
// the interfaces of e (every interface has exactly one white side).
template <typename S>
__global__ void k_white(DevGeo g, const int* __restrict__ white, const S* __restrict__ T, const S* __restrict__ v,
                        const S* __restrict__ t, S* y, double* c) {
  extern __shared__ unsigned char shraw[];
  const int M = g.M, n = g.n, e = white[blockIdx.x];
  S* tb = reinterpret_cast<S*>(shraw);
  S* z = tb + M;
  double* cs = reinterpret_cast<double*>(z + M + (M & 1));
  for (int i = threadIdx.x; i < M; i += blockDim.x) tb[i] = t[(size_t)e * M + i];
  __syncthreads();
  gemv_cm(T + (size_t)e * M * M, tb, z, M);
  __syncthreads();
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    int F = i / n, tt = i % n;
    int e2 = dev_neighbour(g, e, F);
    S vo = v[(size_t)e * M + i];
    y[(size_t)e * M + i] = vo;
    double ci = 0;
    if (e2 >= 0) {
      size_t s = (size_t)e2 * M + (F ^ 1) * n + tt;
      S ys = t[s] + z[i];
      y[s] = ys;
      ci = g.zw ? dev_zw(g, e, F) * (double)vo + dev_zw(g, e2, F ^ 1) * (double)ys : (double)vo + (double)ys;
    }
    cs[i] = ci;
  }
  __syncthreads();
  if (c && threadIdx.x < 4) {
    int F = threadIdx.x;
    int j = dev_iface(g, e, F);
    if (j >= 0) {
      double s = 0;
      for (int tt = 0; tt < n; ++tt) s += cs[F * n + tt];
      c[j] = s;
    }
  }
}

// c = Z^T v: one thread per interface, summing its 2n slots (weighted).
template <typename S>
__global__ void k_zt(DevGeo g, const S* __restrict__ v, double* c) {
  long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= g.d) return;
  const int row = 2 * g.mx - 1, n = g.n, M = g.M;
  int iy = (int)(j / row), rem = (int)(j % row);
  int e1, F1;
  if (rem < g.mx - 1) { e1 = iy * g.mx + rem; F1 = 1; }
  else { e1 = iy * g.mx + rem - (g.mx - 1); F1 = 3; }
  int e2 = dev_neighbour(g, e1, F1);
  const double w1 = dev_zw(g, e1, F1), w2 = dev_zw(g, e2, F1 ^ 1);
  double s = 0;
  for (int t = 0; t < n; ++t)
    s += w1 * (double)v[(size_t)e1 * M + F1 * n + t] + w2 * (double)v[(size_t)e2 * M + (F1 ^ 1) * n + t];
  c[j] = s;
}

// out = H c (FP64, d x d, warp per row).
__global__ void k_coarse(const double* __restrict__ H, const double* __restrict__ c, double* out, int d) {
  const int lane = threadIdx.x & 31;
  const long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (row >= d) return;
  const double* h = H + row * (long long)d;
  double acc = 0;
  for (int j = lane; j < d; j += 32) acc += __ldg(h + j) * __ldg(c + j);
  acc = warp_sum(acc);
  if (lane == 0) out[row] = acc;
}

// w = y - (S Z) chat on one slot (pull form); chat == nullptr gives w = y.
template <typename S>
__device__ __forceinline__ double deflate_slot(const DevGeo& g, const S* __restrict__ y, const double* __restrict__ chat,
                                               const S* __restrict__ Rs, long long s) {
  const int M = g.M, n = g.n;
  int e = (int)(s / M), i = (int)(s % M), F = i / n, t = i % n;
  int e2 = dev_neighbour(g, e, F);
  if (e2 < 0) return 0.0;
  double ys = (double)y[s];
  if (!chat) return ys;
  double acc = dev_zw(g, e, F) * chat[dev_iface(g, e, F)];
  const S* R = Rs + ((size_t)e2 * M + (F ^ 1) * n + t) * 4;
#pragma unroll
  for (int G = 0; G < 4; ++G) {
    int jj = dev_iface(g, e2, G);
    if (jj >= 0) acc += (double)R[G] * chat[jj];
  }
  return ys - acc;
}

// Deflation (Eq. projection1) fused with the first Gram-Schmidt pass:
// w = y - S Z chat; h1 = V[0..nvec)^T w; also ||w||^2.
template <typename S>
__global__ void k_defl_dots(DevGeo g, const S* __restrict__ y, const double* __restrict__ chat,
                            const S* __restrict__ Rs, const S* __restrict__ V, int nvec, S* w, double* part,
                            unsigned* cnt, GState* gs) {
  __shared__ double wsh[kSlotsPerBlock];
  const long long base = (long long)blockIdx.x * blockDim.x, s = base + threadIdx.x;
  double ws = 0;
  if (s < g.kp) {
    S wv = (S)deflate_slot(g, y, chat, Rs, s);
    w[s] = wv;
    ws = (double)wv;
  }
  wsh[threadIdx.x] = ws;
  __syncthreads();
  if (nvec < 0) return;  // deflation only
  block_multidot(V, g.kp, nvec, base, wsh, true, part);
  if (last_block_done(cnt)) {
    finalize_partials(part, gridDim.x, nvec + 1, gs->h1);
    __syncthreads();
    if (threadIdx.x == 0) {
      gs->wnorm0sq = gs->h1[nvec];
      *cnt = 0;
    }
  }
}

// out = a - b
template <typename S>
__global__ void k_sub(long long n, const S* __restrict__ a, const S* __restrict__ b, S* out) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s < n) out[s] = a[s] - b[s];
}

// x = t - Z (chat - chat_b) on interface slots (Eq. deflated_schur assembly).
__global__ void k_assemble(DevGeo g, const double* __restrict__ t, const double* __restrict__ chat,
                           const double* __restrict__ chat_b, double* x) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= g.kp) return;
  const int M = g.M, n = g.n;
  int e = (int)(s / M), i = (int)(s % M), F = i / n;
  int j = dev_iface(g, e, F);
  if (j < 0) { x[s] = 0.0; return; }
  double cb = chat_b ? chat_b[j] : 0.0;
  x[s] = t[s] - dev_zw(g, e, F) * ((chat ? chat[j] : 0.0) - cb);
}

#include "smpm_gmres.cuh"
#include "smpm_prepost.cuh"
#include "smpm_refine.cuh"
#include "smpm_lockstep.cuh"
#include "smpm_batch.cuh"

// y = S v streamed from HBM: a persistent CTA per SM walks its elements
// e = c, c+G, ... and keeps STAGES of them in flight with bulk copies of the
// (contiguous, column-major) T_e into shared-memory buffers, so the factor
// streams at HBM rate while the GEMV of an earlier element runs.  Outputs as
// k_schur (push form).  A copy that never completes (bounded wait) leaves NaN
// in that element's outputs.
template <typename S>
__global__ void __launch_bounds__(256, 2) k_schur_stream(DevGeo g, const S* __restrict__ Tc, const S* v, S* y,
                                                         int stages) {
  extern __shared__ __align__(16) unsigned char raw[];
  const int M = g.M, n = g.n, G = gridDim.x;
  const unsigned mbytes = (unsigned)(M * M * sizeof(S));
  S* buf = reinterpret_cast<S*>(raw);
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(buf + (size_t)stages * M * M);
  S* ve = reinterpret_cast<S*>(mbar + stages);
  S* z = ve + M;
  S* red = z + M;
  const long long nk = (g.nel - blockIdx.x + G - 1) / G;
  if (threadIdx.x == 0) {
    for (int b = 0; b < stages; ++b) mbar_init(mbar + b);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](long long k) {
    if (threadIdx.x != 0 || k >= nk) return;
    const int b = (int)(k % stages);
    const long long e = blockIdx.x + k * G;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar + b)), "r"(mbytes)
                 : "memory");
    bulk_g2s(buf + (size_t)b * M * M, Tc + (size_t)e * M * M, mbytes, mbar + b);
  };
  for (int k = 0; k < stages; ++k) issue(k);
  __shared__ int ok;
  bool failed = false;
  long long waited = 0;  // copies completed or given up
  // register prefetch of the next element's vector entries (thread i < M):
  // own slot i and the neighbour slot its output row feeds
  auto nb_slot = [&](long long e, int i) -> long long {
    const int F = i / n, t = i % n, e2 = dev_neighbour(g, (int)e, F);
    return e2 >= 0 ? (long long)e2 * M + (F ^ 1) * n + t : -1;
  };
  S pv_own = 0, pv_nb = 0;
  if (nk > 0 && threadIdx.x < M) {
    pv_own = v[(long long)blockIdx.x * M + threadIdx.x];
    const long long sl = nb_slot(blockIdx.x, threadIdx.x);
    pv_nb = sl >= 0 ? v[sl] : S(0);
  }
  for (long long k = 0; k < nk; ++k) {
    const long long e = blockIdx.x + k * G;
    const int b = (int)(k % stages);
    S cur_nb = pv_nb;
    if (threadIdx.x < M) ve[threadIdx.x] = pv_own;
    if (k + 1 < nk && threadIdx.x < M) {
      const long long e1 = e + G;
      pv_own = v[e1 * M + threadIdx.x];
      const long long sl = nb_slot(e1, threadIdx.x);
      pv_nb = sl >= 0 ? v[sl] : S(0);
    }
    if (threadIdx.x == 0) ok = (!failed && mbar_wait(mbar + b, (unsigned)((k / stages) & 1))) ? 1 : 0;
    __syncthreads();
    if (ok) {
      waited = k + 1;
      gemv_split(buf + (size_t)b * M * M, M, ve, z, M, M, red);
      issue(k + stages);  // buffer b is free again (gemv_split ends with a barrier)
    } else {
      failed = true;  // stop issuing; the outputs of this CTA become NaN
    }
    if (threadIdx.x < M) {
      const int i = threadIdx.x;
      const long long sl = nb_slot(e, i);
      if (sl >= 0) y[sl] = ok ? cur_nb + z[i] : (S)nan("");
      else y[e * M + i] = ve[i];
    }
    __syncthreads();
  }
  if (failed && threadIdx.x == 0) {  // bounded wait for the copies still in flight
    const long long issued = (waited + stages < nk) ? waited + stages : nk;
    for (long long k = waited; k < issued; ++k) mbar_wait(mbar + (k % stages), (unsigned)((k / stages) & 1));
  }
}


// y_p = S_p v_p for every problem p of a batch in one launch: the elements of
// all problems form one list; CTA c walks entries c, c+G, ... and streams
// their T_e (M_p^2 s bytes each, contiguous, column-major) with bulk copies
// into a shared-memory ring of `ring` bytes, as many elements in flight as
// fit (at most kRingSlots), so small elements keep as many bytes in flight
// as large ones.  Warp 0 owns the ring: its lanes load the metadata of the
// next candidate elements in parallel (one table entry each), lane 0 places
// them at the ring head in order (wrapping to the start when the tail is
// free), and each lane issues its own element's copy and stages its
// metadata in the slot, so the other warps never wait on the element table:
// one element ahead they prefetch into registers the element's own slots and
// the neighbour slots its rows feed.
constexpr int kRingSlots = 16;

template <typename S>
struct ElemMeta {
  const S* T;      // this element's T_e
  long long off;   // slot offset of the problem in the packed vectors
  int e, M, n, mx, my;
  unsigned boff;   // byte offset of the element's copy in the ring (staged copies only)
};

template <typename S>
__global__ void __launch_bounds__(256, 2) k_schur_stream_batch(const ElemMeta<S>* __restrict__ tab, long long nelem,
                                                               const S* v, S* y, unsigned ring, int Mmax) {
  extern __shared__ __align__(16) unsigned char raw[];
  const int G = gridDim.x, lane = threadIdx.x & 31;
  const bool w0 = threadIdx.x < 32;
  unsigned char* buf = raw;
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(raw + ring);
  ElemMeta<S>* meta = reinterpret_cast<ElemMeta<S>*>(mbar + kRingSlots);
  S* ve = reinterpret_cast<S*>(meta + kRingSlots);
  S* z = ve + Mmax;
  S* red = z + Mmax;
  const long long nk = (nelem - blockIdx.x + G - 1) / G;
  if (threadIdx.x == 0) {
    for (int b = 0; b < kRingSlots; ++b) mbar_init(mbar + b);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // ring state, kept identical in every lane of warp 0
  long long issued = 0;
  unsigned head = 0, tail = 0;  // [tail, head) in ring order holds unconsumed copies
  bool empty = true;
  auto refill = [&](long long consumed) {
    if (!w0) return;
    long long lim = consumed + kRingSlots;
    if (lim > nk) lim = nk;
    const int cnt = (int)(lim - issued);
    if (cnt <= 0) return;
    ElemMeta<S> em{};
    if (lane < cnt) em = tab[blockIdx.x + (issued + lane) * G];
    int placed = 0;  // candidates 0 .. placed-1 get a place, in order
    unsigned pos_mine = 0;
    for (int j = 0; j < cnt; ++j) {
      const int Mj = __shfl_sync(0xffffffffu, em.M, j);
      const unsigned need = (unsigned)(Mj * Mj * sizeof(S));
      unsigned pos;
      bool fits = true;
      if (empty) {
        pos = 0;
        head = tail = 0;
      } else if (head == tail) {
        fits = false;
      } else if (head > tail) {
        if (head + need <= ring) pos = head;
        else if (need <= tail) pos = 0;
        else fits = false;
      } else {
        if (head + need <= tail) pos = head;
        else fits = false;
      }
      if (!fits) break;
      if (lane == j) pos_mine = pos;
      head = pos + need;
      empty = false;
      ++placed;
    }
    if (lane < placed) {
      const long long k = issued + lane;
      const int b = (int)(k % kRingSlots);
      em.boff = pos_mine;
      meta[b] = em;
      const unsigned need = (unsigned)(em.M * em.M * sizeof(S));
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar + b)), "r"(need)
                   : "memory");
      bulk_g2s(buf + pos_mine, em.T + (size_t)em.e * em.M * em.M, need, mbar + b);
    }
    issued += placed;
  };
  // neighbour slot fed by row i of element (e, M, n) on an mx x my grid, or -1
  auto nb_slot = [](const ElemMeta<S>& md, int i) -> long long {
    const int F = i / md.n, t = i % md.n, ix = md.e % md.mx, iy = md.e / md.mx;
    int e2;
    switch (F) {
      case 0: e2 = ix > 0 ? md.e - 1 : -1; break;
      case 1: e2 = ix < md.mx - 1 ? md.e + 1 : -1; break;
      case 2: e2 = iy > 0 ? md.e - md.mx : -1; break;
      default: e2 = iy < md.my - 1 ? md.e + md.mx : -1; break;
    }
    return e2 >= 0 ? (long long)e2 * md.M + (F ^ 1) * md.n + t : -1;
  };
  refill(0);
  __syncthreads();  // metadata of the first copies visible
  __shared__ int ok;
  __shared__ long long nissued;
  bool failed = false;
  long long waited = 0;
  S pv_own = 0, pv_nb = 0;
  bool have_pf = false;  // pv_own / pv_nb hold the current element's entries
  if (nk > 0) {
    const ElemMeta<S> md = meta[0];
    if (threadIdx.x < md.M) {
      pv_own = v[md.off + (long long)md.e * md.M + threadIdx.x];
      const long long sl = nb_slot(md, threadIdx.x);
      pv_nb = sl >= 0 ? v[md.off + sl] : S(0);
    }
    have_pf = true;
  }
  for (long long k = 0; k < nk; ++k) {
    const int b = (int)(k % kRingSlots);
    ElemMeta<S> md = meta[b];  // staged before the previous barrier; read before the slot is reused
    const S cur_nb = pv_nb;
    const bool cur_pf = have_pf;
    if (threadIdx.x < md.M) ve[threadIdx.x] = have_pf ? pv_own : v[md.off + (long long)md.e * md.M + threadIdx.x];
    if (threadIdx.x == 0) {
      ok = (!failed && k < issued && mbar_wait(mbar + b, (unsigned)((k / kRingSlots) & 1))) ? 1 : 0;
      nissued = issued;
    }
    __syncthreads();
    have_pf = k + 1 < nissued;
    if (have_pf) {  // prefetch the next element's vector entries (its metadata is staged)
      const ElemMeta<S> m1 = meta[(k + 1) % kRingSlots];
      if (threadIdx.x < m1.M) {
        pv_own = v[m1.off + (long long)m1.e * m1.M + threadIdx.x];
        const long long sl = nb_slot(m1, threadIdx.x);
        pv_nb = sl >= 0 ? v[m1.off + sl] : S(0);
      }
    }
    if (ok) {
      waited = k + 1;
      gemv_split(reinterpret_cast<const S*>(buf + md.boff), md.M, ve, z, md.M, md.M, red);
      if (w0) {  // element k's copy is consumed: the tail moves on
        if (k + 1 < issued) tail = meta[(k + 1) % kRingSlots].boff;
        else empty = true;
      }
      refill(k + 1);
    } else {
      failed = true;
      md = tab[blockIdx.x + k * G];  // no staged copy: metadata from the table
    }
    if (threadIdx.x < md.M) {
      const int i = threadIdx.x;
      const long long sl = nb_slot(md, i);
      if (!ok) {
        y[md.off + (sl >= 0 ? sl : (long long)md.e * md.M + i)] = (S)nan("");
      } else if (sl >= 0) {
        y[md.off + sl] = (cur_pf ? cur_nb : v[md.off + sl]) + z[i];
      } else {
        y[md.off + (long long)md.e * md.M + i] = ve[i];
      }
    }
    __syncthreads();  // also publishes the metadata staged by refill
  }
  if (failed && threadIdx.x == 0)  // bounded wait for the copies still in flight
    for (long long k = waited; k < issued; ++k) mbar_wait(mbar + (k % kRingSlots), (unsigned)((k / kRingSlots) & 1));
}

// Warp-per-element variant of the batched apply: warp w of the grid takes
// elements w, w + W, ... (W warps in all).  Lane l owns rows l, l+32, l+64
// (M <= 96) and walks the columns of T_e straight from global memory (each
// column is M contiguous entries, read by the warp as coalesced 128-byte
// lines), eight columns per step so that 24 independent loads per lane are in
// flight; the element's own slots sit in a per-warp shared-memory row and
// are broadcast column by column.  No CTA barrier, no copy engine: every warp
// is an independent stream of loads, and the SM keeps many of them resident.
template <typename S>
__global__ void __launch_bounds__(256) k_schur_warp_batch(const ElemMeta<S>* __restrict__ tab, long long nelem,
                                                          const S* v, S* y) {
  __shared__ S xs[8][96];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long W = (long long)gridDim.x * (blockDim.x >> 5);
  S* x = xs[wib];
  for (long long k = (long long)blockIdx.x * (blockDim.x >> 5) + wib; k < nelem; k += W) {
    const ElemMeta<S> md = tab[k];
    const int M = md.M, n = md.n;
    const S* vp = v + md.off;
    const S* Te = md.T + (size_t)md.e * M * M;
    for (int i = lane; i < M; i += 32) x[i] = vp[(long long)md.e * M + i];
    __syncwarp();
    const bool r1 = lane + 32 < M, r2 = lane + 64 < M;
    S z0 = 0, z1 = 0, z2 = 0;
    int c = 0;
    for (; c + 8 <= M; c += 8) {
      S a0[8], a1[8], a2[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const S* col = Te + (size_t)(c + u) * M;
        a0[u] = __ldg(col + lane);
        a1[u] = r1 ? __ldg(col + lane + 32) : S(0);
        a2[u] = r2 ? __ldg(col + lane + 64) : S(0);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const S xc = x[c + u];
        z0 += a0[u] * xc;
        z1 += a1[u] * xc;
        z2 += a2[u] * xc;
      }
    }
    for (; c < M; ++c) {
      const S* col = Te + (size_t)c * M;
      const S xc = x[c];
      z0 += __ldg(col + lane) * xc;
      if (r1) z1 += __ldg(col + lane + 32) * xc;
      if (r2) z2 += __ldg(col + lane + 64) * xc;
    }
    const int ix = md.e % md.mx, iy = md.e / md.mx;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int i = lane + 32 * j;
      if (i >= M) break;
      const S zi = j == 0 ? z0 : (j == 1 ? z1 : z2);
      const int F = i / n, t = i % n;
      int e2;
      switch (F) {
        case 0: e2 = ix > 0 ? md.e - 1 : -1; break;
        case 1: e2 = ix < md.mx - 1 ? md.e + 1 : -1; break;
        case 2: e2 = iy > 0 ? md.e - md.mx : -1; break;
        default: e2 = iy < md.my - 1 ? md.e + md.mx : -1; break;
      }
      if (e2 >= 0) {
        const long long sl = md.off + (long long)e2 * M + (F ^ 1) * n + t;
        y[sl] = v[sl] + zi;
      } else {
        y[md.off + (long long)md.e * M + i] = x[i];
      }
    }
    __syncwarp();
  }
}

// Register-streamed apply with K = 2 or 4 warps per element, for element
// lists too short to give every SM enough independent warps at one warp per
// element (a single grid): warp w of the group takes columns
// [w ceil(M/K), (w+1) ceil(M/K)); lane l owns rows l, l+32, l+64 (M <= 96)
// and reads its columns of T_e straight from global memory, eight columns
// per step (24 independent loads per lane in flight).  The group's partial
// products meet in shared memory; the K warps of an element sync on a named
// barrier of their own, so element groups never wait on each other.  A CTA of
// 8 warps takes 8/K elements per step (grid-stride).
template <int K>
__device__ __forceinline__ void group_sync(int grp) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(32 * K) : "memory");
}

template <typename S, int K>
__global__ void __launch_bounds__(256) k_schur_warpk(const ElemMeta<S>* __restrict__ tab, long long nelem, const S* v,
                                                     S* y) {
  constexpr int EPC = 8 / K;  // elements per CTA step
  __shared__ S xs[EPC][96];
  __shared__ S zs[EPC][K][96];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, grp = wib / K, part = wib % K;
  for (long long base = (long long)blockIdx.x * EPC; base < nelem; base += (long long)gridDim.x * EPC) {
    const long long k = base + grp;
    const bool live = k < nelem;
    ElemMeta<S> md{};
    if (live) md = tab[k];
    const int M = md.M;
    S* x = xs[grp];
    if (live)
      for (int i = part * 32 + lane; i < M; i += 32 * K) x[i] = v[md.off + (long long)md.e * M + i];
    group_sync<K>(grp);
    if (live) {
      const S* Te = md.T + (size_t)md.e * M * M;
      const int per = (M + K - 1) / K, c0 = part * per, c1 = min(M, c0 + per);
      const bool r1 = lane + 32 < M, r2 = lane + 64 < M;
      S z0 = 0, z1 = 0, z2 = 0;
      int c = c0;
      for (; c + 8 <= c1; c += 8) {
        S a0[8], a1[8], a2[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const S* col = Te + (size_t)(c + u) * M;
          a0[u] = __ldg(col + lane);
          a1[u] = r1 ? __ldg(col + lane + 32) : S(0);
          a2[u] = r2 ? __ldg(col + lane + 64) : S(0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const S xc = x[c + u];
          z0 += a0[u] * xc;
          z1 += a1[u] * xc;
          z2 += a2[u] * xc;
        }
      }
      for (; c < c1; ++c) {
        const S* col = Te + (size_t)c * M;
        const S xc = x[c];
        z0 += __ldg(col + lane) * xc;
        if (r1) z1 += __ldg(col + lane + 32) * xc;
        if (r2) z2 += __ldg(col + lane + 64) * xc;
      }
      zs[grp][part][lane] = z0;
      if (r1) zs[grp][part][lane + 32] = z1;
      if (r2) zs[grp][part][lane + 64] = z2;
    }
    group_sync<K>(grp);
    if (live) {
      const int n = md.n, ix = md.e % md.mx, iy = md.e / md.mx;
      for (int i = part * 32 + lane; i < M; i += 32 * K) {
        S zi = zs[grp][0][i];
#pragma unroll
        for (int q = 1; q < K; ++q) zi += zs[grp][q][i];
        const int F = i / n, t = i % n;
        int e2;
        switch (F) {
          case 0: e2 = ix > 0 ? md.e - 1 : -1; break;
          case 1: e2 = ix < md.mx - 1 ? md.e + 1 : -1; break;
          case 2: e2 = iy > 0 ? md.e - md.mx : -1; break;
          default: e2 = iy < md.my - 1 ? md.e + md.mx : -1; break;
        }
        if (e2 >= 0) {
          const long long sl = md.off + (long long)e2 * M + (F ^ 1) * n + t;
          y[sl] = v[sl] + zi;
        } else {
          y[md.off + (long long)md.e * M + i] = x[i];
        }
      }
    }
    group_sync<K>(grp);
  }
}

// Register-streamed apply over an element list (M <= 96): one warp per
// element when the list gives every SM enough warps, else 2 or 4.
template <typename S>
cudaError_t launch_schur_warp(const ElemMeta<S>* tab, long long nelem, const S* v, S* y, int sms, cudaStream_t st) {
  const long long want = (long long)sms * 48;  // resident warps per SM worth keeping busy
  if (nelem >= want) {
    k_schur_warp_batch<S><<<(unsigned)sms * 8, 256, 0, st>>>(tab, nelem, v, y);
  } else if (2 * nelem >= want) {
    k_schur_warpk<S, 2><<<(unsigned)((nelem + 3) / 4), 256, 0, st>>>(tab, nelem, v, y);
  } else {
    k_schur_warpk<S, 4><<<(unsigned)((nelem + 1) / 2), 256, 0, st>>>(tab, nelem, v, y);
  }
  return cudaGetLastError();
}

// Element-class-shared apply y = S v.  On an axis-aligned uniform grid T_e
// depends only on which of the element's four faces are interfaces (at most
// 9 classes: interior, 4 edges, 4 corners), so y = v + scatter(T_c X_c) with
// X_c the M x n_c matrix of the own slots of all elements of class c: a real
// dense contraction.  One CTA per tile of up to kClassTile elements of one
// class: thread 0 stages T_c and the tile's element slot vectors in shared
// memory with 1-D bulk copies (all in flight at once, one mbarrier; plain
// loads when v is not 16-byte aligned), thread (rg, eg) accumulates rows
// rg + 16 i (i < ceil(M/16)) of elements eg + 16 j (j < 4) in registers, and
// the products go straight to the neighbours' facing slots.  HBM traffic is
// the vectors only (plus the class matrices once).  A copy that does not
// complete within the bounded wait leaves the tile's outputs NaN.
constexpr int kClassTile = 64;  // elements per CTA tile
inline size_t class_smem(int M, size_t elem) {
  return 16 + ((size_t)M * M + (size_t)(M + 16 / elem) * kClassTile) * elem;
}

template <typename S>
__global__ void __launch_bounds__(256) k_schur_class(DevGeo g, const S* __restrict__ Tcls, const int* __restrict__ tiles,
                                                     const int* __restrict__ elems, const S* __restrict__ v, S* y,
                                                     int bulk) {
  extern __shared__ __align__(16) unsigned char raw[];
  const int M = g.M, n = g.n;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(raw);
  S* Ts = reinterpret_cast<S*>(raw + 16);  // M x M column-major
  const int XS = M + 16 / (int)sizeof(S);  // element stride of Xs: 16 bytes of padding (banks, bulk alignment)
  S* Xs = Ts + (size_t)M * M;              // element-major: Xs[t * XS + k]
  const int cls = tiles[3 * blockIdx.x], start = tiles[3 * blockIdx.x + 1], cnt = tiles[3 * blockIdx.x + 2];
  const S* T = Tcls + (size_t)cls * M * M;
  __shared__ int ok;
  if (bulk) {
    // warp 0 issues the copies: lane 0 arms the mbarrier with the tile's
    // byte count, then every lane copies its own elements (their indices are
    // loaded in parallel, not one after another)
    if (threadIdx.x < 32) {
      const unsigned mm = (unsigned)(M * M * sizeof(S)), col = (unsigned)(M * sizeof(S));
      if (threadIdx.x == 0) {
        mbar_init(bar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                     "r"(mm + (unsigned)cnt * col)
                     : "memory");
        bulk_g2s(Ts, T, mm, bar);
      }
      __syncwarp();
      for (int t = threadIdx.x; t < cnt; t += 32)
        bulk_g2s(Xs + (size_t)t * XS, v + (size_t)__ldg(elems + start + t) * M, col, bar);
      if (threadIdx.x == 0) ok = mbar_wait(bar, 0) ? 1 : 0;
    }
    __syncthreads();
  } else {
    for (int i = threadIdx.x; i < M * M; i += blockDim.x) Ts[i] = T[i];
    for (int i = threadIdx.x; i < M * cnt; i += blockDim.x)
      Xs[(size_t)(i / M) * XS + i % M] = v[(size_t)elems[start + i / M] * M + i % M];
    if (threadIdx.x == 0) ok = 1;
    __syncthreads();
  }
  const int rg = threadIdx.x & 15, eg = threadIdx.x >> 4;  // 16 x 16 thread grid
  constexpr int RT = 8;                                    // rows per thread (M <= 128)
  S acc[RT][4];
#pragma unroll
  for (int i = 0; i < RT; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = S(0);
  const int nr = (M - rg + 15) / 16;
  const S* xb = Xs + (size_t)eg * XS;
  for (int k = 0; k < M; ++k) {
    S b[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = xb[(size_t)16 * j * XS + k];
#pragma unroll
    for (int i = 0; i < RT; ++i) {
      if (i < nr) {
        const S a = Ts[(size_t)k * M + rg + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a * b[j];
      }
    }
  }
  const S bad = ok ? S(0) : S(nan(""));
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int t = eg + 16 * j;
    if (t >= cnt) continue;
    const int e = elems[start + t];
#pragma unroll
    for (int i = 0; i < RT; ++i) {
      const int r = rg + 16 * i;
      if (i >= nr) continue;
      const int F = r / n, tt = r % n, e2 = dev_neighbour(g, e, F);
      if (e2 >= 0) {
        const size_t sl = (size_t)e2 * M + (F ^ 1) * n + tt;
        y[sl] = v[sl] + acc[i][j] + bad;
      } else {
        y[(size_t)e * M + r] = Xs[(size_t)t * XS + r] + bad;
      }
    }
  }
}

template <typename S>
inline size_t schur_stream_batch_smem(unsigned ring, int Mmax) {
  return ring + kRingSlots * (8 + sizeof(ElemMeta<S>)) + (2 * (size_t)Mmax + 256) * sizeof(S) + 64;
}

inline size_t schur_stream_smem(int M, int stages, size_t elem) {
  return (size_t)stages * M * M * elem + stages * 8 + (2 * (size_t)M + 256) * elem + 64;
}

// ------------------------------------------------------------- host side
inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

// ===================================================================== handle
struct smpm_handle_s {
  Geometry g;
  smpm_opts opts{};
  bool factored = false;
  bool op_factored = false;  // operator-only factor step (SMPM_FLAG_OPERATOR_ONLY): S can be applied
  // element classes (face-type masks) for the class-shared apply
  int ncls = 0, ntiles = 0, cls_ok = 0;  // cls_ok: the kernel's shared-memory limit is set
  int apply_kind = 0;                     // kernel of smpm_apply_schur(32): SMPM_APPLY_*
  double* dTcls = nullptr;   // ncls * M*M, column-major
  float* dTcls32 = nullptr;
  int* dtiles = nullptr;     // ntiles * (class, first, count) into dclsel
  int* dclsel = nullptr;     // nel: elements sorted by class
  double* dHT = nullptr;     // H column-major, for the fused coarse solve of the Arnoldi steps
  double* wchatd = nullptr;  // 2 d: its two c_hat buffers
  Factors f;
  DevGeo dg{};
  // device factors
  double *dT = nullptr, *dRs = nullptr, *dG = nullptr, *dX = nullptr, *dH = nullptr;
  double *dfdx = nullptr, *dfdy = nullptr, *dD = nullptr;
  double *dcgeo = nullptr, *drgeo = nullptr;  // per column / row: tau, p, 2/h
  double *dzw = nullptr, *dzwa = nullptr;      // deflation weights (graded grids), forward / adjoint
  double *duL = nullptr, *duS = nullptr, *duC = nullptr, *dwhat = nullptr;
  int *dblack = nullptr, *dwhite = nullptr;
  // workspace
  double *wb = nullptr, *wbS = nullptr, *wV = nullptr, *wt = nullptr, *wy = nullptr, *ww = nullptr;
  double *wx = nullptr, *wrg = nullptr, *wtmp = nullptr;
  double *wc = nullptr, *wchat = nullptr, *wcb = nullptr, *wchatb = nullptr;
  double* wpart = nullptr;
  unsigned* wcnt = nullptr;
  unsigned* wbar = nullptr;
  int* werr = nullptr;
  GState* wgs = nullptr;
  struct {
    int grid = 0, nown_b = 0, nown_w = 0, ES = 0, mats_smem = 0, basis_smem = 0, stream_mats = 0, buf_elems = 0,
        nbuf = 2, warp_elems = 0;
    size_t smem = 0, smem_pp = 0;
  } gm;  // launch shape of the persistent GMRES kernel
  double* wvown = nullptr;
  double* wacc = nullptr;
  // mixed precision: FP32 operator copies and work vectors, FP64 residual
  float *dT32 = nullptr, *dG32 = nullptr, *dX32 = nullptr, *dRs32 = nullptr;
  float* dH32 = nullptr;  // FP32 copy of the coarse inverse, for the FP32 inner solves
  float *wx32 = nullptr, *wt32 = nullptr, *wy32 = nullptr, *wV32 = nullptr, *wrg32 = nullptr, *wvown32 = nullptr;
  double *wr = nullptr, *wcr = nullptr, *wrn = nullptr;
  int *wdone = nullptr, *wnref = nullptr;
  struct {
    int basis_smem = 0, mats_smem = 0, stream_mats = 0, buf_elems = 0, nbuf = 2, warp_elems = 0;
    size_t smem = 0, smem_ref = 0;
  } gm32;
  double *wacc8 = nullptr, *wxs = nullptr, *dZtuS = nullptr;
  // transposed system for the adjoint solve (SMPM_FLAG_ADJOINT)
  double *dTa = nullptr, *dRsa = nullptr, *dGa = nullptr, *dXa = nullptr, *dHa = nullptr;
  // element tables of the register-streamed apply (k_schur_warp_batch / k_schur_warpk)
  ElemMeta<double>* dtab64 = nullptr;
  ElemMeta<float>* dtab32 = nullptr;
  double *dfdxT = nullptr, *dfdyT = nullptr, *duSa = nullptr, *dZtuSa = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // bracket the GMRES kernel of each solve
  cudaEvent_t evp = nullptr, evq = nullptr;  // start of k_pre, end of k_post
  unsigned char* wctl = nullptr;              // [bar x4 | err | pad | acc8] zeroed per solve
  long long* wtrace = nullptr;                // phase trace buffer (SMPM_TRACE set)
  // staging for the host-pointer entry point
  double *sf = nullptr, *sg = nullptr, *su = nullptr;
  size_t sf_n = 0;
  std::vector<void*> allocs;
  long long launches = 0;  // kernels launched by this handle (for reports)
  // lockstep solves of several right-hand sides (allocated on first use, for
  // up to `cap` columns): per-column pre/post state and GMRES vectors,
  // basis, w/w2, column reports and the launch shape
  struct {
    int cap = 0, RC = 1, mats_smem = 0;
    size_t smem = 0;
    double *b = nullptr, *bS = nullptr, *rg = nullptr, *cb = nullptr, *chatb = nullptr, *xs = nullptr;
    double *x = nullptr, *t = nullptr, *y = nullptr, *vg = nullptr, *c = nullptr, *chat = nullptr;
    double *V = nullptr, *W = nullptr, *acc = nullptr, *Rh = nullptr, *yv = nullptr;
    LockColState* cs = nullptr;
    unsigned char* ctl = nullptr;  // barrier counters | err | per column: acc8, done, nref, rn
    PrePostArgs* dP = nullptr;     // 2 cap argument blocks (pre, post)
    // mixed precision: FP32 inner vectors and basis, Z^T r per column,
    // refinement arguments (kMaxRefine cap)
    bool has32 = false;
    float *x32 = nullptr, *t32 = nullptr, *y32 = nullptr, *vg32 = nullptr, *rg32 = nullptr;
    float *V32 = nullptr, *W32 = nullptr;
    double* cr = nullptr;
    RefineArgs* dR = nullptr;
    std::vector<RefineArgs> hR;
    std::vector<PrePostArgs> hP;
    std::vector<LockColState> hcs;
    std::vector<double> hacc;
    std::vector<void*> allocs;
  } lk;
};

namespace {

smpm_status fail(smpm_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

// No C++ exception crosses the C ABI: every entry point that returns a
// status catches what the standard library throws (a failed host
// allocation, e.g. the dense d x d coarse matrix of a very large grid, or a
// container asked for more than it can hold) and reports it as ENOMEM.
smpm_status host_exception() {
  try {
    throw;
  } catch (const std::bad_alloc&) {
    return fail(SMPM_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(SMPM_ENOMEM, std::string("host error: ") + e.what());
  } catch (...) {
    return fail(SMPM_ENOMEM, "unknown host error");
  }
}

#define CU(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return fail(e_ == cudaErrorMemoryAllocation ? SMPM_ENOMEM : SMPM_ECUDA,                     \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                            \
  } while (0)

#define CHECK_LAUNCH()    \
  do {                    \
    ++h->launches;        \
    CU(cudaGetLastError()); \
  } while (0)

template <typename P>
smpm_status dalloc(smpm_handle h, P** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(P) + 16);
  if (e != cudaSuccess) return fail(SMPM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  h->allocs.push_back(q);
  *p = static_cast<P*>(q);
  return SMPM_OK;
}

template <typename P>
smpm_status upload(smpm_handle h, P** p, const std::vector<P>& src, cudaStream_t st) {
  smpm_status s = dalloc(h, p, src.size() ? src.size() : 1);
  if (s != SMPM_OK) return s;
  if (!src.empty()) CU(cudaMemcpyAsync(*p, src.data(), src.size() * sizeof(P), cudaMemcpyHostToDevice, st));
  return SMPM_OK;
}

void free_lock(smpm_handle h) {
  for (void* p : h->lk.allocs) cudaFree(p);
  h->lk.allocs.clear();
  h->lk.cap = 0;
  h->lk.has32 = false;
}

// Frees every device allocation and event of the handle and resets all of
// its device state (pointers, launch shapes, staging sizes) to the state of
// a fresh handle, keeping the geometry and the launch count: no pointer of an
// earlier factor step survives a re-factor with other options.
void free_all(smpm_handle h) {
  free_lock(h);
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  for (cudaEvent_t* ev : {&h->ev0, &h->ev1, &h->evp, &h->evq}) {
    if (*ev) cudaEventDestroy(*ev);
    *ev = nullptr;
  }
  const Geometry g = h->g;
  const smpm_opts opts = h->opts;
  const long long launches = h->launches;
  *h = smpm_handle_s();
  h->g = g;
  h->opts = opts;
  h->launches = launches;
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

// Raise a kernel's dynamic shared-memory limit to the device maximum minus
// its static shared memory.  The limit belongs to the kernel, shared by every
// handle of the process, so it is never lowered to one handle's size.
template <typename K>
cudaError_t set_smem_limit(K* fn, int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, (const void*)fn);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}

// count square blocks of size b x b, each transposed (row-major -> column-major)
std::vector<double> transpose_blocks(const std::vector<double>& src, int b, size_t count) {
  std::vector<double> out(src.size());
  for (size_t k = 0; k < count; ++k)
    for (int i = 0; i < b; ++i)
      for (int j = 0; j < b; ++j) out[k * b * b + (size_t)j * b + i] = src[k * b * b + (size_t)i * b + j];
  return out;
}

size_t elem_smem(int n) { return 3 * (size_t)n * n * sizeof(double); }

// ---- operator launches (FP64) ----------------------------------------
template <typename S>
smpm_status launch_schur_stream(smpm_handle h, const S* T, const S* v, S* y, cudaStream_t st) {
  const DevGeo& g = h->dg;
  int dev = 0, sms = 0, optin = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // two CTAs per SM when at least two stages fit in half the SM's shared
  // memory, else one CTA with as many stages as fit (at most 8)
  int per_sm_smem = 0;
  CU(cudaDeviceGetAttribute(&per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  int cps = 2, stages = 8;
  while (stages > 1 && 2 * (schur_stream_smem(g.M, stages, sizeof(S)) + 1024) > (size_t)per_sm_smem) --stages;
  if (stages < 2) {
    cps = 1;
    stages = 8;
    while (stages > 1 && schur_stream_smem(g.M, stages, sizeof(S)) > (size_t)optin) --stages;
  }
  const size_t smem = schur_stream_smem(g.M, stages, sizeof(S));
  if (smem > (size_t)optin) {  // one matrix does not fit: per-element kernel from global memory
    k_schur<S><<<(unsigned)g.nel, kElemThreads, 2 * g.M * sizeof(S), st>>>(g, T, v, y);
    CHECK_LAUNCH();
    return SMPM_OK;
  }
  CU(set_smem_limit(k_schur_stream<S>, optin));
  const unsigned grid = (unsigned)std::min<long long>((long long)sms * cps, g.nel);
  k_schur_stream<S><<<grid, kElemThreads, smem, st>>>(g, T, v, y, stages);
  CHECK_LAUNCH();
  return SMPM_OK;
}

template <typename S>
smpm_status launch_schur_class(smpm_handle h, const S* T, const S* v, S* y, cudaStream_t st);

// Whether apply kernel kind (SMPM_APPLY_*) can run on h's grid.
bool apply_kind_ok(smpm_handle h, int kind, bool fp32) {
  switch (kind) {
    case SMPM_APPLY_AUTO: case SMPM_APPLY_STREAM: return true;
    case SMPM_APPLY_WARP: case SMPM_APPLY_WARP2: case SMPM_APPLY_WARP4:
      return h->g.M <= 96 && (fp32 ? h->dtab32 != nullptr : h->dtab64 != nullptr);
    case SMPM_APPLY_CLASS: return h->cls_ok && (fp32 ? h->dTcls32 != nullptr : h->dTcls != nullptr);
    default: return false;
  }
}

// y = S v with the handle's apply kernel (SMPM_APPLY_AUTO: one warp per
// element, register-streamed from global memory, for M <= 96 -- 1, 2 or 4
// elements per warp by the element count -- else the shared-memory stream).
template <typename S>
smpm_status launch_schur_kind(smpm_handle h, int kind, const S* v, S* y, cudaStream_t st) {
  const bool fp32 = sizeof(S) == 4;
  const ElemMeta<S>* tab = reinterpret_cast<const ElemMeta<S>*>(fp32 ? (const void*)h->dtab32 : (const void*)h->dtab64);
  const S* T = reinterpret_cast<const S*>(fp32 ? (const void*)h->dT32 : (const void*)h->dT);
  if (kind == SMPM_APPLY_AUTO) kind = apply_kind_ok(h, SMPM_APPLY_WARP, fp32) ? -1 : SMPM_APPLY_STREAM;
  if (kind == SMPM_APPLY_STREAM) return launch_schur_stream<S>(h, T, v, y, st);
  if (kind == SMPM_APPLY_CLASS) {
    const S* Tc = reinterpret_cast<const S*>(fp32 ? (const void*)h->dTcls32 : (const void*)h->dTcls);
    return launch_schur_class<S>(h, Tc, v, y, st);
  }
  int dev = 0, sms = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const long long ne = h->g.nel;
  if (kind == -1) {
    CU(launch_schur_warp<S>(tab, ne, v, y, sms, st));
  } else if (kind == SMPM_APPLY_WARP) {
    k_schur_warp_batch<S><<<(unsigned)sms * 8, 256, 0, st>>>(tab, ne, v, y);
  } else if (kind == SMPM_APPLY_WARP2) {
    k_schur_warpk<S, 2><<<(unsigned)((ne + 3) / 4), 256, 0, st>>>(tab, ne, v, y);
  } else {
    k_schur_warpk<S, 4><<<(unsigned)((ne + 1) / 2), 256, 0, st>>>(tab, ne, v, y);
  }
  CU(cudaGetLastError());
  ++h->launches;
  return SMPM_OK;
}

smpm_status launch_schur(smpm_handle h, const double* v, double* y, cudaStream_t st) {
  return launch_schur_kind<double>(h, h->apply_kind, v, y, st);
}

// t = M^-1 v (t fully written), then optionally y = S t and c = Z^T y.
smpm_status launch_precond(smpm_handle h, const double* v, double* t, double* y, double* c, cudaStream_t st) {
  const DevGeo& g = h->dg;
  const unsigned nb = (unsigned)h->f.black.size(), nw = (unsigned)h->f.white.size();
  if (nw > 0) CU(cudaMemsetAsync(t, 0, g.kp * sizeof(double), st));  // white boundary slots
  k_black<double><<<nb, kElemThreads, 5 * g.M * sizeof(double), st>>>(g, h->dblack, h->dT, h->dG, h->dX, v, t);
  CHECK_LAUNCH();
  if (y) {
    CU(cudaMemsetAsync(y, 0, g.kp * sizeof(double), st));  // black boundary slots
    if (nw > 0) {
      k_white<double><<<nw, kElemThreads, (3 * g.M + 2) * sizeof(double), st>>>(g, h->dwhite, h->dT, v, t, y, c);
      CHECK_LAUNCH();
    }
  }
  return SMPM_OK;
}

smpm_status launch_zt(smpm_handle h, const double* v, double* c, cudaStream_t st) {
  const DevGeo& g = h->dg;
  k_zt<double><<<blocks_for(g.d, 128), 128, 0, st>>>(g, v, c);
  CHECK_LAUNCH();
  return SMPM_OK;
}

smpm_status launch_coarse(smpm_handle h, const double* c, double* chat, cudaStream_t st) {
  const DevGeo& g = h->dg;
  k_coarse<<<blocks_for(g.d * 32, 256), 256, 0, st>>>(h->dH, c, chat, (int)g.d);
  CHECK_LAUNCH();
  return SMPM_OK;
}

// w = y - S Z chat (chat may be null: w = y); nvec >= 0 also runs the first
// Gram-Schmidt pass against V[0..nvec).
smpm_status launch_defl(smpm_handle h, const double* y, const double* chat, int nvec, double* w, cudaStream_t st) {
  const DevGeo& g = h->dg;
  k_defl_dots<double><<<blocks_for(g.kp, kSlotsPerBlock), kSlotsPerBlock, 0, st>>>(
      g, y, chat, h->dRs, h->wV, nvec, w, h->wpart, h->wcnt, h->wgs);
  CHECK_LAUNCH();
  return SMPM_OK;
}

// SMPM_TRACE: per-tag mean SM cycles between consecutive trace points of CTA 0.
smpm_status print_trace(smpm_handle h, cudaStream_t st) {
  std::vector<long long> tr(kTraceCap + 4, 0);
  CU(cudaMemcpyAsync(tr.data(), h->wtrace, kTraceCap * sizeof(long long), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  double sum[80] = {0};
  long long cnt[80] = {0};
  // three regions: the GMRES kernel from 0, the pre kernel from cap/2, the
  // post kernel from 3 cap/4
  for (int r0 : {0, kTraceCap / 2, 3 * (kTraceCap / 4)}) {
    const int r1 = r0 == 0 ? kTraceCap / 2 : r0 + kTraceCap / 4;
    for (int i = r0; i + 3 < r1 && tr[i + 2] != 0; i += 2) {
      int tag = (int)tr[i];
      if (tag >= 0 && tag < 80) {
        sum[tag] += (double)(tr[i + 3] - tr[i + 1]);
        cnt[tag] += 1;
      }
    }
  }
  std::fprintf(stderr, "[smpm trace] mean SM cycles from tag to next trace point (CTA 0)\n");
  for (int t = 0; t < 80; ++t)
    if (cnt[t]) std::fprintf(stderr, "  tag %2d  n %5lld  cycles %10.0f\n", t, cnt[t], sum[t] / cnt[t]);
  CU(cudaMemsetAsync(h->wtrace, 0, kTraceCap * sizeof(long long), st));
  return SMPM_OK;
}

// Shared-memory layout of the owned data of the GMRES kernel, in order of
// preference: resident matrices + basis; streamed matrices (two bulk-copy
// buffers) + basis; streamed matrices with the basis in global memory; all
// global.
struct Layout {
  int basis_smem, mats_smem, stream_mats, buf_elems, nbuf, warp_elems;
  size_t smem;
};

template <typename S>
Layout choose_layout(const Geometry& g, int m, int ES, int nown_b, int nown_w, int precond, bool no_smem,
                     bool force_stream, int smem_optin, bool w_global = false, bool warp = false) {
  Layout L;
  L.warp_elems = warp ? 1 : 0;  // warps read their matrices resident or from global memory: no stream
  L.buf_elems = g.M * g.M + 4 * g.n * g.n;
  L.basis_smem = no_smem ? 0 : 1;
  L.mats_smem = (no_smem || force_stream) ? 0 : 1;
  L.stream_mats = 0;
  L.nbuf = 2;
  auto need = [&]() {
    return gmres_smem_bytes<S>(m, g.M, g.n, ES, nown_b, nown_w, L.basis_smem, L.mats_smem, g.d,
                               L.stream_mats ? L.buf_elems : 0, w_global, L.nbuf, warp);
  };
  if (need() > (size_t)smem_optin) L.mats_smem = 0;
  if (!L.mats_smem && !no_smem && precond > 0 && !warp) {
    L.stream_mats = 1;
    if (need() > (size_t)smem_optin) L.basis_smem = 0;
    if (need() > (size_t)smem_optin) L.stream_mats = 0;
  }
  if (need() > (size_t)smem_optin) L.basis_smem = 0;
  if (L.stream_mats)  // deepest stream that fits: nbuf - 1 copies in flight during each item
    while (L.nbuf < kMaxStreamBufs) {
      ++L.nbuf;
      if (need() > (size_t)smem_optin) {
        --L.nbuf;
        break;
      }
    }
  L.smem = need();
  return L;
}

// Kernel arguments shared by the three cooperative kernels of a solve
// (adj: the operator of the slot-swapped transposed system).
GmresArgs<double> gmres_args(smpm_handle h, double tol, bool adj = false) {
  GmresArgs<double> a{};
  a.g = h->dg;
  a.black = h->dblack;
  a.white = h->dwhite;
  a.nblack = (int)h->f.black.size();
  a.nwhite = (int)h->f.white.size();
  a.Tc = h->dT; a.Gc = h->dG; a.Xc = h->dX; a.Rs = h->dRs; a.H = h->dH;
  if (adj) { a.Tc = h->dTa; a.Gc = h->dGa; a.Xc = h->dXa; a.Rs = h->dRsa; a.H = h->dHa; a.g.zw = h->dzwa; }
  a.vglob = h->wV; a.vown = h->wvown; a.t = h->wt; a.y = h->wy;
  a.c = h->wc; a.chat = h->wchat; a.rhs = h->wrg; a.x = h->wx;
  a.acc = h->wacc; a.gs = h->wgs; a.bar = h->wbar; a.err = h->werr;
  a.precond = h->opts.precond; a.m = h->opts.restart; a.maxit = h->opts.maxit; a.tol = tol;
  a.nown_b = h->gm.nown_b; a.nown_w = h->gm.nown_w; a.ES = h->gm.ES;
  a.mats_smem = h->gm.mats_smem; a.basis_smem = h->gm.basis_smem;
  a.stream_mats = h->gm.stream_mats; a.buf_elems = h->gm.buf_elems; a.nbuf = h->gm.nbuf;
  a.warp_elems = h->gm.warp_elems;
  a.trace = h->wtrace;
  a.trace_cap = h->wtrace ? kTraceCap / 2 : 0;
  a.skip = nullptr;
  a.G = h->gm.grid;
  a.base = 0;
  a.fused = (!adj && h->dHT) ? 1 : 0;
  a.HT = adj ? nullptr : h->dHT;
  a.chatd = h->wchatd;
  return a;
}

GmresArgs<float> gmres_args32(smpm_handle h, double tol) {
  GmresArgs<float> a{};
  a.g = h->dg;
  a.black = h->dblack;
  a.white = h->dwhite;
  a.nblack = (int)h->f.black.size();
  a.nwhite = (int)h->f.white.size();
  a.Tc = h->dT32; a.Gc = h->dG32; a.Xc = h->dX32; a.Rs = h->dRs32; a.H = h->dH32;
  a.vglob = h->wV32; a.vown = h->wvown32; a.t = h->wt32; a.y = h->wy32;
  a.c = h->wc; a.chat = h->wchat; a.rhs = h->wrg32; a.x = h->wx32;
  a.acc = h->wacc; a.gs = h->wgs; a.bar = h->wbar; a.err = h->werr;
  a.precond = h->opts.precond; a.m = h->opts.restart; a.maxit = h->opts.restart; a.tol = tol;
  a.nown_b = h->gm.nown_b; a.nown_w = h->gm.nown_w; a.ES = h->gm.ES;
  a.mats_smem = h->gm32.mats_smem; a.basis_smem = h->gm32.basis_smem;
  a.stream_mats = h->gm32.stream_mats; a.buf_elems = h->gm32.buf_elems; a.nbuf = h->gm32.nbuf;
  a.warp_elems = h->gm32.warp_elems;
  a.trace = nullptr;
  a.trace_cap = 0;
  a.skip = h->wdone;
  a.G = h->gm.grid;
  a.base = 0;
  a.fused = h->dHT ? 1 : 0;
  a.HT = h->dHT;
  a.chatd = h->wchatd;
  return a;
}

// Arguments of k_pre / k_post for one solve (mixed: also the FP32 buffers
// that k_pre clears; adj: the transposed system).  The all-global layout.
PrePostArgs prepost_args(smpm_handle h, double tol, const double* f, const double* gn, double* u, bool mixed,
                         bool adj = false, double* gg = nullptr) {
  const int m = h->opts.restart;
  PrePostArgs P{};
  P.ga = gmres_args(h, tol, adj);
  P.ga.mats_smem = 0;
  P.ga.basis_smem = 0;
  P.ga.stream_mats = 0;
  P.ga.warp_elems = 0;  // the pre/post kernels' shared memory has no per-warp scratch
  P.ga.trace = nullptr;
  P.fdx = h->dfdx; P.fdy = h->dfdy; P.D = h->dD; P.uL = h->duL; P.uS = h->duS; P.what = h->dwhat;
  P.ZtuS = h->dZtuS; P.f = f; P.gn = gn; P.b = h->wb; P.bS = h->wbS; P.rg = h->wrg; P.cb = h->wcb;
  P.chatb = h->wchatb; P.xs = h->wxs; P.u = u; P.acc = h->wacc8;
  double* zs[7] = {h->wx, h->wt, h->wy, h->wV, h->wbS, h->wrg, h->wxs};
  for (int i = 0; i < 7; ++i) P.zero[i] = zs[i];
  P.gacc = h->wacc;
  P.gacc_n = (long long)(2 * m + 1) * (m + 3);
  if (mixed) {
    float* z32[4] = {h->wx32, h->wt32, h->wy32, h->wV32};
    for (int i = 0; i < 4; ++i) P.zero32[i] = z32[i];
    P.cr = h->wcr;
    P.rg32 = h->wrg32;
  }
  if (adj) {
    P.adjoint = 1;
    P.gg = gg;
    P.gn = nullptr;
    P.fdx = h->dfdxT; P.fdy = h->dfdyT; P.uS = h->duSa; P.ZtuS = h->dZtuSa;
  }
  return P;
}

// Arguments of one refinement step after the inner solve with arguments a.
RefineArgs refine_args(smpm_handle h, const GmresArgs<float>& a, double tol) {
  RefineArgs RA{};
  RA.ga = a;
  RA.ga.mats_smem = 0;
  RA.ga.basis_smem = 0;
  RA.ga.stream_mats = 0;
  RA.ga.rhs = h->wrg32;
  RA.Tc64 = h->dT;
  RA.Rs64 = h->dRs;
  RA.xS = h->wxs;
  RA.bS = h->wbS;
  RA.r = h->wr;
  RA.cr = h->wcr;
  RA.chat_r = h->wchatb;
  RA.rgn = h->wacc8 + ACC_RGN;
  RA.rn = h->wrn;
  RA.done = h->wdone;
  RA.nref = h->wnref;
  RA.rhs32 = h->wrg32;
  RA.tol = tol;
  return RA;
}

// One right-hand side, FP32 inner GMRES inside FP64 iterative refinement
// (GMRES-IR): k_pre, then kMaxRefine pairs (k_gmres<float>, k_refine) that
// return at once after convergence, then k_post on the assembled x_S.
smpm_status solve_one_mixed(smpm_handle h, const double* f, const double* gn, double* u, double tol,
                            smpm_report* rep, cudaStream_t st) {
  const int m = h->opts.restart;
  smpm_report R{};
  const long long launches0 = h->launches;
  CU(cudaMemsetAsync(h->wctl, 0, kCtlBytes, st));
  PrePostArgs P = prepost_args(h, tol, f, gn, u, true);
  CU(cudaEventRecord(h->evp, st));
  {
    P.ga.bar = h->wbar + 0;
    void* args[] = {&P};
    CU(cudaLaunchCooperativeKernel((const void*)k_pre, dim3(h->gm.grid), dim3(kGmresThreads), args, h->gm.smem_pp,
                                   st));
    CHECK_LAUNCH();
  }
  CU(cudaEventRecord(h->ev0, st));
  for (int ref = 0; ref < kMaxRefine; ++ref) {
    GmresArgs<float> a = gmres_args32(h, kInnerTol);
    a.bar = h->wbar + 2 + 2 * ref;
    a.its_out = reinterpret_cast<int*>(h->wctl + 592) + ref;
    if (ref == 0 && h->wtrace) {
      a.trace = h->wtrace;
      a.trace_cap = kTraceCap / 2;
    }
    {
      void* args[] = {&a};
      CU(cudaLaunchCooperativeKernel((const void*)k_gmres<float>, dim3(h->gm.grid), dim3(kGmresThreads), args,
                                     h->gm32.smem, st));
      CHECK_LAUNCH();
    }
    RefineArgs RA = refine_args(h, a, tol);
    RA.ga.bar = h->wbar + 3 + 2 * ref;
    RA.rn = h->wrn + ref;
    void* args[] = {&RA};
    CU(cudaLaunchCooperativeKernel((const void*)k_refine, dim3(h->gm.grid), dim3(kGmresThreads), args,
                                   h->gm32.smem_ref, st));
    CHECK_LAUNCH();
  }
  CU(cudaEventRecord(h->ev1, st));
  {
    P.ga.bar = h->wbar + 1;
    P.assembled = 1;
    void* args[] = {&P};
    CU(cudaLaunchCooperativeKernel((const void*)k_post, dim3(h->gm.grid), dim3(kGmresThreads), args, h->gm.smem_pp,
                                   st));
    CHECK_LAUNCH();
    CU(cudaEventRecord(h->evq, st));
  }
  int herr = 0, done = 0, nref = 0;
  double acc8[8], rn[32], scal[8];
  CU(cudaMemcpyAsync(&herr, h->werr, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(&done, h->wdone, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(&nref, h->wnref, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(acc8, h->wacc8, sizeof(acc8), cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(rn, h->wrn, sizeof(rn), cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(scal, reinterpret_cast<char*>(h->wgs) + offsetof(GState, scal), sizeof(scal),
                     cudaMemcpyDeviceToHost, st));
  int its[32];
  CU(cudaMemcpyAsync(its, h->wctl + 592, sizeof(its), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (herr) return fail(SMPM_ETIMEOUT, "a grid barrier or copy wait of the solve kernels timed out");
  if (h->wtrace) {
    std::fprintf(stderr, "[smpm trace] refinement rounds:");
    for (int i = 0; i < nref && i < 32; ++i)
      std::fprintf(stderr, " (%d inner, |r|^2 %.3e)", its[i], rn[i]);
    std::fprintf(stderr, "  |P b_S|^2 %.3e\n", acc8[ACC_RGN]);
    print_trace(h, st);
  }
  R.iterations = (int)scal[5];
  R.refinements = nref;
  R.converged = done ? 1 : 0;
  const double rho = nref > 0 ? std::sqrt(rn[nref - 1]) : 0.0;
  R.gmres_relres = acc8[ACC_RGN] > 0 ? rho / std::sqrt(acc8[ACC_RGN]) : 0.0;
  R.schur_relres = acc8[ACC_BSN] > 0 ? std::sqrt(acc8[ACC_RES] / acc8[ACC_BSN]) : 0.0;
  if (!std::isfinite(R.gmres_relres) || !std::isfinite(R.schur_relres))
    return fail(SMPM_ENAN, "non-finite value in the right-hand side or the refinement");
  {
    float ms = 0;
    CU(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    R.gmres_ms = ms;
    CU(cudaEventElapsedTime(&ms, h->evp, h->ev0));
    R.pre_ms = ms;
    CU(cudaEventElapsedTime(&ms, h->ev1, h->evq));
    R.post_ms = ms;
  }
  R.launches = (int)(h->launches - launches0);
  if (rep) *rep = R;
  if (!done && acc8[ACC_RGN] > 0) return fail(SMPM_ENOTCONV, "iterative refinement did not reach tol");
  return SMPM_OK;
}

// One right-hand side, FP64, Algorithms 1-3: three cooperative launches
// (k_pre, k_gmres, k_post) and one host synchronisation for the report.
// adj: the transposed solve on the adjoint factors (f = dl/du, u = dl/db,
// gg = dl/dg or null), always FP64.
smpm_status solve_one(smpm_handle h, const double* f, const double* gn, double* u, double tol, smpm_report* rep,
                      cudaStream_t st, bool adj = false, double* gg = nullptr) {
  if (h->opts.precision == 1 && !adj) return solve_one_mixed(h, f, gn, u, tol, rep, st);
  const int m = h->opts.restart;
  smpm_report R{};
  const long long launches0 = h->launches;
  // one memset per solve: barrier counters of the three kernels, error flag,
  // pre/post accumulators (contiguous); everything else is zeroed in k_pre
  CU(cudaMemsetAsync(h->wctl, 0, kCtlBytes, st));
  PrePostArgs P = prepost_args(h, tol, f, gn, u, false, adj, gg);
  P.ga.bar = h->wbar + 0;
  if (h->wtrace) {  // pre and post trace into the upper halves of the buffer
    P.ga.trace = h->wtrace + kTraceCap / 2;
    P.ga.trace_cap = kTraceCap / 4;
  }
  {
    void* args[] = {&P};
    CU(cudaEventRecord(h->evp, st));
    CU(cudaLaunchCooperativeKernel((const void*)k_pre, dim3(h->gm.grid), dim3(kGmresThreads), args, h->gm.smem_pp,
                                   st));
    CHECK_LAUNCH();
  }
  CU(cudaEventRecord(h->ev0, st));
  {
    GmresArgs<double> a = gmres_args(h, tol, adj);
    a.bar = h->wbar + 1;
    void* args[] = {&a};
    CU(cudaLaunchCooperativeKernel((const void*)k_gmres<double>, dim3(h->gm.grid), dim3(kGmresThreads), args,
                                   h->gm.smem, st));
    CHECK_LAUNCH();
  }
  CU(cudaEventRecord(h->ev1, st));
  {
    P.ga.bar = h->wbar + 2;
    if (h->wtrace) P.ga.trace = h->wtrace + 3 * (kTraceCap / 4);
    void* args[] = {&P};
    CU(cudaLaunchCooperativeKernel((const void*)k_post, dim3(h->gm.grid), dim3(kGmresThreads), args, h->gm.smem_pp,
                                   st));
    CHECK_LAUNCH();
    CU(cudaEventRecord(h->evq, st));
  }
  if (h->wtrace) print_trace(h, st);
  GState hs;
  int herr = 0;
  double acc8[8];
  CU(cudaMemcpyAsync(&herr, h->werr, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(acc8, h->wacc8, sizeof(acc8), cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(&hs, h->wgs, offsetof(GState, g), cudaMemcpyDeviceToHost, st));
  double scal[8];
  CU(cudaMemcpyAsync(scal, reinterpret_cast<char*>(h->wgs) + offsetof(GState, scal), sizeof(scal),
                     cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (herr) return fail(SMPM_ETIMEOUT, "a grid barrier of the solve kernels timed out");
  if (hs.nan) return fail(SMPM_ENAN, "non-finite value in the right-hand side or the Arnoldi process");
  R.iterations = hs.j;
  R.restarts = scal[7] > 1 ? (int)scal[7] - 1 : 0;
  // an Arnoldi breakdown before the estimate reaches tol (the Krylov space
  // became invariant to round-off, e.g. a tol below round-off on a small
  // system) is reported as EBREAKDOWN with the iterate assembled as usual
  const bool conv = hs.converged || hs.beta0 == 0.0;
  R.converged = conv ? 1 : 0;
  R.gmres_relres = hs.beta0 > 0 ? hs.resid / hs.beta0 : 0.0;
  R.schur_relres = acc8[ACC_BSN] > 0 ? std::sqrt(acc8[ACC_RES] / acc8[ACC_BSN]) : 0.0;
  {
    float ms = 0;
    CU(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    R.gmres_ms = ms;
    CU(cudaEventElapsedTime(&ms, h->evp, h->ev0));
    R.pre_ms = ms;
    CU(cudaEventElapsedTime(&ms, h->ev1, h->evq));
    R.post_ms = ms;
  }
  R.launches = (int)(h->launches - launches0);
  if (rep) *rep = R;
  if (!conv && hs.breakdown) return fail(SMPM_EBREAKDOWN, "Arnoldi breakdown before GMRES reached tol");
  if (!conv) return fail(SMPM_ENOTCONV, "GMRES did not converge within maxit");
  return SMPM_OK;
}

// ---- lockstep solves of several right-hand sides (FP64, Algorithms 2 and 3)
template <typename P>
smpm_status lalloc(smpm_handle h, P** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(P) + 16);
  if (e != cudaSuccess) return fail(SMPM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  h->lk.allocs.push_back(q);
  *p = static_cast<P*>(q);
  return SMPM_OK;
}

// control block of a lockstep solve: 32 barrier counters (pre 0, post 1,
// inner GMRES 2 + 2 ref, refinement 3 + 2 ref), err at 128; column k's block
// at kLockCtlBytes + k kLockColBytes: acc8 (8 doubles) | done, nref (ints at
// +64) | rn[kMaxRefine] at +128
constexpr size_t kLockCtlBytes = 256;  // (kLockColBytes, the column block size, is shared with the batch)

// columns per element work item: the largest of maxrc, ..., 2, 1 that
// divides R and still gives `warps` warps of a CTA an item (all warps busy:
// FP64 needs at least 4 per SM for its pipe, FP32 its loads in flight).
int lock_rc(int R, int nown_b, int maxrc, int warps) {
  for (int c = maxrc; c >= 2; c /= 2)
    if (R % c == 0 && (long long)nown_b * (R / c) >= warps) return c;
  return 1;
}

// Workspace of the lockstep kernels for up to R columns (FP32 inner buffers
// too when the handle is factored for mixed precision).
smpm_status lock_prepare(smpm_handle h, int R) {
  auto& L = h->lk;
  const bool mixed = h->opts.precision == 1;
  if (L.cap >= R && (L.has32 || !mixed)) return SMPM_OK;
  free_lock(h);
  int cap = 2;
  while (cap < R) cap *= 2;
  const Geometry& g = h->g;
  const size_t kp = g.kp, r = g.r, d = g.d, m = h->opts.restart, G = h->gm.grid, ES = h->gm.ES;
  smpm_status s;
  if ((s = lalloc(h, &L.b, cap * r)) || (s = lalloc(h, &L.bS, cap * kp)) || (s = lalloc(h, &L.rg, cap * kp)) ||
      (s = lalloc(h, &L.cb, cap * d)) || (s = lalloc(h, &L.chatb, cap * d)) || (s = lalloc(h, &L.xs, cap * kp)) ||
      (s = lalloc(h, &L.c, cap * d)) || (s = lalloc(h, &L.chat, cap * d)) ||
      (s = lalloc(h, &L.acc, (2 * m + 1) * cap * (m + 3))) || (s = lalloc(h, &L.Rh, cap * m * (m + 1))) ||
      (s = lalloc(h, &L.yv, cap * m)) || (s = lalloc(h, &L.cs, (size_t)cap)) ||
      (s = lalloc(h, &L.ctl, kLockCtlBytes + kLockColBytes * (size_t)cap)) ||
      (s = lalloc(h, &L.dP, 2 * (size_t)cap)))
    return s;
  if (!mixed) {
    if ((s = lalloc(h, &L.x, cap * kp)) || (s = lalloc(h, &L.t, cap * kp)) || (s = lalloc(h, &L.y, cap * kp)) ||
        (s = lalloc(h, &L.vg, cap * kp)) || (s = lalloc(h, &L.V, G * (m + 1) * cap * ES)) ||
        (s = lalloc(h, &L.W, G * 2 * cap * (ES + 1))))
      return s;
  } else {
    if ((s = lalloc(h, &L.x32, cap * kp)) || (s = lalloc(h, &L.t32, cap * kp)) || (s = lalloc(h, &L.y32, cap * kp)) ||
        (s = lalloc(h, &L.vg32, cap * kp)) || (s = lalloc(h, &L.rg32, cap * kp)) ||
        (s = lalloc(h, &L.V32, G * (m + 1) * cap * ES)) || (s = lalloc(h, &L.W32, G * 2 * cap * (ES + 1))) ||
        (s = lalloc(h, &L.cr, cap * d)) || (s = lalloc(h, &L.dR, (size_t)kMaxRefine * cap)))
      return s;
    L.has32 = true;
    L.hR.resize((size_t)kMaxRefine * cap);
  }
  L.cap = cap;
  L.hP.resize(2 * cap);
  L.hcs.resize(cap);
  L.hacc.resize(8 * cap);
  return SMPM_OK;
}

// Launch shape of the lockstep kernel: resident operator matrices when they fit.
template <typename S>
smpm_status lock_shape(smpm_handle h, int R, int optin, int* RC, int* mats, size_t* smem) {
  const Geometry& g = h->g;
  const int m = h->opts.restart;
  *RC = lock_rc(R, h->gm.nown_b, sizeof(S) == 4 ? 8 : 4, kGmresThreads / 32);
  *mats = 1;
  *smem = lock_smem_bytes<S>(m, g.M, g.n, R, *RC, h->gm.nown_b, h->gm.nown_w, true);
  if ((h->opts.flags & SMPM_FLAG_NO_SMEM_RESIDENCY) || *smem > (size_t)optin) {
    *mats = 0;
    *smem = lock_smem_bytes<S>(m, g.M, g.n, R, *RC, h->gm.nown_b, h->gm.nown_w, false);
  }
  if (*smem > (size_t)optin) return fail(SMPM_EINVAL, "lockstep layout does not fit in shared memory");
  CU(set_smem_limit(k_gmres_lock<S>, optin));
  return SMPM_OK;
}

// R right-hand sides of one grid in lockstep.  FP64: k_pre_cols,
// k_gmres_lock<double>, k_post_cols.  Mixed precision: k_pre_cols, then
// kMaxRefine pairs (k_gmres_lock<float>, k_refine_cols) that skip the columns
// already done, then k_post_cols on the assembled x_S.  One host
// synchronisation for the reports.
smpm_status solve_lock(smpm_handle h, const double* f, const double* gn, double* u, double tol, int R,
                       smpm_report* rep, cudaStream_t st) {
  smpm_status s;
  if ((s = lock_prepare(h, R))) return s;
  auto& L = h->lk;
  const Geometry& g = h->g;
  const bool mixed = h->opts.precision == 1;
  const long long launches0 = h->launches;
  int dev = 0, optin = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  int RC = 1, mats = 0;
  size_t smem = 0;
  if ((s = mixed ? lock_shape<float>(h, R, optin, &RC, &mats, &smem) : lock_shape<double>(h, R, optin, &RC, &mats,
                                                                                          &smem)))
    return s;
  CU(set_smem_limit(k_pre_cols, optin));
  CU(set_smem_limit(k_post_cols, optin));
  unsigned* bar = reinterpret_cast<unsigned*>(L.ctl);
  int* err = reinterpret_cast<int*>(L.ctl + 128);
  auto colblk = [&](int k) { return L.ctl + kLockCtlBytes + kLockColBytes * (size_t)k; };
  const int m = h->opts.restart;
  CU(cudaMemsetAsync(L.ctl, 0, kLockCtlBytes + kLockColBytes * (size_t)R, st));
  CU(cudaMemsetAsync(L.acc, 0, sizeof(double) * (size_t)(2 * m + 1) * R * (m + 3), st));
  CU(cudaMemsetAsync(L.cs, 0, sizeof(LockColState) * (size_t)R, st));
  // the work vectors of every column start at zero: slots on physical-boundary
  // faces are never written by the phases, but the white elements read t there
  // (times the zero columns of T_e), so they must hold zeros, not stale values
  {
    const size_t nv = (size_t)R * g.kp;
    if (!mixed) {
      for (double* v : {L.t, L.y, L.vg}) CU(cudaMemsetAsync(v, 0, nv * sizeof(double), st));
    } else {
      for (float* v : {L.t32, L.y32, L.vg32}) CU(cudaMemsetAsync(v, 0, nv * sizeof(float), st));
    }
  }
  // per-column arguments of the pre (k < R) and post (R + k) bodies
  for (int k = 0; k < R; ++k) {
    PrePostArgs P = prepost_args(h, tol, f + (size_t)k * g.r, gn ? gn + (size_t)k * g.kp : nullptr,
                                 u + (size_t)k * g.r, mixed);
    P.b = L.b + (size_t)k * g.r;
    P.bS = L.bS + (size_t)k * g.kp;
    P.rg = L.rg + (size_t)k * g.kp;
    P.cb = L.cb + (size_t)k * g.d;
    P.chatb = L.chatb + (size_t)k * g.d;
    P.xs = L.xs + (size_t)k * g.kp;
    P.acc = reinterpret_cast<double*>(colblk(k));
    P.ga.err = err;
    P.gacc = nullptr;
    P.gacc_n = 0;
    if (!mixed) {
      P.ga.x = L.x + (size_t)k * g.kp;
      double* zs[7] = {P.ga.x, h->wt, h->wy, h->wV, P.bS, P.rg, P.xs};
      for (int i = 0; i < 7; ++i) P.zero[i] = zs[i];
    } else {
      double* zs[7] = {h->wx, h->wt, h->wy, h->wV, P.bS, P.rg, P.xs};
      for (int i = 0; i < 7; ++i) P.zero[i] = zs[i];
      float* z32[4] = {L.x32 + (size_t)k * g.kp, L.t32, L.y32, L.vg32};
      for (int i = 0; i < 4; ++i) P.zero32[i] = z32[i];
      P.cr = L.cr + (size_t)k * g.d;
      P.rg32 = L.rg32 + (size_t)k * g.kp;
    }
    P.ga.bar = bar + 0;
    L.hP[k] = P;
    P.ga.bar = bar + 1;
    P.assembled = mixed ? 1 : 0;
    L.hP[R + k] = P;
  }
  CU(cudaMemcpyAsync(L.dP, L.hP.data(), 2 * R * sizeof(PrePostArgs), cudaMemcpyHostToDevice, st));
  if (mixed) {
    for (int ref = 0; ref < kMaxRefine; ++ref)
      for (int k = 0; k < R; ++k) {
        GmresArgs<float> a = gmres_args32(h, kInnerTol);
        a.x = L.x32 + (size_t)k * g.kp;
        a.t = L.t32;
        a.y = L.y32;
        a.vglob = L.vg32;
        a.rhs = L.rg32 + (size_t)k * g.kp;
        a.err = err;
        a.skip = nullptr;
        RefineArgs RA = refine_args(h, a, tol);
        RA.ga.bar = bar + 3 + 2 * ref;
        RA.xS = L.xs + (size_t)k * g.kp;
        RA.bS = L.bS + (size_t)k * g.kp;
        RA.cr = L.cr + (size_t)k * g.d;
        RA.chat_r = L.chatb + (size_t)k * g.d;
        RA.rgn = reinterpret_cast<double*>(colblk(k)) + ACC_RGN;
        RA.rn = reinterpret_cast<double*>(colblk(k) + 128) + ref;
        RA.done = reinterpret_cast<int*>(colblk(k) + 64);
        RA.nref = reinterpret_cast<int*>(colblk(k) + 68);
        RA.rhs32 = L.rg32 + (size_t)k * g.kp;
        L.hR[(size_t)ref * R + k] = RA;
      }
    CU(cudaMemcpyAsync(L.dR, L.hR.data(), (size_t)kMaxRefine * R * sizeof(RefineArgs), cudaMemcpyHostToDevice, st));
  }
  CU(cudaEventRecord(h->evp, st));
  {
    const PrePostArgs* Ps = L.dP;
    int RR = R;
    void* args[] = {&Ps, &RR};
    CU(cudaLaunchCooperativeKernel((const void*)k_pre_cols, dim3(h->gm.grid), dim3(kGmresThreads), args,
                                   h->gm.smem_pp, st));
    CHECK_LAUNCH();
  }
  CU(cudaEventRecord(h->ev0, st));
  auto lock_fields = [&](auto& A) {
    A.a.err = err;
    A.a.mats_smem = mats; A.a.basis_smem = 0; A.a.stream_mats = 0; A.a.warp_elems = 1;
    A.a.trace = nullptr; A.a.trace_cap = 0; A.a.skip = nullptr; A.a.its_out = nullptr; A.a.wscr = nullptr;
    A.a.c = L.c; A.a.chat = L.chat; A.a.acc = L.acc;
    A.R = R; A.RC = RC; A.vs = g.kp; A.ds = g.d;
    A.cs = L.cs; A.Rh = L.Rh; A.yv = L.yv;
  };
  if (!mixed) {
    LockArgs<double> A{};
    A.a = gmres_args(h, tol);
    lock_fields(A);
    A.a.rhs = L.rg; A.a.x = L.x; A.a.t = L.t; A.a.y = L.y; A.a.vglob = L.vg;
    A.a.bar = bar + 2;
    A.V = L.V; A.W = L.W;
    A.done = nullptr; A.done_stride = 0;
    if (h->wtrace) {
      A.a.trace = h->wtrace;
      A.a.trace_cap = kTraceCap / 2;
    }
    void* args[] = {&A};
    CU(cudaLaunchCooperativeKernel((const void*)k_gmres_lock<double>, dim3(h->gm.grid), dim3(kGmresThreads), args,
                                   smem, st));
    CHECK_LAUNCH();
  } else {
    CU(set_smem_limit(k_refine_cols, optin));
    for (int ref = 0; ref < kMaxRefine; ++ref) {
      LockArgs<float> A{};
      A.a = gmres_args32(h, kInnerTol);
      lock_fields(A);
      A.a.rhs = L.rg32; A.a.x = L.x32; A.a.t = L.t32; A.a.y = L.y32; A.a.vglob = L.vg32;
      A.a.bar = bar + 2 + 2 * ref;
      A.V = L.V32; A.W = L.W32;
      A.done = reinterpret_cast<const int*>(colblk(0) + 64);
      A.done_stride = (int)(kLockColBytes / sizeof(int));
      if (h->wtrace && ref == 0) {
        A.a.trace = h->wtrace;
        A.a.trace_cap = kTraceCap / 2;
      }
      {
        void* args[] = {&A};
        CU(cudaLaunchCooperativeKernel((const void*)k_gmres_lock<float>, dim3(h->gm.grid), dim3(kGmresThreads),
                                       args, smem, st));
        CHECK_LAUNCH();
      }
      {
        const RefineArgs* Rs = L.dR + (size_t)ref * R;
        int RR = R;
        void* args[] = {&Rs, &RR};
        CU(cudaLaunchCooperativeKernel((const void*)k_refine_cols, dim3(h->gm.grid), dim3(kGmresThreads), args,
                                       h->gm32.smem_ref, st));
        CHECK_LAUNCH();
      }
    }
  }
  CU(cudaEventRecord(h->ev1, st));
  {
    const PrePostArgs* Ps = L.dP + R;
    int RR = R;
    void* args[] = {&Ps, &RR};
    CU(cudaLaunchCooperativeKernel((const void*)k_post_cols, dim3(h->gm.grid), dim3(kGmresThreads), args,
                                   h->gm.smem_pp, st));
    CHECK_LAUNCH();
  }
  CU(cudaEventRecord(h->evq, st));
  int herr = 0;
  std::vector<unsigned char> hcol(kLockColBytes * (size_t)R);
  CU(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(hcol.data(), colblk(0), hcol.size(), cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(L.hcs.data(), L.cs, R * sizeof(LockColState), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (herr) return fail(SMPM_ETIMEOUT, "a grid barrier of the lockstep solve kernels timed out");
  if (h->wtrace) print_trace(h, st);
  float gms = 0, pms = 0, qms = 0;
  CU(cudaEventElapsedTime(&gms, h->ev0, h->ev1));
  CU(cudaEventElapsedTime(&pms, h->evp, h->ev0));
  CU(cudaEventElapsedTime(&qms, h->ev1, h->evq));
  smpm_status worst = SMPM_OK;
  for (int k = 0; k < R; ++k) {
    const LockColState& c = L.hcs[k];
    const unsigned char* blk = hcol.data() + kLockColBytes * (size_t)k;
    const double* a8 = reinterpret_cast<const double*>(blk);
    const int done = *reinterpret_cast<const int*>(blk + 64), nref = *reinterpret_cast<const int*>(blk + 68);
    const double* rn = reinterpret_cast<const double*>(blk + 128);
    smpm_report Rp{};
    Rp.iterations = c.its_total;
    Rp.launches = (int)(h->launches - launches0);
    Rp.gmres_ms = gms;
    Rp.pre_ms = pms;
    Rp.post_ms = qms;
    Rp.schur_relres = a8[ACC_BSN] > 0 ? std::sqrt(a8[ACC_RES] / a8[ACC_BSN]) : 0.0;
    bool conv;
    if (!mixed) {
      if (c.nan) return fail(SMPM_ENAN, "non-finite value in a right-hand side or its Arnoldi process");
      Rp.restarts = c.cycles > 1 ? c.cycles - 1 : 0;
      conv = c.converged != 0;
      Rp.gmres_relres = c.beta0 > 0 ? c.resid / c.beta0 : 0.0;
    } else {
      Rp.refinements = nref;
      conv = done != 0 || a8[ACC_RGN] == 0.0;
      const double rho = nref > 0 ? std::sqrt(rn[std::min(nref, kMaxRefine) - 1]) : 0.0;
      Rp.gmres_relres = a8[ACC_RGN] > 0 ? rho / std::sqrt(a8[ACC_RGN]) : 0.0;
      if (!std::isfinite(Rp.gmres_relres) || !std::isfinite(Rp.schur_relres))
        return fail(SMPM_ENAN, "non-finite value in a right-hand side or its refinement");
    }
    Rp.converged = conv ? 1 : 0;
    if (rep) rep[k] = Rp;
    if (!conv && worst == SMPM_OK) worst = (!mixed && c.breakdown) ? SMPM_EBREAKDOWN : SMPM_ENOTCONV;
  }
  if (worst != SMPM_OK)
    return fail(worst, worst == SMPM_EBREAKDOWN ? "Arnoldi breakdown before tol in a lockstep column"
                                                : "a lockstep column did not converge");
  return SMPM_OK;
}

}  // namespace

// ================================================================ C ABI

// ===================================================================== batch
struct smpm_batch_s {
  std::vector<smpm_handle> hs;
  std::vector<int> nrhs;
  std::vector<long long> foff, goff;  // start of problem p's block in the packed f (u) and g
  long long f_len = 0, g_len = 0, ntasks = 0;
  int grid = 0, team_size = 0, nteams = 0, use_graph = 1;
  size_t smem = 0;
  BatchTask* dtasks = nullptr;
  int *dbegin = nullptr, *dteam = nullptr, *derr = nullptr;
  unsigned* dbars = nullptr;
  BatchIO* dio = nullptr;
  TaskReport* drep = nullptr;
  BatchIO* hio = nullptr;        // pinned
  TaskReport* hrep = nullptr;    // pinned
  int* herr = nullptr;           // pinned
  std::vector<void*> allocs;     // device memory of the current team layout
  std::vector<long long> task_of;  // report index of (problem p, rhs k): task_of[foff-like prefix]
  std::vector<long long> task_col; // first right-hand side (report index) of each task
  std::vector<long long> rhs_base;
  cudaStream_t bs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaEvent_t ein = nullptr, eout = nullptr;
  float last_ms = 0;
  // batched apply y_p = S_p v_p: element list and per-problem tables
  ElemMeta<double>* dtab64 = nullptr;
  ElemMeta<float>* dtab32 = nullptr;  // null unless every handle has FP32 factors
  long long nelem = 0, v_len = 0;
  int Mmax = 0;
  int apply_kernel = 1;  // 0: bulk-copy ring (k_schur_stream_batch), 1: warp per element (k_schur_warp_batch)
  int precision = -1;    // -1: each handle's own, 0: FP64, 1: mixed
};

namespace {

void batch_free_layout(smpm_batch b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
  for (void* p : b->allocs) cudaFree(p);
  b->allocs.clear();
  b->dtasks = nullptr;
  b->dbegin = b->dteam = nullptr;
}

template <typename P>
smpm_status balloc(smpm_batch b, P** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(P) + 16);
  if (e != cudaSuccess) return fail(SMPM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  b->allocs.push_back(q);
  *p = static_cast<P*>(q);
  return SMPM_OK;
}

// Lay the batch out for teams of T CTAs: longest-processing-time assignment
// of whole problems to teams, per-problem scratch for that team size, the
// task table (one task per right-hand side) and the launch's shared memory.
smpm_status batch_layout(smpm_batch b, int T) {
  batch_free_layout(b);
  int dev = 0, sms = 0, optin = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (T < 1 || T > sms) return fail(SMPM_EINVAL, "team size must be in [1, number of SMs]");
  const int np = (int)b->hs.size();
  b->grid = sms;
  b->team_size = T;
  b->nteams = sms / T;
  // cost estimate of a problem: right-hand sides x operator entries
  std::vector<double> cost(np);
  std::vector<int> order(np);
  for (int p = 0; p < np; ++p) {
    const Geometry& g = b->hs[p]->g;
    cost[p] = (double)b->nrhs[p] * ((double)g.nel * g.M * g.M + 2e4 * T);
    order[p] = p;
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<double> load(b->nteams, 0.0);
  std::vector<std::vector<int>> plist(b->nteams);
  for (int p : order) {
    int t = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[t] += cost[p];
    plist[t].push_back(p);
  }
  // per-problem layout for G = T (all-global operator and basis)
  struct PL {
    int nown_b, nown_w, ES;
    bool wg;
    Layout lay;  // layout of the GMRES body (FP64, or the FP32 inner solve)
    double* vown64;
    float* vown32;
    double* wscr64;
    float* wscr32;
    int lock;       // 1: the problem's right-hand sides run as lockstep groups
    size_t lsmem;   // shared memory of its lockstep body (bound over its groups)
  };
  std::vector<PL> pl(np);
  size_t smem = 0;
  smpm_status st;
  for (int p = 0; p < np; ++p) {
    smpm_handle h = b->hs[p];
    const Geometry& g = h->g;
    const int nb = (int)h->f.black.size(), nw = (int)h->f.white.size(), m = h->opts.restart;
    PL& L = pl[p];
    L.nown_b = (nb + T - 1) / T;
    L.nown_w = (nw + T - 1) / T;
    L.ES = 2 * g.M * L.nown_b;
    if (L.ES % 2 == 0) L.ES += 1;
    const bool mixed = (b->precision < 0 ? h->opts.precision : b->precision) == 1;
    // the all-global needs of pre/post and refinement, then the richest
    // GMRES layout that fits beside the argument header (resident or
    // streamed operator matrices, resident basis)
    const int budget = optin - kBatchHdr - 1024;
    auto need_fixed = [&](bool wg) {
      size_t a = prepost_smem_bytes(m, g.M, g.n, L.ES, L.nown_b, L.nown_w, g.d, wg);
      if (mixed) a = std::max(a, refine_smem_bytes(m, g.M, g.n, L.ES, L.nown_b, L.nown_w, g.d, wg));
      return a;
    };
    const int precond = h->opts.precond;
    const bool warp = precond > 0 && L.nown_b >= kWarpElemsMin;
    auto lay_for = [&](bool wg) {
      return mixed ? choose_layout<float>(g, m, L.ES, L.nown_b, L.nown_w, precond, false, false, budget, wg, warp)
                   : choose_layout<double>(g, m, L.ES, L.nown_b, L.nown_w, precond, false, false, budget, wg, warp);
    };
    // w, w2 move to global scratch when either the pre/post bodies or the
    // GMRES body (with its per-warp scratch) would not fit beside them
    L.wg = need_fixed(false) > (size_t)budget || lay_for(false).smem > (size_t)budget;
    L.lay = lay_for(L.wg);
    if (mixed && warp)  // the refinement body runs the warp phases too
      L.lay.smem = std::max(L.lay.smem, refine_smem_bytes(m, g.M, g.n, L.ES, L.nown_b, L.nown_w, g.d, L.wg, true));
    // several right-hand sides of a block-Jacobi problem: lockstep groups of
    // up to kLockMaxCols columns when their body fits (bound: the widest tile)
    L.lock = 0;
    L.lsmem = 0;
    if (b->nrhs[p] >= 2 && precond > 0 && !(h->opts.flags & SMPM_FLAG_NO_LOCKSTEP)) {
      const int Rg = std::min(b->nrhs[p], kLockMaxCols);
      L.lsmem = mixed ? lock_smem_bytes<float>(m, g.M, g.n, Rg, 8, L.nown_b, L.nown_w, false)
                      : lock_smem_bytes<double>(m, g.M, g.n, Rg, 4, L.nown_b, L.nown_w, false);
      if (std::max(need_fixed(L.wg), L.lsmem) <= (size_t)budget) L.lock = 1;
    }
    const size_t nd = kBatchHdr + std::max(need_fixed(L.wg), L.lock ? L.lsmem : L.lay.smem);
    if (nd > (size_t)optin - 1024)
      return fail(SMPM_EINVAL, "a problem of the batch is too large for teams of this size");
    smem = std::max(smem, nd);
    L.vown64 = nullptr;
    L.vown32 = nullptr;
    L.wscr64 = nullptr;
    L.wscr32 = nullptr;
    const size_t vn = (size_t)T * (m + 1) * L.ES;
    if (!L.lock && !L.lay.basis_smem && !mixed && (st = balloc(b, &L.vown64, vn))) return st;
    if (!L.lock && !L.lay.basis_smem && mixed && (st = balloc(b, &L.vown32, vn))) return st;
    if (L.wg) {
      if ((st = balloc(b, &L.wscr64, (size_t)T * 2 * (L.ES + 1)))) return st;
      if (mixed && (st = balloc(b, &L.wscr32, (size_t)T * 2 * (L.ES + 1)))) return st;
    }
  }
  // task table: one task per right-hand side, or one per lockstep group of
  // up to kLockMaxCols right-hand sides of a problem (per-column arguments in
  // global memory, work vectors in a workspace of the team sized for the
  // largest group it runs)
  std::vector<BatchTask> tasks;
  std::vector<int> begin(b->nteams + 1, 0);
  b->task_of.assign(b->ntasks, -1);
  b->task_col.clear();
  long long ncol_groups = 0;
  for (int p = 0; p < np; ++p)
    if (pl[p].lock)
      for (int k0 = 0; k0 < b->nrhs[p]; k0 += kLockMaxCols)
        if (std::min(kLockMaxCols, b->nrhs[p] - k0) >= 2) ncol_groups += std::min(kLockMaxCols, b->nrhs[p] - k0);
  PrePostArgs* dPc = nullptr;
  RefineArgs* dRc = nullptr;
  std::vector<PrePostArgs> hPc;
  std::vector<RefineArgs> hRc;
  if (ncol_groups > 0) {
    if ((st = balloc(b, &dPc, 2 * (size_t)ncol_groups)) || (st = balloc(b, &dRc, (size_t)kMaxRefine * ncol_groups)))
      return st;
    hPc.reserve(2 * (size_t)ncol_groups);
    hRc.reserve((size_t)kMaxRefine * ncol_groups);
  }
  for (int t = 0; t < b->nteams; ++t) {
    begin[t] = (int)tasks.size();
    // ---- the team's lockstep workspace: the largest group it runs
    struct {
      size_t R = 0, r = 0, kp = 0, d = 0, acc = 0, Rh = 0, yv = 0, V64 = 0, W64 = 0, V32 = 0, W32 = 0;
      bool f64 = false, f32 = false;
    } need;
    for (int p : plist[t]) {
      if (!pl[p].lock) continue;
      smpm_handle h = b->hs[p];
      const Geometry& g = h->g;
      const size_t R = (size_t)std::min(b->nrhs[p], kLockMaxCols), m = h->opts.restart, ES = pl[p].ES;
      const bool mixed = (b->precision < 0 ? h->opts.precision : b->precision) == 1;
      need.R = std::max(need.R, R);
      need.r = std::max(need.r, (size_t)g.r);
      need.kp = std::max(need.kp, (size_t)g.kp);
      need.d = std::max(need.d, (size_t)g.d);
      need.acc = std::max(need.acc, (2 * m + 1) * R * (m + 3));
      need.Rh = std::max(need.Rh, R * m * (m + 1));
      need.yv = std::max(need.yv, R * m);
      if (mixed) {
        need.f32 = true;
        need.V32 = std::max(need.V32, (size_t)T * (m + 1) * R * ES);
        need.W32 = std::max(need.W32, (size_t)T * 2 * R * (ES + 1));
      } else {
        need.f64 = true;
        need.V64 = std::max(need.V64, (size_t)T * (m + 1) * R * ES);
        need.W64 = std::max(need.W64, (size_t)T * 2 * R * (ES + 1));
      }
    }
    double *wb = nullptr, *wbS = nullptr, *wrg = nullptr, *wcb = nullptr, *wchatb = nullptr, *wxs = nullptr;
    double *wc = nullptr, *wchat = nullptr, *wacc = nullptr, *wRh = nullptr, *wyv = nullptr;
    double *wx = nullptr, *wt = nullptr, *wy = nullptr, *wvg = nullptr, *wV = nullptr, *wW = nullptr, *wcr = nullptr;
    float *wx32 = nullptr, *wt32 = nullptr, *wy32 = nullptr, *wvg32 = nullptr, *wrg32 = nullptr, *wV32 = nullptr,
          *wW32 = nullptr;
    LockColState* wcs = nullptr;
    unsigned char* wctl = nullptr;
    if (need.R > 0) {
      const size_t R = need.R;
      if ((st = balloc(b, &wb, R * need.r)) || (st = balloc(b, &wbS, R * need.kp)) ||
          (st = balloc(b, &wrg, R * need.kp)) || (st = balloc(b, &wcb, R * need.d)) ||
          (st = balloc(b, &wchatb, R * need.d)) || (st = balloc(b, &wxs, R * need.kp)) ||
          (st = balloc(b, &wc, R * need.d)) || (st = balloc(b, &wchat, R * need.d)) ||
          (st = balloc(b, &wacc, need.acc)) || (st = balloc(b, &wRh, need.Rh)) || (st = balloc(b, &wyv, need.yv)) ||
          (st = balloc(b, &wcs, R)) || (st = balloc(b, &wctl, R * kLockColBytes)))
        return st;
      if (need.f64 && ((st = balloc(b, &wx, R * need.kp)) || (st = balloc(b, &wt, R * need.kp)) ||
                       (st = balloc(b, &wy, R * need.kp)) || (st = balloc(b, &wvg, R * need.kp)) ||
                       (st = balloc(b, &wV, need.V64)) || (st = balloc(b, &wW, need.W64))))
        return st;
      if (need.f32 && ((st = balloc(b, &wx32, R * need.kp)) || (st = balloc(b, &wt32, R * need.kp)) ||
                       (st = balloc(b, &wy32, R * need.kp)) || (st = balloc(b, &wvg32, R * need.kp)) ||
                       (st = balloc(b, &wrg32, R * need.kp)) || (st = balloc(b, &wcr, R * need.d)) ||
                       (st = balloc(b, &wV32, need.V32)) || (st = balloc(b, &wW32, need.W32))))
        return st;
      // work vectors start at zero (boundary-face slots are never written)
      for (double* v : {wt, wy, wvg})
        if (v) CU(cudaMemset(v, 0, R * need.kp * sizeof(double)));
      for (float* v : {wt32, wy32, wvg32})
        if (v) CU(cudaMemset(v, 0, R * need.kp * sizeof(float)));
    }
    for (int p : plist[t]) {
      smpm_handle h = b->hs[p];
      const PL& L = pl[p];
      const bool mixed = (b->precision < 0 ? h->opts.precision : b->precision) == 1;
      const double tol = h->opts.tol;
      auto team_fields = [&](auto& a) {
        a.G = T;
        a.base = t * T;
        a.nown_b = L.nown_b;
        a.nown_w = L.nown_w;
        a.ES = L.ES;
        a.mats_smem = 0;
        a.basis_smem = 0;
        a.stream_mats = 0;
        a.bar = b->dbars + t;
        a.err = b->derr;
        a.trace = nullptr;
        a.trace_cap = 0;
        a.skip = nullptr;
        a.its_out = nullptr;
      };
      auto layout_fields = [&](auto& a) {
        a.mats_smem = L.lay.mats_smem;
        a.basis_smem = L.lay.basis_smem;
        a.stream_mats = L.lay.stream_mats;
        a.buf_elems = L.lay.buf_elems;
        a.nbuf = L.lay.nbuf;
        a.warp_elems = L.lay.warp_elems;
      };
      auto single_task = [&](int k) {
        BatchTask bt{};
        bt.P = prepost_args(h, tol, nullptr, nullptr, nullptr, mixed);
        auto team_fields = [&](auto& a) {
          a.G = T;
          a.base = t * T;
          a.nown_b = L.nown_b;
          a.nown_w = L.nown_w;
          a.ES = L.ES;
          a.mats_smem = 0;
          a.basis_smem = 0;
          a.stream_mats = 0;
          a.bar = b->dbars + t;
          a.err = b->derr;
          a.trace = nullptr;
          a.trace_cap = 0;
          a.skip = nullptr;
          a.its_out = nullptr;
        };
        team_fields(bt.P.ga);
        bt.P.ga.vown = nullptr;
        bt.P.ga.wscr = L.wscr64;
        auto layout_fields = [&](auto& a) {
          a.mats_smem = L.lay.mats_smem;
          a.basis_smem = L.lay.basis_smem;
          a.stream_mats = L.lay.stream_mats;
          a.buf_elems = L.lay.buf_elems;
          a.nbuf = L.lay.nbuf;
          a.warp_elems = L.lay.warp_elems;
        };
        if (mixed) {
          bt.a32 = gmres_args32(h, kInnerTol);
          team_fields(bt.a32);
          bt.a32.vown = L.vown32;
          bt.a32.wscr = L.wscr32;
          bt.R = refine_args(h, bt.a32, tol);  // all-global (refine_args clears the layout)
          bt.R.ga.warp_elems = L.lay.warp_elems;
          layout_fields(bt.a32);
        } else {
          bt.a64 = gmres_args(h, tol);
          team_fields(bt.a64);
          layout_fields(bt.a64);
          bt.a64.vown = L.vown64;
          bt.a64.wscr = L.wscr64;
        }
        bt.precision = mixed ? 1 : 0;
        bt.has_g = 1;
        bt.f_off = b->foff[p] + (long long)k * h->g.r;
        bt.u_off = bt.f_off;
        bt.g_off = b->goff[p] + (long long)k * h->g.kp;
        bt.ctl = h->wctl;
        bt.its = reinterpret_cast<int*>(h->wctl + 592);
        bt.rn = h->wrn;
        bt.rep0 = b->rhs_base[p] + k;
        b->task_of[b->rhs_base[p] + k] = b->rhs_base[p] + k;
        b->task_col.push_back(b->rhs_base[p] + k);
        tasks.push_back(bt);
      };
      for (int k0 = 0; k0 < b->nrhs[p]; k0 += (L.lock ? kLockMaxCols : 1)) {
        const int R = L.lock ? std::min(kLockMaxCols, b->nrhs[p] - k0) : 1;
        if (R == 1) {
          single_task(k0);
          continue;
        }
        const Geometry& g = h->g;
        BatchTask bt{};
        bt.P = prepost_args(h, tol, nullptr, nullptr, nullptr, mixed);
        team_fields(bt.P.ga);
        bt.P.ga.vown = nullptr;
        bt.P.ga.wscr = L.wscr64;
        bt.precision = mixed ? 1 : 0;
        bt.has_g = 1;
        bt.f_off = b->foff[p] + (long long)k0 * g.r;
        bt.u_off = bt.f_off;
        bt.g_off = b->goff[p] + (long long)k0 * g.kp;
        bt.ncols = R;
        bt.rep0 = b->rhs_base[p] + k0;
        bt.r_len = g.r;
        bt.kp_len = g.kp;
        bt.lctl = wctl;
        const size_t c0 = hPc.size() / 2;  // first column slot of this group in the argument arrays
        bt.Pc = dPc + 2 * c0;
        bt.Rc = dRc + (size_t)kMaxRefine * c0;
        std::vector<PrePostArgs> pre(R), post(R);
        for (int c = 0; c < R; ++c) {
          PrePostArgs P = bt.P;
          P.b = wb + (size_t)c * g.r;
          P.bS = wbS + (size_t)c * g.kp;
          P.rg = wrg + (size_t)c * g.kp;
          P.cb = wcb + (size_t)c * g.d;
          P.chatb = wchatb + (size_t)c * g.d;
          P.xs = wxs + (size_t)c * g.kp;
          P.acc = reinterpret_cast<double*>(wctl + (size_t)c * kLockColBytes);
          P.gacc = nullptr;
          P.gacc_n = 0;
          if (!mixed) {
            P.ga.x = wx + (size_t)c * g.kp;
            double* zs[7] = {P.ga.x, h->wt, h->wy, h->wV, P.bS, P.rg, P.xs};
            for (int i = 0; i < 7; ++i) P.zero[i] = zs[i];
          } else {
            double* zs[7] = {h->wx, h->wt, h->wy, h->wV, P.bS, P.rg, P.xs};
            for (int i = 0; i < 7; ++i) P.zero[i] = zs[i];
            float* z32[4] = {wx32 + (size_t)c * g.kp, wt32, wy32, wvg32};
            for (int i = 0; i < 4; ++i) P.zero32[i] = z32[i];
            P.cr = wcr + (size_t)c * g.d;
            P.rg32 = wrg32 + (size_t)c * g.kp;
          }
          P.assembled = 0;
          pre[c] = P;
          P.assembled = mixed ? 1 : 0;
          post[c] = P;
        }
        hPc.insert(hPc.end(), pre.begin(), pre.end());
        hPc.insert(hPc.end(), post.begin(), post.end());
        hRc.resize(hRc.size() + (size_t)kMaxRefine * R);
        auto lock_fields = [&](auto& A, int maxrc) {
          team_fields(A.a);
          A.a.mats_smem = 0;
          A.a.basis_smem = 0;
          A.a.stream_mats = 0;
          A.a.warp_elems = 1;
          A.a.wscr = nullptr;
          A.a.vown = nullptr;
          A.a.fused = 0;
          A.a.c = wc;
          A.a.chat = wchat;
          A.a.acc = wacc;
          A.R = R;
          A.RC = lock_rc(R, L.nown_b, maxrc, kGmresThreads / 32);
          A.vs = g.kp;
          A.ds = g.d;
          A.cs = wcs;
          A.Rh = wRh;
          A.yv = wyv;
        };
        if (!mixed) {
          bt.L64.a = gmres_args(h, tol);
          lock_fields(bt.L64, 4);
          bt.L64.a.rhs = wrg;
          bt.L64.a.x = wx;
          bt.L64.a.t = wt;
          bt.L64.a.y = wy;
          bt.L64.a.vglob = wvg;
          bt.L64.V = wV;
          bt.L64.W = wW;
          bt.L64.done = nullptr;
          bt.L64.done_stride = 0;
        } else {
          bt.L32.a = gmres_args32(h, kInnerTol);
          lock_fields(bt.L32, 8);
          bt.L32.a.rhs = wrg32;
          bt.L32.a.x = wx32;
          bt.L32.a.t = wt32;
          bt.L32.a.y = wy32;
          bt.L32.a.vglob = wvg32;
          bt.L32.V = wV32;
          bt.L32.W = wW32;
          bt.L32.done = reinterpret_cast<const int*>(wctl + 64);
          bt.L32.done_stride = (int)(kLockColBytes / sizeof(int));
          for (int ref = 0; ref < kMaxRefine; ++ref)
            for (int c = 0; c < R; ++c) {
              GmresArgs<float> a = gmres_args32(h, kInnerTol);
              team_fields(a);
              a.warp_elems = L.lay.warp_elems;
              a.wscr = L.wscr32;
              a.x = wx32 + (size_t)c * g.kp;
              a.t = wt32;
              a.y = wy32;
              a.vglob = wvg32;
              a.rhs = wrg32 + (size_t)c * g.kp;
              RefineArgs RA = refine_args(h, a, tol);
              RA.ga.warp_elems = L.lay.warp_elems;
              RA.xS = wxs + (size_t)c * g.kp;
              RA.bS = wbS + (size_t)c * g.kp;
              RA.cr = wcr + (size_t)c * g.d;
              RA.chat_r = wchatb + (size_t)c * g.d;
              unsigned char* blk = wctl + (size_t)c * kLockColBytes;
              RA.rgn = reinterpret_cast<double*>(blk) + ACC_RGN;
              RA.rn = reinterpret_cast<double*>(blk + 128) + ref;
              RA.done = reinterpret_cast<int*>(blk + 64);
              RA.nref = reinterpret_cast<int*>(blk + 68);
              RA.rhs32 = wrg32 + (size_t)c * g.kp;
              hRc[(size_t)kMaxRefine * c0 + (size_t)ref * R + c] = RA;
            }
        }
        for (int c = 0; c < R; ++c) b->task_of[b->rhs_base[p] + k0 + c] = b->rhs_base[p] + k0 + c;
        b->task_col.push_back(b->rhs_base[p] + k0);
        tasks.push_back(bt);
      }
    }
  }
  if (!hPc.empty()) {
    CU(cudaMemcpy(dPc, hPc.data(), hPc.size() * sizeof(PrePostArgs), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(dRc, hRc.data(), hRc.size() * sizeof(RefineArgs), cudaMemcpyHostToDevice));
  }
  begin[b->nteams] = (int)tasks.size();
  std::vector<int> team_of(sms, -1);
  for (int c = 0; c < b->nteams * T; ++c) team_of[c] = c / T;
  if ((st = balloc(b, &b->dtasks, tasks.size())) || (st = balloc(b, &b->dbegin, begin.size())) ||
      (st = balloc(b, &b->dteam, team_of.size())))
    return st;
  CU(cudaMemcpy(b->dtasks, tasks.data(), tasks.size() * sizeof(BatchTask), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(b->dbegin, begin.data(), begin.size() * sizeof(int), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(b->dteam, team_of.data(), team_of.size() * sizeof(int), cudaMemcpyHostToDevice));
  b->smem = smem;
  CU(set_smem_limit(k_batch, optin));
  int per = 0;
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch, kGmresThreads, smem));
  if (per < 1) return fail(SMPM_ECUDA, "the batch kernel does not fit on an SM");
  return SMPM_OK;
}

// y_p = S_p v_p for all problems: stages as in launch_schur_stream, sized
// for the largest element matrix of the batch.
template <typename S>
smpm_status batch_apply(smpm_batch b, const ElemMeta<S>* tab, const S* v, S* y, cudaStream_t st) {
  int dev = 0, sms = 0, optin = 0, per_sm_smem = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  CU(cudaDeviceGetAttribute(&per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  const int M = b->Mmax;
  // two CTAs per SM when a ring of two of the largest element matrices fits
  // in half the SM, else one CTA; the ring takes the rest of the CTA's share
  // (less the CTA's reserved and static shared memory: 1 KB each CTA on this
  // part, with margin)
  const size_t fixed = schur_stream_batch_smem<S>(0, M);
  const size_t one = (size_t)M * M * sizeof(S);
  int cps = 2;
  size_t share = (size_t)per_sm_smem / 2 - 2048;
  if (share > (size_t)optin - 1024) share = (size_t)optin - 1024;
  if (share < fixed + 2 * one) {
    cps = 1;
    share = (size_t)optin - 1024;
  }
  if (share < fixed + one) return fail(SMPM_EINVAL, "element matrix too large for the batched apply");
  const unsigned ring = (unsigned)((share - fixed) / 16 * 16);
  const size_t smem = schur_stream_batch_smem<S>(ring, M);
  if (b->apply_kernel == 1 && M <= 96) {  // register-streamed, warps per element
    CU(launch_schur_warp<S>(tab, b->nelem, v, y, sms, st));
    return SMPM_OK;
  }
  CU(set_smem_limit(k_schur_stream_batch<S>, optin));
  const unsigned grid = (unsigned)std::min<long long>((long long)sms * cps, b->nelem);
  k_schur_stream_batch<S><<<grid, kElemThreads, smem, st>>>(tab, b->nelem, v, y, ring, M);
  CU(cudaGetLastError());
  return SMPM_OK;
}

// The device work of one batched solve, in stream order.
smpm_status batch_enqueue(smpm_batch b, cudaStream_t st) {
  CU(cudaMemcpyAsync(b->dio, b->hio, sizeof(BatchIO), cudaMemcpyHostToDevice, st));
  CU(cudaMemsetAsync(b->dbars, 0, sizeof(unsigned) * b->grid, st));
  CU(cudaMemsetAsync(b->derr, 0, 4 * sizeof(int), st));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b->grid);
  cfg.blockDim = dim3(kGmresThreads);
  cfg.dynamicSmemBytes = b->smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int ctl = (int)kCtlBytes;
  CU(cudaLaunchKernelEx(&cfg, k_batch, (const BatchTask*)b->dtasks, (const int*)b->dbegin, (const int*)b->dteam,
                        (const BatchIO*)b->dio, b->drep, ctl));
  CU(cudaMemcpyAsync(b->hrep, b->drep, sizeof(TaskReport) * b->ntasks, cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(b->herr, b->derr, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
  return SMPM_OK;
}

}  // namespace

extern "C" {

void smpm_default_opts(smpm_opts* o) {
  if (!o) return;
  o->tol = 1e-10;
  o->restart = 50;
  o->maxit = 1000;
  o->precision = 0;
  o->precond = 2;
  o->tau_scale = 1.0;
  o->robin_scale = 0.25;
  o->flags = 0;
}

const char* smpm_last_error(void) { return g_last_error.c_str(); }

smpm_status smpm_setup_graded(int mx, int my, int n, const double* xs, const double* ys, smpm_handle* out) try {
  if (!out) return fail(SMPM_EINVAL, "null handle pointer");
  *out = nullptr;
  if (!xs || !ys) return fail(SMPM_EINVAL, "null element edges");
  if (mx < 1 || my < 1 || mx > 4096 || my > 4096) return fail(SMPM_EINVAL, "grid sizes out of range");
  for (int i = 0; i <= mx; ++i)
    if (!std::isfinite(xs[i]) || (i > 0 && !(xs[i] > xs[i - 1])))
      return fail(SMPM_EINVAL, "column edges must be finite and strictly increasing");
  for (int i = 0; i <= my; ++i)
    if (!std::isfinite(ys[i]) || (i > 0 && !(ys[i] > ys[i - 1])))
      return fail(SMPM_EINVAL, "row edges must be finite and strictly increasing");
  smpm_status s = smpm_setup(mx, my, n, xs[mx] - xs[0], ys[my] - ys[0], out);
  if (s != SMPM_OK) return s;
  Geometry& g = (*out)->g;
  g.graded = true;
  g.xe.assign(xs, xs + mx + 1);
  g.ye.assign(ys, ys + my + 1);
  return SMPM_OK;
} catch (...) {
  if (out && *out) {
    smpm_destroy(*out);
    *out = nullptr;
  }
  return host_exception();
}

smpm_status smpm_setup(int mx, int my, int n, double Lx, double Ly, smpm_handle* out) try {
  if (!out) return fail(SMPM_EINVAL, "null handle pointer");
  *out = nullptr;
  if (mx < 1 || my < 1 || mx > 4096 || my > 4096 || n < 2 || n > kMaxN)
    return fail(SMPM_EINVAL, "grid sizes out of range");
  if (!(Lx > 0) || !(Ly > 0) || !std::isfinite(Lx) || !std::isfinite(Ly))
    return fail(SMPM_EINVAL, "domain lengths must be positive and finite");
  smpm_handle h = new (std::nothrow) smpm_handle_s();
  if (!h) return fail(SMPM_ENOMEM, "host allocation failed");
  Geometry& g = h->g;
  g.mx = mx; g.my = my; g.n = n; g.M = 4 * n;
  g.Lx = Lx; g.Ly = Ly; g.hx = Lx / mx; g.hy = Ly / my;
  g.nel = (long long)mx * my;
  g.nn = (long long)n * n;
  g.r = g.nn * g.nel;
  g.kp = 4LL * n * g.nel;
  g.d = (long long)(mx - 1) * my + (long long)mx * (my - 1);
  g.k = 2LL * n * g.d;
  smpm_default_opts(&h->opts);
  *out = h;
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

smpm_status smpm_partition_tile(smpm_handle h, int px, int py, int rank, smpm_tile* t) try {
  if (!h || !t) return fail(SMPM_EINVAL, "null argument");
  if (partition_tile(h->g, px, py, rank, t) != SMPM_OK)
    return fail(SMPM_EINVAL, "tile grid must satisfy 1 <= px <= mx, 1 <= py <= my, 0 <= rank < px py");
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

smpm_status smpm_partition_halo(smpm_handle h, int px, int py, int rank, int side, long long* own,
                                long long* facing) try {
  if (!h) return fail(SMPM_EINVAL, "null handle");
  if (partition_halo(h->g, px, py, rank, side, own, facing) != SMPM_OK)
    return fail(SMPM_EINVAL, "no peer across that side, or tile grid out of range");
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

smpm_status smpm_sizes(smpm_handle h, long long* r, long long* kp, long long* d, long long* k, long long* nblack) try {
  if (!h) return fail(SMPM_EINVAL, "null handle");
  if (r) *r = h->g.r;
  if (kp) *kp = h->g.kp;
  if (d) *d = h->g.d;
  if (k) *k = h->g.k;
  if (nblack) {
    long long c = 0;
    for (long long e = 0; e < h->g.nel; ++e) c += h->g.black((int)e) ? 1 : 0;
    *nblack = c;
  }
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

smpm_status smpm_node_coords(smpm_handle h, double* x, double* y) try {
  if (!h || !x || !y) return fail(SMPM_EINVAL, "null argument");
  const Geometry& g = h->g;
  std::vector<double> xi, w;
  gll(g.n, &xi, &w);
  for (long long e = 0; e < g.nel; ++e) {
    int ix = (int)(e % g.mx), iy = (int)(e / g.mx);
    const double x0 = g.col_x0(ix), y0 = g.row_y0(iy), hx = g.col_h(ix), hy = g.row_h(iy);
    for (int b = 0; b < g.n; ++b)
      for (int a = 0; a < g.n; ++a) {
        long long q = e * g.nn + b * g.n + a;
        x[q] = x0 + (xi[a] + 1.0) * hx / 2.0;
        y[q] = y0 + (xi[b] + 1.0) * hy / 2.0;
      }
  }
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

smpm_status smpm_node_mass(smpm_handle h, double* wq) try {
  if (!h || !wq) return fail(SMPM_EINVAL, "null argument");
  const Geometry& g = h->g;
  std::vector<double> xi, w;
  gll(g.n, &xi, &w);
  for (long long e = 0; e < g.nel; ++e)
    for (int b = 0; b < g.n; ++b)
      for (int a = 0; a < g.n; ++a)
        wq[e * g.nn + b * g.n + a] = w[a] * w[b] * g.hx_of((int)e) * g.hy_of((int)e) / 4.0;
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

}  // extern "C"

namespace {

// Options check shared by the factor entry points.
smpm_status check_factor_opts(smpm_handle h, const smpm_opts* o, smpm_opts* out) {
  if (!h) return fail(SMPM_EINVAL, "null handle");
  smpm_opts opts;
  smpm_default_opts(&opts);
  if (o) opts = *o;
  if (!(opts.tol > 0) || opts.restart < 1 || opts.restart > kMaxRestart || opts.maxit < 1 || opts.precond < 0 ||
      opts.precond > 2 || opts.precision < 0 || opts.precision > 1 || !(opts.tau_scale > 0) ||
      !(opts.robin_scale > 0))
    return fail(SMPM_EINVAL, "bad solver options");
  if (h->g.nel < 2) return fail(SMPM_ENOINTERFACE, "the Schur method needs mx*my >= 2 (one interface at least)");
  if (h->g.d < 2 && opts.precond > 0)
    return fail(SMPM_EINVAL, "with a single interface the only block-Jacobi block is all of the singular S; "
                             "use precond = 0");
  *out = opts;
  return SMPM_OK;
}

// Device half of the factor step: uploads of the host factors in h->f,
// workspaces and launch shapes.
smpm_status factor_device(smpm_handle h, cudaStream_t st);
// The same for an operator-only factor step: T_e (FP64, and FP32 with
// precision 1) and the element tables of the apply kernels.
smpm_status factor_device_operator(smpm_handle h, cudaStream_t st);

}  // namespace

extern "C" {

smpm_status schur_factor(smpm_handle h, const smpm_opts* o, void* stream) try {
  smpm_opts opts;
  smpm_status cs = check_factor_opts(h, o, &opts);
  if (cs != SMPM_OK) return cs;
  free_all(h);
  h->factored = false;
  h->op_factored = false;
  h->opts = opts;
  h->f = Factors();
  std::string err;
  int rc = factor_host(h->g, opts, &h->f, &err);
  if (rc != SMPM_OK) return fail(static_cast<smpm_status>(rc), err);
  if (h->f.operator_only) return factor_device_operator(h, as_stream(stream));
  return factor_device(h, as_stream(stream));
} catch (...) {
  return host_exception();
}

smpm_status smpm_factor_many(const smpm_handle* hs, int count, const smpm_opts* o, void* stream) try {
  if (!hs || count < 1) return fail(SMPM_EINVAL, "bad arguments");
  smpm_opts opts;
  for (int i = 0; i < count; ++i) {
    smpm_status cs = check_factor_opts(hs[i], o, &opts);
    if (cs != SMPM_OK) return cs;
  }
  std::vector<Factors> fs(count);
  std::vector<std::string> errs(count);
  std::vector<int> rc(count, SMPM_OK), order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return hs[a]->g.d * (long long)hs[a]->g.M > hs[b]->g.d * (long long)hs[b]->g.M;
  });
  // one problem per thread, largest first (the factor step's own parallel
  // loops run single-threaded inside this region)
#pragma omp parallel for schedule(dynamic, 1)
  for (int k = 0; k < count; ++k) {
    const int i = order[k];
    rc[i] = factor_host(hs[i]->g, opts, &fs[i], &errs[i]);
  }
  cudaStream_t st = as_stream(stream);
  for (int i = 0; i < count; ++i) {
    if (rc[i] != SMPM_OK) return fail(static_cast<smpm_status>(rc[i]), errs[i]);
    smpm_handle h = hs[i];
    free_all(h);
    h->factored = false;
    h->op_factored = false;
    h->opts = opts;
    h->f = std::move(fs[i]);
    smpm_status s = h->f.operator_only ? factor_device_operator(h, st) : factor_device(h, st);
    if (s != SMPM_OK) return s;
  }
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

}  // extern "C"

namespace {

// Class tables of the class-shared apply: one T per T class of the factor
// step (face types, and on a graded grid the sizes; the copies of T_e within
// a class are identical), tiles of kClassTile elements.
smpm_status upload_classes(smpm_handle h, const std::vector<double>& Tc, cudaStream_t st) {
  const Geometry& g = h->g;
  const size_t MM = (size_t)g.M * g.M;
  std::vector<int> cls_of(g.nel, -1), first;
  std::vector<std::vector<int>> members;
  for (long long e = 0; e < g.nel; ++e) {
    const int key = h->f.tcls[e];
    if (cls_of[key] < 0) {
      cls_of[key] = (int)members.size();
      members.emplace_back();
      first.push_back((int)e);
    }
    members[cls_of[key]].push_back((int)e);
  }
  std::vector<double> Tcls(members.size() * MM);
  for (size_t c = 0; c < members.size(); ++c)
    std::copy(Tc.begin() + (size_t)first[c] * MM, Tc.begin() + (size_t)(first[c] + 1) * MM, Tcls.begin() + c * MM);
  std::vector<int> sel, tiles;
  for (size_t c = 0; c < members.size(); ++c) {
    const int base = (int)sel.size();
    sel.insert(sel.end(), members[c].begin(), members[c].end());
    for (int i = 0; i < (int)members[c].size(); i += kClassTile) {
      tiles.push_back((int)c);
      tiles.push_back(base + i);
      tiles.push_back(std::min(kClassTile, (int)members[c].size() - i));
    }
  }
  smpm_status s;
  if ((s = upload(h, &h->dTcls, Tcls, st)) || (s = upload(h, &h->dtiles, tiles, st)) ||
      (s = upload(h, &h->dclsel, sel, st)))
    return s;
  if (h->opts.precision == 1 && (s = upload(h, &h->dTcls32, std::vector<float>(Tcls.begin(), Tcls.end()), st)))
    return s;
  h->ncls = (int)members.size();
  h->ntiles = (int)(tiles.size() / 3);
  int dev = 0, optin = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (g.M <= 128 && class_smem(g.M, sizeof(double)) <= (size_t)optin) {
    CU(set_smem_limit(k_schur_class<double>, optin));
    CU(set_smem_limit(k_schur_class<float>, optin));
    h->cls_ok = 1;
  }
  return SMPM_OK;
}

smpm_status factor_device_operator(smpm_handle h, cudaStream_t st) {
  const Geometry& g = h->g;
  DevGeo& dg = h->dg;
  dg.mx = g.mx; dg.my = g.my; dg.n = g.n; dg.M = g.M;
  dg.nel = g.nel; dg.kp = g.kp; dg.r = g.r; dg.d = g.d;
  dg.graded = g.graded ? 1 : 0;
  smpm_status s;
  std::vector<double> Tc = transpose_blocks(h->f.T, g.M, g.nel);
  if ((s = upload(h, &h->dT, Tc, st)) || (s = upload(h, &h->dcgeo, h->f.colg, st)) ||
      (s = upload(h, &h->drgeo, h->f.rowg, st)))
    return s;
  dg.cgeo = h->dcgeo;
  dg.rgeo = h->drgeo;
  if (h->opts.precision == 1 && (s = upload(h, &h->dT32, std::vector<float>(Tc.begin(), Tc.end()), st))) return s;
  std::vector<ElemMeta<double>> t64(g.nel);
  std::vector<ElemMeta<float>> t32(h->dT32 ? g.nel : 0);
  for (long long e = 0; e < g.nel; ++e) {
    ElemMeta<double> a{};
    a.T = h->dT; a.e = (int)e; a.M = g.M; a.n = g.n; a.mx = g.mx; a.my = g.my;
    t64[e] = a;
    if (h->dT32) {
      ElemMeta<float> c{};
      c.T = h->dT32; c.e = (int)e; c.M = g.M; c.n = g.n; c.mx = g.mx; c.my = g.my;
      t32[e] = c;
    }
  }
  if ((s = upload(h, &h->dtab64, t64, st))) return s;
  if (h->dT32 && (s = upload(h, &h->dtab32, t32, st))) return s;
  if ((s = upload_classes(h, Tc, st))) return s;
  CU(cudaStreamSynchronize(st));
  h->f.T.clear();
  h->f.T.shrink_to_fit();
  h->op_factored = true;
  return SMPM_OK;
}

smpm_status factor_device(smpm_handle h, cudaStream_t st) {
  const smpm_opts opts = h->opts;
  const Geometry& g = h->g;
  DevGeo& dg = h->dg;
  dg.mx = g.mx; dg.my = g.my; dg.n = g.n; dg.M = g.M;
  dg.nel = g.nel; dg.kp = g.kp; dg.r = g.r; dg.d = g.d;
  dg.graded = g.graded ? 1 : 0;
  smpm_status s;
  // device copies of T_e, G_b and the X_F blocks are column-major
  std::vector<double> Tc = transpose_blocks(h->f.T, g.M, g.nel), Gc = transpose_blocks(h->f.G, g.M, h->f.black.size()),
                      Xc = transpose_blocks(h->f.X, g.n, 4 * h->f.black.size());
  if ((s = upload(h, &h->dT, Tc, st)) || (s = upload(h, &h->dRs, h->f.Rs, st)) ||
      (s = upload(h, &h->dG, Gc, st)) || (s = upload(h, &h->dX, Xc, st)) ||
      (s = upload(h, &h->dH, h->f.H, st)) || (s = upload(h, &h->dfdx, h->f.fdx, st)) ||
      (s = upload(h, &h->dfdy, h->f.fdy, st)) || (s = upload(h, &h->dD, h->f.D, st)) ||
      (s = upload(h, &h->duL, h->f.uL, st)) || (s = upload(h, &h->duS, h->f.uS, st)) ||
      (s = upload(h, &h->duC, h->f.uC, st)) || (s = upload(h, &h->dwhat, h->f.what, st)) ||
      (s = upload(h, &h->dblack, h->f.black, st)) || (s = upload(h, &h->dwhite, h->f.white, st)) ||
      (s = upload(h, &h->dcgeo, h->f.colg, st)) || (s = upload(h, &h->drgeo, h->f.rowg, st)))
    return s;
  dg.cgeo = h->dcgeo;
  dg.rgeo = h->drgeo;
  if (g.graded) {  // uniform grids: every deflation weight is 1 (no table)
    if ((s = upload(h, &h->dzw, h->f.zw, st))) return s;
    if (h->f.has_adjoint && (s = upload(h, &h->dzwa, h->f.zwa, st))) return s;
  }
  dg.zw = h->dzw;
  const size_t kp = g.kp, r = g.r, d = g.d, m = opts.restart;
  const size_t nbs = blocks_for(g.kp, kSlotsPerBlock);
  if ((s = dalloc(h, &h->wb, r)) || (s = dalloc(h, &h->wbS, kp)) || (s = dalloc(h, &h->wV, (m + 1) * kp)) ||
      (s = dalloc(h, &h->wt, kp)) || (s = dalloc(h, &h->wy, kp)) || (s = dalloc(h, &h->ww, kp)) ||
      (s = dalloc(h, &h->wx, kp)) || (s = dalloc(h, &h->wrg, kp)) ||
      (s = dalloc(h, &h->wtmp, kp)) || (s = dalloc(h, &h->wc, d)) || (s = dalloc(h, &h->wchat, d)) ||
      (s = dalloc(h, &h->wcb, d)) || (s = dalloc(h, &h->wchatb, d)) ||
      (s = dalloc(h, &h->wpart, (size_t)3 * (kMaxRestart + 3) * std::max<size_t>(nbs, 1024))) ||
      (s = dalloc(h, &h->wcnt, 8)) || (s = dalloc(h, &h->wgs, 1)))
    return s;
  CU(cudaMemsetAsync(h->wcnt, 0, 8 * sizeof(unsigned), st));
  CU(cudaEventCreate(&h->ev0));
  CU(cudaEventCreate(&h->ev1));
  CU(cudaEventCreate(&h->evp));
  CU(cudaEventCreate(&h->evq));
  if (std::getenv("SMPM_TRACE")) {
    if ((s = dalloc(h, &h->wtrace, kTraceCap))) return s;
    CU(cudaMemsetAsync(h->wtrace, 0, kTraceCap * sizeof(long long), st));
  }
  {
    // persistent GMRES kernel: one CTA per SM at most (all CTAs co-resident);
    // CTA c owns blocks c, c+G, ... and keeps their matrices and its basis
    // slice in shared memory when they fit.
    int dev = 0, sms = 0, smem_optin = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CU(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int nb = (int)h->f.black.size(), nw = (int)h->f.white.size();
    auto& gm = h->gm;
    gm.grid = std::max(1, std::min(sms, std::max(nb, nw)));
    gm.nown_b = (nb + gm.grid - 1) / gm.grid;
    gm.nown_w = (nw + gm.grid - 1) / gm.grid;
    gm.ES = 2 * g.M * gm.nown_b;
    if (gm.ES % 2 == 0) gm.ES += 1;
    const int m = opts.restart;
    const bool no_smem = (opts.flags & SMPM_FLAG_NO_SMEM_RESIDENCY) != 0;
    const bool force_stream = (opts.flags & SMPM_FLAG_STREAM_MATRICES) != 0;
    // one warp per element when every CTA owns several blocks (or on request)
    const bool warp = opts.precond > 0 && !force_stream &&
                      (gm.nown_b >= kWarpElemsMin || (opts.flags & SMPM_FLAG_WARP_ELEMS) != 0);
    {
      Layout L = choose_layout<double>(g, m, gm.ES, gm.nown_b, gm.nown_w, opts.precond, no_smem, force_stream,
                                       smem_optin, false, warp);
      gm.basis_smem = L.basis_smem;
      gm.mats_smem = L.mats_smem;
      gm.stream_mats = L.stream_mats;
      gm.buf_elems = L.buf_elems;
      gm.nbuf = L.nbuf;
      gm.warp_elems = L.warp_elems;
      gm.smem = L.smem;
    }
    CU(set_smem_limit(k_gmres<double>, smem_optin));
    int per_sm = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gmres<double>, kGmresThreads, gm.smem));
    if (per_sm < 1) return fail(SMPM_ECUDA, "the GMRES kernel does not fit on an SM");
    if (opts.precision == 1) {
      // FP32 inner GMRES: FP32 copies of the operator, its own layout, the
      // refinement kernel, FP32 work vectors and the FP64 residual
      Layout L = choose_layout<float>(g, m, gm.ES, gm.nown_b, gm.nown_w, opts.precond, no_smem, force_stream,
                                      smem_optin, false, warp);
      auto& g32 = h->gm32;
      g32.basis_smem = L.basis_smem;
      g32.mats_smem = L.mats_smem;
      g32.stream_mats = L.stream_mats;
      g32.buf_elems = L.buf_elems;
      g32.nbuf = L.nbuf;
      g32.warp_elems = L.warp_elems;
      g32.smem = L.smem;
      CU(set_smem_limit(k_gmres<float>, smem_optin));
      CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gmres<float>, kGmresThreads, g32.smem));
      if (per_sm < 1) return fail(SMPM_ECUDA, "the FP32 GMRES kernel does not fit on an SM");
      g32.smem_ref = refine_smem_bytes(m, g.M, g.n, gm.ES, gm.nown_b, gm.nown_w, g.d, false, g32.warp_elems != 0);
      if (g32.smem_ref > (size_t)smem_optin) return fail(SMPM_EINVAL, "grid too large for the refinement kernel");
      CU(set_smem_limit(k_refine, smem_optin));
      CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_refine, kGmresThreads, g32.smem_ref));
      if (per_sm < 1) return fail(SMPM_ECUDA, "the refinement kernel does not fit on an SM");
      auto to32 = [](const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); };
      if ((s = upload(h, &h->dT32, to32(Tc), st)) || (s = upload(h, &h->dG32, to32(Gc), st)) ||
          (s = upload(h, &h->dX32, to32(Xc), st)) || (s = upload(h, &h->dRs32, to32(h->f.Rs), st)) ||
          (s = upload(h, &h->dH32, to32(h->f.H), st)))
        return s;
      if ((s = dalloc(h, &h->wx32, g.kp)) || (s = dalloc(h, &h->wt32, g.kp)) || (s = dalloc(h, &h->wy32, g.kp)) ||
          (s = dalloc(h, &h->wV32, g.kp)) || (s = dalloc(h, &h->wrg32, g.kp)) || (s = dalloc(h, &h->wr, g.kp)) ||
          (s = dalloc(h, &h->wcr, g.d)))
        return s;
      if (!g32.basis_smem && (s = dalloc(h, &h->wvown32, (size_t)gm.grid * (m + 1) * gm.ES))) return s;
    }
    gm.smem_pp = prepost_smem_bytes(m, g.M, g.n, gm.ES, gm.nown_b, gm.nown_w, g.d);
    if (gm.smem_pp > (size_t)smem_optin) return fail(SMPM_EINVAL, "grid too large for the solve kernels");
    CU(set_smem_limit(k_pre, smem_optin));
    CU(set_smem_limit(k_post, smem_optin));
    for (const void* fn : {(const void*)k_pre, (const void*)k_post}) {
      int per = 0;
      CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kGmresThreads, gm.smem_pp));
      if (per < 1) return fail(SMPM_ECUDA, "the solve kernels do not fit on an SM");
    }
    std::vector<double> ztus(g.d, 0.0);
    for (long long e = 0; e < g.nel; ++e)
      for (int F = 0; F < 4; ++F) {
        int j = h->g.iface((int)e, F);
        if (j < 0) continue;
        for (int t = 0; t < g.n; ++t) ztus[j] += h->f.zw[4 * e + F] * h->f.uS[e * g.M + F * g.n + t];
      }
    if ((s = upload(h, &h->dZtuS, ztus, st))) return s;
    {
      std::vector<ElemMeta<double>> t64(g.nel);
      std::vector<ElemMeta<float>> t32(h->dT32 ? g.nel : 0);
      for (long long e = 0; e < g.nel; ++e) {
        ElemMeta<double> a{};
        a.T = h->dT;
        a.e = (int)e;
        a.M = g.M;
        a.n = g.n;
        a.mx = g.mx;
        a.my = g.my;
        t64[e] = a;
        if (h->dT32) {
          ElemMeta<float> c{};
          c.T = h->dT32;
          c.e = (int)e;
          c.M = g.M;
          c.n = g.n;
          c.mx = g.mx;
          c.my = g.my;
          t32[e] = c;
        }
      }
      if ((s = upload(h, &h->dtab64, t64, st))) return s;
      if (h->dT32 && (s = upload(h, &h->dtab32, t32, st))) return s;
      if ((s = upload_classes(h, Tc, st))) return s;
    }
    if (h->f.has_adjoint) {
      // T~_e = T_e^T: its column-major device copy is T_e row-major
      std::vector<double> Gca = transpose_blocks(h->f.Ga, g.M, h->f.black.size()),
                          Xca = transpose_blocks(h->f.Xa, g.n, 4 * h->f.black.size());
      std::vector<double> ztusa(g.d, 0.0);
      for (long long e = 0; e < g.nel; ++e)
        for (int F = 0; F < 4; ++F) {
          int j = h->g.iface((int)e, F);
          if (j < 0) continue;
          for (int t = 0; t < g.n; ++t) ztusa[j] += h->f.zwa[4 * e + F] * h->f.uSa[e * g.M + F * g.n + t];
        }
      if ((s = upload(h, &h->dTa, h->f.T, st)) || (s = upload(h, &h->dRsa, h->f.Rsa, st)) ||
          (s = upload(h, &h->dGa, Gca, st)) || (s = upload(h, &h->dXa, Xca, st)) ||
          (s = upload(h, &h->dHa, h->f.Ha, st)) || (s = upload(h, &h->dfdxT, h->f.fdxT, st)) ||
          (s = upload(h, &h->dfdyT, h->f.fdyT, st)) || (s = upload(h, &h->duSa, h->f.uSa, st)) ||
          (s = upload(h, &h->dZtuSa, ztusa, st)))
        return s;
    }
    if ((s = dalloc(h, &h->wctl, kCtlBytes)) || (s = dalloc(h, &h->wxs, g.kp))) return s;
    h->wbar = reinterpret_cast<unsigned*>(h->wctl);
    h->werr = reinterpret_cast<int*>(h->wctl + 256);
    h->wdone = reinterpret_cast<int*>(h->wctl + 260);
    h->wnref = reinterpret_cast<int*>(h->wctl + 264);
    h->wacc8 = reinterpret_cast<double*>(h->wctl + 272);
    h->wrn = reinterpret_cast<double*>(h->wctl + 336);
    if ((s = dalloc(h, &h->wacc, (size_t)(2 * m + 1) * (m + 3)))) return s;
    if (!gm.basis_smem && (s = dalloc(h, &h->wvown, (size_t)gm.grid * (m + 1) * gm.ES))) return s;
    if (opts.precond == 2 && g.d * (long long)gm.grid <= kFusedCoarseMaxAdds) {
      std::vector<double> HT((size_t)g.d * g.d);
      for (long long r = 0; r < g.d; ++r)
        for (long long j = 0; j < g.d; ++j) HT[(size_t)j * g.d + r] = h->f.H[(size_t)r * g.d + j];
      if ((s = upload(h, &h->dHT, HT, st)) || (s = dalloc(h, &h->wchatd, 2 * (size_t)g.d))) return s;
    }
  }
  CU(cudaStreamSynchronize(st));
  h->factored = true;
  return SMPM_OK;
}

}  // namespace

extern "C" {

smpm_status schur_solve(smpm_handle h, const double* f, const double* gn, double tol, int nrhs, double* u,
                        smpm_report* rep, void* stream) try {
  if (!h || !f || !u || nrhs < 1) return fail(SMPM_EINVAL, "bad arguments");
  if (!h->factored) return fail(SMPM_ESTATE, "schur_factor has not been called");
  double t = tol > 0 ? tol : h->opts.tol;
  cudaStream_t st = as_stream(stream);
  smpm_status worst = SMPM_OK;
  // several right-hand sides of an FP64 solve with block-Jacobi: lockstep
  // groups of up to kLockMaxCols columns
  const bool lock = nrhs > 1 && h->opts.precond > 0 && !(h->opts.flags & SMPM_FLAG_NO_LOCKSTEP) &&
                    h->gm.stream_mats == 0 && (h->opts.precision == 0 || h->gm32.stream_mats == 0);
  for (int k = 0; lock && k < nrhs; k += kLockMaxCols) {
    const int R = std::min(kLockMaxCols, nrhs - k);
    smpm_status s = R == 1 ? solve_one(h, f + (size_t)k * h->g.r, gn ? gn + (size_t)k * h->g.kp : nullptr,
                                       u + (size_t)k * h->g.r, t, rep ? rep + k : nullptr, st)
                           : solve_lock(h, f + (size_t)k * h->g.r, gn ? gn + (size_t)k * h->g.kp : nullptr,
                                        u + (size_t)k * h->g.r, t, R, rep ? rep + k : nullptr, st);
    if (s == SMPM_ENOTCONV || s == SMPM_EBREAKDOWN) {
      if (worst == SMPM_OK) worst = s;
    } else if (s != SMPM_OK) {
      return s;
    }
  }
  for (int k = 0; !lock && k < nrhs; ++k) {
    smpm_status s = solve_one(h, f + (size_t)k * h->g.r, gn ? gn + (size_t)k * h->g.kp : nullptr,
                              u + (size_t)k * h->g.r, t, rep ? rep + k : nullptr, st);
    if (s == SMPM_ENOTCONV || s == SMPM_EBREAKDOWN) {
      if (worst == SMPM_OK) worst = s;
    } else if (s != SMPM_OK) {
      return s;
    }
  }
  return worst;
} catch (...) {
  return host_exception();
}

smpm_status schur_solve_adjoint(smpm_handle h, const double* gbar_u, double tol, int nrhs, double* gbar_f,
                                double* gbar_g, smpm_report* rep, void* stream) try {
  if (!h || !gbar_u || !gbar_f || nrhs < 1) return fail(SMPM_EINVAL, "bad arguments");
  if (!h->factored) return fail(SMPM_ESTATE, "schur_factor has not been called");
  if (!h->f.has_adjoint) return fail(SMPM_ESTATE, "schur_factor was called without SMPM_FLAG_ADJOINT");
  double t = tol > 0 ? tol : h->opts.tol;
  cudaStream_t st = as_stream(stream);
  smpm_status worst = SMPM_OK;
  for (int k = 0; k < nrhs; ++k) {
    smpm_status s = solve_one(h, gbar_u + (size_t)k * h->g.r, nullptr, gbar_f + (size_t)k * h->g.r, t,
                              rep ? rep + k : nullptr, st, true, gbar_g ? gbar_g + (size_t)k * h->g.kp : nullptr);
    if (s == SMPM_ENOTCONV || s == SMPM_EBREAKDOWN) {
      if (worst == SMPM_OK) worst = s;
    } else if (s != SMPM_OK) {
      return s;
    }
  }
  return worst;
} catch (...) {
  return host_exception();
}

smpm_status schur_solve_host(smpm_handle h, const double* f, const double* gn, double tol, int nrhs, double* u,
                             smpm_report* rep, void* stream) try {
  if (!h || !f || !u || nrhs < 1) return fail(SMPM_EINVAL, "bad arguments");
  if (!h->factored) return fail(SMPM_ESTATE, "schur_factor has not been called");
  cudaStream_t st = as_stream(stream);
  const size_t rn = (size_t)h->g.r * nrhs, gnn = (size_t)h->g.kp * nrhs;
  if (h->sf_n < (size_t)nrhs) {
    smpm_status s;
    if ((s = dalloc(h, &h->sf, rn)) || (s = dalloc(h, &h->sg, gnn)) || (s = dalloc(h, &h->su, rn))) return s;
    h->sf_n = nrhs;
  }
  CU(cudaMemcpyAsync(h->sf, f, rn * sizeof(double), cudaMemcpyHostToDevice, st));
  if (gn) CU(cudaMemcpyAsync(h->sg, gn, gnn * sizeof(double), cudaMemcpyHostToDevice, st));
  smpm_status s = schur_solve(h, h->sf, gn ? h->sg : nullptr, tol, nrhs, h->su, rep, stream);
  if (s != SMPM_OK && s != SMPM_ENOTCONV && s != SMPM_EBREAKDOWN) return s;
  CU(cudaMemcpyAsync(u, h->su, rn * sizeof(double), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  return s;
} catch (...) {
  return host_exception();
}

#define NEED_FACTOR()                                                              \
  do {                                                                             \
    if (!h) return fail(SMPM_EINVAL, "null handle");                               \
    if (!h->factored) return fail(SMPM_ESTATE, "schur_factor has not been called"); \
  } while (0)

#define NEED_OPERATOR()                                                                          \
  do {                                                                                           \
    if (!h) return fail(SMPM_EINVAL, "null handle");                                             \
    if (!h->factored && !h->op_factored) return fail(SMPM_ESTATE, "schur_factor has not been called"); \
  } while (0)

smpm_status smpm_apply_schur(smpm_handle h, const double* v, double* y, void* stream) try {
  NEED_OPERATOR();
  if (!v || !y) return fail(SMPM_EINVAL, "null vector");
  return launch_schur(h, v, y, as_stream(stream));
} catch (...) {
  return host_exception();
}

smpm_status smpm_apply_schur32(smpm_handle h, const float* v, float* y, void* stream) try {
  NEED_OPERATOR();
  if (!v || !y) return fail(SMPM_EINVAL, "null vector");
  if (!h->dT32) return fail(SMPM_ESTATE, "FP32 factors exist only after schur_factor with precision = 1");
  const int kind = apply_kind_ok(h, h->apply_kind, true) ? h->apply_kind : SMPM_APPLY_AUTO;
  return launch_schur_kind<float>(h, kind, v, y, as_stream(stream));
} catch (...) {
  return host_exception();
}

smpm_status smpm_set_apply_kernel(smpm_handle h, int kind) try {
  NEED_OPERATOR();
  if (!apply_kind_ok(h, kind, false)) return fail(SMPM_EINVAL, "apply kernel not available on this grid");
  h->apply_kind = kind;
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

smpm_status smpm_autotune_apply(smpm_handle h, int precision, int reps, int flush, double* ms_out, int* chosen,
                                void* stream) try {
  NEED_OPERATOR();
  if (precision != 0 && precision != 1) return fail(SMPM_EINVAL, "precision must be 0 or 1");
  if (precision == 1 && !h->dT32) return fail(SMPM_ESTATE, "FP32 factors exist only after schur_factor with precision = 1");
  if (reps < 1) reps = 5;
  cudaStream_t st = as_stream(stream);
  const size_t es = precision ? sizeof(float) : sizeof(double);
  void *v = nullptr, *y = nullptr, *fl = nullptr;
  const size_t flush_bytes = flush ? ((size_t)512 << 20) : 0;  // several times L2
  auto release = [&]() {
    if (v) cudaFree(v);
    if (y) cudaFree(y);
    if (fl) cudaFree(fl);
  };
  if (cudaMalloc(&v, h->g.kp * es) != cudaSuccess || cudaMalloc(&y, h->g.kp * es) != cudaSuccess ||
      (flush_bytes && cudaMalloc(&fl, flush_bytes) != cudaSuccess)) {
    release();
    cudaGetLastError();
    return fail(SMPM_ENOMEM, "device allocation failed in the apply autotuner");
  }
  cudaEvent_t a = nullptr, b = nullptr;
  smpm_status res = SMPM_OK;
  int best = SMPM_APPLY_AUTO;
  double best_ms = 1e300;
  if (cudaMemsetAsync(v, 0, h->g.kp * es, st) != cudaSuccess || cudaEventCreate(&a) != cudaSuccess ||
      cudaEventCreate(&b) != cudaSuccess)
    res = fail(SMPM_ECUDA, "autotuner setup failed");
  for (int kind = SMPM_APPLY_WARP; res == SMPM_OK && kind <= SMPM_APPLY_CLASS; ++kind) {
    if (ms_out) ms_out[kind - 1] = -1.0;
    if (!apply_kind_ok(h, kind, precision == 1)) continue;
    std::vector<float> t;
    for (int r = 0; r <= reps && res == SMPM_OK; ++r) {  // r = 0 warms up
      if (fl && cudaMemsetAsync(fl, r & 0xff, flush_bytes, st) != cudaSuccess) res = fail(SMPM_ECUDA, "flush failed");
      if (res != SMPM_OK) break;
      cudaEventRecord(a, st);
      res = precision ? launch_schur_kind<float>(h, kind, (const float*)v, (float*)y, st)
                      : launch_schur_kind<double>(h, kind, (const double*)v, (double*)y, st);
      cudaEventRecord(b, st);
      if (res == SMPM_OK && cudaEventSynchronize(b) != cudaSuccess) res = fail(SMPM_ECUDA, "apply kernel failed");
      float ms = 0;
      if (res == SMPM_OK && r > 0 && cudaEventElapsedTime(&ms, a, b) == cudaSuccess) t.push_back(ms);
    }
    if (res != SMPM_OK || t.empty()) break;
    std::sort(t.begin(), t.end());
    const double med = t[t.size() / 2];
    if (ms_out) ms_out[kind - 1] = med;
    if (med < best_ms) { best_ms = med; best = kind; }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  release();
  if (res != SMPM_OK) return res;
  h->apply_kind = best;
  if (chosen) *chosen = best;
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

}  // extern "C"

namespace {

template <typename S>
smpm_status launch_schur_class(smpm_handle h, const S* T, const S* v, S* y, cudaStream_t st) {
  if (!h->cls_ok) return fail(SMPM_EINVAL, "the class-shared apply needs n <= 32 and its tile in shared memory");
  const int bulk = (reinterpret_cast<uintptr_t>(v) % 16 == 0) ? 1 : 0;  // bulk copies need 16-byte alignment
  k_schur_class<S><<<(unsigned)h->ntiles, 256, class_smem(h->g.M, sizeof(S)), st>>>(h->dg, T, h->dtiles, h->dclsel,
                                                                                      v, y, bulk);
  CHECK_LAUNCH();
  return SMPM_OK;
}

}  // namespace

extern "C" {

smpm_status smpm_apply_schur_class(smpm_handle h, const double* v, double* y, void* stream) try {
  NEED_OPERATOR();
  if (!v || !y) return fail(SMPM_EINVAL, "null vector");
  return launch_schur_class<double>(h, h->dTcls, v, y, as_stream(stream));
} catch (...) {
  return host_exception();
}

smpm_status smpm_apply_schur_class32(smpm_handle h, const float* v, float* y, void* stream) try {
  NEED_OPERATOR();
  if (!v || !y) return fail(SMPM_EINVAL, "null vector");
  if (!h->dTcls32) return fail(SMPM_ESTATE, "FP32 factors exist only after schur_factor with precision = 1");
  return launch_schur_class<float>(h, h->dTcls32, v, y, as_stream(stream));
} catch (...) {
  return host_exception();
}

smpm_status smpm_apply_precond(smpm_handle h, const double* v, double* t, void* stream) try {
  NEED_FACTOR();
  if (!v || !t) return fail(SMPM_EINVAL, "null vector");
  return launch_precond(h, v, t, nullptr, nullptr, as_stream(stream));
} catch (...) {
  return host_exception();
}

smpm_status smpm_apply_schur_precond(smpm_handle h, const double* v, double* y, void* stream) try {
  NEED_FACTOR();
  if (!v || !y) return fail(SMPM_EINVAL, "null vector");
  return launch_precond(h, v, h->wt, y, h->wc, as_stream(stream));
} catch (...) {
  return host_exception();
}

smpm_status smpm_apply_deflation(smpm_handle h, const double* v, double* y, void* stream) try {
  NEED_FACTOR();
  if (!v || !y) return fail(SMPM_EINVAL, "null vector");
  cudaStream_t st = as_stream(stream);
  smpm_status s;
  if ((s = launch_zt(h, v, h->wc, st))) return s;
  if ((s = launch_coarse(h, h->wc, h->wchat, st))) return s;
  return launch_defl(h, v, h->wchat, -1, y, st);
} catch (...) {
  return host_exception();
}

smpm_status smpm_apply_deflation_q(smpm_handle h, const double* v, double* y, void* stream) try {
  NEED_FACTOR();
  if (!v || !y) return fail(SMPM_EINVAL, "null vector");
  cudaStream_t st = as_stream(stream);
  smpm_status s;
  if ((s = launch_schur(h, v, h->wtmp, st))) return s;
  if ((s = launch_zt(h, h->wtmp, h->wc, st))) return s;
  if ((s = launch_coarse(h, h->wc, h->wchat, st))) return s;
  k_assemble<<<blocks_for(h->g.kp, kSlotsPerBlock), kSlotsPerBlock, 0, st>>>(h->dg, v, h->wchat, nullptr, y);
  CHECK_LAUNCH();
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

smpm_status smpm_schur_rhs(smpm_handle h, const double* b, double* bS, void* stream) try {
  NEED_FACTOR();
  if (!b || !bS) return fail(SMPM_EINVAL, "null vector");
  cudaStream_t st = as_stream(stream);
  CU(cudaMemsetAsync(bS, 0, h->g.kp * sizeof(double), st));
  k_schur_rhs<<<(unsigned)h->g.nel, kElemThreads, elem_smem(h->g.n), st>>>(h->dg, h->dfdx, h->dfdy, h->dD, b, bS);
  CHECK_LAUNCH();
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

smpm_status smpm_recover(smpm_handle h, const double* b, const double* x, double* u, void* stream) try {
  NEED_FACTOR();
  if (!b || !x || !u) return fail(SMPM_EINVAL, "null vector");
  k_recover<<<(unsigned)h->g.nel, kElemThreads, elem_smem(h->g.n), as_stream(stream)>>>(h->dg, h->dfdx, h->dfdy, b,
                                                                                        x, u);
  CHECK_LAUNCH();
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

smpm_status smpm_null_vectors(smpm_handle h, double* uL, double* uS, double* uC, void* stream) try {
  NEED_FACTOR();
  cudaStream_t st = as_stream(stream);
  if (uL) CU(cudaMemcpyAsync(uL, h->duL, h->g.r * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (uS) CU(cudaMemcpyAsync(uS, h->duS, h->g.kp * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (uC) CU(cudaMemcpyAsync(uC, h->duC, h->g.d * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

smpm_status smpm_coarse_matrix(smpm_handle h, double* C) try {
  if (!h) return fail(SMPM_EINVAL, "null handle");
  if (h->f.C.empty()) return fail(SMPM_ESTATE, "no factors: call schur_factor or smpm_factor_host_only");
  if (!C) return fail(SMPM_EINVAL, "null pointer");
  std::memcpy(C, h->f.C.data(), h->f.C.size() * sizeof(double));
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

smpm_status smpm_factor_host_only(smpm_handle h, const smpm_opts* o) try {
  if (!h) return fail(SMPM_EINVAL, "null handle");
  smpm_opts opts;
  smpm_default_opts(&opts);
  if (o) opts = *o;
  if (!(opts.tau_scale > 0) || !(opts.robin_scale > 0)) return fail(SMPM_EINVAL, "bad solver options");
  if (h->g.nel < 2) return fail(SMPM_ENOINTERFACE, "the Schur method needs mx*my >= 2 (one interface at least)");
  Factors f;
  std::string err;
  int rc = factor_host(h->g, opts, &f, &err);
  if (rc != SMPM_OK) return fail(static_cast<smpm_status>(rc), err);
  h->f = std::move(f);
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

smpm_status smpm_host_factor(smpm_handle h, const char* name, double* out, long long count, long long* len) try {
  if (!h || !name) return fail(SMPM_EINVAL, "null argument");
  const Factors& f = h->f;
  std::vector<double> tmp;
  const std::vector<double>* src = nullptr;
  std::string nm(name);
  if (nm == "x1d") src = &f.x1d;
  else if (nm == "w1d") src = &f.w1d;
  else if (nm == "D") src = &f.D;
  else if (nm == "T") src = &f.T;
  else if (nm == "G") src = &f.G;
  else if (nm == "X") src = &f.X;
  else if (nm == "C") src = &f.C;
  else if (nm == "H") src = &f.H;
  else if (nm == "c0") src = &f.c0;
  else if (nm == "uC") src = &f.uC;
  else if (nm == "uS") src = &f.uS;
  else if (nm == "B1") src = &f.B1;
  else if (nm == "uL") src = &f.uL;
  else if (nm == "what") src = &f.what;
  else if (nm == "Ta") src = &f.Ta;
  else if (nm == "Ga") src = &f.Ga;
  else if (nm == "Xa") src = &f.Xa;
  else if (nm == "Ha") src = &f.Ha;
  else if (nm == "Rsa") src = &f.Rsa;
  else if (nm == "zw") src = &f.zw;
  else if (nm == "zwa") src = &f.zwa;
  else if (nm == "Rs") src = &f.Rs;
  else if (nm == "uSa") src = &f.uSa;
  else if (nm == "fdx") src = &f.fdx;
  else if (nm == "fdxT") src = &f.fdxT;
  else if (nm == "black") { tmp.assign(f.black.begin(), f.black.end()); src = &tmp; }
  else if (nm == "null_iterations") { tmp.assign(1, (double)f.null_iterations); src = &tmp; }
  else return fail(SMPM_EINVAL, "unknown factor name " + nm);
  if (len) *len = (long long)src->size();
  if (!out) return SMPM_OK;
  if (count != (long long)src->size()) return fail(SMPM_EINVAL, "count does not match the factor length");
  std::memcpy(out, src->data(), src->size() * sizeof(double));
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

void smpm_destroy(smpm_handle h) {
  if (!h) return;
  free_all(h);
  delete h;
}


smpm_status smpm_batch_create(const smpm_handle* hs, int count, const int* nrhs, int team_size, int use_graph,
                              int precision, smpm_batch* out) try {
  if (!hs || count < 1 || !nrhs || !out || precision < -1 || precision > 1)
    return fail(SMPM_EINVAL, "bad arguments");
  *out = nullptr;
  for (int p = 0; p < count; ++p) {
    if (!hs[p] || nrhs[p] < 1) return fail(SMPM_EINVAL, "null handle or nrhs < 1 in the batch");
    if (!hs[p]->factored) return fail(SMPM_ESTATE, "a handle of the batch has not been factored");
    if (precision == 1 && !hs[p]->dT32)
      return fail(SMPM_ESTATE, "mixed precision needs every handle factored with precision 1");
    for (int q = 0; q < p; ++q)
      if (hs[q] == hs[p]) return fail(SMPM_EINVAL, "a handle appears twice in the batch");
  }
  smpm_batch b = new smpm_batch_s();
  b->hs.assign(hs, hs + count);
  b->nrhs.assign(nrhs, nrhs + count);
  b->precision = precision;
  b->use_graph = use_graph ? 1 : 0;
  long long fo = 0, go = 0, rb = 0;
  for (int p = 0; p < count; ++p) {
    b->foff.push_back(fo);
    b->goff.push_back(go);
    b->rhs_base.push_back(rb);
    fo += (long long)nrhs[p] * hs[p]->g.r;
    go += (long long)nrhs[p] * hs[p]->g.kp;
    rb += nrhs[p];
  }
  b->f_len = fo;
  b->g_len = go;
  b->ntasks = rb;
  auto bad = [&](smpm_status st) {
    smpm_batch_destroy(b);
    return st;
  };
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
    return bad(fail(SMPM_ECUDA, "no CUDA device"));
  if (cudaMalloc(&b->dbars, sizeof(unsigned) * sms) || cudaMalloc(&b->derr, 4 * sizeof(int)) ||
      cudaMalloc(&b->dio, sizeof(BatchIO)) || cudaMalloc(&b->drep, sizeof(TaskReport) * b->ntasks) ||
      cudaMallocHost(&b->hio, sizeof(BatchIO)) || cudaMallocHost(&b->hrep, sizeof(TaskReport) * b->ntasks) ||
      cudaMallocHost(&b->herr, 4 * sizeof(int)) || cudaStreamCreateWithFlags(&b->bs, cudaStreamNonBlocking) ||
      cudaEventCreate(&b->ein) || cudaEventCreate(&b->eout))
    return bad(fail(SMPM_ENOMEM, "batch allocation failed"));
  int T = team_size;
  if (T <= 0) {  // default: the smallest team size of the candidate list that fits
    T = sms;
    for (int c : {8, 16, 19, 38, 76})
      if (c <= sms) {
        smpm_status st = batch_layout(b, c);
        if (st == SMPM_OK) {
          T = c;
          break;
        }
      }
  }
  smpm_status st = batch_layout(b, T);
  if (st != SMPM_OK) return bad(st);
  {
    // per-element tables of the batched apply
    std::vector<ElemMeta<double>> t64;
    std::vector<ElemMeta<float>> t32;
    bool all32 = true;
    for (int p = 0; p < count; ++p) all32 = all32 && hs[p]->dT32 != nullptr;
    long long off = 0;
    for (int p = 0; p < count; ++p) {
      smpm_handle h = hs[p];
      for (long long e = 0; e < h->g.nel; ++e) {
        ElemMeta<double> a{};
        a.T = h->dT;
        a.off = off;
        a.e = (int)e;
        a.M = h->g.M;
        a.n = h->g.n;
        a.mx = h->g.mx;
        a.my = h->g.my;
        t64.push_back(a);
        if (all32) {
          ElemMeta<float> c{};
          c.T = h->dT32;
          c.off = off;
          c.e = (int)e;
          c.M = h->g.M;
          c.n = h->g.n;
          c.mx = h->g.mx;
          c.my = h->g.my;
          t32.push_back(c);
        }
      }
      off += h->g.kp;
      b->Mmax = std::max(b->Mmax, h->g.M);
    }
    b->nelem = (long long)t64.size();
    b->v_len = off;
    if (cudaMalloc(&b->dtab64, t64.size() * sizeof(ElemMeta<double>)) ||
        (all32 && cudaMalloc(&b->dtab32, t32.size() * sizeof(ElemMeta<float>))))
      return bad(fail(SMPM_ENOMEM, "batch allocation failed"));
    if (cudaMemcpy(b->dtab64, t64.data(), t64.size() * sizeof(ElemMeta<double>), cudaMemcpyHostToDevice) ||
        (all32 && cudaMemcpy(b->dtab32, t32.data(), t32.size() * sizeof(ElemMeta<float>), cudaMemcpyHostToDevice)))
      return bad(fail(SMPM_ECUDA, "batch table upload failed"));
  }
  *out = b;
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

smpm_status smpm_batch_info(smpm_batch b, long long* f_len, long long* g_len, long long* ntasks, int* team_size,
                            int* nteams, double* last_ms) try {
  if (!b) return fail(SMPM_EINVAL, "null batch");
  if (f_len) *f_len = b->f_len;
  if (g_len) *g_len = b->g_len;
  if (ntasks) *ntasks = b->ntasks;
  if (team_size) *team_size = b->team_size;
  if (nteams) *nteams = b->nteams;
  if (last_ms) *last_ms = b->last_ms;
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

smpm_status smpm_batch_solve(smpm_batch b, const double* f, const double* g, double* u, smpm_report* rep,
                             void* stream) try {
  if (!b || !f || !u) return fail(SMPM_EINVAL, "bad arguments");
  cudaStream_t us = as_stream(stream);
  b->hio->f = f;
  b->hio->g = g;
  b->hio->u = u;
  CU(cudaEventRecord(b->ein, us));
  CU(cudaStreamWaitEvent(b->bs, b->ein, 0));
  if (b->use_graph) {
    if (!b->gexec) {
      CU(cudaStreamBeginCapture(b->bs, cudaStreamCaptureModeThreadLocal));
      smpm_status st = batch_enqueue(b, b->bs);
      cudaGraph_t gr = nullptr;
      cudaError_t e = cudaStreamEndCapture(b->bs, &gr);
      if (st != SMPM_OK) {
        if (gr) cudaGraphDestroy(gr);
        return st;
      }
      if (e != cudaSuccess) return fail(SMPM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      b->graph = gr;
      CU(cudaGraphInstantiate(&b->gexec, b->graph, 0));
    }
    CU(cudaEventRecord(b->ein, b->bs));
    CU(cudaGraphLaunch(b->gexec, b->bs));
  } else {
    CU(cudaEventRecord(b->ein, b->bs));
    smpm_status st = batch_enqueue(b, b->bs);
    if (st != SMPM_OK) return st;
  }
  CU(cudaEventRecord(b->eout, b->bs));
  CU(cudaStreamWaitEvent(us, b->eout, 0));
  CU(cudaStreamSynchronize(b->bs));
  CU(cudaEventElapsedTime(&b->last_ms, b->ein, b->eout));
  if (b->herr[0]) {  // code, first failing task + 1, body (see k_batch)
    std::string where = "unknown";
    const long long t = (long long)b->herr[1] - 1;
    const long long col = (t >= 0 && t < (long long)b->task_col.size()) ? b->task_col[t] : -1;
    for (size_t p = 0; p < b->hs.size() && col >= 0; ++p)
      for (int k = 0; k < b->nrhs[p]; ++k)
        if (b->rhs_base[p] + k == col) where = "problem " + std::to_string(p) + " rhs " + std::to_string(k);
    static const char* what[] = {"?", "start barrier", "pre", "GMRES", "refinement", "post"};
    const int w = (b->herr[2] >= 0 && b->herr[2] <= 5) ? b->herr[2] : 0;
    return fail(SMPM_ETIMEOUT, std::string(b->herr[0] == 2 ? "a matrix copy wait" : "a team barrier") +
                                   " of the batch kernel timed out (first failure: " + where + ", " + what[w] + ")");
  }
  smpm_status worst = SMPM_OK;
  for (size_t p = 0; p < b->hs.size(); ++p)
    for (int k = 0; k < b->nrhs[p]; ++k) {
      const long long i = b->rhs_base[p] + k;
      const TaskReport& t = b->hrep[b->task_of[i]];
      smpm_report R{};
      R.iterations = t.iterations;
      R.restarts = t.restarts;
      R.refinements = t.refinements;
      R.converged = t.converged;
      R.gmres_relres = t.gmres_den > 0 ? t.gmres_num / t.gmres_den : 0.0;
      R.schur_relres = t.bsn2 > 0 ? std::sqrt(t.res2 / t.bsn2) : 0.0;
      R.launches = 1;
      R.gmres_ms = b->last_ms;
      if (!std::isfinite(R.gmres_relres) || !std::isfinite(R.schur_relres))
        return fail(SMPM_ENAN, "non-finite residual in a batched solve");
      if (!t.converged && worst == SMPM_OK) worst = t.breakdown ? SMPM_EBREAKDOWN : SMPM_ENOTCONV;
      if (rep) rep[i] = R;
    }
  if (worst != SMPM_OK)
    return fail(worst, worst == SMPM_EBREAKDOWN ? "Arnoldi breakdown before tol in a batched solve"
                                                : "a batched solve did not converge");
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

smpm_status smpm_batch_autotune(smpm_batch b, const double* f, const double* g, double* u, void* stream,
                                const int* candidates, int ncand, double* ms_out, int* chosen) try {
  if (!b || !f || !u || !candidates || ncand < 1) return fail(SMPM_EINVAL, "bad arguments");
  int best = -1;
  double best_ms = 1e300;
  for (int i = 0; i < ncand; ++i) {
    if (ms_out) ms_out[i] = -1.0;
    if (batch_layout(b, candidates[i]) != SMPM_OK) continue;
    smpm_status st = smpm_batch_solve(b, f, g, u, nullptr, stream);  // warm-up (and graph capture)
    if (st != SMPM_OK && st != SMPM_ENOTCONV) return st;
    st = smpm_batch_solve(b, f, g, u, nullptr, stream);
    if (st != SMPM_OK && st != SMPM_ENOTCONV) return st;
    if (ms_out) ms_out[i] = b->last_ms;
    if (b->last_ms < best_ms) {
      best_ms = b->last_ms;
      best = candidates[i];
    }
  }
  if (best < 0) return fail(SMPM_EINVAL, "no candidate team size fits the batch");
  smpm_status st = batch_layout(b, best);
  if (st != SMPM_OK) return st;
  if (chosen) *chosen = best;
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

smpm_status smpm_batch_task_times(smpm_batch b, int* team, double* begin_ms, double* end_ms) try {
  if (!b) return fail(SMPM_EINVAL, "null batch");
  unsigned long long t0 = ~0ull;
  for (long long i = 0; i < b->ntasks; ++i) t0 = std::min(t0, b->hrep[i].t_begin);
  for (size_t p = 0; p < b->hs.size(); ++p)
    for (int k = 0; k < b->nrhs[p]; ++k) {
      const long long i = b->rhs_base[p] + k;
      const TaskReport& t = b->hrep[b->task_of[i]];
      if (team) team[i] = t.team;
      if (begin_ms) begin_ms[i] = (double)(t.t_begin - t0) * 1e-6;
      if (end_ms) end_ms[i] = (double)(t.t_end - t0) * 1e-6;
    }
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

smpm_status smpm_set_barrier_spin_limit(long long spins) try {
  const long long v = spins > 0 ? spins : (1LL << 28);
  CU(cudaMemcpyToSymbol(g_barrier_spin_limit, &v, sizeof(v)));
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

smpm_status smpm_batch_set_apply_kernel(smpm_batch b, int kind) try {
  if (!b || kind < 0 || kind > 1) return fail(SMPM_EINVAL, "bad arguments");
  b->apply_kernel = kind;
  return SMPM_OK;
} catch (...) {
  return host_exception();
}

smpm_status smpm_batch_apply_schur(smpm_batch b, const double* v, double* y, void* stream) try {
  if (!b || !v || !y) return fail(SMPM_EINVAL, "bad arguments");
  return batch_apply<double>(b, b->dtab64, v, y, as_stream(stream));
} catch (...) {
  return host_exception();
}

smpm_status smpm_batch_apply_schur32(smpm_batch b, const float* v, float* y, void* stream) try {
  if (!b || !v || !y) return fail(SMPM_EINVAL, "bad arguments");
  if (!b->dtab32) return fail(SMPM_ESTATE, "not every handle of the batch was factored with precision 1");
  return batch_apply<float>(b, b->dtab32, v, y, as_stream(stream));
} catch (...) {
  return host_exception();
}

void smpm_batch_destroy(smpm_batch b) {
  if (!b) return;
  if (b->bs) cudaStreamSynchronize(b->bs);
  batch_free_layout(b);
  cudaFree(b->dtab64);
  cudaFree(b->dtab32);
  cudaFree(b->dbars);
  cudaFree(b->derr);
  cudaFree(b->dio);
  cudaFree(b->drep);
  cudaFreeHost(b->hio);
  cudaFreeHost(b->hrep);
  cudaFreeHost(b->herr);
  if (b->ein) cudaEventDestroy(b->ein);
  if (b->eout) cudaEventDestroy(b->eout);
  if (b->bs) cudaStreamDestroy(b->bs);
  delete b;
}

}  // extern "C"

// ============================================ allocation-free deflation
// A variant of the deflation operator y = P v for callers that cannot
// allocate device memory at the time of the call: code running inside a
// framework whose caching allocator owns the free device memory, code that
// must not trigger the implicit device synchronisation of cudaMalloc/cudaFree
// (latency-critical loops), or callers with a fixed memory budget.  Its
// scratch (Z^T v, C^+ Z^T v and a barrier word) lives in the file-scope array
// below, which every GPU that loads this library holds until exit.
namespace {

constexpr long long kNoAllocMaxInterfaces = 32768;  // d limit: 2 x 32768 doubles = 512 KiB
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxInterfaces + 32];

// Device address of g_noalloc_scratch per device, taken once with that device
// current and kept for the life of the process (it does not survive a
// cudaDeviceReset, after which the module is loaded again).
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[256] = {nullptr};

// One cooperative launch: c = Z^T v | c_hat = C^+ c | y = v - S Z c_hat.
// On a barrier timeout (not expected: all CTAs are co-resident) y is NaN.
__global__ void __launch_bounds__(256) k_deflate_noalloc(DevGeo g, const double* __restrict__ H,
                                                         const double* __restrict__ Rs, const double* v, double* y,
                                                         double* scratch) {
  double* c = scratch;
  double* chat = scratch + kNoAllocMaxInterfaces;
  unsigned* bar = reinterpret_cast<unsigned*>(scratch + 2 * kNoAllocMaxInterfaces);
  int* err = reinterpret_cast<int*>(bar + 4);
  unsigned epoch = 0;
  const int n = g.n, M = g.M, row = 2 * g.mx - 1;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x, nthr = (long long)gridDim.x * blockDim.x;
  for (long long j = tid; j < g.d; j += nthr) {  // interface sums, as k_zt
    int iy = (int)(j / row), rem = (int)(j % row), e1, F1;
    if (rem < g.mx - 1) { e1 = iy * g.mx + rem; F1 = 1; }
    else { e1 = iy * g.mx + rem - (g.mx - 1); F1 = 3; }
    int e2 = dev_neighbour(g, e1, F1);
    const double w1 = dev_zw(g, e1, F1), w2 = dev_zw(g, e2, F1 ^ 1);
    double s = 0;
    for (int t = 0; t < n; ++t) s += w1 * v[(size_t)e1 * M + F1 * n + t] + w2 * v[(size_t)e2 * M + (F1 ^ 1) * n + t];
    c[j] = s;
  }
  bool ok = grid_sync(bar, err, epoch, (int)gridDim.x);
  if (ok) {
    const int lane = threadIdx.x & 31;
    const long long nw = nthr >> 5;
    for (long long r = tid >> 5; r < g.d; r += nw) {
      const double* h = H + r * g.d;
      double acc = 0;
      for (long long j = lane; j < g.d; j += 32) acc += __ldg(h + j) * __ldcg(c + j);
      acc = warp_sum(acc);
      if (lane == 0) chat[r] = acc;
    }
    ok = grid_sync(bar, err, epoch, (int)gridDim.x);
  }
  for (long long s = tid; s < g.kp; s += nthr) y[s] = ok ? deflate_slot_cg(g, v, chat, Rs, s) : nan("");
}

}  // namespace

extern "C" smpm_status smpm_apply_deflation_noalloc(smpm_handle h, const double* v, double* y, void* stream) try {
  if (!h) return fail(SMPM_EINVAL, "null handle");
  if (h->g.d > kNoAllocMaxInterfaces)
    return fail(SMPM_EINVAL, "smpm_apply_deflation_noalloc supports at most " +
                                 std::to_string(kNoAllocMaxInterfaces) + " interfaces; this grid has " +
                                 std::to_string(h->g.d));
  if (!h->factored) return fail(SMPM_ESTATE, "schur_factor has not been called");
  if (!v || !y) return fail(SMPM_EINVAL, "null vector");
  cudaStream_t st = as_stream(stream);
  int dev = 0;
  CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return fail(SMPM_EINVAL, "device ordinal out of range");
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      CU(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_noalloc_ptr[dev];
  }
  // the barrier word and the error flag must start at zero; c and c_hat are
  // fully written before they are read
  CU(cudaMemsetAsync(scratch + 2 * kNoAllocMaxInterfaces, 0, 32 * sizeof(double), st));
  int sms = 0;
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DevGeo g = h->dg;
  const double* H = h->dH;
  const double* Rs = h->dRs;
  void* args[] = {&g, &H, &Rs, &v, &y, &scratch};
  CU(cudaLaunchCooperativeKernel((const void*)k_deflate_noalloc, dim3(sms), dim3(256), args, 0, st));
  CHECK_LAUNCH();
  return SMPM_OK;
} catch (...) {
  return host_exception();
}
