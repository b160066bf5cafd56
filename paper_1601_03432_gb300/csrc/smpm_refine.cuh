// One step of GMRES-based iterative refinement (mixed precision):
// the inner GMRES (k_gmres<float>) has solved P S M^-1 y = P r in FP32 with
// the FP64 coarse solve; this cooperative kernel turns y into the FP64
// correction and the next inner right-hand side:
//   R1  owner blocks:   t = M^-1 y                        (FP32 operator)
//   R2  white elements: S t on the black slots, c = Z^T S t (FP64 sums)
//   R3  c_hat = C^+ c                                      (FP64)
//   R4  owner entries:  x_S += t - Z (c_hat - c_hat_r)     (FP64; Eq. deflated_schur
//                       for the correction equation S d = r); y <- 0
//   R5  elements:       r = b_S - S x_S with the FP64 T_e (push form);
//                       ||r||^2 and Z^T r accumulated
//   R6  ||r|| <= tol ||P b_S||: done (all CTAs agree); otherwise
//                       c_hat_r = C^+ Z^T r                (FP64)
//   R7  owner entries:  next inner right-hand side P r = r - S Z c_hat_r (FP32)
#pragma once
// Included inside the anonymous namespace of smpm_solver.cu.

struct alignas(16) RefineArgs {  // 16-byte multiple: staged with 16-byte copies in batched solves
  GmresArgs<float> ga;   // FP32 operator and vectors: x = inner y, t, y, c, chat, rhs (next inner rhs)
  const double* Tc64;    // nel * M*M, FP64 T_e (column-major)
  const double* Rs64;    // FP64 row sums for the deflation of r
  double* xS;            // kp, FP64 Schur iterate
  const double* bS;      // kp, projected b_S
  double* r;             // kp, FP64 residual
  double* cr;            // d, Z^T r (zero on entry, left zero)
  double* chat_r;        // d, C^+ Z^T r of the current residual
  const double* rgn;     // ||P b_S||^2
  double* rn;            // ||r||^2 accumulator of this step (zero on entry)
  int* done;             // set once converged; later launches return at once
  int* nref;             // refinement steps taken
  float* rhs32;          // kp, next inner right-hand side
  double tol;
};

inline size_t refine_smem_bytes(int m, int M, int n, int ES, int nown_b, int nown_w, long long d,
                                bool w_global = false, bool warp_elems = false) {
  return gmres_smem_bytes<float>(m, M, n, ES, nown_b, nown_w, 0, 0, d, 0, w_global, 2, warp_elems) +
         (2 * (size_t)M + 256 + 16) * sizeof(double);
}

// One refinement step by the CTAs of a team; returns 1 when converged (done
// set), 0 when another inner solve follows, -1 when a barrier timed out.
__device__ int refine_body(const RefineArgs& R, unsigned char* smraw, unsigned& epoch) {
  const GmresArgs<float>& a = R.ga;
  const Smem<float> s = carve(a, smraw);
  double* p64 = reinterpret_cast<double*>(s.mats);
  double* z64 = p64 + a.g.M;
  double* red64 = z64 + a.g.M;
  const DevGeo& g = a.g;
  const int n = g.n, M = g.M, G = a.G, rank = team_rank(a);
  int trace_n = 0;
  // ---- R1-R3: t = M^-1 y, S t, c_hat
  if (!black_phase(a, s, (MatStream<float>*)nullptr, a.x, 1.0, (const float*)nullptr)) return -1;
  if (!apply_op(a, s, a.x, 1.0, true, trace_n, epoch)) return -1;
  // ---- R4: x_S += t - Z (c_hat - c_hat_r); y <- 0 for the next inner solve
  for (int i = threadIdx.x; i < a.ES; i += blockDim.x) {
    const long long sl = entry_slot(a, i);
    if (sl < 0) continue;
    const int e = (int)(sl / M), F = (int)(sl % M) / n, j = dev_iface(g, e, F);
    if (j >= 0) R.xS[sl] += (double)__ldcg(a.t + sl) - dev_zw(g, e, F) * (__ldcg(a.chat + j) - R.chat_r[j]);
    a.x[sl] = 0.f;
  }
  if (!grid_sync(a.bar, a.err, epoch, a.G)) return -1;
  // ---- R5: r = b_S - S x_S (FP64), ||r||^2, Z^T r
  double pr = 0;
  if (a.warp_elems) {  // one warp per element (elements rank + k G, k = warp, warp + nwarps, ...)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    double* pw = reinterpret_cast<double*>(s.wb + (size_t)warp * warp_scratch(M));  // 2M doubles fit in 5M floats
    double* zw = pw + M;
    for (long long e = rank + (long long)warp * G; e < g.nel; e += (long long)nwarps * G) {
      for (int i = lane; i < M; i += 32) pw[i] = __ldcg(R.xS + e * M + i);
      __syncwarp();
      warp_gemv(R.Tc64 + (size_t)e * M * M, pw, zw, M, lane);
      for (int i = lane; i < M; i += 32) {  // pw is free again: it takes the residual entries
        const int F = i / n, t = i % n, e2 = dev_neighbour(g, (int)e, F);
        double rr = 0;
        if (e2 >= 0) {
          const size_t sl = (size_t)e2 * M + (F ^ 1) * n + t;
          rr = R.bS[sl] - (__ldcg(R.xS + sl) + zw[i]);
          R.r[sl] = rr;
          pr += rr * rr;
          rr *= dev_zw(g, e2, F ^ 1);  // its weight in Z^T r
        }
        pw[i] = rr;
      }
      __syncwarp();
      if (lane < 4) {  // face F summed by lane F
        const int F = lane, j = dev_iface(g, (int)e, F);
        double sum = 0;
        for (int t = 0; t < n; ++t) sum += pw[F * n + t];
        if (j >= 0 && sum != 0.0) atomicAdd(R.cr + j, sum);
      }
      __syncwarp();
    }
  }
  for (long long e = rank; e < (a.warp_elems ? 0 : g.nel); e += G) {
    for (int i = threadIdx.x; i < M; i += blockDim.x) p64[i] = __ldcg(R.xS + e * M + i);
    __syncthreads();
    gemv_split(R.Tc64 + (size_t)e * M * M, M, p64, z64, M, M, red64);
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
      const int F = i / n, t = i % n, e2 = dev_neighbour(g, (int)e, F);
      double rr = 0;
      if (e2 >= 0) {
        const size_t sl = (size_t)e2 * M + (F ^ 1) * n + t;
        rr = R.bS[sl] - (__ldcg(R.xS + sl) + z64[i]);
        R.r[sl] = rr;
        pr += rr * rr;
        rr *= dev_zw(g, e2, F ^ 1);  // its weight in Z^T r
      }
      red64[i] = rr;
    }
    __syncthreads();
    if (threadIdx.x < 128) {  // face F summed by warp F
      const int F = threadIdx.x >> 5, lane = threadIdx.x & 31;
      double sum = 0;
      for (int t = lane; t < n; t += 32) sum += red64[F * n + t];
      sum = warp_sum(sum);
      const int j = dev_iface(g, (int)e, F);
      if (lane == 0 && j >= 0 && sum != 0.0) atomicAdd(R.cr + j, sum);
    }
    __syncthreads();
  }
  pr = warp_sum(pr);
  if ((threadIdx.x & 31) == 0 && pr != 0.0) atomicAdd(R.rn, pr);
  if (!grid_sync(a.bar, a.err, epoch, a.G)) return -1;
  // ---- R6: convergence test (uniform), else c_hat_r = C^+ Z^T r
  const double rho = sqrt(__ldcg(R.rn)), target = R.tol * sqrt(__ldcg(R.rgn));
  if (rank == 0 && threadIdx.x == 0) *R.nref += 1;
  if (rho <= target) {
    if (rank == 0 && threadIdx.x == 0) *R.done = 1;
    return 1;
  }
  {
    GmresArgs<float> b = a;
    b.c = R.cr;
    b.chat = R.chat_r;
    coarse_rows(b, s);
  }
  if (!grid_sync(a.bar, a.err, epoch, a.G)) return -1;
  // ---- R7: next inner right-hand side P r (FP32); Z^T r back to zero
  for (int i = threadIdx.x; i < a.ES; i += blockDim.x) {
    const long long sl = entry_slot(a, i);
    if (sl < 0) continue;
    R.rhs32[sl] = (float)deflate_slot_cg(g, (const double*)R.r, R.chat_r, R.Rs64, sl);
  }
  for (long long j = (long long)rank * blockDim.x + threadIdx.x; j < g.d; j += (long long)G * blockDim.x)
    R.cr[j] = 0.0;
  return 0;
}

__global__ void __launch_bounds__(256, 1) k_refine(RefineArgs R) {
  extern __shared__ __align__(16) unsigned char smraw[];
  if (*((volatile const int*)R.done)) return;
  unsigned epoch = 0;
  refine_body(R, smraw, epoch);
}
