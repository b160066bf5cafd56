// Cooperative kernels around the GMRES kernel (FP64): the right-hand side
// steps before it and the assembly/recovery steps after it, each one launch
// with grid barriers between its phases.  Ownership follows smpm_gmres.cuh:
// CTA c owns the checkerboard blocks and white elements c, c+G, ..., and for
// node-level work the elements e = c, c+G, ...
//
// k_pre (the projections of Sec. 1.4, the Schur right-hand side of
// Eq. schur_complement_system and the GMRES right-hand side P b_S):
//   P1  b = f + tau g on the owned elements; u_L^T b accumulated
//   P2  b <- b - u_L (u_L^T b); w = A_e^-1 b_e (fast diagonalisation); the
//       Robin fluxes of w are pushed into the neighbours' facing slots
//       (b_S = B A^-1 b); the same pass accumulates u_S^T b_S and, per face,
//       the interface sums Z^T b_S
//   P3  b_S <- b_S - u_S (u_S^T b_S) enters through Z^T b_S - (u_S^T b_S) Z^T u_S;
//       c_hat_b = C^+ Z^T b_S (coarse rows)
//   P4  owner entries: b_S projected in place, rhs = P b_S = b_S - S Z c_hat_b
// k_post (the assembly of Eq. deflated_schur, the recovery u = A^-1 (b - E x)
// and the zero-mean normalisation):
//   Q1  t = M^-1 x on the owned blocks
//   Q2  white elements: y = S t, c = Z^T y
//   Q3  c_hat = C^+ c
//   Q4  owner entries: x_S = t - Z (c_hat - c_hat_b)       [Eq. deflated_schur]
//   Q5  owned elements: u_e = A_e^-1 (b_e - E_e x_S); the pushed products
//       T_e x_S also give the true residual ||b_S - S x_S||^2; GLL-weighted
//       mean of u accumulated
//   Q6  u <- u - mean
//
// With `adjoint` set the same kernels run the transposed solve (reverse-mode
// derivative of u(f, g)), on the factors of the slot-swapped S^T (T~ = T^T,
// see the factor step) and with the transposed element operators:
//   P1  y = gbar (= dl/du); 1^T y accumulated
//   P2  y <- y - w^ (1^T y)  (N^T, N the zero-mean map); w = A_e^-T y_e; the
//       face values of w (E^T A^-T y) are pushed into the facing slots
//   P3, P4, Q1-Q4 unchanged (the transposed factors are passed in)
//   Q5  lam_e = A_e^-T (y_e - B_e^T mu_e) with mu_e the element's own slots of
//       the solution; u_L^T lam accumulated
//   Q6  dl/db = lam - u_L (u_L^T lam) written to u; dl/dg on boundary-face
//       slots = tau_F dl/db at the face node (gg, if given)
#pragma once
// Included inside the anonymous namespace of smpm_solver.cu.

struct alignas(16) PrePostArgs {  // 16-byte multiple: staged with 16-byte copies in batched solves
  GmresArgs<double> ga;  // geometry, ownership, operator matrices, t/y/c/chat buffers
  const double* fdx;
  const double* fdy;
  const double* D;
  const double* uL;
  const double* uS;
  const double* what;
  const double* ZtuS;  // d : Z^T u_S
  const double* f;
  const double* gn;
  double* b;      // r
  double* bS;     // kp
  double* rg;     // kp
  double* cb;     // d : Z^T b_S (accumulated)
  double* chatb;  // d
  double* xs;     // kp
  double* u;      // r
  double* acc;    // 8 FP64 accumulators
  double* zero[7];  // kp-long buffers zeroed in P1 (x, t, y, vglob, b_S, rhs, x_S)
  double* gacc;     // GMRES accumulators, zeroed in P1
  long long gacc_n;
  float* zero32[4];  // kp-long FP32 buffers zeroed in P1 (mixed precision), or null
  double* cr;        // d, zeroed in P1 (mixed precision), or null
  float* rg32;       // kp, FP32 copy of the GMRES right-hand side (mixed precision), or null
  int assembled;     // k_post: x_S is given in xs (skip the assembly)
  int adjoint;       // transposed solve (see above)
  double* gg;        // adjoint: kp, dl/dg per padded slot, or null
};

// accumulator slots
enum { ACC_ULB = 0, ACC_USBS = 1, ACC_MEAN = 2, ACC_RES = 3, ACC_BSN = 4, ACC_RGN = 5 };

__device__ double* fd_scratch(const Smem<double>& s) { return s.mats; }

// b_e (projected or not) is in B; solves U = A_e^-1 B.
__device__ void elem_fd(const PrePostArgs& P, int e, double* B, double* U, double* t1) {
  const DevGeo& g = P.ga.g;
  elem_solve_dev(g.n, fd_x(g, P.fdx, e), fd_y(g, P.fdy, e), B, U, t1);
}

__device__ bool pre_body(const PrePostArgs& P, unsigned char* smraw, unsigned& epoch) {
  const GmresArgs<double>& a = P.ga;
  const Smem<double> s = carve(a, smraw);
  const DevGeo& g = a.g;
  const int n = g.n, nn = n * n, M = g.M, G = a.G, rank = team_rank(a);
  double* B = fd_scratch(s);
  double* U = B + nn;
  double* t1 = U + nn;
  int trace_n = 0;
  GM_TRACE(50);
  // ---- P1: zero the work vectors; b = f + tau g; u_L^T b
  for (long long i = (long long)rank * blockDim.x + threadIdx.x; i < g.kp; i += (long long)G * blockDim.x)
    for (int v = 0; v < 7; ++v) P.zero[v][i] = 0.0;
  for (long long i = (long long)rank * blockDim.x + threadIdx.x; i < P.gacc_n; i += (long long)G * blockDim.x)
    P.gacc[i] = 0.0;
  for (long long i = (long long)rank * blockDim.x + threadIdx.x; i < g.d; i += (long long)G * blockDim.x) {
    P.cb[i] = 0.0;
    if (P.cr) P.cr[i] = 0.0;
  }
  if (P.zero32[0])
    for (long long i = (long long)rank * blockDim.x + threadIdx.x; i < g.kp; i += (long long)G * blockDim.x)
      for (int v = 0; v < 4; ++v) P.zero32[v][i] = 0.f;
  if (rank == 0 && threadIdx.x == 0) a.gs->scal[5] = 0.0;  // inner iterations of the solve
  double part = 0;
  for (long long e = rank; e < g.nel; e += G) {
    for (int q = threadIdx.x; q < nn; q += blockDim.x) {
      const int aa = q % n, bb = q / n;
      const long long gq = e * nn + q;
      double v = P.f[gq];
      if (P.gn) {
        const long long s0 = e * M;
        const double tx = face_geo(g, (int)e, 0)[0], ty = face_geo(g, (int)e, 2)[0];
        if (aa == 0 && dev_neighbour(g, (int)e, 0) < 0) v += tx * P.gn[s0 + bb];
        if (aa == n - 1 && dev_neighbour(g, (int)e, 1) < 0) v += tx * P.gn[s0 + n + bb];
        if (bb == 0 && dev_neighbour(g, (int)e, 2) < 0) v += ty * P.gn[s0 + 2 * n + aa];
        if (bb == n - 1 && dev_neighbour(g, (int)e, 3) < 0) v += ty * P.gn[s0 + 3 * n + aa];
      }
      P.b[gq] = v;
      part += P.adjoint ? v : P.uL[gq] * v;
    }
  }
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0 && part != 0.0) atomicAdd(P.acc + ACC_ULB, part);
  GM_TRACE(51);
  if (!grid_sync(a.bar, a.err, epoch, a.G)) return false;
  GM_TRACE(52);
  // ---- P2: project b; w = A_e^-1 b_e; push fluxes into b_S; u_S^T b_S; Z^T b_S
  const double alpha = __ldcg(P.acc + ACC_ULB);
  double pus = 0;
  for (long long e = rank; e < g.nel; e += G) {
    for (int q = threadIdx.x; q < nn; q += blockDim.x) {
      const long long gq = e * nn + q;
      double v = P.b[gq] - alpha * (P.adjoint ? P.what[gq] : P.uL[gq]);
      P.b[gq] = v;
      B[q] = v;
    }
    __syncthreads();
    elem_fd(P, (int)e, B, U, t1);
    // flux of w into the slot (nbr, opp F, t): -tau' (p' w - n_F . grad w) with
    // tau', p' of the neighbour's face opp F and the gradient in e's own size
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
      const int F = i / n, t = i % n;
      const int e2 = dev_neighbour(g, (int)e, F);
      double val = 0;
      if (e2 >= 0) {
        int aa, bb;
        face_node(n, F, t, &aa, &bb);
        const double* fn = face_geo(g, e2, F ^ 1);
        val = P.adjoint ? U[bb * n + aa]
                        : -fn[0] * (fn[1] * U[bb * n + aa] - normal_deriv(g, P.D, U, F, t, face_geo(g, (int)e, F)[2]));
        const size_t sl = (size_t)e2 * M + (F ^ 1) * n + t;
        P.bS[sl] = val;
        pus += P.uS[sl] * val;
        val *= dev_zw(g, e2, F ^ 1);  // its weight in Z^T b_S
      }
      s.cs[i] = val;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
      const int F = threadIdx.x, j = dev_iface(g, (int)e, F);
      if (j >= 0) {
        double sum = 0;
        for (int t = 0; t < n; ++t) sum += s.cs[F * n + t];
        atomicAdd(P.cb + j, sum);
      }
    }
    __syncthreads();
  }
  pus = warp_sum(pus);
  if ((threadIdx.x & 31) == 0 && pus != 0.0) atomicAdd(P.acc + ACC_USBS, pus);
  GM_TRACE(53);
  if (!grid_sync(a.bar, a.err, epoch, a.G)) return false;
  GM_TRACE(54);
  // ---- P3: c_hat_b = C^+ Z^T (b_S - beta u_S)
  const double beta = __ldcg(P.acc + ACC_USBS);
  if (a.precond == 2) {
    for (int j = rank * blockDim.x + threadIdx.x; j < (int)g.d; j += G * blockDim.x)
      a.c[j] = __ldcg(P.cb + j) - beta * P.ZtuS[j];
    GM_TRACE(55);
    if (!grid_sync(a.bar, a.err, epoch, a.G)) return false;
    GM_TRACE(56);
    coarse_rows(a, s);  // a.c -> a.chat
    GM_TRACE(57);
    if (!grid_sync(a.bar, a.err, epoch, a.G)) return false;
    GM_TRACE(58);
    for (int j = rank * blockDim.x + threadIdx.x; j < (int)g.d; j += G * blockDim.x)
      P.chatb[j] = __ldcg(a.chat + j);
  }
  // ---- P4: owner entries: project b_S, rhs = P b_S
  double bsn = 0, rgn = 0;
  for (int i = threadIdx.x; i < a.ES; i += blockDim.x) {
    const long long sl = entry_slot(a, i);
    if (sl < 0) continue;
    const int e = (int)(sl / M), F = (int)(sl % M) / n;
    if (dev_neighbour(g, e, F) < 0) {
      P.bS[sl] = 0.0;
      P.rg[sl] = 0.0;
      if (P.rg32) P.rg32[sl] = 0.f;
      continue;
    }
    double v = __ldcg(P.bS + sl) - beta * P.uS[sl];
    P.bS[sl] = v;
    bsn += v * v;
    double r = v;
    if (a.precond == 2) {
      // - (S Z c_hat_b) at the slot (pull form), as in the GMRES deflation
      const int ii = (int)(sl % M), t = ii % n, e2 = dev_neighbour(g, e, F);
      double acc = dev_zw(g, e, F) * __ldcg(a.chat + dev_iface(g, e, F));
      const double* R = a.Rs + ((size_t)e2 * M + (F ^ 1) * n + t) * 4;
      for (int G2 = 0; G2 < 4; ++G2) {
        const int jj = dev_iface(g, e2, G2);
        if (jj >= 0) acc += __ldg(R + G2) * __ldcg(a.chat + jj);
      }
      r -= acc;
    }
    P.rg[sl] = r;
    if (P.rg32) P.rg32[sl] = (float)r;
    rgn += r * r;
  }
  bsn = warp_sum(bsn);
  rgn = warp_sum(rgn);
  if ((threadIdx.x & 31) == 0) {
    if (bsn != 0.0) atomicAdd(P.acc + ACC_BSN, bsn);
    if (rgn != 0.0) atomicAdd(P.acc + ACC_RGN, rgn);
  }
  return true;
}

__global__ void __launch_bounds__(256, 1) k_pre(PrePostArgs P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned epoch = 0;
  pre_body(P, smraw, epoch);
}

__device__ bool post_body(const PrePostArgs& P, unsigned char* smraw, unsigned& epoch) {
  const GmresArgs<double>& a = P.ga;
  const Smem<double> s = carve(a, smraw);
  const DevGeo& g = a.g;
  const int n = g.n, nn = n * n, M = g.M, G = a.G, rank = team_rank(a);
  double* B = fd_scratch(s);
  double* U = B + nn;
  double* t1 = U + nn;
  int trace_n = 0;
  // ---- Q1-Q4: x_S
  if (P.assembled) {
    // x_S given (iterative refinement)
  } else if (a.precond == 0) {
    for (int i = threadIdx.x; i < a.ES; i += blockDim.x) {
      const long long sl = entry_slot(a, i);
      if (sl >= 0) P.xs[sl] = __ldcg(a.x + sl);
    }
  } else {
    for (int k = 0; k < a.nown_b; ++k) {
      const int ib = rank + k * G;
      if (ib >= a.nblack) break;
      const int e = a.black[ib];
      for (int i = threadIdx.x; i < 2 * M; i += blockDim.x) {
        const long long sl = block_slot(g, e, i);
        s.w[i] = sl >= 0 ? __ldcg(a.x + sl) : 0.0;
      }
      __syncthreads();
      block_solve(a, s, k, ib, e, s.w);
    }
    if (a.precond == 1) {
      GM_TRACE(61);
      if (!grid_sync(a.bar, a.err, epoch, a.G)) return false;
      GM_TRACE(62);
      for (int i = threadIdx.x; i < a.ES; i += blockDim.x) {
        const long long sl = entry_slot(a, i);
        if (sl >= 0) P.xs[sl] = __ldcg(a.t + sl);
      }
    } else {
      // white step and coarse solve of y = S t, then x_S = t - Z (c_hat - c_hat_b)
      if (!apply_op(a, s, a.x, 1.0, true, trace_n, epoch)) return false;
      for (int i = threadIdx.x; i < a.ES; i += blockDim.x) {
        const long long sl = entry_slot(a, i);
        if (sl < 0) continue;
        const int e = (int)(sl / M), F = (int)(sl % M) / n, j = dev_iface(g, e, F);
        P.xs[sl] = j < 0 ? 0.0 : __ldcg(a.t + sl) - dev_zw(g, e, F) * (__ldcg(a.chat + j) - P.chatb[j]);
      }
    }
  }
  GM_TRACE(63);
  if (!grid_sync(a.bar, a.err, epoch, a.G)) return false;
  GM_TRACE(64);
  // ---- Q5: recovery u_e = A_e^-1 (b_e - E_e x_S), residual b_S - S x_S, mean
  double pm = 0, pr = 0;
  for (long long e = rank; e < g.nel; e += G) {
    for (int q = threadIdx.x; q < nn; q += blockDim.x) B[q] = P.b[e * nn + q];
    for (int i = threadIdx.x; i < M; i += blockDim.x) s.p[i] = __ldcg(P.xs + e * M + i);
    __syncthreads();
    for (int F = 0; F < 4; ++F) {  // faces in turn: a corner node takes both slots
      if (dev_neighbour(g, (int)e, F) >= 0) {
        if (!P.adjoint) {
          for (int t = threadIdx.x; t < n; t += blockDim.x) {
            int aa, bb;
            face_node(n, F, t, &aa, &bb);
            B[bb * n + aa] -= s.p[F * n + t];
          }
        } else {
          // - B_e^T mu: the slot (F, t) feeds, through B, the flux
          // -tau' (p' u(q) - n_F.grad u(q)) at face node q = (F, t), tau' and p'
          // of the neighbour's face opp F; its transpose touches the n nodes
          // on the normal line through q
          const double* fn = face_geo(g, dev_neighbour(g, (int)e, F), F ^ 1);
          const double tau = fn[0], pw = fn[1];
          const double sc = face_geo(g, (int)e, F)[2];
          const int drow = (F & 1) ? n - 1 : 0;   // D row of the face end
          const double sgn = (F & 1) ? 1.0 : -1.0;  // outward normal along the axis
          for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
            const int t = idx / n, k = idx % n;
            const double v = s.p[F * n + t];
            const double dn = sgn * sc * __ldg(P.D + drow * n + k);
            const double coef = -tau * ((k == drow ? pw : 0.0) - dn);
            const int q = F < 2 ? t * n + k : k * n + t;
            B[q] -= coef * v;
          }
        }
      }
      __syncthreads();
    }
    elem_fd(P, (int)e, B, U, t1);
    for (int q = threadIdx.x; q < nn; q += blockDim.x) {
      P.u[e * nn + q] = U[q];
      pm += (P.adjoint ? P.uL[e * nn + q] : P.what[e * nn + q]) * U[q];
    }
    // (S x_S) on the slots facing e: x_S + T_e x_S,e
    gemv_split(a.Tc + (size_t)e * M * M, M, s.p, s.z, M, M, s.red);
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
      const int F = i / n, t = i % n, e2 = dev_neighbour(g, (int)e, F);
      if (e2 < 0) continue;
      const size_t sl = (size_t)e2 * M + (F ^ 1) * n + t;
      const double rr = P.bS[sl] - (__ldcg(P.xs + sl) + s.z[i]);
      pr += rr * rr;
    }
    __syncthreads();
  }
  pm = warp_sum(pm);
  pr = warp_sum(pr);
  if ((threadIdx.x & 31) == 0) {
    if (pm != 0.0) atomicAdd(P.acc + ACC_MEAN, pm);
    if (pr != 0.0) atomicAdd(P.acc + ACC_RES, pr);
  }
  GM_TRACE(65);
  if (!grid_sync(a.bar, a.err, epoch, a.G)) return false;
  GM_TRACE(66);
  // ---- Q6: zero GLL-weighted mean (adjoint: projection out of u_L, dl/dg)
  const double mean = __ldcg(P.acc + ACC_MEAN);
  if (!P.adjoint) {
    for (long long e = rank; e < g.nel; e += G)
      for (int q = threadIdx.x; q < nn; q += blockDim.x) P.u[e * nn + q] -= mean;
    return true;
  }
  for (long long e = rank; e < g.nel; e += G) {
    if (P.gg)
      for (int i = threadIdx.x; i < M; i += blockDim.x) {
        const int F = i / n, t = i % n;
        double v = 0;
        if (dev_neighbour(g, (int)e, F) < 0) {
          int aa, bb;
          face_node(n, F, t, &aa, &bb);
          const long long q = e * nn + bb * n + aa;
          v = face_geo(g, (int)e, F)[0] * (__ldcg(P.u + q) - mean * P.uL[q]);
        }
        P.gg[e * M + i] = v;
      }
    __syncthreads();
    for (int q = threadIdx.x; q < nn; q += blockDim.x) P.u[e * nn + q] -= mean * P.uL[e * nn + q];
  }
  return true;
}

__global__ void __launch_bounds__(256, 1) k_post(PrePostArgs P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned epoch = 0;
  post_body(P, smraw, epoch);
}

inline size_t prepost_smem_bytes(int m, int M, int n, int ES, int nown_b, int nown_w, long long d,
                                 bool w_global = false) {
  return gmres_smem_bytes<double>(m, M, n, ES, nown_b, nown_w, 0, 0, d, 0, w_global) +
         (3 * (size_t)n * n + 64) * sizeof(double);
}
