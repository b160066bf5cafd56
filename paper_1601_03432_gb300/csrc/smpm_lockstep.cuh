// Lockstep GMRES over R right-hand sides ("columns") of one grid: the R
// Arnoldi processes of Algorithm 2 / 3 (GMRES on S M^-1 or P S M^-1) advance
// together, one step at a time, in ONE persistent cooperative launch, so that
// every operator matrix (G_b, X_b, T_e, the coarse C^+) is read once per step
// for all R columns and the five grid barriers of a step are shared.  Each
// element product becomes a small dense GEMM: the M x M matrix times an
// M x RC tile of columns.
//
// Per column, everything of the single-column kernel is kept: its own basis,
// Hessenberg column, FP64 Givens rotations, residual estimate, convergence,
// breakdown and NaN flags, and its own restarts.  A column that converges
// stops (its scale is set to zero: its later basis vectors are zero and its
// Givens state is frozen); the step loop ends when every column has stopped,
// and a restart cycle restarts only the columns still running.  The
// iterates of column rho are exactly those of a single-column solve of that
// right-hand side (same phases, same CGS2 with the lazy v_j and the
// Pythagorean norm); only the order of the atomic dot-product sums differs.
//
// Layouts: column rho of a kp-vector at base + rho * vs; of a d-vector at
// base + rho * ds.  The basis lives in global memory (L2 / HBM): CTA rank's
// slice of basis vector l, column rho at V + ((rank (m+1) + l) R + rho) ES;
// w and w2 likewise (W + (rank 2R + rho) (ES+1), w2 at + R (ES+1)).
// Element work items are (owned element, chunk of RC columns); warp w takes
// items w, w + 8, ...; an item's tile of slot values lives in the warp's
// shared scratch as X[i * RC + rho].
#pragma once
// Included inside the anonymous namespace of smpm_solver.cu, after smpm_gmres.cuh.

constexpr int kLockMaxCols = 16;  // columns of one lockstep launch

struct LockColState {  // per column, written by the team's rank 0 at the end
  double beta0, tolabs, resid;
  int its, converged, breakdown, nan, cycles;
  int its_total;  // Arnoldi steps summed over the launches of a solve (zero before the first)
};

template <typename S>
struct LockArgs {
  GmresArgs<S> a;  // geometry, ownership, matrices, team, barrier, err, precond, m, maxit, tol;
                   // rhs, x, t, y, vglob: column 0 (stride vs); c, chat: column 0 (stride ds);
                   // acc: (2m+1) R (m+3) FP64 accumulators (zero on entry)
  int R;           // columns (a multiple of RC, <= kLockMaxCols)
  int RC;          // columns per element work item (1, 2, 4 or 8)
  long long vs, ds;
  S* V;            // basis, G (m+1) R ES
  S* W;            // w, w2: G 2R (ES+1)
  LockColState* cs;  // R
  double* Rh;        // R m (m+1): Hessenberg R factor per column (written by rank 0)
  double* yv;        // R m: least-squares solution per column
  const int* done;   // per column (stride done_stride ints): nonzero -> the column does not run
  int done_stride;
};

template <typename S>
struct LockSmem {
  double *gcs, *gsn, *gg, *invb, *h1, *h2, *hs1, *hs2, *colv;  // [rho * m3 + l]
  double* misc;                                                // [rho * 8 + k]
  double* scl;                                                 // scale of each column's input
  int* jc;                                                     // steps of the column in this cycle
  int* active;
  int* flags;  // [0]: any column active
  S* wb;       // per-warp tiles: 4 M RC entries per warp
  S* mats;     // resident matrices (a.mats_smem)
};

__host__ __device__ inline size_t lock_tile_elems(int M, int RC) { return 4 * (size_t)M * RC; }

template <typename S>
inline size_t lock_smem_bytes(int m, int M, int n, int R, int RC, int nown_b, int nown_w, bool mats_smem) {
  const size_t m3 = m + 3;
  size_t dbl = 9 * m3 * R + 9 * (size_t)R;
  size_t ints = 2 * (size_t)R + 4;
  size_t sel = (size_t)(kGmresThreads / 32) * lock_tile_elems(M, RC) + 16;
  if (mats_smem) sel += (size_t)nown_b * (2 * (size_t)M * M + 4 * (size_t)n * n) + (size_t)nown_w * M * M;
  return dbl * sizeof(double) + ints * sizeof(int) + 16 + sel * sizeof(S) + 128;
}

template <typename S>
__device__ LockSmem<S> lock_carve(const LockArgs<S>& A, unsigned char* raw) {
  LockSmem<S> s;
  const int m3 = A.a.m + 3, R = A.R;
  double* d = reinterpret_cast<double*>(raw);
  s.gcs = d; d += (size_t)m3 * R;
  s.gsn = d; d += (size_t)m3 * R;
  s.gg = d; d += (size_t)m3 * R;
  s.invb = d; d += (size_t)m3 * R;
  s.h1 = d; d += (size_t)m3 * R;
  s.h2 = d; d += (size_t)m3 * R;
  s.hs1 = d; d += (size_t)m3 * R;
  s.hs2 = d; d += (size_t)m3 * R;
  s.colv = d; d += (size_t)m3 * R;
  s.misc = d; d += 8 * (size_t)R;
  s.scl = d; d += R;
  int* ip = reinterpret_cast<int*>(d);
  s.jc = ip; ip += R;
  s.active = ip; ip += R;
  s.flags = ip; ip += 4;
  S* q = reinterpret_cast<S*>((reinterpret_cast<size_t>(ip) + 15) & ~size_t(15));
  s.wb = q;
  q += (size_t)(blockDim.x / 32) * lock_tile_elems(A.a.g.M, A.RC);
  q = reinterpret_cast<S*>((reinterpret_cast<size_t>(q) + 15) & ~size_t(15));
  s.mats = q;
  return s;
}

// matrices of owned block k / white element k: resident copies or global
template <typename S>
__device__ __forceinline__ const S* lk_G(const LockArgs<S>& A, const LockSmem<S>& s, int k, int ib) {
  const int M = A.a.g.M, n = A.a.g.n;
  return A.a.mats_smem ? s.mats + (size_t)k * (2 * M * M + 4 * n * n) : A.a.Gc + (size_t)ib * M * M;
}
template <typename S>
__device__ __forceinline__ const S* lk_Tb(const LockArgs<S>& A, const LockSmem<S>& s, int k, int e) {
  const int M = A.a.g.M, n = A.a.g.n;
  return A.a.mats_smem ? s.mats + (size_t)k * (2 * M * M + 4 * n * n) + M * M : A.a.Tc + (size_t)e * M * M;
}
template <typename S>
__device__ __forceinline__ const S* lk_X(const LockArgs<S>& A, const LockSmem<S>& s, int k, int ib) {
  const int M = A.a.g.M, n = A.a.g.n;
  return A.a.mats_smem ? s.mats + (size_t)k * (2 * M * M + 4 * n * n) + 2 * M * M : A.a.Xc + (size_t)ib * 4 * n * n;
}
template <typename S>
__device__ __forceinline__ const S* lk_Tw(const LockArgs<S>& A, const LockSmem<S>& s, int k, int e) {
  const int M = A.a.g.M, n = A.a.g.n;
  return A.a.mats_smem ? s.mats + (size_t)A.a.nown_b * (2 * M * M + 4 * n * n) + (size_t)k * M * M
                       : A.a.Tc + (size_t)e * M * M;
}

template <typename S>
__device__ __forceinline__ S* lk_basis(const LockArgs<S>& A, int l, int rho) {
  return A.V + (((size_t)team_rank(A.a) * (A.a.m + 1) + l) * A.R + rho) * A.a.ES;
}
template <typename S>
__device__ __forceinline__ S* lk_w(const LockArgs<S>& A, int rho) {
  return A.W + ((size_t)team_rank(A.a) * 2 * A.R + rho) * (A.a.ES + 1);
}
template <typename S>
__device__ __forceinline__ S* lk_w2(const LockArgs<S>& A, int rho) {
  return A.W + ((size_t)team_rank(A.a) * 2 * A.R + A.R + rho) * (A.a.ES + 1);
}

// Z[r * RC + c] = sum_k Amat[k * M + r] X[k * RC + c] for r < M, c < RC by one
// warp: lane l owns rows l, l+32, l+64, l+96 (M <= 128); Amat column-major in
// shared or global memory; X, Z in the warp's shared scratch.  Every product
// is a plain FMA into one of 4 RC independent accumulators.  Ends with
// __syncwarp.
template <typename S, int RC>
__device__ __forceinline__ void warp_gemm(const S* Amat, const S* X, S* Z, int M, int lane) {
  constexpr int U = sizeof(S) == 4 ? (RC >= 8 ? 4 : 8) : 2;  // columns of A per step (registers: 4 RC + 4 U)
  S acc[4][RC];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int c = 0; c < RC; ++c) acc[j][c] = S(0);
  const int nr = (M - lane + 31) / 32;
  int k = 0;
  for (; k + U <= M; k += U) {
    S av[U][4];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int j = 0; j < 4; ++j) av[u][j] = j < nr ? Amat[(size_t)(k + u) * M + lane + 32 * j] : S(0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int c = 0; c < RC; ++c) {
        const S xc = X[(k + u) * RC + c];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[j][c] += av[u][j] * xc;
      }
    }
  }
  for (; k < M; ++k) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const S av = j < nr ? Amat[(size_t)k * M + lane + 32 * j] : S(0);
#pragma unroll
      for (int c = 0; c < RC; ++c) acc[j][c] += av * X[k * RC + c];
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (j < nr)
#pragma unroll
      for (int c = 0; c < RC; ++c) Z[(lane + 32 * j) * RC + c] = acc[j][c];
  __syncwarp();
}

template <typename S>
__device__ __forceinline__ void warp_gemm_rc(int RC, const S* Amat, const S* X, S* Z, int M, int lane) {
  switch (RC) {
    case 1: warp_gemm<S, 1>(Amat, X, Z, M, lane); break;
    case 2: warp_gemm<S, 2>(Amat, X, Z, M, lane); break;
    case 4: warp_gemm<S, 4>(Amat, X, Z, M, lane); break;
    default: warp_gemm<S, 8>(Amat, X, Z, M, lane); break;
  }
}

// Black block solves for all columns: items (owned block k, chunk q of RC
// columns).  Column rho's input is sc[rho] * (the basis slice when own, else
// the global vector src).  t = M^-1 v on the block: r1 = p - X q,
// a = G r1, z = T_e a, t = [a; q - z].
template <typename S>
__device__ void lk_black(const LockArgs<S>& A, const LockSmem<S>& s, const S* src, const double* sc, int jbasis) {
  const GmresArgs<S>& a = A.a;
  const DevGeo& g = a.g;
  const int M = g.M, n = g.n, G = a.G, rank = team_rank(a), RC = A.RC, Q = A.R / A.RC;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  S* P = s.wb + (size_t)warp * lock_tile_elems(M, RC);  // [p; q]: 2M x RC
  S* Rr = P + 2 * M * RC;                                // r1, later z: M x RC
  S* Aa = Rr + M * RC;                                   // a: M x RC
  for (int it = warp; it < a.nown_b * Q; it += nwarps) {
    const int k = it / Q, c0 = (it % Q) * RC;
    const int ib = rank + k * G;
    if (ib >= a.nblack) continue;
    const int e = a.black[ib];
    for (int idx = lane; idx < 2 * M * RC; idx += 32) {
      const int c = idx / (2 * M), i = idx % (2 * M), rho = c0 + c;
      S v = S(0);
      if (jbasis >= 0) {
        v = (S)(sc[rho] * (double)lk_basis(A, jbasis, rho)[k * 2 * M + i]);
      } else {
        const long long sl = block_slot(g, e, i);
        if (sl >= 0) v = (S)(sc[rho] * (double)ldcg(src + rho * A.vs + sl));
      }
      P[i * RC + c] = v;
    }
    __syncwarp();
    const S* X = lk_X(A, s, k, ib);
    for (int idx = lane; idx < M * RC; idx += 32) {
      const int i = idx / RC, c = idx % RC, F = i / n, t = i % n;
      const S* xf = X + (size_t)F * n * n;
      const S* qf = P + (size_t)(M + F * n) * RC + c;
      S acc = 0;
      for (int cc = 0; cc < n; ++cc) acc += xf[cc * n + t] * qf[cc * RC];
      Rr[idx] = P[idx] - acc;
    }
    __syncwarp();
    warp_gemm_rc(RC, lk_G(A, s, k, ib), Rr, Aa, M, lane);
    warp_gemm_rc(RC, lk_Tb(A, s, k, e), Aa, Rr, M, lane);
    for (int idx = lane; idx < 2 * M * RC; idx += 32) {
      const int c = idx / (2 * M), i = idx % (2 * M), rho = c0 + c;
      const long long sl = block_slot(g, e, i);
      if (sl >= 0) a.t[rho * A.vs + sl] = i < M ? Aa[i * RC + c] : (S)(P[i * RC + c] - Rr[(i - M) * RC + c]);
    }
    __syncwarp();
  }
  __syncthreads();
}

// White elements for all columns: y = S t on the black slots facing e,
// y = sc * v on e's own slots, c = Z^T y on e's interfaces (with_c).
template <typename S>
__device__ void lk_white(const LockArgs<S>& A, const LockSmem<S>& s, const S* v, const double* sc, bool with_c) {
  const GmresArgs<S>& a = A.a;
  const DevGeo& g = a.g;
  const int M = g.M, n = g.n, G = a.G, rank = team_rank(a), RC = A.RC, Q = A.R / A.RC;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  S* P = s.wb + (size_t)warp * lock_tile_elems(M, RC);  // t on e's slots: M x RC
  S* Z = P + M * RC;                                     // T_e t: M x RC
  double* ci = reinterpret_cast<double*>(Z + M * RC + (sizeof(S) == 4 ? (M * RC) & 1 : 0));  // M x RC doubles
  for (int it = warp; it < a.nown_w * Q; it += nwarps) {
    const int k = it / Q, c0 = (it % Q) * RC;
    const int iw = rank + k * G;
    if (iw >= a.nwhite) continue;
    const int e = a.white[iw];
    for (int idx = lane; idx < M * RC; idx += 32) {
      const int c = idx / M, i = idx % M;
      P[i * RC + c] = ldcg(a.t + (c0 + c) * A.vs + (size_t)e * M + i);
    }
    __syncwarp();
    warp_gemm_rc(RC, lk_Tw(A, s, k, e), P, Z, M, lane);
    for (int idx = lane; idx < M * RC; idx += 32) {
      const int c = idx / M, i = idx % M, rho = c0 + c;
      const int F = i / n, tt = i % n, e2 = dev_neighbour(g, e, F);
      const S vo = (S)(sc[rho] * (double)ldcg(v + rho * A.vs + (size_t)e * M + i));
      a.y[rho * A.vs + (size_t)e * M + i] = vo;
      double c1 = 0;
      if (e2 >= 0) {
        const size_t sl = (size_t)e2 * M + (F ^ 1) * n + tt;
        const S ys = ldcg(a.t + rho * A.vs + sl) + Z[i * RC + c];
        a.y[rho * A.vs + sl] = ys;
        c1 = g.zw ? dev_zw(g, e, F) * (double)vo + dev_zw(g, e2, F ^ 1) * (double)ys : (double)vo + (double)ys;
      }
      ci[c * M + i] = c1;
    }
    __syncwarp();
    if (with_c && lane < 4 * RC) {  // face F of column c summed by lane c * 4 + F
      const int c = lane / 4, F = lane % 4, j = dev_iface(g, e, F);
      if (j >= 0) {
        double sum = 0;
        for (int tt = 0; tt < n; ++tt) sum += ci[c * M + F * n + tt];
        a.c[(c0 + c) * A.ds + j] = sum;
      }
    }
    __syncwarp();
  }
  __syncthreads();
}

// c_hat = C^+ c for all columns: the CTA takes a contiguous range of rows,
// one warp per row; lanes read consecutive entries of the row (H row-major)
// and of each column's c, two entries per lane and step, and the loads of the
// next step are issued before the FMAs of this one (software pipelining); the
// R partial sums meet in warp shuffles.
template <typename S, typename HT>
__device__ void lk_coarse_h(const LockArgs<S>& A, const HT* H) {
  const GmresArgs<S>& a = A.a;
  const int d = (int)a.g.d, R = A.R;
  const int per = (d + a.G - 1) / a.G;
  const int r0 = team_rank(a) * per, r1 = min(d, r0 + per);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  constexpr int U = 2, CG = 8;  // entries per lane and step; columns per pass over the row
  const int nfull = d / (32 * U);
  for (int r = r0 + warp; r < r1; r += nwarps) {
    const HT* hr = H + (size_t)r * d;
    for (int c0 = 0; c0 < R; c0 += CG) {
      const int nc = min(CG, R - c0);
      const double* cb = a.c + (size_t)c0 * A.ds;
      HT acc[CG];
#pragma unroll
      for (int c = 0; c < CG; ++c) acc[c] = 0;
      HT h[U], cv[CG][U];
      auto load = [&](int st) {
        const int j = st * 32 * U + lane;
#pragma unroll
        for (int u = 0; u < U; ++u) h[u] = __ldg(hr + j + 32 * u);
#pragma unroll
        for (int c = 0; c < CG; ++c)
          if (c < nc)
#pragma unroll
            for (int u = 0; u < U; ++u) cv[c][u] = (HT)__ldcg(cb + c * A.ds + j + 32 * u);
      };
      if (nfull > 0) load(0);
      for (int st = 0; st < nfull; ++st) {
        HT hh[U], cc[CG][U];
#pragma unroll
        for (int u = 0; u < U; ++u) hh[u] = h[u];
#pragma unroll
        for (int c = 0; c < CG; ++c)
#pragma unroll
          for (int u = 0; u < U; ++u) cc[c][u] = cv[c][u];
        if (st + 1 < nfull) load(st + 1);
#pragma unroll
        for (int c = 0; c < CG; ++c)
          if (c < nc)
#pragma unroll
            for (int u = 0; u < U; ++u) acc[c] += hh[u] * cc[c][u];
      }
      for (int j = nfull * 32 * U + lane; j < d; j += 32) {
        const HT hv = __ldg(hr + j);
#pragma unroll
        for (int c = 0; c < CG; ++c)
          if (c < nc) acc[c] += hv * (HT)__ldcg(cb + c * A.ds + j);
      }
#pragma unroll
      for (int c = 0; c < CG; ++c) {
        if (c < nc) {
          const double v = (double)warp_sum(acc[c]);
          if (lane == 0) a.chat[(c0 + c) * A.ds + r] = v;
        }
      }
    }
  }
}

// FP32 columns: the coarse inverse's FP32 copy (see coarse_rows32).  The R
// coarse vectors are converted to FP32 once per CTA, a chunk of dc entries of
// every column at a time, into the idle warp tiles (converting them on every
// row's pass costs as much as FP64 products); each warp keeps its rows'
// partial sums in c_hat across the chunks.
template <typename S>
__device__ void lk_coarse32_staged(const LockArgs<S>& A, float* cf, int dc) {
  const GmresArgs<S>& a = A.a;
  const int d = (int)a.g.d, R = A.R;
  const int per = (d + a.G - 1) / a.G;
  const int r0 = team_rank(a) * per, r1 = min(d, r0 + per);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  constexpr int CG = 8;
  for (int j0 = 0; j0 < d; j0 += dc) {
    const int len = min(dc, d - j0);
    for (int i = threadIdx.x; i < R * len; i += blockDim.x) {
      const int c = i / len, j = i - c * len;
      cf[(size_t)c * dc + j] = (float)__ldcg(a.c + (size_t)c * A.ds + j0 + j);
    }
    __syncthreads();
    for (int r = r0 + warp; r < r1; r += nwarps) {
      const float* hr = a.H + (size_t)r * d + j0;
      for (int c0 = 0; c0 < R; c0 += CG) {
        const int nc = min(CG, R - c0);
        const float* cc = cf + (size_t)c0 * dc;
        float acc[CG];
#pragma unroll
        for (int c = 0; c < CG; ++c) acc[c] = 0.f;
        int j = lane;
        for (; j + 32 * 7 < len; j += 32 * 8) {  // eight entries per lane per step, loaded first
          float h[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) h[u] = __ldg(hr + j + 32 * u);
#pragma unroll
          for (int c = 0; c < CG; ++c)
            if (c < nc)
#pragma unroll
              for (int u = 0; u < 8; ++u) acc[c] += h[u] * cc[(size_t)c * dc + j + 32 * u];
        }
        for (; j < len; j += 32) {
          const float hv = __ldg(hr + j);
#pragma unroll
          for (int c = 0; c < CG; ++c)
            if (c < nc) acc[c] += hv * cc[(size_t)c * dc + j];
        }
#pragma unroll
        for (int c = 0; c < CG; ++c)
          if (c < nc) {
            const float v = warp_sum(acc[c]);
            double* out = a.chat + (size_t)(c0 + c) * A.ds + r;
            if (lane == 0) *out = (j0 == 0 ? 0.0 : *out) + (double)v;
          }
      }
    }
    __syncthreads();  // the warp tiles take the next chunk, or the next phase
  }
}

template <typename S>
__device__ void lk_coarse(const LockArgs<S>& A, const LockSmem<S>& s) {
  if constexpr (sizeof(S) == 4) {
    const int room = (int)((size_t)(blockDim.x / 32) * lock_tile_elems(A.a.g.M, A.RC));
    const int dc = (room / A.R) & ~31;  // entries per column and chunk
    if (dc >= 256) {
      lk_coarse32_staged(A, reinterpret_cast<float*>(s.wb), dc);
      return;
    }
  }
  lk_coarse_h(A, A.a.H);
}

// op(sc * src) -> y (and c, chat) for all columns; with own_j >= 0 the block
// solves read basis vector own_j (owner slices), else the global src.
template <typename S>
__device__ bool lk_apply(const LockArgs<S>& A, const LockSmem<S>& s, const S* src, const double* sc, int own_j,
                         unsigned& epoch, int& trace_n) {
  const GmresArgs<S>& a = A.a;
  lk_black(A, s, src, sc, own_j);
  GM_TRACE(31);
  if (!grid_sync(a.bar, a.err, epoch, a.G)) return false;
  GM_TRACE(32);
  lk_white(A, s, src, sc, a.precond == 2);
  GM_TRACE(33);
  if (!grid_sync(a.bar, a.err, epoch, a.G)) return false;
  GM_TRACE(34);
  if (a.precond == 2) {
    lk_coarse(A, s);
    GM_TRACE(35);
    if (!grid_sync(a.bar, a.err, epoch, a.G)) return false;
    GM_TRACE(36);
  }
  return true;
}

// Dot products of the owned basis slices with the columns' vectors: for each
// pair (l, rho), l < nl, out[l * R + rho] += sum_i basis(l, rho)[i] vec(rho)[i],
// with l == nl - 1 giving vec.vec.  Work items are (pair, chunk of the ES
// entries), one warp per item: lanes read consecutive entries (coalesced),
// eight entries per lane and step loaded ahead, and the partial sum meets in
// warp shuffles before one FP64 atomic add.  FP32 products are summed in FP32
// over chunks of 16 entries per lane, chunks in FP64.
template <typename S>
__device__ void lk_dots(const LockArgs<S>& A, bool second, int nl, double* out) {
  const int E = A.a.ES, R = A.R, npairs = nl * R;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  int nch = 1;  // chunks per pair: at least two items per warp, chunks of 512 entries or more
  while (npairs * nch < 2 * nwarps && E / (nch * 2) >= 512) nch *= 2;
  const int clen = (E + nch - 1) / nch;
  for (int it = warp; it < npairs * nch; it += nwarps) {
    const int pr = it / nch, ch = it % nch;
    const int l = pr / R, rho = pr % R;
    const S* vec = second ? lk_w2(A, rho) : lk_w(A, rho);
    const S* vl = (l == nl - 1) ? vec : lk_basis(A, l, rho);
    const int i0 = ch * clen, i1 = min(E, i0 + clen);
    double sum = 0;
    if constexpr (sizeof(S) == 4) {
      int i = i0 + lane, cnt = 0;
      float f0 = 0.f;
      for (; i + 7 * 32 < i1; i += 8 * 32) {
        float bv[8], wv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          bv[u] = ldcg(vl + i + 32 * u);
          wv[u] = ldcg(vec + i + 32 * u);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) f0 = fmaf(bv[u], wv[u], f0);
        cnt += 8;
        if (cnt == 16) {
          sum += (double)f0;
          f0 = 0.f;
          cnt = 0;
        }
      }
      for (; i < i1; i += 32) f0 = fmaf(ldcg(vl + i), ldcg(vec + i), f0);
      sum += (double)f0;
    } else {
      double acc[4] = {0, 0, 0, 0};
      int i = i0 + lane;
      for (; i + 7 * 32 < i1; i += 8 * 32) {
        double bv[8], wv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          bv[u] = ldcg(vl + i + 32 * u);
          wv[u] = ldcg(vec + i + 32 * u);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u & 3] += bv[u] * wv[u];
      }
      for (; i < i1; i += 32) acc[0] += ldcg(vl + i) * ldcg(vec + i);
      sum = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    }
    sum = warp_sum(sum);
    if (lane == 0 && sum != 0.0) atomicAdd(out + pr, sum);
  }
}

// dst(rho)[i] = base(rho)[i] - sum_{l < nl} coef[rho * m3 + l] basis(l, rho)[i]
// for every column rho and owned entry i.  Each thread takes CH (column,
// entry) pairs at a time and runs the l loop over all of them, so CH
// independent loads are in flight per step (FP32 arithmetic for FP32 bases).
// With vg, the result is also written to the column's global vector at the
// entry's slot.
template <typename S>
__device__ void lk_combo_pass(const LockArgs<S>& A, bool from_w2, const double* coef, int nl, bool to_basis, int jdst,
                              bool to_vg) {
  constexpr int CH = 16;
  const GmresArgs<S>& a = A.a;
  const int E = a.ES, R = A.R, m3 = a.m + 3;
  const int NP = R * E;
  using C = typename std::conditional<sizeof(S) == 4, float, double>::type;
  for (int p0 = threadIdx.x; p0 < NP; p0 += CH * blockDim.x) {
    C acc[CH];
    int rho_[CH], i_[CH];
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const int p = p0 + q * blockDim.x;
      rho_[q] = p < NP ? p / E : 0;
      i_[q] = p < NP ? p % E : 0;
      const S* bsrc = from_w2 ? lk_w2(A, rho_[q]) : lk_w(A, rho_[q]);
      acc[q] = p < NP ? (C)ldcg(bsrc + i_[q]) : C(0);
    }
    for (int l = 0; l < nl; ++l) {
      S v[CH];
#pragma unroll
      for (int q = 0; q < CH; ++q) v[q] = ldcg(lk_basis(A, l, rho_[q]) + i_[q]);
#pragma unroll
      for (int q = 0; q < CH; ++q) acc[q] -= (C)coef[rho_[q] * m3 + l] * (C)v[q];
    }
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const int p = p0 + q * blockDim.x;
      if (p >= NP) continue;
      const S val = (S)acc[q];
      if (to_basis) {
        lk_basis(A, jdst, rho_[q])[i_[q]] = val;
      } else {
        lk_w2(A, rho_[q])[i_[q]] = val;
      }
      if (to_vg) {
        const long long sl = entry_slot(a, i_[q]);
        if (sl >= 0) a.vglob[rho_[q] * A.vs + sl] = val;
      }
    }
  }
}

// base - sum_{l < nl} coef[l] basis(l, rho)[i] (FP32 arithmetic for FP32 bases)
template <typename S>
__device__ __forceinline__ double lk_combo(const LockArgs<S>& A, double base, const double* coef, int nl, int rho,
                                           int i) {
  if constexpr (sizeof(S) == 4) {
    float r = (float)base;
    for (int l = 0; l < nl; ++l) r = fmaf(-(float)coef[l], ldcg(lk_basis(A, l, rho) + i), r);
    return (double)r;
  } else {
    double r = base;
    for (int l = 0; l < nl; ++l) r -= coef[l] * ldcg(lk_basis(A, l, rho) + i);
    return r;
  }
}

// The lockstep GMRES by the CTAs of a team; false when a wait timed out.
template <typename S>
__device__ __noinline__ bool lock_body(const LockArgs<S>& A, unsigned char* smraw, unsigned& epoch) {
  const LockSmem<S> s = lock_carve(A, smraw);
  const GmresArgs<S>& a = A.a;
  const DevGeo& g = a.g;
  const int M = g.M, n = g.n, m = a.m, m3 = m + 3, R = A.R;
  const int ES = a.ES, G = a.G, rank = team_rank(a);
  int trace_n = 0;

  // resident copies of the owned matrices
  if (a.mats_smem) {
    for (int k = 0; k < a.nown_b; ++k) {
      const int ib = rank + k * G;
      if (ib >= a.nblack) break;
      const int e = a.black[ib];
      S* dst = s.mats + (size_t)k * (2 * M * M + 4 * n * n);
      for (int i = threadIdx.x; i < M * M; i += blockDim.x) {
        dst[i] = a.Gc[(size_t)ib * M * M + i];
        dst[M * M + i] = a.Tc[(size_t)e * M * M + i];
      }
      for (int i = threadIdx.x; i < 4 * n * n; i += blockDim.x) dst[2 * M * M + i] = a.Xc[(size_t)ib * 4 * n * n + i];
    }
    for (int k = 0; k < a.nown_w; ++k) {
      const int iw = rank + k * G;
      if (iw >= a.nwhite) break;
      const int e = a.white[iw];
      S* dst = s.mats + (size_t)a.nown_b * (2 * M * M + 4 * n * n) + (size_t)k * M * M;
      for (int i = threadIdx.x; i < M * M; i += blockDim.x) dst[i] = a.Tc[(size_t)e * M * M + i];
    }
  }
  // misc per column: 0 ||w||^2, 1 ||w2||^2, 2 residual estimate, 3 state (0 running,
  // 1 converged, 2 breakdown, 3 NaN), 5 Arnoldi steps (all cycles), 6 beta0, 7 tol * beta0
  for (int c = threadIdx.x; c < R; c += blockDim.x) {
    // done flags are written by other CTAs (refinement steps of the same
    // launch in a batch): read from L2, never a stale L1 line
    s.active[c] = (A.done && *((volatile const int*)(A.done + (size_t)c * A.done_stride))) ? 0 : 1;
    s.jc[c] = 0;
    for (int k = 0; k < 8; ++k) s.misc[c * 8 + k] = 0;
  }
  int total = 0, cycle = 0;
  __syncthreads();
  bool any_active = true;
  while (true) {
    double* accN = a.acc + (size_t)(2 * m) * R * m3;
    // ---- cycle start: V[0] = rhs - op(x) for every column
    if (cycle > 0) {
      for (int c = threadIdx.x; c < R; c += blockDim.x) s.scl[c] = 1.0;
      __syncthreads();
      if (!lk_apply(A, s, a.x, s.scl, -1, epoch, trace_n)) return false;
    }
    for (int rho = 0; rho < R; ++rho) {
      S* v0 = lk_basis(A, 0, rho);
      double nn = 0;
      for (int i = threadIdx.x; i < ES; i += blockDim.x) {
        const long long sl = entry_slot(a, i);
        S rv = 0;
        if (sl >= 0 && s.active[rho]) {
          double r = (double)ldcg(a.rhs + rho * A.vs + sl);
          if (cycle > 0)
            r -= deflate_slot_cg(g, a.y + rho * A.vs, a.precond == 2 ? a.chat + rho * A.ds : nullptr, a.Rs, sl);
          rv = (S)r;
        }
        if (sl >= 0) a.vglob[rho * A.vs + sl] = rv;
        v0[i] = rv;
        nn += (double)rv * (double)rv;
      }
      nn = warp_sum(nn);
      if ((threadIdx.x & 31) == 0 && nn != 0.0) atomicAdd(accN + rho, nn);
    }
    if (!grid_sync(a.bar, a.err, epoch, a.G)) return false;
    if (threadIdx.x < R) {
      const int c = threadIdx.x;
      const double beta = sqrt(__ldcg(accN + c));
      double* mc = s.misc + c * 8;
      if (cycle == 0) {
        mc[6] = beta;
        mc[7] = a.tol * beta;
      }
      s.jc[c] = 0;
      if (s.active[c]) {
        mc[2] = beta;  // residual estimate
        if (!isfinite(beta)) {
          mc[3] = 3;  // nan
          s.active[c] = 0;
        } else if (beta <= mc[7] || beta == 0.0) {
          mc[3] = 1;  // converged
          s.active[c] = 0;
        }
      }
      s.gg[c * m3] = beta;
      s.invb[c * m3] = s.active[c] ? 1.0 / beta : 0.0;
    }
    __syncthreads();
    any_active = false;
    for (int c = 0; c < R; ++c) any_active |= s.active[c] != 0;
    if (!any_active || total >= a.maxit) break;
    int j = 0;
    for (; j < m && total < a.maxit; ++j) {
      double* accD = a.acc + (size_t)(2 * j) * R * m3;
      double* accE = a.acc + (size_t)(2 * j + 1) * R * m3;
      // ---- A: v_j = w2 - V h2 (scaled later) on the owned entries, then block solves
      GM_TRACE(30);
      if (j > 0) {
        lk_combo_pass(A, true, s.hs2, j, true, j, true);
        __syncthreads();
      }
      for (int c = threadIdx.x; c < R; c += blockDim.x) s.scl[c] = s.invb[c * m3 + j];
      __syncthreads();
      GM_TRACE(37);
      if (!lk_apply(A, s, a.vglob, s.scl, j, epoch, trace_n)) return false;
      // ---- D: w = y - S Z chat on owned entries; V^T w, ||w||^2 (four
      // (column, entry) pairs per thread at a time, their loads interleaved)
      for (int p0 = threadIdx.x; p0 < R * ES; p0 += 4 * blockDim.x) {
        double wv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int p = p0 + q * blockDim.x, rho = p / ES, i = p % ES;
          const long long sl = p < R * ES ? entry_slot(a, i) : -1;
          wv[q] = sl >= 0 ? deflate_slot_cg(g, a.y + rho * A.vs, a.precond == 2 ? a.chat + rho * A.ds : nullptr,
                                            a.Rs, sl)
                          : 0.0;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int p = p0 + q * blockDim.x;
          if (p < R * ES) lk_w(A, p / ES)[p % ES] = (S)wv[q];
        }
      }
      __syncthreads();
      GM_TRACE(38);
      lk_dots(A, false, j + 2, accD);
      GM_TRACE(39);
      if (!grid_sync(a.bar, a.err, epoch, a.G)) return false;
      GM_TRACE(40);
      for (int p = threadIdx.x; p < (j + 2) * R; p += blockDim.x) {
        const int l = p / R, c = p % R;
        double v = __ldcg(accD + p);
        if (l <= j) {
          v *= s.invb[c * m3 + l];
          s.h1[c * m3 + l] = v;
          s.hs1[c * m3 + l] = v * s.invb[c * m3 + l];
        } else {
          s.misc[c * 8 + 0] = v;  // ||w||^2
        }
      }
      __syncthreads();
      // ---- E: w2 = w - V h1; V^T w2, ||w2||^2
      lk_combo_pass(A, false, s.hs1, j + 1, false, 0, false);
      __syncthreads();
      GM_TRACE(41);
      lk_dots(A, true, j + 2, accE);
      GM_TRACE(42);
      if (!grid_sync(a.bar, a.err, epoch, a.G)) return false;
      GM_TRACE(43);
      for (int p = threadIdx.x; p < (j + 2) * R; p += blockDim.x) {
        const int l = p / R, c = p % R;
        double v = __ldcg(accE + p);
        if (l <= j) {
          v *= s.invb[c * m3 + l];
          s.h2[c * m3 + l] = v;
          s.hs2[c * m3 + l] = v * s.invb[c * m3 + l];
        } else {
          s.misc[c * 8 + 1] = v;  // ||w2||^2
        }
      }
      __syncthreads();
      // ---- Givens update of every running column (thread c), replicated in every CTA
      if (threadIdx.x < R) {
        const int c = threadIdx.x;
        double* mc = s.misc + c * 8;
        if (s.active[c]) {
          const double* h1 = s.h1 + c * m3;
          const double* h2 = s.h2 + c * m3;
          double* col = s.colv + c * m3;
          double* gcs = s.gcs + c * m3;
          double* gsn = s.gsn + c * m3;
          double* gg = s.gg + c * m3;
          double q = 0;
          for (int l = 0; l <= j; ++l) {
            q += h2[l] * h2[l];
            col[l] = h1[l] + h2[l];
          }
          const double bsq = mc[1] - q;
          const double ib = bsq > 0 ? rsqrt(bsq) : 0.0;
          const double bnext = bsq > 0 ? bsq * ib : 0.0;
          double xi = col[0];
          for (int i = 0; i < j; ++i) {
            const double x1 = col[i + 1], cc = gcs[i], sn = gsn[i];
            const double cx1 = cc * x1, sx1 = sn * x1;
            col[i] = fma(cc, xi, sx1);
            xi = fma(-sn, xi, cx1);
          }
          col[j] = xi;
          const double hh = col[j] * col[j] + bnext * bnext;
          const double iden = hh > 0 ? rsqrt(hh) : 0.0;
          const double cs = hh > 0 ? col[j] * iden : 1.0, ss = bnext * iden;
          gcs[j] = cs;
          gsn[j] = ss;
          col[j] = hh * iden;
          gg[j + 1] = -ss * gg[j];
          gg[j] = cs * gg[j];
          s.invb[c * m3 + j + 1] = ib;
          const double resid = fabs(gg[j + 1]);
          mc[2] = resid;
          s.jc[c] = j + 1;
          mc[5] += 1;
          if (rank == 0) {
            double* Rc = A.Rh + ((size_t)c * m + j) * (m + 1);
            for (int l = 0; l <= j; ++l) Rc[l] = col[l];
          }
          if (!isfinite(resid) || !isfinite(bnext)) {
            mc[3] = 3;
            s.active[c] = 0;
          } else if (resid <= mc[7]) {
            mc[3] = 1;
            s.active[c] = 0;
          } else if (bsq <= 1e-28 * mc[0]) {
            mc[3] = 2;  // breakdown
            s.active[c] = 0;
          }
          if (!s.active[c]) s.invb[c * m3 + j + 1] = 0.0;
        } else {
          s.invb[c * m3 + j + 1] = 0.0;
        }
      }
      __syncthreads();
      GM_TRACE(44);
      ++total;
      any_active = false;
      for (int c = 0; c < R; ++c) any_active |= s.active[c] != 0;
      if (!any_active) {
        ++j;
        break;
      }
    }
    // ---- end of cycle: y = R^-1 g per column (team rank 0), x += V diag(invb) y
    if (rank == 0 && threadIdx.x < R) {
      const int c = threadIdx.x, jj = s.jc[c];
      const double* gg = s.gg + c * m3;
      double* y = A.yv + (size_t)c * m;
      for (int i = jj - 1; i >= 0; --i) {
        double sum = gg[i];
        for (int k = i + 1; k < jj; ++k) sum -= A.Rh[((size_t)c * m + k) * (m + 1) + i] * y[k];
        y[i] = sum / A.Rh[((size_t)c * m + i) * (m + 1) + i];
      }
    }
    for (size_t i = (size_t)rank * blockDim.x + threadIdx.x; i < (size_t)(2 * m + 1) * R * m3;
         i += (size_t)G * blockDim.x)
      a.acc[i] = 0.0;
    if (!grid_sync(a.bar, a.err, epoch, a.G)) return false;
    for (int p = threadIdx.x; p < R * m; p += blockDim.x) {
      const int c = p / m, l = p % m;
      s.hs1[c * m3 + l] = l < s.jc[c] ? -__ldcg(A.yv + (size_t)c * m + l) * s.invb[c * m3 + l] : 0.0;
    }
    __syncthreads();
    for (int rho = 0; rho < R; ++rho) {
      const int jj = s.jc[rho];
      if (jj == 0) continue;
      for (int i = threadIdx.x; i < ES; i += blockDim.x) {
        const long long sl = entry_slot(a, i);
        if (sl < 0) continue;
        S* xp = a.x + rho * A.vs + sl;
        *xp = (S)lk_combo(A, (double)ldcg(xp), s.hs1 + rho * m3, jj, rho, i);
      }
    }
    if (!grid_sync(a.bar, a.err, epoch, a.G)) return false;
    ++cycle;
    any_active = false;
    for (int c = 0; c < R; ++c) any_active |= s.active[c] != 0;
    if (!any_active || total >= a.maxit) break;
  }
  if (rank == 0 && threadIdx.x < R) {
    const int c = threadIdx.x;
    const double* mc = s.misc + c * 8;
    LockColState st;
    st.beta0 = mc[6];
    st.tolabs = mc[7];
    st.resid = mc[2];
    st.its = (int)mc[5];
    st.converged = (mc[3] == 1 || mc[6] == 0.0) ? 1 : 0;
    st.breakdown = mc[3] == 2 ? 1 : 0;
    st.nan = mc[3] == 3 ? 1 : 0;
    st.cycles = cycle;
    st.its_total = A.cs[c].its_total + st.its;
    A.cs[c] = st;
  }
  return true;
}

// true when every column is marked done (the launch has nothing to do)
template <typename S>
__device__ __forceinline__ bool lock_all_done(const LockArgs<S>& A) {
  if (!A.done) return false;
  for (int c = 0; c < A.R; ++c)
    if (!*((volatile const int*)(A.done + (size_t)c * A.done_stride))) return false;
  return true;
}

template <typename S>
__global__ void __launch_bounds__(256, 1) k_gmres_lock(LockArgs<S> A) {
  extern __shared__ __align__(16) unsigned char smraw[];
  if (lock_all_done(A)) return;
  unsigned epoch = 0;
  lock_body(A, smraw, epoch);
}

// The right-hand-side and recovery bodies of R columns, one launch each: the
// bodies run one column after another (their barrier epoch carries on), each
// with its own arguments; the scratch vectors they share (t, y, c, c_hat)
// are only touched after a barrier that every CTA passes once it is done with
// the previous column.
__global__ void __launch_bounds__(256, 1) k_pre_cols(const PrePostArgs* __restrict__ Ps, int R) {
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned epoch = 0;
  for (int c = 0; c < R; ++c)
    if (!pre_body(Ps[c], smraw, epoch)) return;
}

__global__ void __launch_bounds__(256, 1) k_post_cols(const PrePostArgs* __restrict__ Ps, int R) {
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned epoch = 0;
  for (int c = 0; c < R; ++c)
    if (!post_body(Ps[c], smraw, epoch)) return;
}

// One refinement step (refine_body) for every column not yet done, one
// column after another.  A column's done flag is read before its body starts;
// only its own body (rank 0, after a barrier every CTA passed) sets it.
__global__ void __launch_bounds__(256, 1) k_refine_cols(const RefineArgs* __restrict__ Rs, int R) {
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned epoch = 0;
  for (int c = 0; c < R; ++c) {
    if (*((volatile const int*)Rs[c].done)) continue;
    if (refine_body(Rs[c], smraw, epoch) < 0) return;
  }
}
