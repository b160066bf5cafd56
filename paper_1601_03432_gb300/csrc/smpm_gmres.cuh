// Persistent GMRES kernel for x := GMRES(op, rhs) with op one of
//   S            (Algorithm 1),
//   S M^-1       (Algorithm 2),
//   P S M^-1     (Algorithm 3),
// run as ONE cooperative launch per solve: restarted GMRES(m), classical
// Gram-Schmidt with one re-orthogonalisation (CGS2), FP64 Givens rotations,
// the convergence test on the rotated residual, restarts from the true
// residual.
//
// Work is owned, not redistributed per phase: CTA c owns the checkerboard
// blocks ib = c, c + G, ... (G = grid size) -- the black elements and the
// slots of their blocks, which partition Gamma -- and the white elements
// iw = c, c + G, ...  The owner keeps its blocks' operator matrices (G_b, T_e,
// X_b and the white T_e, column-major) and its slice of the Krylov basis in
// shared memory when they fit, so an Arnoldi step touches L2/HBM only for the
// vectors exchanged between neighbouring elements.  One step:
//   A  owner: v_j = w2 - V h2 on its block slots (lazy, see E), then the
//      block solve t = M^-1 v_j: a = G (p - X q), b = q - T_e a
//   B  white elements: y = S t (y = v on white-owned slots), c = Z^T y
//   C  c_hat = C^+ c (dense FP64 rows spread over all CTAs; Algorithm 3)
//   D  owner: w = y - S Z c_hat; V^T w and ||w||^2, accumulated with FP64
//      atomics in L2
//   E  owner: w2 = w - V h1; V^T w2 and ||w2||^2 likewise; every CTA forms
//      ||v_{j+1}||^2 = ||w2||^2 - ||h2||^2 and applies the same Givens
//      rotations to its own copy, so all CTAs take the same decision.
// Phases are separated by a grid barrier (5 per step for Algorithm 3).  The
// basis is kept unnormalised with the inverse norms replicated in every CTA.
// FP64 products are plain per-thread FMA chains (thread per matrix row, per
// basis vector, per slot): FP64 issue slots are scarce on this part, so the
// hot path uses no warp-shuffle reduction trees.
//
// Data written by other CTAs inside the kernel is read with ld.global.cg: L1
// is not coherent across SMs.  The grid barrier spins with a bound and raises
// an error flag instead of hanging.
#pragma once
// Included inside the anonymous namespace of smpm_solver.cu.

template <typename S>
struct GmresArgs {
  DevGeo g;
  const int* black;
  const int* white;
  int nblack, nwhite;
  const S* Tc;      // nel * M*M, column-major T_e
  const S* Gc;      // nblack * M*M, column-major G_b
  const S* Xc;      // nblack * 4*n*n, column-major X_F blocks
  const S* Rs;      // nel * M*4 row sums of T_e (deflation)
  // d*d row-major coarse inverse: FP64, or its FP32 copy for the FP32 inner
  // solves of the mixed-precision path
  const typename std::conditional<sizeof(S) == 4, float, double>::type* H;
  S* vglob;         // kp : current basis vector (raw), exchanged between CTAs
  S* vown;          // G * (m+1) * ES : basis slices when not resident in smem
  S* t;             // kp
  S* y;             // kp
  double* c;        // d
  double* chat;     // d
  const S* rhs;     // kp
  S* x;             // kp (zero on entry)
  double* acc;      // (2m + 1) * (m + 3) FP64 accumulators (zero on entry)
  GState* gs;
  unsigned* bar;    // barrier counter (zero on entry)
  int* err;
  int precond, m, maxit;
  double tol;
  int nown_b, nown_w;  // blocks / white elements per CTA (ceil)
  int ES;              // entries per CTA in the basis slice (odd, >= 2M nown_b)
  int mats_smem;       // 1: owned matrices resident in shared memory
  int basis_smem;      // 1: basis slice resident in shared memory
  int stream_mats;     // 1: owned matrices streamed through two shared buffers (bulk copies)
  int buf_elems;       // elements of S per stream buffer (>= M*M + 4*n*n, multiple of 16 bytes)
  int nbuf;            // stream buffers (2..kMaxStreamBufs): nbuf - 1 items in flight while one is used
  int warp_elems;      // 1: each warp works on its own block / white element (many per CTA); 0: the
                       // whole CTA works on one element at a time
  long long* trace;
  int trace_cap;
  const int* skip;  // when non-null and set on entry, the kernel returns at once
  int* its_out;     // when non-null: Arnoldi steps of this launch
  int G;            // CTAs working on this solve (a team; the whole grid for one solve)
  int base;         // first CTA of the team: the CTA's rank is blockIdx.x - base
  S* wscr;          // when non-null: per-CTA global scratch for w, w2 (2 (ES+1) per rank)
  // fused coarse solve (Algorithm 3 steps only): each white element adds
  // H[:, j] c_j for its interfaces j into c_hat as soon as c_j is known, so
  // the separate coarse phase and its grid barrier disappear
  int fused;           // 1: use HT / chatd in the Arnoldi steps
  const double* HT;    // d*d, H column-major (HT[j d + r] = H[r][j])
  double* chatd;       // 2 d: c_hat of even / odd steps (accumulated with atomics)
};

// rank of this CTA within the team that works on a solve
template <typename S>
__device__ __forceinline__ int team_rank(const GmresArgs<S>& a) {
  return (int)blockIdx.x - a.base;
}

#define GM_TRACE(tag)                                                                   \
  do {                                                                                  \
    if (a.trace && team_rank(a) == 0 && threadIdx.x == 0 && trace_n + 2 <= a.trace_cap) { \
      a.trace[trace_n++] = (tag);                                                       \
      a.trace[trace_n++] = clock64();                                                   \
    }                                                                                   \
  } while (0)

template <typename S>
__device__ __forceinline__ S ldcg(const S* p) {
  return __ldcg(p);
}

// Team barrier on a monotonic counter: thread 0 of each CTA adds one with
// release semantics and polls with acquire loads until the counter reaches
// the CTA's next epoch (a multiple of the team size G; the team is the whole
// grid for a single solve).  Bounded spin; err is set on timeout and the
// caller unwinds.
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Polls of a barrier wait before it gives up (default 2^28, about a minute
// of polling; smpm_set_barrier_spin_limit lowers it to exercise the timeout).
__device__ long long g_barrier_spin_limit = 1LL << 28;

// work: run by thread 0 between its arrival and its wait (serial work of this
// CTA overlapped with the other CTAs' arrival); it must touch only what no
// other CTA reads before the barrier completes.
template <typename Work>
__device__ bool grid_sync_with(unsigned* bar, int* err, unsigned& epoch, int G, Work&& work) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    epoch += (unsigned)G;
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(bar), "r"(1u) : "memory");
    work();
    long long spins = 0;
    const long long limit = g_barrier_spin_limit;
    while ((int)(ld_acquire(bar) - epoch) < 0) {
      if (++spins > limit) {  // this CTA's own timeout: code 1 unless a failure is recorded
        atomicCAS(err, 0, 1);
        ok = 0;
        break;
      }
      if ((spins & 4095) == 0 && *((volatile int*)err)) {  // another CTA failed: unwind
        ok = 0;
        break;
      }
    }
  }
  __syncthreads();
  return ok != 0;
}

__device__ bool grid_sync(unsigned* bar, int* err, unsigned& epoch, int G) {
  return grid_sync_with(bar, err, epoch, G, [] {});
}

// slot of entry i (< 2M) of the block of black element e: own slots first,
// then the neighbours' slots facing e; -1 where a face has no neighbour.
__device__ __forceinline__ long long block_slot(const DevGeo& g, int e, int i) {
  const int M = g.M, n = g.n;
  if (i < M) return (long long)e * M + i;
  i -= M;
  int F = i / n, t = i % n;
  int e2 = dev_neighbour(g, e, F);
  return e2 >= 0 ? (long long)e2 * M + (F ^ 1) * n + t : -1;
}

// per-warp scratch of the warp-per-element phases: p, q (the block's own and
// facing slots), r1, a, z
__host__ __device__ __forceinline__ int warp_scratch(int M) { return 5 * M; }

template <typename S>
struct Smem {
  double *h1, *h2, *hs1, *hs2, *gcs, *gsn, *gg, *col, *invb, *misc, *cs;
  S *p, *r1, *av, *z, *red;
  S *w, *w2;
  double* cst;  // staged coarse vector c (d)
  double* cpv;  // fused coarse: c_j of the owned white elements' interfaces (4 per element)
  int* cpj;     // and their interface indices (-1: none)
  S* V;     // (m+1) * ES when resident
  S* mats;  // resident matrices, or the two stream buffers
  S* wb;    // warp_elems: per-warp element scratch, kWarpScratch(M) entries per warp
  unsigned long long* mbar;  // mbarriers of the matrix stream (kMaxStreamBufs)
};

template <typename S>
__device__ Smem<S> carve(const GmresArgs<S>& a, unsigned char* raw) {
  Smem<S> s;
  const int m = a.m, M = a.g.M;
  double* d = reinterpret_cast<double*>(raw);
  s.mbar = reinterpret_cast<unsigned long long*>(d); d += kMaxStreamBufs;
  s.h1 = d; d += m + 3;
  s.h2 = d; d += m + 3;
  s.hs1 = d; d += m + 3;
  s.hs2 = d; d += m + 3;
  s.gcs = d; d += m + 3;
  s.gsn = d; d += m + 3;
  s.gg = d; d += m + 3;
  s.col = d; d += m + 3;
  s.invb = d; d += m + 3;
  s.misc = d; d += 16;
  s.cs = d; d += M;
  s.cst = d; d += a.g.d + 1;
  s.cpv = d; d += 4 * (size_t)a.nown_w;
  s.cpj = reinterpret_cast<int*>(d); d += 2 * (size_t)a.nown_w;
  S* q = reinterpret_cast<S*>(d);
  s.p = q; q += M;
  s.r1 = q; q += M;
  s.av = q; q += M;
  s.z = q; q += M;
  s.red = q; q += 256;
  if (a.wscr) {
    s.w = a.wscr + (size_t)team_rank(a) * 2 * (a.ES + 1);
    s.w2 = s.w + a.ES + 1;
  } else {
    s.w = q; q += a.ES + 1;
    s.w2 = q; q += a.ES + 1;
  }
  if (a.warp_elems) {  // 16-byte aligned base; each warp's 5M entries keep that alignment (M = 4n)
    q = reinterpret_cast<S*>((reinterpret_cast<size_t>(q) + 15) & ~size_t(15));
    s.wb = q;
    q += (size_t)(blockDim.x / 32) * warp_scratch(M);
  } else {
    s.wb = nullptr;
  }
  s.V = q;
  if (a.basis_smem) q += (size_t)(m + 1) * a.ES;
  q = reinterpret_cast<S*>((reinterpret_cast<size_t>(q) + 15) & ~size_t(15));
  s.mats = q;
  return s;
}

template <typename S>
inline size_t gmres_smem_bytes(int m, int M, int n, int ES, int nown_b, int nown_w, int basis_smem, int mats_smem,
                               long long d, int stream_elems = 0, bool w_global = false, int nbuf = 2,
                               bool warp_elems = false) {
  size_t dbl = kMaxStreamBufs + 9 * (size_t)(m + 3) + 16 + M + (size_t)d + 1 + 6 * (size_t)nown_w;
  size_t sel = 4 * (size_t)M + 256 + (w_global ? 0 : 2 * (size_t)(ES + 1));
  if (warp_elems) sel += (size_t)(kGmresThreads / 32) * warp_scratch(M) + 16 / sizeof(S);
  if (basis_smem) sel += (size_t)(m + 1) * ES;
  if (mats_smem) sel += (size_t)nown_b * (2 * (size_t)M * M + 4 * (size_t)n * n) + (size_t)nown_w * M * M;
  sel += (size_t)nbuf * stream_elems;
  return dbl * sizeof(double) + sel * sizeof(S) + 128;
}

// pointers to the owned matrices (shared-memory copies or global)
template <typename S>
__device__ __forceinline__ const S* mat_G(const GmresArgs<S>& a, const Smem<S>& s, int k, int ib) {
  const int M = a.g.M, n = a.g.n;
  return a.mats_smem ? s.mats + (size_t)k * (2 * M * M + 4 * n * n) : a.Gc + (size_t)ib * M * M;
}
template <typename S>
__device__ __forceinline__ const S* mat_Tb(const GmresArgs<S>& a, const Smem<S>& s, int k, int e) {
  const int M = a.g.M, n = a.g.n;
  return a.mats_smem ? s.mats + (size_t)k * (2 * M * M + 4 * n * n) + M * M : a.Tc + (size_t)e * M * M;
}
template <typename S>
__device__ __forceinline__ const S* mat_X(const GmresArgs<S>& a, const Smem<S>& s, int k, int ib) {
  const int M = a.g.M, n = a.g.n;
  return a.mats_smem ? s.mats + (size_t)k * (2 * M * M + 4 * n * n) + 2 * M * M : a.Xc + (size_t)ib * 4 * n * n;
}
template <typename S>
__device__ __forceinline__ const S* mat_Tw(const GmresArgs<S>& a, const Smem<S>& s, int k, int e) {
  const int M = a.g.M, n = a.g.n;
  return a.mats_smem ? s.mats + (size_t)a.nown_b * (2 * M * M + 4 * n * n) + (size_t)k * M * M
                     : a.Tc + (size_t)e * M * M;
}

template <typename S>
__device__ __forceinline__ S* basis(const GmresArgs<S>& a, const Smem<S>& s, int l) {
  return a.basis_smem ? s.V + (size_t)l * a.ES : a.vown + ((size_t)team_rank(a) * (a.m + 1) + l) * a.ES;
}

// ---- matrix stream: bulk copies into two shared-memory buffers ------------
// Item sequence of a CTA (cyclic, the order in which the phases use them):
// for each owned block k: [G_k | X_k], [T_e(k)]; then for each owned white
// element: [T_e].  Item i lives in buffer i % nbuf; while it is used the next
// nbuf - 1 items are in flight.  Thread 0 issues; waits are bounded.  Every
// thread orders its earlier shared-memory accesses before the copy engine's
// writes (fence.proxy.async) ahead of the barrier that precedes an issue.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  for (long long spins = 0; spins < (1LL << 22); ++spins) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

template <typename S>
struct MatStream {
  int nb, nw, nitems;
  long long issued, consumed;
};

template <typename S>
__device__ void ms_issue(const GmresArgs<S>& a, const Smem<S>& s, MatStream<S>& ms) {
  if (ms.nitems == 0) return;
  const long long i = ms.issued++;
  if (threadIdx.x != 0) return;
  const int M = a.g.M, n = a.g.n, G = a.G, rank = team_rank(a);
  const int it = (int)(i % ms.nitems), b = (int)(i % a.nbuf);
  S* dst = s.mats + (size_t)b * a.buf_elems;
  unsigned long long* bar = s.mbar + b;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const unsigned mm = (unsigned)(M * M * sizeof(S)), xx = (unsigned)(4 * n * n * sizeof(S));
  if (it < 2 * ms.nb) {
    const int k = it >> 1, ib = rank + k * G;
    if ((it & 1) == 0) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(mm + xx)
                   : "memory");
      bulk_g2s(dst, a.Gc + (size_t)ib * M * M, mm, bar);
      bulk_g2s(dst + (size_t)M * M, a.Xc + (size_t)ib * 4 * n * n, xx, bar);
    } else {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(mm) : "memory");
      bulk_g2s(dst, a.Tc + (size_t)a.black[ib] * M * M, mm, bar);
    }
  } else {
    const int k = it - 2 * ms.nb, iw = rank + k * G;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(mm) : "memory");
    bulk_g2s(dst, a.Tc + (size_t)a.white[iw] * M * M, mm, bar);
  }
}

// wait for the next item; returns its buffer (null on timeout, err set)
template <typename S>
__device__ const S* ms_acquire(const GmresArgs<S>& a, const Smem<S>& s, MatStream<S>& ms) {
  const long long i = ms.consumed;
  const int b = (int)(i % a.nbuf);
  const unsigned parity = (unsigned)((i / a.nbuf) & 1);
  __shared__ int ok;
  if (threadIdx.x == 0) ok = mbar_wait(s.mbar + b, parity) ? 1 : 0;
  __syncthreads();
  if (!ok) {
    if (threadIdx.x == 0) atomicCAS(a.err, 0, 2);  // code 2: a matrix copy did not complete
    return nullptr;
  }
  return s.mats + (size_t)b * a.buf_elems;
}

// done with the current item: the buffer is refilled with item consumed + nbuf
template <typename S>
__device__ void ms_release(const GmresArgs<S>& a, const Smem<S>& s, MatStream<S>& ms) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  ++ms.consumed;
  ms_issue(a, s, ms);
}

// wait (bounded) for the copies still in flight before the body returns,
// then invalidate the stream's mbarriers: the shared memory they occupy is
// reused by the next body of a batched solve.  (A copy that never completed
// leaves its mbarrier as it is: the caller is unwinding with the error flag
// set and reuses nothing.)
template <typename S>
__device__ void ms_drain(const GmresArgs<S>& a, const Smem<S>& s, MatStream<S>& ms) {
  if (!a.stream_mats) return;
  bool all_done = true;
  while (ms.consumed < ms.issued) {
    const long long i = ms.consumed++;
    if (threadIdx.x == 0 && !mbar_wait(s.mbar + (i % a.nbuf), (unsigned)((i / a.nbuf) & 1))) all_done = false;
  }
  __syncthreads();
  if (threadIdx.x == 0 && all_done)
    for (int b = 0; b < a.nbuf; ++b)
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(s.mbar + b)) : "memory");
  __syncthreads();
}

// ---- element phases ---------------------------------------------------------
// Block solve of one black block from the block-slot values vb[0..2M)
// (already scaled), t = M^-1 v on the block, in two halves around the
// matrix stream: (1) r1 = p - X q, a = G r1; (2) z = T_e a, write t.
template <typename S>
__device__ void block_solve_a(const GmresArgs<S>& a, const Smem<S>& s, const S* G, const S* X, const S* vb) {
  const int M = a.g.M, n = a.g.n;
  int P = 1;
  while (P * 2 * M <= (int)blockDim.x && P < 8) P *= 2;
  const int t = threadIdx.x, r = t % M, part = t / M;
  if (part < P) {
    const int F = r / n, tt = r % n;
    const S* xf = X + (size_t)F * n * n;
    const S* xq = vb + M + F * n;
    S acc = 0;
    for (int c = part; c < n; c += P) acc += xf[c * n + tt] * xq[c];
    s.red[part * M + r] = acc;
  }
  __syncthreads();
  for (int i = t; i < M; i += blockDim.x) {
    S sum = s.red[i];
    for (int p = 1; p < P; ++p) sum += s.red[p * M + i];
    s.r1[i] = vb[i] - sum;
  }
  __syncthreads();
  gemv_split(G, M, s.r1, s.av, M, M, s.red);
}

template <typename S>
__device__ void block_solve_b(const GmresArgs<S>& a, const Smem<S>& s, int e, const S* T, const S* vb) {
  const int M = a.g.M;
  gemv_split(T, M, s.av, s.z, M, M, s.red);
  for (int i = threadIdx.x; i < 2 * M; i += blockDim.x) {
    long long sl = block_slot(a.g, e, i);
    if (sl < 0) continue;
    a.t[sl] = i < M ? s.av[i] : (S)(vb[i] - s.z[i - M]);
  }
  __syncthreads();
}

template <typename S>
__device__ void block_solve(const GmresArgs<S>& a, const Smem<S>& s, int k, int ib, int e, const S* vb) {
  block_solve_a(a, s, mat_G(a, s, k, ib), mat_X(a, s, k, ib), vb);
  block_solve_b(a, s, e, mat_Tb(a, s, k, e), vb);
}

// White element: y = S t on the black slots facing e, y = sc*v on e's slots,
// c = Z^T y on e's interfaces (with_c).
template <typename S>
__device__ void white_step(const GmresArgs<S>& a, const Smem<S>& s, const S* Tw, int e, const S* v, double sc,
                           bool with_c, int kstage = -1) {
  const DevGeo& g = a.g;
  const int M = g.M, n = g.n;
  for (int i = threadIdx.x; i < M; i += blockDim.x) s.p[i] = ldcg(a.t + (size_t)e * M + i);
  __syncthreads();
  gemv_split(Tw, M, s.p, s.z, M, M, s.red);
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    int F = i / n, tt = i % n;
    int e2 = dev_neighbour(g, e, F);
    S vo = (S)(sc * (double)ldcg(v + (size_t)e * M + i));
    a.y[(size_t)e * M + i] = vo;
    double ci = 0;
    if (e2 >= 0) {
      size_t sl = (size_t)e2 * M + (F ^ 1) * n + tt;
      S ys = ldcg(a.t + sl) + s.z[i];
      a.y[sl] = ys;
      ci = g.zw ? dev_zw(g, e, F) * (double)vo + dev_zw(g, e2, F ^ 1) * (double)ys : (double)vo + (double)ys;
    }
    s.cs[i] = ci;
  }
  __syncthreads();
  if (with_c && threadIdx.x < 128) {  // face F summed by warp F
    const int F = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double sum = 0;
    for (int tt = lane; tt < n; tt += 32) sum += s.cs[F * n + tt];
    sum = warp_sum(sum);
    const int j = dev_iface(g, e, F);
    if (lane == 0 && j >= 0) a.c[j] = sum;
    if (lane == 0 && kstage >= 0) {
      s.cpv[kstage * 4 + F] = sum;
      s.cpj[kstage * 4 + F] = j;
    }
  }
  __syncthreads();
}

// Push form y = S (sc*v) for element e (Algorithm 1).
template <typename S>
__device__ void push_step(const GmresArgs<S>& a, const Smem<S>& s, int e, const S* v, double sc) {
  const DevGeo& g = a.g;
  const int M = g.M, n = g.n;
  for (int i = threadIdx.x; i < M; i += blockDim.x) s.p[i] = (S)(sc * (double)ldcg(v + (size_t)e * M + i));
  __syncthreads();
  gemv_split(a.Tc + (size_t)e * M * M, M, s.p, s.z, M, M, s.red);
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    int F = i / n, tt = i % n;
    int e2 = dev_neighbour(g, e, F);
    if (e2 >= 0) {
      size_t sl = (size_t)e2 * M + (F ^ 1) * n + tt;
      a.y[sl] = (S)(sc * (double)ldcg(v + sl)) + s.z[i];
    } else {
      a.y[(size_t)e * M + i] = s.p[i];
    }
  }
  __syncthreads();
}

// c_hat = H c: CTA c takes a contiguous range of rows; c is staged in shared
// memory and P lanes split each row (H row-major: lanes read consecutive
// columns), partial sums meet in warp shuffles.  Each lane keeps eight loads
// in flight (16-byte loads when rows start 16-byte aligned, i.e. d even), so
// that a matrix larger than L2 streams at HBM rate; such a matrix is read
// with the evict-first hint, which keeps the Krylov basis resident in L2.
__device__ __forceinline__ double2 ld_h2(const double* p, bool stream) {
  return stream ? __ldcs(reinterpret_cast<const double2*>(p)) : __ldg(reinterpret_cast<const double2*>(p));
}
__device__ __forceinline__ double ld_h1(const double* p, bool stream) { return stream ? __ldcs(p) : __ldg(p); }

// The FP32 inner solves of the mixed-precision path apply the coarse
// inverse in FP32 (its FP32 copy, FP32 products and sums): an inner solve
// needs only a relative 1e-4, and every refinement sweep recomputes the
// residual in FP64.
__device__ void coarse_rows32(const float* __restrict__ H32, const double* c, double* chat, int d, int r0, int r1,
                              float* cf) {
  for (int j = threadIdx.x; j < d; j += blockDim.x) cf[j] = (float)__ldcg(c + j);
  __syncthreads();
  const int rows = r1 - r0;
  int P = 32;
  while (P > 1 && P * rows > 2 * (int)blockDim.x) P >>= 1;
  const int lane = threadIdx.x % P, grp = threadIdx.x / P, ngrp = blockDim.x / P;
  const bool vec = (d & 3) == 0;  // rows start 16-byte aligned
  for (int rb = 0; rb < rows; rb += ngrp) {
    const int r = r0 + rb + grp;
    float sum = 0.f;
    if (r < r1) {
      const float* hr = H32 + (size_t)r * d;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      int j = vec ? 4 * lane : lane;
      if (vec) {
        for (; j + 28 * P < d; j += 32 * P) {
          float4 h[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) h[u] = __ldg(reinterpret_cast<const float4*>(hr + j + 4 * u * P));
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int jj = j + 4 * u * P;
            acc[u & 3] += h[u].x * cf[jj] + h[u].y * cf[jj + 1] + h[u].z * cf[jj + 2] + h[u].w * cf[jj + 3];
          }
        }
        for (; j < d; j += 4 * P) {
          const float4 h = __ldg(reinterpret_cast<const float4*>(hr + j));
          acc[0] += h.x * cf[j] + h.y * cf[j + 1] + h.z * cf[j + 2] + h.w * cf[j + 3];
        }
      } else {
        for (; j + 7 * P < d; j += 8 * P) {
          float h[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) h[u] = __ldg(hr + j + u * P);
#pragma unroll
          for (int u = 0; u < 8; ++u) acc[u & 3] += h[u] * cf[j + u * P];
        }
        for (; j < d; j += P) acc[0] += __ldg(hr + j) * cf[j];
      }
      sum = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    }
    for (int o = P / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, P);
    if (lane == 0 && r < r1) chat[r] = (double)sum;
  }
}

template <typename S>
__device__ void coarse_rows(const GmresArgs<S>& a, const Smem<S>& s) {
  const int d = (int)a.g.d;
  const int per = (d + a.G - 1) / a.G;
  const int r0 = team_rank(a) * per, r1 = min(d, r0 + per);
  if (r0 >= r1) return;
  if constexpr (sizeof(S) == 4) {
    coarse_rows32(a.H, a.c, a.chat, d, r0, r1, reinterpret_cast<float*>(s.cst));
    return;
  } else {
  for (int j = threadIdx.x; j < d; j += blockDim.x) s.cst[j] = __ldcg(a.c + j);
  __syncthreads();
  const bool stream = (size_t)d * d * sizeof(double) > ((size_t)48 << 20);
  const bool vec = (d & 1) == 0;
  const int rows = r1 - r0;
  int P = 32;
  while (P > 1 && P * rows > 2 * (int)blockDim.x) P >>= 1;
  const int lane = threadIdx.x % P, grp = threadIdx.x / P, ngrp = blockDim.x / P;
  const double* cs = s.cst;
  for (int rb = 0; rb < rows; rb += ngrp) {  // uniform trip count per warp
    const int r = r0 + rb + grp;
    double sum = 0;
    if (r < r1) {
      const double* hr = a.H + (size_t)r * d;
      double acc[4] = {0, 0, 0, 0};
      if (vec) {
        int j = 2 * lane;
        for (; j + 30 * P < d; j += 32 * P) {
          double2 h[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) h[u] = ld_h2(hr + j + 2 * u * P, stream);
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int jj = j + 2 * u * P;
            acc[u & 3] += h[u].x * cs[jj] + h[u].y * cs[jj + 1];
          }
        }
        for (; j < d; j += 2 * P) {
          const double2 h = ld_h2(hr + j, stream);
          acc[0] += h.x * cs[j] + h.y * cs[j + 1];
        }
      } else {
        int j = lane;
        for (; j + 7 * P < d; j += 8 * P) {
          double h[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) h[u] = ld_h1(hr + j + u * P, stream);
#pragma unroll
          for (int u = 0; u < 8; ++u) acc[u & 3] += h[u] * cs[j + u * P];
        }
        for (; j < d; j += P) acc[0] += ld_h1(hr + j, stream) * cs[j];
      }
      sum = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    }
    for (int o = P / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, P);
    if (lane == 0 && r < r1) a.chat[r] = sum;
  }
  }
}

// w = y - S Z chat for one slot (pull form); chat == nullptr gives w = y.
template <typename S>
__device__ __forceinline__ double deflate_slot_cg(const DevGeo& g, const S* y, const double* chat,
                                                  const S* __restrict__ Rs, long long sl) {
  const int M = g.M, n = g.n;
  int e = (int)(sl / M), i = (int)(sl % M), F = i / n, t = i % n;
  int e2 = dev_neighbour(g, e, F);
  if (e2 < 0) return 0.0;
  double ys = (double)ldcg(y + sl);
  if (!chat) return ys;
  double acc = __ldcg(chat + dev_iface(g, e, F));
  if (g.zw) acc *= dev_zw(g, e, F);  // uniform grids: weight 1, no FP64 multiply
  const S* R = Rs + ((size_t)e2 * M + (F ^ 1) * n + t) * 4;
#pragma unroll
  for (int G = 0; G < 4; ++G) {
    int jj = dev_iface(g, e2, G);
    if (jj >= 0) acc += (double)__ldg(R + G) * __ldcg(chat + jj);
  }
  return ys - acc;
}

// Dot products of the owned basis slice with vec (ES entries) for l < nl,
// l == nl - 1 giving vec.vec: P lanes per l (P a power of two <= 32, P*nl <=
// blockDim when possible) read consecutive entries; partial sums meet in warp
// shuffles and are added atomically to out[l] (FP64, in L2).
template <typename S>
__device__ void owned_dots(const GmresArgs<S>& a, const Smem<S>& s, const S* vec, int nl, double* out) {
  const int E = a.ES;
  int P = 32;
  while (P > 1 && P * nl > (int)blockDim.x) P >>= 1;
  const int ngrp = blockDim.x / P, lane = threadIdx.x % P, grp = threadIdx.x / P;
  for (int lb = 0; lb < nl; lb += ngrp) {  // uniform trip count per warp
    const int l = lb + grp;
    double sum = 0;
    if (l < nl) {
      const S* vl = (l == nl - 1) ? vec : basis(a, s, l);
      // eight entries per step, loaded before they are used: with the basis
      // in global memory each lane keeps eight independent loads in flight
      if constexpr (sizeof(S) == 4) {
        // FP32 products summed in FP32 over chunks of 16, chunks added in FP64
        int i = lane, cnt = 0;
        float f0 = 0.f;
        for (; i + 7 * P < E; i += 8 * P) {
          float bv[8], wv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            bv[u] = (float)vl[i + u * P];
            wv[u] = (float)vec[i + u * P];
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
        for (; i < E; i += P) f0 = fmaf((float)vl[i], (float)vec[i], f0);
        sum += (double)f0;
      } else {
        double acc[4] = {0, 0, 0, 0};
        int i = lane;
        for (; i + 7 * P < E; i += 8 * P) {
          double bv[8], wv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            bv[u] = (double)vl[i + u * P];
            wv[u] = (double)vec[i + u * P];
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) acc[u & 3] += bv[u] * wv[u];
        }
        for (; i < E; i += P) acc[0] += (double)vl[i] * (double)vec[i];
        sum = (acc[0] + acc[1]) + (acc[2] + acc[3]);
      }
    }
    for (int o = P / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, P);
    if (l < nl && lane == 0 && sum != 0.0) atomicAdd(out + l, sum);
  }
}

// base[i] - sum_{l < nl} coef[l] * basis(l)[i] for one owned entry; FP32
// arithmetic for FP32 bases (coefficients rounded once), FP64 otherwise.
template <typename S>
__device__ __forceinline__ double basis_combo(const GmresArgs<S>& a, const Smem<S>& s, double base, const double* coef,
                                              int nl, int i) {
  if constexpr (sizeof(S) == 4) {
    float r = (float)base;
    for (int l = 0; l < nl; ++l) r = fmaf(-(float)coef[l], (float)basis(a, s, l)[i], r);
    return (double)r;
  } else {
    double r = base;
    for (int l = 0; l < nl; ++l) r -= coef[l] * (double)basis(a, s, l)[i];
    return r;
  }
}

template <typename S>
__device__ __forceinline__ long long entry_slot(const GmresArgs<S>& a, int i) {
  const int M2 = 2 * a.g.M;
  int k = i / M2, ii = i % M2;
  int ib = team_rank(a) + k * a.G;
  if (k >= a.nown_b || ib >= a.nblack) return -1;
  return block_slot(a.g, a.black[ib], ii);
}

// ---- warp-per-element phases -------------------------------------------
// z[r] = sum_c A[c*M + r] x[c] for r < M by one warp: lane l owns rows
// l, l+32, ... (up to NR of them, M <= 32 NR); A column-major in shared or
// global memory (read-only), U columns per step with all their loads issued
// first (U NR independent loads per lane in flight: from global memory each
// step is one round trip); x and z in the warp's shared scratch.  Ends with
// __syncwarp.
template <typename S, int U, int NR>
__device__ __forceinline__ void warp_gemv_u(const S* A, const S* x, S* z, int M, int lane) {
  S acc[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) acc[j] = S(0);
  const int nr = (M - lane + 31) / 32;  // rows of this lane (0..NR)
  int c = 0;
  for (; c + U <= M; c += U) {
    S av[U][NR];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int j = 0; j < NR; ++j) av[u][j] = j < nr ? A[(size_t)(c + u) * M + lane + 32 * j] : S(0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const S xc = x[c + u];
#pragma unroll
      for (int j = 0; j < NR; ++j) acc[j] += av[u][j] * xc;
    }
  }
  for (; c < M; ++c) {
    const S xc = x[c];
#pragma unroll
    for (int j = 0; j < NR; ++j)
      if (j < nr) acc[j] += A[(size_t)c * M + lane + 32 * j] * xc;
  }
#pragma unroll
  for (int j = 0; j < NR; ++j)
    if (j < nr) z[lane + 32 * j] = acc[j];
  __syncwarp();
}

template <typename S>
__device__ __forceinline__ void warp_gemv(const S* A, const S* x, S* z, int M, int lane) {
  // lane owns rows lane + 32 j; U columns of loads are issued before their
  // FMAs, so a warp keeps U * NR loads in flight (M <= 64: 16 columns x 2
  // rows, else 8 x 4): matrices streamed from HBM need the bytes in flight
  // more than the FP64 pipe needs short chains
  if (M <= 64)
    warp_gemv_u<S, 16, 2>(A, x, z, M, lane);
  else
    warp_gemv_u<S, 8, 4>(A, x, z, M, lane);
}

// Black block solves with one warp per owned block (blocks k = warp,
// warp + nwarps, ...): vb = sc * (own slice or src), r1 = p - X q, a = G r1,
// z = T_e a, t = [a; q - z] on the block's slots.
template <typename S>
__device__ void black_phase_warps(const GmresArgs<S>& a, const Smem<S>& s, const S* src, double sc, const S* own) {
  const DevGeo& g = a.g;
  const int M = g.M, n = g.n, G = a.G, rank = team_rank(a);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  S* p = s.wb + (size_t)warp * warp_scratch(M);
  S* q = p + M;
  S* r1 = q + M;
  S* av = r1 + M;
  S* z = av + M;
  for (int k = warp; k < a.nown_b; k += nwarps) {
    const int ib = rank + k * G;
    if (ib >= a.nblack) break;
    const int e = a.black[ib];
    for (int i = lane; i < 2 * M; i += 32) {
      S v;
      if (own) {
        v = (S)(sc * (double)own[k * 2 * M + i]);
      } else {
        const long long sl = block_slot(g, e, i);
        v = sl >= 0 ? (S)(sc * (double)ldcg(src + sl)) : S(0);
      }
      p[i] = v;  // p and q are contiguous: q = p + M
    }
    __syncwarp();
    const S* X = mat_X(a, s, k, ib);
    for (int i = lane; i < M; i += 32) {
      const int F = i / n, t = i % n;
      const S* xf = X + (size_t)F * n * n;
      S acc = 0;
      for (int c = 0; c < n; ++c) acc += xf[c * n + t] * q[F * n + c];
      r1[i] = p[i] - acc;
    }
    __syncwarp();
    warp_gemv(mat_G(a, s, k, ib), r1, av, M, lane);
    warp_gemv(mat_Tb(a, s, k, e), av, z, M, lane);
    for (int i = lane; i < 2 * M; i += 32) {
      const long long sl = block_slot(g, e, i);
      if (sl >= 0) a.t[sl] = i < M ? av[i] : (S)(q[i - M] - z[i - M]);
    }
    __syncwarp();
  }
  __syncthreads();
}

// White elements with one warp per element: y = S t on the black slots
// facing e, y = sc*v on e's slots, c = Z^T y on e's interfaces (with_c).
template <typename S>
__device__ void white_phase_warps(const GmresArgs<S>& a, const Smem<S>& s, const S* v, double sc, bool with_c,
                                  bool stage = false) {
  const DevGeo& g = a.g;
  const int M = g.M, n = g.n, G = a.G, rank = team_rank(a);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  S* p = s.wb + (size_t)warp * warp_scratch(M);
  S* z = p + M;
  double* ci = reinterpret_cast<double*>(z + M + (M & 1));  // M doubles (within the 5M scratch for S = float
                                                             // and for S = double)
  for (int k = warp; k < a.nown_w; k += nwarps) {
    const int iw = rank + k * G;
    if (iw >= a.nwhite) break;
    const int e = a.white[iw];
    for (int i = lane; i < M; i += 32) p[i] = ldcg(a.t + (size_t)e * M + i);
    __syncwarp();
    warp_gemv(mat_Tw(a, s, k, e), p, z, M, lane);
    for (int i = lane; i < M; i += 32) {
      const int F = i / n, tt = i % n, e2 = dev_neighbour(g, e, F);
      const S vo = (S)(sc * (double)ldcg(v + (size_t)e * M + i));
      a.y[(size_t)e * M + i] = vo;
      double c1 = 0;
      if (e2 >= 0) {
        const size_t sl = (size_t)e2 * M + (F ^ 1) * n + tt;
        const S ys = ldcg(a.t + sl) + z[i];
        a.y[sl] = ys;
        c1 = g.zw ? dev_zw(g, e, F) * (double)vo + dev_zw(g, e2, F ^ 1) * (double)ys : (double)vo + (double)ys;
      }
      ci[i] = c1;
    }
    __syncwarp();
    if (with_c && lane < 4) {  // face F summed by lane F
      const int F = lane, j = dev_iface(g, e, F);
      double sum = 0;
      if (j >= 0) {
        for (int tt = 0; tt < n; ++tt) sum += ci[F * n + tt];
        a.c[j] = sum;
      }
      if (stage) {
        s.cpv[k * 4 + F] = sum;
        s.cpj[k * 4 + F] = j;
      }
    }
    __syncwarp();
  }
  __syncthreads();
}

// black block solves of this CTA from the global vector sc * src
template <typename S>
__device__ bool black_phase(const GmresArgs<S>& a, const Smem<S>& s, MatStream<S>* ms, const S* src, double sc,
                            const S* own) {
  if (a.warp_elems) {
    black_phase_warps(a, s, src, sc, own);
    return true;
  }
  const DevGeo& g = a.g;
  const int M = g.M, G = a.G;
  for (int k = 0; k < a.nown_b; ++k) {
    int ib = team_rank(a) + k * G;
    if (ib >= a.nblack) break;
    int e = a.black[ib];
    for (int i = threadIdx.x; i < 2 * M; i += blockDim.x) {
      if (own) {
        s.w[i] = (S)(sc * (double)own[k * 2 * M + i]);
      } else {
        long long sl = block_slot(g, e, i);
        s.w[i] = sl >= 0 ? (S)(sc * (double)ldcg(src + sl)) : S(0);
      }
    }
    __syncthreads();
    if (ms) {
      const S* GX = ms_acquire(a, s, *ms);
      if (!GX) return false;
      block_solve_a(a, s, GX, GX + (size_t)M * M, s.w);
      ms_release(a, s, *ms);
      const S* T = ms_acquire(a, s, *ms);
      if (!T) return false;
      block_solve_b(a, s, e, T, s.w);
      ms_release(a, s, *ms);
    } else {
      block_solve(a, s, k, ib, e, s.w);
    }
  }
  return true;
}

// op(sc * src) -> y (and c, chat).  With t_done the owners have already
// written t = M^-1 v for their blocks.  With chat_acc (fused coarse solve,
// Algorithm 3 only) the white phase also adds H[:, j] c_j for the interfaces
// of the CTA's white elements into chat_acc (zero on entry), and there is no
// separate coarse phase: c_hat is complete after the white phase's barrier.
template <typename S>
__device__ bool apply_op(const GmresArgs<S>& a, const Smem<S>& s, const S* src, double sc, bool t_done,
                         int& trace_n, unsigned& epoch, MatStream<S>* ms = nullptr, double* chat_acc = nullptr) {
  const DevGeo& g = a.g;
  const int G = a.G;
  if (a.precond == 0) {
    for (long long e = team_rank(a); e < g.nel; e += G) push_step(a, s, (int)e, src, sc);
    return grid_sync(a.bar, a.err, epoch, a.G);
  }
  if (!t_done && !black_phase(a, s, ms, src, sc, (const S*)nullptr)) return false;
  GM_TRACE(20);
  if (!grid_sync(a.bar, a.err, epoch, a.G)) return false;
  GM_TRACE(21);
  const bool fuse = chat_acc && a.precond == 2;
  if (fuse)
    for (int q = threadIdx.x; q < 4 * a.nown_w; q += blockDim.x) s.cpj[q] = -1;
  __syncthreads();
  if (a.warp_elems) white_phase_warps(a, s, src, sc, a.precond == 2, fuse);
  for (int k = 0; k < (a.warp_elems ? 0 : a.nown_w); ++k) {
    int iw = team_rank(a) + k * G;
    if (iw >= a.nwhite) break;
    if (ms) {
      const S* T = ms_acquire(a, s, *ms);
      if (!T) return false;
      white_step(a, s, T, a.white[iw], src, sc, a.precond == 2, fuse ? k : -1);
      ms_release(a, s, *ms);
    } else {
      white_step(a, s, mat_Tw(a, s, k, a.white[iw]), a.white[iw], src, sc, a.precond == 2, fuse ? k : -1);
    }
  }
  if (fuse) {  // c_hat += sum over this CTA's interfaces j of H[:, j] c_j
    __syncthreads();
    const int d = (int)g.d, nq = 4 * a.nown_w;
    for (int r = threadIdx.x; r < d; r += blockDim.x) {
      double acc = 0;
      for (int q = 0; q < nq; ++q) {
        const int j = s.cpj[q];
        if (j >= 0) acc += __ldg(a.HT + (size_t)j * d + r) * s.cpv[q];
      }
      if (acc != 0.0) atomicAdd(chat_acc + r, acc);
    }
  }
  GM_TRACE(22);
  if (!grid_sync(a.bar, a.err, epoch, a.G)) return false;
  GM_TRACE(23);
  if (a.precond == 2 && !fuse) {
    coarse_rows(a, s);
    GM_TRACE(24);
    if (!grid_sync(a.bar, a.err, epoch, a.G)) return false;
    GM_TRACE(25);
  }
  return true;
}

// Givens update of Hessenberg column j (thread 0; every CTA runs it on its
// own copy): the j earlier rotations applied to s.col, the new rotation from
// s.col[j] and the subdiagonal entry s.misc[4], the rotated right-hand side
// gg and its last entry |gg[j+1]| (the residual estimate) in s.misc[2].
template <typename S>
__device__ void givens_column(const GmresArgs<S>& a, const Smem<S>& s, int j, int rank) {
  const double bnext = s.misc[4];
  // the rotated entry is carried in a register: one dependent FMA per
  // rotation (the products with the unrotated entries do not depend on the
  // chain); the operands of eight rotations are loaded into registers ahead
  // of them, so only the FMA chain is serial
  double xi = s.col[0];
  int i0 = 0;
  for (; i0 + 8 <= j; i0 += 8) {
    double x1[8], c[8], sn[8], out[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      x1[u] = s.col[i0 + u + 1];
      c[u] = s.gcs[i0 + u];
      sn[u] = s.gsn[i0 + u];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const double cx1 = c[u] * x1[u], sx1 = sn[u] * x1[u];
      out[u] = fma(c[u], xi, sx1);
      xi = fma(-sn[u], xi, cx1);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) s.col[i0 + u] = out[u];
  }
  for (int i = i0; i < j; ++i) {
    const double x1 = s.col[i + 1], c = s.gcs[i], sn = s.gsn[i];
    const double cx1 = c * x1, sx1 = sn * x1;
    s.col[i] = fma(c, xi, sx1);
    xi = fma(-sn, xi, cx1);
  }
  const double hh = xi * xi + bnext * bnext;
  const double iden = hh > 0 ? rsqrt(hh) : 0.0;
  const double cc = hh > 0 ? xi * iden : 1.0, ss = bnext * iden;
  s.gcs[j] = cc;
  s.gsn[j] = ss;
  s.col[j] = hh * iden;
  s.gg[j + 1] = -ss * s.gg[j];
  s.gg[j] = cc * s.gg[j];
  s.misc[2] = fabs(s.gg[j + 1]);
  if (rank == 0) {
    a.gs->g[j] = s.gg[j];
    a.gs->g[j + 1] = s.gg[j + 1];
  }
}

// column j of the triangular factor (rotated Hessenberg column), for the
// end-of-cycle solve: all threads of CTA 0, after givens_column
template <typename S>
__device__ __forceinline__ void store_rcol(const GmresArgs<S>& a, const Smem<S>& s, int j, int rank) {
  if (rank != 0) return;
  double* Rc = a.gs->R + (size_t)j * (kMaxRestart + 1);
  for (int l = threadIdx.x; l <= j; l += blockDim.x) Rc[l] = s.col[l];
}

// One GMRES solve by the CTAs of a team (the whole grid for k_gmres).
// epoch: the team barrier's epoch, carried across consecutive bodies.
// Returns false when a barrier or copy wait timed out (err set).
template <typename S>
__device__ bool gmres_body(const GmresArgs<S>& a, unsigned char* smraw, unsigned& epoch) {
  const Smem<S> s = carve(a, smraw);
  const DevGeo& g = a.g;
  const int M = g.M, n = g.n, m = a.m;
  const int ES = a.ES, G = a.G, rank = team_rank(a);
  const int m3 = m + 3;
  int trace_n = 0;

  // ---- matrix stream (owned matrices too large for shared memory)
  MatStream<S> msd;
  msd.nb = 0;
  msd.nw = 0;
  for (int k = 0; k < a.nown_b; ++k) msd.nb += (rank + k * G < a.nblack) ? 1 : 0;
  for (int k = 0; k < a.nown_w; ++k) msd.nw += (rank + k * G < a.nwhite) ? 1 : 0;
  msd.nitems = 2 * msd.nb + msd.nw;
  msd.issued = msd.consumed = 0;
  MatStream<S>* ms = a.stream_mats ? &msd : nullptr;
  if (ms) {
    // shared memory written by an earlier body (batched solves) before the
    // copy engine writes it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int b = 0; b < a.nbuf; ++b) mbar_init(s.mbar + b);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    for (int b = 0; b < a.nbuf; ++b) ms_issue(a, s, msd);
  }
#define GM_FAIL()           \
  do {                      \
    ms_drain(a, s, msd);    \
    return false;           \
  } while (0)

  // ---- resident copies of the owned matrices
  if (a.mats_smem) {
    for (int k = 0; k < a.nown_b; ++k) {
      int ib = rank + k * G;
      if (ib >= a.nblack) break;
      int e = a.black[ib];
      S* dst = s.mats + (size_t)k * (2 * M * M + 4 * n * n);
      for (int i = threadIdx.x; i < M * M; i += blockDim.x) {
        dst[i] = a.Gc[(size_t)ib * M * M + i];
        dst[M * M + i] = a.Tc[(size_t)e * M * M + i];
      }
      for (int i = threadIdx.x; i < 4 * n * n; i += blockDim.x) dst[2 * M * M + i] = a.Xc[(size_t)ib * 4 * n * n + i];
    }
    for (int k = 0; k < a.nown_w; ++k) {
      int iw = rank + k * G;
      if (iw >= a.nwhite) break;
      int e = a.white[iw];
      S* dst = s.mats + (size_t)a.nown_b * (2 * M * M + 4 * n * n) + (size_t)k * M * M;
      for (int i = threadIdx.x; i < M * M; i += blockDim.x) dst[i] = a.Tc[(size_t)e * M * M + i];
    }
  }

  int total = 0, cycle = 0, jlast = 0;
  bool converged = false, breakdown = false, nan = false;
  double tolabs = 0, beta0 = 0, resid = 0;
  __syncthreads();
  while (true) {
    double* accN = a.acc + (size_t)(2 * m) * m3;
    // ---- cycle start: V[0] = rhs - op(x)
    if (cycle > 0) {
      if (!apply_op(a, s, a.x, 1.0, false, trace_n, epoch, ms)) GM_FAIL();
    }
    {
      S* v0 = basis(a, s, 0);
      double nn = 0;
      for (int i = threadIdx.x; i < ES; i += blockDim.x) {
        long long sl = entry_slot(a, i);
        S rv = 0;
        if (sl >= 0) {
          double r = (double)ldcg(a.rhs + sl);
          if (cycle > 0) r -= deflate_slot_cg(g, a.y, a.precond == 2 ? a.chat : nullptr, a.Rs, sl);
          rv = (S)r;
          a.vglob[sl] = rv;
        }
        v0[i] = rv;
        nn += (double)rv * (double)rv;
      }
      nn = warp_sum(nn);
      if ((threadIdx.x & 31) == 0 && nn != 0.0) atomicAdd(accN, nn);
    }
    const bool fused = a.fused && a.precond == 2;
    if (fused)  // both c_hat buffers of the fused coarse solve start at zero
      for (long long i = (long long)rank * blockDim.x + threadIdx.x; i < 2 * g.d; i += (long long)G * blockDim.x)
        a.chatd[i] = 0.0;
    if (!grid_sync(a.bar, a.err, epoch, a.G)) GM_FAIL();
    const double beta = sqrt(__ldcg(accN));
    if (cycle == 0) {
      beta0 = beta;
      tolabs = a.tol * beta;
    }
    resid = beta;
    if (!isfinite(beta)) { nan = true; break; }
    if (beta <= tolabs || beta == 0.0) { converged = true; break; }
    if (threadIdx.x == 0) {
      s.gg[0] = beta;
      s.invb[0] = 1.0 / beta;
    }
    __syncthreads();
    int j = 0, pending = -1;  // pending: the step whose Givens rotation is deferred
    for (; j < m && total < a.maxit; ++j) {
      double* accD = a.acc + (size_t)(2 * j) * m3;
      double* accE = a.acc + (size_t)(2 * j + 1) * m3;
      const double ivj = s.invb[j];
      GM_TRACE(1);
      // ---- A: finalize V[j] on the owned entries (j > 0), then block solves
      S* vj = basis(a, s, j);
      if (j > 0) {
        for (int i = threadIdx.x; i < ES; i += blockDim.x) {
          S rv = (S)basis_combo(a, s, (double)s.w2[i], s.hs2, j, i);
          vj[i] = rv;
          long long sl = entry_slot(a, i);
          if (sl >= 0) a.vglob[sl] = rv;
        }
        __syncthreads();
      }
      // fused coarse solve: this step accumulates c_hat into buffer j & 1; the
      // other buffer was last read in the previous step's phase D (before its
      // barrier) and is cleared here for the next step
      double* chat_j = fused ? a.chatd + (size_t)(j & 1) * g.d : nullptr;
      if (fused) {
        double* nxt = a.chatd + (size_t)((j + 1) & 1) * g.d;
        for (long long i = (long long)rank * blockDim.x + threadIdx.x; i < g.d; i += (long long)G * blockDim.x)
          nxt[i] = 0.0;
      }
      if (a.precond == 0) {
        if (!grid_sync(a.bar, a.err, epoch, a.G)) GM_FAIL();  // neighbours read v_j
        if (!apply_op(a, s, a.vglob, ivj, false, trace_n, epoch, ms)) GM_FAIL();
      } else {
        if (!black_phase(a, s, ms, (const S*)nullptr, ivj, vj)) GM_FAIL();
        if (!apply_op(a, s, a.vglob, ivj, true, trace_n, epoch, ms, chat_j)) GM_FAIL();
      }
      GM_TRACE(4);
      // ---- D: w = y - S Z chat on owned entries; V^T w, ||w||^2
      const double* chat_d = a.precond == 2 ? (fused ? chat_j : a.chat) : nullptr;
      for (int i = threadIdx.x; i < ES; i += blockDim.x) {
        long long sl = entry_slot(a, i);
        s.w[i] = sl >= 0 ? (S)deflate_slot_cg(g, a.y, chat_d, a.Rs, sl) : S(0);
      }
      __syncthreads();
      owned_dots(a, s, s.w, j + 2, accD);
      GM_TRACE(5);
      if (!grid_sync_with(a.bar, a.err, epoch, a.G, [&] {
            if (pending >= 0) givens_column(a, s, pending, rank);
          }))
        GM_FAIL();
      GM_TRACE(6);
      if (pending >= 0) {  // the previous step's rotation and convergence test
        store_rcol(a, s, pending, rank);
        resid = s.misc[2];
        pending = -1;
        if (!isfinite(resid)) { nan = true; break; }
        if (resid <= tolabs) { converged = true; break; }  // j columns: this step is dropped
      }
      for (int l = threadIdx.x; l < j + 2; l += blockDim.x) {
        double v = __ldcg(accD + l);
        if (l <= j) {
          v *= s.invb[l];
          s.h1[l] = v;
          s.hs1[l] = v * s.invb[l];
        } else {
          s.misc[0] = v;  // ||w||^2
        }
      }
      __syncthreads();
      // ---- E: w2 = w - V h1; V^T w2, ||w2||^2
      for (int i = threadIdx.x; i < ES; i += blockDim.x) s.w2[i] = (S)basis_combo(a, s, (double)s.w[i], s.hs1, j + 1, i);
      __syncthreads();
      owned_dots(a, s, s.w2, j + 2, accE);
      GM_TRACE(8);
      if (!grid_sync(a.bar, a.err, epoch, a.G)) GM_FAIL();
      GM_TRACE(9);
      for (int l = threadIdx.x; l < j + 2; l += blockDim.x) {
        double v = __ldcg(accE + l);
        if (l <= j) {
          v *= s.invb[l];
          s.h2[l] = v;
          s.hs2[l] = v * s.invb[l];
        } else {
          s.misc[1] = v;  // ||w2||^2
        }
      }
      __syncthreads();
      GM_TRACE(10);
      if (threadIdx.x < 32) {  // ||h2||^2 and h1 + h2 in warp 0
        double q = 0;
        for (int l = threadIdx.x; l <= j; l += 32) {
          q += s.h2[l] * s.h2[l];
          s.col[l] = s.h1[l] + s.h2[l];
        }
        q = warp_sum(q);
        if (threadIdx.x == 0) s.misc[5] = q;
      }
      __syncthreads();
      GM_TRACE(11);
      // ---- F: ||w2|| (Pythagorean) and the breakdown test now; the Givens
      // rotation of column j -- a serial FP64 chain in thread 0, replicated in
      // every CTA -- runs inside the next step's first grid barrier, while the
      // other CTAs arrive, and its convergence test is read after it.  A step
      // that converged thus costs one extra step of work, whose results
      // (v_{j+1}, t, the dot products) are never used.
      if (threadIdx.x == 0) {
        const double bsq = s.misc[1] - s.misc[5];
        const double ib = bsq > 0 ? rsqrt(bsq) : 0.0;
        s.invb[j + 1] = ib;
        s.misc[3] = (bsq <= 1e-28 * s.misc[0]) ? 1.0 : 0.0;
        s.misc[4] = bsq > 0 ? bsq * ib : 0.0;  // the new subdiagonal entry
      }
      __syncthreads();
      GM_TRACE(13);
      ++total;
      if (!isfinite(s.misc[4]) || s.misc[3] != 0.0 || j + 1 >= m || total >= a.maxit) {
        // last step of the cycle: rotate now
        if (threadIdx.x == 0) givens_column(a, s, j, rank);
        __syncthreads();
        store_rcol(a, s, j, rank);
        resid = s.misc[2];
        if (!isfinite(resid) || !isfinite(s.misc[4])) { nan = true; ++j; break; }
        if (resid <= tolabs) { converged = true; ++j; break; }
        if (s.misc[3] != 0.0) { breakdown = true; ++j; break; }
        continue;
      }
      pending = j;
    }
    jlast = j;
    if (nan) break;
    __syncthreads();  // the columns of R written by all threads of CTA 0
    // ---- end of cycle: y = R^-1 g (warp 0 of CTA 0, column by column: y_k,
    // then the entries above it lose R_ik y_k in parallel over the lanes),
    // x += V diag(invb) y on owned entries
    if (rank == 0 && threadIdx.x < 32) {
      const int m1 = kMaxRestart + 1, lane = threadIdx.x;
      for (int l = lane; l < j; l += 32) s.col[l] = a.gs->g[l];
      __syncwarp();
      for (int k = j - 1; k >= 0; --k) {
        const double* Rk = a.gs->R + (size_t)k * m1;
        const double yk = s.col[k] / Rk[k];
        __syncwarp();
        for (int i = lane; i < k; i += 32) s.col[i] = fma(-Rk[i], yk, s.col[i]);
        if (lane == 0) a.gs->y[k] = yk;
        __syncwarp();
      }
    }
    // the accumulators are consumed: zero them for the next cycle
    for (size_t i = (size_t)rank * blockDim.x + threadIdx.x; i < (size_t)(2 * m + 1) * m3;
         i += (size_t)G * blockDim.x)
      a.acc[i] = 0.0;
    if (!grid_sync(a.bar, a.err, epoch, a.G)) GM_FAIL();
    for (int l = threadIdx.x; l < j; l += blockDim.x) s.hs1[l] = -__ldcg(a.gs->y + l) * s.invb[l];
    __syncthreads();
    for (int i = threadIdx.x; i < ES; i += blockDim.x) {
      long long sl = entry_slot(a, i);
      if (sl < 0) continue;
      a.x[sl] = (S)basis_combo(a, s, (double)ldcg(a.x + sl), s.hs1, j, i);
    }
    if (!grid_sync(a.bar, a.err, epoch, a.G)) GM_FAIL();
    ++cycle;
    if (converged || breakdown || total >= a.maxit) break;
  }
  if (rank == 0 && threadIdx.x == 0) {
    a.gs->beta0 = beta0;
    a.gs->tolabs = tolabs;
    a.gs->resid = resid;
    a.gs->j = total;
    a.gs->converged = converged ? 1 : 0;
    a.gs->breakdown = breakdown ? 1 : 0;
    a.gs->nan = nan ? 1 : 0;
    a.gs->scal[7] = cycle;
    a.gs->scal[6] = jlast;
    a.gs->scal[5] += total;  // iterations over all launches of a solve
    if (a.its_out) *a.its_out = total;
  }
  ms_drain(a, s, msd);
  return true;
#undef GM_FAIL
}

template <typename S>
__global__ void __launch_bounds__(256, 1) k_gmres(GmresArgs<S> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  if (a.skip && *((volatile const int*)a.skip)) return;
  unsigned epoch = 0;
  gmres_body(a, smraw, epoch);
}
