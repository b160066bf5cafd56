// Batched solves: many right-hand sides of many independent problems (grids
// of different sizes) in ONE persistent cooperative launch.
//
// The CTAs of the launch are split into teams (contiguous CTA ranges, fixed
// for the launch).  Each team works through its own list of tasks, one task
// = one right-hand side of one problem, all right-hand sides of a problem on
// the same team, and runs for each task the bodies of the single-solve
// kernels in order: pre_body, then gmres_body<double> (FP64) or up to
// kMaxRefine pairs (gmres_body<float>, refine_body) (mixed precision), then
// post_body.  Team barriers replace the grid barriers; a team's barrier epoch
// runs on across its tasks.  The task's arguments are staged in shared
// memory (header of the dynamic buffer) and the bodies carve the rest.
#pragma once
// Included inside the anonymous namespace of smpm_solver.cu.

struct alignas(16) BatchTask {
  PrePostArgs P;          // FP64 pre/post arguments (all-global layout)
  GmresArgs<double> a64;  // FP64 GMRES (its own layout: resident or streamed matrices, basis)
  GmresArgs<float> a32;   // FP32 inner GMRES (mixed precision)
  RefineArgs R;           // refinement step (mixed precision)
  int precision;          // 0 FP64, 1 FP32 inner + FP64 refinement
  int has_g;
  long long f_off, g_off, u_off;  // offsets into the packed f, g, u of a call
  unsigned char* ctl;     // the problem's control block (zeroed per task from byte 256)
  int* its;               // inner iterations per refinement step (in ctl)
  double* rn;             // ||r||^2 per refinement step (in ctl)
  // lockstep group (ncols >= 2): ncols right-hand sides of the problem in one
  // lockstep GMRES; per-column arguments live in global memory and are staged
  // one at a time behind this header
  int ncols;
  long long rep0;                // report index of the group's first column
  long long r_len, kp_len;       // node and slot vector lengths of the problem
  LockArgs<double> L64;
  LockArgs<float> L32;
  const PrePostArgs* Pc;         // 2 R: pre (c), post (R + c)
  const RefineArgs* Rc;          // kMaxRefine R: refinement step ref of column c at ref R + c
  unsigned char* lctl;           // column blocks (kLockColBytes each): acc8 | done, nref | rn
};

struct BatchIO {
  const double* f;
  const double* g;
  double* u;
};

struct TaskReport {
  int iterations, restarts, refinements, converged;
  double gmres_num, gmres_den;  // relres = num / den
  double res2, bsn2;            // ||b_S - S x_S||^2, ||b_S||^2
  unsigned long long t_begin, t_end;  // global timer (ns) at the task's start and end on its team's first CTA
  int team, breakdown;  // breakdown: an FP64 solve ended on an Arnoldi breakdown before tol
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

constexpr size_t kLockColBytes = 256;  // column block of a lockstep solve's control area
constexpr int kBatchTaskBytes = (int)((sizeof(BatchTask) + 127) / 128 * 128);
// header: the task, then staging for one column's pre/post and refinement arguments
constexpr int kBatchHdr = (int)((kBatchTaskBytes + sizeof(PrePostArgs) + sizeof(RefineArgs) + 127) / 128 * 128);

// copy n bytes (a multiple of 16) from global memory into shared memory, all threads
__device__ __forceinline__ void stage16(void* dst, const void* src, int n) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(dst);
  for (int i = threadIdx.x; i < n / 16; i += blockDim.x) d[i] = s[i];
}

// A lockstep group task: pre bodies of the R columns, the lockstep GMRES
// (FP64, or up to kMaxRefine rounds of FP32 lockstep GMRES and per-column
// refinement), post bodies, reports.  Returns the failing body (0: none).
__device__ __noinline__ int batch_group(BatchTask& T, unsigned char* smraw, unsigned char* body, const BatchIO* io,
                           TaskReport* rep, int team, unsigned& epoch) {
  PrePostArgs& Pst = *reinterpret_cast<PrePostArgs*>(smraw + kBatchTaskBytes);
  RefineArgs& Rst = *reinterpret_cast<RefineArgs*>(smraw + kBatchTaskBytes + sizeof(PrePostArgs));
  const int R = T.ncols;
  const GmresArgs<double>& ga = T.P.ga;
  const int rank = team_rank(ga);
  const unsigned long long t_begin = global_ns();
  auto stage_p = [&](int i, int c) {
    __syncthreads();
    stage16(&Pst, T.Pc + i, (int)sizeof(PrePostArgs));
    __syncthreads();
    if (threadIdx.x == 0) {
      Pst.f = io->f + T.f_off + (size_t)c * T.r_len;
      Pst.u = io->u + T.u_off + (size_t)c * T.r_len;
      Pst.gn = (T.has_g && io->g) ? io->g + T.g_off + (size_t)c * T.kp_len : nullptr;
    }
    __syncthreads();
  };
  // column blocks, lockstep accumulators and column reports start at zero
  if (rank == 0) {
    for (int i = threadIdx.x; i < R * (int)(kLockColBytes / 4); i += blockDim.x) reinterpret_cast<int*>(T.lctl)[i] = 0;
    for (int i = threadIdx.x; i < R * (int)(sizeof(LockColState) / 4); i += blockDim.x)
      reinterpret_cast<int*>(T.precision == 0 ? T.L64.cs : T.L32.cs)[i] = 0;
  }
  {
    const GmresArgs<double>& a = T.P.ga;
    const size_t nacc = (size_t)(2 * a.m + 1) * R * (a.m + 3);
    double* acc = T.precision == 0 ? T.L64.a.acc : T.L32.a.acc;
    for (size_t i = (size_t)rank * blockDim.x + threadIdx.x; i < nacc; i += (size_t)a.G * blockDim.x) acc[i] = 0.0;
  }
  if (!grid_sync(ga.bar, ga.err, epoch, ga.G)) return 1;
  for (int c = 0; c < R; ++c) {
    stage_p(c, c);
    if (!pre_body(Pst, body, epoch)) return 2;
  }
  if (T.precision == 0) {
    if (!lock_body<double>(T.L64, body, epoch)) return 3;
  } else {
    for (int ref = 0; ref < kMaxRefine; ++ref) {
      // every column's done flag was written before the last barrier
      bool all = true;
      for (int c = 0; c < R; ++c)
        all = all && *((volatile const int*)(T.lctl + (size_t)c * kLockColBytes + 64)) != 0;
      if (all) break;
      if (!lock_body<float>(T.L32, body, epoch)) return 3;
      for (int c = 0; c < R; ++c) {
        if (*((volatile const int*)(T.lctl + (size_t)c * kLockColBytes + 64))) continue;
        __syncthreads();
        stage16(&Rst, T.Rc + (size_t)ref * R + c, (int)sizeof(RefineArgs));
        __syncthreads();
        if (refine_body(Rst, body, epoch) < 0) return 4;
      }
      if (!grid_sync(ga.bar, ga.err, epoch, ga.G)) return 4;
    }
  }
  for (int c = 0; c < R; ++c) {
    stage_p(R + c, c);
    if (!post_body(Pst, body, epoch)) return 5;
  }
  if (!grid_sync(ga.bar, ga.err, epoch, ga.G)) return 5;
  if (rank == 0 && threadIdx.x < R) {
    const int c = threadIdx.x;
    const unsigned char* blk = T.lctl + (size_t)c * kLockColBytes;
    const double* a8 = reinterpret_cast<const double*>(blk);
    const LockColState& cs = (T.precision == 0 ? T.L64.cs : T.L32.cs)[c];
    TaskReport r{};
    r.res2 = __ldcg(a8 + ACC_RES);
    r.bsn2 = __ldcg(a8 + ACC_BSN);
    r.iterations = cs.its_total;
    if (T.precision == 0) {
      r.restarts = cs.cycles > 1 ? cs.cycles - 1 : 0;
      r.converged = cs.converged;
      r.breakdown = cs.breakdown;
      r.gmres_num = cs.resid;
      r.gmres_den = cs.beta0;
    } else {
      const int nref = *reinterpret_cast<const int*>(blk + 68);
      const double* rn = reinterpret_cast<const double*>(blk + 128);
      r.refinements = nref;
      r.converged = (*reinterpret_cast<const int*>(blk + 64) != 0 || __ldcg(a8 + ACC_RGN) == 0.0) ? 1 : 0;
      r.gmres_num = nref > 0 ? sqrt(__ldcg(rn + min(nref, kMaxRefine) - 1)) : 0.0;
      r.gmres_den = sqrt(__ldcg(a8 + ACC_RGN));
    }
    r.t_begin = t_begin;
    r.t_end = global_ns();
    r.team = team;
    rep[T.rep0 + c] = r;
  }
  return 0;
}

__global__ void __launch_bounds__(256, 1) k_batch(const BatchTask* __restrict__ tasks, const int* __restrict__ begin,
                                                  const int* __restrict__ team_of, const BatchIO* io,
                                                  TaskReport* rep, int ctl_bytes) {
  extern __shared__ __align__(16) unsigned char smraw[];
  BatchTask& T = *reinterpret_cast<BatchTask*>(smraw);
  unsigned char* body = smraw + kBatchHdr;
  const int team = team_of[blockIdx.x];
  if (team < 0) return;  // CTA outside every team
  unsigned epoch = 0;
  for (int t = begin[team]; t < begin[team + 1]; ++t) {
    __syncthreads();  // every thread is done with the previous task's arguments
    {
      const int4* src = reinterpret_cast<const int4*>(tasks + t);
      int4* dst = reinterpret_cast<int4*>(smraw);
      for (int i = threadIdx.x; i < (int)(sizeof(BatchTask) / 16); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    if (T.ncols >= 2) {  // lockstep group
      const int where = batch_group(T, smraw, body, io, rep, team, epoch);
      if (where) {
        if (threadIdx.x == 0 && atomicCAS(T.P.ga.err + 1, 0, t + 1) == 0) T.P.ga.err[2] = where;
        return;
      }
      continue;
    }
    if (threadIdx.x == 0) {
      T.P.f = io->f + T.f_off;
      T.P.u = io->u + T.u_off;
      T.P.gn = (T.has_g && io->g) ? io->g + T.g_off : nullptr;
      T.P.assembled = 0;
    }
    __syncthreads();
    const int rank = team_rank(T.P.ga);
    const unsigned long long t_begin = global_ns();
    // per-solve control block of the problem (accumulators, flags, counts)
    if (rank == 0)
      for (int i = 256 / 4 + threadIdx.x; i < ctl_bytes / 4; i += blockDim.x) reinterpret_cast<int*>(T.ctl)[i] = 0;
    // on a failed wait the first failing task and body are recorded beside
    // the error code (err[1] = task + 1, err[2] = body: 1 start, 2 pre,
    // 3 GMRES, 4 refinement, 5 post)
    auto failed = [&](int where) {
      if (threadIdx.x == 0 && atomicCAS(T.P.ga.err + 1, 0, t + 1) == 0) T.P.ga.err[2] = where;
    };
    if (!grid_sync(T.P.ga.bar, T.P.ga.err, epoch, T.P.ga.G)) return failed(1);
    if (!pre_body(T.P, body, epoch)) return failed(2);
    if (T.precision == 0) {
      if (!gmres_body<double>(T.a64, body, epoch)) return failed(3);
    } else {
      for (int ref = 0; ref < kMaxRefine; ++ref) {
        __syncthreads();
        if (threadIdx.x == 0) {
          T.a32.its_out = T.its + ref;
          T.R.ga.its_out = T.its + ref;
          T.R.rn = T.rn + ref;
        }
        __syncthreads();
        if (!gmres_body<float>(T.a32, body, epoch)) return failed(3);
        const int st = refine_body(T.R, body, epoch);
        if (st < 0) return failed(4);
        if (st == 1) break;
      }
      __syncthreads();
      if (threadIdx.x == 0) T.P.assembled = 1;
      __syncthreads();
    }
    if (!post_body(T.P, body, epoch)) return failed(5);
    // every CTA of the team is past the task's last reads of the problem's
    // control block (the zero-mean step reads its accumulator after the last
    // barrier of post_body) before rank 0 reads the report and the next task
    // clears the block
    if (!grid_sync(T.P.ga.bar, T.P.ga.err, epoch, T.P.ga.G)) return failed(5);
    if (rank == 0 && threadIdx.x == 0) {
      const GState* gs = T.P.ga.gs;
      const double* acc8 = T.P.acc;
      TaskReport r{};
      r.res2 = __ldcg(acc8 + ACC_RES);
      r.bsn2 = __ldcg(acc8 + ACC_BSN);
      if (T.precision == 0) {
        r.iterations = gs->j;
        r.restarts = gs->scal[7] > 1 ? (int)gs->scal[7] - 1 : 0;
        r.converged = (gs->converged || gs->beta0 == 0.0) ? 1 : 0;
        r.breakdown = gs->breakdown;
        r.gmres_num = gs->resid;
        r.gmres_den = gs->beta0;
      } else {
        const int nref = *T.R.nref;
        r.iterations = (int)gs->scal[5];
        r.refinements = nref;
        r.converged = *T.R.done;
        r.gmres_num = nref > 0 ? sqrt(__ldcg(T.rn + nref - 1)) : 0.0;
        r.gmres_den = sqrt(__ldcg(acc8 + ACC_RGN));
      }
      r.t_begin = t_begin;
      r.t_end = global_ns();
      r.team = team;
      rep[T.rep0] = r;
    }
  }
}
// stage16 copies these with 16-byte loads and stores
static_assert(sizeof(PrePostArgs) % 16 == 0 && alignof(PrePostArgs) >= 16, "PrePostArgs: 16-byte copies");
static_assert(sizeof(RefineArgs) % 16 == 0 && alignof(RefineArgs) >= 16, "RefineArgs: 16-byte copies");
static_assert(sizeof(BatchTask) % 16 == 0, "BatchTask: 16-byte copies");
