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

constexpr int kBatchHdr = (int)((sizeof(BatchTask) + 127) / 128 * 128);

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
      rep[t] = r;
    }
  }
}
