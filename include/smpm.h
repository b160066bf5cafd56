/*
 * smpm.h -- C ABI of the GB300 solver for the deflated Schur-complement
 * method of Joshi & Diamessis, "A deflated Schur complement method for the
 * iterative solution of a high-order discontinuous element discretization of
 * the Poisson equation" (arXiv 1601.03432).
 *
 * The library solves the 2-D Poisson-Neumann problem (Eq. poisson)
 *     lap u = f on [0,Lx]x[0,Ly],   n.grad u = g on the boundary,
 * discretised by the spectral multidomain penalty method (Sec. 1.2,
 * Eq. smpm_poisson) on an my x mx grid of elements with n x n GLL points each,
 * by Algorithm 3 (Sec. 2): GMRES on the deflated, block-Jacobi preconditioned
 * Schur complement system, with the null-space projections of Sec. 1.4.
 *
 * Layouts (all arrays are plain float64, no padding between elements):
 *   node vectors (length r = n*n*mx*my): element e = iy*mx + ix, then node
 *     (a, b) at e*n*n + b*n + a (a = x index, fastest).
 *   slot vectors (length kp = 4*n*mx*my): one slot per (element, face, face
 *     node) at e*4n + F*n + t, faces F = W,E,S,N = 0,1,2,3, t increasing along
 *     the face.  Slots on physical-boundary faces are padding for interface
 *     vectors (Sec. 1.3: interfaces carry 2n nodes, n on either side) and
 *     carry the Neumann data g for the solve.
 *
 * Ownership: the handle owns every device factor it allocates; the caller
 * owns every buffer it passes.  Device pointers must be valid on the current
 * CUDA device for the given stream.  Calls on one handle are not thread-safe.
 * Every entry point returns an smpm_status; on error the output buffers are
 * unspecified unless stated.  smpm_last_error() gives a message (per host
 * thread).  No C++ exception leaves the library: a failed host allocation in
 * any entry point is reported as SMPM_ENOMEM.  The library never checks the
 * length of a caller's buffer (lengths come from the handle); a short buffer
 * is undefined behaviour, so the Python binding checks lengths before the
 * call.
 */
#ifndef SMPM_H
#define SMPM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct smpm_handle_s* smpm_handle;
typedef struct smpm_batch_s* smpm_batch;   /* opaque; a set of factored handles solved together */

typedef enum {
  SMPM_OK = 0,
  SMPM_EINVAL = 1,        /* bad argument (sizes, null pointers, options)        */
  SMPM_ENOINTERFACE = 2,  /* mx*my < 2: no interface, A is singular (Sec. 1.3)  */
  SMPM_ENOMEM = 3,        /* device or host allocation failed                   */
  SMPM_ECUDA = 4,         /* a CUDA call failed                                 */
  SMPM_ENOTCONV = 5,      /* GMRES did not reach tol within maxit (u = best)    */
  SMPM_EBREAKDOWN = 6,    /* Arnoldi breakdown before tol                       */
  SMPM_ENAN = 7,          /* NaN/Inf met in the input or the iteration          */
  SMPM_ESTATE = 8,        /* call order violated (e.g. solve before factor)     */
  SMPM_ETIMEOUT = 9       /* a bounded device-side wait gave up (no hang)       */
} smpm_status;

/* Solver options.  precond: 0 = none (Algorithm 1), 1 = block-Jacobi
 * (Algorithm 2), 2 = block-Jacobi + deflation (Algorithm 3, default).
 * precision: 0 = FP64 throughout; 1 = FP32 inner GMRES inside FP64 iterative
 * refinement.  tau_scale scales the penalty tau_F = -tau_scale n(n-1)/h_perp
 * and robin_scale the Robin identity weight p_F = robin_scale n(n-1)/h_perp
 * of Eq. smpm_poisson (defaults 1 and 0.25). */
typedef struct {
  double tol;          /* relative residual target of GMRES (default 1e-10)  */
  int restart;         /* GMRES restart length m (default 50, max 200)        */
  int maxit;           /* maximum Arnoldi steps in total (default 1000)       */
  int precision;       /* 0 FP64, 1 FP32-inner + FP64 refinement              */
  int precond;         /* 0, 1, 2 as above                                    */
  double tau_scale;    /* default 1.0                                         */
  double robin_scale;  /* default 0.25                                        */
  int flags;           /* SMPM_FLAG_* bits (default 0)                        */
} smpm_opts;

/* flags: keep the GMRES operator matrices and Krylov basis in global memory
 * even when they fit in shared memory; stream the operator matrices through
 * shared memory with bulk copies even when they would fit resident (the
 * large-grid layouts, selectable for testing). */
#define SMPM_FLAG_NO_SMEM_RESIDENCY 1
#define SMPM_FLAG_STREAM_MATRICES 2
#define SMPM_FLAG_ADJOINT 4        /* also build the transposed system for schur_solve_adjoint */
#define SMPM_FLAG_WARP_ELEMS 8     /* one warp per block / element in the GMRES phases even when few
                                      are owned per CTA (the default from 4 per CTA; for testing) */
#define SMPM_FLAG_ROBIN_LITERAL 16 /* Robin flux R = I + n.grad with identity weight p_F = 1 on every face
                                      (the literal form of Sec. 1.2); robin_scale is then unused */
#define SMPM_FLAG_NO_LOCKSTEP 32    /* solve several right-hand sides one after another instead of in
                                      lockstep (for testing) */
#define SMPM_FLAG_OPERATOR_ONLY 64  /* schur_factor builds only the element factors T_e of S (no block-
                                      Jacobi, coarse or null-space factors): smpm_apply_schur and
                                      smpm_apply_schur32 work, every other call returns ESTATE.  For
                                      applying S on grids whose dense coarse step would not fit */

/* Per-solve report, written by schur_solve when the pointer is non-null. */
typedef struct {
  int iterations;        /* Arnoldi steps (all restarts, all refinement sweeps) */
  int restarts;          /* GMRES restarts                                       */
  int refinements;       /* outer refinement sweeps (precision 1), else 0        */
  int converged;         /* 1 if the GMRES estimate reached tol                  */
  double gmres_relres;   /* final GMRES residual estimate / ||P b_S||            */
  double schur_relres;   /* ||b_S - S x_S|| / ||b_S|| recomputed in FP64          */
  int launches;          /* CUDA kernels launched by this solve                  */
  double gmres_ms;       /* device time of the GMRES kernel (CUDA events)        */
  double pre_ms;         /* device time of the right-hand-side kernel            */
  double post_ms;        /* device time of the assembly/recovery kernel          */
} smpm_report;

/* Fill o with the defaults listed above. */
void smpm_default_opts(smpm_opts* o);

/* Geometry of Sec. 1.2: an my x mx Cartesian grid of elements on
 * [0,Lx]x[0,Ly] with n GLL points per direction (2 <= n <= 32,
 * 1 <= mx, my <= 4096).  No device work.  Errors: EINVAL, ENOMEM. */
smpm_status smpm_setup(int mx, int my, int n, double Lx, double Ly, smpm_handle* h);

/* Graded grid (Sec. 1.2 admits any smooth invertible element map; this is
 * the axis-aligned case with sizes of their own): element (ix, iy) covers
 * [xs[ix], xs[ix+1]] x [ys[iy], ys[iy+1]].  xs: host, mx+1 finite, strictly
 * increasing column edges; ys: host, my+1 row edges; both copied.  The
 * penalty tau_F and the Robin weight p_F of every face use the size of the
 * element that owns the face; the neighbour's gradient uses the neighbour's
 * size.  B 1, the right null vector of S, then differs between the two sides
 * of an interface, and the deflation vectors z_j of Sec. 2 are its
 * restrictions to interface j divided by the mean of the two sides (the
 * 0/1 indicators of the paper on a uniform grid; indicators alone leave B 1
 * outside the coarse space and GMRES stagnates on strongly graded grids).
 * Other limits and errors as smpm_setup. */
smpm_status smpm_setup_graded(int mx, int my, int n, const double* xs, const double* ys, smpm_handle* h);

/* Sizes: r = n^2 mx my nodes, kp = 4 n mx my slots, d interfaces, k = 2 n d
 * real interface slots, nblack checkerboard blocks.  Any pointer may be null. */
smpm_status smpm_sizes(smpm_handle h, long long* r, long long* kp, long long* d,
                       long long* k, long long* nblack);

/* Host arrays x, y (length r each) of the node coordinates (element map of
 * Sec. 1.2), for building f and g. */
smpm_status smpm_node_coords(smpm_handle h, double* x, double* y);

/* Host array (length r) of the GLL quadrature weight of every node. */
smpm_status smpm_node_mass(smpm_handle h, double* w);

/* Factor step (Sec. 1.3 - 2): element operators A_e and their tensor-product
 * inverses, the per-element interface factors T_e = B_e A_e^-1 E_e, the
 * block-Jacobi blocks M_b = S[block, block] (Fig. 2) in the reduced form
 * G_b = (I - X_b Y_b)^-1, the coarse matrix C = Z^T S Z and its regularised
 * inverse, and the null vectors u_L, u_S, u_C (Sec. 1.4).  Computed on the
 * host in FP64 and uploaded; o may be null for the defaults.  stream is a
 * cudaStream_t (null = legacy default stream).  Errors: EINVAL (also for
 * precond > 0 on a grid with a single interface, whose only block-Jacobi
 * block is the whole singular S), ENOINTERFACE, ENOMEM (also, before any
 * work, when the dense coarse step's 3 (d+1)^2 host doubles (5 with
 * SMPM_FLAG_ADJOINT) exceed the
 * machine's physical memory, and for any failed host allocation), ECUDA.
 * No C++ exception leaves any entry point of this library. */
smpm_status schur_factor(smpm_handle h, const smpm_opts* o, void* stream);

/* schur_factor with the same options for count distinct handles: the host
 * factor steps run in parallel (one handle per host thread, largest grids
 * first), then each handle's device part runs in turn on stream.  Stops at
 * the first failing handle (its status and message are returned; handles
 * after it are left unfactored). */
smpm_status smpm_factor_many(const smpm_handle* hs, int count, const smpm_opts* o, void* stream);

/* Algorithm 3 (or 1/2 per opts.precond) for nrhs right-hand sides.
 *   f : device, r * nrhs, right-hand side of Eq. poisson at the nodes
 *   g : device, kp * nrhs or null (= 0), Neumann data on boundary-face slots
 *       (interface slots are ignored)
 *   u : device, r * nrhs, output, normalised to zero GLL-weighted mean
 *   tol <= 0 takes opts.tol.  rep (host, nrhs entries) may be null.
 * The right-hand side b = f + tau g is projected out of u_L (Eq.
 * regularize_poisson) and b_S out of u_S (Eq. regularize_schur).
 * With nrhs > 1, FP64 and block-Jacobi (precond 1 or 2), the right-hand
 * sides are solved in lockstep, up to 16 at a time: their Arnoldi processes
 * advance together in one launch, so each step reads the operator matrices
 * once for all of them (each element product is a small dense GEMM); every
 * column keeps its own basis, Givens rotations, convergence and restarts,
 * and its report is its own.  SMPM_FLAG_NO_LOCKSTEP solves them one after
 * another instead.
 * Errors: EINVAL, ESTATE (no factor), ENOTCONV (u holds the last iterate),
 * EBREAKDOWN (Arnoldi breakdown before tol; u assembled as for ENOTCONV),
 * ENAN, ETIMEOUT, ECUDA. */
smpm_status schur_solve(smpm_handle h, const double* f, const double* g, double tol,
                        int nrhs, double* u, smpm_report* rep, void* stream);

/* Reverse-mode derivative of schur_solve: for a loss l(u) with
 * gbar_u = dl/du, returns gbar_f = dl/df and gbar_g = dl/dg.  The solve is
 * linear in (f, g): b = f + tau g (Eq. smpm_poisson), b~ = b - u_L u_L^T b
 * (Eq. regularize_poisson), L z = b~, u = z - (w^T z / 1^T w) 1, so
 *   dl/db = Pi lam,  L^T lam = N^T gbar_u,  N^T y = y - w (1^T y) / 1^T w,
 * with Pi = I - u_L u_L^T.  L^T lam = N^T gbar_u is solved by Algorithm 3 on
 * the transposed Schur system S^T = I + E^T A^-T B^T (Sec. 1.3 transposed):
 * transposed block-Jacobi blocks, the same interface indicators Z, coarse
 * matrix C^T (left null vector c0, right null vector u_C), left null vector
 * B 1 of S^T; then lam = A^-T (y - B^T mu) for the interface solution mu.
 *   gbar_u : device, r * nrhs
 *   gbar_f : device, r * nrhs, output (dl/df = dl/db)
 *   gbar_g : device, kp * nrhs, output or null; tau_F dl/db at the face node
 *            on physical-boundary slots, 0 on interface slots
 * Always FP64 (also on a handle factored with precision 1).  Needs
 * schur_factor with SMPM_FLAG_ADJOINT in opts.flags (else ESTATE).  rep and
 * errors as schur_solve. */
smpm_status schur_solve_adjoint(smpm_handle h, const double* gbar_u, double tol, int nrhs,
                                double* gbar_f, double* gbar_g, smpm_report* rep, void* stream);

/* As schur_solve, with f, g and u in HOST memory: the library copies the
 * inputs to its device staging buffers, solves, and copies u back before
 * returning (the stream is synchronised). */
smpm_status schur_solve_host(smpm_handle h, const double* f, const double* g, double tol,
                             int nrhs, double* u, smpm_report* rep, void* stream);

/* ---- single operators on device slot/node vectors (one right-hand side);
 * these are the building blocks of the solve, exported for testing. -------- */

/* y = S v, S = I + B A^-1 E (Eq. schur_complement_system); v, y: kp. */
smpm_status smpm_apply_schur(smpm_handle h, const double* v, double* y, void* stream);
/* y = S v in FP32 with the FP32 copy of the T_e factors (the operator of the
 * inner GMRES of the mixed-precision path); v, y: kp floats.  Needs
 * schur_factor with precision = 1 (else ESTATE). */
smpm_status smpm_apply_schur32(smpm_handle h, const float* v, float* y, void* stream);
/* t = M^-1 v, block-Jacobi of Sec. 2 / Fig. 2; v, t: kp. */
smpm_status smpm_apply_precond(smpm_handle h, const double* v, double* t, void* stream);
/* y = S M^-1 v computed in the fused checkerboard form; v, y: kp. */
smpm_status smpm_apply_schur_precond(smpm_handle h, const double* v, double* y, void* stream);
/* y = P v, P = I - S Z C^-1 Z^T (Eq. projection1) with the regularised C^-1. */
smpm_status smpm_apply_deflation(smpm_handle h, const double* v, double* y, void* stream);
/* y = Q v, Q = I - Z C^-1 Z^T S (Eq. projection2). */
smpm_status smpm_apply_deflation_q(smpm_handle h, const double* v, double* y, void* stream);
/* y = S v as smpm_apply_schur / smpm_apply_schur32, by the element-class-
 * shared path: on the axis-aligned uniform grids of this library T_e depends
 * only on which faces of the element are interfaces (at most 9 classes), so
 * the apply is one dense product T_c X_c per class (X_c: the own slots of the
 * class's elements side by side) and only the vectors stream from HBM.  The
 * paper's method keeps per-element factors (mapped elements, Sec. 1.2); this
 * is a property of uniform grids.  Needs n <= 32.  Errors as
 * smpm_apply_schur. */
smpm_status smpm_apply_schur_class(smpm_handle h, const double* v, double* y, void* stream);
smpm_status smpm_apply_schur_class32(smpm_handle h, const float* v, float* y, void* stream);

/* Kernels of y = S v (smpm_apply_schur, smpm_apply_schur32 and the S apply
 * inside the deflation entry points): AUTO picks by thresholds (one warp per
 * element for 4n <= 96, 1, 2 or 4 elements per warp by the element count, else
 * the shared-memory stream); WARP: persistent CTAs, one warp per element,
 * T_e read column by column from global memory; WARP2 / WARP4: 2 or 4 warps
 * per element; STREAM: bulk copies of T_e into a shared-memory ring; CLASS:
 * the element-class-shared product (smpm_apply_schur_class). */
enum { SMPM_APPLY_AUTO = 0, SMPM_APPLY_WARP = 1, SMPM_APPLY_WARP2 = 2, SMPM_APPLY_WARP4 = 3,
       SMPM_APPLY_STREAM = 4, SMPM_APPLY_CLASS = 5 };

/* Fix the apply kernel of h.  Errors: ESTATE (not factored), EINVAL (kind
 * not available on this grid: WARP* need 4n <= 96, CLASS its tile in shared
 * memory). */
smpm_status smpm_set_apply_kernel(smpm_handle h, int kind);

/* Time every available apply kernel on h's grid in precision 0 (FP64) or 1
 * (FP32, needs precision-1 factors): reps timed launches each after one
 * warm-up (median of the CUDA-event times; reps < 1 means 5), with a 512 MiB
 * write between launches when flush != 0 so that T_e comes from HBM.  The
 * fastest becomes h's apply kernel.  ms_out (host, 5 entries, may be null):
 * the median per kind WARP..CLASS, -1 where not available; chosen (may be
 * null): the kind kept.  Scratch vectors are allocated and freed inside;
 * synchronises the stream.  Errors: ESTATE, EINVAL, ENOMEM, ECUDA. */
smpm_status smpm_autotune_apply(smpm_handle h, int precision, int reps, int flush, double* ms_out, int* chosen,
                                void* stream);

/* b_S = B A^-1 b (right-hand side of Eq. schur_complement_system); b: r, bS: kp. */
smpm_status smpm_schur_rhs(smpm_handle h, const double* b, double* bS, void* stream);
/* u = A^-1 (b - E x) (back-substitution of Sec. 1.3); b: r, x: kp, u: r. */
smpm_status smpm_recover(smpm_handle h, const double* b, const double* x, double* u, void* stream);
/* Null vectors (device outputs): u_L (r), u_S (kp), u_C (d). Any may be null. */
smpm_status smpm_null_vectors(smpm_handle h, double* uL, double* uS, double* uC, void* stream);
/* Host copy of C = Z^T S Z (d*d, row-major). */
smpm_status smpm_coarse_matrix(smpm_handle h, double* C);

/* Host part of schur_factor only (no device work, no GPU needed): builds the
 * FP64 factors in host memory so that they can be inspected with
 * smpm_host_factor.  A later schur_factor recomputes them. */
smpm_status smpm_factor_host_only(smpm_handle h, const smpm_opts* o);

/* Copy the host factor array `name` into out (host, count doubles; count must
 * equal the array length, returned through *len when out is null).  Names:
 * "x1d","w1d","D" (Sec. 1.2), "T" (nel*(4n)^2, T_e row-major), "G", "X"
 * (block-Jacobi, per black element), "black" (black element ids as doubles),
 * "C","H","c0","uC" (coarse, Sec. 2), "uS","B1" (kp), "uL","what" (r),
 * "null_iterations" (1 value). */
smpm_status smpm_host_factor(smpm_handle h, const char* name, double* out, long long count, long long* len);

/* y = P v exactly as smpm_apply_deflation, for callers that cannot allocate
 * device memory when they call: code inside a framework whose caching
 * allocator already owns the free device memory, latency-critical loops that
 * must not hit the implicit device synchronisation of cudaMalloc/cudaFree,
 * or callers with a fixed memory budget.  The paper has no counterpart; this
 * is a property of the library interface only.
 *   v, y : device, kp doubles (caller-owned; y must not alias v)
 * The call allocates nothing: its scratch (Z^T v, C^+ Z^T v and a barrier
 * word) is a file-scope device array of 2*32768 + 32 doubles (~512 KiB) that
 * every GPU loading this library holds until exit.  Grids with more than
 * 32768 interfaces are rejected with SMPM_EINVAL.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  The address is
 * kept for the life of the process: it is not valid after cudaDeviceReset
 * (or any other teardown of the device's primary context), so do not call
 * this entry point again after one.  Every call shares the one array: calls
 * that overlap on the GPU (different streams, threads or handles) race and
 * must be serialised by the caller.  Asynchronous on stream: the status only
 * covers the checks and the launch.  A failed internal grid barrier (not
 * expected: every CTA is co-resident) still returns SMPM_OK and leaves y =
 * NaN, so a caller that must detect it checks y.
 * Errors: EINVAL, ESTATE, ECUDA. */
smpm_status smpm_apply_deflation_noalloc(smpm_handle h, const double* v, double* y, void* stream);

/* Testing hook for the failure path of the device-side waits.  Every grid
 * or team barrier of the solve kernels polls at most `spins` times (default
 * 2^28, restored by spins <= 0) before it sets the kernel's error flag and
 * unwinds; the solve then returns SMPM_ETIMEOUT with no kernel left waiting,
 * and the context stays usable.  A small value makes real waits run out.
 * Applies to the current device; call it between solves (it synchronises
 * with the device like cudaMemcpyToSymbol).  Errors: ECUDA. */
smpm_status smpm_set_barrier_spin_limit(long long spins);

/* ---- batched solves: many right-hand sides of many independent grids ----
 * One persistent cooperative launch runs every right-hand side of every
 * problem of the batch (Algorithm 3 per right-hand side, each problem with
 * the precision, preconditioner and tol of its own schur_factor).  The
 * launch's CTAs form teams of team_size CTAs; whole problems are assigned to
 * teams (longest estimated work first, onto the least-loaded team) and a
 * team solves its problems' right-hand sides one after another with team
 * barriers in place of grid barriers.  The paper solves one system at a
 * time; batching is a property of this library.
 *
 * smpm_batch_create: hs[count] factored handles (distinct; their device
 * workspaces are used by the batch, so do not solve on them concurrently),
 * nrhs[count] >= 1 right-hand sides each.  team_size <= 0 picks the smallest
 * of 8, 16, 19, 38, 76 that fits (each problem's solve state must fit the
 * shared memory of one CTA at that team size), else all SMs as one team.
 * use_graph != 0 captures the batch's device work (argument copy, barrier
 * resets, the launch, the report copy) in a CUDA graph on the first solve
 * and replays it afterwards.  precision: -1 each handle's own, 0 FP64 for all,
 * 1 mixed precision for all (every handle factored with precision 1).
 * Errors: EINVAL, ESTATE, ENOMEM, ECUDA. */
smpm_status smpm_batch_create(const smpm_handle* hs, int count, const int* nrhs, int team_size, int use_graph,
                              int precision, smpm_batch* out);

/* Sizes of the packed arrays (problem-major, right-hand-side-major within a
 * problem: problem p's k-th right-hand side starts at the sum over q < p of
 * nrhs_q r_q, plus k r_p, for f and u, and likewise with kp for g), the
 * number of tasks (right-hand sides), the current team size and team count,
 * and the device time of the last batched solve (ms).  Any pointer may be
 * null. */
smpm_status smpm_batch_info(smpm_batch b, long long* f_len, long long* g_len, long long* ntasks, int* team_size,
                            int* nteams, double* last_ms);

/* Solve the whole batch.  f, u: device, f_len doubles (packed as above; u is
 * written, zero-mean per right-hand side); g: device, g_len doubles, or null
 * for g = 0.  rep: host, ntasks entries in the packed order, or null.
 * Ordered after prior work on stream; returns after the batch has finished.
 * Errors: EINVAL, ENOTCONV (some right-hand side did not converge; u holds
 * its last iterate), ENAN, ETIMEOUT, ECUDA. */
smpm_status smpm_batch_solve(smpm_batch b, const double* f, const double* g, double* u, smpm_report* rep,
                             void* stream);

/* Autotuner: lays the batch out for each of candidates[ncand] team sizes
 * that fits, times one solve of (f, g) after a warm-up solve (u is
 * overwritten), keeps the fastest.  ms_out (host, ncand, may be null)
 * receives each candidate's time (-1 when it does not fit); chosen (may be
 * null) the team size kept. */
smpm_status smpm_batch_autotune(smpm_batch b, const double* f, const double* g, double* u, void* stream,
                                const int* candidates, int ncand, double* ms_out, int* chosen);

/* Per right-hand side of the last batched solve (packed order): the team
 * that solved it and its start and end on the device's global timer, in ms
 * from the earliest start.  Host arrays of ntasks entries; any may be null. */
smpm_status smpm_batch_task_times(smpm_batch b, int* team, double* begin_ms, double* end_ms);

/* y_p = S_p v_p (Eq. schur_complement_system) for every problem p of the
 * batch in one launch (one vector per problem): v, y device, packed
 * problem-major with kp_p entries each (v_len = sum of kp_p).  By default one
 * warp per element reads the element's T_e column by column straight from
 * global memory with many loads in flight (see smpm_batch_set_apply_kernel).
 * The FP32 variant needs every handle factored with precision 1.
 * Asynchronous on stream.  Errors: EINVAL, ESTATE, ECUDA. */
smpm_status smpm_batch_apply_schur(smpm_batch b, const double* v, double* y, void* stream);
smpm_status smpm_batch_apply_schur32(smpm_batch b, const float* v, float* y, void* stream);

/* Kernel of the batched apply: 1 (default) warps per element reading T_e
 * from global memory (element matrices up to 96 x 96, i.e. n <= 24; larger
 * ones take kind 0), 0 bulk copies of T_e into a shared-memory ring per CTA
 * (measured slower; kept selectable).  Errors: EINVAL. */
smpm_status smpm_batch_set_apply_kernel(smpm_batch b, int kind);

/* Release the batch (not its handles; null is ignored). */
void smpm_batch_destroy(smpm_batch b);

/* Element-tile domain decomposition for running one grid on several devices
 * (Sec. 2's block structure is local to elements and their neighbours; the
 * method shards by tiles of elements).  Host only, no device work.  The
 * mx x my elements are split into px x py contiguous tiles; rank
 * ty * px + tx owns element columns [ix0, ix1) and rows [iy0, iy1), with
 * ix0 = tx mx / px (integer division), so tile sizes differ by at most one,
 * and the interface slots of its own elements.  Per step of Algorithm 3 a
 * rank exchanges with each peer across a cut: the Schur apply's pushed
 * products (push form: T_e v_e destined for the peer's slots), the
 * block-Jacobi block inputs and outputs of black elements on the cut, and
 * the partial interface sums of Z^T v (an all-reduce of d values, after
 * which the coarse solve is replicated); the Gram-Schmidt dot products are
 * all-reduced. */
typedef struct {
  int px, py, rank;
  int ix0, ix1, iy0, iy1;  /* owned element columns [ix0, ix1) and rows [iy0, iy1) */
  long long nel_owned;
  int npeers;              /* ranks sharing a cut with this tile (<= 4) */
  int peers[4];            /* peer across the tile's W, E, S, N side, -1 if none */
  long long halo[4];       /* slots on that cut (n per cut interface), 0 if none */
} smpm_tile;

/* Tile of rank in the px x py decomposition of h's grid.  Errors: EINVAL
 * (px > mx, py > my, rank out of range, null argument). */
smpm_status smpm_partition_tile(smpm_handle h, int px, int py, int rank, smpm_tile* t);

/* Halo of rank across side (0 W, 1 E, 2 S, 3 N): own[k] is rank's padded
 * slot (e, side, s) on the cut face of its boundary element e, facing[k] the
 * peer's slot (nbr(e, side), opposite side, s) across it; k runs along the cut
 * (element row or column ascending, then s), so rank's facing list towards a
 * peer equals the peer's own list towards rank.  own, facing: host arrays of
 * halo[side] entries (either may be null).  Errors: EINVAL (also for a side
 * without a peer). */
smpm_status smpm_partition_halo(smpm_handle h, int px, int py, int rank, int side, long long* own,
                                long long* facing);

/* Release every resource of h (null is ignored). */
void smpm_destroy(smpm_handle h);

/* Message of the last error on this thread ("" if none). */
const char* smpm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SMPM_H */
