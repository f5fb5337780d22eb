/*
 * sem.h -- C ABI of libsem: matrix-free tensor-product GLL spectral-element
 * operators for periodic viscous Burgers, their tangent and transpose products,
 * and the explicit Runge-Kutta forward / discrete-adjoint sweeps built on them,
 * on one NVIDIA GB300 (sm_103a).
 *
 * Method: Marin, Constantinescu, Smith, "A scalable matrix-free spectral element
 * approach for unsteady PDE constrained optimization using PETSc/TAO",
 * arXiv:1806.01422.  Each entry point names the section / equation it implements.
 *
 * Conventions shared by every call
 * --------------------------------
 * Grid.  d in {1,2,3}; E elements per direction; order N (n = N+1 GLL points per
 *   direction); periodic box [0, L)^d, L = 2*pi for d = 1 and 1 otherwise unless
 *   sem_opts.L is set.  Unique nodes per direction G = E*N.
 * Vectors.  A "state" is d*G^d doubles (sem_ndof), structure of arrays by
 *   component: index ((c*G + g_{d-1})*G + ...)*G + g_0, so x_0 is the fastest
 *   index.  Component c is the velocity along x_c (d = 1: the scalar u).
 *   Node g along an axis sits at x = e*h + (xi_i + 1)*h/2 with e = g / N,
 *   i = g % N, h = L/E and xi the GLL points on [-1, 1] (sem_coords).
 * Pointers.  State pointers are DEVICE pointers owned by the caller, 8-byte
 *   aligned, not overlapping any output of the same call (else SEM_ERR_ALIAS).
 *   `stream` is a cudaStream_t (NULL = legacy default stream).  Every call is
 *   stream-ordered and returns after enqueueing, except where a host output
 *   (J_host) is documented as synchronising the stream.
 * Ownership.  The handle owns its workspaces, the forward trajectory and the
 *   checkpoint slots; they are allocated on first use on the device current at
 *   that time and freed by sem_destroy.
 * Errors.  Every int-returning call returns SEM_OK (0) or a negative code;
 *   sem_last_error() returns a thread-local message for the last failure.
 *   Argument errors are detected on the host before anything is enqueued.
 */
#ifndef SEM_H
#define SEM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sem_ctx* sem_t;

/* status codes */
#define SEM_OK             0
#define SEM_ERR_ARG       -1  /* bad dimension, size, order, pointer or option */
#define SEM_ERR_ALIAS     -2  /* an output overlaps an input */
#define SEM_ERR_OOM       -3  /* device allocation failed or checkpoint budget exceeded */
#define SEM_ERR_NONFINITE -4  /* a NaN/Inf appeared in the forward or adjoint sweep */
#define SEM_ERR_STATE     -5  /* sem_rk_adjoint without a completed sem_rk_forward */
#define SEM_ERR_CUDA      -6  /* a CUDA runtime call failed (message has the CUDA error) */

/* explicit Runge-Kutta schemes (Butcher tableaux) */
#define SEM_RK4      0  /* classic 4-stage, 4th order */
#define SEM_SSPRK3   1  /* Shu-Osher SSP 3-stage, 3rd order */
#define SEM_EULER    2  /* forward Euler (the case of Sec. 4.1) */
#define SEM_BS3      4  /* Bogacki-Shampine 3-stage, 3rd order; with sem_set_adaptive the
                           3(2) pair with adaptive step sizes */
/* implicit scheme */
#define SEM_CN       3  /* Crank-Nicolson (Sec. 6.3): u_{n+1} - u_n = dt/2 (F(u_n) + F(u_{n+1})),
                           Newton with matrix-free GMRES per step; FP64 single-instance
                           handles only; stores every state u_0 .. u_N whatever the
                           checkpoint mode; its adjoint solves with (I - dt/2 J^T)
                           (see sem_set_solver) */

/* arithmetic of the element kernels */
#define SEM_PREC_FP64       0  /* everything in FP64 */
#define SEM_PREC_FP32_BULK  1  /* FP32 contractions, pointwise products and sums of
                                  the <= 2^d element contributions per node; FP64
                                  RK stage accumulation, objective and adjoint
                                  accumulation */
#define SEM_PREC_FP64_DF    2  /* the FP64 form with its element kernels (contractions
                                  and pointwise products) in double-float arithmetic
                                  on the FP32 pipe: pairs of floats, about 48
                                  significand bits, compensated dot products; inputs,
                                  element results, assembly, states and every
                                  reduction in FP64.  Results agree with the FP64 form
                                  to about 1e-13 relative (the 1e-11 bound holds). */

/* trajectory storage for the adjoint sweep (Sec. 5.3, Sec. 5.4) */
#define SEM_CKPT_AUTO      0  /* STAGES if it fits ckpt_budget_bytes, else STATES, else BINOMIAL */
#define SEM_CKPT_STAGES    1  /* store every stage value of every step: adjoint = s J^T per step */
#define SEM_CKPT_STATES    2  /* store every step's state; recompute its stages in the adjoint */
#define SEM_CKPT_BINOMIAL  3  /* ckpt_slots state slots, revolve-optimal recomputation */
#define SEM_CKPT_TWO_LEVEL 4  /* every step's state: as many as ckpt_budget_bytes allow
                                 (less a 3-state staging ring) in device memory, the rest in
                                 pinned host memory (sem_set_host_tier); AUTO picks it after
                                 STATES when a host budget is set */

typedef struct {
    int    dim;                /* 1, 2 or 3 */
    int    E;                  /* elements per direction, >= 1 (>= 2 recommended) */
    int    N;                  /* polynomial order, 1..15 (n = N+1 <= 16 points) */
    double nu;                 /* viscosity, >= 0 */
    double L;                  /* box edge; <= 0 selects the default (2 pi for d = 1, else 1) */
    int    precision;          /* SEM_PREC_* */
    int    ckpt_mode;          /* SEM_CKPT_* */
    int    ckpt_slots;         /* BINOMIAL: number of state slots (>= 1) */
    size_t ckpt_budget_bytes;  /* device bytes the trajectory may use; 0 = no limit */
} sem_opts;

/* Create a handle for the periodic grid of Sec. 3.2 (affine elements, GLL basis).
 * Host-only: computes the GLL tables; no device memory is touched.
 * Returns SEM_ERR_ARG for dim not in {1,2,3}, E < 1, N not in [1,15], nu < 0,
 * non-finite nu, or a null `out`. */
int sem_create(int dim, int E, int N, double nu, sem_t* out);
int sem_create_ex(const sem_opts* opts, sem_t* out);

/* Free the handle and every device buffer it owns (after synchronising the device
 * work the handle enqueued).  NULL is ignored. */
void sem_destroy(sem_t h);

/* d * (E*N)^d: unique periodic scalar unknowns (Sec. 6.3 counts unknowns this way). */
size_t sem_ndof(sem_t h);

/* Host array x[G]: coordinates of the unique nodes along one axis (same on every axis). */
int sem_coords(sem_t h, double* x_host);

/* f = F(u) = M^-1 Q^T [ -nu sum_j D_j^T B D_j Q u_c - B sum_j (Q u_j) o D_j (Q u_c) ]
 * Eq. rhsvec (Sec. 3.3) with the sign of Eq. burgers23d, in the explicit form
 * du/dt = M^-1 P[u] of Sec. 3.4.  u, f: device states. */
int sem_rhs(sem_t h, const double* u, double* f, void* stream);

/* jw = J(u) w, the tangent of sem_rhs (eq. jacvec). */
int sem_jac_apply(sem_t h, const double* u, const double* w, double* jw, void* stream);

/* jtv = J(u)^T v, the Euclidean transpose of sem_jac_apply (eq. jactransvec, the
 * paper's contribution): jtv = Q^T L^T Q M^-1 v with one shared divergence for the
 * viscous and D_j^T[u_j o w] terms. */
int sem_jacT_apply(sem_t h, const double* u, const double* v, double* jtv, void* stream);

/* Forward sweep (Sec. 4.1, Fig. 1): u_{k+1} = RK step of u_k for k < nsteps, from
 * u0 to uT (device states; uT must not overlap u0).  Stores what the adjoint
 * needs according to the
 * handle's checkpoint mode.  dt > 0, nsteps >= 1.  Returns SEM_ERR_NONFINITE if
 * the final state is not finite (the check synchronises the stream), SEM_ERR_OOM
 * if the trajectory does not fit the budget or the device. */
int sem_rk_forward(sem_t h, int scheme, double dt, int nsteps,
                   const double* u0, double* uT, void* stream);

/* Backward sweep: lam0 = (d u_N / d u_0)^T lamT along the last forward sweep
 * (eqs. adjointloop, initadj, gradient with the RK tableau; Euclidean adjoint).
 * SEM_ERR_STATE if no forward sweep was recorded.  Checks finiteness like
 * sem_rk_forward. */
int sem_rk_adjoint(sem_t h, const double* lamT, double* lam0, void* stream);

/* J_host = 1/2 (u - u_obs)^T M (u - u_obs) and lam = M (u - u_obs) (eqs. ourcost,
 * initadj).  Synchronises `stream` to write *J_host.  lam may be NULL. */
int sem_objective(sem_t h, const double* u, const double* u_obs,
                  double* J_host, double* lam, void* stream);

/* One gradient evaluation of the misfit J(u0) = 1/2 ||u_N(u0) - u_obs||_M^2
 * (Fig. 1): forward sweep, objective, terminal adjoint, backward sweep.
 * grad = dJ/du0 (Euclidean).  Synchronises `stream` to write *J_host. */
int sem_objective_grad(sem_t h, int scheme, double dt, int nsteps,
                       const double* u0, const double* u_obs,
                       double* J_host, double* grad, void* stream);

/* CUDA-graph execution of sem_objective_grad (and sem_batch_objective_grad):
 * with enable != 0 the first call records the whole launch sequence of the
 * gradient evaluation (forward sweep with trajectory storage, misfit, terminal
 * adjoint, backward sweep) into a CUDA graph on a private stream, after making
 * every allocation it needs, and each later call with the same scheme, dt,
 * nsteps and u0 / u_obs / grad pointers replays that graph on `stream`.  A
 * call with other arguments records a new graph.  With opt-in kernel timing
 * (sem_profile) enabled while recording, the sampled launches' event pairs
 * become nodes of the graph and every replay adds their times to the
 * counters of sem_profile_read.  enable = 0 releases the graph. */
int sem_set_graph(sem_t h, int enable);
long long sem_graph_replays(sem_t h);   /* graph launches so far; -1 for a null handle */

/* Host-only: optimal number of extra forward steps (advances) the binomial
 * schedule spends to reverse `nsteps` steps from a stored start state with
 * `slots` further state slots (Sec. 5.3, revolve).  Returns SEM_ERR_ARG for
 * nsteps < 1, slots < 0 or a null pointer. */
int sem_ckpt_plan(int nsteps, int slots, long long* advances);

/* Work counters of the last sweeps on this handle: out3[0] = F applies in the
 * last forward sweep, out3[1] = F applies the last adjoint sweep spent on
 * recomputation (stage taping and checkpoint replays), out3[2] = J^T applies in
 * the last adjoint sweep.  Host-only. */
int sem_sweep_stats(sem_t h, long long* out3);

/* Frozen advection: the linear problems of Sec. 6.1 (advection-diffusion with
 * a given velocity).  With a != NULL (a device state, copied on `stream`), the
 * time integrators of this handle (sem_rk_forward, sem_rk_adjoint and
 * sem_objective_grad, every scheme) integrate the linear equation
 *     du/dt = J(a) u = nu Lap u - (a . grad) u - (u . grad) a,
 * the tangent of F at the fixed field a (eq. jacvec); for a constant field a
 * this is u_t + a . grad u = nu Lap u, component by component.  Their adjoints
 * use J(a)^T at every stage, so the forward sweep of an explicit scheme stores
 * no trajectory.  sem_rhs, sem_jac_apply and sem_jacT_apply are unaffected.
 * a == NULL returns the handle to Burgers.  Either call discards the recorded
 * forward sweep and any recorded gradient graph. */
int sem_set_advection(sem_t h, const double* a, void* stream);

/* Contraction engine of the element kernels (no counterpart in the paper, whose
 * element products are BLAS calls, Sec. 3.3 and 6.3).
 * SEM_CONTRACT_CUDA_CORE (default): the 1D contractions are even-odd split FMA
 * chains on the CUDA cores.  SEM_CONTRACT_TENSOR: for 3D handles of order N = 15
 * (16 points per direction), the F(u) element pass applies each 16 x 16 matrix to
 * the 256 lines of a direction as one matrix product on the tensor cores: tcgen05
 * MMAs with split-TF32 operands and FP32 accumulation in the FP32-bulk form
 * (three TF32 products per contraction, near FP32 accuracy), DMMA (mma.sync
 * m8n8k4, FP64) in the FP64 form.  J and J^T keep the CUDA-core kernels.  Returns
 * SEM_ERR_ARG for other grids, for FP64-DF and for batch handles.  Discards a
 * recorded gradient graph. */
#define SEM_CONTRACT_CUDA_CORE 0
#define SEM_CONTRACT_TENSOR    1
int sem_set_contraction(sem_t h, int mode);

/* Programmatic dependent launch (process-wide; on by default; no counterpart in
 * the paper).  Element and assembly kernels are launched with the programmatic
 * stream-serialization attribute: the next kernel's blocks may be scheduled
 * while the previous one finishes, each kernel waiting for its predecessor's
 * completion and memory before it reads anything, so only launch latency is
 * hidden and results are unchanged.  enable = 0 launches them the ordinary way
 * (for comparison).  Affects launches made after the call, and graphs recorded
 * after it. */
int sem_set_dependent_launch(int enable);

/* Element-kernel and assembly launches made by operator applies since the last
 * forward sweep began (its adjoint sweep included; a recorded gradient graph
 * replays the launches counted while it was recorded).  Host-only. */
int sem_launch_count(sem_t h, long long* launches);

/* Adaptive step sizes (Sec. 5.1: the step follows an estimate of the local
 * truncation error, weighted by absolute and relative tolerances).  With atol > 0
 * or rtol > 0, sweeps with scheme SEM_BS3 (sem_rk_forward, sem_objective_grad)
 * integrate over the horizon T = dt * nsteps starting from the trial step dt:
 * each attempted step also evaluates F(u_{n+1}) for the second-order companion
 * of the Bogacki-Shampine 3(2) pair; the error E = u_{n+1} - uhat_{n+1} is taken
 * in the RMS norm weighted by 1 / (atol + rtol max(|u_n|, |u_{n+1}|)); a step is
 * accepted when that norm is <= 1 and the next trial step is
 * dt min(fmax, max(0.2, 0.9 err^(-1/3))), fmax = 5 (1 right after a rejection);
 * the last step ends on T.  Each attempt synchronises the stream once to read the
 * norm.  Every accepted state is kept on the device (growing the trajectory
 * buffer, within ckpt_budget_bytes when set); sem_rk_adjoint differentiates the
 * accepted steps with their sizes held fixed.  FP64 form only; never captured in
 * a CUDA graph.  atol = rtol = 0 turns adaptivity off (SEM_BS3 then takes nsteps
 * fixed steps). */
int sem_set_adaptive(sem_t h, double atol, double rtol);

/* Accepted and rejected steps of the last adaptive sweep, and the first
 * min(cap, accepted) accepted step sizes in dts (may be NULL when cap = 0).
 * Zeros when the last sweep was not adaptive.  Host-only. */
int sem_adaptive_steps(sem_t h, int* accepted, int* rejected, double* dts, int cap);

/* Second level of the trajectory store (Sec. 5.4: the paper's checkpoints may
 * live in RAM or on disk).  host_bytes > 0 lets SEM_CKPT_TWO_LEVEL (and AUTO, when
 * every step's state does not fit the device budget) keep states in up to
 * host_bytes of pinned host memory, allocated at the next forward sweep that needs
 * them.  The forward sweep copies each host-tier state from a device staging slot
 * on a second stream while the following steps compute; the adjoint sweep loads
 * them back up to three steps ahead.  Results are bitwise equal to
 * SEM_CKPT_STATES.  Gradient evaluations that use the host tier run without a
 * CUDA graph.  0 releases the host buffer (after synchronising the device).
 * Returns SEM_ERR_OOM from the sweep if the states do not fit both levels. */
int sem_set_host_tier(sem_t h, size_t host_bytes);

/* Storage used by the last forward sweep: out4[0] its SEM_CKPT_* mode (0 when none
 * was recorded or the sweep was linear), out4[1] vectors held on the device,
 * out4[2] states held in host memory, out4[3] binomial slots.  Host-only. */
int sem_trajectory_info(sem_t h, long long* out4);

/* Settings of the SEM_CN solves (Sec. 6.3 names the scheme; the solver is this
 * library's): Newton stops when |delta| <= newton_rtol max(|u_{n+1}|, 1) (2-norms);
 * each linear system (I - dt/2 J(u)) x = b or (I - dt/2 J(u)^T) x = b runs
 * restarted GMRES(krylov_m) from x = 0 until |b - A x| <= krylov_rtol |b|,
 * failing with SEM_ERR_NONFINITE after krylov_maxit Arnoldi steps (likewise
 * Newton after 30 iterations).  Defaults 1e-12, 1e-12, 30, 2000.
 * 1 <= krylov_m <= 38.  Host-only apart from freeing the Krylov basis when
 * krylov_m changes.  The solves synchronise their stream once per Arnoldi step,
 * so with SEM_CN sem_objective_grad runs without a CUDA graph. */
int sem_set_solver(sem_t h, double newton_rtol, double krylov_rtol, int krylov_m, int krylov_maxit);

/* Counters of the last SEM_CN sweeps: out4[0] Newton iterations and out4[1]
 * Arnoldi steps of the forward sweep, out4[2] Arnoldi steps of the adjoint
 * sweep, out4[3] operator applies of both.  Host-only. */
int sem_solver_stats(sem_t h, long long* out4);

/* Opt-in kernel timing (no counterpart in the paper; used by the benchmarks).
 * With every = n > 0, one launch in n of each kind on this handle is bracketed
 * by a pair of CUDA events on its stream (every = 0 turns timing off).
 * sem_profile_read waits for the recorded events and returns the summed device
 * time in ms (ms4) and the number of timed launches (count4) per kind:
 * [0] F element kernel, [1] J element kernel, [2] J^T element kernel,
 * [3] gather-scatter assembly; reset != 0 clears them.  bytes4 (may be NULL)
 * receives the algorithmic bytes of the timed launches, summed the same way:
 * for the assembly the element-local values read once plus every epilogue
 * source read and every output written once (8 bytes per unknown each); 0 for
 * the element kernels.  Each timed launch costs two event records; the stream
 * waits once per 4096 timed launches. */
int sem_profile(sem_t h, int every);
int sem_profile_read(sem_t h, double* ms4, long long* count4, double* bytes4, int reset);

/* ---------------------------------------------------------------- batches
 * Many independent optimisation problems of uneven size (the paper solves one;
 * this serves ensembles of them).  sem_batch_create makes one handle for
 * `count` independent periodic 2D viscous-Burgers instances on [0, L)^2,
 * instance k with E[k] elements per direction of order N[k] in {3, 5, 7, 9}
 * and viscosity nu[k] >= 0.  `common` (may be NULL) supplies L and the
 * checkpoint mode, slots and budget; precision must be SEM_PREC_FP64.
 * The handle works with every state entry point (sem_rhs, sem_jac_apply,
 * sem_jacT_apply, sem_rk_forward, sem_rk_adjoint, sem_objective,
 * sem_objective_grad) on PACKED vectors: instance k occupies
 * [offset, offset + ndof) of sem_batch_layout, in the single-instance layout.
 * All instances advance with the same scheme and dt; each operator pass is one
 * persistent launch over all instances' elements plus one gather-scatter
 * launch, and every instance's result is bitwise equal to its own handle's.
 * The misfit of sem_objective / sem_objective_grad is the sum over instances.
 * Host-only; SEM_ERR_ARG for count < 1, null arrays or an unsupported instance. */
int sem_batch_create(int count, const int* E, const int* N, const double* nu,
                     const sem_opts* common, sem_t* out);
int sem_batch_count(sem_t h);   /* 0 for a single-instance handle */
int sem_batch_layout(sem_t h, int k, size_t* offset, size_t* ndof);
int sem_batch_coords(sem_t h, int k, double* x_host);   /* instance k's G node coordinates */

/* Autotuner of the batched element kernel: times the J^T element pass with
 * 64, 128, 192 and 256 threads per block (elements per block = threads / (N+1)
 * per instance) and keeps the fastest; ms4 (may be NULL) receives the four
 * times, *threads the choice.  The first operator apply on a batch runs it
 * when it has not run yet; both synchronise `stream`. */
int sem_batch_autotune(sem_t h, double* ms4, int* threads, void* stream);

/* sem_objective_grad for a batch with the per-instance misfits J_host[count]. */
int sem_batch_objective_grad(sem_t h, int scheme, double dt, int nsteps,
                             const double* u0, const double* u_obs,
                             double* J_host, double* grad, void* stream);

/* Size of the fixed device array used by sem_rhs_noalloc (16 MiB). */
#define SEM_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)

/* f = F(u) exactly as sem_rhs computes it (the element kernels of the handle's
 * precision: FP64, FP64-DF or FP32-bulk, and the same gather-scatter), but
 * without allocating any device memory.  The paper has no counterpart; this
 * serves callers that cannot call cudaMalloc, e.g. hosts whose device memory
 * belongs to their own pool, or loops that must not take the synchronisation
 * an allocation can cause.  It works on a handle that has not yet allocated
 * its own workspace.
 * The element-local scratch is a file-scope device array of
 * SEM_NOALLOC_SCRATCH_BYTES on every GPU that loads the library, kept until the
 * process exits; grids needing more (d * E^d * (N+1)^d values of 4 bytes in the
 * FP32-bulk form, 8 otherwise) return SEM_ERR_ARG, and so do handles of
 * sem_batch_create.  The first call on a device looks the array up with that
 * device current, so make it before any stream capture.  All calls share the
 * array: calls whose kernels overlap on the GPU race and must be ordered by the
 * caller.  Arguments and errors otherwise as sem_rhs. */
int sem_rhs_noalloc(sem_t h, const double* u, double* f, void* stream);

/* Thread-local text of the last error ("" if none). */
const char* sem_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SEM_H */
