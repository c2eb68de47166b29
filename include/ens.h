/*
 * ens.h -- C ABI of the GB300 ensemble ODE/SDE solver (libens.so).
 *
 * The operation: solve N independent copies of one small differential equation
 *     du/dt = f(u, p, t),  u(t0) = u0            (ODE, arXiv 2304.06835 Sec. 3.1)
 *     dX = a(X,t) dt + b(X,t) dW                  (SDE, Sec. 3.3)
 * each with its own parameters p_j, initial state u0_j and time span [t0_j, tf_j]
 * (the ensemble problem of Sec. 5.1.1: the U, P and F matrices).  One GPU thread integrates
 * one trajectory with the whole step loop in registers (EnsembleGPUKernel, Sec. 5.2,
 * the one-thread-per-trajectory kernel listing).
 *
 * Conventions shared by every entry point:
 *   - Return value: ENS_OK or an ENS_E* code.  On error nothing was launched and
 *     ens_last_error() returns a message (thread-local, valid until the next call).
 *   - Array pointers passed to ens_solve* / ens_adjoint / ens_mlp_* are DEVICE pointers
 *     owned by the caller, except where a parameter says HOST.  The library never frees
 *     or allocates caller memory; it allocates only its own small scratch (queue counters,
 *     adjoint replay buffers, staging for ens_solve_host), owned by the handle and freed
 *     by ens_destroy.
 *   - Calls are asynchronous on `cuda_stream` (a cudaStream_t, NULL = legacy default
 *     stream) unless stated otherwise.  Calls that share a handle must be ordered on one
 *     stream (they share the handle's scratch).
 *   - Per-trajectory numerical failures do not fail a call: they go to status[i].
 *   - N = 0 is a no-op that returns ENS_OK.
 */
#ifndef ENS_H_
#define ENS_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ens_handle ens_handle;

/* return codes */
enum { ENS_OK = 0, ENS_EINVAL = 1, ENS_ENOTSUP = 2, ENS_ECUDA = 3, ENS_ENOMEM = 4 };

/* right-hand sides compiled into the library (Appendix models):
 *   LORENZ    D=3 P=3  p=(sigma, rho, beta)   f = (sigma(y2-y1), y1(rho-y3)-y2, y1 y2 - beta y3)
 *             (Appendix, Lorenz problem; the paper writes beta as gamma)
 *   ROBERTSON D=3 P=3  p=(k1, k2, k3)         f = (-k1 y1 + k3 y2 y3, k1 y1 - k3 y2 y3 - k2 y2^2,
 *                                                   k2 y2^2)   (Appendix, Robertson equation)
 *   GBM       D=1 P=2  p=(mu, sigma)          a = mu X, b = sigma X   (Appendix, linear SDE);
 *             ODE algorithms integrate the drift only (u' = mu u).
 *   CRN       D=4 P=6  u=([sigma], A1, A2, A3), p=(S, D, tau, nu0, n, eta); 8 Wiener processes
 *             (Appendix, sigma-factor CRN; Chemical Langevin form):
 *               a = (nu0 + H - [sigma], ([sigma] - A1)/tau, (A1 - A2)/tau, (A2 - A3)/tau),
 *               H = (S[sigma])^n / ((S[sigma])^n + (D A3)^n + 1);
 *               noise of [sigma]: eta(sqrt(nu0 + H) dW1 - sqrt([sigma]) dW2), of A_i:
 *               eta(sqrt(A_{i-1}/tau) dW_{2i+1} - sqrt(A_i/tau) dW_{2i+2}) with A_0 = [sigma].
 *             Square-root arguments and the two Hill bases are taken as max(., 0) (the form
 *             is undefined for negative amounts, which a discrete path can reach).
 *             Euler-Maruyama only.
 *   BALL      D=2 P=2  u=(x, v), p=(g, e)       f = (v, -g)   (Appendix, bouncing ball;
 *             Sec. 6.5 events).  Event: x reaching 0 from above sets v <- -e v.  Each
 *             accepted step's dense output (see ens_opts.dense) is checked at 10 evenly
 *             spaced points; the first crossing is located by the Illinois method to 4 ulp
 *             of the step, the state there takes the affect and the integration restarts
 *             from it.  A crossing and recrossing between two checkpoints is not seen, so a
 *             step much longer than the shortest flight needs ens_opts.dtmax.
 *             TSIT5_ADAPTIVE only.
 *   OREGO     D=3  P=3   p=(k1, k2, k3)  Oregonator: f = (k1 (y2 + y1 (1 - k2 y1 - y2)),
 *             (y3 - (1 + y1) y2) / k1, k3 (y1 - y3)) (Appendix; the first equation's leading
 *             sign read as +, the Field-Noyes model: with the printed minus the printed initial
 *             state runs to -infinity).
 *   HIRES     D=8  P=12  p = its 12 distinct rate constants in order of appearance
 *             (1.71, 0.43, 8.32, 0.0007, 8.75, 10.03, 0.035, 1.12, 1.745, 280, 0.69, 1.81);
 *             a constant printed in several equations is one parameter (Appendix, HIRES).
 *   POLLU     D=20 P=25  p=(k1..k25): the printed equations, which are exactly the sum over
 *             25 mass-action reactions ("k7 u9", "2 k18 u16" read as k7 y9, 2 k18 y16)
 *             (Appendix, POLLU).  HIRES and POLLU take the Rosenbrock methods (ROS23,
 *             RODAS4, RODAS5P), one trajectory per thread; their W is factored by a sparse
 *             LU on the fixed Jacobian pattern (a minimum-degree order and its fill decided
 *             at compile time; a column whose partial pivoting would exchange rows sends
 *             the step to a dense LU with row exchanges). */
enum { ENS_RHS_LORENZ = 1, ENS_RHS_ROBERTSON = 2, ENS_RHS_GBM = 3, ENS_RHS_CRN = 4,
       ENS_RHS_BALL = 5, ENS_RHS_OREGO = 6, ENS_RHS_HIRES = 7, ENS_RHS_POLLU = 8 };

/* algorithms:
 *   TSIT5_FIXED    Tsitouras 5(4) pair, fixed step dt (GPUTsit5, Sec. 5.2.1; RK step Sec. 3.1)
 *   TSIT5_ADAPTIVE same with the embedded error estimate, scaled RMS ratio q and PI control
 *                  h_new = eta q_{n-1}^{beta2} q_n^{beta1} h (Sec. 3.1)
 *   RK4            classic 4-stage Runge-Kutta, fixed step (explicit RK family, Sec. 3.1)
 *   ROS23          Rosenbrock23, the Shampine-Reichelt 2(3) Rosenbrock-W pair with a 3x3 LU of
 *                  W = I - h d J held in registers (GPURosenbrock23, Sec. 5.2.1; Sec. 3.2.1)
 *   EM             Euler-Maruyama, fixed step, X += a h + sum_m b_m sqrt(h) Z_{k,m} over the
 *                  model's M Wiener processes (diagonal noise for GBM, M = 1; non-diagonal
 *                  for the CRN, M = 8) (GPUEM, Sec. 5.2.2; Sec. 3.3).  Z_{k,m} is normal
 *                  number k*M + m of the trajectory's Philox stream (see ens_normals).
 *   RODAS4         Rodas4, the stiffly accurate 4(3) Rosenbrock method of Hairer and Wanner
 *                  (GPURodas4, Sec. 5.2.1; Sec. 3.2.1), 6 stages, one LU of W = I - h gamma J
 *                  per attempt; adaptive with the PI control of TSIT5_ADAPTIVE (k = 4)
 *   RODAS5P        Rodas5P, Steinebach's stiffly accurate 5(4) Rosenbrock method (GPURodas5P,
 *                  Sec. 5.2.1), 8 stages; adaptive (k = 5).
 *   SIEA           weak order 2 stochastic Runge-Kutta step, fixed step, diagonal noise
 *                  (GPUSIEA, Sec. 5.2.2; the improved-Euler-type member of the SRK family of
 *                  Sec. 3.3): Ybar = X + a h + b dW, Y+- = X + a h +- b sqrt(h),
 *                  X += (a(X) + a(Ybar)) h/2 + (b(Y+) + b(Y-) + 2 b(X)) dW/4
 *                       + (b(Y+) - b(Y-)) (dW^2 - h) / (4 sqrt(h)), dW = sqrt(h) Z_k
 *                  (the normals of EM's stream); models with diagonal noise only (GBM).
 * The Rosenbrock methods save at save times by stepping onto them (no interpolation) and need
 * a model with a Jacobian (not the CRN or the bouncing ball). */
enum {
  ENS_TSIT5_FIXED = 1, ENS_TSIT5_ADAPTIVE = 2, ENS_RK4 = 3, ENS_ROS23 = 4, ENS_EM = 5,
  ENS_RODAS4 = 6, ENS_RODAS5P = 7, ENS_SIEA = 8
};

/* element type of every floating-point array of a call */
enum { ENS_F32 = 0, ENS_F64 = 1 };

/* array layouts (the paper's n x N state matrix U is the SOA layout, Sec. 5.1.1):
 *   ROWMAJOR  params[N][P], u0[N][D], tspan[N][2], out[N][S][D]
 *   SOA       params[P][N], u0[D][N], tspan[2][N], out[S][D][N]  (coalesced) */
enum { ENS_LAYOUT_ROWMAJOR = 0, ENS_LAYOUT_SOA = 1 };

/* per-trajectory status codes written to status[i] */
enum { ENS_TRAJ_OK = 0, ENS_TRAJ_MAXITERS = 1, ENS_TRAJ_DT_MIN = 2, ENS_TRAJ_NONFINITE = 3 };

/* scheduling of trajectories onto threads */
enum {
  ENS_SCHED_AUTO = 0,       /* adaptive algorithms: PERSISTENT; fixed-step: DIRECT */
  ENS_SCHED_DIRECT = 1,     /* thread i integrates trajectories i, i+grid, ... */
  ENS_SCHED_PERSISTENT = 2  /* resident grid; a lane that finishes fetches the next trajectory
                               from an atomic queue (per-lane refill) */
};

/* order in which the persistent schedule hands out trajectories */
enum {
  ENS_ORDER_AUTO = 0,   /* adaptive algorithms: COST; fixed-step: INDEX */
  ENS_ORDER_INDEX = 1,  /* 0, 1, 2, ... */
  ENS_ORDER_COST = 2    /* longest expected work first: key (tf - t0) / h0 with h0 the
                           Hairer-Norsett-Wanner starting step (adaptive) or dt (fixed),
                           counting-sorted on the device into 1024 log-spaced buckets */
};

#define ENS_MAX_SAVE 256

typedef struct {
  int alg;                /* ENS_TSIT5_FIXED ... ENS_SIEA */
  int dtype;              /* ENS_F32 / ENS_F64 */
  int layout;             /* ENS_LAYOUT_* */
  double dt;              /* fixed-step size (TSIT5_FIXED, RK4, EM), > 0 */
  double abstol, reltol;  /* adaptive tolerances; abstol >= 1e-30, reltol >= 0 */
  double dt0;             /* adaptive first step; <= 0: Hairer-Norsett-Wanner starting step */
  long long maxiters;     /* per-trajectory cap on step attempts (>= 1); the fixed-step
                             methods take at most 2^31 - 2 steps whatever the cap (a longer
                             span stops there with ENS_TRAJ_MAXITERS) */
  const double* saveat;   /* HOST array of n_save ascending times, copied during the call;
                             NULL/0: only the final state is written (S = 1) */
  int n_save;             /* 0 .. ENS_MAX_SAVE */
  unsigned long long seed;   /* SDE: Philox4x32-10 key */
  long long index_offset;    /* SDE: trajectory i draws from stream index_offset + i */
  int schedule;           /* ENS_SCHED_* */
  int block;              /* threads per block; 0 = tuned / default.  Adaptive Tsit5 with
                             dense = 1 or a step record stages its output in shared memory
                             and takes at most 512 (more: ENS_ECUDA, too many resources). */
  int tpt;                /* trajectories per thread (1, 2 or 4); 0 = tuned / default.  The
                             Rosenbrock kernels, dense output and the step record run one.
                             FP32 on the final-state output, adaptive Tsit5 (persistent
                             schedule) and fixed-step Tsit5 / RK4 (direct schedule) run 2 as
                             one lockstep pair on the paired FP32 instructions (the default
                             for the fixed-step ones).  Every shape gives each trajectory the
                             result of 1. */
  int refill_min;         /* persistent schedule: a warp refills its idle trajectory slots
                             once at least this many of them are idle (1..32; 0 = default 4),
                             counted over all the warp's slots (32 x trajectories per thread);
                             one pass then gives each thread with an idle slot one new
                             trajectory.  Batching refills trades idle slots for fewer
                             divergent refill passes. */
  int order;              /* ENS_ORDER_* (persistent schedule only) */
  int blocks_per_sm;      /* persistent schedule: resident blocks per SM (0 = as many as fit;
                             -1, -2, -3 = that many quarters of them, as ens_autotune reports;
                             otherwise <= 64).  Fewer resident lanes each take more
                             trajectories from the queue, which shortens the drain at the end
                             of the queue. */
  int dense;              /* TSIT5_ADAPTIVE with save times: 0 = the steps are cut to land on
                             each save time; 1 = the steps run to tf uncut and each save time
                             s in a step [t_n, t_n + h] takes the dense output
                             u_n + h sum_i b_i(theta) k_i, theta = (s - t_n)/h: a C1
                             continuous extension of order 4 of the Tsit5 pair (Sec. 5.1.1
                             solution storage), so the steps and the final state are those
                             of the solve without save times.  Other algorithms ignore it. */
  double dtmax;           /* adaptive methods: largest step; <= 0: none.  Finite. */
  int step_cap;           /* adaptive methods, n_save = 0: > 0 stores every accepted step
                             (the paper's full-solution storage, Sec. 5.1.1).  out is then
                             [N][step_cap][D] (SOA: [step_cap][D][N]): entry k is the state
                             after k accepted steps (entry 0: u0; after an event, the state
                             that took the affect).  Entries past a trajectory's count are
                             not written.  Storing stops at step_cap; the solve goes on. */
  void* step_t;           /* device, opts->dtype: [N][step_cap] (SOA [step_cap][N]) times of
                             the entries, or NULL */
  int* step_n;            /* device int32 [N]: accepted steps + 1 (may exceed step_cap), or
                             NULL.  (ens_solve and ens_solve_noalloc; ens_solve_host
                             rejects a step record.) */
  /* measurement aid: two cudaEvent_t (or NULL), recorded on the solve's stream just before
     and just after the integrator kernel itself (not the longest-first ordering before it),
     so that the kernel's own duration can be read with cudaEventElapsedTime.  Both or none;
     batch plans and ens_solve_host ignore them. */
  void* kernel_start;
  void* kernel_stop;
} ens_opts;

/* Fill *o with defaults: TSIT5_ADAPTIVE, F32, SOA, abstol=reltol=1e-6, maxiters=1e6, auto. */
void ens_opts_default(ens_opts* o);

/* Create a solver handle for right-hand side `rhs_id` with state dimension D and parameter
 * count P (ENS_EINVAL unless they match the model).  Binds to the current CUDA device. */
int ens_create(ens_handle** h, int rhs_id, int D, int P);

/* Destroy a handle and free its scratch.  Waits for work the handle launched to finish. */
int ens_destroy(ens_handle* h);

/* Solve N trajectories (Sec. 5.1.1 ensemble problem; algorithms above).
 *   params, u0, tspan : device arrays in opts->dtype and opts->layout (read only)
 *   out               : device array [N][S][D] (layout) written with the state at each save
 *                       time (S = n_save) or the final state (S = 1).  Save times outside
 *                       [t0, tf] of a trajectory, or after a failure, are written as NaN.
 *                       Adaptive methods step exactly onto save times (adaptive Tsit5 with
 *                       opts->dense: the dense output at them, steps not cut); fixed-step
 *                       methods record after step ceil((s - t0)/dt - 1e-12).  With
 *                       opts->step_cap > 0: the every-step record instead (see ens_opts).
 *   status            : device int8 [N] (ENS_TRAJ_*) or NULL
 *   stats             : device int32 [3][N] = accepted steps, rejected steps, f evaluations,
 *                       or NULL
 * Validation (ENS_EINVAL): null arrays, N < 0, unsupported (rhs, alg) pair (EM needs an
 * SDE model: GBM or CRN; the CRN takes EM only),
 * dt <= 0 for fixed-step, tolerances out of range, n_save > ENS_MAX_SAVE or unsorted. */
int ens_solve(ens_handle* h, long long N, const void* params, const void* u0, const void* tspan,
              const ens_opts* opts, void* out, signed char* status, int* stats,
              void* cuda_stream);

/* Same as ens_solve with HOST arrays (pageable or pinned): copies inputs to the device,
 * solves, copies out/status/stats back and synchronises the stream before returning.
 * From 2^20 trajectories the work runs in 2 chunks whose copies, on a stream of the
 * handle, overlap the other chunk's solve; the results equal one solve over all N (same
 * launch shape, SDE streams by index)
 * (the paper's high-level path that passes the problem to the GPU and returns the result
 * to the CPU, Sec. 6.1). */
int ens_solve_host(ens_handle* h, long long N, const void* params, const void* u0,
                   const void* tspan, const ens_opts* opts, void* out, signed char* status,
                   int* stats, void* cuda_stream);

/* Launch-shape autotuner (the occupancy tuning the paper leaves to KernelAbstractions,
 * Sec. 5.1): runs the solve of ens_solve (same arguments, outputs really written) with every
 * candidate launch shape -- block in {64, 128, 256, 512}, and for the persistent schedule
 * trajectories per thread in {1, 2} (1 only for the kernels that run one: Rosenbrock23, dense
 * output, step record) and resident blocks per SM in {all that fit, 3/4, 1/2 of that}; a
 * nonzero opts->block / opts->tpt / opts->blocks_per_sm pins that value; shapes that do not
 * fit the kernel are skipped --
 * timing each (one warm-up, best of two), and records the fastest in a process-wide cache
 * keyed by (model, algorithm, dtype, layout, floor(log2 N), output kind -- final state, save
 * times, dense save times or step record --, SM count).  Later
 * ens_solve / ens_batch_create calls with block = tpt = blocks_per_sm = 0 use the cached
 * shape.  Returns it in *block / *tpt / *blocks_per_sm (> 0 a cap, 0 all that fit, < 0 that
 * many quarters of the blocks that fit) and its time in *best_ms.  Synchronises the stream. */
int ens_autotune(ens_handle* h, long long N, const void* params, const void* u0,
                 const void* tspan, const ens_opts* opts, void* out, signed char* status,
                 int* stats, void* cuda_stream, int* block, int* tpt, int* blocks_per_sm,
                 float* best_ms);

/* Work estimate per trajectory (the key the longest-first order of the persistent schedule
 * sorts by, and the cost that balances the shards of one ensemble across ranks, as the
 * paper's MPI path scatters one ensemble, Sec. 6.3): keys[i] = the expected number of steps
 * of trajectory i -- (tf - t0) / dt for fixed-step methods, (tf - t0) / h0 for adaptive ones
 * with h0 the starting step (opts->dt0 if > 0, else the Hairer-Norsett-Wanner starting step
 * the solve itself takes).  Same arguments and checks as ens_solve, without outputs; keys is
 * a device float [N].  Asynchronous on cuda_stream. */
int ens_cost_keys(ens_handle* h, long long N, const void* params, const void* u0,
                  const void* tspan, const ens_opts* opts, float* keys, void* cuda_stream);

/* Batched ensembles: several sub-problems (different models, methods, sizes and time spans)
 * solved by one call -- the uneven-work case of Sec. 6.4 (trajectories whose step counts
 * differ) widened to mixed stiff / non-stiff / stochastic work.  A plan validates the items,
 * optionally autotunes each one, allocates its scratch and, with ENS_BATCH_GRAPH, captures the
 * whole batch into one CUDA graph: the items run as concurrent persistent (or direct) kernels
 * on forked streams, longest measured item first, joined back onto the caller's stream.
 * Flags:
 *   ENS_BATCH_GRAPH     capture into a CUDA graph; ens_batch_run is one graph launch
 *   ENS_BATCH_AUTOTUNE  run ens_autotune's search on every item during creation (the items'
 *                       outputs are written by the trial solves)
 *   ENS_BATCH_SERIAL    no concurrency: the items run one after another on the caller stream
 *   ENS_BATCH_FUSED     one persistent kernel for all items: every warp works through the
 *                       items' queues in the plan's order (longest measured first), taking the
 *                       next item's trajectories once the current item's queue is drained and
 *                       its lanes are done, so one item's tail overlaps the next item's work.
 *                       Available for items of three kinds, at most one of each, without save
 *                       times or step records: Lorenz FP32 TSIT5_ADAPTIVE, Robertson FP32
 *                       ROS23, GBM FP32 EM (one trajectory per thread, block 128);
 *                       ENS_ENOTSUP otherwise.
 * With GRAPH and AUTOTUNE (and more than one item) the plan also captures the serial order
 * and, when the items allow it, the fused kernel, times every graph at creation (one warm-up
 * and three timed launches each, writing the items' outputs) and keeps the fastest:
 * concurrent persistent kernels, each sized for the whole GPU, can crowd one another.
 * Each item's opts are those of ens_solve; saveat is copied at creation.  The plan keeps the
 * item pointers: ens_batch_run re-solves whatever the input arrays hold at that time. */
#define ENS_BATCH_MAX_ITEMS 16
enum { ENS_BATCH_GRAPH = 1, ENS_BATCH_AUTOTUNE = 2, ENS_BATCH_SERIAL = 4, ENS_BATCH_FUSED = 8 };

typedef struct {
  int rhs_id;               /* ENS_RHS_* */
  long long N;
  const void* params;       /* device arrays as for ens_solve */
  const void* u0;
  const void* tspan;
  void* out;
  signed char* status;      /* or NULL */
  int* stats;               /* or NULL */
  ens_opts opts;
} ens_batch_item;

typedef struct {
  int schedule, block, tpt; /* launch shape the plan uses */
  int blocks_per_sm;        /* persistent: > 0 a cap, 0 all that fit, < 0 that fraction x 4 */
  float tuned_ms;           /* autotuned solve time of the item alone (0 if not tuned) */
  int launch_position;      /* position in the launch order (-1: empty item) */
  int graph;                /* 1 if the plan runs as a CUDA graph */
  int serial;               /* 1 if the items run one after another */
  float graph_ms_concurrent;  /* GRAPH|AUTOTUNE: measured time of the concurrent graph, */
  float graph_ms_serial;      /* of the serial one, */
  float graph_ms_fused;       /* and of the fused kernel (0: not measured) */
  int fused;                /* 1 if the plan runs the fused kernel */
  unsigned long long lane_slots;  /* lane slots the item's persistent loops issued in the last
                                     run (iterations x 32 x trajectories per thread; 0 for a
                                     direct-schedule item): the item's attempts divided by this
                                     is its lane efficiency.  Reading it synchronises with the
                                     device. */
} ens_batch_item_info;

typedef struct ens_batch ens_batch;

/* Create a plan (may synchronise cuda_stream: autotuning and graph capture do). */
int ens_batch_create(ens_batch** b, const ens_batch_item* items, int n_items, int flags,
                     void* cuda_stream);
/* Solve every item (asynchronous on cuda_stream). */
int ens_batch_run(ens_batch* b, void* cuda_stream);
int ens_batch_info(const ens_batch* b, int item, ens_batch_item_info* info);
/* Waits for the device, then frees the plan. */
int ens_batch_destroy(ens_batch* b);

/* Discrete adjoint of a fixed-step explicit Runge-Kutta solve (TSIT5_FIXED or RK4).
 * The paper differentiates through its solvers with automatic differentiation (Sec. 6.5);
 * here the reverse mode of the step map of Sec. 3.1 (U_i = u_n + h sum_j a_ij k_j,
 * k_i = f(U_i, p), u_{n+1} = u_n + h sum_i b_i k_i) is written out: per step, with
 * lambda = dL/du_{n+1}, the stage adjoints kbar_i = h b_i lambda + h sum_{l>i} a_li Ubar_l,
 * Ubar_i = f_u(U_i)^T kbar_i, dL/dp += f_p(U_i)^T kbar_i, dL/du_n = lambda + sum_i Ubar_i.
 * The result is the exact gradient of the discrete map (not of the ODE), up to rounding.
 *
 * Checkpointing: u is stored every `checkpoint_every` = K steps; the reverse pass replays
 * each K-step segment from its checkpoint, storing the stage inputs, then transposes it.
 *   max_steps  : upper bound on any trajectory's step count n = ceil((tf - t0)/dt - 1e-12).
 *                Trajectories with more steps get status MAXITERS, NaN state and gradients.
 *   ckpt       : device array of ens_adjoint_ckpt_elems(N, D, max_steps, K) elements of
 *                opts->dtype, laid out [C][D][N], C = ceil(max_steps / K).
 * Options used: alg, dtype, layout, dt (others ignored).  Arrays follow opts->layout like
 * ens_solve: params [N][P], u0 [N][D], tspan [N][2], out / grad_out / grad_u0 [N][D],
 * grad_p [N][P] (ROWMAJOR) or their transposes (SOA).  Asynchronous on cuda_stream.
 * Errors: ENS_EINVAL for another algorithm, dt <= 0, max_steps < 1, K < 1, null arrays;
 * ENS_ENOMEM when the handle's scratch cannot be allocated. */

/* Elements of the checkpoint array (C * D * N), or -1 for invalid arguments. */
long long ens_adjoint_ckpt_elems(long long N, int D, long long max_steps, int checkpoint_every);

/* Forward pass with checkpoints: writes out = u(tf) (or skips it if out is NULL), ckpt, and
 * status (OK or MAXITERS; NULL allowed). */
int ens_adjoint_forward(ens_handle* h, long long N, const void* params, const void* u0,
                        const void* tspan, const ens_opts* opts, long long max_steps,
                        int checkpoint_every, void* out, void* ckpt, signed char* status,
                        void* cuda_stream);

/* Reverse pass: grad_out = dL/du(tf) in; grad_p = dL/dp and grad_u0 = dL/du0 out.  ckpt is
 * the array written by ens_adjoint_forward with the same arguments, or NULL, in which case
 * the forward pass runs first into handle-owned scratch.  The handle also owns the segment
 * buffer of K * S * D * N elements (S = 6 stages for TSIT5_FIXED, 4 for RK4). */
int ens_adjoint(ens_handle* h, long long N, const void* params, const void* u0, const void* tspan,
                const ens_opts* opts, long long max_steps, int checkpoint_every, const void* ckpt,
                const void* grad_out, void* grad_p, void* grad_u0, void* cuda_stream);

/* Learned surrogate (no counterpart in the paper: an addition to the ensemble method).
 * A multilayer perceptron with widths 6 -> 256 -> 256 -> 256 -> 3 and exact-erf GELU maps a
 * Lorenz problem x = (sigma, rho, beta, u0_1, u0_2, u0_3) to its state u(tf); `members`
 * independently initialised copies form an ensemble whose disagreement gates a fallback to
 * the solver.  BF16 operands, FP32 accumulation, every product on the tcgen05 tensor cores
 * (gelu(z) = z Phi(z), the exact erf form, with erf evaluated by Abramowitz & Stegun 7.1.26,
 * absolute error <= 1.5e-7):
 *   x_n = bf16(2 (x - lo)/(hi - lo) - 1),  Z_l = H_{l-1} W_l^T + b_l,  H_l = bf16(gelu(Z_l)),
 *   y = Z_4 * y_std + y_mean.
 * Parameters per member: FP32, flat in the order W_1 [256][6], b_1 [256], W_2 [256][256],
 * b_2, W_3 [256][256], b_3, W_4 [3][256], b_4 [3] (ens_mlp_n_params() = 134,147 values).
 * Arrays are device arrays; x [B][6] and y [B][3] FP32 row-major.  Calls are asynchronous
 * unless stated; calls on one network share its workspace and must be ordered on one stream.
 * A wait for the tensor cores that exceeds one second sets an error flag that ens_mlp_check
 * reports (the results of that call are then invalid). */
typedef struct ens_mlp ens_mlp;
long long ens_mlp_n_params(void);
/* box: HOST [6][2] (lo, hi) of the inputs, used to normalise x and by the gate.  batch_max:
 * rows of the workspace (a multiple of 128); longer forward calls are processed in chunks.
 * Parameters are drawn uniform in +-1/sqrt(fan_in) from Philox4x32-10 keyed by `seed`.
 * Synchronises the stream. */
int ens_mlp_create(ens_mlp** m, int members, long long batch_max, const double* box,
                   unsigned long long seed, void* cuda_stream);
int ens_mlp_destroy(ens_mlp* m);
/* output de-standardisation y = z * y_std + y_mean (HOST arrays of 3); synchronises. */
int ens_mlp_set_scaling(ens_mlp* m, const double* y_mean, const double* y_std, void* cuda_stream);
/* copy member's FP32 parameters to `get` and/or replace them from `set` (device, n_params) */
int ens_mlp_params(ens_mlp* m, int member, float* get, const float* set, void* cuda_stream);
/* Forward + backward of one member on a minibatch (B <= batch_max): the gradient of the mean
 * squared error on standardised targets, L = sum (z - (y - y_mean)/y_std)^2 / (3B), is kept
 * for ens_mlp_adam and copied to `grad` (n_params, or NULL); the loss to *loss (device
 * double, or NULL).  Row b of the minibatch is x[idx[b]], y[idx[b]] when idx (device int64
 * [B]) is given, else x[b], y[b]. */
int ens_mlp_grad(ens_mlp* m, int member, long long B, const float* x, const float* y,
                 const long long* idx, float* grad, double* loss, void* cuda_stream);
/* One Adam step (Kingma & Ba; beta1 0.9, beta2 0.999, eps 1e-8, step count t >= 1) of one
 * member with the gradient of the last ens_mlp_grad call. */
int ens_mlp_adam(ens_mlp* m, int member, float lr, int t, void* cuda_stream);
/* Inference: y [E'][B][3] for member (E' = 1) or all members (member = -1, E' = members).
 * By default one fused persistent kernel computes all layers of all requested members with
 * the activations kept on chip (warp-specialised: TMA weight streaming, tcgen05 MMAs of two
 * 128-sample tiles in flight, epilogue warps); flags = ENS_MLP_LAYERWISE runs the same
 * arithmetic layer by layer through global memory (identical results). */
#define ENS_MLP_LAYERWISE 1
int ens_mlp_forward(ens_mlp* m, int member, long long B, const float* x, float* y, int flags,
                    void* cuda_stream);
/* Gate: y_mean [B][3] = mean over the members of y_members [members][B][3] (NULL to skip);
 * spread [B] = the largest per-component population standard deviation over the members
 * (NULL to skip; the statistic a gate threshold is calibrated on);
 * fallback[b] = 1 when x_b leaves the box or spread[b] exceeds tau; *n_fallback (device, or
 * NULL) is incremented by the
 * number of fallbacks (zero it first).  With fb_index given, every fallback sample is also
 * appended, at a slot taken from *n_fallback, to a compacted solver problem in ROWMAJOR FP32
 * layout: fb_index[slot] = b, fb_params[slot] = (sigma, rho, beta), fb_u0[slot] = u0,
 * fb_tspan[slot] = (t0, t1) (each array has room for B rows; slot order is arbitrary). */
int ens_mlp_gate(ens_mlp* m, long long B, const float* x, const float* y_members, float tau,
                 float* y_mean, float* spread, unsigned char* fallback, unsigned long long* n_fallback,
                 long long* fb_index, float* fb_params, float* fb_u0, float* fb_tspan, double t0,
                 double t1, void* cuda_stream);
/* y[fb_index[i]] = u[i] (rows of 3) for i < n: the solver's answers for the fallbacks. */
int ens_mlp_scatter(long long n, const long long* fb_index, const float* u, float* y,
                    void* cuda_stream);
/* Synchronise the stream and report a tensor-core wait timeout of an earlier call. */
int ens_mlp_check(ens_mlp* m, void* cuda_stream);
/* Test aid: out[i] = gelu(z[i]) (which = 0) or gelu'(z[i]) (which = 1) evaluated exactly as the
 * network kernels evaluate them (device arrays of n floats). */
int ens_mlp_activation(int which, long long n, const float* z, float* out, void* cuda_stream);

/* Ensemble moments for Monte Carlo estimation (Sec. 3.3: the expectation and variance of an
 * SDE's solution estimated over the ensemble), and the exchange step of a sharded ensemble:
 * each rank reduces its own trajectories, then the ranks' results are merged
 * (ens_moments_combine) into the whole ensemble's.
 *   out    : device array in `dtype`, the layout of ens_solve's output ([N][S][D] row-major,
 *            [S][D][N] SOA); the moments are over save slot `slot` (0 <= slot < S; S = 1 for a
 *            final-state solve)
 *   status : device int8 [N] or NULL; with it only trajectories with status 0 count
 *   scratch: device double [ENS_MOMENTS_BLOCKS * (2D + 1)], caller-owned: the partial
 *            results of the first pass (overwritten)
 *   result : device double [2D + 1]: result[j] = mean of x_j, result[D + j] = M2_j = sum over
 *            the counted trajectories of (x_j - mean_j)^2 (j < D), result[2D] = n, the number
 *            of trajectories counted; written, not accumulated.  The unbiased variance is
 *            M2_j / (n - 1).  With n = 0 every entry is 0.
 * FP64 arithmetic; groups are joined by the pairwise update of Chan, Golub and LeVeque (no
 * cancellation of raw power sums when |mean| >> std); deterministic (fixed merge orders in
 * two passes: ENS_MOMENTS_BLOCKS blocks, then one).  Asynchronous on cuda_stream; calls
 * sharing a scratch array must be ordered on one stream.  ENS_EINVAL for bad sizes, slot,
 * dtype, layout or null pointers. */
#define ENS_MOMENTS_BLOCKS 608
int ens_moments(long long N, int D, int dtype, int layout, int S, int slot, const void* out,
                const signed char* status, double* scratch, double* result, void* cuda_stream);

/* Merge the ens_moments results of n_parts disjoint groups of trajectories (e.g. the ranks of
 * a sharded ensemble, gathered in rank order) into the moments of their union, by the same
 * pairwise update, in the order given.  HOST arrays: parts [n_parts][2D + 1], result
 * [2D + 1], both in ens_moments' result layout (mean, M2, n).  Synchronous, no device work.
 * ENS_EINVAL for n_parts < 1, D < 1 or null pointers. */
int ens_moments_combine(int n_parts, int D, const double* parts, double* result);

/* Raw Philox4x32-10 words (Salmon et al. SC'11) of the SDE streams: for trajectory
 * j < n_traj and call c < n_calls, out[(c*4 + w)*n_traj + j] = word w of
 * Philox(counter = (c lo, c hi, (index_offset+j) lo, hi), key = (seed lo, seed hi)).
 * Device array out; used to check the generator bit-exactly. */
int ens_philox4x32_10(unsigned long long seed, long long index_offset, long long n_traj,
                      long long n_calls, unsigned int* out, void* cuda_stream);

/* The standard normals Z_k (k < n_per) of trajectory j's stream (Euler-Maruyama step s of a
 * model with M Wiener processes uses Z_{s*M} .. Z_{s*M+M-1}): out[k*n_traj + j] in `dtype` (F32: 4 normals per Philox call, F64: 2).  Box-Muller of the
 * uniforms ((x>>9)+0.5)*2^-23 (F32) or ((x0:x1 >> 12)+0.5)*2^-52 (F64),
 * exact and inside (0,1). */
int ens_normals(unsigned long long seed, long long index_offset, long long n_traj,
                long long n_per, int dtype, void* out, void* cuda_stream);

/* Measurement aid (no counterpart in the paper): times `blocks` x `threads` threads that each
 * run 8 independent FMA chains for 16*iters steps in `dtype`, synchronising the stream, and
 * writes the achieved FMA instructions per second (lane-level) to *ops_per_s.  Used to
 * measure the FP32 / FP64 FMA-pipe rate that bounds the solver. */
int ens_probe_fma(int dtype, long long iters, int blocks, int threads, double* ops_per_s,
                  void* cuda_stream);

/* No counterpart in the paper.  The ensemble solve of ens_solve (same options, same
 * device-array arguments, same results) for callers that must not allocate device memory:
 * a framework that owns all device memory through its own pool, a real-time loop that cannot
 * pay cudaMalloc's implicit synchronisation, a plugin whose host forbids allocations.  It
 * needs no handle and calls no cudaMalloc, cudaFree or allocating library routine; its
 * scratch (queue counter, cost-order permutation and keys, bucket cursors) lives in one
 * fixed device array of the library, about 6 MiB, that every GPU loading the library holds
 * until the process exits.  The first call on a device looks up that array's device address
 * (once per device): make that first call before any stream capture.  The address is kept for
 * the life of the process, so a caller that destroys the device's context (cudaDeviceReset)
 * must not call this entry point again in that process.  All calls share the array: a call
 * clears what must start at zero, and calls that overlap on the GPU (other streams or host
 * threads) race on it, so order them on one stream.
 * Errors: ENS_EINVAL when N > ENS_NOALLOC_MAX_N; otherwise exactly those of ens_solve (the
 * same argument checks run first). */
#define ENS_NOALLOC_MAX_N 1048576LL
int ens_solve_noalloc(int rhs_id, long long N, const void* params, const void* u0,
                      const void* tspan, const ens_opts* opts, void* out, signed char* status,
                      int* stats, void* cuda_stream);

const char* ens_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ENS_H_ */
