/*
 * varsim.h -- C ABI of the GB300 (sm_103a) Green's-function thermal solver.
 *
 * The library computes the steady and transient temperature rise of a die
 * whose leakage power and silicon conductivity vary across the die and depend
 * on temperature, following the Green's-function method of Sultan & Sarangi
 * ("VarSim", arXiv 2307.12119):
 *   - T = f_sp * P: temperature is the Green's function convolved with the
 *     power map (Sec. II-B, Eq. 2);
 *   - the radially symmetric Green's function is obtained from its Hankel
 *     transform (Sec. II-F, Eq. 8; Appendix, Theorem I);
 *   - die edges are handled by mirror images (Sec. IV-F);
 *   - leakage P = P_dyn + P_leak0 (1 + beta dT) (Eqs. 5, 13) and the
 *     conductivity factor f_sp(T) = f_sp0 (1 + alpha dT) (Eq. 12) are resolved
 *     by iterating power -> temperature -> leakage/conductivity to a stated
 *     tolerance (the convergence loop of Sec. V-C), preconditioned by the
 *     mean/variation split into a shift-invariant and a shift-variant part
 *     (Sec. IV-C, Eqs. 18-26);
 *   - the transient uses a single-pole response per spatial frequency and
 *     superposition of power differences (Sec. IV-D/E, Eqs. 27-37).
 *
 * Conventions for every call:
 *   - Maps are row-major float32 [n][n] (x fastest), one value per grid cell.
 *     Power inputs are watts PER CELL; temperatures are kelvin ABOVE AMBIENT.
 *     Geometry is SI (metres, W/(m K), W/(m^2 K), J/(m^2 K)).
 *   - Map pointers are caller-owned CUDA device memory, contiguous, 16-byte
 *     aligned. The library never frees or retains them past the call (a batch
 *     plan retains them until vs_plan_free, see below).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Work is asynchronous on it unless a call says otherwise.
 *   - Errors are returned as vs_status codes; no call aborts, exits or traps.
 *     vs_last_error() gives a human-readable message for the calling thread.
 *   - Handles (vs_kernel, vs_plan) are library-owned until their free call.
 *     A vs_kernel is read-only after creation and may be shared by calls on
 *     different streams.
 */
#ifndef VARSIM_H
#define VARSIM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VS_OK = 0,
  VS_ERR_INVALID_ARG = 1,    /* bad pointer, size or parameter */
  VS_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  VS_ERR_OOM = 3,            /* device allocation failed */
  VS_ERR_NO_CONVERGENCE = 4, /* residual above tol after max_iter, or growing */
  VS_ERR_RUNAWAY = 5,        /* beta*mu*max(K) >= 1 (thermal runaway) or
                                1 - alpha*s*u <= 0.05 (conductivity model breaks) */
  VS_ERR_NONFINITE = 6,      /* NaN/Inf met in a map */
  VS_ERR_TIMEOUT = 7         /* an internal wait on other CTAs (a grid barrier or
                                an exchange between phases) gave up */
} vs_status;

#define VS_MAX_LAYERS 8
#define VS_MIN_N 8
#define VS_MAX_N 2048

/* Layer stack below the die surface (chip parameter table, Sec. V-A).
 * Layer 0 is the power-dissipating silicon; the temperature is read in its
 * top plane. Layers are in perfect contact; the bottom of the last layer sees
 * a convective coefficient h; the top surface and the side walls are
 * adiabatic. heat_cap_J_m2K is the areal thermal capacitance C of the
 * transient model (Eq. 27); it is only used when a time step is given.
 *
 * Spreader wider than the die (Sec. II-B: the Green's function is a
 * fast-decaying part plus a constant carried by the heat spreader). With
 * spreader_layer = i in [1, n_layers) and spreader_side_m >= the die side,
 * layers i .. n_layers-1 form a square spreader of that side, centred under
 * the die, with its own adiabatic walls. It changes only that constant: the
 * uniform mode of the kernel takes the die layers in series with the
 * spreader's mean impedance over the die footprint (its cosine series, FP64
 * on the GPU); every other mode keeps the die-sized stack. spreader_layer = 0
 * (a zero-initialised struct) or a side equal to the die's is the die-sized
 * stack. Against a finite-volume solve of the actual geometry this reading is
 * within about 1 % of the rise for sources inside the die and about 8 % at
 * its corners (2.5 mm of overhang on a 10 mm die), where the wider spreader
 * draws heat sideways. */
typedef struct {
  int n_layers;                          /* 1 .. VS_MAX_LAYERS */
  double thickness_m[VS_MAX_LAYERS];     /* > 0 */
  double kappa_W_mK[VS_MAX_LAYERS];      /* > 0 */
  double h_conv_W_m2K;                   /* > 0 */
  double heat_cap_J_m2K;                 /* > 0 if dt_s > 0 */
  int spreader_layer;                    /* 0 (die-sized) or 1 .. n_layers-1 */
  double spreader_side_m;                /* >= die side when spreader_layer > 0 */
} vs_stack;

/* Square die of side die_m split into n x n square cells (the paper's grid,
 * Sec. V-A uses 64 x 64). n must be a power of two in [VS_MIN_N, VS_MAX_N]. */
typedef struct {
  int n;
  double die_m;
} vs_grid;

/* Options of the Green's-function build.
 *   quad_nodes: Gauss-Legendre nodes of the Hankel quadrature (0 => 256,
 *               allowed 64..1024);
 *   rel_tol:    truncation tolerance of the real-space radius and of the
 *               spectral alias sum (0 => 1e-13, allowed 1e-16..1e-6);
 *   dt_s:       time step of the transient (0 => no transient tables). */
typedef struct {
  int quad_nodes;
  double rel_tol;
  double dt_s;
} vs_kernel_opts;

#define VS_PREC_FP32 0        /* FP32 fast cosine transforms (SIMT, any n) */
#define VS_PREC_BF16_SPLIT 1  /* cosine transforms as tcgen05 tensor-core GEMMs in
                                 BF16 hi/lo split precision with FP32 accumulation
                                 (x = hi + lo, products hi*hi + hi*lo + lo*hi);
                                 n = 128 .. 1024 (power of two). Two engines:
                                 - n = 256 with cold starts, engine AUTO or
                                   CLUSTER: one CTA pair per map keeps the map on
                                   chip; every transform is two half-size GEMMs
                                   (the even/odd symmetry of the DCT-II), the
                                   start and preconditioner are those of the FP32
                                   engines (the die's uniform mode);
                                 - otherwise (engine STREAMED, other n, warm
                                   starts): a persistent engine that streams the
                                   map through global memory between GEMM passes,
                                   outputs in chunks of 256 columns, b = beta mu,
                                   theta_0 = 0 (or the warm start).
                                 The rounding of the split (~1e-3 K at 30-130 K
                                 rises) suits update tolerances of ~1e-2 K. */

/* Execution engines of the FP32 steady solve (identical arithmetic, different
 * data movement). Both precondition the iteration
 *   u <- K/(1 - b K) * (P_dyn + P_leak0 (1 + beta theta) - b u)
 * (every scalar b has the same fixed point). A cold map (no theta_init)
 * first solves the uniform mode of its die, the scalar fixed point
 *   u_bar = K[0][0] (mean P_dyn + mu (1 + beta theta_bar)),
 *   theta_bar = u_bar / (1 - alpha u_bar),
 * from the means of its inputs; every cell then starts at theta_bar and
 * b = beta mu (1 + 2 alpha u_bar) (about the mean of beta P_leak0 dtheta/du,
 * so the iteration is left with the variation alone). On the 256 x 256 bench
 * maps this takes 3.0 instead of 4.4 iterations at 1e-2 K. A warm start
 * (theta_init given) keeps b = beta mu.
 *   VS_ENGINE_STREAMED: one cooperative launch over all maps of a plan; the
 *     spectral work map streams through global memory between the row and
 *     column phases, phases separated by grid barriers; any n.
 *   VS_ENGINE_CLUSTER: one thread-block cluster of n/32 CTAs per map that
 *     keeps the map in shared memory for the whole solve (transposes through
 *     distributed shared memory, cluster barriers); n in [32, 256]; one launch
 *     per distinct n of a plan.
 *   VS_ENGINE_AUTO: the cluster engine when precision is FP32 and every map
 *     has n in [32, 256], the streamed engine otherwise.
 * The transient solve and vs_solve_steady_noalloc always use the streamed
 * engine; VS_PREC_BF16_SPLIT has its own tensor-core engines (above), where
 * engine CLUSTER asks for the on-chip pair engine. */
#define VS_ENGINE_AUTO 0
#define VS_ENGINE_STREAMED 1
#define VS_ENGINE_CLUSTER 2

#define VS_COND_LINEAR 0      /* theta = s u / (1 - alpha s u) (Eqs. 11-12) */
#define VS_COND_KIRCHHOFF 1   /* kappa = kappa_amb (T / T_amb)^-eta (Eq. 10) through the
                                 Kirchhoff transform: theta = T_amb ((1 + (1 - eta) s u /
                                 T_amb)^(1 / (1 - eta)) - 1) */
#define VS_MAX_LEAK_POINTS 16

/* Stopping rules of the steady fixed point (the paper iterates until the
 * temperatures settle and states no rule).
 *   VS_STOP_UPDATE (0): stop when the update max |theta_n - theta_{n-1}| <= tol_K.
 *   VS_STOP_ESTIMATE (1): stop when an a-posteriori estimate of the error
 *     max |theta_n - theta*| is <= tol_K. For a contraction with factor q the
 *     error of iterate n is at most r_n q / (1 - q), r_n the update; q is
 *     estimated from the last two updates with a safety factor of 4,
 *     q = min(0.9, 4 r_n / r_{n-1}), from the second iteration on (the first
 *     iteration uses the update rule). It stops where the error, not the
 *     update, reaches tol_K: on the 256 x 256 bench maps at 1e-2 K it takes
 *     about 2.1 instead of 3.0 iterations, with errors <= 5e-3 K against the
 *     converged map. */
#define VS_STOP_UPDATE 0
#define VS_STOP_ESTIMATE 1

/* Parameters of a solve.
 *   beta_per_K : temperature coefficient of leakage (Eq. 5), >= 0
 *   alpha_per_K: temperature coefficient of the Green's function (Eq. 12), >= 0
 *   tol_K      : stop when max |theta_n - theta_{n-1}| <= tol_K (> 0), or by
 *                the stopping rule stop_rule
 *   max_iter   : 1 .. 1000
 *   precision  : VS_PREC_FP32 or VS_PREC_BF16_SPLIT
 *   engine     : VS_ENGINE_AUTO (0, what a zero-initialised struct selects),
 *                VS_ENGINE_STREAMED or VS_ENGINE_CLUSTER; asking for the
 *                cluster engine where it does not apply is VS_ERR_INVALID_ARG
 * Physics variants (zero-initialised = the linear models above):
 *   conductivity: VS_COND_LINEAR, or VS_COND_KIRCHHOFF with eta (> 0, != 1)
 *                 and t_amb_K (> 0); alpha_per_K is then unused
 *   leak_points : 0 => P_leak = P_leak0 (1 + beta theta); 2 .. 16 =>
 *                 P_leak = P_leak0 g(theta), g piecewise linear through
 *                 (leak_theta_K[i], leak_g[i]) (theta strictly increasing, g
 *                 finite), the end segments extended (Sec. II-E). The
 *                 iteration then preconditions with the table's slope at
 *                 theta = 0 instead of beta_per_K (the fixed point is the
 *                 same); that slope also enters the runaway check.
 * A variant needs FP32 and a steady solve: the cluster engine (one launch
 * shape, update-load batch 2; a cold map starts from theta_0 = 0) or the
 * streamed engine, VS_ENGINE_AUTO choosing as for the linear models; the
 * tensor-core engines, the transient and vs_solve_steady_noalloc return
 * VS_ERR_INVALID_ARG for it.
 *   stop_rule  : VS_STOP_UPDATE (0, what a zero-initialised struct selects) or
 *                VS_STOP_ESTIMATE, on every steady engine and for the per-step
 *                fixed point of a transient with implicit leakage (a lagged
 *                transient has no fixed point and ignores it). */
typedef struct {
  double beta_per_K;
  double alpha_per_K;
  double tol_K;
  int max_iter;
  int precision;
  int engine;
  int conductivity;
  double eta;
  double t_amb_K;
  int leak_points;
  double leak_theta_K[VS_MAX_LEAK_POINTS];
  double leak_g[VS_MAX_LEAK_POINTS];
  int stop_rule;
} vs_solve_params;

/* Per-map outcome. status is a vs_status; iterations counts the applications
 * of the convolution, each followed by the update and the convergence check
 * (0 for a map stopped before its first, e.g. a runaway at the start);
 * residual_K is the last max |theta_n - theta_{n-1}| (theta_0 is the start:
 * 0, the warm start's map, or the die's uniform-mode temperature); mu_W is the
 * mean of P_leak0 (W per cell); fell_back is 1 for a map of a warm-started
 * solve that did not converge from the network's start and was solved again
 * cold (vs_warm_plan_info with fallback), else 0. */
typedef struct {
  int status;
  int iterations;
  double residual_K;
  double mu_W;
  int fell_back;
} vs_solve_info;

typedef struct vs_kernel_t* vs_kernel;
typedef struct vs_plan_t* vs_plan;
typedef struct vs_model_t* vs_model;

/* ------------------------------------------------------------------------ */
/* Green's function build (Sec. II-B, Eq. 2; Sec. II-F Eq. 8; Theorem I;    */
/* images Sec. IV-F).                                                       */
/* ------------------------------------------------------------------------ */

/* Builds the imaged, cell-averaged Green's function of (stack, grid) in the
 * cosine basis of the die, K[p][q], p,q in [0,n), on the GPU:
 *   1. stack spectrum g(k) (impedance recursion of the heat equation, Eq. 1);
 *   2. Hankel quadrature (Eq. 8, Theorem I normalisation) of the top-layer
 *      (fast-decaying part, Sec. II-B) Green's function at every lattice
 *      radius, FP64: G1(r) = halfspace_disc(r) - sum_i w_i J0(k_i r);
 *   3. fold of the lattice into the 2n-periodic mirror-imaged kernel and its
 *      cosine transform;
 *   4. spectral (Poisson) sum of the remaining smooth spreader part.
 * If opts->dt_s > 0 the per-mode decay factors of the transient are built too.
 * Synchronises `stream` before returning. *out is NULL on failure.
 * Errors: VS_ERR_INVALID_ARG (sizes, non-positive physics), VS_ERR_OOM,
 * VS_ERR_CUDA. */
int vs_make_kernel(const vs_stack* stack, const vs_grid* grid,
                   const vs_kernel_opts* opts, vs_kernel* out, void* stream);

void vs_free_kernel(vs_kernel k);

/* Grid side n of a kernel, or -1 for NULL. */
int vs_kernel_n(vs_kernel k);

/* Copies the FP64 cosine-basis kernel K[p][q] (n*n doubles, row p) to host
 * memory `out_host`. Blocking. Errors: VS_ERR_INVALID_ARG, VS_ERR_CUDA. */
int vs_kernel_spectrum(vs_kernel k, double* out_host);

/* Copies the top-layer radial Green's function table G1(cell*sqrt(m)) for
 * m = 0..m_max to `out_host` (entries for m that are not a sum of two squares
 * are 0). m_max is written to *m_max_out; pass out_host = NULL to query it.
 * Blocking. */
int vs_kernel_radial(vs_kernel k, double* out_host, int* m_max_out);

/* Evaluates the Hankel quadrature of step 2 above for arbitrary radii:
 * out_dev[i] = G1(r_dev[i]) in K/W for the top layer of `stack` with the
 * source disc of one cell of `grid`. r_dev, out_dev: device float64 arrays of
 * length count. quad_nodes as in vs_kernel_opts. Asynchronous on `stream`. */
int vs_hankel_radial(const vs_stack* stack, const vs_grid* grid, int quad_nodes,
                     const double* r_dev, double* out_dev, int count, void* stream);

/* ------------------------------------------------------------------------ */
/* Steady solve (Eqs. 13-26; convergence loop of Sec. V-C).                 */
/* ------------------------------------------------------------------------ */

/* Solves u = L[P_dyn + P_leak0 (1 + beta theta)], theta = s u / (1 - alpha s u)
 * for one map, where L is the convolution with the imaged Green's function.
 * Iterates the mean/variation split (shift-invariant kernel
 * K/(1 - beta mu K), Eq. 21 with alpha = 0) until max |dtheta| <= tol.
 *   p_dyn, p_leak0: W per cell; s_kappa: conductivity multiplier (NULL => 1);
 *   theta: output, K above ambient.
 * info_host (may be NULL) is filled after an internal stream synchronisation.
 * Returns the map's status (VS_OK, VS_ERR_NO_CONVERGENCE, VS_ERR_RUNAWAY,
 * VS_ERR_NONFINITE) or an argument/CUDA error. */
int vs_solve_steady(vs_kernel k, const float* p_dyn, const float* p_leak0,
                    const float* s_kappa, const vs_solve_params* params,
                    float* theta, vs_solve_info* info_host, void* stream);

/* Allocation-free variant of vs_solve_steady. The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory
 * while solving -- e.g. services that reserve their device-memory budget up
 * front, or latency-critical loops where cudaMalloc/cudaFree (which can
 * synchronise the device) are not allowed. It makes no cudaMalloc, cudaFree
 * or other allocating call; its scratch lives in a fixed, file-scope device
 * array of about 1.02 MiB that every GPU loading the library holds until the
 * process exits.
 *   Limit: n <= 512 (the work map of a 512 x 512 grid fills the array);
 *          larger grids return VS_ERR_INVALID_ARG with a message.
 *   Arguments, layout, outputs and statuses are those of vs_solve_steady,
 *   except that it always runs the FP32 streamed engine: params->precision
 *   other than VS_PREC_FP32, or params->engine = VS_ENGINE_CLUSTER, return
 *   VS_ERR_INVALID_ARG.
 *   The first call on each device resolves the array's device address
 *   (cudaGetSymbolAddress) and keeps it for the life of the process; make
 *   that first call outside any stream capture. The address belongs to the
 *   device's primary context: after cudaDeviceReset the module may load
 *   elsewhere, so do not call this entry point again in that process.
 *   Every call re-initialises the parts of the array that must start at zero,
 *   but all calls share the one array: calls whose GPU work overlaps (different
 *   streams or host threads without ordering) race and corrupt each other.
 *   Synchronises `stream` before returning. */
int vs_solve_steady_noalloc(vs_kernel k, const float* p_dyn, const float* p_leak0,
                            const float* s_kappa, const vs_solve_params* params,
                            float* theta, vs_solve_info* info_host, void* stream);

/* ------------------------------------------------------------------------ */
/* Batched steady solve: many maps (possibly of different grid sizes), one  */
/* launch per run (cluster engine: one per distinct grid size).             */
/* ------------------------------------------------------------------------ */

typedef struct {
  vs_kernel k;             /* Green's function of this map's geometry */
  const float* p_dyn;      /* device, [n][n] */
  const float* p_leak0;    /* device, [n][n] */
  const float* s_kappa;    /* device, [n][n], or NULL => 1 */
  float* theta;            /* device output, [n][n] */
  const float* theta_init; /* device [n][n] initial temperature (warm start of the
                              fixed point, e.g. from vs_warm_apply), or NULL: the
                              FP32 engines then start from the die's uniform-mode
                              temperature, the tensor-core engine from 0 */
} vs_batch_item;

/* Creates a plan for n_items maps: uploads the item table and picks the
 * engine (params->engine). Streamed engine: allocates the scratch (4 bytes per
 * cell plus small per-map state) and picks the launch shape (tuned once per
 * mix of grid sizes and cached). Cluster engine: no spectral scratch, maps
 * grouped by grid size. The item pointers are retained until vs_plan_free.
 * Synchronises `stream`. */
int vs_plan_create(const vs_batch_item* items_host, int n_items,
                   const vs_solve_params* params, vs_plan* out, void* stream);

/* Launch-shape autotuner (the paper has no counterpart). A plan's shape is
 * one integer: on the cluster engine the update-load batch (1, 2 or 4
 * positions whose inputs a thread loads before using them: the depth of the
 * global-load pipelining), on the streamed engine the task size (2048, 4096,
 * 8192 or 16384 elements of a map per row or column task). vs_plan_create
 * tunes plans of at least 64 maps: it times every candidate on the plan itself
 * (a warm-up and two timed runs each, CUDA events on `stream`; the runs write
 * the plan's theta) and keeps the fastest. The choice is cached for the
 * process per engine, mix of grid sizes and power-of-two batch bucket, so
 * later plans of the same kind reuse it untimed. VS_AUTOTUNE=0 in the
 * environment keeps the defaults (batch 2, 8192 elements). The shape changes
 * data movement only: on the cluster engine every shape gives bit-identical
 * maps. vs_plan_create_shaped forces a shape (0 = as vs_plan_create);
 * VS_ERR_INVALID_ARG for a shape the engine does not have. */
int vs_plan_create_shaped(const vs_batch_item* items_host, int n_items,
                          const vs_solve_params* params, int shape, vs_plan* out, void* stream);
/* The plan's shape, and the candidates its creation timed: *n_timed of them
 * (0 when forced, cached or not tuned), their shapes and times in ms (arrays
 * of at least 4, may be NULL). */
int vs_plan_shape(vs_plan plan, int* shape_out, int* n_timed, int* cand_shapes, double* cand_ms);

/* Runs the plan: one launch (streamed engine: cooperative and persistent;
 * cluster engine: one per distinct grid size, a cluster per map) that
 * iterates every map to its own convergence. Asynchronous; makes no host
 * allocation or synchronisation, so it can be captured in a CUDA graph.
 * Per-map results go to the plan's device info array (vs_plan_info). A plan
 * owns its scratch: runs of one plan must be ordered (e.g. on one stream);
 * different plans, and kernels shared between them, may run concurrently. */
int vs_plan_run(vs_plan plan, void* stream);

/* Copies the per-map vs_solve_info of the last run to host memory
 * (n_items entries) after synchronising `stream`. Returns the worst status. */
int vs_plan_info(vs_plan plan, vs_solve_info* info_host, void* stream);

/* Number of kernel launches one vs_plan_run makes (for launch accounting). */
int vs_plan_launches(vs_plan plan);

void vs_plan_free(vs_plan plan);

/* Convenience: create + run + info + free. info_host may be NULL.
 * Returns the worst per-map status. */
int vs_solve_batch(const vs_batch_item* items_host, int n_items,
                   const vs_solve_params* params, vs_solve_info* info_host,
                   void* stream);

/* Batched steady solve from and to HOST memory (the paper has no counterpart;
 * the solve itself is that of vs_solve_batch, Eqs. 13-26). count maps of
 * grid k->n: p_dyn, p_leak0, s_kappa (NULL => 1) and theta are host arrays
 * [count][n][n]. The maps go through the GPU in chunks of chunk_maps maps
 * (0 => a sixteenth of the batch, at most about 1 GiB of device buffers per
 * chunk): the host-to-device copies of
 * the next chunk and the device-to-host copy of the previous one overlap the
 * solve of the current one (internal streams and events, two device buffer
 * slots). The overlap needs page-locked host memory (cudaHostAlloc, or
 * torch's pin_memory); pageable arrays work but serialise the copies. Every
 * map gets exactly the result vs_solve_batch gives it. Ordered after work
 * already queued on `stream`; returns when theta (and info_host, count entries,
 * if not NULL) are complete in host memory. Allocates its device buffers per
 * call (a vs_host_plan, below, keeps them). Returns the worst per-map status. */
int vs_solve_batch_host(vs_kernel k, int count, const float* p_dyn, const float* p_leak0,
                        const float* s_kappa, float* theta, const vs_solve_params* params,
                        vs_solve_info* info_host, int chunk_maps, void* stream);

/* The same as a reusable object: vs_host_plan_create allocates the internal
 * streams, the two device buffer slots (4 arrays of chunk maps each, 3 without
 * s), pinned staging for the per-map outcomes and the plans of the chunks, for
 * `count` maps of grid k->n with (with_s = 1) or without (0) a conductivity
 * field; chunk_maps as above. The chunk plans take the launch shape the
 * autotuner cached for their kind, else the default, without timing runs
 * (their buffers hold no maps yet). The kernel must outlive the host plan.
 * vs_host_plan_run then solves one batch of host arrays exactly as
 * vs_solve_batch_host does (same ordering on `stream`, same return), with no
 * allocation; s_kappa must be non-NULL exactly when with_s = 1
 * (VS_ERR_INVALID_ARG otherwise). Runs of one host plan must not overlap.
 * vs_host_plan_free releases everything (NULL is a no-op). */
typedef struct vs_host_plan_t* vs_host_plan;
int vs_host_plan_create(vs_kernel k, int count, int with_s, const vs_solve_params* params,
                        int chunk_maps, vs_host_plan* out);
int vs_host_plan_run(vs_host_plan plan, const float* p_dyn, const float* p_leak0,
                     const float* s_kappa, float* theta, vs_solve_info* info_host, void* stream);
void vs_host_plan_free(vs_host_plan plan);

/* ------------------------------------------------------------------------ */
/* Transient (Sec. IV-D/E, Eqs. 27-37).                                     */
/* ------------------------------------------------------------------------ */

/* Time-varying power P_dyn,n (n = 1..n_steps, piecewise constant over steps
 * of dt_s given at kernel build) with leakage lagged one step,
 * P_n = P_dyn,n + P_leak0 (1 + beta theta_{n-1}), theta_0 = 0.
 * Superposition of power differences (Eq. 36) with the single-pole step
 * response g(k)(1 - exp(-t / (C g(k)))) of every cosine mode (Eq. 35), run as
 * the equivalent per-mode recursion. The sub-cell alias part of the kernel is
 * taken as settled within one step.
 *   p_dyn_trace: [n_steps][n][n]; theta_trace: output [n_steps][n][n].
 * info_host (may be NULL) filled after synchronisation; iterations = steps. */
int vs_solve_transient(vs_kernel k, int n_steps, const float* p_dyn_trace,
                       const float* p_leak0, const float* s_kappa,
                       const vs_solve_params* params, float* theta_trace,
                       vs_solve_info* info_host, void* stream);

/* Variants of the transient (Sec. IV-E).
 *   window : 0 => untruncated superposition (as vs_solve_transient). K >= 1 =>
 *            the step response of every power difference of age >= K steps is
 *            taken as settled, S_j = S_inf = K~ for j >= K, which telescopes to
 *            u_n = sum_{j<K} S_j * (P_{n-j+1} - P_{n-j}) + K~ * P_{n-K+1}
 *            (the paper uses K = 5 steps of 1 ms); at most VS_MAX_WINDOW.
 *   leakage: VS_LEAK_LAGGED (P_n uses theta_{n-1}) or VS_LEAK_IMPLICIT: every
 *            step iterates theta_n <- phi(u_n(P_dyn,n + P_leak0 (1 + beta
 *            theta_n))) from theta_{n-1} until max |change| <= tol_K or
 *            max_iter iterations (the history then holds the source of the
 *            last iteration). */
#define VS_LEAK_LAGGED 0
#define VS_LEAK_IMPLICIT 1
#define VS_MAX_WINDOW 256
typedef struct {
  int window;
  int leakage;
} vs_transient_opts;

/* vs_solve_transient with options (opts NULL => window 0, lagged leakage).
 * n = 256, 512, 1024 without the combination of a window with implicit
 * leakage run on one persistent launch (a CTA per 2-8 rows; the phases
 * exchange tagged words with lagged leakage and meet at grid barriers with
 * implicit leakage); the rest on the general streamed engine. Device state on
 * the persistent launch: (2 + max(0, window - 1)) * n * n floats. info_host:
 * lagged, iterations = steps; implicit, iterations = fixed-point iterations
 * summed over the steps, residual_K = the largest final change of a step, and
 * status VS_ERR_NO_CONVERGENCE if a step reached max_iter without meeting the
 * stopping rule (stop_rule of vs_solve_params). */
int vs_solve_transient_ex(vs_kernel k, int n_steps, const float* p_dyn_trace,
                          const float* p_leak0, const float* s_kappa,
                          const vs_solve_params* params, const vs_transient_opts* opts,
                          float* theta_trace, vs_solve_info* info_host, void* stream);

/* ------------------------------------------------------------------------ */
/* One-shot closed form (Sec. IV-C: Eqs. 21, 25, 26), the paper's own       */
/* alternative to iterating the fixed point.                                */
/* ------------------------------------------------------------------------ */

/* For `count` maps of one kernel ([count][n][n] device float32, 16-byte
 * aligned; s_kappa may be NULL => 1):
 *   u = L_det * (P_dyn + P_leak0) + (P_leak0 - mu) . r,  theta = phi(u),
 *   L_det = K~ / (1 - beta mu K~)  (Eq. 21 without its alpha term, which the
 *   paper derives through Lemma I; alpha acts through phi as in the solve),
 *   r = beta L_det^2 * (P_dyn + P_leak0)            (VS_CF_CONV: Eq. 25 to
 *       first order in the variation, applied to the power map), or
 *   r = (beta L_det^2 * impulse at cell (n/2, n/2)) sum(P_dyn + P_leak0)
 *                                                   (VS_CF_IMPULSE: Eq. 26's
 *       total-power scaling of the impulse response, literally),
 * with * the mirror-image convolution and . the Hadamard product. No
 * iteration: the result differs from the fixed point of vs_solve_steady by
 * the approximation. n = 32 .. 256: one launch, a thread-block cluster per
 * map (the cluster engine's layout), plus a small descriptor table from the
 * stream-ordered allocator; other n: four kernel launches and scratch of
 * 8 bytes per cell from the stream-ordered allocator. The two forms compute
 * the same (to rounding). info_host (may be NULL => no synchronisation)
 * gets status VS_OK, VS_ERR_RUNAWAY or VS_ERR_NONFINITE per map,
 * iterations 0, residual_K 0 and mu_W. */
#define VS_CF_CONV 0
#define VS_CF_IMPULSE 1
int vs_solve_closed_form(vs_kernel k, int count, const float* p_dyn, const float* p_leak0,
                         const float* s_kappa, const vs_solve_params* params, int mode,
                         float* theta, vs_solve_info* info_host, void* stream);

/* ------------------------------------------------------------------------ */
/* Learned warm start of the fixed point. The paper iterates power ->       */
/* temperature -> leakage until convergence (Sec. V-C); these calls predict */
/* most of the remaining correction after the first iterate so that the     */
/* iteration can start closer to its fixed point. The solve still decides   */
/* convergence, so a poor prediction costs iterations, not accuracy.        */
/* ------------------------------------------------------------------------ */

/* Small U-Net on resolution x resolution inputs (3 channels -> 1): convs
 * 3->C, C->C, pool, C->2C, 2C->2C, pool, 2C->2C, up + skip -> C, up + skip -> C,
 * C->1 (3x3, zero padding, ReLU except the last). BF16 weights, FP32
 * activations and accumulation; He-uniform initialisation from `seed`.
 * base_channels C in [1, 64]; resolution a multiple of 4 in [8, 256].
 * Parameters are laid out as all weights [co][ci][3][3] layer by layer, then
 * all biases. */
int vs_model_create(int base_channels, int resolution, unsigned long long seed, vs_model* out);
void vs_free_model(vs_model m);
long long vs_model_nparams(vs_model m);
/* Host FP32 copies of the master parameters (n = vs_model_nparams). Setting
 * them also resets the optimiser state. Blocking. */
int vs_model_get_params(vs_model m, float* host);
int vs_model_set_params(vs_model m, const float* host);
/* y[b][0][R][R] = net(x[b][3][R][R]) for `batch` samples (device arrays).
 * The model's forward, gradient and training calls (and the warm plans that
 * hold it) share its activation buffers: calls on one model must be ordered,
 * e.g. on one stream; different models are independent. */
int vs_model_forward(vs_model m, const float* x, float* y, int batch, void* stream);
/* The same forward with the convolutions as tcgen05 implicit GEMMs (BF16
 * activations and weights, FP32 accumulation) wherever a layer's shape fits
 * (its image a multiple of 128 pixels, padded weights <= 64 KB), the SIMT
 * kernels elsewhere. Within BF16 rounding of vs_model_forward; the warm plan's
 * prediction stage runs it. */
int vs_model_forward_tc(vs_model m, const float* x, float* y, int batch, void* stream);
/* Mean-squared-error loss against t[b][1][R][R] and its parameter gradient
 * (host arrays; grad_host may be NULL). No update. Blocking. */
int vs_model_loss_grad(vs_model m, const float* x, const float* t, int batch,
                       double* loss_host, float* grad_host, void* stream);
/* Adam training (lr, beta1 0.9, beta2 0.999) on n_samples pairs (x, t) in
 * device memory for `epochs` shuffled passes of `batch`; *loss_host = MSE of
 * the last batch. Blocking. */
int vs_model_train(vs_model m, const float* x, const float* t, int n_samples, int epochs,
                   int batch, float lr, unsigned long long seed, double* loss_host, void* stream);
/* Checkpoint (base channels, resolution, parameters) to / from a file. */
int vs_model_save(vs_model m, const char* path);
int vs_model_load(const char* path, vs_model* out);
/* Base channel count C and input resolution R of a model (e.g. one loaded
 * from a checkpoint). */
int vs_model_shape(vs_model m, int* base_channels, int* resolution);

/* Features of `count` maps [count][n][n] for the warm start, averaged over
 * (n/R)^2 blocks: x[b] = {theta1/100, 10 (P_leak0/mean - 1), 30 (s - 1)}
 * ([count][3][R][R]); s_kappa may be NULL. */
int vs_warm_features(const float* theta1, const float* p_leak0, const float* s_kappa,
                     int count, int n, int resolution, float* x_out, void* stream);
/* Training target t[b] = block average of (theta_star - theta1) / 10. */
int vs_warm_target(const float* theta_star, const float* theta1, int count, int n,
                   int resolution, float* t_out, void* stream);
/* theta_init = theta1 + 10 * bilinear upsampling of y to n x n. */
int vs_warm_apply(const float* theta1, const float* y, int count, int n, int resolution,
                  float* theta_init, void* stream);

/* Warm-started batched solve of `count` maps of one kernel's grid, in three
 * stages that a run can take together or apart (bit mask `stages`):
 *   VS_WARM_FIRST   one fixed-point iteration from theta_0 = 0 -> theta1;
 *   VS_WARM_PREDICT features of theta1, network, theta_init = theta1 +
 *                   predicted correction (vs_warm_features, vs_model_forward,
 *                   vs_warm_apply);
 *   VS_WARM_SOLVE   the batched solve (vs_plan_run) from theta_init -> theta.
 * p_dyn, p_leak0, s_kappa (NULL => 1), theta, theta1, theta_init: device
 * float32 [count][n][n], caller-owned, retained until vs_warm_plan_free;
 * theta1 and theta_init may be written by the caller between stages (e.g. to
 * run the solve from another start). The model's resolution must divide n.
 * The plan owns the network's input and output buffers and both solve plans.
 * A run is asynchronous and allocation-free (graph-capturable). Synchronises
 * `stream` on create. */
#define VS_WARM_FIRST 1
#define VS_WARM_PREDICT 2
#define VS_WARM_SOLVE 4
#define VS_WARM_ALL 7
typedef struct vs_warm_plan_t* vs_warm_plan;
int vs_warm_plan_create(vs_kernel k, int count, const float* p_dyn, const float* p_leak0,
                        const float* s_kappa, float* theta, float* theta1, float* theta_init,
                        vs_model model, const vs_solve_params* params, vs_warm_plan* out,
                        void* stream);
int vs_warm_plan_run(vs_warm_plan plan, int stages, void* stream);
/* Kernel launches of one full run (VS_WARM_ALL). */
int vs_warm_plan_launches(vs_warm_plan plan);
/* Per-map outcome of the last solve stage into info_host[count] (blocking).
 * With `fallback` != 0, the maps whose status is not VS_OK are solved again
 * from theta_0 = 0 (vs_solve_batch) and their entries replaced, with
 * fell_back = 1; fell_back_host (may be NULL) gets the same flags. Returns the
 * worst per-map status, or the launch-level error. */
int vs_warm_plan_info(vs_warm_plan plan, vs_solve_info* info_host, int fallback,
                      int* fell_back_host, void* stream);
void vs_warm_plan_free(vs_warm_plan plan);

/* Split-precision tensor-core transform (the building block of
 * VS_PREC_BF16_SPLIT), exposed for testing: for each of `rows` rows,
 *   out[r][j] = sum_k in[r][k] C[j][k],  C[j][k] = cos(pi j (2k+1) / 2n)
 * (forward DCT-II of Sec. IV-F's mirror-imaged rows) or, with inverse != 0,
 *   out[r][j] = sum_k in[r][k] w_k cos(pi k (2j+1) / 2n) / n, w_0 = 1, w_k = 2
 * (its exact inverse). in/out: device float32 [rows][n], rows a multiple of
 * 128, n a power of two in [128, 1024], 16-byte aligned. Asynchronous on
 * `stream`. */
int vs_tc_transform(const float* in, float* out, int rows, int n, int inverse, void* stream);

/* ------------------------------------------------------------------------ */

const char* vs_status_string(int status);
const char* vs_last_error(void);      /* thread-local, never NULL */
const char* vs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* VARSIM_H */
