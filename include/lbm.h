/*
 * lbm.h -- C ABI of the GB300 (sm_103a) Ehrenfest-regularised lattice
 * Boltzmann library (liblbm.so).
 *
 * Method: Brownlee, Gorban, Levesley, "Stable simulation of fluid flow with
 * high-Reynolds number using Ehrenfests' steps" (2007).  One time step is
 *   free flight (Sec. 3, exact shift on the lattice, Sec. 3.2) with the
 *   boundary rules of Sec. 4.2, moments M = m(f) (Sec. 2), quasiequilibrium
 *   f*_M (Sec. 4.1 / Sec. 4.2 / (argmax)), nonequilibrium entropy
 *   dS = sum_i f_i ln(f_i / f*_i) ((DelS), Sec. 3.3), the LBGK step
 *   f + 2 beta (f* - f) ((lbgkLB)), and the Ehrenfests' step f <- f* at the
 *   k sites with the largest dS > delta (all of them if fewer qualify)
 *   (Sec. 3.2 last paragraph; (ESLB)).
 *
 * Conventions for every entry point:
 *   - All functions are extern "C", never throw, and return an int status:
 *     LB_OK (0) or a negative LB_ERR_* code; lb_last_error() then gives a
 *     thread-local message.  Invalid arguments are rejected before any work
 *     is queued (LB_ERR_ARG).
 *   - Population arrays exchanged with the caller are FP64, laid out
 *     [Q][ny][nx] (population plane, row, x fastest), populations in the
 *     paper's numbering: D1Q3 {rest, left, right} = {0, -1, +1} (Sec. 4.1);
 *     D2Q9 0 rest, 1..4 E N W S, 5..8 NE NW SW SE (Sec. 4.2).
 *   - Field arrays (rho, u_x, u_y, 2E, dS) are FP64 [ny][nx]; site index
 *     = y * nx + x.  Solid (obstacle) sites hold no populations: they read
 *     back as 0 (dS: NaN) and are never selected.
 *   - Unless a function says otherwise, pointers are HOST pointers owned by
 *     the caller and only read / written during the call.  The library owns
 *     all device memory it allocates (cudaMalloc in lb_create) and frees it
 *     in lb_destroy.
 *   - Work is queued on the stream given to lb_create (NULL: the library
 *     creates its own non-blocking stream).  Calls that return data to host
 *     memory synchronise that stream.  One handle must not be used from two
 *     threads at once.
 *   - Exactly one GPU: the device current at lb_create.
 */
#ifndef LBM_H
#define LBM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_handle lb_handle;

/* Lattices: Sec. 4.1 (D1Q3, velocities {0, -1, +1}) and Sec. 4.2 (D2Q9). */
enum lb_lattice { LB_D1Q3 = 0, LB_D2Q9 = 1 };

/* Quasiequilibria:
 *   LB_EQ_POLY      polynomial (Sec. 4.1 formulas; D2Q9 the standard
 *                   second-order form W_i rho (1 + 3 v.u + 9/2 (v.u)^2 - 3/2 u^2));
 *   LB_EQ_ENTROPIC  entropic for mass and momentum (Sec. 4.1 closed form,
 *                   Sec. 4.2 product formula);
 *   LB_EQ_ENTROPIC_ENERGY      entropic with the energy constraint as well,
 *                   M = (rho, rho u1, rho u2, 2E) ((argmax), Lagrange form of
 *                   Sec. 3.3), solved per site by Newton from the polynomial
 *                   start point (FP32 iterations, then finishing steps to a
 *                   residual of 1e-12 with the residual in float-float for
 *                   FP32 / FP16 storage, in FP64 for FP64 storage);
 *   LB_EQ_ENTROPIC_ENERGY_MLP  as above, Newton warm-started by the 4-64-64-4
 *                   network loaded with lb_set_mlp (BF16 tensor cores). */
enum lb_equilibrium {
    LB_EQ_POLY = 0,
    LB_EQ_ENTROPIC = 1,
    LB_EQ_ENTROPIC_ENERGY = 2,
    LB_EQ_ENTROPIC_ENERGY_MLP = 3
};

/* Storage of the populations in device memory (the arithmetic type is FP64
 * for LB_F64 and FP32 otherwise):
 *   LB_F64      f in FP64;  LB_F32  f in FP32;
 *   LB_F32_DEV  g = f - W_i rho0 (rho0 = 1) in FP32;
 *   LB_F16_DEV  g = f - W_i rho0 in FP16.
 * The deviation forms collide in deviation variables and recompute dS in
 * FP64 for sites whose FP32 dS lies within a relative 1e-3 of delta. */
enum lb_precision { LB_F64 = 0, LB_F32 = 1, LB_F32_DEV = 2, LB_F16_DEV = 3 };

/* Boundary kinds of the four sides (Sec. 4.2 boundary paragraph):
 *   LB_BB         half-way bounce-back (no-slip);
 *   LB_FREESLIP   specular reflection (y sides only);
 *   LB_INLET_EQ   incoming populations = quasiequilibrium of (rho_in, u_in)
 *                 (x sides only);
 *   LB_OUTLET_EQ  incoming populations = quasiequilibrium of the density and
 *                 velocity of the penultimate column (x sides only; the
 *                 outlet rule of Sec. 4.2);
 *   LB_PERIODIC   wrap-around (both sides of an axis);
 *   LB_OUTLET_COPY zero-gradient outflow: an incoming population arrives as
 *                 if the column beyond the side were a copy of the side
 *                 column (it is taken from the side column itself, row
 *                 y - v_y, or y where that leaves the lattice; x sides only).
 *                 Not in the paper: its equilibrium outlet feeds back the
 *                 reverse flow of vortices leaving the channel.
 * The obstacle is a solid rectangle [x0, x0+w) x [y0, y0+h) (w = 0: none);
 * it must keep at least one fluid site to the y walls and two columns to an
 * outlet.  obstacle_wall selects the rule on its faces (the paper leaves it
 * open, pointing to kinetic boundary conditions, Sec. 4.2):
 *   LB_WALL_BOUNCE_BACK  half-way bounce-back, f_i(x) = f'_{-i}(x) (no-slip);
 *   LB_WALL_DIFFUSE      diffuse kinetic wall at rest (Maxwell's diffuse
 *                        reflection): the populations entering x from the
 *                        obstacle are W_i rho_w, rho_w such that they carry
 *                        exactly the mass f'_{-i}(x) that x sent into it,
 *                        f_i = W_i sum_B f'_{-j} / sum_B W_j over the set B
 *                        of x's links into the obstacle.
 * A zero-initialised struct selects bounce-back.  Any other value: LB_ERR_ARG. */
enum lb_bc { LB_BB = 0, LB_FREESLIP = 1, LB_INLET_EQ = 2, LB_OUTLET_EQ = 3, LB_PERIODIC = 4,
             LB_OUTLET_COPY = 5 };
enum lb_wall { LB_WALL_BOUNCE_BACK = 0, LB_WALL_DIFFUSE = 1 };

typedef struct lb_boundaries {
    int kind_x0, kind_x1, kind_y0, kind_y1;
    double rho_in;
    double u_in[2];
    int obstacle_x0, obstacle_y0, obstacle_w, obstacle_h;
    int obstacle_wall;          /* lb_wall */
} lb_boundaries;

/* Status codes. */
#define LB_OK 0
#define LB_ERR_ARG (-1)         /* invalid argument; nothing was queued */
#define LB_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define LB_ERR_NONFINITE (-3)   /* a non-finite moment appeared (sticky) */
#define LB_ERR_NEWTON (-4)      /* a Newton solve missed 1e-12 (sticky) */
#define LB_ERR_TIMEOUT (-5)     /* a bounded device wait gave up (sticky) */
#define LB_ERR_OOM (-6)         /* device allocation failed */
#define LB_ERR_STATE (-7)       /* call not valid in the handle's state */

/* Create a run.  lattice: lb_lattice; nx, ny: grid (ny = 1 for D1Q3;
 * nx >= 3, ny >= 3 for D2Q9); equilibrium: lb_equilibrium; nu > 0: kinematic
 * viscosity, giving the LBGK parameter beta = 1 / (1 + 6 nu) (the paper
 * writes omega = 2 beta in (lbgkLB) and leaves nu(beta) to the standard
 * relation nu = (1/omega - 1/2)/3); delta: Ehrenfests' tolerance (any real;
 * dS > delta is strict); k >= 0: Ehrenfests' sites per step (0 turns the
 * regulariser off); bc: boundaries (NULL: bounce-back on every side, no
 * obstacle); precision: lb_precision; cuda_stream: a cudaStream_t or NULL.
 * The populations start at zero; call lb_init_equilibrium or lb_set_state.
 * On success *out receives the handle. */
int lb_create(int lattice, int nx, int ny, int equilibrium, double nu, double delta, int k,
              const lb_boundaries* bc, int precision, void* cuda_stream, lb_handle** out);

/* Free the handle and all its device memory.  NULL is a no-op. */
void lb_destroy(lb_handle* h);

/* Set the state to the quasiequilibrium of the given fields (Sec. 4.1 and
 * Sec. 4.2 both start on the quasiequilibrium manifold).  rho, ux: host
 * [ny][nx]; uy: host [ny][nx] or NULL (D1Q3 / zero); e2: host [ny][nx] or
 * NULL, the energy 2E for LB_EQ_ENTROPIC_ENERGY* (NULL: isothermal). */
int lb_init_equilibrium(lb_handle* h, const double* rho, const double* ux, const double* uy,
                        const double* e2);

/* Pre-collision populations of the current time step, host [Q][ny][nx]
 * FP64 (checkpoint).  lb_set_state loads them back (resume); a step after
 * lb_set_state continues exactly as the run that was saved. */
int lb_get_state(lb_handle* h, double* f);
int lb_set_state(lb_handle* h, const double* f);

/* Advance n >= 0 time steps.  Asynchronous: work is queued on the stream
 * and the call returns the sticky status of work already completed. */
int lb_step(lb_handle* h, int n);

/* Wait for all queued work (steps and asynchronous transfers); return the
 * sticky status. */
int lb_sync(lb_handle* h);

/* Moments of the current pre-collision state: rho, u_x, u_y and 2E (each
 * [ny][nx] FP64; uy and e2 may be NULL).  on_device != 0: the pointers are
 * device pointers and the call does not synchronise. */
int lb_moments(lb_handle* h, double* rho, double* ux, double* uy, double* e2, int on_device);

/* Asynchronous forms of lb_set_state and of lb_moments with host arrays:
 * the call queues the transfer and returns.  The uploaded state replaces
 * the run's after the work already queued (its copies may start earlier);
 * the moments are those of the state after the work already queued.  f must
 * stay unchanged, and rho, ux, uy, e2 hold the moments, only after lb_sync
 * (or a synchronous call of the same kind).
 * Uploads and downloads use separate copy streams and staging memory, so a
 * state upload queued after lb_moments_async overlaps that download (the
 * serving loop set_state_async, step, moments_async).  Host arrays in pinned
 * memory (cudaHostAlloc) make the copies truly asynchronous; with pageable
 * memory the calls are correct but the driver serialises the copies.
 * Results equal those of the synchronous calls bit for bit. */
int lb_set_state_async(lb_handle* h, const double* f);
int lb_moments_async(lb_handle* h, double* rho, double* ux, double* uy, double* e2);

/* Sites that took the Ehrenfests' step in the last completed step (order
 * unspecified).  idx: host array of cap ints; *count receives the number
 * (which may exceed cap; only cap are written). */
int lb_selected(lb_handle* h, int* idx, int cap, int* count);

/* Per-step number of Ehrenfests' sites for the last n steps (oldest
 * first).  At most the log capacity (lb_set_log_capacity) is kept. */
int lb_counts(lb_handle* h, int* per_step, int n);

/* Velocity probe (Sec. 4.2.1): log u_x of the pre-collision state at (x, y)
 * once per step.  lb_probe copies the last n samples (oldest first). */
int lb_set_probe(lb_handle* h, int x, int y);
int lb_probe(lb_handle* h, double* ux_series, int n);

/* Capacity (steps) of the count and probe logs; default 65536.  Resets
 * both logs. */
int lb_set_log_capacity(lb_handle* h, int steps);

/* Nonequilibrium entropy dS (DelS) of the current pre-collision state at
 * every site, evaluated exactly (no pre-filter) in the run's arithmetic
 * type.  ds: [ny][nx] FP64, host or (on_device != 0) device. */
int lb_delta_s(lb_handle* h, double* ds, int on_device);

/* Test hook: the selection rule alone.  Among the n values ds[0..n)
 * (host FP64), select the k largest with ds > delta (all of them if fewer
 * qualify), ties to the lower index, through the same block top-k and
 * global radix-select kernels as lb_step.  idx_out: host array of at least
 * min(n, k) ints (order unspecified); *count receives the number selected.
 * Runs on an internal stream and synchronises. */
int lb_select_only(const double* ds, int n, double delta, int k, int* idx_out, int* count);

/* Largest n accepted by lb_select_only_noalloc. */
#define LB_NOALLOC_MAX_N 262144

/* lb_select_only_noalloc -- the paper has no counterpart to this entry point;
 * it exists for callers that cannot allocate device memory: hosts whose own
 * allocator has reserved the device memory and hands it out itself, and
 * real-time loops that must not take cudaMalloc's implicit device
 * synchronisation or its latency.  It makes the same selection as lb_select_only: among
 * ds[0..n) the k largest values > delta (all of them if fewer qualify), ties
 * to the lower index, through the same kernels.
 *   ds:      DEVICE pointer to n FP64 values (read; may be NULL when n = 0);
 *   idx_out: DEVICE pointer to min(n, k) ints (written; order unspecified;
 *            may be NULL when n = 0 or k = 0);
 *   count:   DEVICE pointer to one int (written: the number selected);
 *   cuda_stream: the stream the work is queued on (NULL: the legacy default
 *            stream).  The call is asynchronous: the outputs are valid once
 *            the stream has reached this work.
 * It calls no cudaMalloc, cudaFree or other allocating routine.  Its working
 * memory is one fixed device array of about 3 MB per GPU (room for
 * LB_NOALLOC_MAX_N candidates), held by every GPU that loads the library
 * until the process exits; n > LB_NOALLOC_MAX_N is rejected with LB_ERR_ARG.
 * The first call on a device looks up that array's device address (and sets
 * the select kernel's shared-memory limit) with that device current; make
 * that first call before any stream capture.  All calls share the array:
 * calls that overlap on the GPU (different streams, or different host
 * threads, without ordering between them) race and give wrong results. */
int lb_select_only_noalloc(const double* ds, int n, double delta, int k, int* idx_out, int* count,
                           void* cuda_stream);

/* Test hook: for the next nsteps steps, use the given selections instead of
 * selecting (replay of another implementation's choices).  counts[t] sites
 * for step t, their indices concatenated in idx.  Host arrays. */
int lb_replay_selection(lb_handle* h, const int* counts, const int* idx, int nsteps);

/* Collision (Sec. 4.1): LB_COLLISION_LBGK (lbgkLB, the default),
 * f' = f + 2 beta (f* - f); or LB_COLLISION_ELBM (elbmLB),
 * f' = f + alpha beta (f* - f) with alpha the nontrivial root of
 * S(f + alpha (f* - f)) = S(f) per site (FP64, to 1e-15; alpha = 2 at
 * f = f*; the positivity limit when the entropy still exceeds S(f) there).
 * ELBM needs LB_EQ_ENTROPIC (LB_ERR_ARG otherwise); Ehrenfests' steps apply
 * to it as to LBGK.  Synchronises the run's stream. */
enum lb_collision { LB_COLLISION_LBGK = 0, LB_COLLISION_ELBM = 1 };
int lb_set_collision(lb_handle* h, int collision);

/* ---- Learned form ------------------------------------------------------
 * The 4-64-64-4 ReLU network that gives the energy Newton solve of
 * LB_EQ_ENTROPIC_ENERGY_MLP its start point.  The Lagrange form of the
 * quasiequilibrium (Sec. 3.3) is ln(f*_i / W_i) = mu . (1, v_x, v_y, |v|^2);
 * the network maps the standardised features (rho, u_x, u_y,
 * 2E/rho - |u|^2) to (mu - mu0) / out_scale, mu0 = (ln rho - 3/2 |u|^2,
 * 3 u_x, 3 u_y, 0) being the polynomial start point.  The paper does not
 * use a network; it is this implementation's way to shorten the solve.
 *
 * Parameters: n = lb_mlp_param_count() FP32 values, in this order:
 * W1[64][4], b1[64], W2[64][64], b2[64], W3[4][64], b3[4] (trainable), then
 * mean[4], inv_std[4] (input standardisation) and out_scale[4].  Evaluation
 * (inference and the forward pass of training) rounds the standardised
 * inputs, the weights and the hidden activations to BF16 and accumulates in
 * FP32 on the tensor cores.
 *
 * lb_set_mlp: host array of n parameters (all finite), copied into the
 * run (the run must use LB_EQ_ENTROPIC_ENERGY_MLP; lb_step fails with
 * LB_ERR_STATE until it has been called).  Synchronises the run's stream. */
int lb_mlp_param_count(void);
int lb_set_mlp(lb_handle* h, const float* params, int n);

/* Initial parameters (host array of n = lb_mlp_param_count()): weights
 * uniform in +-sqrt(6 / fan_in) from SplitMix64(seed), zero biases,
 * mean 0, inv_std 1, out_scale 1. */
int lb_mlp_init(float* params, int n, unsigned long long seed);

/* Training data (Sec. 3.3 with the moments M = (rho, rho u, 2E) of
 * (argmax)).  Device arrays of n samples: rho, ux, uy and escale; sample i
 * has 2E = escale[i] x (2E of the isothermal entropic equilibrium of
 * Sec. 4.2 at rho, u).  Its multipliers mu are found by Newton from mu0
 * (FP32 iterations, FP64 steps to a residual of 1e-12 or below).  Outputs
 * (device): feat[n][4] = (rho, u_x, u_y, 2E/rho - |u|^2) and
 * dmu[n][4] = mu - mu0 (FP32); mu[n][4] (FP64, optional); stats (optional,
 * 4 counters, added to): FP32 iterations, FP64 iterations, samples, samples
 * whose residual missed 1e-12.  Asynchronous on the stream (NULL: the
 * default stream). */
int lb_energy_dataset(const double* rho, const double* ux, const double* uy, const double* escale,
                      long long n, float* feat, float* dmu, double* mu, unsigned long long* stats,
                      void* cuda_stream);

/* Sets mean, inv_std (1 / standard deviation) of the features and out_scale
 * (root mean square of dmu) of the device parameter vector from n samples
 * (device arrays as written by lb_energy_dataset).  Asynchronous. */
int lb_mlp_normalise(float* params, const float* feat, const float* dmu, long long n, void* cuda_stream);

/* The network's outputs y[n][4] for features feat[n][4]; device arrays,
 * asynchronous. */
int lb_mlp_forward(const float* params, const float* feat, long long n, float* y, void* cuda_stream);

/* Loss L = mean over the n samples and the 4 outputs of
 * (y - dmu / out_scale)^2 and its gradient with respect to the parameters
 * (grad[lb_mlp_param_count()]; the normalisation entries get 0), taken
 * through the BF16 roundings as if they were the identity.  Device arrays;
 * loss: one float (device, may be NULL).  Deterministic.  Asynchronous. */
int lb_mlp_grad(const float* params, const float* feat, const float* dmu, int n, float* grad,
                float* loss, void* cuda_stream);

/* One Adam step t >= 1 (b1 = 0.9, b2 = 0.999, eps = 1e-8) on the trainable
 * entries: m, v are the moment estimates (device, lb_mlp_param_count()
 * floats each, zero before step 1).  Asynchronous. */
int lb_mlp_adam(float* params, const float* grad, float* m, float* v, long long t, double lr,
                void* cuda_stream);

/* Mini-batch Adam over n samples (consecutive batches of `batch`, the last
 * one shorter), `epochs` passes; the learning rate decays geometrically
 * from lr0 at the first step to lr1 at the last.  params (device) in and
 * out; loss_log (device, optional): mean batch loss of each epoch.
 * Asynchronous; allocates its working memory on the stream. */
int lb_mlp_train(float* params, const float* feat, const float* dmu, long long n, int batch, int epochs,
                 double lr0, double lr1, float* loss_log, void* cuda_stream);

/* Newton statistics of the energy forms since the last reset: total
 * FP32 iterations, finishing iterations (float-float for FP32 / FP16
 * storage, FP64 for FP64 storage), sites solved, and sites that missed
 * 1e-12. */
int lb_newton_stats(lb_handle* h, long long* it32, long long* it64, long long* sites,
                    long long* fails, int reset);

/* Kernel timing for measurement: when enabled, every launch of lb_step (one
 * per time step: stream-collide with the selection and the Ehrenfests' step
 * fused into its last block) is bracketed by CUDA events on the run's
 * stream (graphs are not used).  lb_kernel_times returns the summed
 * milliseconds and launch counts since the last reset (synchronises); the
 * select figures count stand-alone select launches, which lb_step no
 * longer makes. */
int lb_set_timing(lb_handle* h, int enable);
int lb_kernel_times(lb_handle* h, double* collide_ms, long long* collide_launches,
                    double* select_ms, long long* select_launches, int reset);

/* Tile shape of the D2Q9 stream-collide kernel.  Register-fed shapes (sites
 * per thread in x, warps per block, minimum resident blocks per SM):
 * 0 = 1, 8, 3;  1 = 1, 8, 4;  2 = 2, 8, 2;  3 = 4, 8, 1.
 * Shared-memory-staged shapes (tensor-memory-accelerator copies, for every
 * population plane, of the R rows of the R x C-site block tile's sources in
 * that plane plus 16 bytes of halo columns; R rows, C columns, STAGES tiles
 * in flight per block): 4 = 8 x 128, STAGES 2 (default of FP64 storage);
 * 5 = 6 x 128, STAGES 3 (default of FP16 storage and of FP32 storage, plain
 * and deviation, above 600 000 sites; FP32 storage with the polynomial
 * quasiequilibrium up to 600 000 sites defaults to the register-fed shape
 * 1);  6 = 8 x 64, STAGES 2 (three blocks
 * per SM).  The
 * energy-constrained forms are built for shapes 0 (1, 8, 2: 128 registers
 * per thread), 1 (2 and 3 run 1), 4 and 5, and refuse 6 (LB_ERR_ARG); their
 * defaults: 1 for FP64 storage, 4 for FP32 / FP16 storage (Newton start and
 * network warm start alike).  Results do not depend on the shape; only the
 * speed does. */
int lb_set_tile_shape(lb_handle* h, int shape);

/* ------------------------------------------------------------------------
 * One run sharded in x over several handles (one per GPU): each handle holds
 * a slab of columns plus one ghost column on every side that faces another
 * slab.  The selection of Sec. 3.2 is global -- the k sites of the whole
 * grid with the largest dS > delta -- so each step is:
 *   lb_slab_collide     stream + collide of the slab (ghost columns hold the
 *                       neighbours' post-collision populations of the
 *                       previous step), ending with the slab's own k best
 *                       candidates;
 *   lb_slab_candidates  those candidates (key, global site index) to the
 *                       host; the caller gathers every slab's and keeps the
 *                       k best of the union (key descending, global index
 *                       ascending) -- the same set one unsharded run selects;
 *   lb_slab_apply       that global selection: the Ehrenfests' step at the
 *                       slab's own selected sites; completes the step;
 *   lb_slab_ghost       pack the populations leaving through a face into a
 *                       device buffer / unpack the neighbour's into the ghost
 *                       column, before the next lb_slab_collide.
 * lb_step is refused on a slab.  D2Q9 only.
 * ------------------------------------------------------------------------ */

/* Make h (created with the slab's local grid: its nx counts the ghost
 * columns; boundary kinds of the global run on its outer sides, any
 * non-periodic kind on a side facing another slab; obstacle in local
 * coordinates) a slab.  ghost_left / ghost_right: 1 where another slab lies
 * on that side, else 0; global_x0: global x of the slab's first own column;
 * global_nx: columns of the whole grid.  A slab owns at least three columns.
 * Allocates the slab's candidate and selection lists (device). */
int lb_set_slab(lb_handle* h, int ghost_left, int ghost_right, int global_x0, int global_nx);

/* Queue the slab's stream + collide launch (asynchronous); its last block
 * keeps the slab's k best candidates instead of applying them. */
int lb_slab_collide(lb_handle* h);

/* The slab's candidates of the collided step (synchronises): keys (host,
 * monotone uint64 images of dS, larger = larger dS) and global site indices
 * (y * global_nx + x), at most cap of them; *count = how many (<= k). */
int lb_slab_candidates(lb_handle* h, unsigned long long* keys, long long* global_idx, int cap, int* count);

/* Apply the step's global selection (m host global site indices, any
 * order, m <= k): f' <- f* at the slab's own sites among them (Sec. 3.2;
 * (ESLB)); logs the slab's share of the count; completes the step
 * (synchronises). */
int lb_slab_apply(lb_handle* h, const long long* global_idx, int m);

/* Ghost exchange of the completed step (asynchronous on the run's stream):
 * direction 0 packs the three populations that leave through side (0 left,
 * 1 right) -- those moving toward that neighbour, of the slab's first or
 * last own column -- into buf; direction 1 writes buf into the ghost column
 * on that side.  buf: DEVICE array of 3 * ny values of the storage type
 * (planes 3, 6, 7 or 1, 5, 8, each [ny]), owned by the caller. */
int lb_slab_ghost(lb_handle* h, int side, void* buf, int direction);

/* Run facts (out: 8 entries): out[0] = Q, out[1] = padded row length
 * (elements), out[2] = bytes per stored population, out[3] = algorithmic
 * bytes per site update (read Q + write Q populations), out[4] = launches
 * per step (1), out[5] = blocks of the persistent stream-collide grid,
 * out[6] = its resident blocks per SM, out[7] = tile shape.
 * beta_out (nullable) receives beta. */
int lb_info(lb_handle* h, long long* out, double* beta_out);

/* Thread-local message of the last failed call ("" if none). */
const char* lb_last_error(void);

/* ---- Batched form ------------------------------------------------------
 * Many independent D2Q9 runs (each one the method of Sec. 3.2 on its own
 * grid) advanced together and replayed as CUDA graphs of 32 steps, by one of
 * three launch strategies (variants):
 *   0, 1  the batched kernel: per time step, one stream-collide launch
 *         covers the work of every run (a flat list of each run's edge
 *         columns and block tiles, taken by a persistent grid; 8-row tiles
 *         with 2 stages, or 4-row tiles with 3 stages), then one launch
 *         performs every run's selection and Ehrenfests' step (a block per
 *         run);
 *   2     every run's own stream-collide kernel, each run a chain of steps
 *         in its own concurrent branch of the graph.
 * Results are bit-identical to stepping each run alone with lb_step.  The paper runs
 * one flow at a time; the batch is this implementation's way to fill the
 * GPU with small runs (parameter sweeps). */
typedef struct lb_run_desc {
    int lattice;            /* LB_D2Q9 */
    int nx, ny;
    int equilibrium;        /* LB_EQ_POLY or LB_EQ_ENTROPIC, the same for every run */
    double nu, delta;
    int k;
    lb_boundaries bc;
    int precision;          /* the same for every run */
} lb_run_desc;

typedef struct lb_batch lb_batch;

/* Creates the runs (as lb_create would, on one stream: cuda_stream, or a
 * new one when NULL).  Fails with LB_ERR_ARG for other lattices or
 * equilibria, mixed precisions or equilibria, or more than 4096 runs. */
int lb_batch_create(const lb_run_desc* runs, int nruns, void* cuda_stream, lb_batch** out);
void lb_batch_destroy(lb_batch* b);

/* The run r of the batch (owned by the batch; NULL if out of range): use it
 * to initialise, read and log the run.  Stepping it alone with lb_step
 * makes the next lb_batch_step fail with LB_ERR_STATE. */
lb_handle* lb_batch_run(lb_batch* b, int r);

/* Advances every run by n steps (batched launches).  Asynchronous; errors
 * of the runs are reported by the next call, as for lb_step. */
int lb_batch_step(lb_batch* b, int n);

/* The same n steps through each run's own lb_step, one run after another
 * (the baseline the batched launches are measured against). */
int lb_batch_step_sequential(lb_batch* b, int n);

int lb_batch_sync(lb_batch* b);

/* Launch strategy (variant 0, 1 or 2, above; 0 after lb_batch_create).
 * Synchronises. */
int lb_batch_set_variant(lb_batch* b, int variant);

/* Autotuner: when cache_path (may be NULL) holds an entry for this device
 * and batch (device name, SM count, storage, equilibrium, run sizes), its
 * variant is used; otherwise every variant is timed as it runs in
 * production, over `steps` steps rounded up to whole graphs of 32 (CUDA
 * events around the graph replays, after one warm-up graph), the fastest is
 * chosen and written to the cache (a JSON object).  Timing advances every
 * run by 1 + variants x 32 x (1 + ceil(steps / 32)) steps (all variants
 * compute identical results).  variant_out may be NULL. */
int lb_batch_autotune(lb_batch* b, int steps, const char* cache_path, int* variant_out);

/* Per-launch CUDA events (graphs are not used while enabled), summed by
 * lb_batch_kernel_times (synchronises). */
int lb_batch_set_timing(lb_batch* b, int enable);
int lb_batch_kernel_times(lb_batch* b, double* ms, long long* launches, int reset);

/* out[8]: runs, sites, work items of the batched kernel (each run's tiles,
 * plus its edge items: the x = 0 and x = nx - 1 columns, 32 x tile rows
 * sites each), grid blocks, blocks per SM, variant, tile rows, steps per
 * graph. */
int lb_batch_info(lb_batch* b, long long* out);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
