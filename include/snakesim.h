/*
 * snakesim.h -- C-ABI of the GB300 soft-snake simulator.
 *
 * The library advances batches of soft robotic snakes built from 1D pneumatic
 * actuators (Gasoto et al., "A Validated Physical Model For Real-Time Simulation of
 * Soft Robotic Snakes", arXiv 1904.02833).  Each snake is a chain of particles
 * (Sec. IV-A, Eq. 1: q_i = [x y z], lumped mass M_i = m 1_3) held together by compliant
 * constraints c(q, p) + E lambda = 0 (Sec. IV, equations of motion).  Per env-step of
 * length dt the library runs n_sub substeps of first-order implicit time stepping
 * (Sec. IV-D); each substep
 *   a1  samples the open-loop gait a_k = clamp(sin(w t + alpha k) + phi, -1, 1) A (Eq. 9),
 *   a2  filters the two antagonistic chamber pressures of every link (Sec. III) through a
 *       first-order inflate / deflate latency,
 *   a3  turns pressure into rest curvature (Eq. 3-4: a chamber's rest length scales with
 *       eps(p) = 1 + p / Y; with an inextensible centre layer this is a rest angle
 *       G (p_R - p_L) L0 per node),
 *   a4  predicts positions under gravity,
 *   a5  relaxes the Schur system of Eq. 8 with its own diagonal (the Jacobi
 *       preconditioner of Sec. IV-D) over stretch, yaw/pitch bend, ground contact
 *       (Eq. 7) and Coulomb friction rows, in parallel, with compliance alpha / h^2,
 *   a6  measures the normalised residual and stops at the tolerance or the cap,
 *   a7  updates velocities from the displacement with exponential damping.
 * Thousands of snakes of uneven length run together: the snakes are grouped by length
 * into lane layouts (8, 16 or 32 lanes per snake, 1-4 nodes per lane), and each layout
 * runs one persistent kernel that takes its snakes from a device-side work queue.
 *
 * Conventions (every call):
 *   - Every call returns a SimStatus; nothing aborts or throws across the ABI.  The text
 *     of the last error of the calling thread is available from sim_last_error().
 *   - Work is enqueued on the CUDA stream given to sim_create (a cudaStream_t passed as
 *     void*, 0 = legacy default stream) and is asynchronous unless stated otherwise.
 *   - The library owns its device buffers (allocated in sim_create, freed in
 *     sim_destroy).  Caller buffers are only read or written during the call, or by work
 *     enqueued by it on the handle's stream.
 *   - Buffers flagged is_device = 1 are device pointers (e.g. from torch tensors);
 *     is_device = 0 means host memory (copies are synchronous with the stream).
 *   - Node arrays hold the snakes back to back: snake s owns nodes
 *     [node_off[s], node_off[s+1]) with node_off[s+1] - node_off[s] = n_links * seg + 1,
 *     and links [link_off[s], link_off[s+1]).
 *   - A handle is used by one host thread at a time.
 */
#ifndef SNAKESIM_H_
#define SNAKESIM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct SimHandle SimHandle; /* opaque, owned by the library */

typedef enum {
  SIM_OK = 0,
  SIM_NOT_CONVERGED = 1, /* warning: some snake hit the iteration cap above tol */
  SIM_EINVAL = -1,       /* bad argument; nothing was enqueued */
  SIM_ECUDA = -2,        /* a CUDA call failed; see sim_last_error() */
  SIM_ENOMEM = -3,       /* device allocation failed */
  SIM_ENAN = -4          /* a snake's state became non-finite */
} SimStatus;

/* Warm-start modes of the multipliers at the start of every substep. */
enum { SIM_WARM_COLD = 0, SIM_WARM_PREVIOUS = 1, SIM_WARM_LEARNED = 2 };

/* Global solver settings. */
typedef struct {
  double dt;          /* env-step length [s] (1/60 in the paper's real-time setting)     */
  int32_t n_sub;      /* substeps per env-step, h = dt / n_sub                           */
  int32_t iters;      /* cap on Jacobi updates per substep                               */
  float tol;          /* residual tolerance; 0 runs exactly `iters` updates              */
  float omega;        /* Jacobi relaxation (1/3: a node touches at most 3 bend rows)     */
  float gravity[3];   /* [m/s^2]                                                         */
  int32_t contact;    /* 1: ground plane z = 0 with Coulomb friction                     */
  int32_t warm;       /* SIM_WARM_*                                                      */
  float beta;         /* weight of the previous substep's multipliers in a warm start:   *
                       * PREVIOUS starts from beta lambda_prev, LEARNED from              *
                       * beta_net lambda_prev + m g h^2 y (y: the network's output) on    *
                       * the rows the network predicts and from beta lambda_prev on the   *
                       * others and at the substeps between network substeps             */
  int32_t latency;    /* chamber model, SIM_LATENCY_*                                    */
  /* SIM_LATENCY_LAW only (Sec. V-A, Eq. 11-12; pressures in units of the maximum):      *
   * every law_dt seconds (rounded to whole substeps, at least one) each chamber moves    *
   * towards its target p^ at the end of that period: inflating by                        *
   * p_source k_inflate ((p^ - p) / p_source)^2, deflating by min(p k_deflate, t_p),      *
   * never past p^; it holds its value in between.                                        */
  float k_inflate;    /* (0, 1]; the paper's fitted value 0.23                           */
  float k_deflate;    /* (0, 1]; the paper's fitted value 0.23                           */
  float t_p;          /* > 0; the paper's 0.68 psi of an 8 psi maximum = 0.085           */
  float p_source;     /* > 0; source pressure                                            */
  float law_dt;       /* >= 0 [s]; the paper's time step 0.0083 s                        */
  int32_t solver;     /* SIM_SOLVER_*                                                    */
  int32_t pcr_iters;  /* SIM_SOLVER_NEWTON_PCR: PCR iterations per Newton step (>= 1; the *
                       * paper uses 20)                                                   */
  /* SIM_WARM_LEARNED only:                                                               */
  int32_t net_rows;   /* SIM_NET_ROWS_*: the row kinds the network predicts               */
  int32_t net_every;  /* the network runs at substeps s with s % net_every == 0 (0 is     *
                       * read as 1); the substeps in between start from beta lambda_prev  *
                       * and run in the same launch as the network substep before them   */
  float beta_net;     /* weight of lambda_prev under the network's prediction, <= 1; a    *
                       * negative value means beta                                        */
} SimConfig;

/* Row kinds the network predicts in the learned warm start: all six (stretch, yaw, pitch,
 * contact, friction x / y), the bilateral rows only (stretch, yaw, pitch), or the stretch
 * rows only; the other rows then start from beta lambda_prev. */
enum { SIM_NET_ROWS_ALL = 0, SIM_NET_ROWS_BILATERAL = 1, SIM_NET_ROWS_STRETCH = 2 };

/* Substep solvers: the Jacobi relaxation of Eq. 8 (`iters` caps its updates), or the
 * paper's Newton steps with a preconditioned conjugate residual solve of the Schur system
 * (Sec. IV-D) over the bilateral rows, for contact-free substeps only (`contact` = 0;
 * `iters` caps the matrix-vector products; the update counts report them). */
enum { SIM_SOLVER_JACOBI = 0, SIM_SOLVER_NEWTON_PCR = 1 };

/* Chamber models: first-order latency with the per-snake tau_inf / tau_def (exact
 * exponential relaxation every substep), or the paper's discrete law (Sec. V-A). */
enum { SIM_LATENCY_EXP = 0, SIM_LATENCY_LAW = 1 };

/* Per-snake parameters (host layout, 96 bytes). */
typedef struct {
  int32_t n_links;      /* soft links; nodes = n_links * seg_per_link + 1               */
  int32_t seg_per_link; /* segments per link (rigid connector at every link boundary)   */
  int32_t n_fixed;      /* leading nodes clamped in place (cantilever: 2)               */
  float mu_side;        /* > 0: anisotropic friction (the wheels and scales of Sec. V):   *
                         * mu along the body, mu_side across it, friction pair limited *
                         * to the ellipse of the body frame; 0: isotropic mu            */
  float L0;             /* segment rest length [m]                                       */
  float mass;           /* node mass [kg]                                                */
  float alpha_s;        /* stretch compliance [m/N]                                      */
  float alpha_b;        /* bend compliance [m/N]; bend rows are L0 x angle               */
  float gain;           /* rest curvature per unit pressure G [rad/m]                    */
  float tau_inf;        /* inflation time constant [s]                                   */
  float tau_def;        /* deflation time constant [s]                                   */
  float mu;             /* Coulomb friction coefficient                                  */
  float damping;        /* velocity damping rate d [1/s]: v <- v exp(-d h)               */
  float radius;         /* contact radius r: contact row z - r >= 0 [m]                  */
  float gait_amp;       /* A of Eq. 9 (pressure normalised to [0, 1])                    */
  float gait_freq;      /* f [Hz], the sine is sin(2 pi f t + k lag)                     */
  float gait_lag;       /* phase shift between links alpha [rad]                         */
  float gait_offset;    /* phi of Eq. 9                                                  */
  float gait_scale;     /* sine scale (1 in Eq. 9; 0 gives a constant command)           */
  float gait_alternate; /* 1: sign (-1)^k on link k (pressure on alternating sides)      */
  float x0, y0, z0;     /* position of node 0 [m]                                        */
  float yaw0;           /* initial heading [rad]                                         */
} SnakeParams;

/* Creates a simulator for n_snakes snakes (params: host array of n_snakes) in the
 * straight initial pose (node i at (x0, y0, z0) + i L0 (cos yaw0, sin yaw0, 0)), at
 * rest, chambers empty, multipliers zero, time 0.  `stream` is a cudaStream_t (void*).
 * Errors: SIM_EINVAL (null pointers, n_snakes < 1, n_links < 1, seg_per_link < 1,
 * n_fixed outside [0, nodes], non-positive L0 / mass / dt / n_sub, iters < 0),
 * SIM_ENOMEM, SIM_ECUDA.  On error *out is NULL. */
SimStatus sim_create(const SimConfig* cfg, int n_snakes, const SnakeParams* params,
                     void* stream, SimHandle** out);

/* Replaces the solver settings (dt, n_sub, iters, tol, omega, gravity, contact, warm)
 * for subsequent steps.  Same validation as sim_create. */
SimStatus sim_set_config(SimHandle* h, const SimConfig* cfg);

/* Overrides the gait: u[total_links] in [-1, 1] is the command of every link for every
 * substep of subsequent sim_step calls (u > 0 drives the right chamber, u < 0 the
 * left, Sec. III); u = NULL returns to the gait of Eq. 9.  The values are copied
 * (stream-ordered) into a library buffer; the caller may reuse u after the call.
 * Errors: SIM_EINVAL for a null handle. */
SimStatus sim_set_pressure(SimHandle* h, const float* u, int is_device);

/* Advances every snake by n_steps env-steps (asynchronous).  n_steps >= 0.
 * The per-snake residual (max over the steps' substeps of the residual after the last
 * update) and update counts (sum over substeps of the last env-step) are kept for
 * sim_get_state.  Errors: SIM_EINVAL, SIM_ECUDA. */
SimStatus sim_step(SimHandle* h, int n_steps);

/* Reads the state.  Any pointer may be NULL.  pos, vel: [total_nodes][3] float;
 * press: [total_links][2] (p_R, p_L); resid: [n_snakes] float; iters: [n_snakes] int32.
 * is_device = 0 copies to host memory and synchronises the stream; is_device = 1
 * enqueues device-to-device copies. */
SimStatus sim_get_state(SimHandle* h, float* pos, float* vel, float* press, float* resid,
                        int32_t* iters, int is_device);

/* Overwrites the state (any pointer may be NULL: that part is kept).  Layouts as in
 * sim_get_state; lam: [total_nodes][6] multipliers (stretch, yaw, pitch, contact,
 * friction x, friction y of the rows a node owns). */
SimStatus sim_set_state(SimHandle* h, const float* pos, const float* vel, const float* press,
                        const float* lam, int is_device);

/* Reads the multipliers [total_nodes][6] (layout as in sim_set_state). */
SimStatus sim_get_lambda(SimHandle* h, float* lam, int is_device);

/* Sizes: total nodes, total links, snakes; and the env-step counter (time = step * dt). */
SimStatus sim_get_info(SimHandle* h, int64_t* n_nodes, int64_t* n_links, int32_t* n_snakes,
                       int64_t* step_index);

/* Sets the env-step counter (the gait time is step_index * dt). */
SimStatus sim_set_step_index(SimHandle* h, int64_t step_index);

/* Device pointers of the library-owned state, for zero-copy use from torch:
 * pos4/vel4 [total_nodes] float4 (x, y, z, inverse mass) / (vx, vy, vz, 0),
 * press2 [total_links] float2, lam [total_nodes][6] float.  Valid until sim_destroy. */
SimStatus sim_device_state(SimHandle* h, void** pos4, void** vel4, void** press2, void** lam);

/* Per-snake status of the last step: 0 ok, SIM_NOT_CONVERGED, SIM_ENAN (host array
 * [n_snakes], synchronises the stream).  Returns the worst status. */
SimStatus sim_get_status(SimHandle* h, int32_t* status);

/* Chooses the lanes per snake and nodes per lane of every snake-length bucket by
 * timing candidate layouts with CUDA events (the state is restored afterwards).
 * Runs synchronously.  Errors: SIM_EINVAL, SIM_ECUDA. */
SimStatus sim_autotune(SimHandle* h, int n_steps);

/* Current layout of a bucket of snakes with `nodes` nodes: lanes per snake (8, 16, 32)
 * and nodes per lane (1..4); 0 if no snake has that length. */
SimStatus sim_get_layout(SimHandle* h, int nodes, int32_t* lanes, int32_t* nodes_per_lane);

/* Forces the layout of a bucket (lanes in {8, 16, 32}, nodes_per_lane in 1..4,
 * lanes * nodes_per_lane >= nodes).  Errors: SIM_EINVAL. */
SimStatus sim_set_layout(SimHandle* h, int nodes, int lanes, int nodes_per_lane);

/* Captures sim_step(h, n_steps) in a CUDA graph on first use and replays it
 * afterwards (the graph is rebuilt when the configuration or layout changes). */
SimStatus sim_step_graph(SimHandle* h, int n_steps);

/* Saves / restores the whole simulation state (positions, velocities, pressures,
 * multipliers, per-snake residual, update count and status, env-step counter, substep
 * position of split stepping and, inside a split env-step, the begun substep's
 * features) in a library-owned snapshot; stream-ordered.  Restoring without a saved
 * snapshot is SIM_EINVAL. */
SimStatus sim_snapshot_save(SimHandle* h);
SimStatus sim_snapshot_restore(SimHandle* h);

/* ---------------------------------------------------------------- calibration adjoint
 * Gradients for calibrating five per-snake parameters theta = (alpha_b, damping d,
 * tau_inflate, tau_deflate, gain G) against observed trajectories (no counterpart in the
 * paper, which tunes its latency gains by hand, Sec. VI-B).
 *
 * sim_calib_forward runs n_steps env-steps from the current state with theta (device
 * FP32 [n_snakes][5]) replacing those parameters, every substep starting cold and
 * applying exactly `iters` Jacobi updates (the configuration's tol and warm start are
 * not used; the gait of Eq. 9 drives the links, a command override is ignored).  It
 * writes the last node's position after every env-step to tips (device FP32
 * [n_steps][n_snakes][3]), keeps the state every ckpt_every env-steps as a checkpoint,
 * and advances the simulator.
 * sim_calib_backward takes d L / d tips (device [n_steps][n_snakes][3]) and writes
 * d L / d theta (device [n_snakes][5]) for the executed discrete map: each checkpoint
 * segment is recomputed, its substeps are walked in reverse and, inside each, the K
 * iterates are recomputed and transposed (clamps and the friction projection take the
 * derivative of the branch they took).  Working memory grows with ckpt_every x n_sub
 * substep states per snake.  Errors: SIM_EINVAL, SIM_ENOMEM, SIM_ECUDA. */
SimStatus sim_calib_forward(SimHandle* h, const float* theta, int n_steps, int ckpt_every,
                            float* tips);
SimStatus sim_calib_backward(SimHandle* h, const float* tips_bar, float* grad_theta);

/* Kernel launches made by this handle so far (the count the benchmark reports). */
SimStatus sim_launch_count(SimHandle* h, int64_t* launches);

/* Per-layout kernel timing.  sim_kernel_timing(h, 1) makes the following sim_step /
 * sim_split_* calls (not sim_step_graph) launch the layouts' solver kernels one after
 * another on the handle's stream (instead of overlapping them on forked streams) with a
 * CUDA event pair around every launch; sim_kernel_times synchronises the handle's stream and
 * returns, per lane layout id (lanes 8/16/32 x nodes per lane 1..4: id = 4 (lanes / 16,
 * i.e. 0, 1, 2) + nodes per lane - 1), the summed kernel time in ms and the launch count
 * (host arrays of 12), then forgets the recorded launches.  Errors: SIM_EINVAL, SIM_ECUDA. */
SimStatus sim_kernel_timing(SimHandle* h, int enable);
SimStatus sim_kernel_times(SimHandle* h, float* ms, int64_t* launches);

/* Frees the handle and its device buffers (synchronises the stream).  NULL is ok. */
SimStatus sim_destroy(SimHandle* h);

/* Splits a batch for several GPUs: the snakes are independent (each one's substeps touch
 * only its own nodes, Sec. IV), so one batch runs as contiguous snake ranges, one handle
 * per range and GPU, with no exchange between them.  params: host [n_snakes];
 * first: host int32 [parts + 1], receives the ranges: part p owns snakes
 * [first[p], first[p + 1]), first[0] = 0, first[parts] = n_snakes.  The ranges are
 * balanced by node count (n_links * seg_per_link + 1 per snake): boundary p is the snake
 * boundary whose node prefix sum is nearest to p / parts of the total (the lower one on
 * a tie), kept non-decreasing, so every part holds the ideal share to within the nodes of
 * one snake (parts beyond the number of snakes may be empty).  Host computation only (no
 * CUDA call, no GPU needed).  Errors: SIM_EINVAL (n_snakes < 1, parts < 1, null
 * pointers, a snake with n_links or seg_per_link < 1). */
SimStatus sim_partition(int n_snakes, const SnakeParams* params, int parts, int32_t* first);

/* Measures the FP32 arithmetic roof the solvers are compared against: enqueues on
 * `stream` n_blocks blocks of 256 threads, each thread running `iters` rounds of 16 x 8
 * independent fused multiply-adds (256 FLOP per round and thread), and writes one
 * float per thread to out_dev (device, n_blocks * 256 floats) so that nothing is
 * optimised away.  The caller times it (FLOP = n_blocks * 256 * iters * 256).
 * Errors: SIM_EINVAL (n_blocks < 1, iters < 1, null out_dev), SIM_ECUDA. */
SimStatus sim_fp32_fma_probe(float* out_dev, int n_blocks, int iters, void* stream);

/* ---------------------------------------------------------------- learned warm start
 * A small network predicts the multipliers each substep starts from, so that fewer
 * Jacobi updates reach the tolerance (no counterpart in the paper, which solves every
 * step with Newton + PCR from scratch, Sec. IV-D).  Per constraint row it reads 24
 * features (row kind, the row's node positions and velocities in the row's frame, the
 * rest angle, the previous substep's multiplier; written by the solver, bf16, padded to
 * 32 per row) and computes lambda0 / (m g h^2) = w3 . silu(W2 silu(W1 f + b1) + b2) + b3
 * with hidden width 128, BF16 operands and FP32 accumulation on the tensor cores.
 * Parameter vector (FP32, MLP_NUM_PARAMS): W1 [128][24], b1 [128], W2 [128][128],
 * b2 [128], w3 [128], b3. */
#define MLP_NUM_PARAMS 19841
typedef struct MlpHandle MlpHandle;

/* Creates a network with all parameters zero, bound to `stream` (cudaStream_t). */
SimStatus mlp_create(void* stream, MlpHandle** out);
/* Sets / reads the FP32 parameter vector; setting also resets the Adam moments. */
SimStatus mlp_set_params(MlpHandle* m, const float* params, int is_device);
SimStatus mlp_get_params(MlpHandle* m, float* params, int is_device);
/* out[r] for feat [rows][32] bf16 (device pointers, feat 16-byte aligned).
 * Synchronises the stream; SIM_EINVAL for a misaligned feat, SIM_ECUDA if a tensor-core
 * wait timed out.  The training calls below take feat with the same layout and
 * alignment. */
SimStatus mlp_forward(MlpHandle* m, const void* feat, int64_t rows, float* out);
/* Gradient of L = scale * sum_r (y_r - target_r)^2 into grad[MLP_NUM_PARAMS] and L into
 * *loss (device pointers, either may be NULL).  Synchronises the stream. */
SimStatus mlp_grad(MlpHandle* m, const void* feat, const float* target, int64_t rows,
                   float scale, float* grad, float* loss);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on the mean squared error over the rows;
 * *loss (device, may be NULL) receives the loss before the step.  Asynchronous. */
SimStatus mlp_train_step(MlpHandle* m, const void* feat, const float* target, int64_t rows,
                         float lr, float* loss);
/* Synchronises and reports a timed-out tensor-core wait of earlier asynchronous calls. */
SimStatus mlp_check(MlpHandle* m);
/* Self-test of the bounded waits the network kernels use on tensor-core completions (no
 * counterpart in the paper): on `stream` (cudaStream_t) one block allocates tensor memory,
 * waits at most `polls` polls on a barrier that nothing arrives on, records that the wait
 * ran out and frees its tensor memory before returning, as the network kernels do when a
 * completion never arrives (they then report SIM_ECUDA).  *timed_out (host) receives 1
 * when the wait ran out, the expected result; the device stays usable.  Synchronises
 * `stream`.  Errors: SIM_EINVAL (polls < 1, null pointer), SIM_ECUDA. */
SimStatus mlp_wait_selftest(uint32_t polls, void* stream, int32_t* timed_out);
SimStatus mlp_destroy(MlpHandle* m);

/* Allocation-free forward pass, for callers that cannot allocate device memory (a
 * control loop with a hard real-time budget that must not stall on the allocator, or a
 * host application whose device memory belongs to its own allocator and offers this
 * library none).  No counterpart in the paper.
 * params: device FP32 parameter vector of n_params = MLP_NUM_PARAMS values (layout as
 * above, owned by the caller); feat: device bf16 [rows][32]; out: device FP32 [rows];
 * stream: cudaStream_t; feat must be 16-byte aligned.  Calls no cudaMalloc / cudaFree:
 * the bfloat16 weight copies and the timeout flag live in a fixed file-scope device array
 * of MLP_NOALLOC_SCRATCH_BYTES bytes, held by every GPU that loads the library until the
 * process exits.  The first call on a device, with that device current, looks up the
 * array's device address and sets the kernel's shared-memory limit; make that first
 * call before any stream capture begins.  The set-up is keyed on the device's current
 * context, so the first call after a cudaDeviceReset repeats it.  The array is shared by
 * every call on a device and keeps the last call's contents (the call clears the flag it
 * needs at zero), so calls whose GPU work overlaps (other streams, other threads) race;
 * order them on one stream.  Synchronises `stream`.  Errors: SIM_EINVAL (null pointers,
 * rows < 0, a misaligned feat, n_params other than MLP_NUM_PARAMS -- the array holds
 * exactly one network's weights), SIM_ECUDA. */
#define MLP_NOALLOC_SCRATCH_BYTES 41216
SimStatus mlp_forward_noalloc(const float* params, int32_t n_params, const void* feat,
                              int64_t rows, float* out, void* stream);

/* Attaches a network to a simulator (NULL detaches).  With warm = SIM_WARM_LEARNED every
 * substep starts from the network's multipliers; sim_step then runs each substep as
 * solver launch -> network -> solver launch (captured together by sim_step_graph).
 * The network must outlive its use by the simulator. */
SimStatus sim_set_mlp(SimHandle* h, MlpHandle* m);

/* Substep-by-substep stepping (used to log training data).  sim_split_begin starts the
 * next env-step: it runs the gait, latency filter and prediction of substep 0 and writes
 * the features of every row.  sim_split_finish completes the current substep (warm start
 * per the configuration, iterations, velocities) and begins the next one, writing its
 * features; after the last substep the env-step counter advances.  Rows are
 * 6 * total_nodes (six slots per node).  In the learned warm start only the row kinds
 * the network predicts (net_rows) are written; the rows of the other kinds keep what an
 * earlier write left there (zero in a new handle). */
SimStatus sim_split_begin(SimHandle* h);
SimStatus sim_split_finish(SimHandle* h);
/* Device pointer of the feature buffer [rows][32] bf16 and the row count.  The rows of
 * one snake are consecutive (six per node, node by node) but the snakes are grouped by
 * lane layout (so that the network runs once per layout on a contiguous range): snake s
 * starts at row first_row[s] (sim_feature_offsets, host array of n_snakes). */
SimStatus sim_features(SimHandle* h, void** feat, int64_t* rows);
SimStatus sim_feature_offsets(SimHandle* h, int32_t* first_row);

/* Training rows of the learned warm start, for the substep in progress of split stepping
 * (after sim_split_begin, before the sim_split_finish that completes it).  The network's
 * output y enters the warm start as lambda0 = beta lambda_prev + m g h^2 y, so the
 * target that makes the warm start land on a reference solution lambda_star is
 *   y* = (lambda_star - beta lambda_prev) / (m g h^2)
 * with m the snake's node mass, g = 9.81 m/s^2 and h = dt / n_sub of the current
 * configuration.  For every existing row of the substep whose kind has its features
 * written (the rows whose features carry a row kind: stretch rows of nodes 0 .. N-2,
 * yaw and pitch rows of nodes 1 .. N-2, and with contact on the contact and two friction
 * rows of every free node; in the learned warm start only the kinds of net_rows, as
 * configured at this call), snake by snake
 * and node by node with the row kinds in order, the call copies the row's 32 bf16
 * features to feat_out and writes y* to target_out.
 * lam_star, lam_prev: device FP32 [nodes][6] in node order (the layout of
 * sim_get_lambda; typically lambda_prev read before the substep and lambda_star after
 * solving it to a tight tolerance from a snapshot).  feat_out: device bf16
 * [capacity][32], 16-byte aligned; target_out: device FP32 [capacity].  *n_rows (host)
 * receives the number of existing rows; with feat_out and target_out both NULL only
 * the count is returned.  Asynchronous on the handle's stream.  Errors: SIM_EINVAL (no
 * substep in progress, capacity below the row count, misaligned or missing buffers,
 * beta outside [0, 1]), SIM_ECUDA. */
SimStatus sim_training_rows(SimHandle* h, const float* lam_star, const float* lam_prev, float beta,
                            void* feat_out, float* target_out, int64_t capacity, int64_t* n_rows);

/* Text of the last error raised on the calling thread ("" if none). */
const char* sim_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SNAKESIM_H_ */
