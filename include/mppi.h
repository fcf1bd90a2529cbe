/*
 * mppi.h - C ABI of the GB300 (sm_103a) MPPI motion planner.
 *
 * One call of mppi_plan() is one iteration of the Model Predictive Path Integral
 * planner of Testouri, Elghazaly and Frank, "Towards a Safe Real-Time Motion
 * Planning Framework for Autonomous Driving Systems: A Model Predictive Path
 * Integral Approach" (arXiv 2308.01654), Algorithm 1 (one pass of its loop):
 *
 *   1. draw K Gaussian perturbations eps ~ N(0, Sigma) of the control sequence
 *      (Algorithm 1 GenerateRandomNoise; Eq. (1)),
 *   2. roll every perturbed sequence out through the kinematic bicycle model
 *      (Eq. (5), explicit Euler) over T steps and add up the step cost
 *      (Eq. (6)-(9) and the five terms of Sec. IV-C, Eq. (12)-(18)),
 *   3. take the minimum cost and the min-shifted softmin weights with
 *      temperature lambda (Eq. (11)),
 *   4. move the nominal controls by the weighted average perturbation (Eq. (11)),
 *   5. smooth with the 5-point Savitzky-Golay filter (Eq. (19)), roll out the
 *      optimal trajectory x* and shift the warm start (Algorithm 1, last lines).
 *
 * Conventions
 *  - Channel 0 of a control is the acceleration a [m/s^2], channel 1 the
 *    steering angle delta [rad].  States are (x [m], y [m], yaw [rad], v [m/s]).
 *  - Arrays are row-major and tightly packed, element type double unless noted.
 *  - Host arrays belong to the caller and are only read (inputs) or written
 *    (outputs) during the call.  Device arrays passed to the *_device entry
 *    points must stay valid until the work queued on the context's stream has
 *    finished.
 *  - Every function returns an mppi_status (0 = MPPI_OK, negative = error);
 *    nothing is thrown across the ABI.  mppi_last_error() gives a message.
 *  - A context is not thread-safe: use one context per host thread.
 *  - All arithmetic of the iteration runs in this library's CUDA kernels; there
 *    is no CPU fallback.  Without a usable GPU mppi_create() fails with
 *    MPPI_ERR_CUDA.
 */
#ifndef MPPI_H
#define MPPI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPPI_MAX_EGO 8          /* ego-vehicle circles */
#define MPPI_MAX_T 1024         /* horizon steps */
#define MPPI_MAX_REF 4096       /* reference polyline vertices (held in shared memory) */
#define MPPI_MAX_CIRC 1024      /* obstacle circles */

/* Opaque planner context: owns the device buffers, a stream and the warm start. */
typedef struct mppi_ctx mppi_ctx;

typedef enum {
    MPPI_OK = 0,
    MPPI_ERR_ARG = -1,       /* invalid argument or non-finite input */
    MPPI_ERR_OOM = -2,       /* device or pinned host allocation failed */
    MPPI_ERR_CUDA = -3,      /* a CUDA call failed (message in mppi_last_error) */
    MPPI_ERR_NUMERIC = -4,   /* no sample cost was finite; the controls are left unchanged */
    MPPI_ERR_TIMEOUT = -5,   /* a bounded device wait ran out */
    MPPI_ERR_CAPACITY = -6   /* a size exceeds a fixed capacity of the library or context */
} mppi_status;

/* Obstacle circle C_k = {x_k, y_k, r_k} (Sec. III, Fig. 3) with a constant velocity:
   its centre at rollout step t (state x_{t+1}) is (x, y) + (vx, vy) * (t + 1) * dt. */
typedef struct {
    double x, y, r, vx, vy;
} mppi_circle;

/* Covers an oriented rectangular object with circles (Sec. III-C, Fig. 3; Algorithm 1,
   ApproximateObstacles: the paper shows an object as three circles along its length and
   gives no construction, so this is one).  The rectangle has centre (x, y), heading yaw
   [rad], length along the heading and width across it [m]; it is cut into n equal slices
   along its length and each slice gets the circle through its four corners, centred on the
   centre line (radius sqrt((length/2n)^2 + (width/2)^2)), so the circles cover the
   rectangle.  n = 0 picks n = ceil(length / width).  Every circle gets the object's
   velocity (vx, vy).  out: caller-owned array of max_out circles.  Returns the number of
   circles written, MPPI_ERR_ARG for non-finite values, length or width <= 0 or n < 0, or
   MPPI_ERR_CAPACITY when n exceeds max_out.  Host code; needs no GPU. */
int32_t mppi_box_to_circles(double x, double y, double yaw, double length, double width, double vx, double vy,
                            int32_t n, mppi_circle* out, int32_t max_out);

/* Hyper-parameters (Algorithm 1 "Given": M = K, T, lambda, gamma, Sigma, R, D, Z). */
typedef struct {
    int32_t K;                  /* samples (rollouts), >= 1 */
    int32_t T;                  /* horizon steps, 1 ..  MPPI_MAX_T */
    double dt;                  /* step [s], > 0 */
    double wheelbase;           /* l of Eq. (5) [m], > 0 */
    double sigma[2];            /* noise standard deviations per channel, >= 0 */
    double u_min[2], u_max[2];  /* control box; u + eps is clamped into it */
    double lam;                 /* softmin temperature lambda, > 0 */
    double gamma;               /* alpha = (gamma - 1) / (2 gamma) of Eq. (9), > 0 */
    double R[2];                /* diagonal control weight of Eq. (8) */
    double w_dist, w_target, w_yaw, w_speed, w_safe;   /* Eq. (18): 15, 7, 120, 5, 25 */
    double w_terminal;          /* terminal cost phi(x_T) = w_terminal * q_x(x_T); 0 = none */
    double v_ref;               /* reference speed v^r of Eq. (15) [m/s] */
    double v_max;               /* speed cap v_G on the rollouts; +inf disables it */
    double d_safe_c, d_safe_0;  /* d_safe = d_safe_c * v + d_safe_0, Eq. (16) */
    int32_t collision_only;     /* 1: c_safe only where d_obj <= 0 (Sec. IV-C, object avoidance) */
    int32_t n_ego;              /* ego circles, 0 .. MPPI_MAX_EGO */
    double ego_offset[MPPI_MAX_EGO];  /* centre offset along the heading from (x, y) [m] */
    double ego_radius[MPPI_MAX_EGO];  /* radius [m] */
    int32_t ref_mode;           /* 0: closest point of the polyline, 1: closest vertex */
    int32_t sg_enable;          /* 1: Savitzky-Golay smoothing (Eq. (19)) */
    int32_t shift;              /* 1: warm start u_t <- u*_{t+1} (receding horizon) */
    int32_t noise_bf16;         /* 1: store the noise as bfloat16 (half the bytes) */
    uint64_t seed;              /* Philox key */
    uint32_t session;           /* Philox counter word 3: independent streams per session */
    int32_t group;              /* lanes per sample in the rollout kernel: 0 = choose; 1,2,4,8,16,32 = the
                                   lanes split the search and obstacle work of each step; -2,-4,-8,-16 = that
                                   many lanes split the steps (lane p evaluates the cost of steps p, p+|g|, ...) */
    int32_t block;              /* threads per block of the rollout kernel: 0 = choose, else a multiple of 32 up to
                                   896 (the batch engine and the server take at most 448) */
    int32_t model;              /* 0: state (x, y, yaw, v), control (a, delta) with delta the steering angle;
                                   1: the steering-rate form of Eq. (5): state (x, y, yaw, v, delta),
                                   control (a, omega), delta advanced by omega * dt.  Model 1 makes x0
                                   5 entries and each row of x_out 5 entries (single-plan entry points
                                   only: the batch engine and the server run model 0). */
    int32_t cost_to_go;         /* 1: the update of step t weighs each sample by its cost from step t on
                                   (Eq. (11) read per step: S_min, softmin weights and normaliser per step);
                                   0: by its whole cost.  Single-plan entry points only. */
} mppi_params;

/* Results of one iteration. */
typedef struct {
    int32_t argmin;             /* index of the lowest-cost sample (ties: lowest index) */
    int32_t n_finite;           /* samples with a finite cost */
    double s_min;               /* lowest cost S_min */
    double eta;                 /* sum of the softmin weights exp(-(S_k - S_min) / lambda) */
    uint64_t iter;              /* iteration index used for the noise counter */
} mppi_info;

/* Fills *p with the defaults: the paper's cost weights, gamma = 1, R = lam / sigma^2,
   three ego circles of radius 1.1 m at 0, 1.35 and 2.7 m, SG on, no shift, seed 0. */
int mppi_default_params(mppi_params* p, int32_t K, int32_t T, double dt);

/* Creates a planner on CUDA device `device`.  cuda_stream is a cudaStream_t to
   queue work on (NULL: the context creates its own non-blocking stream).  The
   context owns all device buffers; they are sized here for params->K and T,
   a reference of up to max_ref vertices and max_circ circles (0: the library
   maxima); later calls do not allocate.  The nominal controls start at zero. */
int mppi_create(const mppi_params* params, int device, void* cuda_stream, int32_t max_ref,
                int32_t max_circ, mppi_ctx** out_ctx);

/* Frees every resource of the context; NULL is accepted. */
int mppi_destroy(mppi_ctx* ctx);

/* Changes the stream later work is queued on (NULL: the context's own stream). */
int mppi_set_stream(mppi_ctx* ctx, void* cuda_stream);

/* One MPPI iteration from host buffers; returns when the outputs are written.
   x0[4]          initial state (Algorithm 1 GetInitialState)
   ref_xy[n_ref][2] reference polyline vertices, n_ref >= 2 (the road model B, Eq. (3))
   circ[n_circ]   obstacle circles (Algorithm 1 ApproximateObstacles), may be NULL if 0
   centres        optional [T][n_circ][2] predicted centres per step (overrides vx, vy)
   u_out[T][2]    smoothed controls u* (Algorithm 1 SavitzkyGolayFilter)
   x_out[T+1][4]  optimal trajectory x*, x_out[0] = x0
   info           optional results record
   The warm start (the context's nominal controls) is updated in place.
   Errors: MPPI_ERR_ARG for bad sizes or non-finite inputs (nothing changes),
   MPPI_ERR_CAPACITY above the context's capacities, MPPI_ERR_NUMERIC when no
   sample cost is finite (controls unchanged, outputs not written). */
int mppi_plan(mppi_ctx* ctx, const double* x0, const double* ref_xy, int32_t n_ref,
              const mppi_circle* circ, int32_t n_circ, const double* centres,
              double* u_out, double* x_out, mppi_info* info);

/* The same iteration with every array in device memory (same layouts; circ is
   [n_circ][5] doubles).  Queued on the context's stream and returns at once
   when info is NULL; with a host info pointer it waits and reports the status.
   Non-finite device inputs turn the iteration into a no-op whose status is
   reported by the next call that waits (mppi_sync). */
int mppi_plan_device(mppi_ctx* ctx, const double* d_x0, const double* d_ref_xy, int32_t n_ref,
                     const double* d_circ, int32_t n_circ, const double* d_centres,
                     double* d_u_out, double* d_x_out, mppi_info* info);

/* ------------------------------------------------------------------------------------
   K-partitioned iteration (the multi-GPU form of one iteration).  Both sums of the update,
   Eq. (11), run over the samples, so K splits into slices, one per context (normally one per
   GPU), with two exchanges between them:
     1. mppi_slice_costs on every slice: noise, rollouts and costs of the slice's samples and
        the slice's lowest cost; the caller takes the minimum over the slices (ties: the lowest
        global index) and the sum of the finite counts;
     2. mppi_slice_sums on every slice with that global minimum: the slice's softmin normaliser
        eta = sum_k exp(-(S_k - S_min) / lambda) and its weighted noise sums
        du[t][c] = sum_k w_k eps'_{t,k,c} (binary64, not divided by eta); the caller adds them
        up over the slices;
     3. mppi_slice_finalize on every slice with the totals: u += du / eta, clamp, Savitzky-Golay
        (Eq. (19)), x* and the warm start, the same on every slice.
   A context holds the K = params->K samples k_offset .. k_offset + K - 1 of the whole plan: the
   Philox counter takes the global index, so the noise, the costs and the result do not depend
   on how the samples are split.  The sums match the unsplit iteration to the rounding of
   binary64 additions when every slice but the last holds a multiple of 2048 samples (the
   weighted sums' binary32 partials then group the same samples), otherwise to that of the
   binary32 partials.  The slices must share every parameter but K and the iteration counter
   (mppi_set_controls).  The cost-to-go form is refused (MPPI_ERR_ARG).  Errors: as for
   mppi_plan; a stage out of order is MPPI_ERR_ARG. */
int mppi_slice_costs(mppi_ctx* ctx, int64_t k_offset, const double* x0, const double* ref_xy, int32_t n_ref,
                     const mppi_circle* circ, int32_t n_circ, const double* centres, double* s_min, int32_t* argmin,
                     int32_t* n_finite);
/* s_min: the global minimum; eta and du[T][2]: this slice's sums (host outputs). */
int mppi_slice_sums(mppi_ctx* ctx, double s_min, double* eta, double* du);
/* eta, du[T][2], n_finite: the totals over all slices; s_min and argmin (global index) are
   reported in info.  u_out[T][2] and x_out[T+1][nx] as for mppi_plan. */
int mppi_slice_finalize(mppi_ctx* ctx, double eta, const double* du, int32_t n_finite, double s_min, int32_t argmin,
                        double* u_out, double* x_out, mppi_info* info);

/* Autotuner: times the rollout kernel for every lanes-per-sample group (1..32, -2..-16) and
   block size (64, 128, 256, and sizes that spread the lanes evenly over the SMs with
   1 to 4 resident blocks each, up to 896 threads) on the given inputs (host arrays, as for mppi_plan) and
   keeps the fastest for this context; *group and *block receive the choice (either
   may be NULL).  The warm start and the iteration counter are not changed.  With a
   cache_path (may be NULL) the choice is looked up first and stored after tuning,
   keyed by GPU name, K, T, n_ref, n_circ and the noise precision (one text line per
   entry).  Errors as for mppi_plan. */
int mppi_autotune(mppi_ctx* ctx, const double* x0, const double* ref_xy, int32_t n_ref,
                  const mppi_circle* circ, int32_t n_circ, const double* centres,
                  const char* cache_path, int32_t* group, int32_t* block);

/* Work counters of the rollout kernel's pruned searches for one iteration on the given
   inputs (host arrays, as for mppi_plan), summed over all samples and steps, in this
   order: range boxes tested (the vertex prefix and suffix boxes around the scanned window
   and beyond each chunk of a side walk, and the level-2 boxes of groups of 16 chunks),
   chunk boxes tested (4 segments each),
   segments evaluated, binary64 near-tie refinements, circles tested by
   the broad phase, candidate circles evaluated, and square roots taken for d_obj (one
   per candidate circle within the safety band of the nearest ego circle when the ego
   radii are equal and d_safe is constant, else one per (ego, circle) pair in the band).  Divide by K*T for
   per-rollout-step figures.  Runs an instrumented copy of the rollout kernel; the
   warm start and the iteration counter are not changed. */
#define MPPI_N_STATS 7
int mppi_rollout_stats(mppi_ctx* ctx, const double* x0, const double* ref_xy, int32_t n_ref,
                       const mppi_circle* circ, int32_t n_circ, const double* centres,
                       uint64_t* counters);

/* Waits for the context's queued work and returns the status of the last iteration. */
int mppi_sync(mppi_ctx* ctx, mppi_info* info);

/* Debug (failure-path testing without a device fault; no counterpart in the paper): the next
   iteration of the context writes these status flags into its device record between the
   rollout and the update, as a kernel that detected the condition would.  MPPI_FLAG_TIMEOUT
   makes that iteration end with MPPI_ERR_TIMEOUT (as when a bounded device wait runs out) and
   MPPI_FLAG_NONFINITE_INPUT with MPPI_ERR_ARG; either way the warm start and the iteration
   counter are left as they were and the context stays usable.  One-shot; the iteration runs
   uncaptured.  MPPI_ERR_ARG for other bits. */
#define MPPI_FLAG_NONFINITE_INPUT 1
#define MPPI_FLAG_TIMEOUT 2
int mppi_debug_inject_flags(mppi_ctx* ctx, int32_t flags);

/* Debug (no counterpart in the paper): the library built with -DMPPI_CHECKS (libmppi_checks.so)
   tests every index the rollout kernels read from the staged scene, the circle index, the
   controls and the centre table against its array's length, and the block's dynamic shared
   memory against the scene it stages; a violation is counted and the read moved to index 0, so
   nothing traps.  *enabled = 1 in that build (0 otherwise, where the checks are compiled out);
   *hits = the violations counted since the last call (then reset; 0 in the normal build).
   mppi_debug_check_selftest runs, on `device`, one kernel with two out-of-range indices and
   reports the count it leaves (2 in the checks build, 0 otherwise). */
int mppi_debug_check_hits(int32_t* enabled, uint64_t* hits);
int mppi_debug_check_selftest(int device, uint64_t* hits);

/* Warm start I/O (checkpoint / resume): U[T][2] host doubles and the iteration index. */
int mppi_set_controls(mppi_ctx* ctx, const double* U, uint64_t iter);
int mppi_get_controls(mppi_ctx* ctx, double* U, uint64_t* iter);

/* Debug / parity views of the last iteration (host outputs, waits for the stream):
   S[K] sample costs; z[T][K][2] unit normals as float (bf16 widened exactly). */
int mppi_get_costs(mppi_ctx* ctx, double* S);
int mppi_get_noise(mppi_ctx* ctx, float* z);

/* Raw Philox4x32-10 words on the device for n host counters ctr[n][4] and key
   (seed low, seed high): the generator used by the noise kernel. out[n][4]. */
int mppi_philox(uint64_t seed, const uint32_t* ctr, int32_t n, uint32_t* out);

/* Per-kernel timing with CUDA events on the context's stream (the library's own
   tracing; no effect on results).  on = 1: each iteration records MPPI_N_KERNELS + 1
   events; mppi_kernel_times() waits for the last iteration and writes the durations in
   milliseconds of its stages, in launch order: prep (scene preparation and noise, one
   launch), noise (the bfloat16 form's fix-up; empty otherwise), rollout (ends with the
   argmin), argmin (empty), weights, wsum, finalize.  An event between two kernels ends
   their chaining (the second kernel is otherwise scheduled while the first drains), so
   on = 1 lengthens the iteration.
   on = 2: only the two events around the rollout kernel; mppi_kernel_times() writes its
   duration and NaN for the others.  on = 0: off.  Other values: MPPI_ERR_ARG. */
#define MPPI_N_KERNELS 7
int mppi_set_profiling(mppi_ctx* ctx, int32_t on);
int mppi_kernel_times(mppi_ctx* ctx, float* ms, int32_t n);

/* ------------------------------------------------------------------------------------
   Batched planning: many independent iterations (different K, T, references, obstacles)
   computed together by one fixed kernel sequence captured in a CUDA graph, with one
   persistent rollout kernel over all plans' samples (the longest plans first).  Each
   plan's warm start lives in a device slot of the batch object; a plan's result does not
   depend on the other plans of its submission.  Several submissions may be in flight
   (one per pipeline); the caller must not use a slot in two submissions in flight.
   ------------------------------------------------------------------------------------ */
typedef struct mppi_batch mppi_batch;

typedef struct {
    const mppi_params* params;  /* this plan's hyper-parameters (noise_bf16 must be the batch's) */
    int32_t slot;               /* warm-start slot, 0 .. max_slots-1, distinct within a submission */
    const double* x0;           /* [4] */
    const double* ref_xy;       /* [n_ref][2] */
    int32_t n_ref;
    const mppi_circle* circ;    /* [n_circ] */
    int32_t n_circ;
    const double* centres;      /* optional [T][n_circ][2] */
    double* u_out;              /* [T][2], written by mppi_batch_wait when status is MPPI_OK */
    double* x_out;              /* [T+1][4] */
    mppi_info* info;            /* optional */
    int32_t status;             /* written by mppi_batch_wait: this plan's mppi_status */
} mppi_request;

/* Capacities: max_slots warm-start slots; at most max_batch plans, max_samples samples
   (sum of K) and max_rollout_steps rollout steps (sum of K*T) per submission; T, n_ref and
   n_circ of any plan up to max_T, max_ref, max_circ; pipelines = submissions that may be
   in flight at once (1..16).  All device and pinned memory is allocated here. */
int mppi_batch_create(int32_t max_slots, int32_t max_batch, int64_t max_samples, int64_t max_rollout_steps,
                      int32_t max_T, int32_t max_ref, int32_t max_circ, int32_t noise_bf16, int32_t pipelines,
                      int device, mppi_batch** out);
int mppi_batch_destroy(mppi_batch* batch);

/* Queues one iteration of each of the n plans (inputs are copied before it returns) on
   a free pipeline and returns its ticket; MPPI_ERR_CAPACITY when every pipeline is busy.
   mppi_batch_wait(ticket) waits and writes the outputs, status and info of every plan;
   it returns MPPI_OK, or the status of the first failed plan.  mppi_batch_plan does both. */
int mppi_batch_submit(mppi_batch* batch, mppi_request* req, int32_t n, int32_t* ticket);
int mppi_batch_wait(mppi_batch* batch, int32_t ticket);
int mppi_batch_plan(mppi_batch* batch, mppi_request* req, int32_t n);

/* Times the persistent rollout kernel for every lanes-per-sample group (1..32 splitting the
   work of each step, -2, -4, -8 splitting the steps) and block size (64, 128, 256, 448) on
   this submission's plans (without changing any slot) and keeps the fastest; *group and
   *block receive the choice (either may be NULL). */
int mppi_batch_autotune(mppi_batch* batch, mppi_request* req, int32_t n, int32_t* group, int32_t* block);

/* Sets the persistent rollout kernel's launch shape directly (e.g. a shape tuned earlier):
   group as for mppi_batch_autotune, block a multiple of 32 up to 448 holding at least 16
   samples.  MPPI_ERR_ARG for other values, MPPI_ERR_CAPACITY while a submission is in flight
   or when the shape does not fit the shared memory of a block.  No counterpart in the paper. */
int mppi_batch_set_launch(mppi_batch* batch, int32_t group, int32_t block);

/* Warm start of one slot: U[T][2] and its iteration index (the Philox counter word 2). */
int mppi_batch_set_controls(mppi_batch* batch, int32_t slot, const double* U, int32_t T, uint64_t iter);
int mppi_batch_get_controls(mppi_batch* batch, int32_t slot, double* U, int32_t T, uint64_t* iter);
/* Parity view (debug): the sample costs S[K] (Eq. (6), binary64) of plan i of the last submission
   that completed on pipeline `ticket` (the ticket mppi_batch_submit returned).  K must be that plan's
   K.  MPPI_ERR_CAPACITY while the pipeline has a submission in flight (its costs are being
   overwritten), MPPI_ERR_ARG for a plan or K the last submission did not have. */
int mppi_batch_get_costs(mppi_batch* batch, int32_t ticket, int32_t i, double* S, int32_t K);
const char* mppi_batch_last_error(mppi_batch* batch);

/* ------------------------------------------------------------------------------------
   Serving: a continuous-batching planning server for many vehicle sessions.  Requests
   arrive at any time (mppi_server_enqueue copies the inputs and returns at once).  A
   scheduler thread forms a micro-batch whenever one of the `pipelines` is free, taking
   queued requests in arrival order while their device footprint (noise K*T*8 bytes, or
   *4 with bfloat16 noise, costs and weights K*12 bytes, the scene) fits the free part of
   hbm_budget_bytes and the per-batch capacities; a session is never in two batches in
   flight, so its requests run in order against its device-resident warm start (session
   id = warm-start slot).  Up to `pipelines` batches overlap on the GPU; requests that
   arrive meanwhile join the next batch.  Results, with the latency from enqueue to
   completion, are collected with mppi_server_poll.
   ------------------------------------------------------------------------------------ */
typedef struct mppi_server mppi_server;

typedef struct {
    int32_t max_sessions;       /* sessions (and warm-start slots), ids 0 .. max_sessions-1 */
    int32_t max_batch;          /* plans per micro-batch (<= 1024) */
    int64_t max_samples;        /* sum of K per micro-batch */
    int64_t max_rollout_steps;  /* sum of K*T per micro-batch */
    int32_t max_T, max_ref, max_circ;
    int32_t pipelines;          /* micro-batches in flight at once (1..16) */
    int32_t noise_bf16;
    int32_t device;
    int64_t hbm_budget_bytes;   /* admission limit on the footprint of all requests in flight */
    double max_wait_us;         /* a batch may wait this long to grow while others run (0: never waits) */
    double watchdog_ms;         /* host-side watchdog: a micro-batch still running this long after its
                                   submission is abandoned (0: off; see mppi_server_set_watchdog) */
} mppi_server_config;

typedef struct {
    uint64_t request_id;
    int32_t session;
    int32_t status;             /* mppi_status of the plan */
    int32_t T;
    double latency_us;          /* completion - enqueue */
    double queue_us;            /* submission to the GPU - enqueue */
    mppi_info info;
} mppi_result;

int mppi_server_create(const mppi_server_config* cfg, mppi_server** out);
int mppi_server_destroy(mppi_server* server);   /* waits for the batches in flight */

/* Tunes the batch engine's rollout launch shape on n_plans copies of one request
   (the server must be idle). */
int mppi_server_autotune(mppi_server* server, const mppi_params* params, const double* x0, const double* ref_xy,
                         int32_t n_ref, const mppi_circle* circ, int32_t n_circ, int32_t n_plans,
                         int32_t* group, int32_t* block);

/* Thread-safe; the arrays are copied before it returns. */
int mppi_server_enqueue(mppi_server* server, const mppi_params* params, int32_t session, const double* x0,
                        const double* ref_xy, int32_t n_ref, const mppi_circle* circ, int32_t n_circ,
                        const double* centres, uint64_t* request_id);

/* Moves up to max completed results into out[] (waiting up to wait_ms for the first);
   with u_out / x_out (may be NULL) also their u* [max_T][2] and x* [max_T+1][4] per result.
   A result whose T exceeds max_T while u_out or x_out is given has status MPPI_ERR_CAPACITY
   and its rows are not written (its info is). */
int mppi_server_poll(mppi_server* server, mppi_result* out, int32_t max, double* u_out, double* x_out,
                     int32_t max_T, int32_t wait_ms, int32_t* n_out);

/* Queue depth, requests in flight, micro-batches submitted and plans completed so far. */
int mppi_server_pending(mppi_server* server, int32_t* queued, int32_t* in_flight, uint64_t* batches,
                        uint64_t* plans);

/* Warm start of an idle session (checkpoint / resume). */
int mppi_server_set_controls(mppi_server* server, int32_t session, const double* U, int32_t T, uint64_t iter);

/* Host-side watchdog (no counterpart in the paper): a micro-batch still running watchdog_ms
   after its submission is abandoned.  Its requests complete at once with MPPI_ERR_TIMEOUT
   (latency stamped then, u* and x* not given); the device work cannot be stopped, so their
   sessions, HBM budget and pipeline stay taken until it has ended, when its results are dropped
   (the sessions' warm starts are what that work left).  0 turns the watchdog off.
   mppi_server_timeouts gives the number of requests completed that way so far. */
int mppi_server_set_watchdog(mppi_server* server, double watchdog_ms);
int mppi_server_timeouts(mppi_server* server, uint64_t* n);

/* Session table to and from a file (checkpoint / resume of every session's warm start and
   iteration counter; no counterpart in the paper): the server must be idle (no request queued
   or in flight), else MPPI_ERR_CAPACITY.  The file holds "MPPISNAP", version 1, max_sessions,
   max_T, then per session its counter and U[max_T][2] in this host's byte order; restore
   refuses (MPPI_ERR_ARG) a file of another size or version, or a truncated one. */
int mppi_server_snapshot(mppi_server* server, const char* path);
int mppi_server_restore(mppi_server* server, const char* path);
const char* mppi_server_last_error(mppi_server* server);

/* Allocation-free lowest-cost search.  The paper has no counterpart: this is a
   service for callers that cannot allocate GPU memory while they plan, such as a
   vehicle control cycle that must not stall on cudaMalloc (which can synchronise
   the device or fail under memory pressure) or software that may only use memory
   reserved at start-up.  It does what the argmin step of mppi_plan does, on device
   costs d_S[K] (binary64, caller-owned): *d_s_min = the lowest finite cost,
   *d_argmin = its index (ties: lowest index; -1 if none is finite), *d_n_finite =
   the number of finite costs (all three caller-owned device memory).  The work is
   queued on cuda_stream (NULL: the legacy default stream); wait on it before
   reading the outputs.
   Its scratch is a fixed 16 KB array inside the library, reserved on every GPU that
   loads the library until the process exits; nothing is allocated per call.  The
   first call on a device looks up that array's device address (once per device,
   with the device current): make that first call before any stream capture.  All
   calls on a device share the array, so calls that may overlap on the GPU (on
   different streams without ordering) race; serialise them.
   Errors are returned as status codes only (no message is stored, since storing
   one could allocate): MPPI_ERR_ARG for NULL pointers or K < 1, MPPI_ERR_CAPACITY
   for K > MPPI_NOALLOC_MAX_K, MPPI_ERR_CUDA when a CUDA call fails. */
#define MPPI_NOALLOC_MAX_K (1 << 28)
int mppi_argmin_noalloc(const double* d_S, int32_t K, double* d_s_min, int32_t* d_argmin,
                        int32_t* d_n_finite, void* cuda_stream);

const char* mppi_status_string(int status);
const char* mppi_last_error(mppi_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* MPPI_H */
