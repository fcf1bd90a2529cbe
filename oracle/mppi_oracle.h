/*
 * mppi_oracle.h - plain, slow FP64 CPU oracle of one MPPI iteration.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this code.  It shares no source, header,
 * table or helper with the CUDA library; the two meet only in the seeded
 * inputs they both read.
 *
 * Paper: Testouri, Elghazaly, Frank, "Towards a Safe Real-Time Motion Planning
 * Framework for Autonomous Driving Systems: A Model Predictive Path Integral
 * Approach" (arXiv 2308.01654).  Each function cites the passage it follows:
 *   Eq. (1)    stochastic dynamics x_{t+1} = F(x_t, u_t + eps_t), eps ~ N(0, Sigma)
 *   Eq. (5)    kinematic bicycle model
 *   Eq. (6)-(9) trajectory cost, running cost split, control cost, alpha(gamma)
 *   Eq. (11)   min-shifted softmin update of the input sequence
 *   Eq. (12)-(18) the five step costs, the safe distance and the weighted total
 *   Eq. (19)   5-point Savitzky-Golay filter
 *   Algorithm 1 the iteration: noise, parallel rollouts, min, update, smoothing,
 *              optimal rollout, warm-start shift
 * (equation numbers count the paper's numbered displays in order)
 *
 * Arithmetic is IEEE double throughout; loops are scalar and in index order;
 * the nearest-segment search is a global brute force.
 */
#ifndef MPPI_ORACLE_H
#define MPPI_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_EGO 8

typedef struct {
    int32_t K, T;
    double dt, wheelbase;
    double sigma[2], u_min[2], u_max[2];   /* channel 0 = acceleration a, 1 = steering delta */
    double lam, gamma, R[2];               /* R is diagonal */
    double w_dist, w_target, w_yaw, w_speed, w_safe, w_terminal;
    double v_ref, v_max;                   /* v_max = +inf disables the speed cap */
    double d_safe_c, d_safe_0;
    int32_t collision_only;
    int32_t n_ego;
    double ego_offset[ORC_MAX_EGO], ego_radius[ORC_MAX_EGO];
    int32_t ref_mode;                      /* 0 = nearest point on segment, 1 = nearest vertex */
    int32_t sg_enable, shift, noise_bf16;
    uint64_t seed;
    uint32_t session;
    int32_t model;                         /* 0: state (x, y, yaw, v), control (a, delta);
                                              1: state (x, y, yaw, v, delta), control (a, omega) */
    int32_t cost_to_go;                    /* 1: the update of step t weighs each sample by the cost
                                              still to come from step t (Eq. (11) read per step) */
} orc_params;

/* state entries of a model: 4 or 5 */
#define ORC_NX(p) ((p)->model == 1 ? 5 : 4)

typedef struct { double x, y, r, vx, vy; } orc_circle;

typedef struct {
    int32_t argmin;
    int32_t n_finite;
    double s_min;
    double eta;
} orc_info;

/* ---- noise (Algorithm 1, GenerateRandomNoise; Eq. (1) eps ~ N(0, Sigma)) ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform24(uint32_t word);
void orc_box_muller(double u0, double u1, double* z0, double* z1);
double orc_round_bf16(double z);
/* z[(t*K + k)*2 + c], unit normals (not yet scaled by sigma) */
void orc_noise(const orc_params* p, uint32_t iter, double* z);

/* ---- dynamics (Eq. (5), explicit Euler) ---- */
void orc_bicycle_step(const double x[4], double a, double delta, double dt, double wheelbase,
                      double out[4]);
/* the steering-rate form: the steering angle is the fifth state, driven by omega */
void orc_bicycle5_step(const double x[5], double a, double omega, double dt, double wheelbase,
                       double out[5]);

/* ---- cost pieces (Sec. IV-C, Eq. (12)-(18)) ---- */
/* Closest reference point to (px,py); returns squared distance, the winning segment
   (or vertex) index and the reference yaw.  *margin_m receives how far (metres) the
   point is from a place where the reference yaw would switch. */
double orc_nearest_ref(const double* ref_xy, int32_t n_ref, int32_t mode, double px, double py,
                       int32_t* idx, double* theta_r, double* margin_m);
double orc_wrap_angle(double d);
/* d_obj of Eq. (16) for the ego circles of state x against the circle centres at one step */
double orc_obstacle_distance(const orc_params* p, const double x[4], const orc_circle* circ,
                             const double* centres_xy, int32_t n_circ);

/* ---- one sample's trajectory cost S(tau_m) (Eq. (6), Algorithm 1 inner loop) ----
   z_k[t*2 + c] are this sample's unit normals; U[t*2 + c] the nominal controls.
   eps_out (optional) receives eps'_t = clamp(u_t + sigma*z_t) - u_t, [T][2].
   margin (optional) receives the smallest discontinuity margin seen along the rollout. */
double orc_rollout_cost(const orc_params* p, const double x0[4], const double* U, const double* z_k,
                        const double* ref_xy, int32_t n_ref, const orc_circle* circ, int32_t n_circ,
                        const double* centres, double* eps_out, double* margin);
/* The same with the cost from every step on: ctg[t] = sum of the step costs s >= t plus the
   terminal cost (ctg[0] is the returned S up to summation order). */
double orc_rollout_cost_ctg(const orc_params* p, const double x0[4], const double* U, const double* z_k,
                            const double* ref_xy, int32_t n_ref, const orc_circle* circ, int32_t n_circ,
                            const double* centres, double* eps_out, double* margin, double* ctg);

/* ---- update (Eq. (11)), smoothing (Eq. (19)) and optimal rollout ---- */
/* eps[(t*K + k)*2 + c]; dU[t*2 + c] = sum_k w_k eps'_{t,k} / eta.  Returns n_finite. */
int32_t orc_softmin_update(int32_t K, int32_t T, const double* S, const double* eps, double lam,
                           double* dU, orc_info* info, double* weights);
/* Eq. (11) with a per-step cost: Sctg[t*K + k] is sample k's cost from step t on; each step
   gets its own S_min and softmin weights.  eta_t[T] (optional) receives the normalisers.
   Returns the number of samples whose total cost Sctg[0][k] is finite. */
int32_t orc_softmin_update_ctg(int32_t K, int32_t T, const double* Sctg, const double* eps, double lam,
                               double* dU, double* eta_t);
void orc_savgol5(int32_t T, const double* u_in, int32_t stride, double* u_out);
void orc_rollout_states(const orc_params* p, const double x0[4], const double* u, double* xs);

/* ---- one full MPPI iteration (Algorithm 1, one pass of the while loop) ----
   U: in/out nominal controls [T][2] (the warm start).  u_star [T][2], x_star [T+1][NX]
   (NX = 4, or 5 for model 1; x0 has NX entries).
   S_out [K], margin_out [K], eps_out [T][K][2] optional (NULL to skip).
   Returns 0 on success, -1 on invalid arguments, -4 when no sample cost is finite
   (U is left unchanged then). */
int orc_plan(const orc_params* p, uint32_t iter, const double x0[4],
             const double* ref_xy, int32_t n_ref, const orc_circle* circ, int32_t n_circ,
             const double* centres, double* U, double* u_star, double* x_star,
             double* S_out, double* margin_out, double* eps_out, orc_info* info);

/* Sample costs only for samples [k0, k0+count): the bounded CPU baseline. */
int orc_costs_range(const orc_params* p, uint32_t iter, const double x0[4], const double* U,
                    const double* ref_xy, int32_t n_ref, const orc_circle* circ, int32_t n_circ,
                    const double* centres, int32_t k0, int32_t count, double* S_out);

int orc_num_threads(void);
void orc_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
