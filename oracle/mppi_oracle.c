/*
 * mppi_oracle.c - plain FP64 CPU oracle of one MPPI iteration (arXiv 2308.01654).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline leg of the benchmark, never by the library.  It shares no code with
 * the CUDA path.  Every step is written in the paper's order (Algorithm 1) in
 * double precision with scalar loops; reductions run serially in index order.
 * OpenMP may split the *independent* per-sample rollouts across threads; that
 * does not change any result.
 *
 * Readings of points the paper leaves open (each is listed in the design notes):
 *  - noise: Philox4x32-10 (Salmon et al., SC'11), key = seed, counter =
 *    (floor(t/2), k, iter, session); uniform u = ((w >> 8) | 1) * 2^-24;
 *    Box-Muller; even t use words 0,1, odd t words 2,3;
 *  - Sigma holds standard deviations (Table I lists sigma values);
 *  - "checks the generated noise" (Sec. III-A): u + eps is clamped to the
 *    control box and eps' = clamp(u + eps) - u is used everywhere after;
 *  - dynamics: explicit Euler on Eq. (5) with (x, y, yaw, v) and control
 *    (a, delta); every right-hand side is evaluated at x_t;
 *  - state cost on x_{t+1}; c_target compares P_{t+1} with P_t (P_0 = x0);
 *  - closest waypoint = closest point of the polyline (segment projection),
 *    ties to the lowest segment; reference yaw = that segment's direction;
 *    target point = last vertex;
 *  - yaw error wrapped as d - 2*pi*rint(d / 2*pi);
 *  - ego circles at offsets along the heading; d_obj = min over ego circle e
 *    and obstacle circle k of |E_e - O_k| - r_k - r_e;
 *  - softmin over the total trajectory cost S_m (Eq. (11) with the tilde-t
 *    index read as the whole-trajectory cost); non-finite costs weigh 0;
 *  - u + du is clamped, Savitzky-Golay with replicated edges, clamped again;
 *  - warm start: u_t <- u*_{t+1}, last entry repeated.
 */
#include "mppi_oracle.h"

#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double ORC_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------ */
/* Noise: Algorithm 1 "GenerateRandomNoise(Sigma)", eps ~ N(0, Sigma) of Eq. (1) */
/* ------------------------------------------------------------------------ */

/* Philox4x32 with 10 rounds, as published by Salmon, Moraes, Dror and Shaw
   ("Parallel random numbers: as easy as 1, 2, 3", SC'11): each round multiplies
   counter words 0 and 2 by two odd constants, and the new counter is formed from
   the high/low halves of those products XORed with words 1 and 3 and the round
   key; the key is advanced by the two Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Top 24 bits of a word, forced odd, scaled by 2^-24: a value in (0, 1) that is
   exact in both binary32 and binary64. */
double orc_uniform24(uint32_t word)
{
    return (double)((word >> 8) | 1u) * (1.0 / 16777216.0);
}

/* Box-Muller: two independent uniforms -> two independent standard normals. */
void orc_box_muller(double u0, double u1, double* z0, double* z1)
{
    double r = sqrt(-2.0 * log(u0));
    double ang = 2.0 * ORC_PI * u1;
    *z0 = r * cos(ang);
    *z1 = r * sin(ang);
}

/* Round to the nearest bfloat16 value (8 significant bits), ties to even. */
double orc_round_bf16(double z)
{
    if (z == 0.0 || !isfinite(z)) return z;
    int e;
    double m = frexp(z, &e);          /* z = m * 2^e, 0.5 <= |m| < 1 */
    double q = rint(m * 256.0);       /* 8 significant bits, default mode = ties-to-even */
    return ldexp(q, e - 8);
}

void orc_noise(const orc_params* p, uint32_t iter, double* z)
{
    const uint32_t key[2] = {(uint32_t)(p->seed & 0xFFFFFFFFu), (uint32_t)(p->seed >> 32)};
    for (int32_t t = 0; t < p->T; ++t) {
        for (int32_t k = 0; k < p->K; ++k) {
            uint32_t ctr[4] = {(uint32_t)(t / 2), (uint32_t)k, iter, p->session};
            uint32_t w[4];
            orc_philox4x32_10(ctr, key, w);
            uint32_t wa = (t % 2 == 0) ? w[0] : w[2];
            uint32_t wb = (t % 2 == 0) ? w[1] : w[3];
            double z0, z1;
            orc_box_muller(orc_uniform24(wa), orc_uniform24(wb), &z0, &z1);
            if (p->noise_bf16) {
                z0 = orc_round_bf16(z0);
                z1 = orc_round_bf16(z1);
            }
            size_t i = ((size_t)t * (size_t)p->K + (size_t)k) * 2;
            z[i] = z0;
            z[i + 1] = z1;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Dynamics: Eq. (5) kinematic bicycle, one explicit Euler step               */
/* ------------------------------------------------------------------------ */

void orc_bicycle_step(const double x[4], double a, double delta, double dt, double wheelbase,
                      double out[4])
{
    double px = x[0], py = x[1], yaw = x[2], v = x[3];
    double dx = v * cos(yaw);
    double dy = v * sin(yaw);
    double dyaw = v * tan(delta) / wheelbase;
    double dv = a;
    out[0] = px + dx * dt;
    out[1] = py + dy * dt;
    out[2] = yaw + dyaw * dt;
    out[3] = v + dv * dt;
}

/* Eq. (5) with the steering angle as the fifth state and the steering rate omega as the
   second control: every right-hand side at x_t, delta advanced by omega * dt. */
void orc_bicycle5_step(const double x[5], double a, double omega, double dt, double wheelbase,
                       double out[5])
{
    orc_bicycle_step(x, a, x[4], dt, wheelbase, out);
    out[4] = x[4] + omega * dt;
}

static double clampd(double v, double lo, double hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

/* Optional speed cap v_G (Sec. III-A lists the target speed among the checked
   constraints): the acceleration may not take v above v_max within one step. */
static double capped_accel(const orc_params* p, double a, double v)
{
    if (isfinite(p->v_max)) {
        double lim = (p->v_max - v) / p->dt;
        if (a > lim) a = lim;
        if (a < p->u_min[0]) a = p->u_min[0];
    }
    return a;
}

/* ------------------------------------------------------------------------ */
/* Cost pieces: Sec. IV-C, Eq. (12)-(18)                                      */
/* ------------------------------------------------------------------------ */

double orc_wrap_angle(double d)
{
    return d - 2.0 * ORC_PI * rint(d / (2.0 * ORC_PI));
}

/* Closest point of segment i to (px,py) and its squared distance; *tau receives
   the unclamped projection parameter and *len the segment length. */
static double seg_dist2(const double* ref, int32_t i, double px, double py, double* qx, double* qy,
                        double* tau, double* len)
{
    double ax = ref[2 * i], ay = ref[2 * i + 1];
    double bx = ref[2 * i + 2], by = ref[2 * i + 3];
    double ex = bx - ax, ey = by - ay;
    double l2 = ex * ex + ey * ey;
    double s = 0.0;
    if (l2 > 0.0) s = ((px - ax) * ex + (py - ay) * ey) / l2;
    *tau = s;
    *len = sqrt(l2);
    if (s <= 0.0) {
        *qx = ax; *qy = ay;
    } else if (s >= 1.0) {
        *qx = bx; *qy = by;
    } else {
        *qx = ax + s * ex; *qy = ay + s * ey;
    }
    double dx = px - *qx, dy = py - *qy;
    return dx * dx + dy * dy;
}

static double seg_heading(const double* ref, int32_t i)
{
    return atan2(ref[2 * i + 3] - ref[2 * i + 1], ref[2 * i + 2] - ref[2 * i]);
}

/* Eq. (12) needs the closest waypoint W_t; Eq. (14) its reference yaw. */
double orc_nearest_ref(const double* ref, int32_t n_ref, int32_t mode, double px, double py,
                       int32_t* idx, double* theta_r, double* margin_m)
{
    double best = INFINITY;
    int32_t bi = 0;
    if (mode == 0) {
        for (int32_t i = 0; i + 1 < n_ref; ++i) {
            double qx, qy, tau, len;
            double d2 = seg_dist2(ref, i, px, py, &qx, &qy, &tau, &len);
            if (d2 < best) {
                best = d2;
                bi = i;
            }
        }
        double th = seg_heading(ref, bi);
        if (margin_m) {
            /* Distance the point may move before a segment of another heading wins:
               first-order distance to the set where the two distances tie,
               (d_j - d_i) / |grad d_j - grad d_i|, with grad d the unit vector from the
               closest point to P.  Two segments clamped to one shared vertex tie
               exactly; that tie only ends where one of the clamps releases. */
            double bqx, bqy, btau, blen;
            seg_dist2(ref, bi, px, py, &bqx, &bqy, &btau, &blen);
            double dbest = sqrt(best);
            double gbx = dbest > 0.0 ? (px - bqx) / dbest : 0.0;
            double gby = dbest > 0.0 ? (py - bqy) / dbest : 0.0;
            double m = INFINITY;
            for (int32_t i = 0; i + 1 < n_ref; ++i) {
                if (i == bi || seg_heading(ref, i) == th) continue;
                double qx, qy, tau, len;
                double d2 = seg_dist2(ref, i, px, py, &qx, &qy, &tau, &len);
                double mi;
                if (qx == bqx && qy == bqy) {
                    double mt = (tau <= 0.0) ? -tau * len : (tau - 1.0) * len;
                    double mb = (btau <= 0.0) ? -btau * blen : (btau >= 1.0 ? (btau - 1.0) * blen : 0.0);
                    mi = fmin(fabs(mt), fabs(mb));
                } else {
                    double d = sqrt(d2);
                    double gx = d > 0.0 ? (px - qx) / d : 0.0, gy = d > 0.0 ? (py - qy) / d : 0.0;
                    double gn = sqrt((gx - gbx) * (gx - gbx) + (gy - gby) * (gy - gby));
                    mi = gn > 0.0 ? (d - dbest) / gn : INFINITY;
                }
                if (mi < m) m = mi;
            }
            *margin_m = m;
        }
        *idx = bi;
        *theta_r = th;
        return best;
    }
    /* mode 1: closest vertex; yaw of its outgoing segment (incoming for the last vertex) */
    for (int32_t j = 0; j < n_ref; ++j) {
        double dx = px - ref[2 * j], dy = py - ref[2 * j + 1];
        double d2 = dx * dx + dy * dy;
        if (d2 < best) {
            best = d2;
            bi = j;
        }
    }
    int32_t sj = bi < n_ref - 1 ? bi : n_ref - 2;
    double th = seg_heading(ref, sj);
    if (margin_m) {
        double dbest = sqrt(best);
        double bx = px - ref[2 * bi], by = py - ref[2 * bi + 1];
        double gbx = dbest > 0.0 ? bx / dbest : 0.0, gby = dbest > 0.0 ? by / dbest : 0.0;
        double m = INFINITY;
        for (int32_t j = 0; j < n_ref; ++j) {
            int32_t s = j < n_ref - 1 ? j : n_ref - 2;
            if (j == bi || seg_heading(ref, s) == th) continue;
            double dx = px - ref[2 * j], dy = py - ref[2 * j + 1];
            double d = sqrt(dx * dx + dy * dy);
            double gx = d > 0.0 ? dx / d : 0.0, gy = d > 0.0 ? dy / d : 0.0;
            double gn = sqrt((gx - gbx) * (gx - gbx) + (gy - gby) * (gy - gby));
            double mi = gn > 0.0 ? (d - dbest) / gn : INFINITY;
            if (mi < m) m = mi;
        }
        *margin_m = m;
    }
    *idx = bi;
    *theta_r = th;
    return best;
}

/* Eq. (16): d_obj, the smallest clearance between any ego circle and any obstacle circle. */
double orc_obstacle_distance(const orc_params* p, const double x[4], const orc_circle* circ,
                             const double* centres_xy, int32_t n_circ)
{
    double dmin = INFINITY;
    for (int32_t e = 0; e < p->n_ego; ++e) {
        double ex = x[0] + p->ego_offset[e] * cos(x[2]);
        double ey = x[1] + p->ego_offset[e] * sin(x[2]);
        for (int32_t k = 0; k < n_circ; ++k) {
            double cx = centres_xy[2 * k], cy = centres_xy[2 * k + 1];
            double d = sqrt((ex - cx) * (ex - cx) + (ey - cy) * (ey - cy)) - circ[k].r - p->ego_radius[e];
            if (d < dmin) dmin = d;
        }
    }
    return dmin;
}

/* Obstacle centres at step index s (= t + 1): the per-step table if given, else
   constant-velocity motion O_k + V_k * s * dt (the dynamic obstacles O^d(t) of Eq. (2)). */
static void centres_at(const orc_params* p, const orc_circle* circ, int32_t n_circ,
                       const double* centres, int32_t t, double* out)
{
    for (int32_t k = 0; k < n_circ; ++k) {
        if (centres) {
            out[2 * k] = centres[((size_t)t * n_circ + k) * 2];
            out[2 * k + 1] = centres[((size_t)t * n_circ + k) * 2 + 1];
        } else {
            double s = (double)(t + 1) * p->dt;
            out[2 * k] = circ[k].x + circ[k].vx * s;
            out[2 * k + 1] = circ[k].y + circ[k].vy * s;
        }
    }
}

/* State-dependent step cost q_x on x_{t+1} (Eq. (12)-(18)); P_t is the previous position. */
static double state_cost(const orc_params* p, const double xn[4], double prev_x, double prev_y,
                         const double* ref, int32_t n_ref, const orc_circle* circ, int32_t n_circ,
                         const double* cxy, double* margin)
{
    int32_t idx;
    double theta_r, m_ref;
    double c_dist = orc_nearest_ref(ref, n_ref, p->ref_mode, xn[0], xn[1], &idx, &theta_r,
                                    margin ? &m_ref : NULL);                        /* Eq. (12) */
    double tx = ref[2 * (n_ref - 1)], ty = ref[2 * (n_ref - 1) + 1];
    double dn = (xn[0] - tx) * (xn[0] - tx) + (xn[1] - ty) * (xn[1] - ty);
    double dp = (prev_x - tx) * (prev_x - tx) + (prev_y - ty) * (prev_y - ty);
    double c_target = dn > dp ? 1.0 : 0.0;                                           /* Eq. (13) */
    double dyaw = orc_wrap_angle(xn[2] - theta_r);
    double c_yaw = dyaw * dyaw;                                                      /* Eq. (14) */
    double c_speed = (xn[3] - p->v_ref) * (xn[3] - p->v_ref);                        /* Eq. (15) */
    double d_obj = orc_obstacle_distance(p, xn, circ, cxy, n_circ);                  /* Eq. (16) */
    double d_safe = p->d_safe_c * xn[3] + p->d_safe_0;
    double gap = d_safe - d_obj;
    double c_safe = gap > 0.0 ? gap * gap : 0.0;                                     /* Eq. (17) */
    if (p->collision_only && !(d_obj <= 0.0)) c_safe = 0.0;
    if (margin) {
        double m = m_ref;
        double mt = 0.5 * fabs(sqrt(dn) - sqrt(dp));
        if (mt < m) m = mt;
        double h = fabs(orc_wrap_angle(xn[2] - theta_r));
        double mw = ORC_PI - h;           /* distance of the yaw error from the wrap at +-pi */
        if (mw < m) m = mw;
        if (p->collision_only && fabs(d_obj) < m) m = fabs(d_obj);
        if (m < *margin) *margin = m;
    }
    return p->w_dist * c_dist + p->w_target * c_target + p->w_yaw * c_yaw + p->w_speed * c_speed +
           p->w_safe * c_safe;                                                       /* Eq. (18) */
}

/* Eq. (8)-(9): q_u = alpha eps^T R u + u^T R eps + 1/2 u^T R u, R diagonal. */
static double control_cost(const orc_params* p, const double u[2], const double ep[2])
{
    double alpha = (p->gamma - 1.0) / (2.0 * p->gamma);
    double eRu = ep[0] * p->R[0] * u[0] + ep[1] * p->R[1] * u[1];
    double uRe = u[0] * p->R[0] * ep[0] + u[1] * p->R[1] * ep[1];
    double uRu = u[0] * p->R[0] * u[0] + u[1] * p->R[1] * u[1];
    return alpha * eRu + uRe + 0.5 * uRu;
}

/* Algorithm 1, inner loop for one sample m: roll out F(x_t, u_t + eps_t) and add up
   the running cost (Eq. (6)-(7)), then the terminal cost. */
double orc_rollout_cost(const orc_params* p, const double x0[4], const double* U, const double* z_k,
                        const double* ref, int32_t n_ref, const orc_circle* circ, int32_t n_circ,
                        const double* centres, double* eps_out, double* margin)
{
    return orc_rollout_cost_ctg(p, x0, U, z_k, ref, n_ref, circ, n_circ, centres, eps_out, margin, NULL);
}

double orc_rollout_cost_ctg(const orc_params* p, const double x0[4], const double* U, const double* z_k,
                            const double* ref, int32_t n_ref, const orc_circle* circ, int32_t n_circ,
                            const double* centres, double* eps_out, double* margin, double* ctg)
{
    double x[5] = {x0[0], x0[1], x0[2], x0[3], p->model == 1 ? x0[4] : 0.0};
    double prev_x = x0[0], prev_y = x0[1];
    double* cxy = n_circ > 0 ? (double*)malloc(sizeof(double) * 2 * (size_t)n_circ) : NULL;
    double S = 0.0, last_qx = 0.0;
    if (margin) *margin = INFINITY;
    for (int32_t t = 0; t < p->T; ++t) {
        const double u[2] = {U[2 * t], U[2 * t + 1]};
        double v[2], ep[2];
        for (int c = 0; c < 2; ++c) {
            double eps = p->sigma[c] * z_k[2 * t + c];
            v[c] = clampd(u[c] + eps, p->u_min[c], p->u_max[c]);
            ep[c] = v[c] - u[c];
        }
        if (eps_out) {
            eps_out[2 * t] = ep[0];
            eps_out[2 * t + 1] = ep[1];
        }
        double a = capped_accel(p, v[0], x[3]);
        double xn[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        if (p->model == 1)
            orc_bicycle5_step(x, a, v[1], p->dt, p->wheelbase, xn);
        else
            orc_bicycle_step(x, a, v[1], p->dt, p->wheelbase, xn);
        centres_at(p, circ, n_circ, centres, t, cxy);
        double qx = state_cost(p, xn, prev_x, prev_y, ref, n_ref, circ, n_circ, cxy, margin);
        double qu = control_cost(p, u, ep);
        S += qx + qu;
        if (ctg) ctg[t] = qx + qu;          /* step costs for now, summed from the end below */
        last_qx = qx;
        prev_x = xn[0];
        prev_y = xn[1];
        memcpy(x, xn, sizeof(x));
    }
    S += p->w_terminal * last_qx;       /* phi(x_T) */
    if (ctg) {
        double acc = p->w_terminal * last_qx;
        for (int32_t t = p->T - 1; t >= 0; --t) {
            acc += ctg[t];
            ctg[t] = acc;
        }
    }
    free(cxy);
    return S;
}

/* ------------------------------------------------------------------------ */
/* Update, smoothing, optimal rollout                                          */
/* ------------------------------------------------------------------------ */

/* Algorithm 1 after the rollouts: S_min, then Eq. (11) for every t. */
int32_t orc_softmin_update(int32_t K, int32_t T, const double* S, const double* eps, double lam,
                           double* dU, orc_info* info, double* weights)
{
    double smin = INFINITY;
    int32_t arg = -1, n_fin = 0;
    for (int32_t k = 0; k < K; ++k) {
        if (!isfinite(S[k])) continue;
        ++n_fin;
        if (S[k] < smin) {
            smin = S[k];
            arg = k;
        }
    }
    if (info) {
        info->argmin = arg;
        info->n_finite = n_fin;
        info->s_min = smin;
        info->eta = 0.0;
    }
    if (n_fin == 0) return 0;
    double* w = weights ? weights : (double*)malloc(sizeof(double) * (size_t)K);
    double eta = 0.0;
    for (int32_t k = 0; k < K; ++k) {
        w[k] = isfinite(S[k]) ? exp(-(S[k] - smin) / lam) : 0.0;
        eta += w[k];
    }
    for (int32_t t = 0; t < T; ++t) {
        for (int c = 0; c < 2; ++c) {
            double num = 0.0;
            for (int32_t k = 0; k < K; ++k) num += w[k] * eps[((size_t)t * K + k) * 2 + c];
            dU[2 * t + c] = num / eta;
        }
    }
    if (info) info->eta = eta;
    if (!weights) free(w);
    return n_fin;
}

/* Eq. (11) read per step: at each t the weights come from the cost still to come. */
int32_t orc_softmin_update_ctg(int32_t K, int32_t T, const double* Sctg, const double* eps, double lam,
                               double* dU, double* eta_t)
{
    int32_t n_fin = 0;
    for (int32_t k = 0; k < K; ++k)
        if (isfinite(Sctg[k])) ++n_fin;
    for (int32_t t = 0; t < T; ++t) {
        const double* St = Sctg + (size_t)t * K;
        double smin = INFINITY;
        for (int32_t k = 0; k < K; ++k)
            if (isfinite(St[k]) && St[k] < smin) smin = St[k];
        double eta = 0.0, num[2] = {0.0, 0.0};
        if (isfinite(smin)) {
            for (int32_t k = 0; k < K; ++k) {
                const double w = isfinite(St[k]) ? exp(-(St[k] - smin) / lam) : 0.0;
                eta += w;
                for (int c = 0; c < 2; ++c) num[c] += w * eps[((size_t)t * K + k) * 2 + c];
            }
        }
        for (int c = 0; c < 2; ++c) dU[2 * t + c] = eta > 0.0 ? num[c] / eta : 0.0;
        if (eta_t) eta_t[t] = eta;
    }
    return n_fin;
}

/* Eq. (19): u*_t = (-3 u_{t-2} + 12 u_{t-1} + 17 u_t + 12 u_{t+1} - 3 u_{t+2}) / 35,
   indices outside [0, T-1] replaced by the nearest end. */
void orc_savgol5(int32_t T, const double* u_in, int32_t stride, double* u_out)
{
    static const double coef[5] = {-3.0, 12.0, 17.0, 12.0, -3.0};
    for (int32_t t = 0; t < T; ++t) {
        double acc = 0.0;
        for (int j = -2; j <= 2; ++j) {
            int32_t s = t + j;
            if (s < 0) s = 0;
            if (s > T - 1) s = T - 1;
            acc += coef[j + 2] * u_in[(size_t)s * stride];
        }
        u_out[(size_t)t * stride] = acc / 35.0;
    }
}

/* Algorithm 1: x*_{t+1} = F(x*_t, u*_t), noise free. xs is [T+1][NX]. */
void orc_rollout_states(const orc_params* p, const double x0[4], const double* u, double* xs)
{
    const int nx = ORC_NX(p);
    memcpy(xs, x0, (size_t)nx * sizeof(double));
    for (int32_t t = 0; t < p->T; ++t) {
        double a = capped_accel(p, u[2 * t], xs[nx * t + 3]);
        if (nx == 5)
            orc_bicycle5_step(xs + 5 * t, a, u[2 * t + 1], p->dt, p->wheelbase, xs + 5 * (t + 1));
        else
            orc_bicycle_step(xs + 4 * t, a, u[2 * t + 1], p->dt, p->wheelbase, xs + 4 * (t + 1));
    }
}

static int all_finite(const double* v, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!isfinite(v[i])) return 0;
    return 1;
}

static int validate(const orc_params* p, const double x0[4], const double* ref, int32_t n_ref,
                    const orc_circle* circ, int32_t n_circ, const double* centres, const double* U)
{
    if (!p || p->K < 1 || p->T < 1 || n_ref < 2 || n_circ < 0) return -1;
    if (!(p->dt > 0.0) || !(p->lam > 0.0) || !(p->wheelbase > 0.0) || !(p->gamma > 0.0)) return -1;
    if (p->n_ego < 0 || p->n_ego > ORC_MAX_EGO) return -1;
    if (p->model != 0 && p->model != 1) return -1;
    for (int c = 0; c < 2; ++c)
        if (!(p->sigma[c] >= 0.0) || !(p->u_min[c] <= p->u_max[c])) return -1;
    if (!all_finite(x0, (size_t)ORC_NX(p)) || !all_finite(ref, 2 * (size_t)n_ref) || !all_finite(U, 2 * (size_t)p->T))
        return -1;
    if (n_circ > 0 && !all_finite((const double*)circ, 5 * (size_t)n_circ)) return -1;
    if (centres && !all_finite(centres, (size_t)p->T * n_circ * 2)) return -1;
    return 0;
}

int orc_costs_range(const orc_params* p, uint32_t iter, const double x0[4], const double* U,
                    const double* ref, int32_t n_ref, const orc_circle* circ, int32_t n_circ,
                    const double* centres, int32_t k0, int32_t count, double* S_out)
{
    if (validate(p, x0, ref, n_ref, circ, n_circ, centres, U)) return -1;
    if (k0 < 0 || count < 0 || k0 + count > p->K) return -1;
    const uint32_t key[2] = {(uint32_t)(p->seed & 0xFFFFFFFFu), (uint32_t)(p->seed >> 32)};
#pragma omp parallel for schedule(dynamic, 4)
    for (int32_t j = 0; j < count; ++j) {
        int32_t k = k0 + j;
        double* zk = (double*)malloc(sizeof(double) * 2 * (size_t)p->T);
        for (int32_t t = 0; t < p->T; ++t) {
            uint32_t ctr[4] = {(uint32_t)(t / 2), (uint32_t)k, iter, p->session};
            uint32_t w[4];
            orc_philox4x32_10(ctr, key, w);
            uint32_t wa = (t % 2 == 0) ? w[0] : w[2];
            uint32_t wb = (t % 2 == 0) ? w[1] : w[3];
            orc_box_muller(orc_uniform24(wa), orc_uniform24(wb), &zk[2 * t], &zk[2 * t + 1]);
            if (p->noise_bf16) {
                zk[2 * t] = orc_round_bf16(zk[2 * t]);
                zk[2 * t + 1] = orc_round_bf16(zk[2 * t + 1]);
            }
        }
        S_out[j] = orc_rollout_cost(p, x0, U, zk, ref, n_ref, circ, n_circ, centres, NULL, NULL);
        free(zk);
    }
    return 0;
}

int orc_plan(const orc_params* p, uint32_t iter, const double x0[4],
             const double* ref, int32_t n_ref, const orc_circle* circ, int32_t n_circ,
             const double* centres, double* U, double* u_star, double* x_star,
             double* S_out, double* margin_out, double* eps_out, orc_info* info)
{
    if (validate(p, x0, ref, n_ref, circ, n_circ, centres, U)) return -1;
    const int32_t K = p->K, T = p->T;
    const size_t KT2 = (size_t)K * T * 2;

    /* Algorithm 1: eps <- GenerateRandomNoise(Sigma) (unit normals, scaled in the rollout) */
    double* z = (double*)malloc(sizeof(double) * KT2);
    orc_noise(p, iter, z);

    /* Algorithm 1: for m in parallel: roll out and accumulate S(tau_m) */
    double* S = S_out ? S_out : (double*)malloc(sizeof(double) * K);
    double* eps = eps_out ? eps_out : (double*)malloc(sizeof(double) * KT2);
    double* ctg = p->cost_to_go ? (double*)malloc(sizeof(double) * (size_t)K * T) : NULL;
#pragma omp parallel
    {
        double* zk = (double*)malloc(sizeof(double) * 2 * (size_t)T);
        double* ek = (double*)malloc(sizeof(double) * 2 * (size_t)T);
        double* ck = (double*)malloc(sizeof(double) * (size_t)T);
#pragma omp for schedule(dynamic, 16)
        for (int32_t k = 0; k < K; ++k) {
            for (int32_t t = 0; t < T; ++t) {
                zk[2 * t] = z[((size_t)t * K + k) * 2];
                zk[2 * t + 1] = z[((size_t)t * K + k) * 2 + 1];
            }
            double m;
            S[k] = orc_rollout_cost_ctg(p, x0, U, zk, ref, n_ref, circ, n_circ, centres, ek, &m,
                                        ctg ? ck : NULL);
            if (ctg)
                for (int32_t t = 0; t < T; ++t) ctg[(size_t)t * K + k] = ck[t];
            if (margin_out) margin_out[k] = m;
            for (int32_t t = 0; t < T; ++t) {
                eps[((size_t)t * K + k) * 2] = ek[2 * t];
                eps[((size_t)t * K + k) * 2 + 1] = ek[2 * t + 1];
            }
        }
        free(zk);
        free(ek);
        free(ck);
    }

    /* Algorithm 1: S_min, then the update of Eq. (11) */
    double* dU = (double*)malloc(sizeof(double) * 2 * (size_t)T);
    orc_info local;
    int32_t n_fin = orc_softmin_update(K, T, S, eps, p->lam, dU, &local, NULL);
    if (ctg) {
        /* the per-step reading replaces the update; S_min, the argmin and eta stay those of
           the whole cost (step 0) */
        double* eta_t = (double*)malloc(sizeof(double) * (size_t)T);
        orc_softmin_update_ctg(K, T, ctg, eps, p->lam, dU, eta_t);
        local.eta = eta_t[0];
        free(eta_t);
        free(ctg);
    }
    if (info) *info = local;
    int rc = 0;
    if (n_fin == 0) {
        rc = -4;
    } else {
        double* un = (double*)malloc(sizeof(double) * 2 * (size_t)T);
        for (int32_t t = 0; t < T; ++t)
            for (int c = 0; c < 2; ++c)
                un[2 * t + c] = clampd(U[2 * t + c] + dU[2 * t + c], p->u_min[c], p->u_max[c]);
        /* Algorithm 1: u* <- SavitzkyGolayFilter(Z, u), bounds re-imposed */
        if (p->sg_enable) {
            for (int c = 0; c < 2; ++c) orc_savgol5(T, un + c, 2, u_star + c);
            for (int32_t t = 0; t < T; ++t)
                for (int c = 0; c < 2; ++c)
                    u_star[2 * t + c] = clampd(u_star[2 * t + c], p->u_min[c], p->u_max[c]);
        } else {
            memcpy(u_star, un, sizeof(double) * 2 * (size_t)T);
        }
        /* Algorithm 1: optimal trajectory x* */
        orc_rollout_states(p, x0, u_star, x_star);
        /* Algorithm 1: warm start for the next cycle */
        for (int32_t t = 0; t < T; ++t) {
            int32_t s = p->shift ? (t + 1 < T ? t + 1 : T - 1) : t;
            U[2 * t] = u_star[2 * s];
            U[2 * t + 1] = u_star[2 * s + 1];
        }
        free(un);
    }
    free(dU);
    free(z);
    if (!S_out) free(S);
    if (!eps_out) free(eps);
    return rc;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads the sample loops use from now on (timing only: the results do not depend on it). */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
