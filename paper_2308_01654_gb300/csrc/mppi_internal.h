// mppi_internal.h - types shared by the kernels and the C ABI implementation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mppi {

// Largest block of the single-plan rollout kernel: it is compiled for 896 lanes per SM (at
// most 72 registers a thread), as one block of 896 or several smaller ones.  One block per SM
// matters: two co-resident blocks of one wave do not progress alike (the second ran ~16 %
// slower), and the second then finished alone at half occupancy.
constexpr int MAX_ROLLOUT_THREADS = 896;

// Largest block of the batched planner's rollout kernel (two per SM).
constexpr int BATCH_MAX_THREADS = 448;

// Per-context device record: iteration counter, status and the reduction results.
struct __align__(16) DevState {
    unsigned long long iter;     // next iteration index (low 32 bits enter the Philox counter)
    int32_t flags;               // FLAG_* raised by kernels
    int32_t status;              // mppi_status of the last iteration
    double s_min;                // lowest sample cost
    double eta;                  // sum of softmin weights
    int32_t argmin;
    int32_t n_finite;
    unsigned int ticket;         // last-block-done counter of the argmin reduction (rollout kernel)
    int32_t jb0;                 // reference segment closest to x0
    unsigned long long jkey;     // packed (distance bits, index) for the jb0 search
    float4 x0f;                  // (0, 0, yaw0, v0): x0 in the local frame
    unsigned long long iter_used;  // iteration index of the last finished iteration
    int32_t moving;              // some obstacle circle has a nonzero velocity
    float delta0f;               // steering angle of x0 (model 1)
    int32_t multi_head;          // the reference polyline has segments of more than one heading
    int32_t pad_;
};

// Byte offsets of the arrays in the scene blob that the rollout kernel stages into
// shared memory with one bulk copy.  Every offset is a multiple of 16.
struct SceneLayout {
    int T, n_ref, n_seg, n_l1, n_l2, n_circ;   // chunks of REF_L1 segments, groups of REF_L2 chunks
    int off_ctl;     // float4 [T]       (u_a, u_d, g_a, g_d): nominal controls and control-cost slopes
    int off_c0;      // float  [T]       1/2 u^T R u
    int off_vert;    // float2 [n_ref]   vertices, local frame
    int off_seg;     // float4 [n_seg]   (ex, ey, ex/|e|^2, ey/|e|^2)
    int off_head;    // float  [n_seg]   heading of each segment
    int off_l1;      // float4 [n_l1]    level-1 chunk boxes
    // the circles are stored sorted by their key s = p . d (p: the first centre, d: the lane direction)
    int off_circ;    // float4 [n_circ]  (x, y, r, (d_safe_0 + r + r_ego)^2 when d_safe is constant)
    int off_vel;     // float2 [n_circ]  velocities
    int off_disp;    // float  [n_circ]  bound on the distance a centre moves in one step
    int off_proj;    // float4           (dx, dy, 0, 0): unit direction of the lane (first to last vertex)
    int off_order;   // int    [n_circ]  input index of each sorted circle (its column of the centre table)
    int off_skey;    // float  [n_circ]  the sorted keys
    int bytes;       // the staged part (all of the above), a multiple of 16
    // after the staged part, read from global memory (through L1) by the segment search:
    int off_pbox;    // float4 [n_ref]   box of the vertices 0 .. i
    int off_sbox;    // float4 [n_ref]   box of the vertices i .. n_ref - 1
    int total;       // the whole scene buffer, a multiple of 16
};

// Per-plan constants in the precision the kernels use.
struct PlanConst {
    int K, T;
    float dt, dt_over_L;
    float sig_a, sig_d, amin, amax, dmin, dmax;
    float w_dist, w_target, w_yaw, w_speed, w_safe, w_terminal;
    float v_ref, v_max;
    int vcap;
    float d_safe_c, d_safe_0;
    int collision_only;
    int n_ego;
    int ego_same_radius;     // all ego radii equal: the band limit is per circle
    float ego_off[8], ego_rad[8];
    float ego_omin, ego_omax, ego_rmax;   // extent of the ego circles along the heading, largest radius
    int ref_mode;
    int has_table;           // per-step centre table given
    uint32_t key0, key1, session;
    // double-precision parameters of the update and the optimal rollout
    double lam, dt_d, wheelbase_d, amin_d, amax_d, dmin_d, dmax_d, v_max_d;
    double g_a, g_d;         // (1 + alpha) R_a, (1 + alpha) R_d
    double half_Ra, half_Rd; // R / 2
    int sg_enable, shift;
    // last, so the members above keep their offsets (the weighted-sum kernel measurably
    // slows down when they move)
    int model;               // 0: control (a, delta); 1: state carries delta, control (a, omega)
    int cost_to_go;          // 1: per-step weights from the cost still to come
    double inv_dt_d;         // 1 / dt
    double dt_over_wb_d;     // dt / wheelbase
    float inv_lam_f;         // 1 / lambda
    uint32_t k_offset;       // global index of sample 0 (a K-slice of a partitioned plan; else 0)
};

SceneLayout make_layout(int T, int n_ref, int n_circ);

struct PlanBuffers {
    DevState* state;
    unsigned char* scene;    // SceneLayout::bytes
    float2* table;           // [T][n_circ] centres, local frame (when given)
    void* z;                 // [T][K] float2 or bf16x2
    double* S;               // [K]
    float* w;                // [K] softmin weights
    double* eta_part;        // [n_wblk]
    ulonglong2* kmin_part;   // [K] per rollout block: (cost order key, (finite count << 32) | index)
    double* du_part;         // [n_kt][T][2]
    double* du;              // [T][2] sum over the k-tiles (wsum's last block per step tile), or null
    unsigned* tt_count;      // [n_tt] k-tile blocks done per step tile (zero between launches)
    double* U;               // [T][2] nominal controls (the warm start)
    unsigned long long* stats;  // [7] work counters (STATS launches only)
    unsigned* fix_count;     // bfloat16 noise: pairs whose rounding is taken again in binary64
    uint2* fix_list;         // [NOISE_FIX_CAP] their (step pair j, sample k); null: decided in place
    float* ctg_prefix;       // [T][K] cost of steps 0..t-1 per sample (cost-to-go form), or null
    float* wt;               // [T][K] per-step softmin weights (cost-to-go form)
    double* eta_t;           // [T] per-step normalisers (cost-to-go form)
    int n_wblk, n_kt, n_tt, kt_size;
    int tt_len;              // steps per step tile of the weighted sum (<= WS_TT)
};

// Shared memory each rollout block builds after the staged blob: the level-2 boxes, the
// circle index (a float4 of scalars and CIRC_BUCKETS + 1 bucket starts into the sorted
// circles) and a float4 of search scalars.
constexpr int CIRC_BUCKETS = 64;

__host__ __device__ inline size_t block_extra_bytes(const SceneLayout& L) {
    return (size_t)16 * L.n_l2 + 32 + (size_t)4 * ((CIRC_BUCKETS + 1 + 3) & ~3);
}

// Per-thread slots after the block's extras: the compensated steering angle of the
// steering-rate model (float2 per thread of the block), kept out of the registers of the
// other model; none for the 4-state model.
__host__ __device__ inline size_t steer_slots_bytes(int threads, bool model1) {
    return model1 ? (size_t)8 * threads : 0;
}

// Capacity of the deferred bfloat16 rounding list (pairs beyond it are decided in place).
constexpr unsigned NOISE_FIX_CAP = 1u << 16;

struct PlanInputs {
    const double* x0;        // [4]
    const double* ref;       // [n_ref][2]
    const double* circ;      // [n_circ][5]
    const double* centres;   // [T][n_circ][2] or null
    int n_ref, n_circ;
    double* u_out;           // [T][2]
    double* x_out;           // [T+1][4]
    DevState* state_out = nullptr;   // when set, finalize copies the device record here (pinned host)
};

// Launch the whole iteration (prep, noise, rollout, reductions, update) on a stream.
// ev: optional array of N_KERNELS + 1 events; ev_mode 1 records them around every kernel
// (per-kernel timing: the prep stage is the prep + noise launch, the noise stage the bf16
// fix-up, the argmin stage empty since the rollout kernel ends with the argmin), 2 only ev[2]
// and ev[3] around the rollout (the rest stays chained).
constexpr int N_KERNELS = 7;   // prep, noise, rollout, argmin, weights, wsum, finalize
// inject: status flags written into the device record between the rollout and the weights
// (debug: the failure path without a fault; 0 = none; the source must outlive the launch).
cudaError_t launch_iteration(const PlanConst& pc, const SceneLayout& L, const PlanBuffers& b,
                             const PlanInputs& in, int group, int threads, int noise_bf16, cudaStream_t st,
                             cudaEvent_t* ev = nullptr, int ev_mode = 1, const int* inject = nullptr);

// The iteration split at the two exchanges of a K-partitioned plan (each context holds the
// slice of samples k_offset .. k_offset + K - 1): costs (prep, noise, rollout with the slice's
// S_min and argmin), sums (softmin weights against the global S_min and the weighted noise
// sums), finalize (update, smoothing, x*, warm start from the summed eta and du).
cudaError_t launch_slice_costs(const PlanConst& pc, const SceneLayout& L, const PlanBuffers& b,
                               const PlanInputs& in, int group, int threads, int noise_bf16, cudaStream_t st);
cudaError_t launch_slice_sums(const PlanConst& pc, const SceneLayout& L, const PlanBuffers& b, int noise_bf16,
                              cudaStream_t st);
cudaError_t launch_slice_finalize(const PlanConst& pc, const PlanBuffers& b, const PlanInputs& in, cudaStream_t st);

// prep + noise only (no change to the warm start or the iteration counter) and the
// reset of the fields prep accumulates into; used by the autotuner.
cudaError_t launch_prep_noise(const PlanConst& pc, const SceneLayout& L, const PlanBuffers& b,
                              const PlanInputs& in, int noise_bf16, cudaStream_t st);
cudaError_t launch_reset_state(DevState* st, cudaStream_t s);

// Bounds-checking debug build (MPPI_CHECKS): the index violations counted by the kernels of
// each translation unit since the last call (then reset; 0 in the normal build), and a kernel
// with two out-of-range indices that the checks must count (a4: 4 ints, out: 1 int).
cudaError_t take_check_hits_kernels(unsigned long long* hits);
cudaError_t take_check_hits_batch(unsigned long long* hits);
cudaError_t run_check_selftest(int* a4, int* out, cudaStream_t st);

// Raw Philox words for n counters (device buffers).
cudaError_t launch_philox(uint2 key, const uint4* ctr, uint4* out, int n, cudaStream_t st);

// Rollout kernel only (for timing and tuning); requires prep and noise of the same plan.
cudaError_t launch_rollout(const PlanConst& pc, const SceneLayout& L, const PlanBuffers& b, int group,
                           int threads, int noise_bf16, cudaStream_t st);

// Rollout with work counters (1 lane per sample): accumulates into b.stats.
cudaError_t launch_rollout_stats(const PlanConst& pc, const SceneLayout& L, const PlanBuffers& b, int noise_bf16,
                                 cudaStream_t st);

// Dynamic shared memory of a rollout block: the staged blob, the extras the block builds and
// the steering slots (threads of the block; model1: the steering-rate model).
size_t rollout_smem_bytes(const SceneLayout& L, int threads, bool model1);

// Resident rollout blocks per SM for a launch shape (0 if it cannot launch).
// ext: the steering-rate model or the cost-to-go form is on (PlanConst model / cost_to_go)
int rollout_max_blocks_per_sm(int group, int threads, int noise_bf16, size_t smem, bool ext);

}  // namespace mppi
