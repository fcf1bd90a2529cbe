// mppi_api.cu - the C ABI of include/mppi.h: contexts, buffers, validation, launch order.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "mppi.h"
#include "mppi_device.cuh"
#include "mppi_internal.h"

using namespace mppi;

struct mppi_ctx {
    mppi_params p;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    int cap_ref = 0, cap_circ = 0;
    PlanConst pc{};
    PlanBuffers b{};
    double* d_in = nullptr;      // x0 | ref | circ | centres (binary64, device)
    double* d_out = nullptr;     // u_out [T][2] | x_out [T+1][nx]
    int nx = 4;                  // state entries: 4, or 5 for the steering-rate model
    double* h_in = nullptr;      // pinned staging of the same layout
    double* h_out = nullptr;     // pinned staging of outputs
    DevState* h_state = nullptr; // pinned copy of the device record
    // device addresses of the two pinned buffers: mppi_plan's finalize writes u*, x* and the
    // record straight into host memory (no copy back)
    double* h_out_dev = nullptr;
    DevState* h_state_dev = nullptr;
    size_t in_elems = 0, out_elems = 0;
    int group = 1;
    int threads = 128;
    int profiling = 0;
    // the host-buffer iteration captured as a CUDA graph, per input shape
    cudaGraphExec_t graph = nullptr;
    long long graph_key = -1, seen_key = -1;
    size_t graph_n_in = 0;
    cudaEvent_t ev[N_KERNELS + 1] = {};
    // K-partitioned iteration: the inputs staged by mppi_slice_costs and the stage reached
    // (0 none, 1 costs done, 2 sums done)
    PlanInputs slice_in{};
    int slice_stage = 0;
    // debug: status flags the next iteration raises between its rollout and its update
    int inject_flags = 0;
    std::string err;
};

static thread_local std::string g_err;

static int fail(mppi_ctx* c, int status, const std::string& msg) {
    if (c) c->err = msg;
    g_err = msg;
    return status;
}

static int cuda_fail(mppi_ctx* c, cudaError_t e, const char* what) {
    return fail(c, MPPI_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

// Every value finite: no exponent field all ones (inf, NaN).  Adding one unit of the exponent
// field to the masked exponent carries into the top bit only from all ones, so the pass is
// integer and, or and add without branches, and the compiler vectorises it.
static bool finite_all(const double* v, size_t n) {
    const uint64_t exp_mask = 0x7ff0000000000000ull, exp_one = 0x0010000000000000ull;
    uint64_t bad = 0;
    for (size_t i = 0; i < n; ++i) {
        uint64_t bits;
        memcpy(&bits, v + i, sizeof(bits));
        bad |= (bits & exp_mask) + exp_one;
    }
    return (bad >> 63) == 0;
}

static bool valid_group(int g) {
    return g == 0 || g == 1 || g == 2 || g == 4 || g == 8 || g == 16 || g == 32 || g == -2 || g == -4 || g == -8 ||
           g == -16;
}

static bool valid_block(int b) { return b >= 32 && b <= MAX_ROLLOUT_THREADS && b % 32 == 0; }

static int check_params(const mppi_params* p, std::string& why) {
    if (!p) { why = "params is NULL"; return MPPI_ERR_ARG; }
    if (p->K < 1) { why = "K must be >= 1"; return MPPI_ERR_ARG; }
    if (p->T < 1 || p->T > MPPI_MAX_T) { why = "T must be in [1, MPPI_MAX_T]"; return MPPI_ERR_ARG; }
    if (!(p->dt > 0.0) || !isfinite(p->dt)) { why = "dt must be finite and > 0"; return MPPI_ERR_ARG; }
    if (!(p->wheelbase > 0.0) || !isfinite(p->wheelbase)) { why = "wheelbase must be > 0"; return MPPI_ERR_ARG; }
    if (!(p->lam > 0.0)) { why = "lam must be > 0"; return MPPI_ERR_ARG; }
    if (!(p->gamma > 0.0) || !isfinite(p->gamma)) { why = "gamma must be > 0"; return MPPI_ERR_ARG; }
    for (int c = 0; c < 2; ++c) {
        if (!(p->sigma[c] >= 0.0) || !isfinite(p->sigma[c])) { why = "sigma must be finite and >= 0"; return MPPI_ERR_ARG; }
        if (!isfinite(p->u_min[c]) || !isfinite(p->u_max[c]) || !(p->u_min[c] <= p->u_max[c])) {
            why = "u_min <= u_max must hold with finite bounds";
            return MPPI_ERR_ARG;
        }
        if (!isfinite(p->R[c])) { why = "R must be finite"; return MPPI_ERR_ARG; }
    }
    if (p->n_ego < 0 || p->n_ego > MPPI_MAX_EGO) { why = "n_ego must be in [0, MPPI_MAX_EGO]"; return MPPI_ERR_ARG; }
    const double w[] = {p->w_dist, p->w_target, p->w_yaw, p->w_speed, p->w_safe, p->w_terminal,
                        p->v_ref, p->d_safe_c, p->d_safe_0};
    if (!finite_all(w, sizeof(w) / sizeof(w[0]))) { why = "weights and speeds must be finite"; return MPPI_ERR_ARG; }
    if (isnan(p->v_max)) { why = "v_max must not be NaN"; return MPPI_ERR_ARG; }
    for (int e = 0; e < p->n_ego; ++e)
        if (!isfinite(p->ego_offset[e]) || !isfinite(p->ego_radius[e])) { why = "ego circles must be finite"; return MPPI_ERR_ARG; }
    if (p->ref_mode != 0 && p->ref_mode != 1) { why = "ref_mode must be 0 or 1"; return MPPI_ERR_ARG; }
    if (p->model != 0 && p->model != 1) { why = "model must be 0 or 1"; return MPPI_ERR_ARG; }
    if (p->cost_to_go != 0 && p->cost_to_go != 1) { why = "cost_to_go must be 0 or 1"; return MPPI_ERR_ARG; }
    if (!valid_group(p->group)) {
        why = "group must be 0, 1, 2, 4, 8, 16, 32, -2, -4, -8 or -16";
        return MPPI_ERR_ARG;
    }
    if (!(p->block == 0 || valid_block(p->block))) {
        why = "block must be 0 or a multiple of 32 in [32, 896]";
        return MPPI_ERR_ARG;
    }
    return MPPI_OK;
}

static int auto_group(int K) {
    // enough lanes to keep every SM busy when K is small; one lane per sample when K is large
    const long long target = 152LL * 512LL;
    int g = 1;
    while (g < 32 && (long long)K * g * 2 <= target) g *= 2;
    return g;
}

static PlanConst make_const(const mppi_params& p) {
    PlanConst c{};
    c.K = p.K;
    c.T = p.T;
    c.model = p.model;
    c.cost_to_go = p.cost_to_go;
    c.dt = (float)p.dt;
    c.dt_over_L = (float)(p.dt / p.wheelbase);
    c.sig_a = (float)p.sigma[0];
    c.sig_d = (float)p.sigma[1];
    c.amin = (float)p.u_min[0];
    c.amax = (float)p.u_max[0];
    c.dmin = (float)p.u_min[1];
    c.dmax = (float)p.u_max[1];
    c.w_dist = (float)p.w_dist;
    c.w_target = (float)p.w_target;
    c.w_yaw = (float)p.w_yaw;
    c.w_speed = (float)p.w_speed;
    c.w_safe = (float)p.w_safe;
    c.w_terminal = (float)p.w_terminal;
    c.v_ref = (float)p.v_ref;
    c.vcap = isfinite(p.v_max) ? 1 : 0;
    c.v_max = c.vcap ? (float)p.v_max : 0.0f;
    c.d_safe_c = (float)p.d_safe_c;
    c.d_safe_0 = (float)p.d_safe_0;
    c.collision_only = p.collision_only ? 1 : 0;
    c.n_ego = p.n_ego;
    c.ego_same_radius = 1;
    for (int e = 0; e < 8; ++e) {
        c.ego_off[e] = e < p.n_ego ? (float)p.ego_offset[e] : 0.0f;
        c.ego_rad[e] = e < p.n_ego ? (float)p.ego_radius[e] : 0.0f;
        if (e < p.n_ego && p.ego_radius[e] != p.ego_radius[0]) c.ego_same_radius = 0;
    }
    c.ego_omin = 0.0f;
    c.ego_omax = 0.0f;
    c.ego_rmax = 0.0f;
    for (int e = 0; e < p.n_ego; ++e) {
        c.ego_omin = e == 0 ? c.ego_off[0] : fminf(c.ego_omin, c.ego_off[e]);
        c.ego_omax = e == 0 ? c.ego_off[0] : fmaxf(c.ego_omax, c.ego_off[e]);
        c.ego_rmax = e == 0 ? c.ego_rad[0] : fmaxf(c.ego_rmax, c.ego_rad[e]);
    }
    c.ref_mode = p.ref_mode;
    c.has_table = 0;
    c.key0 = (uint32_t)(p.seed & 0xffffffffull);
    c.key1 = (uint32_t)(p.seed >> 32);
    c.session = p.session;
    c.lam = p.lam;
    c.dt_d = p.dt;
    c.wheelbase_d = p.wheelbase;
    c.inv_dt_d = 1.0 / p.dt;
    c.inv_lam_f = (float)(1.0 / p.lam);
    c.dt_over_wb_d = p.dt / p.wheelbase;
    c.amin_d = p.u_min[0];
    c.amax_d = p.u_max[0];
    c.dmin_d = p.u_min[1];
    c.dmax_d = p.u_max[1];
    c.v_max_d = p.v_max;
    const double alpha = (p.gamma - 1.0) / (2.0 * p.gamma);
    c.g_a = (1.0 + alpha) * p.R[0];
    c.g_d = (1.0 + alpha) * p.R[1];
    c.half_Ra = 0.5 * p.R[0];
    c.half_Rd = 0.5 * p.R[1];
    c.sg_enable = p.sg_enable ? 1 : 0;
    c.shift = p.shift ? 1 : 0;
    return c;
}

// Shared with the batched planner (same validation and conversion for every plan).
namespace mppi {
int check_params_shared(const mppi_params* p, std::string& why) { return check_params(p, why); }
PlanConst make_const_shared(const mppi_params& p) { return make_const(p); }
}  // namespace mppi

static void free_all(mppi_ctx* c) {
    PlanBuffers& b = c->b;
    void* dev[] = {b.state, b.scene, b.table, b.z, b.S, b.w, b.eta_part, b.kmin_part, b.du_part, b.du,
                   b.tt_count, b.U, b.stats, b.fix_count, b.fix_list, b.ctg_prefix, b.wt, b.eta_t, c->d_in, c->d_out};
    for (void* p : dev)
        if (p) cudaFree(p);
    if (c->h_in) cudaFreeHost(c->h_in);
    if (c->h_out) cudaFreeHost(c->h_out);
    if (c->h_state) cudaFreeHost(c->h_state);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
}

extern "C" {

int mppi_default_params(mppi_params* p, int32_t K, int32_t T, double dt) {
    if (!p) return MPPI_ERR_ARG;
    memset(p, 0, sizeof(*p));
    p->K = K;
    p->T = T;
    p->dt = dt;
    p->wheelbase = 2.7;
    p->sigma[0] = 0.5;
    p->sigma[1] = 0.05;
    p->u_min[0] = -3.0;
    p->u_max[0] = 3.0;
    p->u_min[1] = -0.5;
    p->u_max[1] = 0.5;
    p->lam = 1.0;
    p->gamma = 1.0;
    p->R[0] = p->lam / (p->sigma[0] * p->sigma[0]);
    p->R[1] = p->lam / (p->sigma[1] * p->sigma[1]);
    p->w_dist = 15.0;
    p->w_target = 7.0;
    p->w_yaw = 120.0;
    p->w_speed = 5.0;
    p->w_safe = 25.0;
    p->w_terminal = 0.0;
    p->v_ref = 30.0 / 3.6;
    p->v_max = INFINITY;
    p->d_safe_c = 0.0;
    p->d_safe_0 = 0.5;
    p->n_ego = 3;
    p->ego_offset[0] = 0.0;
    p->ego_offset[1] = 1.35;
    p->ego_offset[2] = 2.7;
    p->ego_radius[0] = p->ego_radius[1] = p->ego_radius[2] = 1.1;
    p->sg_enable = 1;
    return MPPI_OK;
}

int mppi_create(const mppi_params* params, int device, void* cuda_stream, int32_t max_ref, int32_t max_circ,
                mppi_ctx** out_ctx) {
    std::string why;
    if (!out_ctx) return fail(nullptr, MPPI_ERR_ARG, "out_ctx is NULL");
    *out_ctx = nullptr;
    int rc = check_params(params, why);
    if (rc != MPPI_OK) return fail(nullptr, rc, why);
    if (max_ref < 0 || max_ref > MPPI_MAX_REF || max_circ < 0 || max_circ > MPPI_MAX_CIRC)
        return fail(nullptr, MPPI_ERR_CAPACITY, "max_ref / max_circ above the library maxima");
    mppi_ctx* c = new (std::nothrow) mppi_ctx();
    if (!c) return fail(nullptr, MPPI_ERR_OOM, "host allocation failed");
    c->p = *params;
    c->device = device;
    c->cap_ref = max_ref ? max_ref : MPPI_MAX_REF;
    c->cap_circ = max_circ ? max_circ : MPPI_MAX_CIRC;
    c->group = params->group ? params->group : auto_group(params->K);
    c->threads = params->block ? params->block : 128;
    c->pc = make_const(*params);
    auto bail = [&](int status) {
        free_all(c);
        delete c;
        return status;
    };
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return bail(cuda_fail(nullptr, e, "cudaSetDevice"));
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(cuda_fail(nullptr, e, "cudaStreamCreate"));
        c->stream = c->own_stream;
    }
    const int K = params->K, T = params->T;
    PlanBuffers& b = c->b;
    b.n_wblk = (int)std::min<long long>((K + 255) / 256, 296);
    b.kt_size = 256 * WS_J;
    b.n_kt = (K + b.kt_size - 1) / b.kt_size;
    // steps per tile of the weighted sum: the longest of 8, 4, 2, 1 that still gives six
    // blocks per SM (small plans otherwise run on a handful of SMs; at the roofline size
    // 1600 shorter blocks finish 2 us sooner than 800: less tail among co-resident blocks)
    int n_sm = 0;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n_sm <= 0) n_sm = 152;
    b.tt_len = WS_TT;
    while (b.tt_len > 1 && (long long)b.n_kt * ((T + b.tt_len - 1) / b.tt_len) < 6LL * n_sm) b.tt_len /= 2;
    b.n_tt = (T + b.tt_len - 1) / b.tt_len;
    const SceneLayout Lmax = make_layout(T, c->cap_ref, c->cap_circ);
    const size_t zbytes = (size_t)T * K * (params->noise_bf16 ? 4 : 8);
    c->nx = params->model == 1 ? 5 : 4;
    c->in_elems = 8 + 2 * (size_t)c->cap_ref + 5 * (size_t)c->cap_circ + 2 * (size_t)T * c->cap_circ;
    c->out_elems = 2 * (size_t)T + (size_t)c->nx * (size_t)(T + 1);
    struct A {
        void** p;
        size_t n;
    } allocs[] = {
        {(void**)&b.state, sizeof(DevState)},
        {(void**)&b.scene, (size_t)Lmax.total},
        {(void**)&b.table, sizeof(float2) * (size_t)T * std::max(c->cap_circ, 1)},
        {(void**)&b.z, zbytes},
        {(void**)&b.S, sizeof(double) * K},
        {(void**)&b.w, sizeof(float) * K},
        {(void**)&b.eta_part, sizeof(double) * b.n_wblk},
        // one record per rollout block: at most K blocks (|group| <= 32 lanes a sample, >= 32 threads)
        {(void**)&b.kmin_part, sizeof(ulonglong2) * (size_t)K},
        {(void**)&b.du_part, sizeof(double) * 2 * (size_t)T * b.n_kt},
        {(void**)&b.du, sizeof(double) * 2 * (size_t)T},
        {(void**)&b.tt_count, sizeof(unsigned) * (size_t)b.n_tt},
        {(void**)&b.U, sizeof(double) * 2 * (size_t)T},
        {(void**)&b.stats, sizeof(unsigned long long) * 8},
        {(void**)&b.fix_count, sizeof(unsigned)},
        {(void**)&b.fix_list, sizeof(uint2) * (c->p.noise_bf16 ? NOISE_FIX_CAP : 1u)},
        {(void**)&b.ctg_prefix, sizeof(float) * (c->p.cost_to_go ? (size_t)K * T : 1u)},
        {(void**)&b.wt, sizeof(float) * (c->p.cost_to_go ? (size_t)K * T : 1u)},
        {(void**)&b.eta_t, sizeof(double) * (size_t)T},
        {(void**)&c->d_in, sizeof(double) * c->in_elems},
        {(void**)&c->d_out, sizeof(double) * c->out_elems},
    };
    for (auto& a : allocs) {
        e = cudaMalloc(a.p, a.n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(nullptr, MPPI_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e)));
        }
    }
    if (cudaMallocHost((void**)&c->h_in, sizeof(double) * c->in_elems) != cudaSuccess ||
        cudaMallocHost((void**)&c->h_out, sizeof(double) * c->out_elems) != cudaSuccess ||
        cudaMallocHost((void**)&c->h_state, sizeof(DevState)) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(nullptr, MPPI_ERR_OOM, "pinned host allocation failed"));
    }
    if (cudaHostGetDevicePointer((void**)&c->h_out_dev, c->h_out, 0) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&c->h_state_dev, c->h_state, 0) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(nullptr, MPPI_ERR_CUDA, "pinned host buffers are not mapped for the device"));
    }
    DevState s0;
    memset(&s0, 0, sizeof(s0));
    s0.jkey = ~0ull;
    e = cudaMemcpyAsync(b.state, &s0, sizeof(s0), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.U, 0, sizeof(double) * 2 * (size_t)T, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.tt_count, 0, sizeof(unsigned) * (size_t)b.n_tt, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.fix_count, 0, sizeof(unsigned), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bail(cuda_fail(nullptr, e, "context initialisation"));
    *out_ctx = c;
    return MPPI_OK;
}

int mppi_destroy(mppi_ctx* c) {
    if (!c) return MPPI_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
    return MPPI_OK;
}

int mppi_set_stream(mppi_ctx* c, void* cuda_stream) {
    if (!c) return fail(nullptr, MPPI_ERR_ARG, "ctx is NULL");
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    c->stream = cuda_stream ? (cudaStream_t)cuda_stream : c->own_stream;
    if (!c->stream) {
        CK(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking), "cudaStreamCreate");
        c->stream = c->own_stream;
    }
    return MPPI_OK;
}

static int check_sizes(mppi_ctx* c, int32_t n_ref, int32_t n_circ) {
    if (n_ref < 2) return fail(c, MPPI_ERR_ARG, "n_ref must be >= 2");
    if (n_circ < 0) return fail(c, MPPI_ERR_ARG, "n_circ must be >= 0");
    if (n_ref > c->cap_ref || n_circ > c->cap_circ)
        return fail(c, MPPI_ERR_CAPACITY, "reference or circle count above the context capacity");
    const SceneLayout L = make_layout(c->p.T, n_ref, n_circ);
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    if ((int)rollout_smem_bytes(L, c->threads, c->p.model == 1) + 1024 > max_smem)
        return fail(c, MPPI_ERR_CAPACITY, "reference + circles + horizon exceed shared memory");
    return MPPI_OK;
}

static int enqueue(mppi_ctx* c, const PlanInputs& in, int has_table) {
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    const SceneLayout L = make_layout(c->p.T, in.n_ref, in.n_circ);
    PlanConst pc = c->pc;
    pc.has_table = has_table;
    // an armed injection is copied from pageable memory (staged before the call returns)
    const int inject = c->inject_flags;
    c->inject_flags = 0;
    CK(launch_iteration(pc, L, c->b, in, c->group, c->threads, c->p.noise_bf16, c->stream,
                        c->profiling ? c->ev : nullptr, c->profiling, inject ? &inject : nullptr),
       "kernel launch");
    return MPPI_OK;
}

static void fill_info(const DevState& s, mppi_info* info) {
    if (!info) return;
    info->argmin = s.argmin;
    info->n_finite = s.n_finite;
    info->s_min = s.s_min;
    info->eta = 0.0;
    info->iter = s.iter_used;
}

static int wait_status(mppi_ctx* c, mppi_info* info, bool state_copied = false) {
    if (!state_copied)
        CK(cudaMemcpyAsync(c->h_state, c->b.state, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream),
           "state copy");
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    const DevState& s = *c->h_state;
    if (info) {
        fill_info(s, info);
        info->eta = s.eta;
    }
    if (s.status == MPPI_ERR_ARG) return fail(c, MPPI_ERR_ARG, "non-finite input detected on the device");
    if (s.status == MPPI_ERR_TIMEOUT) return fail(c, MPPI_ERR_TIMEOUT, "a bounded device wait ran out");
    if (s.status == MPPI_ERR_NUMERIC) return fail(c, MPPI_ERR_NUMERIC, "no sample cost was finite");
    return s.status;
}

// Validates host inputs, packs them into the pinned staging buffer and (with copy) queues
// their copy into the context's device input buffer; n_in receives the staged doubles.
static int stage_host_inputs(mppi_ctx* c, const double* x0, const double* ref_xy, int32_t n_ref,
                             const mppi_circle* circ, int32_t n_circ, const double* centres, PlanInputs& in,
                             bool copy = true, size_t* n_in_out = nullptr) {
    if (!x0 || !ref_xy || (n_circ > 0 && !circ)) return fail(c, MPPI_ERR_ARG, "NULL array argument");
    int rc = check_sizes(c, n_ref, n_circ);
    if (rc != MPPI_OK) return rc;
    const int T = c->p.T;
    const size_t nr = 2 * (size_t)n_ref, nc = 5 * (size_t)n_circ, nt = centres ? 2 * (size_t)T * n_circ : 0;
    if (!finite_all(x0, (size_t)c->nx) || !finite_all(ref_xy, nr) || (nc && !finite_all((const double*)circ, nc)) ||
        (centres && !finite_all(centres, nt)))
        return fail(c, MPPI_ERR_ARG, "non-finite input");
    double* h = c->h_in;
    // x0 in the first 8 entries (4 or 5 used): the reference stays 16-byte aligned
    memcpy(h, x0, (size_t)c->nx * sizeof(double));
    memcpy(h + 8, ref_xy, nr * sizeof(double));
    if (nc) memcpy(h + 8 + nr, circ, nc * sizeof(double));
    if (nt) memcpy(h + 8 + nr + nc, centres, nt * sizeof(double));
    const size_t n_in = 8 + nr + nc + nt;
    if (n_in_out) *n_in_out = n_in;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    if (copy)
        CK(cudaMemcpyAsync(c->d_in, h, n_in * sizeof(double), cudaMemcpyHostToDevice, c->stream), "input copy");
    in.x0 = c->d_in;
    in.ref = c->d_in + 8;
    in.circ = c->d_in + 8 + nr;
    in.centres = nt ? c->d_in + 8 + nr + nc : nullptr;
    in.n_ref = n_ref;
    in.n_circ = n_circ;
    in.u_out = c->d_out;
    in.x_out = c->d_out + 2 * (size_t)T;
    return MPPI_OK;
}

// The whole host-buffer iteration (input copy, kernels, output and status copies) in
// stream order; captured into a graph by mppi_plan.
static cudaError_t plan_sequence(mppi_ctx* c, const PlanInputs& in, size_t n_in) {
    cudaError_t e = cudaMemcpyAsync(c->d_in, c->h_in, n_in * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return e;
    const SceneLayout L = make_layout(c->p.T, in.n_ref, in.n_circ);
    PlanConst pc = c->pc;
    pc.has_table = in.centres ? 1 : 0;
    return launch_iteration(pc, L, c->b, in, c->group, c->threads, c->p.noise_bf16, c->stream, nullptr);
}

int mppi_plan(mppi_ctx* c, const double* x0, const double* ref_xy, int32_t n_ref, const mppi_circle* circ,
              int32_t n_circ, const double* centres, double* u_out, double* x_out, mppi_info* info) {
    if (!c) return fail(nullptr, MPPI_ERR_ARG, "ctx is NULL");
    if (!u_out || !x_out) return fail(c, MPPI_ERR_ARG, "NULL array argument");
    const int T = c->p.T;
    PlanInputs in;
    size_t n_in = 0;
    int rc = stage_host_inputs(c, x0, ref_xy, n_ref, circ, n_circ, centres, in, false, &n_in);
    if (rc != MPPI_OK) return rc;
    // outputs and the record go straight to the pinned host buffers (written by finalize)
    in.u_out = c->h_out_dev;
    in.x_out = c->h_out_dev + 2 * (size_t)T;
    in.state_out = c->h_state_dev;
    if (c->profiling || c->inject_flags) {
        // traced or injected iterations run uncaptured
        CK(cudaMemcpyAsync(c->d_in, c->h_in, n_in * sizeof(double), cudaMemcpyHostToDevice, c->stream), "input copy");
        rc = enqueue(c, in, in.centres ? 1 : 0);
        if (rc != MPPI_OK) return rc;
        rc = wait_status(c, info, true);
    } else {
        // shape key: the graph bakes in sizes, the layout and the launch shape
        const long long key =
            ((((long long)n_ref * 2048 + n_circ) * 2 + (in.centres ? 1 : 0)) * 64 + (c->group + 8)) * 1024 + c->threads;
        if (c->graph && key == c->graph_key && n_in == c->graph_n_in) {
            CK(cudaGraphLaunch(c->graph, c->stream), "graph launch");
        } else if (key == c->seen_key) {
            // second iteration with this shape: capture it (the first ran uncaptured and set up
            // every kernel attribute outside the capture)
            if (c->graph) {
                cudaGraphExecDestroy(c->graph);
                c->graph = nullptr;
            }
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
            const cudaError_t es = plan_sequence(c, in, n_in);
            const cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
            if (es != cudaSuccess || ee != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return cuda_fail(c, es != cudaSuccess ? es : ee, "graph capture");
            }
            const cudaError_t ei = cudaGraphInstantiate(&c->graph, g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) return cuda_fail(c, ei, "graph instantiate");
            c->graph_key = key;
            c->graph_n_in = n_in;
            CK(cudaGraphLaunch(c->graph, c->stream), "graph launch");
        } else {
            CK(plan_sequence(c, in, n_in), "kernel launch");
            c->seen_key = key;
        }
        rc = wait_status(c, info, true);
    }
    if (rc != MPPI_OK) return rc;
    memcpy(u_out, c->h_out, 2 * (size_t)T * sizeof(double));
    memcpy(x_out, c->h_out + 2 * (size_t)T, (size_t)c->nx * (size_t)(T + 1) * sizeof(double));
    return MPPI_OK;
}

int mppi_plan_device(mppi_ctx* c, const double* d_x0, const double* d_ref_xy, int32_t n_ref, const double* d_circ,
                     int32_t n_circ, const double* d_centres, double* d_u_out, double* d_x_out, mppi_info* info) {
    if (!c) return fail(nullptr, MPPI_ERR_ARG, "ctx is NULL");
    if (!d_x0 || !d_ref_xy || !d_u_out || !d_x_out || (n_circ > 0 && !d_circ))
        return fail(c, MPPI_ERR_ARG, "NULL array argument");
    int rc = check_sizes(c, n_ref, n_circ);
    if (rc != MPPI_OK) return rc;
    PlanInputs in;
    in.x0 = d_x0;
    in.ref = d_ref_xy;
    in.circ = n_circ > 0 ? d_circ : c->d_in;
    in.centres = d_centres;
    in.n_ref = n_ref;
    in.n_circ = n_circ;
    in.u_out = d_u_out;
    in.x_out = d_x_out;
    rc = enqueue(c, in, d_centres ? 1 : 0);
    if (rc != MPPI_OK) return rc;
    if (info) return wait_status(c, info);
    return MPPI_OK;
}

int mppi_debug_check_hits(int32_t* enabled, uint64_t* hits) {
    if (!enabled || !hits) return fail(nullptr, MPPI_ERR_ARG, "NULL argument");
#ifdef MPPI_CHECKS
    *enabled = 1;
#else
    *enabled = 0;
#endif
    unsigned long long a = 0, b = 0;
    cudaError_t e = take_check_hits_kernels(&a);
    if (e == cudaSuccess) e = take_check_hits_batch(&b);
    if (e != cudaSuccess) return fail(nullptr, MPPI_ERR_CUDA, std::string("check counters: ") + cudaGetErrorString(e));
    *hits = a + b;
    return MPPI_OK;
}

int mppi_debug_check_selftest(int device, uint64_t* hits) {
    if (!hits) return fail(nullptr, MPPI_ERR_ARG, "NULL argument");
    cudaError_t e = cudaSetDevice(device);
    int* d = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&d, 5 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(d, 0, 5 * sizeof(int));
    unsigned long long before = 0, after = 0;
    if (e == cudaSuccess) e = take_check_hits_kernels(&before);
    if (e == cudaSuccess) e = run_check_selftest(d, d + 4, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = take_check_hits_kernels(&after);
    if (d) cudaFree(d);
    if (e != cudaSuccess) return fail(nullptr, MPPI_ERR_CUDA, std::string("check self-test: ") + cudaGetErrorString(e));
    *hits = after;
    return MPPI_OK;
}

int mppi_debug_inject_flags(mppi_ctx* c, int32_t flags) {
    if (!c) return fail(nullptr, MPPI_ERR_ARG, "ctx is NULL");
    if (flags & ~(FLAG_NONFINITE_INPUT | FLAG_TIMEOUT)) return fail(c, MPPI_ERR_ARG, "unknown flag bits");
    c->inject_flags = flags;
    return MPPI_OK;
}

// ------------------------------------------------------------------------------------
// K-partitioned iteration (one slice of the samples per context; see include/mppi.h)
// ------------------------------------------------------------------------------------
int mppi_slice_costs(mppi_ctx* c, int64_t k_offset, const double* x0, const double* ref_xy, int32_t n_ref,
                     const mppi_circle* circ, int32_t n_circ, const double* centres, double* s_min, int32_t* argmin,
                     int32_t* n_finite) {
    if (!c) return fail(nullptr, MPPI_ERR_ARG, "ctx is NULL");
    if (!s_min || !argmin || !n_finite) return fail(c, MPPI_ERR_ARG, "NULL output argument");
    if (c->p.cost_to_go) return fail(c, MPPI_ERR_ARG, "the K-partitioned iteration runs the whole-cost weights");
    if (k_offset < 0 || k_offset + (int64_t)c->p.K > (int64_t)INT32_MAX)
        return fail(c, MPPI_ERR_ARG, "k_offset must be >= 0 and the global sample indices below 2^31");
    c->slice_stage = 0;
    PlanInputs in;
    int rc = stage_host_inputs(c, x0, ref_xy, n_ref, circ, n_circ, centres, in);
    if (rc != MPPI_OK) return rc;
    const SceneLayout L = make_layout(c->p.T, in.n_ref, in.n_circ);
    PlanConst pc = c->pc;
    pc.has_table = in.centres ? 1 : 0;
    pc.k_offset = (uint32_t)k_offset;
    CK(launch_slice_costs(pc, L, c->b, in, c->group, c->threads, c->p.noise_bf16, c->stream), "kernel launch");
    CK(cudaMemcpyAsync(c->h_state, c->b.state, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream), "state copy");
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    const DevState& s = *c->h_state;
    if (s.flags & FLAG_NONFINITE_INPUT) rc = fail(c, MPPI_ERR_ARG, "non-finite input detected on the device");
    else if (s.flags & FLAG_TIMEOUT) rc = fail(c, MPPI_ERR_TIMEOUT, "a bounded device wait ran out");
    if (rc != MPPI_OK) {
        CK(launch_reset_state(c->b.state, c->stream), "state reset");
        CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
        return rc;
    }
    *s_min = s.n_finite > 0 ? s.s_min : INFINITY;
    *argmin = s.n_finite > 0 ? (int32_t)(s.argmin + k_offset) : -1;
    *n_finite = s.n_finite;
    c->slice_in = in;
    c->slice_stage = 1;
    return MPPI_OK;
}

int mppi_slice_sums(mppi_ctx* c, double s_min, double* eta, double* du) {
    if (!c) return fail(nullptr, MPPI_ERR_ARG, "ctx is NULL");
    if (!eta || !du) return fail(c, MPPI_ERR_ARG, "NULL output argument");
    if (c->slice_stage != 1) return fail(c, MPPI_ERR_ARG, "mppi_slice_costs must come first");
    if (isnan(s_min)) return fail(c, MPPI_ERR_ARG, "s_min is NaN");
    const int T = c->p.T;
    const SceneLayout L = make_layout(T, c->slice_in.n_ref, c->slice_in.n_circ);
    CK(cudaMemcpyAsync(&c->b.state->s_min, &s_min, sizeof(double), cudaMemcpyHostToDevice, c->stream), "s_min copy");
    CK(launch_slice_sums(c->pc, L, c->b, c->p.noise_bf16, c->stream), "kernel launch");
    CK(cudaMemcpyAsync(c->h_out, c->b.du, sizeof(double) * 2 * (size_t)T, cudaMemcpyDeviceToHost, c->stream),
       "sums copy");
    std::vector<double> parts((size_t)c->b.n_wblk);
    CK(cudaMemcpyAsync(parts.data(), c->b.eta_part, sizeof(double) * parts.size(), cudaMemcpyDeviceToHost, c->stream),
       "eta copy");
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    double e = 0.0;
    for (double v : parts) e += v;      // block order
    *eta = e;
    memcpy(du, c->h_out, sizeof(double) * 2 * (size_t)T);
    c->slice_stage = 2;
    return MPPI_OK;
}

int mppi_slice_finalize(mppi_ctx* c, double eta, const double* du, int32_t n_finite, double s_min, int32_t argmin,
                        double* u_out, double* x_out, mppi_info* info) {
    if (!c) return fail(nullptr, MPPI_ERR_ARG, "ctx is NULL");
    if (!du || !u_out || !x_out) return fail(c, MPPI_ERR_ARG, "NULL array argument");
    if (c->slice_stage != 2) return fail(c, MPPI_ERR_ARG, "mppi_slice_sums must come first");
    const int T = c->p.T;
    if (!finite_all(du, 2 * (size_t)T) || isnan(eta) || n_finite < 0)
        return fail(c, MPPI_ERR_ARG, "non-finite sums or a negative count");
    // the exchanged totals take the place of this slice's own: du, eta (first partial, the
    // others zero), the finite count and the global minimum
    memcpy(c->h_out, du, sizeof(double) * 2 * (size_t)T);
    CK(cudaMemcpyAsync(c->b.du, c->h_out, sizeof(double) * 2 * (size_t)T, cudaMemcpyHostToDevice, c->stream),
       "sums copy");
    CK(cudaMemsetAsync(c->b.eta_part, 0, sizeof(double) * (size_t)c->b.n_wblk, c->stream), "eta reset");
    CK(cudaMemcpyAsync(c->b.eta_part, &eta, sizeof(double), cudaMemcpyHostToDevice, c->stream), "eta copy");
    CK(cudaMemcpyAsync(&c->b.state->n_finite, &n_finite, sizeof(int32_t), cudaMemcpyHostToDevice, c->stream),
       "count copy");
    CK(cudaMemcpyAsync(&c->b.state->s_min, &s_min, sizeof(double), cudaMemcpyHostToDevice, c->stream), "s_min copy");
    CK(cudaMemcpyAsync(&c->b.state->argmin, &argmin, sizeof(int32_t), cudaMemcpyHostToDevice, c->stream),
       "argmin copy");
    PlanInputs in = c->slice_in;
    in.u_out = c->d_out;
    in.x_out = c->d_out + 2 * (size_t)T;
    in.state_out = nullptr;
    CK(launch_slice_finalize(c->pc, c->b, in, c->stream), "kernel launch");
    CK(cudaMemcpyAsync(c->h_out, c->d_out, sizeof(double) * c->out_elems, cudaMemcpyDeviceToHost, c->stream),
       "output copy");
    c->slice_stage = 0;
    const int rc = wait_status(c, info);
    if (rc != MPPI_OK) return rc;
    memcpy(u_out, c->h_out, 2 * (size_t)T * sizeof(double));
    memcpy(x_out, c->h_out + 2 * (size_t)T, (size_t)c->nx * (size_t)(T + 1) * sizeof(double));
    return MPPI_OK;
}

static std::string gpu_name(int device) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return "unknown";
    std::string n = prop.name;
    for (auto& ch : n)
        if (ch == ' ' || ch == '|') ch = '_';
    return n;
}

static std::string tune_key(mppi_ctx* c, int n_ref, int n_circ) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s|%d|%d|%d|%d|%d|r3", gpu_name(c->device).c_str(), c->p.K, c->p.T, n_ref, n_circ,
             c->p.noise_bf16);
    return buf;
}

static bool cache_lookup(const char* path, const std::string& key, int& g, int& t) {
    if (!path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        char k[300];
        int gg, tt;
        float ms;
        if (sscanf(line, "%299s %d %d %f", k, &gg, &tt, &ms) == 4 && key == k) {
            g = gg;
            t = tt;
            found = true;   // the last entry for a key wins
        }
    }
    fclose(f);
    return found;
}

static void cache_store(const char* path, const std::string& key, int g, int t, float ms) {
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %.6f\n", key.c_str(), g, t, ms);
    fclose(f);
}

int mppi_autotune(mppi_ctx* c, const double* x0, const double* ref_xy, int32_t n_ref, const mppi_circle* circ,
                  int32_t n_circ, const double* centres, const char* cache_path, int32_t* group, int32_t* block) {
    if (!c) return fail(nullptr, MPPI_ERR_ARG, "ctx is NULL");
    const std::string key = tune_key(c, n_ref, n_circ);
    int g = 0, t = 0;
    if (cache_lookup(cache_path, key, g, t) && g != 0 && valid_group(g) && valid_block(t)) {
        c->group = g;
        c->threads = t;
    } else {
        PlanInputs in;
        int rc = stage_host_inputs(c, x0, ref_xy, n_ref, circ, n_circ, centres, in);
        if (rc != MPPI_OK) return rc;
        const SceneLayout L = make_layout(c->p.T, n_ref, n_circ);
        PlanConst pc = c->pc;
        pc.has_table = in.centres ? 1 : 0;
        CK(launch_prep_noise(pc, L, c->b, in, c->p.noise_bf16, c->stream), "prep/noise launch");
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0), "cudaEventCreate");
        CK(cudaEventCreate(&e1), "cudaEventCreate");
        float best = INFINITY;
        int bg = c->group, bt = c->threads;
        int n_sm = 0;
        CK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, c->device), "device attribute");
        const bool model1 = c->p.model == 1;
        const bool ext = c->p.model == 1 || c->p.cost_to_go != 0;
        // lanes per sample: > 0 split the work of each step, < 0 split the steps
        const int groups[] = {1, 2, 4, 8, 16, 32, -2, -4, -8, -16};
        cudaError_t err = cudaSuccess;
        for (int gi = 0; gi < 10 && err == cudaSuccess; ++gi) {
            const int G = groups[gi];
            const long long lanes = (long long)c->p.K * (G < 0 ? -G : G);
            if (G != 1 && lanes > 4LL * n_sm * 2048) continue;  // far more lanes than the GPU holds
            // candidate block sizes: fixed ones, and "balanced" ones that give every SM the same
            // number of lanes when m blocks per SM are resident together
            int cand[8], nc = 0;
            cand[nc++] = 64;
            cand[nc++] = 128;
            cand[nc++] = 256;
            for (int m = 1; m <= 4; ++m) {
                long long per = (lanes + (long long)n_sm * m - 1) / ((long long)n_sm * m);
                int th = (int)(((per + 31) / 32) * 32);
                if (th < 32 || th > MAX_ROLLOUT_THREADS) continue;
                if (rollout_max_blocks_per_sm(G, th, c->p.noise_bf16, rollout_smem_bytes(L, th, model1), ext) < m)
                    continue;
                bool dup = false;
                for (int i = 0; i < nc; ++i) dup |= cand[i] == th;
                if (!dup) cand[nc++] = th;
            }
            for (int bi = 0; bi < nc && err == cudaSuccess; ++bi) {
                if (rollout_max_blocks_per_sm(G, cand[bi], c->p.noise_bf16, rollout_smem_bytes(L, cand[bi], model1),
                                              ext) < 1)
                    continue;
                err = launch_rollout(pc, L, c->b, G, cand[bi], c->p.noise_bf16, c->stream);  // warm-up
                if (err == cudaSuccess) err = cudaEventRecord(e0, c->stream);
                for (int r = 0; r < 3 && err == cudaSuccess; ++r)
                    err = launch_rollout(pc, L, c->b, G, cand[bi], c->p.noise_bf16, c->stream);
                if (err == cudaSuccess) err = cudaEventRecord(e1, c->stream);
                if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                float ms = 0.0f;
                if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
                if (err == cudaSuccess && ms < best) {
                    best = ms;
                    bg = G;
                    bt = cand[bi];
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (err == cudaSuccess) err = launch_reset_state(c->b.state, c->stream);
        if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
        if (err != cudaSuccess) return cuda_fail(c, err, "autotune");
        c->group = bg;
        c->threads = bt;
        cache_store(cache_path, key, bg, bt, best / 3.0f);
    }
    if (group) *group = c->group;
    if (block) *block = c->threads;
    return MPPI_OK;
}

int mppi_rollout_stats(mppi_ctx* c, const double* x0, const double* ref_xy, int32_t n_ref, const mppi_circle* circ,
                       int32_t n_circ, const double* centres, uint64_t* counters) {
    if (!c || !counters) return fail(c, MPPI_ERR_ARG, "NULL argument");
    PlanInputs in;
    int rc = stage_host_inputs(c, x0, ref_xy, n_ref, circ, n_circ, centres, in);
    if (rc != MPPI_OK) return rc;
    const SceneLayout L = make_layout(c->p.T, n_ref, n_circ);
    PlanConst pc = c->pc;
    pc.has_table = in.centres ? 1 : 0;
    CK(cudaMemsetAsync(c->b.stats, 0, sizeof(unsigned long long) * 8, c->stream), "stats reset");
    CK(launch_prep_noise(pc, L, c->b, in, c->p.noise_bf16, c->stream), "prep/noise launch");
    CK(launch_rollout_stats(pc, L, c->b, c->p.noise_bf16, c->stream), "rollout launch");
    CK(launch_reset_state(c->b.state, c->stream), "state reset");
    unsigned long long h[8] = {};
    CK(cudaMemcpyAsync(h, c->b.stats, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "stats copy");
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    for (int i = 0; i < MPPI_N_STATS; ++i) counters[i] = h[i];
    return MPPI_OK;
}

int mppi_sync(mppi_ctx* c, mppi_info* info) {
    if (!c) return fail(nullptr, MPPI_ERR_ARG, "ctx is NULL");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    return wait_status(c, info);
}

int mppi_set_controls(mppi_ctx* c, const double* U, uint64_t iter) {
    if (!c || !U) return fail(c, MPPI_ERR_ARG, "NULL argument");
    if (!finite_all(U, 2 * (size_t)c->p.T)) return fail(c, MPPI_ERR_ARG, "non-finite controls");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    CK(cudaMemcpyAsync(c->b.U, U, sizeof(double) * 2 * c->p.T, cudaMemcpyHostToDevice, c->stream), "controls copy");
    unsigned long long it = iter;
    CK(cudaMemcpyAsync(&c->b.state->iter, &it, sizeof(it), cudaMemcpyHostToDevice, c->stream), "iter copy");
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    return MPPI_OK;
}

int mppi_get_controls(mppi_ctx* c, double* U, uint64_t* iter) {
    if (!c || !U) return fail(c, MPPI_ERR_ARG, "NULL argument");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    CK(cudaMemcpyAsync(U, c->b.U, sizeof(double) * 2 * c->p.T, cudaMemcpyDeviceToHost, c->stream), "controls copy");
    CK(cudaMemcpyAsync(c->h_state, c->b.state, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream), "state copy");
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    if (iter) *iter = c->h_state->iter;
    return MPPI_OK;
}

int mppi_get_costs(mppi_ctx* c, double* S) {
    if (!c || !S) return fail(c, MPPI_ERR_ARG, "NULL argument");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    CK(cudaMemcpyAsync(S, c->b.S, sizeof(double) * c->p.K, cudaMemcpyDeviceToHost, c->stream), "cost copy");
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    return MPPI_OK;
}

int mppi_get_noise(mppi_ctx* c, float* z) {
    if (!c || !z) return fail(c, MPPI_ERR_ARG, "NULL argument");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    const size_t n = 2 * (size_t)c->p.T * c->p.K;
    if (!c->p.noise_bf16) {
        CK(cudaMemcpyAsync(z, c->b.z, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "noise copy");
        CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
        return MPPI_OK;
    }
    // bfloat16 -> binary32 is an exact widening: the 16 bits become the top half
    uint16_t* tmp = (uint16_t*)malloc(n * sizeof(uint16_t));
    if (!tmp) return fail(c, MPPI_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaMemcpyAsync(tmp, c->b.z, n * sizeof(uint16_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        free(tmp);
        return cuda_fail(c, e, "noise copy");
    }
    for (size_t i = 0; i < n; ++i) {
        const uint32_t bits = (uint32_t)tmp[i] << 16;
        memcpy(&z[i], &bits, 4);
    }
    free(tmp);
    return MPPI_OK;
}

int mppi_philox(uint64_t seed, const uint32_t* ctr, int32_t n, uint32_t* out) {
    mppi_ctx* c = nullptr;
    if (!ctr || !out || n < 0) return fail(nullptr, MPPI_ERR_ARG, "bad argument");
    if (n == 0) return MPPI_OK;
    uint4 *d_ctr = nullptr, *d_out = nullptr;
    const size_t bytes = sizeof(uint4) * (size_t)n;
    CK(cudaMalloc(&d_ctr, bytes), "cudaMalloc");
    cudaError_t e = cudaMalloc(&d_out, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(d_ctr, ctr, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = launch_philox(make_uint2((uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32)), d_ctr, d_out, n, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, d_out, bytes, cudaMemcpyDeviceToHost);
    cudaFree(d_ctr);
    if (d_out) cudaFree(d_out);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "philox");
    return MPPI_OK;
}

int mppi_set_profiling(mppi_ctx* c, int32_t on) {
    if (!c) return fail(nullptr, MPPI_ERR_ARG, "ctx is NULL");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    if (on < 0 || on > 2) return fail(c, MPPI_ERR_ARG, "profiling mode must be 0, 1 or 2");
    if (on && !c->ev[0])
        for (auto& e : c->ev) CK(cudaEventCreate(&e), "cudaEventCreate");
    c->profiling = on;
    return MPPI_OK;
}

int mppi_kernel_times(mppi_ctx* c, float* ms, int32_t n) {
    if (!c || !ms || n < N_KERNELS) return fail(c, MPPI_ERR_ARG, "ms must hold MPPI_N_KERNELS floats");
    if (!c->profiling) return fail(c, MPPI_ERR_ARG, "profiling is off");
    if (c->profiling == 2) {
        CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
        for (int i = 0; i < N_KERNELS; ++i) ms[i] = NAN;
        CK(cudaEventElapsedTime(&ms[2], c->ev[2], c->ev[3]), "cudaEventElapsedTime");
        return MPPI_OK;
    }
    CK(cudaEventSynchronize(c->ev[N_KERNELS]), "cudaEventSynchronize");
    for (int i = 0; i < N_KERNELS; ++i) CK(cudaEventElapsedTime(&ms[i], c->ev[i], c->ev[i + 1]), "cudaEventElapsedTime");
    return MPPI_OK;
}

const char* mppi_status_string(int status) {
    switch (status) {
        case MPPI_OK: return "MPPI_OK";
        case MPPI_ERR_ARG: return "MPPI_ERR_ARG: invalid argument";
        case MPPI_ERR_OOM: return "MPPI_ERR_OOM: allocation failed";
        case MPPI_ERR_CUDA: return "MPPI_ERR_CUDA: CUDA error";
        case MPPI_ERR_NUMERIC: return "MPPI_ERR_NUMERIC: no finite sample cost";
        case MPPI_ERR_TIMEOUT: return "MPPI_ERR_TIMEOUT: bounded device wait ran out";
        case MPPI_ERR_CAPACITY: return "MPPI_ERR_CAPACITY: size above capacity";
        default: return "unknown status";
    }
}

const char* mppi_last_error(mppi_ctx* c) { return c ? c->err.c_str() : g_err.c_str(); }

}  // extern "C"
