// mppi_batch.cu - many independent MPPI iterations per launch (the batched planner).
//
// A submission carries n plans with their own K, T, reference, obstacles and warm-start
// slot.  All n are computed by one fixed sequence of kernels captured once in a CUDA
// graph: per-plan scene preparation, noise over the flattened (plan, step pair, sample)
// space, ONE persistent rollout kernel whose blocks pull (plan, sample block) tiles, longest
// plans first, from an atomic counter and re-stage a plan's scene into shared memory by
// TMA only when the plan changes, per-plan reductions, and per-plan smoothing and optimal
// rollout.  The per-sample arithmetic is the single-plan path's (mppi_iter.cuh), so a
// plan's result does not depend on which other plans share its submission.
//
// Warm starts live in device slots shared by all pipelines; a pipeline (stream + buffers
// + graph) holds one submission in flight, so several submissions can overlap.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "mppi.h"
#include "mppi_device.cuh"
#include "mppi_internal.h"
#include "mppi_iter.cuh"

namespace mppi {

// One plan of a submission (device descriptor).
struct __align__(16) BatchInst {
    PlanConst pc;
    SceneLayout L;
    int slot;
    int n_kt;             // k-tiles of the weighted sum
    long long z_off;      // noise offset (pairs)
    long long s_off;      // sample offset (S, w)
    long long scene_off;  // bytes
    long long in_off;     // doubles: x0 | ref | circ | centres
    long long table_off;  // float2
    long long out_off;    // doubles: u [T][2] | x [T+1][4]
    long long du_off;     // doubles: [n_kt][T][2]
};

struct __align__(16) BatchHeader {
    int n;                       // plans in this submission
    int n_tiles;                 // rollout tiles
    unsigned tile_counter;       // next rollout tile (zeroed before the rollout kernel)
    int flags;                   // FLAG_TIMEOUT
    long long noise_total;       // sum over plans of K * ceil(T / 2)
    long long wsum_total;        // sum over plans of ceil(T / WS_TT) * n_kt
};

// Per-plan results written by the batched finalize.
struct __align__(16) OutInfo {
    double s_min, eta;
    int argmin, n_finite, status, pad;
    unsigned long long iter;
};

struct BatchArgs {
    BatchHeader* hdr;
    const BatchInst* inst;
    const long long* noise_prefix;   // [n + 1]
    const long long* wsum_prefix;    // [n + 1]
    const int2* tiles;               // (plan, first sample)
    const double* in;                // inputs arena
    double* out;                     // outputs arena
    OutInfo* info;                   // [n]
    DevState* slots;
    double* slot_U;                  // [max_slots][max_T][2]
    int max_T;
    unsigned char* scene;
    float2* table;
    void* z;
    double* S;
    float* w;
    double* du;
};

__device__ __forceinline__ int find_plan(const long long* prefix, int n, long long q) {
    int lo = 0, hi = n;  // prefix[lo] <= q < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= q) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void plan_views(const BatchArgs& a, const BatchInst& d, PlanInputs& in, PlanBuffers& b) {
    const double* x = a.in + d.in_off;
    in.x0 = x;
    in.ref = x + 4;
    in.circ = x + 4 + 2 * d.L.n_ref;
    in.centres = d.pc.has_table ? x + 4 + 2 * d.L.n_ref + 5 * d.L.n_circ : nullptr;
    in.n_ref = d.L.n_ref;
    in.n_circ = d.L.n_circ;
    in.u_out = a.out + d.out_off;
    in.x_out = a.out + d.out_off + 2 * d.pc.T;
    memset(&b, 0, sizeof(b));
    b.state = a.slots + d.slot;
    b.scene = a.scene + d.scene_off;
    b.table = a.table + d.table_off;
    b.S = a.S + d.s_off;
    b.w = a.w + d.s_off;
    b.du_part = a.du + d.du_off;
    b.U = a.slot_U + (size_t)d.slot * a.max_T * 2;
    b.eta_part = &b.state->eta;
    b.n_wblk = 1;
    b.n_kt = d.n_kt;
    b.kt_size = 256 * WS_J;
}

__global__ void __launch_bounds__(256) batch_prep_kernel(BatchArgs a) {
    const int i = blockIdx.x;
    if (i >= a.hdr->n) return;
    const BatchInst& d = a.inst[i];
    PlanInputs in;
    PlanBuffers b;
    plan_views(a, d, in, b);
    prep_scene(d.pc, d.L, in, b, threadIdx.x, blockDim.x);
}

template <bool BF16>
__global__ void __launch_bounds__(256) batch_noise_kernel(BatchArgs a) {
    __shared__ long long pre[1025];
    const int n = a.hdr->n;
    for (int i = threadIdx.x; i <= n; i += blockDim.x) pre[i] = a.noise_prefix[i];
    __syncthreads();
    const long long total = a.hdr->noise_total;
    using NT = typename NoiseT<BF16>::type;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = find_plan(pre, n, q);
        const BatchInst& d = a.inst[i];
        const int K = d.pc.K, T = d.pc.T;
        const long long local = q - pre[i];
        const int j = (int)(local / K), k = (int)(local - (long long)j * K);
        const uint32_t it = (uint32_t)a.slots[d.slot].iter;
        const uint4 wv = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)k, it, d.pc.session),
                                       make_uint2(d.pc.key0, d.pc.key1));
        NT* z = reinterpret_cast<NT*>(a.z) + d.z_off;
        z[(size_t)(2 * j) * K + k] = make_noise<BF16>(uniform24(wv.x), uniform24(wv.y));
        if (2 * j + 1 < T) z[(size_t)(2 * j + 1) * K + k] = make_noise<BF16>(uniform24(wv.z), uniform24(wv.w));
    }
}

// G lanes per sample; TIME: they split the steps, else the work of each step (rollout_sample).
template <int G, bool TIME, bool BF16>
__global__ void __launch_bounds__(BATCH_MAX_THREADS, 2) batch_rollout_kernel(BatchArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned long long bar;
    __shared__ PlanConst s_pc;
    __shared__ SceneLayout s_L;
    __shared__ float4 s_x0;
    __shared__ int s_tile, s_plan, s_moving, s_multi, s_jb0;
    if (threadIdx.x == 0) {
        bulk_init(&bar);
        s_plan = -1;
    }
    __syncthreads();
    uint32_t phase = 0;
    const int n_tiles = a.hdr->n_tiles;
    using NT = typename NoiseT<BF16>::type;
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(&a.hdr->tile_counter, 1u);
        __syncthreads();
        const int tile = s_tile;
        if (tile >= n_tiles) break;
        const int2 td = a.tiles[tile];
        if (td.x != s_plan) {
            __syncthreads();   // every thread has read s_plan and is done with the previous scene
            if (threadIdx.x == 0) {
                const BatchInst& d = a.inst[td.x];
                s_pc = d.pc;
                s_L = d.L;
                const DevState* st = a.slots + d.slot;
                s_x0 = st->x0f;
                s_moving = st->moving;
                s_multi = st->multi_head;
                s_jb0 = (int)(st->jkey & 0xffffffffu);
                s_plan = td.x;
                bulk_issue(smem, a.scene + d.scene_off, d.L.bytes, &bar);
            }
            __syncthreads();
            if (!__syncthreads_and(bulk_wait(&bar, phase, &a.hdr->flags))) return;
            check_smem(s_L, false);
            phase ^= 1u;
            build_boxes(smem, s_L);
        }
        const BatchInst& d = a.inst[td.x];
        const int k = td.y + (int)threadIdx.x / G;   // G lanes per sample
        rollout_sample<G, TIME, BF16, false, false>(s_pc, s_L, smem, a.scene + d.scene_off,
                                       reinterpret_cast<const NT*>(a.z) + d.z_off,
                                       a.table + d.table_off, s_x0, 0.0f, s_moving != 0, s_multi != 0, s_jb0, k,
                                       a.S + d.s_off,
                                       nullptr);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) batch_argmin_kernel(BatchArgs a) {
    const int i = blockIdx.x;
    if (i >= a.hdr->n) return;
    const BatchInst& d = a.inst[i];
    const double* S = a.S + d.s_off;
    MinRec r{INFINITY, 0x7fffffff, 0};
    for (int k = threadIdx.x; k < d.pc.K; k += blockDim.x) {
        const double s = S[k];
        if (isfinite(s)) {
            r.n += 1;
            if (s < r.v) {
                r.v = s;
                r.i = k;
            }
        }
    }
    r = block_min(r);
    if (threadIdx.x == 0) {
        DevState* st = a.slots + d.slot;
        st->s_min = r.v;
        st->argmin = r.n > 0 ? r.i : -1;
        st->n_finite = r.n;
    }
}

__global__ void __launch_bounds__(256) batch_weights_kernel(BatchArgs a) {
    const int i = blockIdx.x;
    if (i >= a.hdr->n) return;
    const BatchInst& d = a.inst[i];
    DevState* st = a.slots + d.slot;
    const double smin = st->s_min;
    const double* S = a.S + d.s_off;
    float* w = a.w + d.s_off;
    double acc = 0.0;
    for (int k = threadIdx.x; k < d.pc.K; k += blockDim.x) {
        const float wk = softmin_weight(S[k], smin, d.pc.inv_lam_f);
        w[k] = wk;
        acc += (double)wk;
    }
    acc = block_sum_d(acc);
    if (threadIdx.x == 0) st->eta = acc;
}

template <bool BF16>
__global__ void __launch_bounds__(256) batch_wsum_kernel(BatchArgs a) {
    __shared__ long long pre[1025];
    const int n = a.hdr->n;
    for (int i = threadIdx.x; i <= n; i += blockDim.x) pre[i] = a.wsum_prefix[i];
    __syncthreads();
    using NT = typename NoiseT<BF16>::type;
    for (long long q = blockIdx.x; q < a.hdr->wsum_total; q += gridDim.x) {
        const int i = find_plan(pre, n, q);
        const BatchInst& d = a.inst[i];
        const int local = (int)(q - pre[i]);
        const int tt = local / d.n_kt, kt = local - tt * d.n_kt;
        const float4* ctl = reinterpret_cast<const float4*>(a.scene + d.scene_off + d.L.off_ctl);
        wsum_tile<BF16>(d.pc, ctl, reinterpret_cast<const NT*>(a.z) + d.z_off, a.w + d.s_off, kt, tt * WS_TT,
                        256 * WS_J, a.du + d.du_off);
    }
}

__global__ void __launch_bounds__(1024) batch_finalize_kernel(BatchArgs a) {
    const int i = blockIdx.x;
    if (i >= a.hdr->n) return;
    const BatchInst& d = a.inst[i];
    PlanInputs in;
    PlanBuffers b;
    plan_views(a, d, in, b);
    if (threadIdx.x == 0 && (a.hdr->flags & FLAG_TIMEOUT)) atomicOr(&b.state->flags, FLAG_TIMEOUT);
    __syncthreads();
    finalize_block(d.pc, b, in);
    __syncthreads();
    if (threadIdx.x == 0) {
        const DevState* st = b.state;
        OutInfo o;
        o.s_min = st->s_min;
        o.eta = st->eta;
        o.argmin = st->argmin;
        o.n_finite = st->n_finite;
        o.status = st->status;
        o.pad = 0;
        o.iter = st->iter_used;
        a.info[i] = o;
    }
}

template <int G, bool TIME, bool BF16>
static cudaError_t set_rollout_smem(size_t smem) {
    return cudaFuncSetAttribute(batch_rollout_kernel<G, TIME, BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(smem < 48 * 1024 ? 48 * 1024 : smem));
}

template <int G, bool TIME, bool BF16>
static int batch_blocks_per_sm(int threads, size_t smem) {
    int n = 0;
    if (set_rollout_smem<G, TIME, BF16>(smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_rollout_kernel<G, TIME, BF16>, threads, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

// Lanes per sample as the group value: g > 0 split the work of each step, g < 0 split the steps.
#define MPPI_BATCH_GROUPS(X) X(1, 1, false) X(2, 2, false) X(4, 4, false) X(8, 8, false) X(16, 16, false) \
    X(32, 32, false) X(-2, 2, true) X(-4, 4, true) X(-8, 8, true)

// The shared-memory attribute must already be set (batch_max_blocks does it), so this
// only launches and may be captured into a graph.
template <bool BF16>
static cudaError_t launch_batch_rollout_b(const BatchArgs& a, int G, int threads, int blocks, size_t smem,
                                          cudaStream_t st) {
    switch (G) {
#define CASE(gv, g, time)                                                            \
    case gv: {                                                                       \
        batch_rollout_kernel<g, time, BF16><<<blocks, threads, smem, st>>>(a);       \
        return cudaGetLastError();                                                   \
    }
        MPPI_BATCH_GROUPS(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

static int batch_max_blocks(int G, int bf16, int threads, size_t smem) {
    switch (G) {
#define CASE(gv, g, time)                                                                                    \
    case gv: return bf16 ? batch_blocks_per_sm<g, time, true>(threads, smem) : batch_blocks_per_sm<g, time, false>(threads, smem);
        MPPI_BATCH_GROUPS(CASE)
#undef CASE
        default: return 0;
    }
}

static int lanes_of(int G) { return G < 0 ? -G : G; }

// Debug build: the index violations this translation unit's kernels counted (then reset).
cudaError_t take_check_hits_batch(unsigned long long* hits) {
#ifdef MPPI_CHECKS
    cudaError_t e = cudaMemcpyFromSymbol(hits, g_check_hits, sizeof(unsigned long long));
    const unsigned long long zero = 0;
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_check_hits, &zero, sizeof(zero));
    return e;
#else
    *hits = 0;
    return cudaSuccess;
#endif
}

}  // namespace mppi

using namespace mppi;

namespace {

constexpr int ALIGN = 256;
size_t up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

struct Pipeline {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_G = 0, graph_threads = 0;
    // device buffers
    unsigned char* d_stage = nullptr;   // header | inst | prefixes | tiles | inputs
    double* d_out = nullptr;            // outputs | info
    unsigned char* scene = nullptr;
    float2* table = nullptr;
    void* z = nullptr;
    double* S = nullptr;
    float* w = nullptr;
    double* du = nullptr;
    // host staging
    unsigned char* h_stage = nullptr;
    unsigned char* h_out = nullptr;
    size_t stage_used = 0, out_used = 0;
    std::vector<mppi_request*> pending;
    std::vector<long long> out_offsets;
    std::vector<long long> s_offsets;   // per plan of the last submission: offset of its costs in S
    std::vector<int> s_counts;          // and its K (kept after the wait for mppi_batch_get_costs)
    bool busy = false;
    BatchArgs args{};
};

}  // namespace

struct mppi_batch {
    int device = 0;
    int max_slots = 0, max_batch = 0, max_T = 0, max_ref = 0, max_circ = 0, noise_bf16 = 0;
    long long max_samples = 0, max_steps = 0, max_tiles = 0;
    size_t max_scene = 0, rollout_smem = 0, max_in = 0, max_out = 0, stage_bytes = 0, out_bytes = 0;
    // offsets inside the staging buffer
    size_t off_inst = 0, off_npre = 0, off_wpre = 0, off_tiles = 0, off_in = 0;
    DevState* slots = nullptr;
    double* slot_U = nullptr;
    int G = 0, threads = 0, n_sm = 0;
    std::vector<Pipeline> pipes;
    std::string err;
    std::mutex mu;
};

static thread_local std::string g_batch_err;

static int bfail(mppi_batch* b, int status, const std::string& msg) {
    if (b) b->err = msg;
    g_batch_err = msg;
    return status;
}

#define BCK(call, what)                                                                           \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return bfail(B, MPPI_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// the single-plan path's parameter conversion, validation and sizes
namespace mppi {
int check_params_shared(const mppi_params* p, std::string& why);
PlanConst make_const_shared(const mppi_params& p);
}  // namespace mppi

static void free_pipe(Pipeline& p) {
    void* dev[] = {p.d_stage, p.d_out, p.scene, p.table, p.z, p.S, p.w, p.du};
    for (void* q : dev)
        if (q) cudaFree(q);
    if (p.h_stage) cudaFreeHost(p.h_stage);
    if (p.h_out) cudaFreeHost(p.h_out);
    if (p.graph) cudaGraphExecDestroy(p.graph);
    if (p.done) cudaEventDestroy(p.done);
    if (p.stream) cudaStreamDestroy(p.stream);
}

static void free_batch(mppi_batch* B) {
    for (auto& p : B->pipes) free_pipe(p);
    if (B->slots) cudaFree(B->slots);
    if (B->slot_U) cudaFree(B->slot_U);
}

static size_t out_elems(int T) { return 2 * (size_t)T + 4 * (size_t)(T + 1); }

extern "C" {

int mppi_batch_create(int32_t max_slots, int32_t max_batch, int64_t max_samples, int64_t max_rollout_steps,
                      int32_t max_T, int32_t max_ref, int32_t max_circ, int32_t noise_bf16, int32_t pipelines,
                      int device, mppi_batch** out) {
    if (!out) return bfail(nullptr, MPPI_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (max_slots < 1 || max_batch < 1 || max_batch > 1024 || max_samples < 1 || max_rollout_steps < 1 ||
        max_T < 1 || max_T > MPPI_MAX_T || max_ref < 2 || max_ref > MPPI_MAX_REF || max_circ < 0 ||
        max_circ > MPPI_MAX_CIRC || pipelines < 1 || pipelines > 16)
        return bfail(nullptr, MPPI_ERR_ARG, "batch capacities out of range");
    mppi_batch* B = new (std::nothrow) mppi_batch();
    if (!B) return bfail(nullptr, MPPI_ERR_OOM, "host allocation failed");
    B->device = device;
    B->max_slots = max_slots;
    B->max_batch = max_batch;
    B->max_T = max_T;
    B->max_ref = max_ref;
    B->max_circ = max_circ;
    B->noise_bf16 = noise_bf16 ? 1 : 0;
    B->max_samples = max_samples;
    B->max_steps = max_rollout_steps;
    B->max_tiles = max_samples / 16 + max_batch;
    const SceneLayout Lmax = make_layout(max_T, max_ref, max_circ);
    B->max_scene = up((size_t)Lmax.total);
    B->rollout_smem = up(rollout_smem_bytes(Lmax, BATCH_MAX_THREADS, false));   // blob and the boxes built after it
    B->max_in = 4 + 2 * (size_t)max_ref + 5 * (size_t)max_circ + 2 * (size_t)max_T * max_circ;
    B->max_out = out_elems(max_T);
    auto bail = [&](int st) {
        free_batch(B);
        delete B;
        return st;
    };
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return bail(bfail(nullptr, MPPI_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e)));
    cudaDeviceGetAttribute(&B->n_sm, cudaDevAttrMultiProcessorCount, device);
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (B->rollout_smem + 1024 > (size_t)max_smem)
        return bail(bfail(nullptr, MPPI_ERR_CAPACITY, "scene of max_T, max_ref, max_circ exceeds shared memory"));
    // staging layout
    size_t o = up(sizeof(BatchHeader));
    B->off_inst = o;  o += up(sizeof(BatchInst) * (size_t)max_batch);
    B->off_npre = o;  o += up(sizeof(long long) * ((size_t)max_batch + 1));
    B->off_wpre = o;  o += up(sizeof(long long) * ((size_t)max_batch + 1));
    B->off_tiles = o; o += up(sizeof(int2) * (size_t)B->max_tiles);
    B->off_in = o;    o += up(sizeof(double) * B->max_in * (size_t)max_batch);
    B->stage_bytes = o;
    B->out_bytes = up(sizeof(double) * B->max_out * (size_t)max_batch) + up(sizeof(OutInfo) * (size_t)max_batch);
    if (cudaMalloc(&B->slots, sizeof(DevState) * (size_t)max_slots) != cudaSuccess ||
        cudaMalloc(&B->slot_U, sizeof(double) * 2 * (size_t)max_T * max_slots) != cudaSuccess)
        return bail(bfail(nullptr, MPPI_ERR_OOM, "slot allocation failed"));
    std::vector<DevState> s0((size_t)max_slots);
    memset(s0.data(), 0, sizeof(DevState) * s0.size());
    for (auto& s : s0) s.jkey = ~0ull;
    if (cudaMemcpy(B->slots, s0.data(), sizeof(DevState) * s0.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(B->slot_U, 0, sizeof(double) * 2 * (size_t)max_T * max_slots) != cudaSuccess)
        return bail(bfail(nullptr, MPPI_ERR_CUDA, "slot initialisation failed"));
    const long long max_kt_tiles = max_samples / (256 * WS_J) + max_batch;
    B->pipes.resize((size_t)pipelines);
    for (auto& p : B->pipes) {
        const size_t zb = (size_t)max_rollout_steps * (B->noise_bf16 ? 4 : 8);
        bool ok = cudaStreamCreateWithFlags(&p.stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&p.done, cudaEventDisableTiming) == cudaSuccess &&
                  cudaMalloc(&p.d_stage, B->stage_bytes) == cudaSuccess &&
                  cudaMalloc(&p.d_out, B->out_bytes) == cudaSuccess &&
                  cudaMalloc(&p.scene, B->max_scene * (size_t)max_batch) == cudaSuccess &&
                  cudaMalloc(&p.table, sizeof(float2) * (size_t)max_T * std::max(max_circ, 1) * max_batch) ==
                      cudaSuccess &&
                  cudaMalloc(&p.z, zb) == cudaSuccess && cudaMalloc(&p.S, sizeof(double) * max_samples) == cudaSuccess &&
                  cudaMalloc(&p.w, sizeof(float) * max_samples) == cudaSuccess &&
                  cudaMalloc(&p.du, sizeof(double) * 2 * (size_t)max_T * max_kt_tiles) == cudaSuccess &&
                  cudaMallocHost(&p.h_stage, B->stage_bytes) == cudaSuccess &&
                  cudaMallocHost(&p.h_out, B->out_bytes) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return bail(bfail(nullptr, MPPI_ERR_OOM, "pipeline allocation failed"));
        }
        BatchArgs& a = p.args;
        a.hdr = reinterpret_cast<BatchHeader*>(p.d_stage);
        a.inst = reinterpret_cast<const BatchInst*>(p.d_stage + B->off_inst);
        a.noise_prefix = reinterpret_cast<const long long*>(p.d_stage + B->off_npre);
        a.wsum_prefix = reinterpret_cast<const long long*>(p.d_stage + B->off_wpre);
        a.tiles = reinterpret_cast<const int2*>(p.d_stage + B->off_tiles);
        a.in = reinterpret_cast<const double*>(p.d_stage + B->off_in);
        a.out = p.d_out;
        a.info = reinterpret_cast<OutInfo*>(reinterpret_cast<unsigned char*>(p.d_out) +
                                            up(sizeof(double) * B->max_out * (size_t)max_batch));
        a.slots = B->slots;
        a.slot_U = B->slot_U;
        a.max_T = max_T;
        a.scene = p.scene;
        a.table = p.table;
        a.z = p.z;
        a.S = p.S;
        a.w = p.w;
        a.du = p.du;
    }
    // default launch shape of the rollout until mppi_batch_autotune chooses
    B->G = 4;
    B->threads = 128;
    *out = B;
    return MPPI_OK;
}

int mppi_batch_destroy(mppi_batch* B) {
    if (!B) return MPPI_OK;
    cudaSetDevice(B->device);
    for (auto& p : B->pipes)
        if (p.stream) cudaStreamSynchronize(p.stream);
    free_batch(B);
    delete B;
    return MPPI_OK;
}

}  // extern "C"

static bool finite_n(const double* v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!isfinite(v[i])) return false;
    return true;
}

// Builds the staging image of a submission in p.h_stage; returns the status.
static int build_submission(mppi_batch* B, Pipeline& p, mppi_request* req, int n) {
    if (n < 1 || n > B->max_batch) return bfail(B, MPPI_ERR_CAPACITY, "number of plans outside [1, max_batch]");
    std::vector<char> used((size_t)B->max_slots, 0);
    BatchHeader* H = reinterpret_cast<BatchHeader*>(p.h_stage);
    BatchInst* I = reinterpret_cast<BatchInst*>(p.h_stage + B->off_inst);
    long long* npre = reinterpret_cast<long long*>(p.h_stage + B->off_npre);
    long long* wpre = reinterpret_cast<long long*>(p.h_stage + B->off_wpre);
    int2* tiles = reinterpret_cast<int2*>(p.h_stage + B->off_tiles);
    double* inp = reinterpret_cast<double*>(p.h_stage + B->off_in);
    long long z_off = 0, s_off = 0, in_off = 0, table_off = 0, out_off = 0, du_off = 0, scene_off = 0;
    long long noise = 0, wsum = 0, n_tiles = 0;
    const int spt = B->threads / lanes_of(B->G);   // samples per rollout tile
    p.out_offsets.assign((size_t)n, 0);
    p.s_offsets.assign((size_t)n, 0);
    p.s_counts.assign((size_t)n, 0);
    std::vector<std::pair<double, int>> cost((size_t)n);
    for (int i = 0; i < n; ++i) {
        mppi_request& r = req[i];
        std::string why;
        if (!r.params || check_params_shared(r.params, why) != MPPI_OK)
            return bfail(B, MPPI_ERR_ARG, "plan " + std::to_string(i) + ": " + (r.params ? why : "params NULL"));
        const mppi_params& pr = *r.params;
        if (pr.model != 0 || pr.cost_to_go != 0)
            return bfail(B, MPPI_ERR_ARG, "the batch engine runs model 0 with whole-cost weights");
        if (pr.noise_bf16 != B->noise_bf16) return bfail(B, MPPI_ERR_ARG, "noise precision differs from the batch's");
        if (r.slot < 0 || r.slot >= B->max_slots || used[(size_t)r.slot])
            return bfail(B, MPPI_ERR_ARG, "slot out of range or used twice in one submission");
        used[(size_t)r.slot] = 1;
        if (!r.x0 || !r.ref_xy || !r.u_out || !r.x_out || (r.n_circ > 0 && !r.circ) || r.n_ref < 2 || r.n_circ < 0)
            return bfail(B, MPPI_ERR_ARG, "plan " + std::to_string(i) + ": bad arrays");
        if (pr.T > B->max_T || r.n_ref > B->max_ref || r.n_circ > B->max_circ)
            return bfail(B, MPPI_ERR_CAPACITY, "plan " + std::to_string(i) + ": size above the batch capacity");
        const int T = pr.T, K = pr.K;
        const size_t nr = 2 * (size_t)r.n_ref, nc = 5 * (size_t)r.n_circ, nt = r.centres ? 2 * (size_t)T * r.n_circ : 0;
        if (!finite_n(r.x0, 4) || !finite_n(r.ref_xy, nr) || (nc && !finite_n((const double*)r.circ, nc)) ||
            (nt && !finite_n(r.centres, nt)))
            return bfail(B, MPPI_ERR_ARG, "plan " + std::to_string(i) + ": non-finite input");
        BatchInst& d = I[i];
        memset(&d, 0, sizeof(d));
        d.pc = make_const_shared(pr);
        d.pc.has_table = nt ? 1 : 0;
        d.L = make_layout(T, r.n_ref, r.n_circ);
        d.slot = r.slot;
        d.n_kt = (K + 256 * WS_J - 1) / (256 * WS_J);
        d.z_off = z_off;
        d.s_off = s_off;
        d.scene_off = scene_off;
        d.in_off = in_off;
        d.table_off = table_off;
        d.out_off = out_off;
        d.du_off = du_off;
        double* x = inp + in_off;
        memcpy(x, r.x0, 4 * sizeof(double));
        memcpy(x + 4, r.ref_xy, nr * sizeof(double));
        if (nc) memcpy(x + 4 + nr, r.circ, nc * sizeof(double));
        if (nt) memcpy(x + 4 + nr + nc, r.centres, nt * sizeof(double));
        npre[i] = noise;
        wpre[i] = wsum;
        noise += (long long)K * ((T + 1) / 2);
        wsum += (long long)((T + WS_TT - 1) / WS_TT) * d.n_kt;
        p.out_offsets[(size_t)i] = out_off;
        p.s_offsets[(size_t)i] = s_off;
        p.s_counts[(size_t)i] = K;
        z_off += (long long)K * T;
        s_off += K;
        scene_off += (long long)up((size_t)d.L.total);
        in_off += (long long)(4 + nr + nc + nt);
        table_off += (long long)T * std::max(r.n_circ, 1);
        out_off += (long long)out_elems(T);
        du_off += 2LL * T * d.n_kt;
        cost[(size_t)i] = {(double)T * (700.0 + 20.0 * r.n_circ + 2.0 * r.n_ref / 16.0), i};
    }
    if (s_off > B->max_samples || z_off > B->max_steps)
        return bfail(B, MPPI_ERR_CAPACITY, "submission above the batch's sample or rollout-step capacity");
    npre[n] = noise;
    wpre[n] = wsum;
    // rollout tiles, most expensive plans first
    std::stable_sort(cost.begin(), cost.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    for (auto& c : cost) {
        const int i = c.second;
        for (int k0 = 0; k0 < I[i].pc.K; k0 += spt) {
            if (n_tiles >= B->max_tiles) return bfail(B, MPPI_ERR_CAPACITY, "too many rollout tiles");
            tiles[n_tiles++] = make_int2(i, k0);
        }
    }
    memset(H, 0, sizeof(*H));
    H->n = n;
    H->n_tiles = (int)n_tiles;
    H->noise_total = noise;
    H->wsum_total = wsum;
    // the staged region is contiguous up to the end of the used inputs
    p.stage_used = B->off_in + sizeof(double) * (size_t)in_off;
    p.out_used = (size_t)out_off;
    return MPPI_OK;
}

static cudaError_t enqueue_kernels(mppi_batch* B, Pipeline& p, int per_sm) {
    const BatchArgs& a = p.args;
    const cudaStream_t st = p.stream;
    cudaError_t e;
    batch_prep_kernel<<<B->max_batch, 256, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int grid = B->n_sm * 8;
    if (B->noise_bf16) batch_noise_kernel<true><<<grid, 256, 0, st>>>(a);
    else batch_noise_kernel<false><<<grid, 256, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(&a.hdr->tile_counter, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
    const size_t smem = B->rollout_smem;
    if (B->noise_bf16) e = launch_batch_rollout_b<true>(a, B->G, B->threads, B->n_sm * per_sm, smem, st);
    else e = launch_batch_rollout_b<false>(a, B->G, B->threads, B->n_sm * per_sm, smem, st);
    if (e != cudaSuccess) return e;
    batch_argmin_kernel<<<B->max_batch, 256, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    batch_weights_kernel<<<B->max_batch, 256, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (B->noise_bf16) batch_wsum_kernel<true><<<grid, 256, 0, st>>>(a);
    else batch_wsum_kernel<false><<<grid, 256, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    batch_finalize_kernel<<<B->max_batch, 1024, 0, st>>>(a);
    return cudaGetLastError();
}

// The kernel sequence of a pipeline, captured once per rollout launch shape.
static cudaError_t ensure_graph(mppi_batch* B, Pipeline& p) {
    if (p.graph && p.graph_G == B->G && p.graph_threads == B->threads) return cudaSuccess;
    if (p.graph) {
        cudaGraphExecDestroy(p.graph);
        p.graph = nullptr;
    }
    // configure function attributes outside the capture
    const int per_sm = batch_max_blocks(B->G, B->noise_bf16, B->threads, B->rollout_smem);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(p.stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t ek = enqueue_kernels(B, p, per_sm);
    e = cudaStreamEndCapture(p.stream, &g);
    if (ek != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return ek;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&p.graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
    p.graph_G = B->G;
    p.graph_threads = B->threads;
    return cudaSuccess;
}

extern "C" {

int mppi_batch_submit(mppi_batch* B, mppi_request* req, int32_t n, int32_t* ticket) {
    if (!B || !req || !ticket) return bfail(B, MPPI_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(B->mu);
    BCK(cudaSetDevice(B->device), "cudaSetDevice");
    int pi = -1;
    for (size_t i = 0; i < B->pipes.size(); ++i)
        if (!B->pipes[i].busy) {
            pi = (int)i;
            break;
        }
    if (pi < 0) return bfail(B, MPPI_ERR_CAPACITY, "every pipeline has a submission in flight");
    Pipeline& p = B->pipes[(size_t)pi];
    int rc = build_submission(B, p, req, n);
    if (rc != MPPI_OK) return rc;
    BCK(ensure_graph(B, p), "graph capture");
    BCK(cudaMemcpyAsync(p.d_stage, p.h_stage, p.stage_used, cudaMemcpyHostToDevice, p.stream), "input copy");
    BCK(cudaGraphLaunch(p.graph, p.stream), "graph launch");
    BCK(cudaMemcpyAsync(p.h_out, p.d_out, sizeof(double) * p.out_used, cudaMemcpyDeviceToHost, p.stream),
        "output copy");
    BCK(cudaMemcpyAsync(p.h_out + up(sizeof(double) * B->max_out * (size_t)B->max_batch), p.args.info,
                        sizeof(OutInfo) * (size_t)n, cudaMemcpyDeviceToHost, p.stream),
        "info copy");
    BCK(cudaEventRecord(p.done, p.stream), "event record");
    p.pending.assign((size_t)n, nullptr);
    for (int i = 0; i < n; ++i) p.pending[(size_t)i] = &req[i];
    p.busy = true;
    *ticket = pi;
    return MPPI_OK;
}

int mppi_batch_wait(mppi_batch* B, int32_t ticket) {
    if (!B || ticket < 0 || ticket >= (int)B->pipes.size()) return bfail(B, MPPI_ERR_ARG, "bad ticket");
    Pipeline& p = B->pipes[(size_t)ticket];
    if (!p.busy) return bfail(B, MPPI_ERR_ARG, "ticket has no submission in flight");
    BCK(cudaSetDevice(B->device), "cudaSetDevice");
    cudaError_t e = cudaEventSynchronize(p.done);
    std::lock_guard<std::mutex> lock(B->mu);
    p.busy = false;
    if (e != cudaSuccess) return bfail(B, MPPI_ERR_CUDA, std::string("batch: ") + cudaGetErrorString(e));
    const OutInfo* info = reinterpret_cast<const OutInfo*>(p.h_out + up(sizeof(double) * B->max_out * (size_t)B->max_batch));
    const double* outs = reinterpret_cast<const double*>(p.h_out);
    int worst = MPPI_OK;
    for (size_t i = 0; i < p.pending.size(); ++i) {
        mppi_request& r = *p.pending[i];
        const OutInfo& o = info[i];
        r.status = o.status;
        if (o.status == MPPI_OK) {
            const int T = r.params->T;
            memcpy(r.u_out, outs + p.out_offsets[i], 2 * (size_t)T * sizeof(double));
            memcpy(r.x_out, outs + p.out_offsets[i] + 2 * T, 4 * (size_t)(T + 1) * sizeof(double));
        } else if (worst == MPPI_OK) {
            worst = o.status;
        }
        if (r.info) {
            r.info->argmin = o.argmin;
            r.info->n_finite = o.n_finite;
            r.info->s_min = o.s_min;
            r.info->eta = o.eta;
            r.info->iter = o.iter;
        }
    }
    p.pending.clear();
    if (worst != MPPI_OK) return bfail(B, worst, "some plans of the submission failed (see their status)");
    return MPPI_OK;
}

}  // extern "C"

// 1 when the submission on the ticket's pipeline has finished on the device, 0 while it runs,
// MPPI_ERR_* on a bad ticket or a failed query (the server's watchdog polls it).
int batch_ticket_done(mppi_batch* B, int32_t ticket) {
    if (!B || ticket < 0 || ticket >= (int)B->pipes.size()) return MPPI_ERR_ARG;
    Pipeline& p = B->pipes[(size_t)ticket];
    if (!p.busy) return MPPI_ERR_ARG;
    if (cudaSetDevice(B->device) != cudaSuccess) return MPPI_ERR_CUDA;
    const cudaError_t e = cudaEventQuery(p.done);
    if (e == cudaSuccess) return 1;
    if (e == cudaErrorNotReady) return 0;
    return MPPI_ERR_CUDA;
}

extern "C" {

int mppi_batch_plan(mppi_batch* B, mppi_request* req, int32_t n) {
    int32_t t = -1;
    int rc = mppi_batch_submit(B, req, n, &t);
    if (rc != MPPI_OK) return rc;
    return mppi_batch_wait(B, t);
}

int mppi_batch_autotune(mppi_batch* B, mppi_request* req, int32_t n, int32_t* group, int32_t* block) {
    if (!B || !req) return bfail(B, MPPI_ERR_ARG, "NULL argument");
    BCK(cudaSetDevice(B->device), "cudaSetDevice");
    Pipeline& p = B->pipes[0];
    if (p.busy) return bfail(B, MPPI_ERR_CAPACITY, "pipeline 0 has a submission in flight");
    const int saveG = B->G, saveT = B->threads;
    float best = INFINITY;
    int bg = saveG, bt = saveT;
    const int groups[] = {1, 2, 4, 8, 16, 32, -2, -4, -8};
    const int sizes[] = {64, 128, 256, BATCH_MAX_THREADS};
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0), "cudaEventCreate");
    BCK(cudaEventCreate(&e1), "cudaEventCreate");
    int rc = MPPI_OK;
    // prep and noise once (the warm starts and counters of the slots are not changed)
    B->G = 4;
    B->threads = 128;
    rc = build_submission(B, p, req, n);
    cudaError_t e = cudaSuccess;
    if (rc == MPPI_OK) e = cudaMemcpyAsync(p.d_stage, p.h_stage, p.stage_used, cudaMemcpyHostToDevice, p.stream);
    if (rc == MPPI_OK && e == cudaSuccess) {
        batch_prep_kernel<<<B->max_batch, 256, 0, p.stream>>>(p.args);
        if (B->noise_bf16) batch_noise_kernel<true><<<B->n_sm * 8, 256, 0, p.stream>>>(p.args);
        else batch_noise_kernel<false><<<B->n_sm * 8, 256, 0, p.stream>>>(p.args);
        e = cudaGetLastError();
    }
    for (int gi = 0; gi < 9 && rc == MPPI_OK && e == cudaSuccess; ++gi) {
        for (int si = 0; si < 4 && e == cudaSuccess; ++si) {
            const int G = groups[gi], th = sizes[si];
            if (th / lanes_of(G) < 16) continue;   // at least 16 samples per tile
            const int per_sm = batch_max_blocks(G, B->noise_bf16, th, B->rollout_smem);
            if (per_sm < 1) continue;
            B->G = G;
            B->threads = th;
            rc = build_submission(B, p, req, n);   // tiles depend on samples per tile
            if (rc != MPPI_OK) break;
            e = cudaMemcpyAsync(p.d_stage, p.h_stage, p.stage_used, cudaMemcpyHostToDevice, p.stream);
            float ms = 0.0f;
            for (int r = 0; r < 2 && e == cudaSuccess; ++r) {
                if (e == cudaSuccess) e = cudaMemsetAsync(&p.args.hdr->tile_counter, 0, sizeof(unsigned), p.stream);
                if (e == cudaSuccess) e = cudaEventRecord(e0, p.stream);
                if (e == cudaSuccess)
                    e = B->noise_bf16 ? launch_batch_rollout_b<true>(p.args, G, th, B->n_sm * per_sm, B->rollout_smem, p.stream)
                                      : launch_batch_rollout_b<false>(p.args, G, th, B->n_sm * per_sm, B->rollout_smem, p.stream);
                if (e == cudaSuccess) e = cudaEventRecord(e1, p.stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            }
            if (e == cudaSuccess && ms < best) {
                best = ms;
                bg = G;
                bt = th;
            }
        }
    }
    // leave the slots as they were: prep only accumulated the per-iteration fields
    for (int i = 0; i < n && rc == MPPI_OK && e == cudaSuccess; ++i) e = launch_reset_state(B->slots + req[i].slot, p.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p.stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B->G = (rc == MPPI_OK && e == cudaSuccess) ? bg : saveG;
    B->threads = (rc == MPPI_OK && e == cudaSuccess) ? bt : saveT;
    if (rc != MPPI_OK) return rc;
    if (e != cudaSuccess) return bfail(B, MPPI_ERR_CUDA, std::string("batch autotune: ") + cudaGetErrorString(e));
    if (group) *group = B->G;
    if (block) *block = B->threads;
    return MPPI_OK;
}

int mppi_batch_set_launch(mppi_batch* B, int32_t group, int32_t block) {
    if (!B) return bfail(B, MPPI_ERR_ARG, "NULL argument");
    bool known = false;
#define CASE(gv, g, time) known |= group == gv;
    MPPI_BATCH_GROUPS(CASE)
#undef CASE
    if (!known || block < 32 || block > BATCH_MAX_THREADS || block % 32 != 0 || block / lanes_of(group) < 16)
        return bfail(B, MPPI_ERR_ARG, "group must be 1..32 or -2, -4, -8; block a multiple of 32 up to 448 with "
                                      "at least 16 samples per block");
    for (auto& p : B->pipes)
        if (p.busy) return bfail(B, MPPI_ERR_CAPACITY, "a submission is in flight");
    BCK(cudaSetDevice(B->device), "cudaSetDevice");
    if (batch_max_blocks(group, B->noise_bf16, block, B->rollout_smem) < 1)
        return bfail(B, MPPI_ERR_CAPACITY, "launch shape does not fit the shared memory of a block");
    B->G = group;
    B->threads = block;
    return MPPI_OK;
}

int mppi_batch_set_controls(mppi_batch* B, int32_t slot, const double* U, int32_t T, uint64_t iter) {
    if (!B || !U || slot < 0 || slot >= B->max_slots || T < 1 || T > B->max_T) return bfail(B, MPPI_ERR_ARG, "bad argument");
    if (!finite_n(U, 2 * (size_t)T)) return bfail(B, MPPI_ERR_ARG, "non-finite controls");
    BCK(cudaSetDevice(B->device), "cudaSetDevice");
    BCK(cudaMemcpy(B->slot_U + (size_t)slot * B->max_T * 2, U, sizeof(double) * 2 * T, cudaMemcpyHostToDevice),
        "controls copy");
    unsigned long long it = iter;
    BCK(cudaMemcpy(&B->slots[slot].iter, &it, sizeof(it), cudaMemcpyHostToDevice), "iter copy");
    return MPPI_OK;
}

int mppi_batch_get_controls(mppi_batch* B, int32_t slot, double* U, int32_t T, uint64_t* iter) {
    if (!B || !U || slot < 0 || slot >= B->max_slots || T < 1 || T > B->max_T) return bfail(B, MPPI_ERR_ARG, "bad argument");
    BCK(cudaSetDevice(B->device), "cudaSetDevice");
    BCK(cudaMemcpy(U, B->slot_U + (size_t)slot * B->max_T * 2, sizeof(double) * 2 * T, cudaMemcpyDeviceToHost),
        "controls copy");
    unsigned long long it = 0;
    BCK(cudaMemcpy(&it, &B->slots[slot].iter, sizeof(it), cudaMemcpyDeviceToHost), "iter copy");
    if (iter) *iter = it;
    return MPPI_OK;
}

int mppi_batch_get_costs(mppi_batch* B, int32_t ticket, int32_t i, double* S, int32_t K) {
    if (!B || !S || ticket < 0 || ticket >= (int)B->pipes.size()) return bfail(B, MPPI_ERR_ARG, "bad argument");
    std::lock_guard<std::mutex> lock(B->mu);
    Pipeline& p = B->pipes[(size_t)ticket];
    if (p.busy) return bfail(B, MPPI_ERR_CAPACITY, "the pipeline has a submission in flight");
    if (i < 0 || i >= (int)p.s_counts.size() || K != p.s_counts[(size_t)i])
        return bfail(B, MPPI_ERR_ARG, "no such plan in the pipeline's last submission, or K differs");
    BCK(cudaSetDevice(B->device), "cudaSetDevice");
    BCK(cudaMemcpy(S, p.S + p.s_offsets[(size_t)i], sizeof(double) * (size_t)K, cudaMemcpyDeviceToHost), "costs copy");
    return MPPI_OK;
}

const char* mppi_batch_last_error(mppi_batch* B) { return B ? B->err.c_str() : g_batch_err.c_str(); }

}  // extern "C"
