// mppi_kernels.cu - the CUDA kernels of one MPPI iteration (arXiv 2308.01654, Algorithm 1), sm_103a.
//
//   prep      reference polyline, obstacle circles and controls -> scene blob (local frame, binary32)
//   noise     Philox4x32-10 + Box-Muller -> z[T][K]                    (Algorithm 1 GenerateRandomNoise)
//             (prep and noise are one launch, their blocks side by side)
//   rollout   fused Euler rollout of Eq. (5) + step costs of Eq. (12)-(18) -> S[K]
//             with S_min and its index from the rollout's last block      (Algorithm 1, S_min)
//   weights   w_k = exp(-(S_k - S_min) / lambda), eta partials in binary64  (Eq. (11))
//   wsum      sum_k w_k eps'_{t,k} per step, eps' recomputed from z      (Eq. (11))
//   finalize  u + du, clamp, Savitzky-Golay (Eq. (19)), clamp, x* by prefix scans, warm start
#include <math.h>

#include <atomic>

#include "mppi_device.cuh"
#include "mppi_internal.h"
#include "mppi_iter.cuh"
#include "mppi_trace.h"

namespace mppi {

static inline int align16(int x) { return (x + 15) & ~15; }

SceneLayout make_layout(int T, int n_ref, int n_circ) {
    SceneLayout L;
    L.T = T;
    L.n_ref = n_ref;
    L.n_seg = n_ref - 1;
    L.n_l1 = (L.n_seg + REF_L1 - 1) / REF_L1;
    L.n_l2 = (L.n_l1 + REF_L2 - 1) / REF_L2;
    L.n_circ = n_circ;
    int o = 0;
    L.off_ctl = o;  o = align16(o + 16 * T);
    L.off_c0 = o;   o = align16(o + 4 * T);
    L.off_vert = o; o = align16(o + 8 * n_ref);
    L.off_seg = o;  o = align16(o + 16 * L.n_seg);
    L.off_head = o; o = align16(o + 4 * L.n_seg);
    L.off_l1 = o;   o = align16(o + 16 * L.n_l1);
    L.off_circ = o; o = align16(o + 16 * n_circ);
    L.off_vel = o;  o = align16(o + 8 * n_circ);
    L.off_disp = o; o = align16(o + 4 * n_circ);
    L.off_proj = o; o = align16(o + 16);
    L.off_order = o; o = align16(o + 4 * n_circ);
    L.off_skey = o; o = align16(o + 4 * n_circ);
    L.bytes = o;
    L.off_pbox = o; o = align16(o + 16 * n_ref);
    L.off_sbox = o; o = align16(o + 16 * n_ref);
    L.total = o;
    return L;
}

// the staged blob and what each block builds after it (block_extra_bytes)
size_t rollout_smem_bytes(const SceneLayout& L, int threads, bool model1) {
    return (size_t)L.bytes + block_extra_bytes(L) + steer_slots_bytes(threads, model1);
}

// A launch chained to the previous kernel on the stream (programmatic stream serialisation,
// see pdl_wait): its blocks may be scheduled while the predecessor drains.
template <typename... KArgs, typename... Args>
static cudaError_t launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                  Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// -----------------------------------------------------------------------------
// noise: one thread per (step pair j, sample k); coalesced stores along k.  The
// bfloat16 form stores the binary32 normals rounded and lists the pairs that lie within
// the binary32 error bound of a rounding midpoint; noise_fix_kernel takes their rounding
// again on the exact (binary64) normals, so the stored codes are those of the exact values.
// -----------------------------------------------------------------------------
template <bool BF16>
__device__ __forceinline__ void noise_pair(const PlanConst& pc, const DevState* st, typename NoiseT<BF16>::type* z,
                                           unsigned* fix_count, uint2* fix_list, int k, int j) {
    if (k >= pc.K) return;
    const uint32_t it = (uint32_t)st->iter;
    // the counter takes the sample's global index (k_offset: first sample of a K-slice)
    const uint4 w = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)k + pc.k_offset, it, pc.session),
                                  make_uint2(pc.key0, pc.key1));
    const size_t K = (size_t)pc.K;
    const bool two = 2 * j + 1 < pc.T;
    const unsigned long long keep = l2_keep_policy();
    if constexpr (BF16) {
        const float2 za = box_muller(uniform24(w.x), uniform24(w.y));
        const float2 zb = box_muller(uniform24(w.z), uniform24(w.w));
        store_keep(z + (size_t)(2 * j) * K + k, NoiseT<true>::pack(za), keep);
        if (two) store_keep(z + (size_t)(2 * j + 1) * K + k, NoiseT<true>::pack(zb), keep);
        const bool fix = near_bf16_midpoint(za.x) || near_bf16_midpoint(za.y) ||
                         (two && (near_bf16_midpoint(zb.x) || near_bf16_midpoint(zb.y)));
        if (fix) {
            const unsigned i = atomicAdd(fix_count, 1u);
            if (i < NOISE_FIX_CAP) {
                fix_list[i] = make_uint2((unsigned)j, (unsigned)k);
            } else {
                z[(size_t)(2 * j) * K + k] = make_noise<true>(uniform24(w.x), uniform24(w.y));
                if (two) z[(size_t)(2 * j + 1) * K + k] = make_noise<true>(uniform24(w.z), uniform24(w.w));
            }
        }
    } else {
        store_keep(z + (size_t)(2 * j) * K + k, make_noise<false>(uniform24(w.x), uniform24(w.y)), keep);
        if (two) store_keep(z + (size_t)(2 * j + 1) * K + k, make_noise<false>(uniform24(w.z), uniform24(w.w)), keep);
    }
}

// -----------------------------------------------------------------------------
// prep + noise, the first launch of an iteration.  prep makes one pass over the inputs:
// positions are shifted into a frame centred on (x0, y0) in binary64 before rounding, so
// binary32 keeps its resolution where the rollouts happen.  Its blocks come first in the grid
// (prep_x blocks for each phase of prep_scene), the noise blocks (nkb per step pair) after
// them: prep needs the inputs and noise only the seed and the iteration counter, so the two
// run side by side, and the next kernel chains to this one launch.  Launch bounds of the
// noise (eight blocks of 256 per SM).
// -----------------------------------------------------------------------------
template <bool BF16>
__global__ void __launch_bounds__(256, 8) prep_noise_kernel(PlanConst pc, SceneLayout L, PlanInputs in,
                                                            PlanBuffers b, int prep_x, int nkb,
                                                            typename NoiseT<BF16>::type* z) {
    const int n_prep = prep_x * PREP_PHASES;
    const int lin = (int)blockIdx.x;
    if (lin < n_prep) {
        pdl_trigger();
        const int phase = lin / prep_x, bx = lin - phase * prep_x;
        prep_scene(pc, L, in, b, bx * blockDim.x + threadIdx.x, prep_x * blockDim.x, phase);
        return;
    }
    const int r = lin - n_prep, j = r / nkb, kb = r - j * nkb;
    noise_pair<BF16>(pc, b.state, z, b.fix_count, b.fix_list, kb * blockDim.x + threadIdx.x, j);
}

// One warp per block and four blocks per SM, so the few binary64 Box-Muller pairs spread
// over every SM's binary64 pipe.
__global__ void __launch_bounds__(32) noise_fix_kernel(PlanConst pc, const DevState* st, __nv_bfloat162* z,
                                                       const unsigned* fix_count, const uint2* fix_list) {
    pdl_wait();
    pdl_trigger();
    const unsigned n = min(*fix_count, NOISE_FIX_CAP);
    const uint32_t it = (uint32_t)st->iter;
    const size_t K = (size_t)pc.K;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint2 jk = fix_list[i];
        const uint4 w = philox4x32_10(make_uint4(jk.x, jk.y + pc.k_offset, it, pc.session), make_uint2(pc.key0, pc.key1));
        z[(size_t)(2 * jk.x) * K + jk.y] = make_noise<true>(uniform24(w.x), uniform24(w.y));
        if (2 * (int)jk.x + 1 < pc.T)
            z[(size_t)(2 * jk.x + 1) * K + jk.y] = make_noise<true>(uniform24(w.z), uniform24(w.w));
    }
}

static cudaError_t launch_prep_noise_k(const PlanConst& pc, const SceneLayout& L, const PlanBuffers& b,
                                       const PlanInputs& in, int noise_bf16, cudaStream_t st) {
    int items = L.n_ref;
    items = max(items, L.T);
    items = max(items, L.n_circ);
    if (in.centres) items = max(items, L.T * L.n_circ);
    const int prep_x = min(max((items + 255) / 256, 1), 148);
    const int nkb = (pc.K + 255) / 256, njp = (pc.T + 1) / 2;
    const long long blocks = (long long)prep_x * PREP_PHASES + (long long)nkb * njp;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (noise_bf16)
        prep_noise_kernel<true><<<(unsigned)blocks, 256, 0, st>>>(pc, L, in, b, prep_x, nkb,
                                                                  reinterpret_cast<__nv_bfloat162*>(b.z));
    else
        prep_noise_kernel<false><<<(unsigned)blocks, 256, 0, st>>>(pc, L, in, b, prep_x, nkb,
                                                                   reinterpret_cast<float2*>(b.z));
    return cudaGetLastError();
}

// the bfloat16 form's fix-up of the listed pairs, chained after the prep + noise launch
static cudaError_t launch_noise_fix(const PlanConst& pc, const PlanBuffers& b, cudaStream_t st) {
    return launch_chained(noise_fix_kernel, dim3(4 * 152), dim3(32), 0, st, pc, (const DevState*)b.state,
                          reinterpret_cast<__nv_bfloat162*>(b.z), (const unsigned*)b.fix_count,
                          (const uint2*)b.fix_list);
}

__global__ void philox_kernel(uint2 key, const uint4* ctr, uint4* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], key);
}

// SIMPLE: the plan's parameters allow the specialised step (see rollout_sample); the block then
// takes it when scene preparation found the circles static and the lane of one heading, and the
// general step otherwise (a block-uniform choice; both give the same bits).
template <int G, bool TIME, bool BF16, bool STATS, bool EXT, bool SIMPLE = false>
__global__ void __launch_bounds__(MAX_ROLLOUT_THREADS, 1) rollout_kernel(PlanConst pc, SceneLayout L, PlanBuffers b,
                                                        const typename NoiseT<BF16>::type* __restrict__ z) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned long long bar;
    pdl_wait();
    check_smem(L, pc.model == 1);
    const bool staged = __syncthreads_and(stage_to_smem(smem, b.scene, L.bytes, &bar, &b.state->flags));
    if (staged) {
        build_boxes(smem, L);
        const int k = (blockIdx.x * blockDim.x + threadIdx.x) / G;
        const bool moving = b.state->moving != 0, multi = b.state->multi_head != 0;
        if (SIMPLE && !moving && !multi)
            rollout_sample<G, TIME, BF16, STATS, EXT, true>(pc, L, smem, b.scene, z, b.table, b.state->x0f, b.state->delta0f,
                                                           false, false, (int)(b.state->jkey & 0xffffffffu), k, b.S,
                                                           b.stats, nullptr);
        else
            rollout_sample<G, TIME, BF16, STATS, EXT>(pc, L, smem, b.scene, z, b.table, b.state->x0f, b.state->delta0f, moving,
                                                      multi, (int)(b.state->jkey & 0xffffffffu), k, b.S, b.stats,
                                                      pc.cost_to_go ? b.ctg_prefix : nullptr);
    }
    pdl_trigger();   // after the block's samples: the rollout may run in several waves
    rollout_argmin_tail(pc.K, b, (int)(blockIdx.x * blockDim.x / G), (int)(blockDim.x / G), staged);
}

// -----------------------------------------------------------------------------
// softmin weights in binary64 (Eq. (11)); eta partial sums per block.
// -----------------------------------------------------------------------------
__global__ void __launch_bounds__(256) weights_kernel(int K, float inv_lam, PlanBuffers b) {
    pdl_wait();
    pdl_trigger();
    const double smin = b.state->s_min;
    double acc = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
        const float w = softmin_weight(b.S[k], smin, inv_lam);
        b.w[k] = w;
        acc += (double)w;
    }
    acc = block_sum_d(acc);
    if (threadIdx.x == 0) b.eta_part[blockIdx.x] = acc;
}

// -----------------------------------------------------------------------------
// cost-to-go form of Eq. (11): one block per step t.  The cost of sample k from step t on is
// S_k - P_{t,k} (P: its cost of the steps before t, written by the rollout); the block takes
// their minimum, then the weights exp(-(S~ - min) / lambda) (softmin_weight) and their
// binary64 sum, the step's normaliser.
// -----------------------------------------------------------------------------
__global__ void __launch_bounds__(256) ctg_weights_kernel(int K, float inv_lam, PlanBuffers b) {
    pdl_wait();
    pdl_trigger();
    const int t = blockIdx.x;
    const float* P = b.ctg_prefix + (size_t)t * K;
    MinRec r{INFINITY, 0x7fffffff, 0};
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const double s = b.S[k] - (double)P[k];
        if (isfinite(s) && s < r.v) {
            r.v = s;
            r.i = k;
        }
    }
    r = block_min(r);
    __shared__ double s_min;
    if (threadIdx.x == 0) s_min = r.v;
    __syncthreads();
    const double smin = s_min;
    double acc = 0.0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const float w = softmin_weight(b.S[k] - (double)P[k], smin, inv_lam);
        b.wt[(size_t)t * K + k] = w;
        acc += (double)w;
    }
    acc = block_sum_d(acc);
    if (threadIdx.x == 0) b.eta_t[t] = acc;
}

// -----------------------------------------------------------------------------
// wsum: per step t, sum_k w_k eps'_{t,k}.  Each thread owns J samples of a k-tile,
// recomputes eps' from z exactly as the rollout did, accumulates in binary32 over
// its J samples and its warp (32 x J products), and the per-warp partials are
// added in binary64.
// -----------------------------------------------------------------------------
// The last k-tile block of a step tile (ticket) adds the k-tile partials of its steps in
// k-tile order into du, so the one-block update reads 2T sums instead of 2T x n_kt partials.
template <int TT>
__device__ __forceinline__ void wsum_ticket(const PlanConst& pc, const PlanBuffers& b) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&b.tt_count[blockIdx.y], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int T = pc.T, t0 = blockIdx.y * TT, n = 2 * (min(T, t0 + TT) - t0);
    const int n_kt = gridDim.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const size_t e = (size_t)2 * t0 + i;
        double num = 0.0;
        int kt = 0;
        for (; kt + 8 <= n_kt; kt += 8) {
            double v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = __ldcg(&b.du_part[(size_t)(kt + j) * 2 * T + e]);
#pragma unroll
            for (int j = 0; j < 8; ++j) num += v[j];
        }
        for (; kt < n_kt; ++kt) num += __ldcg(&b.du_part[(size_t)kt * 2 * T + e]);
        b.du[e] = num;
    }
    if (threadIdx.x == 0) b.tt_count[blockIdx.y] = 0u;
}

template <bool BF16, bool CTG, int TT>
__global__ void __launch_bounds__(256) wsum_kernel(PlanConst pc, SceneLayout L, PlanBuffers b,
                                                   const typename NoiseT<BF16>::type* __restrict__ z) {
    pdl_wait();
    pdl_trigger();
    const float4* ctl = reinterpret_cast<const float4*>(b.scene + L.off_ctl);
    wsum_tile<BF16, CTG, TT>(pc, ctl, z, b.w, blockIdx.x, blockIdx.y * TT, b.kt_size, b.du_part, b.wt);
    wsum_ticket<TT>(pc, b);
}

// The weighted sum with its noise tile staged in shared memory: thread 0 issues one bulk copy
// per step row of the tile (the row's kt_size samples are contiguous in the noise), each
// completing on its own mbarrier, while the threads load their weights; the arithmetic of
// wsum_tile then takes the rows in turn, each after a bounded wait for it (the same bits as
// wsum_kernel).  All of a tile's rows are requested at once instead of one step at a time.
// Used for bfloat16 noise when every row starts on a 16-byte boundary (K a multiple of 4) and
// for whole-cost weights.
template <bool BF16, int TT>
__global__ void __launch_bounds__(256) wsum_staged_kernel(PlanConst pc, SceneLayout L, PlanBuffers b,
                                                          const typename NoiseT<BF16>::type* __restrict__ z) {
    using NT = typename NoiseT<BF16>::type;
    extern __shared__ __align__(16) unsigned char ws_tile[];
    __shared__ unsigned long long bar[TT];
    const int K = pc.K, T = pc.T, kt = blockIdx.x, t0 = blockIdx.y * TT;
    const int rows = min(T, t0 + TT) - t0;
    if (threadIdx.x == 0)
        for (int r = 0; r < rows; ++r) bulk_init(&bar[r]);
    pdl_wait();
    pdl_trigger();
    __syncthreads();
    const int k0 = kt * b.kt_size, nk = min(b.kt_size, K - k0);
    if (threadIdx.x == 0) {
        const uint32_t dst_a = (uint32_t)__cvta_generic_to_shared(ws_tile);
        const uint32_t row_bytes = (uint32_t)nk * (uint32_t)sizeof(NT);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int r = 0; r < rows; ++r) {
            const uint32_t bar_a = (uint32_t)__cvta_generic_to_shared(&bar[r]);
            const NT* src = z + (size_t)(t0 + r) * K + k0;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a), "r"(row_bytes)
                         : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             dst_a + (uint32_t)(r * b.kt_size * (int)sizeof(NT))),
                         "l"(src), "r"(row_bytes), "r"(bar_a)
                         : "memory");
        }
    }
    const float4* ctl = reinterpret_cast<const float4*>(b.scene + L.off_ctl);
    wsum_tile<BF16, false, TT, true>(pc, ctl, reinterpret_cast<const NT*>(ws_tile), b.w, kt, t0, b.kt_size,
                                     b.du_part, nullptr, [&](int r) { bulk_wait(&bar[r], 0u, &b.state->flags); });
    wsum_ticket<TT>(pc, b);
}

// -----------------------------------------------------------------------------
// finalize (see finalize_block)
// -----------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) finalize_kernel(PlanConst pc, PlanBuffers b, PlanInputs in) {
    pdl_wait();
    finalize_block(pc, b, in);
}

// -----------------------------------------------------------------------------
// host-side launchers
// -----------------------------------------------------------------------------
// The staged form takes its tile as dynamic shared memory (up to 128 KB): opt in once per
// instantiation to the largest size it can be given.
template <bool BF16, int TT>
static cudaError_t launch_wsum_staged(const PlanConst& pc, const SceneLayout& L, const PlanBuffers& b,
                                      const typename NoiseT<BF16>::type* z, dim3 grid, size_t smem,
                                      cudaStream_t st) {
    static std::atomic<bool> done{false};
    if (!done.load(std::memory_order_acquire)) {
        const cudaError_t e = cudaFuncSetAttribute(wsum_staged_kernel<BF16, TT>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)((size_t)TT * 256 * WS_J * sizeof(typename NoiseT<BF16>::type)));
        if (e != cudaSuccess) return e;
        done.store(true, std::memory_order_release);
    }
    return launch_chained(wsum_staged_kernel<BF16, TT>, grid, dim3(256), smem, st, pc, L, b, z);
}

template <bool BF16, bool CTG>
static cudaError_t launch_wsum(const PlanConst& pc, const SceneLayout& L, const PlanBuffers& b,
                               const typename NoiseT<BF16>::type* z, dim3 grid, cudaStream_t st) {
    using NT = typename NoiseT<BF16>::type;
    // bfloat16 noise: the staged form (24-27 us against 31 us on the 65,536 x 200 workload: a
    // 4-byte load per sample keeps too few bytes in flight).  binary32 noise: the register form
    // (29 us against 35 us staged, whose 64 KB tiles leave three blocks per SM)
    if constexpr (BF16 && !CTG) {
        if (pc.K % 4 == 0 && reinterpret_cast<uintptr_t>(z) % 16 == 0) {
            const size_t smem = (size_t)b.tt_len * b.kt_size * sizeof(NT);
            switch (b.tt_len) {
                case 8: return launch_wsum_staged<BF16, 8>(pc, L, b, z, grid, smem, st);
                case 4: return launch_wsum_staged<BF16, 4>(pc, L, b, z, grid, smem, st);
                case 2: return launch_wsum_staged<BF16, 2>(pc, L, b, z, grid, smem, st);
                case 1: return launch_wsum_staged<BF16, 1>(pc, L, b, z, grid, smem, st);
                default: return cudaErrorInvalidValue;
            }
        }
    }
    switch (b.tt_len) {
        case 8: return launch_chained(wsum_kernel<BF16, CTG, 8>, grid, dim3(256), 0, st, pc, L, b, z);
        case 4: return launch_chained(wsum_kernel<BF16, CTG, 4>, grid, dim3(256), 0, st, pc, L, b, z);
        case 2: return launch_chained(wsum_kernel<BF16, CTG, 2>, grid, dim3(256), 0, st, pc, L, b, z);
        case 1: return launch_chained(wsum_kernel<BF16, CTG, 1>, grid, dim3(256), 0, st, pc, L, b, z);
        default: return cudaErrorInvalidValue;
    }
}
// Opt an instantiation of the rollout kernel in to the device's whole shared memory per block,
// once: every launch and occupancy query then passes its own size (which depends on the block
// for the steering-rate model), and none lowers the limit under another.
template <int G, bool TIME, bool BF16, bool STATS, bool EXT, bool SIMPLE = false>
static cudaError_t allow_rollout_smem() {
    static std::atomic<bool> done{false};   // contexts may be driven from several host threads
    if (done.load(std::memory_order_acquire)) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, rollout_kernel<G, TIME, BF16, STATS, EXT, SIMPLE>);
    // the dynamic part may take what the kernel's static shared memory leaves
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(rollout_kernel<G, TIME, BF16, STATS, EXT, SIMPLE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) done.store(true, std::memory_order_release);
    return e;
}

template <int G, bool TIME, bool BF16, bool STATS, bool EXT, bool SIMPLE = false>
static cudaError_t launch_rollout_t(const PlanConst& pc, const SceneLayout& L, const PlanBuffers& b, int threads,
                                    cudaStream_t st) {
    const size_t smem = rollout_smem_bytes(L, threads, pc.model == 1);
    cudaError_t e = allow_rollout_smem<G, TIME, BF16, STATS, EXT, SIMPLE>();
    if (e != cudaSuccess) return e;
    const long long total = (long long)pc.K * G;
    const int blocks = (int)((total + threads - 1) / threads);
    return launch_chained(rollout_kernel<G, TIME, BF16, STATS, EXT, SIMPLE>, dim3(blocks), dim3(threads), smem, st, pc,
                          L, b, reinterpret_cast<const typename NoiseT<BF16>::type*>(b.z));
}

// The launch shapes: lanes per sample as the group value (g > 0 split the work of each
// step, g < 0 split the steps).
#define MPPI_ROLLOUT_GROUPS(X) X(1, 1, false) X(2, 2, false) X(4, 4, false) X(8, 8, false) X(16, 16, false) \
    X(32, 32, false) X(-2, 2, true) X(-4, 4, true) X(-8, 8, true) X(-16, 16, true)

// The lane splits with a specialised instantiation (the ones the autotuner picks; the others run
// the general kernel).
#define MPPI_SIMPLE_GROUPS(X) X(1, 1, false) X(2, 2, false) X(4, 4, false) X(-2, 2, true) X(-4, 4, true) X(-8, 8, true)

// The plan's parameters allow the specialised rollout step (rollout_sample's SIMPLE): three ego
// circles of one radius, a constant safety band, no collision-only switch, no speed cap, the
// segment form of the closest waypoint, no centre table, the 4-state model with whole-cost weights.
static bool simple_plan(const PlanConst& pc) {
    return pc.n_ego == 3 && pc.ego_same_radius && pc.d_safe_c == 0.0f && !pc.collision_only && !pc.vcap &&
           pc.ref_mode == 0 && !pc.has_table && pc.model == 0 && !pc.cost_to_go;
}

template <bool BF16>
static bool launch_rollout_simple(const PlanConst& pc, const SceneLayout& L, const PlanBuffers& b, int group,
                                  int threads, cudaStream_t st, cudaError_t* e) {
    switch (group) {
#define CASE(gv, g, time) \
    case gv: *e = launch_rollout_t<g, time, BF16, false, false, true>(pc, L, b, threads, st); return true;
        MPPI_SIMPLE_GROUPS(CASE)
#undef CASE
        default: return false;
    }
}

template <bool BF16, bool EXT>
static cudaError_t launch_rollout_b(const PlanConst& pc, const SceneLayout& L, const PlanBuffers& b, int group,
                                    int threads, cudaStream_t st) {
    cudaError_t es = cudaSuccess;
    if (!EXT && simple_plan(pc) && launch_rollout_simple<BF16>(pc, L, b, group, threads, st, &es)) return es;
    switch (group) {
#define CASE(gv, g, time) \
    case gv: return launch_rollout_t<g, time, BF16, false, EXT>(pc, L, b, threads, st);
        MPPI_ROLLOUT_GROUPS(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

template <int G, bool TIME, bool BF16, bool EXT>
static int max_blocks_t(int threads, size_t smem) {
    int n = 0;
    if (allow_rollout_smem<G, TIME, BF16, false, EXT>() != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rollout_kernel<G, TIME, BF16, false, EXT>, threads, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

template <bool BF16, bool EXT>
static int max_blocks_b(int group, int threads, size_t smem) {
    switch (group) {
#define CASE(gv, g, time) \
    case gv: return max_blocks_t<g, time, BF16, EXT>(threads, smem);
        MPPI_ROLLOUT_GROUPS(CASE)
#undef CASE
        default: return 0;
    }
}

// ext: the steering-rate model or the cost-to-go form is on (the other instantiation)
static bool ext_of(const PlanConst& pc) { return pc.model == 1 || pc.cost_to_go != 0; }

int rollout_max_blocks_per_sm(int group, int threads, int noise_bf16, size_t smem, bool ext) {
    if (ext)
        return noise_bf16 ? max_blocks_b<true, true>(group, threads, smem) : max_blocks_b<false, true>(group, threads, smem);
    return noise_bf16 ? max_blocks_b<true, false>(group, threads, smem) : max_blocks_b<false, false>(group, threads, smem);
}

cudaError_t launch_rollout_stats(const PlanConst& pc, const SceneLayout& L, const PlanBuffers& b, int noise_bf16,
                                 cudaStream_t st) {
    if (ext_of(pc))
        return noise_bf16 ? launch_rollout_t<1, false, true, true, true>(pc, L, b, 128, st)
                          : launch_rollout_t<1, false, false, true, true>(pc, L, b, 128, st);
    return noise_bf16 ? launch_rollout_t<1, false, true, true, false>(pc, L, b, 128, st)
                      : launch_rollout_t<1, false, false, true, false>(pc, L, b, 128, st);
}

cudaError_t launch_rollout(const PlanConst& pc, const SceneLayout& L, const PlanBuffers& b, int group,
                           int threads, int noise_bf16, cudaStream_t st) {
    if (threads < 32 || threads > MAX_ROLLOUT_THREADS || threads % 32 != 0) return cudaErrorInvalidValue;
    if (ext_of(pc))
        return noise_bf16 ? launch_rollout_b<true, true>(pc, L, b, group, threads, st)
                          : launch_rollout_b<false, true>(pc, L, b, group, threads, st);
    return noise_bf16 ? launch_rollout_b<true, false>(pc, L, b, group, threads, st)
                      : launch_rollout_b<false, false>(pc, L, b, group, threads, st);
}

cudaError_t launch_prep_noise(const PlanConst& pc, const SceneLayout& L, const PlanBuffers& b,
                              const PlanInputs& in, int noise_bf16, cudaStream_t st) {
    cudaError_t e;
    if (b.fix_count && (e = cudaMemsetAsync(b.fix_count, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
    if ((e = launch_prep_noise_k(pc, L, b, in, noise_bf16, st)) != cudaSuccess) return e;
    return noise_bf16 ? launch_noise_fix(pc, b, st) : cudaSuccess;
}

// resets the per-iteration fields that prep accumulates into (after a prep without finalize)
__global__ void reset_state_kernel(DevState* st) {
    st->flags = 0;
    st->moving = 0;
    st->multi_head = 0;
    st->jkey = ~0ull;
}

cudaError_t launch_reset_state(DevState* st, cudaStream_t s) {
    reset_state_kernel<<<1, 1, 0, s>>>(st);
    return cudaGetLastError();
}

cudaError_t launch_iteration(const PlanConst& pc, const SceneLayout& L, const PlanBuffers& b,
                             const PlanInputs& in, int group, int threads, int noise_bf16, cudaStream_t st,
                             cudaEvent_t* ev, int ev_mode, const int* inject) {
    // ev_mode 1: an event before the first kernel and after each (every boundary timed, none
    // chained); 2: only the two around the rollout (ev[2], ev[3]), the other kernels stay chained
    cudaError_t e;
    int stage = 0;
    auto mark = [&]() -> cudaError_t {
        cudaError_t r = cudaGetLastError();
        if (r != cudaSuccess || !ev) return r;
        const int s = stage++;
        if (ev_mode == 2 && s != 2 && s != 3) return cudaSuccess;
        return cudaEventRecord(ev[s], st);
    };
    TraceScope iteration("mppi iteration");
    if (ev && ev_mode != 2 && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
    ++stage;
    // prep and noise in one launch (the "prep" stage), the bf16 fix-up chained after it (the "noise" stage)
    {
        TraceScope r("prep + noise");
        if ((e = launch_prep_noise_k(pc, L, b, in, noise_bf16, st)) != cudaSuccess) return e;
    }
    if ((e = mark()) != cudaSuccess) return e;
    if (noise_bf16) {
        TraceScope r("bf16 noise fix-up");
        if ((e = launch_noise_fix(pc, b, st)) != cudaSuccess) return e;
    }
    if ((e = mark()) != cudaSuccess) return e;
    {
        TraceScope r("rollout + cost + argmin");
        if ((e = launch_rollout(pc, L, b, group, threads, noise_bf16, st)) != cudaSuccess) return e;
    }
    if ((e = mark()) != cudaSuccess) return e;
    // argmin: folded into the rollout kernel (its last block); the stage keeps its event
    if ((e = mark()) != cudaSuccess) return e;
    if (inject && (e = cudaMemcpyAsync(&b.state->flags, inject, sizeof(int), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return e;
    {
        TraceScope r("softmin weights");
        if (pc.cost_to_go)
            e = launch_chained(ctg_weights_kernel, dim3(pc.T), dim3(256), 0, st, pc.K, pc.inv_lam_f, b);
        else
            e = launch_chained(weights_kernel, dim3(b.n_wblk), dim3(256), 0, st, pc.K, pc.inv_lam_f, b);
    }
    if (e != cudaSuccess) return e;
    if ((e = mark()) != cudaSuccess) return e;
    {
        TraceScope r("weighted noise sums");
        dim3 grid(b.n_kt, b.n_tt);
        const bool ctg = pc.cost_to_go != 0;
        if (noise_bf16) {
            const __nv_bfloat162* zb = reinterpret_cast<const __nv_bfloat162*>(b.z);
            e = ctg ? launch_wsum<true, true>(pc, L, b, zb, grid, st) : launch_wsum<true, false>(pc, L, b, zb, grid, st);
        } else {
            const float2* zf = reinterpret_cast<const float2*>(b.z);
            e = ctg ? launch_wsum<false, true>(pc, L, b, zf, grid, st) : launch_wsum<false, false>(pc, L, b, zf, grid, st);
        }
        if (e != cudaSuccess) return e;
        if ((e = mark()) != cudaSuccess) return e;
    }
    {
        TraceScope r("update + smoothing + x*");
        if ((e = launch_chained(finalize_kernel, dim3(1), dim3(((pc.T + 31) / 32) * 32), 0, st, pc, b, in)) !=
            cudaSuccess)
            return e;
    }
    return mark();
}

cudaError_t launch_slice_costs(const PlanConst& pc, const SceneLayout& L, const PlanBuffers& b,
                               const PlanInputs& in, int group, int threads, int noise_bf16, cudaStream_t st) {
    cudaError_t e;
    if ((e = launch_prep_noise_k(pc, L, b, in, noise_bf16, st)) != cudaSuccess) return e;
    if (noise_bf16 && (e = launch_noise_fix(pc, b, st)) != cudaSuccess) return e;
    return launch_rollout(pc, L, b, group, threads, noise_bf16, st);
}

cudaError_t launch_slice_sums(const PlanConst& pc, const SceneLayout& L, const PlanBuffers& b, int noise_bf16,
                              cudaStream_t st) {
    cudaError_t e = launch_chained(weights_kernel, dim3(b.n_wblk), dim3(256), 0, st, pc.K, pc.inv_lam_f, b);
    if (e != cudaSuccess) return e;
    const dim3 grid(b.n_kt, b.n_tt);
    if (noise_bf16) return launch_wsum<true, false>(pc, L, b, reinterpret_cast<const __nv_bfloat162*>(b.z), grid, st);
    return launch_wsum<false, false>(pc, L, b, reinterpret_cast<const float2*>(b.z), grid, st);
}

cudaError_t launch_slice_finalize(const PlanConst& pc, const PlanBuffers& b, const PlanInputs& in, cudaStream_t st) {
    return launch_chained(finalize_kernel, dim3(1), dim3(((pc.T + 31) / 32) * 32), 0, st, pc, b, in);
}

// Debug build: the index violations this translation unit's kernels counted (then reset), and a
// self-test kernel whose two indices are out of range (the check keeps its reads in bounds).
__global__ void check_selftest_kernel(const int* a, int* out) {
#ifdef MPPI_CHECKS
    out[0] = a[IX(-1, 4)] + a[IX(4, 4)];   // both indices are replaced by 0 and counted
#else
    out[0] = a[0];                          // the normal build has no checks: no stray index
#endif
}

cudaError_t take_check_hits_kernels(unsigned long long* hits) {
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

cudaError_t run_check_selftest(int* a4, int* out, cudaStream_t st) {
    check_selftest_kernel<<<1, 1, 0, st>>>(a4, out);
    return cudaGetLastError();
}

cudaError_t launch_philox(uint2 key, const uint4* ctr, uint4* out, int n, cudaStream_t st) {
    philox_kernel<<<(n + 255) / 256, 256, 0, st>>>(key, ctr, out, n);
    return cudaGetLastError();
}

}  // namespace mppi
