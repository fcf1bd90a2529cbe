// mppi_iter.cuh - device building blocks of one MPPI iteration (arXiv 2308.01654, Algorithm 1)
// shared by the single-plan kernels (mppi_kernels.cu) and the batched ones (mppi_batch.cu):
// scene preparation, noise, the fused rollout + cost of one sample, the reductions and the
// smoothing / optimal-rollout block.
#pragma once

#include <math.h>

#include "mppi_device.cuh"
#include "mppi_internal.h"

namespace mppi {

// -----------------------------------------------------------------------------
// prep: positions are shifted into a frame centred on (x0, y0) in binary64 before
// rounding, so binary32 keeps its resolution where the rollouts happen.
// -----------------------------------------------------------------------------
__device__ __forceinline__ float2 local_vertex(const double* ref, int i, double ox, double oy) {
    return make_float2((float)(ref[2 * i] - ox), (float)(ref[2 * i + 1] - oy));
}

// (min x, min y, max x, max y) of two boxes
__device__ __forceinline__ float4 box_union(float4 a, float4 b) {
    return make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fmaxf(a.z, b.z), fmaxf(a.w, b.w));
}

__device__ __forceinline__ float4 seg_record(const double* ref, int i, double ox, double oy) {
    const float2 a = local_vertex(ref, i, ox, oy), b = local_vertex(ref, i + 1, ox, oy);
    const float ex = b.x - a.x, ey = b.y - a.y;
    const float l2 = fmaf(ex, ex, ey * ey);
    const float inv = l2 > 0.0f ? 1.0f / l2 : 0.0f;
    return make_float4(ex, ey, ex * inv, ey * inv);
}

// Heading of segment i: the direction is formed in binary64 and its angle taken in binary32
// (each component rounded to 2^-24 relative, atan2f within a few ulp: a few 1e-7 rad, the
// same order as storing the angle as a binary32), which keeps scene preparation off the slow
// binary64 transcendental path.
__device__ __forceinline__ float seg_heading(const double* ref, int i) {
    const double hx = ref[2 * i + 2] - ref[2 * i], hy = ref[2 * i + 3] - ref[2 * i + 1];
    return atan2f((float)hy, (float)hx);
}

// Unit lane direction (first to last vertex), formed in binary64 and rounded: the axis the
// circles are sorted on.
__device__ __forceinline__ float2 lane_direction(const double* ref, int n_ref) {
    const double ex = ref[2 * (n_ref - 1)] - ref[0], ey = ref[2 * (n_ref - 1) + 1] - ref[1];
    const double el = sqrt(ex * ex + ey * ey);
    const bool ok = el > 0.0 && isfinite(el);
    return make_float2(ok ? (float)(ex / el) : 1.0f, ok ? (float)(ey / el) : 0.0f);
}

// Sort key of circle j: its first centre (the first row of the centre table when one is given,
// else the given centre) in the local frame, projected on the lane direction; non-finite keys
// sort last.
__device__ __forceinline__ float circle_key(const PlanInputs& in, int j, double ox, double oy, float2 pj) {
    const double* c = in.centres ? in.centres + 2 * j : in.circ + 5 * j;
    const float px = (float)(c[0] - ox), py = (float)(c[1] - oy);
    const float key = fmaf(px, pj.x, py * pj.y);
    return isfinite(key) ? key : INFINITY;
}

// Position of circle k in the sorted order (key, then index): one permutation of the circles.
__device__ __forceinline__ int circle_rank(const PlanInputs& in, int k, float kk, double ox, double oy, float2 pj,
                                           int j0, int dj) {
    int rank = 0;
    for (int j = j0; j < in.n_circ; j += dj) {
        const float sj = circle_key(in, j, ox, oy, pj);
        rank += (sj < kk || (sj == kk && j < k)) ? 1 : 0;
    }
    return rank;
}

// The preparation in independent phases: 0 controls and x0, 1 vertices, 2 segments and the
// segment nearest x0, 3 level-1 boxes, 4 circles and the lane direction, 5 the per-step
// centre table, 6 the largest step of each tabulated centre, 7 the prefix and suffix boxes of
// the vertices.  phase < 0 runs them all in turn (one block per plan in the batched planner);
// the single-plan kernel gives each phase its own row of blocks, so the phases run side by side
// instead of one after another.
constexpr int PREP_PHASES = 8;

__device__ __forceinline__ void prep_scene(const PlanConst& pc, const SceneLayout& L, const PlanInputs& in,
                                           const PlanBuffers& b, int tid, int nth, int phase = -1) {
    const double ox = in.x0[0], oy = in.x0[1];
    unsigned char* sc = b.scene;
    float4* ctl = reinterpret_cast<float4*>(sc + L.off_ctl);
    float* c0 = reinterpret_cast<float*>(sc + L.off_c0);
    float2* vert = reinterpret_cast<float2*>(sc + L.off_vert);
    float4* seg = reinterpret_cast<float4*>(sc + L.off_seg);
    float* head = reinterpret_cast<float*>(sc + L.off_head);
    float4* l1 = reinterpret_cast<float4*>(sc + L.off_l1);
    float4* circ = reinterpret_cast<float4*>(sc + L.off_circ);
    float2* vel = reinterpret_cast<float2*>(sc + L.off_vel);
    float* disp = reinterpret_cast<float*>(sc + L.off_disp);
    const bool all = phase < 0;
    const int lane = tid & 31, wid = tid >> 5, nwarps = nth >> 5;
    bool bad = false;

    if (all || phase == 0) {
        if (tid == 0) {
            for (int i = 0; i < (pc.model == 1 ? 5 : 4); ++i) bad |= !isfinite(in.x0[i]);
            b.state->x0f = make_float4(0.0f, 0.0f, (float)in.x0[2], (float)in.x0[3]);
            b.state->delta0f = pc.model == 1 ? (float)in.x0[4] : 0.0f;
        }
        for (int t = tid; t < L.T; t += nth) {
            const double ua = b.U[2 * t], ud = b.U[2 * t + 1];
            ctl[t] = make_float4((float)ua, (float)ud, (float)(pc.g_a * ua), (float)(pc.g_d * ud));
            c0[t] = (float)(pc.half_Ra * ua * ua + pc.half_Rd * ud * ud);
        }
    }
    if (all || phase == 1) {
        for (int i = tid; i < L.n_ref; i += nth) {
            bad |= !isfinite(in.ref[2 * i]) || !isfinite(in.ref[2 * i + 1]);
            vert[i] = local_vertex(in.ref, i, ox, oy);
        }
    }
    if (all || phase == 2) {
        // closest segment (or vertex) to x0 itself, the rollouts' first warm start: a packed
        // (distance bits, index) minimum, reduced in the warp before one atomic per warp
        unsigned long long best = ~0ull;
        const float h0 = seg_heading(in.ref, 0);
        bool multi = false;
        for (int i = tid; i < L.n_seg; i += nth) {
            const float4 s = seg_record(in.ref, i, ox, oy);
            seg[i] = s;
            head[i] = seg_heading(in.ref, i);
            multi |= head[i] != h0;
            const float2 a = local_vertex(in.ref, i, ox, oy);
            const float d2 = pc.ref_mode == 0 ? seg_dist2(0.0f, 0.0f, a, s) : fmaf(a.x, a.x, a.y * a.y);
            const unsigned long long key = ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)i;
            best = key < best ? key : best;
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
            best = other < best ? other : best;
        }
        if (lane == 0 && best != ~0ull) atomicMin(&b.state->jkey, best);
        // one heading throughout: no two segments can be in the binary64 near-tie of the search
        if (__any_sync(0xffffffffu, multi) && lane == 0) atomicOr(&b.state->multi_head, 1);
    }
    if (all || phase == 3) {
        // level-1 boxes: one thread per chunk (its REF_L1 + 1 vertex loads are independent)
        for (int c = tid; c < L.n_l1; c += nth) {
            const int v0 = c * REF_L1, v1 = min(v0 + REF_L1, L.n_seg);
            float4 bb = make_float4(INFINITY, INFINITY, -INFINITY, -INFINITY);
#pragma unroll
            for (int j = 0; j <= REF_L1; ++j) {
                if (v0 + j <= v1) {
                    const float2 p = local_vertex(in.ref, v0 + j, ox, oy);
                    bb.x = fminf(bb.x, p.x); bb.y = fminf(bb.y, p.y);
                    bb.z = fmaxf(bb.z, p.x); bb.w = fmaxf(bb.w, p.y);
                }
            }
            l1[c] = bb;
        }
    }
    if (all || phase == 4) {
        // the circles are stored sorted by their key along the lane direction (circle_rank), with
        // the original index of each sorted position (for the centre table) and the sorted keys
        const float2 pj = lane_direction(in.ref, L.n_ref);
        int* order = reinterpret_cast<int*>(sc + L.off_order);
        float* skey = reinterpret_cast<float*>(sc + L.off_skey);
        // one warp per circle: the lanes count the circles ordered before it in strides of 32
        for (int k = wid; k < L.n_circ; k += nwarps) {
            const double* c = in.circ + 5 * k;
            const float kk = circle_key(in, k, ox, oy, pj);
            const int pos = __reduce_add_sync(0xffffffffu, (unsigned)circle_rank(in, k, kk, ox, oy, pj, lane, 32));
            if (lane != 0) continue;
            for (int j = 0; j < 5; ++j) bad |= !isfinite(c[j]);
            const float r = (float)c[2];
            // band limit (m + r + r_ego)^2 for the constant-d_safe, equal-ego-radius case
            const float m = pc.collision_only ? fmaxf(pc.d_safe_0, 0.0f) : pc.d_safe_0;
            const float lim = m + r + pc.ego_rad[0];
            circ[pos] = make_float4((float)(c[0] - ox), (float)(c[1] - oy), r, lim > 0.0f ? lim * lim : -1.0f);
            vel[pos] = make_float2((float)c[3], (float)c[4]);
            order[pos] = k;
            skey[pos] = kk;
            if (c[3] != 0.0 || c[4] != 0.0) atomicOr(&b.state->moving, 1);
            // bound on the step of a constant-velocity centre, |v| dt with 0.1 % and 1e-5 m to spare
            // (binary32 square root: its error is far inside that margin)
            if (!in.centres) disp[pos] = sqrtf((float)(c[3] * c[3] + c[4] * c[4])) * pc.dt * 1.001f + 1e-5f;
        }
        if (tid == 0) *reinterpret_cast<float4*>(sc + L.off_proj) = make_float4(pj.x, pj.y, 0.0f, 0.0f);
    }
    if (in.centres && (all || phase == 5)) {
        for (int i = tid; i < L.T * L.n_circ; i += nth) {
            const double cx = in.centres[2 * i], cy = in.centres[2 * i + 1];
            bad |= !isfinite(cx) || !isfinite(cy);
            b.table[i] = make_float2((float)(cx - ox), (float)(cy - oy));
        }
    }
    if (in.centres && (all || phase == 6)) {
        // the largest step of each tabulated centre (from the rounded entries the rollouts
        // read): one warp per circle, the lanes stride over the steps
        for (int k = wid; k < L.n_circ; k += nwarps) {
            double m = 0.0;
            for (int t = 1 + lane; t < L.T; t += 32) {
                const double* a = in.centres + 2 * ((size_t)(t - 1) * L.n_circ + k);
                const double* q = in.centres + 2 * ((size_t)t * L.n_circ + k);
                const double dx = (double)(float)(q[0] - ox) - (double)(float)(a[0] - ox);
                const double dy = (double)(float)(q[1] - oy) - (double)(float)(a[1] - oy);
                m = fmax(m, fabs(dx) + fabs(dy));    // >= the Euclidean step
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
            // the circle's sorted position (its place in phase 4's order), counted by the warp
            const float2 pj = lane_direction(in.ref, L.n_ref);
            const int pos = __reduce_add_sync(
                0xffffffffu, (unsigned)circle_rank(in, k, circle_key(in, k, ox, oy, pj), ox, oy, pj, lane, 32));
            if (lane == 0) disp[pos] = isfinite(m) ? (float)(m * 1.001) + 1e-5f : INFINITY;
        }
    }
    if ((all || phase == 7) && tid < (int)blockDim.x) {
        // prefix and suffix boxes of the vertices, by the first block of the phase (every thread of
        // it takes part): each thread a run of consecutive vertices, the runs combined in order by a
        // warp scan and a scan of the warp totals; the suffix pass takes the runs in reverse
        float4* pre = reinterpret_cast<float4*>(sc + L.off_pbox);
        float4* suf = reinterpret_cast<float4*>(sc + L.off_sbox);
        __shared__ float4 s_wbox[32];
        const float4 empty = make_float4(INFINITY, INFINITY, -INFINITY, -INFINITY);
        const int nb = blockDim.x, th = threadIdx.x, nw = (nb + 31) >> 5;
        const int run = (L.n_ref + nb - 1) / nb;
        for (int dir = 0; dir < 2; ++dir) {
            const int r = dir ? nb - 1 - th : th;
            const int i0 = min(r * run, L.n_ref), i1 = min(i0 + run, L.n_ref);
            float4 agg = empty;
            for (int i = i0; i < i1; i += 4) {          // four independent loads in flight
                float2 v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = local_vertex(in.ref, min(i + q, i1 - 1), ox, oy);
#pragma unroll
                for (int q = 0; q < 4; ++q) agg = box_union(agg, make_float4(v[q].x, v[q].y, v[q].x, v[q].y));
            }
            float4 inc = agg;          // inclusive scan in thread order within the warp
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                float4 u;
                u.x = __shfl_up_sync(0xffffffffu, inc.x, o);
                u.y = __shfl_up_sync(0xffffffffu, inc.y, o);
                u.z = __shfl_up_sync(0xffffffffu, inc.z, o);
                u.w = __shfl_up_sync(0xffffffffu, inc.w, o);
                if (lane >= o) inc = box_union(inc, u);
            }
            if (lane == 31) s_wbox[wid] = inc;
            __syncthreads();
            if (wid == 0) {
                float4 t = lane < nw ? s_wbox[lane] : empty;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    float4 u;
                    u.x = __shfl_up_sync(0xffffffffu, t.x, o);
                    u.y = __shfl_up_sync(0xffffffffu, t.y, o);
                    u.z = __shfl_up_sync(0xffffffffu, t.z, o);
                    u.w = __shfl_up_sync(0xffffffffu, t.w, o);
                    if (lane >= o) t = box_union(t, u);
                }
                if (lane < nw) s_wbox[lane] = t;
            }
            __syncthreads();
            // this thread's exclusive prefix: the earlier warps and the earlier lanes of its warp
            float4 carry = wid > 0 ? s_wbox[wid - 1] : empty;
            float4 prev;
            prev.x = __shfl_up_sync(0xffffffffu, inc.x, 1);
            prev.y = __shfl_up_sync(0xffffffffu, inc.y, 1);
            prev.z = __shfl_up_sync(0xffffffffu, inc.z, 1);
            prev.w = __shfl_up_sync(0xffffffffu, inc.w, 1);
            if (lane > 0) carry = box_union(carry, prev);
            for (int i = i0; i < i1; i += 4) {
                // the run in groups of four (forward for the prefix, backward for the suffix)
                float2 v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int iq = dir == 0 ? min(i + q, i1 - 1) : max(i1 - 1 - (i - i0) - q, i0);
                    v[q] = local_vertex(in.ref, iq, ox, oy);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (i + q >= i1) break;
                    carry = box_union(carry, make_float4(v[q].x, v[q].y, v[q].x, v[q].y));
                    if (dir == 0) pre[i + q] = carry;
                    else suf[i1 - 1 - (i - i0) - q] = carry;
                }
            }
            __syncthreads();           // s_wbox is reused by the second pass
        }
    }
    if (bad) atomicOr(&b.state->flags, FLAG_NONFINITE_INPUT);
}

// -----------------------------------------------------------------------------
// noise: one thread per (step pair j, sample k); coalesced stores along k.
// The bfloat16 store is a rounding decision: it is taken on the exact normal
// (binary64 Box-Muller) whenever the binary32 normal lies within its error bound
// of a rounding midpoint, so the stored code is the one of the exact value.
// -----------------------------------------------------------------------------
template <bool BF16>
__device__ __forceinline__ typename NoiseT<BF16>::type make_noise(float u0, float u1) {
    const float2 zf = box_muller(u0, u1);
    if constexpr (BF16) {
        if (near_bf16_midpoint(zf.x) || near_bf16_midpoint(zf.y)) {
            const double2 zd = box_muller_f64(u0, u1);
            __nv_bfloat162 r;
            r.x = bf16_from_f64(zd.x);
            r.y = bf16_from_f64(zd.y);
            return r;
        }
    }
    return NoiseT<BF16>::pack(zf);
}

// -----------------------------------------------------------------------------
// 1-D bulk (TMA) copy global -> shared, completion on an mbarrier, bounded wait.
// -----------------------------------------------------------------------------
// Pieces of the staging, for kernels that stage several times with one barrier:
// bulk_init (thread 0, once; the caller synchronises), bulk_issue (thread 0: one
// expect_tx arrival and the copies in 32 KB pieces), bulk_wait (all threads; waits for
// the given phase parity with an iteration limit and raises FLAG_TIMEOUT instead of
// hanging).
__device__ __forceinline__ void bulk_init(unsigned long long* bar) {
    const uint32_t bar_a = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void bulk_issue(unsigned char* dst, const unsigned char* src, int bytes,
                                           unsigned long long* bar) {
    const uint32_t bar_a = (uint32_t)__cvta_generic_to_shared(bar);
    const uint32_t dst_a = (uint32_t)__cvta_generic_to_shared(dst);
    // order earlier generic-proxy accesses of the buffer before the asynchronous writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a), "r"(bytes) : "memory");
    constexpr int CHUNK = 32768;
    for (int off = 0; off < bytes; off += CHUNK) {
        const int n = min(CHUNK, bytes - off);
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         dst_a + off),
                     "l"(src + off), "r"(n), "r"(bar_a)
                     : "memory");
    }
}

__device__ __forceinline__ bool bulk_wait(unsigned long long* bar, uint32_t parity, int* flags) {
    const uint32_t bar_a = (uint32_t)__cvta_generic_to_shared(bar);
    uint32_t done = 0;
    for (int it = 0; it < (1 << 22) && !done; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar_a), "r"(parity)
            : "memory");
    }
    if (!done && threadIdx.x == 0) atomicOr(flags, FLAG_TIMEOUT);
    // the block reports the timeout but stays resident for a second bounded wait, so a copy that
    // is only late can still land before the block exits (a block must not exit while a bulk
    // copy into its shared memory is in flight); a copy that never completes cannot be told
    // apart from this on the device, so the block returns after the second limit either way
    for (int it = 0; it < (1 << 22) && !done; ++it) {
        uint32_t late = 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(late)
            : "r"(bar_a), "r"(parity)
            : "memory");
        if (late) break;
    }
    return done != 0;
}

// One-shot staging of a whole buffer (phase 0 of a fresh barrier).
__device__ __forceinline__ bool stage_to_smem(unsigned char* dst, const unsigned char* src, int bytes,
                                              unsigned long long* bar, int* flags) {
    if (threadIdx.x == 0) bulk_init(bar);
    __syncthreads();
    if (threadIdx.x == 0) bulk_issue(dst, src, bytes, bar);
    return bulk_wait(bar, 0u, flags);
}

// -----------------------------------------------------------------------------
// rollout + cost.  G lanes (a power of two <= 32) work on one sample: they run the
// dynamics redundantly (identical bits) and split the reference search and the
// obstacle pairs, combining with shuffles inside the group.
// -----------------------------------------------------------------------------
template <int G>
__device__ __forceinline__ unsigned group_mask() {
    if constexpr (G == 32) {
        return 0xffffffffu;
    } else {
        const unsigned lane = threadIdx.x & 31u;
        return ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
    }
}


template <int G>
__device__ __forceinline__ float group_min(float v, unsigned mask) {
#pragma unroll
    for (int o = G / 2; o >= 1; o >>= 1) v = fminf(v, __shfl_xor_sync(mask, v, o, G));
    return v;
}

// Work done by the pruned searches of one lane (only counted in the STATS instantiation):
// range boxes (prefix, suffix, level-2), chunk boxes, segments, binary64 refinements,
// broad-phase circle tests, candidate circles, square roots taken for d_obj.
struct Counters {
    unsigned l2, l1, seg, refine, circ, cand, pair;
};

// (squared distance, index) as one ordered 64-bit key: the minimum key is the smallest
// distance and, among equal distances, the lowest index.
__device__ __forceinline__ unsigned long long dkey(float d2, int i) {
    return ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)i;
}

template <int G>
__device__ __forceinline__ unsigned long long group_min_key(unsigned long long k, unsigned mask) {
#pragma unroll
    for (int o = G / 2; o >= 1; o >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(mask, k, o, G);
        k = ok < k ? ok : k;
    }
    return k;
}

// REF_L1 consecutive segments from i0 (a level-1 chunk, or the search window); the lanes of a
// group split them.
template <int G, bool STATS>
__device__ __forceinline__ void scan_chunk(float px, float py, const float2* vert, const float4* seg, int i0,
                                           int n_seg, int lane_g, unsigned long long& best, Counters& cnt) {
    constexpr int PER = (REF_L1 + G - 1) / G;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int o = lane_g + q * G;
        const int i = i0 + o;
        if (o < REF_L1 && i < n_seg) {
            if (STATS) cnt.seg++;
            const unsigned long long k = dkey(seg_dist2(px, py, vert[IX(i, n_seg)], seg[IX(i, n_seg)]), i);
            best = k < best ? k : best;
        }
    }
}

// The boxes of the segment search: the staged chunk boxes (l1), the level-2 boxes each rollout
// block builds in shared memory right after the staged blob (each the union of REF_L2 chunk
// boxes), and the prefix and suffix boxes of the vertices that scene preparation leaves in
// global memory after the staged part, pre[i] = box of the vertices 0 .. i (the segments
// 0 .. i-1) and suf[i] = box of the vertices i .. n_ref-1 (the segments i .. n_seg-1).
struct RefBoxes {
    const float4* l1;
    const float4* l2;
    const float4* pre;
    const float4* suf;
};

__device__ __forceinline__ RefBoxes ref_boxes(const unsigned char* smem, const unsigned char* gscene,
                                              const SceneLayout& L) {
    RefBoxes r;
    r.l1 = reinterpret_cast<const float4*>(smem + L.off_l1);
    r.l2 = reinterpret_cast<const float4*>(smem + L.bytes);
    r.pre = reinterpret_cast<const float4*>(gscene + L.off_pbox);
    r.suf = reinterpret_cast<const float4*>(gscene + L.off_sbox);
    return r;
}

// The circle index: the circles are stored sorted by their key along the lane direction; the
// block adds CIRC_BUCKETS buckets of equal key width over the finite keys and the scalars the
// broad phase needs to bound where a circle can be at step t.
struct CircleIndex {
    const int* order;       // [n_circ] input index of each sorted circle (its centre-table column)
    const int* start;       // [CIRC_BUCKETS + 1] first sorted position of each bucket
    float smin, inv_w;      // bucket b holds the keys from smin + b / inv_w (inv_w = 0: one range)
    float dmax, rmax;       // largest step bound and radius over the circles
    float dx, dy;           // lane direction
};

__device__ __forceinline__ const unsigned char* circle_index_base(const unsigned char* smem, const SceneLayout& L) {
    return smem + L.bytes + 16 * L.n_l2;
}

__device__ __forceinline__ CircleIndex circle_index(const unsigned char* smem, const SceneLayout& L) {
    const unsigned char* e = circle_index_base(smem, L);
    const float4 sc = *reinterpret_cast<const float4*>(e);
    const float4 pj = *reinterpret_cast<const float4*>(smem + L.off_proj);
    CircleIndex c;
    c.order = reinterpret_cast<const int*>(smem + L.off_order);
    c.start = reinterpret_cast<const int*>(e + 32);
    c.smin = sc.x;
    c.inv_w = sc.y;
    c.dmax = sc.z;
    c.rmax = sc.w;
    c.dx = pj.x;
    c.dy = pj.y;
    return c;
}

// The search scalar the block derives from the staged segments: 4 x the longest segment, the
// length term of the pruning bound (prune_lim).
__device__ __forceinline__ float search_lfac(const unsigned char* smem, const SceneLayout& L) {
    return *reinterpret_cast<const float*>(circle_index_base(smem, L) + 16);
}

// First position in skey[0, n) whose key is >= v (n if none).
__device__ __forceinline__ int lower_bound_f(const float* skey, int n, float v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (skey[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}


__device__ __forceinline__ void build_boxes(unsigned char* smem, const SceneLayout& L) {
    const float4* l1 = reinterpret_cast<const float4*>(smem + L.off_l1);
    float4* l2 = reinterpret_cast<float4*>(smem + L.bytes);
    for (int g = threadIdx.x; g < L.n_l2; g += blockDim.x) {
        float4 a = l1[g * REF_L2];
        const int c1 = min((g + 1) * REF_L2, L.n_l1);
        for (int c = g * REF_L2 + 1; c < c1; ++c) a = box_union(a, l1[c]);
        l2[g] = a;
    }
    // circle index.  Scene preparation stored the circles sorted by their key (the first centre
    // projected on the lane direction, non-finite keys last) with the sorted keys; the block adds
    // the bucket starts over the keys and the largest step bound and radius.
    __shared__ unsigned s_dmax, s_rmax, s_lmax;
    __shared__ int s_nfin;
    if (threadIdx.x == 0) {
        s_dmax = 0u;
        s_rmax = 0u;
        s_lmax = 0u;
    }
    __syncthreads();
    const float4* circ = reinterpret_cast<const float4*>(smem + L.off_circ);
    const float* disp = reinterpret_cast<const float*>(smem + L.off_disp);
    const float* skey = reinterpret_cast<const float*>(smem + L.off_skey);
    for (int k = threadIdx.x; k < L.n_circ; k += blockDim.x) {
        atomicMax(&s_dmax, __float_as_uint(fmaxf(disp[k], 0.0f)));     // non-negative: bits order as values
        atomicMax(&s_rmax, __float_as_uint(fmaxf(circ[k].z, 0.0f)));
    }
    {
        // the longest segment (a NaN length, from non-finite input, gives an infinite bound)
        const float4* seg = reinterpret_cast<const float4*>(smem + L.off_seg);
        float lm = 0.0f;
        for (int i = threadIdx.x; i < L.n_seg; i += blockDim.x) {
            const float l = sqrtf(fmaf(seg[i].x, seg[i].x, seg[i].y * seg[i].y));
            lm = l >= lm ? l : (l < lm ? lm : INFINITY);
        }
        atomicMax(&s_lmax, __float_as_uint(lm));
    }
    if (threadIdx.x == 0) s_nfin = lower_bound_f(skey, L.n_circ, INFINITY);
    __syncthreads();
    unsigned char* e = const_cast<unsigned char*>(circle_index_base(smem, L));
    int* start = reinterpret_cast<int*>(e + 32);
    if (threadIdx.x == 0)
        *reinterpret_cast<float4*>(e + 16) = make_float4(4.0f * __uint_as_float(s_lmax), 0.0f, 0.0f, 0.0f);
    const int nfin = s_nfin;
    const float smin = nfin > 0 ? skey[0] : 0.0f;
    const float bw = nfin > 0 ? (skey[nfin - 1] - smin) / (float)CIRC_BUCKETS : 0.0f;
    const float inv_w = (bw > 0.0f && isfinite(bw)) ? 1.0f / bw : 0.0f;
    for (int b = threadIdx.x; b <= CIRC_BUCKETS; b += blockDim.x)
        start[b] = b == 0 ? 0 : (b == CIRC_BUCKETS ? L.n_circ : lower_bound_f(skey, nfin, fmaf((float)b, bw, smin)));
    if (threadIdx.x == 0)
        *reinterpret_cast<float4*>(e) = make_float4(smin, inv_w, __uint_as_float(s_dmax), __uint_as_float(s_rmax));
    __syncthreads();
}

// Distance from a squared distance as d2 * rsqrt(d2) (a few ulp, against the many more
// instructions of the correctly rounded square root); the argument of the reciprocal square
// root is raised to the smallest normal, so 0 gives 0 without a compare and a select (and a
// subnormal d2 gives at most 1.1e-19 m).  The obstacle term uses it only inside the safety
// band, where c_safe is continuous in it.
__device__ __forceinline__ float dist_of(float d2) { return d2 * rsqrtf(fmaxf(d2, 1.17549435e-38f)); }

// The pruning bound of the segment search: a box whose computed squared distance from p exceeds
// prune_lim(best) holds no segment whose computed squared distance (seg_dist2) is at or below
// best.  The rounding in seg_dist2 is relative to the differences it forms (p - a, the projection
// on e, the residual), so it is a few 2^-24 of (distance + segment length); a segment's far end
// a + e lies within 2^-24 |e| of its vertex (e is the rounded difference of the two binary32
// vertices), hence of its box; box_dist2 is within a few 2^-24 relative.  The bound allows 2^-20
// of (2 distance + 4 longest segment) on the distance (lfac = 4 x the longest segment), plus
// 2^-20 relative: several times the sum of those terms, and independent of how far p is from
// the origin of the frame.
__device__ __forceinline__ float prune_lim(float best2, float lfac) {
    const float d = dist_of(best2);
    const float e = 0x1p-20f * fmaf(2.0f, d, lfac);
    const float r = fmaf(d, 0x1p-20f, d + e);
    return r * r;
}

__device__ __forceinline__ float key_dist2(unsigned long long key) { return __uint_as_float((unsigned)(key >> 32)); }

// The chunks lo .. hi-1 under the level-2 boxes (the search's rare fallback: out of line, so the
// common path keeps its registers).
template <int G, bool STATS>
__device__ __noinline__ void search_range(float px, float py, const float2* vert, const float4* seg,
                                             const RefBoxes& rb, int n_seg, int lo, int hi, int lane_g,
                                             unsigned mask, float lfac, unsigned long long& best, Counters& cnt) {
#pragma unroll 1
    for (int g = lo / REF_L2; g <= (hi - 1) / REF_L2; ++g) {
        if (STATS) cnt.l2++;
        if (box_dist2(px, py, rb.l2[IX(g, (hi - 1) / REF_L2 + 1)]) > prune_lim(key_dist2(best), lfac))
            continue;
        const int c1 = min(hi, (g + 1) * REF_L2);
#pragma unroll 1
        for (int c = max(lo, g * REF_L2); c < c1; ++c) {
            if (STATS) cnt.l1++;
            if (box_dist2(px, py, rb.l1[IX(c, hi)]) <= prune_lim(key_dist2(best), lfac)) {
                scan_chunk<G, STATS>(px, py, vert, seg, c * REF_L1, n_seg, lane_g, best, cnt);
                best = group_min_key<G>(best, mask);
            }
        }
    }
}

// One side of the search beyond the window: from chunk c outward (dir -1: towards the start,
// +1: towards the end), a chunk whose box passes is scanned, and the walk stops as soon as the
// vertex box of everything beyond the chunk fails; after SIDE_WALK chunks the rest of the side is
// searched under the level-2 boxes.  On a curved lane the box of everything before (or after) a
// point spans the curve's width, so it passes for most rollouts off the lane: the walk then
// ends after the few chunks within the rollout's distance instead of testing every level-2 box.
constexpr int SIDE_WALK = 8;

template <int G, bool STATS>
__device__ __forceinline__ void side_walk(float px, float py, const float2* vert, const float4* seg,
                                          const RefBoxes& rb, int n_seg, int n_l1, int lane_g, unsigned mask,
                                          float lfac, int c, int dir, unsigned long long& best, Counters& cnt) {
    for (int s = 0;; ++s) {
        float lim = prune_lim(key_dist2(best), lfac);
        if (STATS) cnt.l1++;
        if (box_dist2(px, py, rb.l1[IX(c, n_l1)]) <= lim) {
            scan_chunk<G, STATS>(px, py, vert, seg, c * REF_L1, n_seg, lane_g, best, cnt);
            best = group_min_key<G>(best, mask);
            lim = prune_lim(key_dist2(best), lfac);
        }
        // the chunks beyond c: 0 .. c-1 (the vertices 0 .. REF_L1 c) or c+1 .. n_l1-1 (the
        // vertices REF_L1 (c+1) .. n_seg)
        if (dir < 0 ? c == 0 : c == n_l1 - 1) return;
        if (STATS) cnt.l2++;
        const float4 bb = dir < 0 ? __ldg(rb.pre + IX(REF_L1 * c, n_seg + 1))
                                  : __ldg(rb.suf + IX(REF_L1 * (c + 1), n_seg + 1));
        if (box_dist2(px, py, bb) > lim) return;
        c += dir;
        if (s + 1 == SIDE_WALK) {
            if (dir < 0) search_range<G, STATS>(px, py, vert, seg, rb, n_seg, 0, c + 1, lane_g, mask, lfac, best, cnt);
            else search_range<G, STATS>(px, py, vert, seg, rb, n_seg, c, n_l1, lane_g, mask, lfac, best, cnt);
            return;
        }
    }
}

// Closest point of the polyline (ties -> lowest segment).  The window of REF_L1 segments around
// the hint jh (from jh - 1, moved inside the polyline) is scanned first; the prefix box of the
// vertices before it and the suffix box of those after it bound the rest, and a side whose box
// passes is searched outward from the window (side_walk; on a straight lane rare: the window
// keeps a segment on either side of the hint).  A box is skipped only when its lower bound exceeds the best
// distance by more than binary32 rounding can account for (prune_lim), so no segment that can
// be the closest is missed and the result does not depend on jh.  Two segments that share a
// vertex can be closer than binary32 resolves (next to the vertex on the outside of a bend
// their distances differ by a second-order term): the winner's neighbours of another heading
// are re-ordered against it in binary64 when their binary32 distances are within 4e-6.
template <int G, bool STATS>
__device__ __forceinline__ void nearest_segment(float px, float py, const float2* vert, const float4* seg,
                                                const float* head, const RefBoxes& rb, int n_seg, int n_l1,
                                                int lane_g, unsigned mask, int jh, bool refine, float lfac,
                                                int& jb, float& best2, Counters& cnt) {
    const int w0 = max(min(jh - 1, n_seg - REF_L1), 0), w1 = w0 + REF_L1;
    unsigned long long best = ~0ull;
    scan_chunk<G, STATS>(px, py, vert, seg, w0, n_seg, lane_g, best, cnt);
    best = group_min_key<G>(best, mask);
    // segments 0 .. w0-1 lie in the box of the vertices 0 .. w0, segments w1 .. n_seg-1 in that of
    // the vertices w1 .. n_seg: when neither box can hold a closer segment, the common case, the
    // search ends here
    const float lim0 = prune_lim(key_dist2(best), lfac);
    const bool left = w0 >= 1 && box_dist2(px, py, __ldg(rb.pre + IX(w0, n_seg + 1))) <= lim0;
    const bool right = w1 < n_seg && box_dist2(px, py, __ldg(rb.suf + IX(w1, n_seg + 1))) <= lim0;
    if (STATS) cnt.l2 += (w0 >= 1 ? 1 : 0) + (w1 < n_seg ? 1 : 0);
    if (left) side_walk<G, STATS>(px, py, vert, seg, rb, n_seg, n_l1, lane_g, mask, lfac, (w0 - 1) / REF_L1, -1, best,
                                  cnt);
    if (right) side_walk<G, STATS>(px, py, vert, seg, rb, n_seg, n_l1, lane_g, mask, lfac, w1 / REF_L1, 1, best, cnt);
    float b2 = __uint_as_float((unsigned)(best >> 32));
    int bi = (int)(best & 0xffffffffu);
    const int b0 = bi;
    const float hb = refine ? head[IX(b0, n_seg)] : 0.0f;
#pragma unroll
    for (int dlt = -1; refine && dlt <= 1; dlt += 2) {
        const int j = b0 + dlt;
        if (j < 0 || j >= n_seg || head[IX(j, n_seg)] == hb) continue;
        const float dj = seg_dist2(px, py, vert[IX(j, n_seg)], seg[IX(j, n_seg)]);
        if (fabsf(dj - b2) <= 4e-6f * b2 + 1e-20f) {
            if (STATS) cnt.refine++;
            const double db = seg_dist2_f64(px, py, vert[IX(bi, n_seg)], vert[IX(bi + 1, n_seg + 1)]);
            const double dd = seg_dist2_f64(px, py, vert[IX(j, n_seg)], vert[IX(j + 1, n_seg + 1)]);
            if (dd < db || (dd == db && j < bi)) {
                bi = j;
                b2 = dj;
            }
        }
    }
    jb = bi;
    best2 = b2;
}

template <int G>
__device__ __forceinline__ void group_argmin(float& d2, int& idx, unsigned mask) {
#pragma unroll
    for (int o = G / 2; o >= 1; o >>= 1) {
        const float od = __shfl_xor_sync(mask, d2, o, G);
        const int oi = __shfl_xor_sync(mask, idx, o, G);
        if (od < d2 || (od == d2 && oi < idx)) {
            d2 = od;
            idx = oi;
        }
    }
}

// Closest vertex (ties -> lowest index), same hierarchy (chunk c covers vertices c*L1 .. c*L1+L1).
template <int G>
__device__ __forceinline__ void nearest_vertex(float px, float py, const float2* vert, const float4* l1,
                                               const float4* l2, int n_ref, int n_l1, int n_l2, int lane_g,
                                               unsigned mask, int& jb, float& best2) {
    float dx = px - vert[IX(jb, n_ref)].x, dy = py - vert[IX(jb, n_ref)].y;
    float b2 = fmaf(dx, dx, dy * dy);
    int bi = jb;
    for (int g = 0; g < n_l2; ++g) {
        if (box_dist2(px, py, l2[IX(g, n_l2)]) > prune_lim(b2, 0.0f)) continue;
        const int c1 = min((g + 1) * REF_L2, n_l1);
        for (int c = g * REF_L2; c < c1; ++c) {
            if (box_dist2(px, py, l1[IX(c, n_l1)]) > prune_lim(b2, 0.0f)) continue;
            const int i1 = min((c + 1) * REF_L1 + 1, n_ref);
            for (int i = c * REF_L1 + lane_g; i < i1; i += G) {
                const float ex = px - vert[IX(i, n_ref)].x, ey = py - vert[IX(i, n_ref)].y;
                const float d2 = fmaf(ex, ex, ey * ey);
                if (d2 < b2 || (d2 == b2 && i < bi)) {
                    b2 = d2;
                    bi = i;
                }
            }
            group_argmin<G>(b2, bi, mask);
        }
    }
    jb = bi;
    best2 = b2;
}

// Kahan-compensated accumulator: the value is hi - lo.
__device__ __forceinline__ void kahan_add(float& hi, float& lo, float inc) {
    const float y = inc - lo;
    const float t = hi + y;
    lo = (t - hi) - y;
    hi = t;
}

// Centre at rollout step t (state x_{t+1}) of the circle c at sorted position pos: from the
// centre table (column order[pos]), or moved at constant velocity from the given centre.
__device__ __forceinline__ float2 circle_centre(const float4& c, const float2* vel, const int* order,
                                                const float2* table, int n_circ, int t, int pos, float st,
                                                bool has_table, bool moving) {
    if (has_table) return table[(size_t)t * n_circ + order[IX(pos, n_circ)]];
    if (!moving) return make_float2(c.x, c.y);
    const float2 vv = vel[IX(pos, n_circ)];
    return make_float2(fmaf(vv.x, st, c.x), fmaf(vv.y, st, c.y));
}


// Warp min / max of a float: one redux.sync on binary32 (a NaN lane is ignored, like fminf and
// fmaxf; the results only bound the warp's broad phase).
__device__ __forceinline__ float warp_min_f(float v) {
    float r;
    asm("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ float warp_max_f(float v) {
    float r;
    asm("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}

// d_obj of Eq. (16) restricted to the pairs that can lie inside the safety band (the
// only pairs that change c_safe), with a warp-wide broad phase: the lanes test the
// circles against the bounding box of every ego circle of the warp, and only the
// circles that pass (ballot) get the exact per-pair test.  A circle is skipped only
// when no ego circle of the warp can come within the band of it, so the result equals
// the brute-force minimum over all in-band pairs.  The lanes of a warp may be at
// different steps t (all within tb0..tb1, the same for the whole warp): the broad phase
// then tests each circle's centre at tb0 with the band widened by the farthest it can
// move in tb1 - tb0 steps.
template <int G, bool STATS, bool SIMPLE = false>
__device__ __forceinline__ float obstacle_min(const PlanConst& pc, const unsigned char* smem, const SceneLayout& L,
                                              const float4* circ, const float2* vel,
                                              const float* disp, const float2* table, int n_circ, int t, int tb0,
                                              int tb1,
                                              bool has_table, bool moving, bool dconst, float nx, float ny,
                                              float cnth, float snth, float mband, int lane, int lane_g,
                                              unsigned mask, Counters& cnt) {
    // box of the ego circle centres of the whole warp
    const float xa = fmaf(pc.ego_omin, cnth, nx), xb = fmaf(pc.ego_omax, cnth, nx);
    const float ya = fmaf(pc.ego_omin, snth, ny), yb = fmaf(pc.ego_omax, snth, ny);
    const float bx0 = warp_min_f(fminf(xa, xb)), bx1 = warp_max_f(fmaxf(xa, xb));
    const float by0 = warp_min_f(fminf(ya, yb)), by1 = warp_max_f(fmaxf(ya, yb));
    const float mmax = dconst ? mband : warp_max_f(mband);
    const float st = (float)(t + 1) * pc.dt, st0 = (float)(tb0 + 1) * pc.dt;
    // the sorted positions whose circles can reach the warp box: a circle's key moves by at
    // most dmax per step from its step-0 value, and projecting on the lane direction does not
    // increase distances, so every circle the box test below can pass lies in [lo, hi)
    const CircleIndex ci = circle_index(smem, L);
    int lo = 0, hi = n_circ;
    {
        const float qx0 = bx0 * ci.dx, qx1 = bx1 * ci.dx, qy0 = by0 * ci.dy, qy1 = by1 * ci.dy;
        const float slo = fminf(qx0, qx1) + fminf(qy0, qy1), shi = fmaxf(qx0, qx1) + fmaxf(qy0, qy1);
        const float reach = (mmax + ci.rmax + pc.ego_rmax) * 1.0001f + 1e-4f + ci.dmax * (float)(2 * tb1 + 2) +
                            1e-3f + 1e-5f * (fabsf(slo) + fabsf(shi));
        const float f0 = (slo - reach - ci.smin) * ci.inv_w, f1 = (shi + reach - ci.smin) * ci.inv_w;
        if (ci.inv_w > 0.0f && isfinite(f0) && isfinite(f1)) {
            const int b0 = f0 < 1.0f ? 0 : (int)fminf(floorf(f0) - 1.0f, (float)CIRC_BUCKETS);
            const int b1 = f1 < -1.0f ? -1 : (int)fminf(floorf(f1) + 1.0f, (float)(CIRC_BUCKETS - 1));
            lo = ci.start[IX(b0, CIRC_BUCKETS + 1)];
            hi = ci.start[IX(b1 + 1, CIRC_BUCKETS + 1)];
        }
    }
    float dobj = INFINITY;
    for (int base = lo; base < hi; base += 32) {
        const int pos = base + lane;
        bool hit = false;
        if (pos < hi) {
            if (STATS) cnt.circ++;
            const float4 c = circ[IX(pos, n_circ)];
            const float2 cc = circle_centre(c, vel, ci.order, table, n_circ, tb0, pos, st0, has_table, moving);
            const float lim = (mmax + c.z + pc.ego_rmax) * 1.0001f + 1e-4f;
            const float ext = tb1 != tb0 && (has_table || moving) ? disp[IX(pos, n_circ)] * (float)(tb1 - tb0) : 0.0f;
            const float dx = fmaxf(fmaxf(bx0 - cc.x, cc.x - bx1), 0.0f);
            const float dy = fmaxf(fmaxf(by0 - cc.y, cc.y - by1), 0.0f);
            hit = lim > 0.0f && fmaf(dx, dx, dy * dy) <= (lim + ext) * (lim + ext);
        }
        unsigned m = __ballot_sync(0xffffffffu, hit);
        for (int j = 0; m; ++j) {
            const int bit = __ffs(m) - 1;
            m &= m - 1;
            if (G > 1 && (j & (G - 1)) != lane_g) continue;
            if (STATS) cnt.cand++;
            const int pos2 = base + bit;
            const float4 c = circ[IX(pos2, n_circ)];
            const float2 cc = circle_centre(c, vel, ci.order, table, n_circ, t, pos2, st, has_table, moving);
            // the circle centre in the ego frame, along the heading (al) and across it (pr): the
            // squared distance to the ego circle at offset o along the heading is (al - o)^2 + pr^2
            const float wx = cc.x - nx, wy = cc.y - ny;
            const float al = fmaf(wx, cnth, wy * snth);
            const float pr = fmaf(wx, snth, -(wy * cnth));
            const float p2 = pr * pr;
            if (dconst) {
                // equal ego radii: the closest ego circle gives the pair minimum (sqrt and the
                // subtraction are monotone), one square root per circle
                float d2m;
                if (SIMPLE || pc.n_ego == 3) {        // the paper's ego model: three circles, no bound checks
                    const float e0 = al - pc.ego_off[0], e1 = al - pc.ego_off[1], e2 = al - pc.ego_off[2];
                    d2m = fminf(fminf(fmaf(e0, e0, p2), fmaf(e1, e1, p2)), fmaf(e2, e2, p2));
                } else {
                    d2m = INFINITY;
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        if (e >= pc.n_ego) break;
                        const float de = al - pc.ego_off[e];
                        d2m = fminf(d2m, fmaf(de, de, p2));
                    }
                }
                // every candidate enters the minimum: a pair outside the band has a clearance above
                // the band, so it neither lowers the minimum below an in-band pair's nor, alone,
                // brings the clearance under d_safe (c_safe stays 0, as with no pair)
                if (STATS && d2m <= c.w) cnt.pair++;
                dobj = fminf(dobj, dist_of(d2m) - (c.z + pc.ego_rad[0]));
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    if (e >= pc.n_ego) break;
                    const float R = c.z + pc.ego_rad[e];
                    const float lim = mband + R;
                    const float de = al - pc.ego_off[e];
                    const float d2 = fmaf(de, de, p2);
                    if (lim > 0.0f && d2 <= lim * lim) {
                        if (STATS) cnt.pair++;
                        dobj = fminf(dobj, dist_of(d2) - R);
                    }
                }
            }
        }
    }
    return group_min<G>(dobj, mask);
}

// The scene blob as staged in shared memory (base: its first byte; the level-2 boxes follow it).
struct Scene {
    const unsigned char* base;
    const unsigned char* gscene;   // the scene buffer in global memory (the search's vertex boxes)
    const float4* ctl;
    const float* c0;
    const float2* vert;
    const float4* seg;
    const float* head;
    const float4* l1;
    const float4* circ;
    const float2* vel;
    const float* disp;
};

__device__ __forceinline__ Scene scene_of(const SceneLayout& L, const unsigned char* smem,
                                          const unsigned char* gscene) {
    Scene s;
    s.base = smem;
    s.gscene = gscene;
    s.ctl = reinterpret_cast<const float4*>(smem + L.off_ctl);
    s.c0 = reinterpret_cast<const float*>(smem + L.off_c0);
    s.vert = reinterpret_cast<const float2*>(smem + L.off_vert);
    s.seg = reinterpret_cast<const float4*>(smem + L.off_seg);
    s.head = reinterpret_cast<const float*>(smem + L.off_head);
    s.l1 = reinterpret_cast<const float4*>(smem + L.off_l1);
    s.circ = reinterpret_cast<const float4*>(smem + L.off_circ);
    s.vel = reinterpret_cast<const float2*>(smem + L.off_vel);
    s.disp = reinterpret_cast<const float*>(smem + L.off_disp);
    return s;
}

// x_t of one rollout with compensated (Kahan) accumulation (the value of each
// coordinate is hi - lo), the direction of its yaw and |P_t - T_P|^2.
struct Roll {
    float px, py, th, v, px_c, py_c, th_c, v_c, sth, cth, tdp;
};

// The steering angle of the steering-rate model (value hi - lo, compensated like the other
// states) lives in this thread's shared-memory slot.
__device__ __forceinline__ float2* steer_slot(const unsigned char* smem, const SceneLayout& L) {
    return reinterpret_cast<float2*>(const_cast<unsigned char*>(smem) + L.bytes + block_extra_bytes(L)) +
           threadIdx.x;
}

// What the state cost of one step needs beyond the search: x_{t+1} (binary32 head and
// compensation), its yaw direction, and the cheap terms c_target (Eq. 13), the speed
// error, d_safe (Eq. 17) and the control cost of Eq. (8).
struct StepIn {
    float nx, ny, px_c, py_c, th, th_c, snth, cnth, c_target, dv, ds, qu;
};

// Eq. (5): explicit Euler from x_t to x_{t+1} under the perturbed controls of step t.
// EXT: compiled with the steering-rate model and the cost-to-go form (otherwise both are
// compiled out: model 0 and whole-cost weights).
template <bool BF16, bool EXT, bool SIMPLE = false>
__device__ __forceinline__ StepIn dyn_step(const PlanConst& pc, const float4 ct, float c0t, float2 zz, float2 tp,
                                           Roll& r, float2* ds) {
    const Perturbed pe = perturb(ct.x, ct.y, zz, pc.sig_a, pc.sig_d, pc.amin, pc.amax, pc.dmin, pc.dmax);
    const float vt = r.v - r.v_c;
    float acc = pe.va;
    if (!SIMPLE && pc.vcap) acc = fmaxf(fminf(acc, (pc.v_max - vt) / pc.dt), pc.amin);
    // model 0: the steering angle is the control; model 1: it is the state, advanced by the
    // steering rate (the second control) after its tangent is taken (right-hand side at x_t)
    float tn;
    if (EXT && pc.model == 1) {
        float2 d = *ds;
        tn = tanf(d.x);
        kahan_add(d.x, d.y, __fmul_rn(pe.vd, pc.dt));
        *ds = d;
    } else {
        tn = tanf(pe.vd);
    }
    // the increments are rounded products (no fused multiply-add), the same expressions as
    // the time-split form below, so both give the same bits
    kahan_add(r.px, r.px_c, __fmul_rn(__fmul_rn(vt, r.cth), pc.dt));
    kahan_add(r.py, r.py_c, __fmul_rn(__fmul_rn(vt, r.sth), pc.dt));
    kahan_add(r.th, r.th_c, __fmul_rn(__fmul_rn(vt, tn), pc.dt_over_L));
    kahan_add(r.v, r.v_c, __fmul_rn(acc, pc.dt));
    StepIn s;
    s.nx = r.px;
    s.ny = r.py;
    s.px_c = r.px_c;
    s.py_c = r.py_c;
    s.th = r.th;
    s.th_c = r.th_c;
    sincosf(r.th, &s.snth, &s.cnth);
    // Eq. (13): progress towards the target point
    const float tx = (s.nx - tp.x) - r.px_c, ty = (s.ny - tp.y) - r.py_c;
    const float tdn = fmaf(tx, tx, ty * ty);
    s.c_target = tdn > r.tdp ? 1.0f : 0.0f;
    r.tdp = tdn;
    s.dv = (r.v - pc.v_ref) - r.v_c;
    s.ds = fmaf(pc.d_safe_c, r.v - r.v_c, pc.d_safe_0);
    s.qu = fmaf(ct.z, pe.ea, fmaf(ct.w, pe.ed, c0t));
    r.sth = s.snth;
    r.cth = s.cnth;
    return s;
}

// Weighted state cost of Eq. (18) at x_{t+1}: the closest waypoint (Eq. 12, 14, search on
// the binary32 position from the warm start jb) and the obstacle term (Eq. 16-17).
template <int G, bool STATS, bool SIMPLE = false>
__device__ __forceinline__ float state_cost(const PlanConst& pc, const SceneLayout& L, const Scene& sc,
                                            const float2* table, const StepIn& s, int t, int tb0, int tb1,
                                            bool has_table, bool moving, bool multi_head, bool dconst, int lane,
                                            int lane_g, unsigned mask, int& jb, Counters& cnt) {
    float d2r;
    if (SIMPLE || pc.ref_mode == 0) {
        // search hint: the last closest segment moved on by the projection of the new position on
        // it, in units of its length (on a lane of equal segments, the segment that holds the
        // projection)
        int jh;
        {
            const float2 pa = sc.vert[IX(jb, L.n_ref)];
            const float4 ps = sc.seg[IX(jb, L.n_seg)];
            const float tq = fminf(fmaxf(fmaf(s.nx - pa.x, ps.z, (s.ny - pa.y) * ps.w), -64.0f), 64.0f);
            jh = min(max(jb + (int)floorf(tq), 0), L.n_seg - 1);
        }
        nearest_segment<G, STATS>(s.nx, s.ny, sc.vert, sc.seg, sc.head, ref_boxes(sc.base, sc.gscene, L), L.n_seg, L.n_l1,
                                  lane_g, mask, jh, multi_head, search_lfac(sc.base, L), jb, d2r, cnt);
    } else {
        nearest_vertex<G>(s.nx, s.ny, sc.vert, sc.l1, ref_boxes(sc.base, sc.gscene, L).l2, L.n_ref, L.n_l1, L.n_l2, lane_g, mask,
                          jb, d2r);
    }
    const float thr = sc.head[IX(min(jb, L.n_seg - 1), L.n_seg)];
    {
        // c_dist on the compensated position: closest point of the winning segment or vertex
        const float2 a = sc.vert[IX(jb, L.n_ref)];
        float qx = a.x, qy = a.y;
        if (SIMPLE || pc.ref_mode == 0) {
            const float4 sg = sc.seg[IX(jb, L.n_seg)];
            const float tau = fmaf(s.nx - a.x, sg.z, (s.ny - a.y) * sg.w);
            if (tau >= 1.0f) {
                qx = sc.vert[IX(jb + 1, L.n_ref)].x;
                qy = sc.vert[IX(jb + 1, L.n_ref)].y;
            } else if (tau > 0.0f) {
                qx = fmaf(tau, sg.x, a.x);
                qy = fmaf(tau, sg.y, a.y);
            }
        }
        const float dx = (s.nx - qx) - s.px_c, dy = (s.ny - qy) - s.py_c;
        d2r = fmaf(dx, dx, dy * dy);
    }
    const float dyaw = wrap_pi((s.th - thr) - s.th_c);

    // Eq. (16)-(17): ego circles against obstacle circles
    const float mband = (!SIMPLE && pc.collision_only) ? fmaxf(s.ds, 0.0f) : s.ds;
    float dobj = INFINITY;
    if (L.n_circ > 0)
        dobj = obstacle_min<G, STATS, SIMPLE>(pc, sc.base, L, sc.circ, sc.vel, sc.disp, table, L.n_circ, t, tb0, tb1, has_table, moving, dconst,
                                      s.nx, s.ny, s.cnth, s.snth, mband, lane, lane_g, mask, cnt);
    const float gap = s.ds - dobj;
    float c_safe = gap > 0.0f ? gap * gap : 0.0f;
    if (!SIMPLE && pc.collision_only && !(dobj <= 0.0f)) c_safe = 0.0f;

    // Eq. (18) weighted state cost
    return fmaf(pc.w_dist, d2r,
                fmaf(pc.w_target, s.c_target,
                     fmaf(pc.w_yaw, dyaw * dyaw, fmaf(pc.w_speed, s.dv * s.dv, pc.w_safe * c_safe))));
}

// Debug build: the block's dynamic shared memory must hold the staged blob, what the block
// builds after it and the steering slots; a shortfall is counted (the normal build has no check).
__device__ __forceinline__ void check_smem(const SceneLayout& L, bool model1) {
#ifdef MPPI_CHECKS
    unsigned dyn = 0;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    if (threadIdx.x == 0 && (size_t)L.bytes + block_extra_bytes(L) + steer_slots_bytes(blockDim.x, model1) > dyn)
        atomicAdd(&g_check_hits, 1ull);
#else
    (void)L;
    (void)model1;
#endif
}

// One sample's rollout and cost (Algorithm 1 inner loop), by the G lanes of its group.
// smem holds the staged scene blob; z the noise [T][K]; x0 = (0, 0, yaw0, v0) in the local
// frame; jb0 the segment closest to x0; S[k] receives the cost.  Every lane of the warp
// must call it (the broad phase and the group reductions are warp / group collective).
//
// TIME = false: the G lanes run the dynamics redundantly (identical bits) and split the
// reference search and the obstacle pairs of every step, combining with shuffles.
// TIME = true: the G lanes split the steps.  In each block of G steps lane p perturbs the
// controls of step t0 + p and takes its steering tangent; yaw and speed, which do not
// depend on the position, are then advanced through the block by every lane from the
// shuffled controls, lane p takes the sine and cosine of its step's yaw, and the positions
// follow from the shuffled directions (same operations as one lane per sample, identical
// bits).  Lane p evaluates the state cost of its step (the reference search warm-started
// from its own previous step) and the step costs are added in step order, so S is bit for
// bit that of G = 1.
// SIMPLE: the plan's scene has static circles without a centre table, three ego circles of one
// radius, a constant safety band, no collision-only switch, no speed cap, the segment form of
// the closest waypoint and a lane of one heading; those decisions are then compile-time
// constants (the same arithmetic, so the same bits, with fewer instructions).
template <int G, bool TIME, bool BF16, bool STATS, bool EXT, bool SIMPLE = false>
__device__ __forceinline__ void rollout_sample(const PlanConst& pc, const SceneLayout& L, const unsigned char* smem,
                                               const unsigned char* gscene,
                                               const typename NoiseT<BF16>::type* __restrict__ z,
                                               const float2* table, float4 x0, float d0, bool moving,
                                               bool multi_head, int jb0, int k, double* S_out,
                                               unsigned long long* stats,
                                               float* prefix = nullptr) {
    const Scene sc = scene_of(L, smem, gscene);
    const int lane = threadIdx.x & 31;
    const int lane_g = threadIdx.x & (G - 1);
    const unsigned mask = group_mask<G>();
    const int K = pc.K, T = pc.T;
    const int kk = min(k, K - 1);               // whole groups past K run along (shuffle safety)
    const bool has_table = !SIMPLE && pc.has_table != 0;
    const float2 tp = sc.vert[L.n_ref - 1];     // target point T_P: last vertex
    const bool dconst = SIMPLE || (pc.d_safe_c == 0.0f && pc.ego_same_radius);
    if (SIMPLE) {
        moving = false;
        multi_head = false;
    }

    Roll r;
    r.px = x0.x;
    r.py = x0.y;
    r.th = x0.z;
    r.v = x0.w;
    r.px_c = r.py_c = r.th_c = r.v_c = 0.0f;
    if (EXT && pc.model == 1) *steer_slot(smem, L) = make_float2(d0, 0.0f);
    sincosf(r.th, &r.sth, &r.cth);
    r.tdp = fmaf(tp.x, tp.x, tp.y * tp.y);      // |P_0 - T_P|^2 with P_0 = (0, 0)
    int jb = jb0;              // closest segment of the last evaluated step
    float s_hi = 0.0f, s_c = 0.0f, q_last = 0.0f;
    Counters cnt{0, 0, 0, 0, 0, 0, 0};

    if constexpr (!TIME) {
        // the noise is read one step ahead (its latency is spent on the previous step's work)
        typename NoiseT<BF16>::type znext = z[kk];
        for (int t = 0; t < T; ++t) {
            const typename NoiseT<BF16>::type zcur = znext;
            znext = z[(size_t)min(t + 1, T - 1) * K + kk];
            const float2 zz = noise_value<BF16>(zcur);
            const StepIn s = dyn_step<BF16, EXT, SIMPLE>(pc, sc.ctl[IX(t, T)], sc.c0[IX(t, T)], zz, tp, r,
                                                         steer_slot(smem, L));
            const float qx = state_cost<G, STATS, SIMPLE>(pc, L, sc, table, s, t, t, t, has_table, moving, multi_head,
                                                  dconst, lane, lane_g, mask, jb, cnt);
            if (EXT && prefix && lane_g == 0 && k < K) prefix[(size_t)t * K + k] = s_hi - s_c;   // cost of steps < t
            kahan_add(s_hi, s_c, qx + s.qu);    // Eq. (6)
            q_last = qx;
        }
    } else {
        // the noise of a lane's own step is read one block of steps ahead (the load's latency is
        // then spent on the previous block's work; the two-lane plain form and the general split)
        typename NoiseT<BF16>::type zpre = z[(size_t)min(lane_g, min(G, T) - 1) * K + kk];
        for (int t0 = 0; t0 < T; t0 += G) {
            // nv real steps in this block; past the last step a lane re-evaluates step T - 1
            // (the warp stays converged)
            const int nv = min(G, T - t0);
            const int my = min(lane_g, nv - 1);
            const int tm = t0 + my;
            StepIn e;
            if constexpr (G == 2 && !EXT) {
                // two lanes, plain form: lane p perturbs the controls of step t0 + p and takes their
                // tangent; yaw and speed advance through both steps in both lanes from the shuffled
                // controls; lane p takes the sine and cosine of the yaw after its own step, and the
                // positions advance through both steps from the shuffled directions.  The same
                // operations as one lane per sample (dyn_step), so the same bits, with one tangent
                // and one sine/cosine per step instead of two.
                const typename NoiseT<BF16>::type zcur = zpre;
                {
                    const int tn = t0 + G;      // the next block's own step (T - 1 past the end)
                    const int tmn = tn < T ? tn + min(lane_g, min(G, T - tn) - 1) : T - 1;
                    zpre = z[(size_t)tmn * K + kk];
                }
                const float4 ct = sc.ctl[IX(tm, T)];
                const Perturbed pe = perturb(ct.x, ct.y, noise_value<BF16>(zcur), pc.sig_a, pc.sig_d, pc.amin,
                                             pc.amax, pc.dmin, pc.dmax);
                const float tn_own = tanf(pe.vd);
                // step t0 (lane 0's controls)
                const float va0 = __shfl_sync(mask, pe.va, 0, 2), tn0 = __shfl_sync(mask, tn_own, 0, 2);
                const float vt0 = r.v - r.v_c;
                float acc = va0;
                if (!SIMPLE && pc.vcap) acc = fmaxf(fminf(acc, (pc.v_max - vt0) / pc.dt), pc.amin);
                kahan_add(r.th, r.th_c, __fmul_rn(__fmul_rn(vt0, tn0), pc.dt_over_L));
                kahan_add(r.v, r.v_c, __fmul_rn(acc, pc.dt));
                float th_own = r.th, thc_own = r.th_c, v_own = r.v, vc_own = r.v_c;
                // step t0 + 1 (lane 1's controls), when there is one: computed on copies and taken
                // by selects (no branch; the same operations, so the same bits)
                const bool two = nv == 2, mine = my == 1;
                const float va1 = __shfl_sync(mask, pe.va, 1, 2), tn1 = __shfl_sync(mask, tn_own, 1, 2);
                const float vt1 = r.v - r.v_c;
                {
                    acc = va1;
                    if (!SIMPLE && pc.vcap) acc = fmaxf(fminf(acc, (pc.v_max - vt1) / pc.dt), pc.amin);
                    float th2 = r.th, thc2 = r.th_c, v2 = r.v, vc2 = r.v_c;
                    kahan_add(th2, thc2, __fmul_rn(__fmul_rn(vt1, tn1), pc.dt_over_L));
                    kahan_add(v2, vc2, __fmul_rn(acc, pc.dt));
                    th_own = mine ? th2 : th_own;
                    thc_own = mine ? thc2 : thc_own;
                    v_own = mine ? v2 : v_own;
                    vc_own = mine ? vc2 : vc_own;
                    r.th = two ? th2 : r.th;
                    r.th_c = two ? thc2 : r.th_c;
                    r.v = two ? v2 : r.v;
                    r.v_c = two ? vc2 : r.v_c;
                }
                sincosf(th_own, &e.snth, &e.cnth);
                // positions: step t0 moves along the carried direction, step t0 + 1 along lane 0's
                const float cn0 = __shfl_sync(mask, e.cnth, 0, 2), sn0 = __shfl_sync(mask, e.snth, 0, 2);
                kahan_add(r.px, r.px_c, __fmul_rn(__fmul_rn(vt0, r.cth), pc.dt));
                kahan_add(r.py, r.py_c, __fmul_rn(__fmul_rn(vt0, r.sth), pc.dt));
                float tx = (r.px - tp.x) - r.px_c, ty = (r.py - tp.y) - r.py_c;
                float tdn = fmaf(tx, tx, ty * ty);
                e.nx = r.px;
                e.ny = r.py;
                e.px_c = r.px_c;
                e.py_c = r.py_c;
                e.c_target = tdn > r.tdp ? 1.0f : 0.0f;
                r.tdp = tdn;
                {
                    float px2 = r.px, pxc2 = r.px_c, py2 = r.py, pyc2 = r.py_c;
                    kahan_add(px2, pxc2, __fmul_rn(__fmul_rn(vt1, cn0), pc.dt));
                    kahan_add(py2, pyc2, __fmul_rn(__fmul_rn(vt1, sn0), pc.dt));
                    const float tx2 = (px2 - tp.x) - pxc2, ty2 = (py2 - tp.y) - pyc2;
                    const float tdn2 = fmaf(tx2, tx2, ty2 * ty2);
                    e.nx = mine ? px2 : e.nx;
                    e.ny = mine ? py2 : e.ny;
                    e.px_c = mine ? pxc2 : e.px_c;
                    e.py_c = mine ? pyc2 : e.py_c;
                    e.c_target = mine ? (tdn2 > r.tdp ? 1.0f : 0.0f) : e.c_target;
                    r.px = two ? px2 : r.px;
                    r.px_c = two ? pxc2 : r.px_c;
                    r.py = two ? py2 : r.py;
                    r.py_c = two ? pyc2 : r.py_c;
                    r.tdp = two ? tdn2 : r.tdp;
                }
                r.cth = __shfl_sync(mask, e.cnth, nv - 1, 2);
                r.sth = __shfl_sync(mask, e.snth, nv - 1, 2);
                e.th = th_own;
                e.th_c = thc_own;
                e.dv = (v_own - pc.v_ref) - vc_own;
                // d_safe of Eq. (17): the specialised step has d_safe_c = 0
                e.ds = SIMPLE ? pc.d_safe_0 : fmaf(pc.d_safe_c, v_own - vc_own, pc.d_safe_0);
                e.qu = fmaf(ct.z, pe.ea, fmaf(ct.w, pe.ed, sc.c0[IX(tm, T)]));
            } else if constexpr (G <= 2) {
                // two lanes with the steering-rate model or the cost-to-go form: both lanes
                // integrate both steps
#pragma unroll 1
                for (int j = 0; j < nv; ++j) {
                    const int t = t0 + j;
                    const float2 zz = NoiseT<BF16>::load(z + (size_t)t * K + kk);
                    const StepIn q = dyn_step<BF16, EXT, SIMPLE>(pc, sc.ctl[IX(t, T)], sc.c0[IX(t, T)], zz, tp, r,
                                                                 steer_slot(smem, L));
                    if (j == my) e = q;
                }
            } else {
            // own step: perturbed controls and the steering tangent (independent of the state)
            const typename NoiseT<BF16>::type zcur = zpre;
            {
                const int tn = t0 + G;
                const int tmn = tn < T ? tn + min(lane_g, min(G, T - tn) - 1) : T - 1;
                zpre = z[(size_t)tmn * K + kk];
            }
            const float4 ct = sc.ctl[IX(tm, T)];
            const Perturbed pe = perturb(ct.x, ct.y, noise_value<BF16>(zcur), pc.sig_a, pc.sig_d,
                                         pc.amin, pc.amax, pc.dmin, pc.dmax);
            float tn_own;
            if (EXT && pc.model == 1) {
                // steering angle through the block (every lane); the tangent of the angle at
                // the start of the own step
                float2 d = *steer_slot(smem, L);
                float d_own = d.x;
#pragma unroll 1
                for (int j = 0; j < nv; ++j) {
                    const float w = __shfl_sync(mask, pe.vd, j, G);
                    if (j == my) d_own = d.x;
                    kahan_add(d.x, d.y, __fmul_rn(w, pc.dt));
                }
                *steer_slot(smem, L) = d;
                tn_own = tanf(d_own);
            } else {
                tn_own = tanf(pe.vd);
            }
            // yaw and speed through the block: every lane, the lanes' controls by shuffle
            float vt_own = 0.0f, th_own = 0.0f, thc_own = 0.0f, v_own = 0.0f, vc_own = 0.0f;
#pragma unroll 1
            for (int j = 0; j < nv; ++j) {
                const float va = __shfl_sync(mask, pe.va, j, G);
                const float tn = __shfl_sync(mask, tn_own, j, G);
                const float vt = r.v - r.v_c;
                float acc = va;
                if (!SIMPLE && pc.vcap) acc = fmaxf(fminf(acc, (pc.v_max - vt) / pc.dt), pc.amin);
                kahan_add(r.th, r.th_c, __fmul_rn(__fmul_rn(vt, tn), pc.dt_over_L));
                kahan_add(r.v, r.v_c, __fmul_rn(acc, pc.dt));
                if (j == my) {
                    vt_own = vt;
                    th_own = r.th;
                    thc_own = r.th_c;
                    v_own = r.v;
                    vc_own = r.v_c;
                }
            }
            sincosf(th_own, &e.snth, &e.cnth);
            // positions through the block: the yaw direction before step j is lane j-1's
            // (the carried one for j = 0)
#pragma unroll 1
            for (int j = 0; j < nv; ++j) {
                const float vt = __shfl_sync(mask, vt_own, j, G);
                const float cn = __shfl_sync(mask, e.cnth, j > 0 ? j - 1 : 0, G);
                const float sn = __shfl_sync(mask, e.snth, j > 0 ? j - 1 : 0, G);
                const float cj = j > 0 ? cn : r.cth, sj = j > 0 ? sn : r.sth;
                kahan_add(r.px, r.px_c, __fmul_rn(__fmul_rn(vt, cj), pc.dt));
                kahan_add(r.py, r.py_c, __fmul_rn(__fmul_rn(vt, sj), pc.dt));
                // Eq. (13): progress towards the target point
                const float tx = (r.px - tp.x) - r.px_c, ty = (r.py - tp.y) - r.py_c;
                const float tdn = fmaf(tx, tx, ty * ty);
                if (j == my) {
                    e.nx = r.px;
                    e.ny = r.py;
                    e.px_c = r.px_c;
                    e.py_c = r.py_c;
                    e.c_target = tdn > r.tdp ? 1.0f : 0.0f;
                }
                r.tdp = tdn;
            }
            r.cth = __shfl_sync(mask, e.cnth, nv - 1, G);
            r.sth = __shfl_sync(mask, e.snth, nv - 1, G);
            e.th = th_own;
            e.th_c = thc_own;
            e.dv = (v_own - pc.v_ref) - vc_own;
            e.ds = fmaf(pc.d_safe_c, v_own - vc_own, pc.d_safe_0);
            e.qu = fmaf(ct.z, pe.ea, fmaf(ct.w, pe.ed, sc.c0[IX(tm, T)]));
            }
            const int tb1 = min(t0 + G - 1, T - 1);
            const float qx = state_cost<1, STATS, SIMPLE>(pc, L, sc, table, e, tm, t0, tb1, has_table, moving, multi_head,
                                                  dconst, lane, 0, mask, jb, cnt);
            const float c = qx + e.qu;
            float pre_own = 0.0f;
#pragma unroll
            for (int j = 0; j < G; ++j) {
                const float cj = __shfl_sync(mask, c, j, G);
                const float qj = __shfl_sync(mask, qx, j, G);
                if (t0 + j < T) {
                    if (EXT && j == lane_g) pre_own = s_hi - s_c;
                    kahan_add(s_hi, s_c, cj);   // Eq. (6), in step order
                    q_last = qj;
                }
            }
            if (EXT && prefix && lane_g < nv && k < K) prefix[(size_t)(t0 + lane_g) * K + k] = pre_own;   // cost of steps < t
        }
    }
    if (lane_g == 0 && k < K) {
        double S = (double)s_hi - (double)s_c;
        if (pc.w_terminal != 0.0f) S += (double)pc.w_terminal * (double)q_last;
        S_out[k] = S;
    }
    if (STATS && k < K) {
        const unsigned v7[7] = {cnt.l2, cnt.l1, cnt.seg, cnt.refine, cnt.circ, cnt.cand, cnt.pair};
        for (int i = 0; i < 7; ++i) atomicAdd(stats + i, (unsigned long long)v7[i]);
    }
}
// -----------------------------------------------------------------------------
// reductions
// -----------------------------------------------------------------------------
struct MinRec {
    double v;
    int i;
    int n;
};

__device__ __forceinline__ MinRec min_combine(MinRec a, MinRec b) {
    MinRec r;
    r.n = a.n + b.n;
    if (b.v < a.v || (b.v == a.v && b.i < a.i)) {
        r.v = b.v;
        r.i = b.i;
    } else {
        r.v = a.v;
        r.i = a.i;
    }
    return r;
}

__device__ __forceinline__ MinRec warp_min(MinRec a) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        MinRec b;
        b.v = __shfl_xor_sync(0xffffffffu, a.v, o);
        b.i = __shfl_xor_sync(0xffffffffu, a.i, o);
        b.n = __shfl_xor_sync(0xffffffffu, a.n, o);
        a = min_combine(a, b);
    }
    return a;
}

static __device__ MinRec block_min(MinRec a) {
    __shared__ double sv[32];
    __shared__ int si[32], sn[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    a = warp_min(a);
    if (lane == 0) {
        sv[w] = a.v;
        si[w] = a.i;
        sn[w] = a.n;
    }
    __syncthreads();
    if (w == 0) {
        MinRec r{INFINITY, 0x7fffffff, 0};
        if (lane < nw) r = MinRec{sv[lane], si[lane], sn[lane]};
        a = warp_min(r);
    }
    __syncthreads();
    return a;
}

// -----------------------------------------------------------------------------
// argmin with integer keys: a finite binary64 cost maps to a 64-bit key with the same order
// (sign bit set: all bits flipped, else the sign bit set; -0 is taken as +0), so the
// reductions compare integers instead of using the binary64 pipe.  Ties go to the lowest
// index; n counts the finite costs.
// -----------------------------------------------------------------------------
struct KeyRec {
    unsigned long long key;
    int i;
    int n;
};

__device__ __forceinline__ unsigned long long order_key(double s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(s + 0.0);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double key_value(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

__device__ __forceinline__ KeyRec key_combine(KeyRec a, KeyRec b) {
    KeyRec r = (b.key < a.key || (b.key == a.key && b.i < a.i)) ? b : a;
    r.n = a.n + b.n;
    return r;
}

static __device__ KeyRec block_keymin(KeyRec a) {
    __shared__ unsigned long long sk[32];
    __shared__ int si[32], sn[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        KeyRec b;
        b.key = __shfl_xor_sync(0xffffffffu, a.key, o);
        b.i = __shfl_xor_sync(0xffffffffu, a.i, o);
        b.n = __shfl_xor_sync(0xffffffffu, a.n, o);
        a = key_combine(a, b);
    }
    if (lane == 0) {
        sk[w] = a.key;
        si[w] = a.i;
        sn[w] = a.n;
    }
    __syncthreads();
    if (w == 0) {
        a = lane < nw ? KeyRec{sk[lane], si[lane], sn[lane]} : KeyRec{~0ull, 0x7fffffff, 0};
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            KeyRec b;
            b.key = __shfl_xor_sync(0xffffffffu, a.key, o);
            b.i = __shfl_xor_sync(0xffffffffu, a.i, o);
            b.n = __shfl_xor_sync(0xffffffffu, a.n, o);
            a = key_combine(a, b);
        }
    }
    __syncthreads();
    return a;
}

// The argmin of Algorithm 1 (S_min and its sample) folded into the end of the rollout kernel:
// each block reduces the costs of its own samples k0 .. k0 + nk - 1 (written by the block
// before the barrier) into one record, and the last block to finish (ticket) combines the
// records of all blocks in block order.  Every block takes part, also one whose staging
// timed out (with an empty record), so the ticket always completes and returns to zero.
__device__ __forceinline__ void rollout_argmin_tail(int K, const PlanBuffers& b, int k0, int nk, bool valid) {
    __shared__ bool last;
    __syncthreads();
    KeyRec r{~0ull, 0x7fffffff, 0};
    const int k = k0 + (int)threadIdx.x;
    if (valid && (int)threadIdx.x < nk && k < K) {
        const double s = b.S[k];
        if (isfinite(s)) r = KeyRec{order_key(s), k, 1};
    }
    r = block_keymin(r);
    if (threadIdx.x == 0) {
        b.kmin_part[blockIdx.x] = make_ulonglong2(r.key, ((unsigned long long)(unsigned)r.n << 32) | (unsigned)r.i);
        __threadfence();
        last = atomicAdd(&b.state->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    KeyRec q{~0ull, 0x7fffffff, 0};
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        const ulonglong2 p = __ldcg(&b.kmin_part[i]);
        q = key_combine(q, KeyRec{p.x, (int)(unsigned)(p.y & 0xffffffffull), (int)(p.y >> 32)});
    }
    q = block_keymin(q);
    if (threadIdx.x == 0) {
        b.state->s_min = q.n > 0 ? key_value(q.key) : INFINITY;
        b.state->argmin = q.n > 0 ? q.i : -1;
        b.state->n_finite = q.n;
        b.state->ticket = 0u;
    }
}

static __device__ double block_sum_d(double v) {
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < nw ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}

// Block-wide inclusive scans in binary64 over the first nwa warps of the block; the other
// warps add nothing and only take part in the barriers.  The active warps add in the same
// order whatever the block size (warp scan, then the scan of the warp totals).
static __device__ double block_scan_incl(double v, double* sh, int nwa) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w < nwa) {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double n = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += n;
        }
        if (lane == 31) sh[w] = v;
    }
    __syncthreads();
    if (w == 0) {
        double s = lane < nwa ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double n = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += n;
        }
        sh[lane] = s;
    }
    __syncthreads();
    if (w > 0 && w < nwa) v += sh[w - 1];
    __syncthreads();
    return v;
}

// Two independent scans in one pass (one set of barriers).
static __device__ double2 block_scan2_incl(double2 v, double2* sh, int nwa) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w < nwa) {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double nx = __shfl_up_sync(0xffffffffu, v.x, o);
            const double ny = __shfl_up_sync(0xffffffffu, v.y, o);
            if (lane >= o) {
                v.x += nx;
                v.y += ny;
            }
        }
        if (lane == 31) sh[w] = v;
    }
    __syncthreads();
    if (w == 0) {
        double2 s = lane < nwa ? sh[lane] : make_double2(0.0, 0.0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double nx = __shfl_up_sync(0xffffffffu, s.x, o);
            const double ny = __shfl_up_sync(0xffffffffu, s.y, o);
            if (lane >= o) {
                s.x += nx;
                s.y += ny;
            }
        }
        sh[lane] = s;
    }
    __syncthreads();
    if (w > 0 && w < nwa) {
        v.x += sh[w - 1].x;
        v.y += sh[w - 1].y;
    }
    __syncthreads();
    return v;
}

__device__ __forceinline__ double clampd(double x, double lo, double hi) { return fmin(fmax(x, lo), hi); }

// -----------------------------------------------------------------------------
// Softmin weight of Eq. (11), exp(-(S - S_min) / lambda): the difference is formed in
// binary64 (costs are large next to their spread), rounded to binary32 and scaled by
// 1 / lambda, and the exponential is taken in binary32 (relative error of the weight a few
// 1e-7 times the exponent, far below the update's tolerance); zero for a non-finite cost.
// binary64 transcendentals are the slow path on this part.
// -----------------------------------------------------------------------------
__device__ __forceinline__ float softmin_weight(double s, double smin, float inv_lam) {
    return isfinite(s) ? expf((float)(smin - s) * inv_lam) : 0.0f;
}

// -----------------------------------------------------------------------------
// wsum tile: per step t in [t0, t0 + TT) (TT <= WS_TT, a compile-time bound so the step
// loop unrolls; the partial of each step does not depend on how the steps are tiled), sum
// over the k-tile kt (kt_size samples)
// of w_k eps'_{t,k}.  Each thread owns WS_J samples, recomputes eps' from z exactly
// as the rollout did, accumulates in binary32 over its samples and its warp (32 x WS_J
// products); the per-warp partials are added in binary64 into du_part[kt][T][2].
// -----------------------------------------------------------------------------

// STAGED: z is the tile itself in shared memory (row t - t0 of kt_size samples, landed by
// the caller's bulk copies; wait_tile(r) waits for row r before its products are taken, so
// the later rows land while the earlier ones are summed); otherwise z is the noise in global
// memory.  Both read the same values in the same order: the same bits.
template <bool BF16, bool CTG = false, int TT = WS_TT, bool STAGED = false, typename Wait = int>
__device__ __forceinline__ void wsum_tile(const PlanConst& pc, const float4* ctl,
                                          const typename NoiseT<BF16>::type* __restrict__ z, const float* w, int kt,
                                          int t0, int kt_size, double* du_part, const float* wt = nullptr,
                                          Wait wait_tile = 0) {
    static_assert(TT >= 1 && TT <= WS_TT, "step tile");
    __shared__ float red[8][TT][2];
    const int K = pc.K, T = pc.T;
    const int t1 = min(T, t0 + TT);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float wj[WS_J];
    int kj[WS_J];
#pragma unroll
    for (int j = 0; j < WS_J; ++j) {
        kj[j] = kt * kt_size + j * blockDim.x + threadIdx.x;
        wj[j] = kj[j] < K ? w[kj[j]] : 0.0f;
    }
    for (int t = t0; t < t1; ++t) {
        const float4 ct = ctl[t];
        if constexpr (STAGED) wait_tile(t - t0);
        float aa = 0.0f, ad = 0.0f;
        if (CTG) {                 // cost-to-go form: weights of this step
#pragma unroll
            for (int j = 0; j < WS_J; ++j) wj[j] = kj[j] < K ? wt[(size_t)t * K + kj[j]] : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < WS_J; ++j) {
            if (kj[j] < K) {
                float2 zz;
                if constexpr (STAGED)
                    zz = noise_value<BF16>(z[(t - t0) * kt_size + j * blockDim.x + threadIdx.x]);
                else
                    zz = load_last<BF16>(z + (size_t)t * K + kj[j]);
                const Perturbed pe =
                    perturb(ct.x, ct.y, zz, pc.sig_a, pc.sig_d, pc.amin, pc.amax, pc.dmin, pc.dmax);
                aa = fmaf(wj[j], pe.ea, aa);
                ad = fmaf(wj[j], pe.ed, ad);
            }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            aa += __shfl_xor_sync(0xffffffffu, aa, o);
            ad += __shfl_xor_sync(0xffffffffu, ad, o);
        }
        if (lane == 0) {
            red[warp][t - t0][0] = aa;
            red[warp][t - t0][1] = ad;
        }
    }
    __syncthreads();
    const int nw = blockDim.x >> 5;
    for (int i = threadIdx.x; i < (t1 - t0) * 2; i += blockDim.x) {
        double s = 0.0;
        for (int wi = 0; wi < nw; ++wi) s += (double)red[wi][i >> 1][i & 1];
        du_part[((size_t)kt * T + t0 + (i >> 1)) * 2 + (i & 1)] = s;
    }
    __syncthreads();
}

// -----------------------------------------------------------------------------
// finalize: u <- clamp(u + du), u* = clamp(SG(u)), x* = F-rollout of u*, warm start.
// One block with blockDim.x >= T (every launch gives T rounded up to a warp, or 1024), so a
// thread holds at most two of the 2T control entries and at most one step.  x* is a chain
// of prefix sums: v_t from sum a dt, yaw from sum v tan(delta)/L dt, x and y from sum
// v (cos, sin) dt; with the speed cap v_{t+1} is a clamp of v_t and one thread steps the
// speeds through, the other sums stay scans.  The sums run in binary64; tan, sin and cos
// are taken in binary32 (relative error a few 1e-8 per term, far below the rollouts' own
// rounding).  binary64 arithmetic is scarce on this part (a few lanes per SM and clock),
// so divisions are replaced by products with reciprocals formed once (1 / eta, 1 / 35,
// 1 / dt, dt / L): each such product is within an ulp of the quotient.
// -----------------------------------------------------------------------------
// The device record into a host-mapped mirror (16-byte words), so a host-buffer iteration needs
// no copy back of its status.
__device__ __forceinline__ void copy_state(const DevState* st, DevState* out) {
    if (!out) return;
    const ulonglong2* src = reinterpret_cast<const ulonglong2*>(st);
    ulonglong2* dst = reinterpret_cast<ulonglong2*>(out);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(DevState) / 16); ++i) dst[i] = src[i];
}

__device__ __forceinline__ void finalize_block(const PlanConst& pc, const PlanBuffers& b, const PlanInputs& in) {
    __shared__ double s_un[2 * 1024];
    __shared__ double s_us[2 * 1024];
    __shared__ double s_v[1024 + 1];
    __shared__ double2 s_scan2[32];
    __shared__ double s_scan[32];
    __shared__ double s_eta, s_inv_eta;
    __shared__ int s_status;
    DevState* st = b.state;
    const int T = pc.T;
    const int t = threadIdx.x, bd = blockDim.x;
    const int nwa = (T + 31) >> 5;                 // warps that hold steps
    const bool ctg = pc.cost_to_go != 0;

    // this thread's control entries i0 = t and i1 = t + bd: their nominal values and the sums
    // over the k-tiles of the weighted noise (k-tile order), all loads issued up front
    const int i0 = t, i1 = t + bd;
    const bool h0 = i0 < 2 * T, h1 = i1 < 2 * T;
    const double U0 = h0 ? b.U[i0] : 0.0, U1 = h1 ? b.U[i1] : 0.0;
    double n0 = 0.0, n1 = 0.0;
    if (b.du) {                                    // already summed by the weighted-sum kernel
        if (h0) n0 = b.du[i0];
        if (h1) n1 = b.du[i1];
    } else {
        const double* dp = b.du_part;
        const size_t stride = 2 * (size_t)T;
        int kt = 0;
        for (; kt + 16 <= b.n_kt; kt += 16) {
            double a0[16], a1[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                a0[j] = h0 ? dp[(size_t)(kt + j) * stride + i0] : 0.0;
                a1[j] = h1 ? dp[(size_t)(kt + j) * stride + i1] : 0.0;
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                n0 += a0[j];
                n1 += a1[j];
            }
        }
        for (; kt < b.n_kt; ++kt) {
            if (h0) n0 += dp[(size_t)kt * stride + i0];
            if (h1) n1 += dp[(size_t)kt * stride + i1];
        }
    }
    {
        // eta: the per-block partial sums of the weights kernel, reduced by the whole block
        double e = 0.0;
        for (int i = t; i < b.n_wblk; i += bd) e += b.eta_part[i];
        e = block_sum_d(e);
        if (t == 0) {
            const int flags = st->flags, nf = st->n_finite;
            s_status = (flags & FLAG_NONFINITE_INPUT) ? -1 : (flags & FLAG_TIMEOUT) ? -5 : nf == 0 ? -4 : 0;
            s_eta = ctg ? b.eta_t[0] : e;     // cost-to-go form: reported eta of step 0
            s_inv_eta = 1.0 / e;
        }
    }
    __syncthreads();
    if (t == 0 && b.fix_count) *b.fix_count = 0u;    // the bf16 fix-up list of the next iteration's noise
    if (s_status != 0) {
        if (t == 0) {
            st->status = s_status;
            st->flags = 0;
            st->moving = 0;
            st->multi_head = 0;
            st->jkey = ~0ull;
            copy_state(st, in.state_out);
        }
        return;
    }
    const double eta = s_eta, inv_eta = s_inv_eta;
    const int ch = t & 1;                          // bd is a multiple of 32: i0 and i1 share the channel
    const double lo = ch ? pc.dmin_d : pc.amin_d, hi = ch ? pc.dmax_d : pc.amax_d;
    if (h0) s_un[i0] = clampd(U0 + (ctg ? n0 / b.eta_t[i0 >> 1] : n0 * inv_eta), lo, hi);
    if (h1) s_un[i1] = clampd(U1 + (ctg ? n1 / b.eta_t[i1 >> 1] : n1 * inv_eta), lo, hi);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int i = r ? i1 : i0;
        if (!(r ? h1 : h0)) continue;
        const int tt = i >> 1;
        double val;
        if (pc.sg_enable) {
            const double cf[5] = {-3.0, 12.0, 17.0, 12.0, -3.0};
            double acc = 0.0;
#pragma unroll
            for (int j = -2; j <= 2; ++j) {
                const int s = min(max(tt + j, 0), T - 1);
                acc += cf[j + 2] * s_un[2 * s + ch];
            }
            val = clampd(acc * (1.0 / 35.0), lo, hi);
        } else {
            val = s_un[i];
        }
        s_us[i] = val;
        in.u_out[i] = val;
    }
    __syncthreads();

    // x*.  Model 1 carries the steering angle as a fifth state: delta_t = delta_0 + sum of omega dt.
    const bool m1 = pc.model == 1;
    const int nx = m1 ? 5 : 4;
    const double x0 = in.x0[0], y0 = in.x0[1], th0 = in.x0[2], v0 = in.x0[3], d0 = m1 ? in.x0[4] : 0.0;
    if (t == 0) {
        in.x_out[0] = x0; in.x_out[1] = y0; in.x_out[2] = th0; in.x_out[3] = v0;
        if (m1) in.x_out[4] = d0;
    }
    const double dt = pc.dt_d;
    const bool on = t < T;
    const double a = on ? s_us[2 * t] : 0.0, dl = on ? s_us[2 * t + 1] : 0.0;
    double2 p1 = make_double2(0.0, 0.0);           // (v_{t+1} - v0 without the cap, delta_{t+1} - delta0)
    if (!pc.vcap || m1)
        p1 = block_scan2_incl(make_double2(on && !pc.vcap ? a * dt : 0.0, on && m1 ? dl * dt : 0.0), s_scan2, nwa);
    double vt, vn;                                  // v_t and v_{t+1}
    if (pc.vcap) {
        if (t == 0) {
            double v = v0;
            for (int s = 0; s < T; ++s) {
                double as = s_us[2 * s];
                const double lim = (pc.v_max_d - v) * pc.inv_dt_d;
                if (as > lim) as = lim;
                if (as < pc.amin_d) as = pc.amin_d;
                s_v[s] = v;
                v = v + as * dt;
            }
            s_v[T] = v;
        }
        __syncthreads();
        vt = on ? s_v[t] : 0.0;
        vn = on ? s_v[t + 1] : 0.0;
    } else {
        vt = v0 + (p1.x - (on ? a * dt : 0.0));
        vn = v0 + p1.x;
    }
    double steer = dl;
    if (m1) steer = d0 + (p1.y - (on ? dl * dt : 0.0));                     // delta_t
    const double dth = on ? vt * (double)tanf((float)steer) * pc.dt_over_wb_d : 0.0;
    const double pth = block_scan_incl(dth, s_scan, nwa);                    // yaw_{t+1} - yaw0
    const double tht = th0 + (pth - dth);                                    // yaw_t
    float sn = 0.0f, cs = 0.0f;
    if (on) sincosf((float)tht, &sn, &cs);
    const double2 pxy = block_scan2_incl(make_double2(on ? vt * (double)cs * dt : 0.0, on ? vt * (double)sn * dt : 0.0),
                                         s_scan2, nwa);
    if (on) {
        double* o = in.x_out + (size_t)nx * (t + 1);
        o[0] = x0 + pxy.x;
        o[1] = y0 + pxy.y;
        o[2] = th0 + pth;
        o[3] = vn;
        if (m1) o[4] = d0 + p1.y;
    }
    // warm start for the next iteration (Algorithm 1, last loop)
    for (int i = t; i < 2 * T; i += bd) {
        const int tt = i >> 1, c = i & 1;
        const int src = pc.shift ? min(tt + 1, T - 1) : tt;
        b.U[i] = s_us[2 * src + c];
    }
    if (t == 0) {
        st->status = 0;
        st->eta = eta;
        st->iter_used = st->iter;
        st->iter += 1ull;
        st->flags = 0;
        st->moving = 0;
        st->multi_head = 0;
        st->jkey = ~0ull;
        copy_state(st, in.state_out);
    }
}


}  // namespace mppi
