// mppi_device.cuh - device math of the MPPI iteration (arXiv 2308.01654), sm_103a.
//
// Shared by the noise, rollout and update kernels so that each quantity that two
// kernels must agree on (the noise words, the clamped perturbation eps') comes
// from one function and is bit-identical wherever it is recomputed.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mppi {

// Chunking of the reference polyline for the exact bounded nearest-segment search:
// level-1 chunks of L1 segments, level-2 groups of L2 level-1 chunks.
constexpr int REF_L1 = 4;
constexpr int REF_L2 = 16;

// Tiles of the weighted noise sum (Eq. 11): WS_J samples per thread (256 threads, so
// 256 * WS_J samples per k-tile) and WS_TT steps per tile.
constexpr int WS_J = 8;
constexpr int WS_TT = 8;

// Status bits raised on the device (DevState::flags).
constexpr int FLAG_NONFINITE_INPUT = 1;
constexpr int FLAG_TIMEOUT = 2;

// -----------------------------------------------------------------------------
// Bounds-checking debug build (compiled with MPPI_CHECKS): IX(i, n) tests an index against
// the length of the array it reads; one outside [0, n) is counted and replaced by 0, so the
// access stays inside the array and nothing traps.  The normal build compiles IX to the index.
// -----------------------------------------------------------------------------
#ifdef MPPI_CHECKS
static __device__ unsigned long long g_check_hits;   // one counter per translation unit
__device__ __forceinline__ int checked_index(long long i, long long n) {
    if (i >= 0 && i < n) return (int)i;
    atomicAdd(&g_check_hits, 1ull);
    return 0;
}
#define IX(i, n) ::mppi::checked_index((long long)(i), (long long)(n))
#else
#define IX(i, n) (i)
#endif

// -----------------------------------------------------------------------------
// Programmatic dependent launch.  The kernels of an iteration after the first are launched
// with programmatic stream serialisation: a kernel may be scheduled while its predecessor
// drains, and waits here (griddepcontrol.wait: until the predecessor grid has completed and
// its memory operations are visible) before it reads anything.  Every chained kernel waits
// before its first dependent access, so grids still complete strictly in stream order.
// pdl_trigger lets the next kernel be scheduled before this one ends; single-wave kernels
// call it, kernels with many waves leave it to their exit so the next kernel's blocks do not
// take SM space from their later waves.  Without the launch attribute both return at once.
// -----------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// -----------------------------------------------------------------------------
// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11):
// ten rounds of two 32x32->64 multiplications whose halves are XORed with the
// other two counter words and the round key; the key advances by the Weyl
// increments between rounds.  Noise of sample k at steps 2j and 2j+1 uses the
// counter (j, k, iter, session) with key (seed low, seed high).
// -----------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = mulhi32(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = mulhi32(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Uniform in (0, 1): the top 24 bits forced odd, times 2^-24 (exact in binary32).
__device__ __forceinline__ float uniform24(uint32_t w) {
    return (float)((w >> 8) | 1u) * 0x1p-24f;
}

// Box-Muller in binary32: sqrt(-2 ln u0) * (cos, sin)(2 pi u1).
__device__ __forceinline__ float2 box_muller(float u0, float u1) {
    const float r = sqrtf(-2.0f * logf(u0));
    float s, c;
    sincospif(2.0f * u1, &s, &c);
    return make_float2(r * c, r * s);
}

// Box-Muller in binary64 (the slow path of the bfloat16 store).
__device__ __forceinline__ double2 box_muller_f64(float u0, float u1) {
    const double r = sqrt(-2.0 * log((double)u0));
    double s, c;
    sincospi(2.0 * (double)u1, &s, &c);
    return make_double2(r * c, r * s);
}

// Round a binary64 value to the nearest bfloat16 (8 significant bits, ties to even)
// in one step: add half of the dropped 45-bit field (plus the kept LSB for ties) and
// truncate; the result has 8 significant bits, so the final conversion is exact.
__device__ __forceinline__ __nv_bfloat16 bf16_from_f64(double z) {
    unsigned long long b = (unsigned long long)__double_as_longlong(z);
    const unsigned long long lsb = (b >> 45) & 1ull;
    b += 0x0FFFFFFFFFFFull + lsb;
    b &= ~0x1FFFFFFFFFFFull;
    return __float2bfloat16_rn((float)__longlong_as_double((long long)b));
}

// True when a binary32 normal may sit on the other side of a bfloat16 rounding midpoint than
// the exact normal: within the binary32 Box-Muller error bound of the midpoint.  That bound is
// relative (u = 2^-24): logf is within 1 ulp (2u relative) and the scaling by -2 is exact;
// sqrtf halves that (u) and rounds (u); sincospif is within 1 ulp (2u) of an exact argument,
// so relatively also next to its zeros; the product rounds (u).  In all |z - z_exact| <= 5u |z|
// ~ 2.98e-7 |z| to first order, and the window is 3.2e-7 |z|.  (|z| is never below ~1e-10:
// u0 <= 1 - 2^-24, and the sine and cosine of pi times an odd multiple of 2^-23 exceed 3e-7.)
__device__ __forceinline__ bool near_bf16_midpoint(float z) {
    const float mid = __uint_as_float((__float_as_uint(z) & 0xFFFF0000u) | 0x8000u);
    return fabsf(z - mid) <= 3.2e-7f * fabsf(z);
}

// -----------------------------------------------------------------------------
// Noise storage: [T][K] of (z_a, z_delta), binary32 pairs or bfloat16 pairs.
// -----------------------------------------------------------------------------
template <bool BF16> struct NoiseT;
template <> struct NoiseT<false> {
    using type = float2;
    __device__ __forceinline__ static float2 load(const type* p) { return __ldg(p); }
    __device__ __forceinline__ static type pack(float2 z) { return z; }
};
template <> struct NoiseT<true> {
    using type = __nv_bfloat162;
    __device__ __forceinline__ static float2 load(const type* p) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
    }
    __device__ __forceinline__ static type pack(float2 z) { return __floats2bfloat162_rn(z.x, z.y); }
};

// -----------------------------------------------------------------------------
// L2 residency of the noise.  z is written once and read twice (rollout, then weighted sum);
// it is smaller than L2 but, stored with the default policy, about half of it is evicted before
// the second read.  The noise kernel stores it with an evict-last policy and the weighted sum,
// its last reader, loads it as streaming data.
// -----------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long l2_keep_policy() {
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void store_keep(float2* p, float2 v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y), "l"(pol)
                 : "memory");
}

__device__ __forceinline__ void store_keep(__nv_bfloat162* p, __nv_bfloat162 v, unsigned long long pol) {
    const unsigned bits = *reinterpret_cast<const unsigned*>(&v);
    asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(p), "r"(bits), "l"(pol) : "memory");
}

// a noise value already in registers or shared memory, as binary32
template <bool BF16>
__device__ __forceinline__ float2 noise_value(typename NoiseT<BF16>::type v) {
    if constexpr (BF16) return __bfloat1622float2(v);
    else return v;
}

// last read of the noise: streaming load
template <bool BF16>
__device__ __forceinline__ float2 load_last(const typename NoiseT<BF16>::type* p) {
    if constexpr (BF16) {
        const unsigned bits = __ldcs(reinterpret_cast<const unsigned*>(p));
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&bits));
    } else {
        return __ldcs(p);
    }
}

// -----------------------------------------------------------------------------
// Control perturbation with the noise check of Sec. III-A: v = clamp(u + sigma z)
// and eps' = v - u.  Written with explicit rounding so the rollout and the update
// kernels produce the same bits.
// -----------------------------------------------------------------------------
struct Perturbed {
    float va, vd;    // applied controls
    float ea, ed;    // eps' = applied - nominal
};

__device__ __forceinline__ Perturbed perturb(float ua, float ud, float2 z, float sa, float sd,
                                             float amin, float amax, float dmin, float dmax) {
    Perturbed p;
    p.va = fminf(fmaxf(__fmaf_rn(sa, z.x, ua), amin), amax);
    p.vd = fminf(fmaxf(__fmaf_rn(sd, z.y, ud), dmin), dmax);
    p.ea = __fsub_rn(p.va, ua);
    p.ed = __fsub_rn(p.vd, ud);
    return p;
}

// yaw error wrapped into [-pi, pi]: d - 2 pi rint(d / 2 pi)
__device__ __forceinline__ float wrap_pi(float d) {
    const float k = rintf(d * 0.15915494309189535f);
    return fmaf(-6.283185307179586f, k, d);
}

// Squared distance from p to the segment from a along e, s = (ex, ey, ex/|e|^2, ey/|e|^2):
// the projection parameter is clamped to [0, 1] and d = (p - a) - tau e.  (Whether the
// clamped end equals the next vertex bit for bit does not matter here: ties between two
// segments that share a vertex are settled in binary64, see nearest_segment.)
__device__ __forceinline__ float seg_dist2(float px, float py, float2 a, float4 s) {
    const float dax = px - a.x, day = py - a.y;
    const float tau = __saturatef(fmaf(dax, s.z, day * s.w));
    const float dx = fmaf(-tau, s.x, dax), dy = fmaf(-tau, s.y, day);
    return fmaf(dx, dx, dy * dy);
}

// The same distance in binary64 from the binary32 inputs: used to settle near ties
// between two segments, where the two binary32 distances cannot be ordered (next to a
// vertex on the outside of a bend the gap is second order in the offset).
__device__ __forceinline__ double seg_dist2_f64(float px, float py, float2 a, float2 b) {
    const double ax = a.x, ay = a.y, ex = (double)b.x - ax, ey = (double)b.y - ay;
    const double dax = (double)px - ax, day = (double)py - ay;
    const double l2 = ex * ex + ey * ey;
    const double tau = l2 > 0.0 ? (dax * ex + day * ey) / l2 : 0.0;
    double qx, qy;
    if (tau <= 0.0) {
        qx = ax; qy = ay;
    } else if (tau >= 1.0) {
        qx = b.x; qy = b.y;
    } else {
        qx = ax + tau * ex;
        qy = ay + tau * ey;
    }
    const double dx = (double)px - qx, dy = (double)py - qy;
    return dx * dx + dy * dy;
}

// Squared distance from p to an axis-aligned box (minx, miny, maxx, maxy).
__device__ __forceinline__ float box_dist2(float px, float py, float4 bb) {
    const float dx = fmaxf(fmaxf(bb.x - px, px - bb.z), 0.0f);
    const float dy = fmaxf(fmaxf(bb.y - py, py - bb.w), 0.0f);
    return fmaf(dx, dx, dy * dy);
}

}  // namespace mppi
