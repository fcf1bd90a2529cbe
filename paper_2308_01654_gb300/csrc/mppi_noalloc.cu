// mppi_noalloc.cu - the allocation-free entry point mppi_argmin_noalloc().
//
// Some callers cannot call cudaMalloc at the time they plan: a vehicle's control cycle
// that must not stall (cudaMalloc may synchronise the device and can fail under memory
// pressure), or code that may only use memory reserved when the program started.  For
// them the lowest-cost search over the sample costs (the argmin step of the iteration)
// is offered without any allocation: its scratch lives in a fixed array in this file,
// reserved on every GPU that loads the library until the process exits.
#include <mutex>

#include "mppi.h"
#include "mppi_device.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = 1024;

struct __align__(16) ArgminScratch {
    double v[NA_MAX_BLOCKS];   // per-block lowest cost
    int i[NA_MAX_BLOCKS];      // its index
    int n[NA_MAX_BLOCKS];      // finite costs seen by the block
    unsigned int ticket;       // blocks finished; must start at zero
};

// The scratch: 16 KB + 16 B, shared by every call on a device.
static __device__ __align__(256) unsigned char g_argmin_scratch[sizeof(ArgminScratch)];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[MAX_DEVICES] = {};

struct Rec {
    double v;
    int i;
    int n;
};

__device__ __forceinline__ Rec combine(Rec a, Rec b) {
    Rec r;
    r.n = a.n + b.n;
    const bool take_b = b.v < a.v || (b.v == a.v && b.i < a.i);
    r.v = take_b ? b.v : a.v;
    r.i = take_b ? b.i : a.i;
    return r;
}

__device__ Rec block_reduce(Rec a) {
    __shared__ double sv[32];
    __shared__ int si[32], sn[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        Rec b{__shfl_xor_sync(0xffffffffu, a.v, o), __shfl_xor_sync(0xffffffffu, a.i, o),
              __shfl_xor_sync(0xffffffffu, a.n, o)};
        a = combine(a, b);
    }
    if (lane == 0) {
        sv[w] = a.v;
        si[w] = a.i;
        sn[w] = a.n;
    }
    __syncthreads();
    if (w == 0) {
        a = lane < nw ? Rec{sv[lane], si[lane], sn[lane]} : Rec{INFINITY, 0x7fffffff, 0};
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            Rec b{__shfl_xor_sync(0xffffffffu, a.v, o), __shfl_xor_sync(0xffffffffu, a.i, o),
                  __shfl_xor_sync(0xffffffffu, a.n, o)};
            a = combine(a, b);
        }
    }
    __syncthreads();
    return a;
}

// Lowest finite cost and its index (ties -> lowest index), with the count of finite costs.
// The blocks write their partial results into the scratch; the last block to finish
// (ticket) combines them and writes the outputs.
__global__ void __launch_bounds__(NA_THREADS) argmin_noalloc_kernel(const double* __restrict__ S, int K,
                                                                    ArgminScratch* sc, double* s_min,
                                                                    int32_t* argmin, int32_t* n_finite) {
    Rec r{INFINITY, 0x7fffffff, 0};
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
        const double s = S[k];
        if (isfinite(s)) {
            r.n += 1;
            if (s < r.v) {
                r.v = s;
                r.i = k;
            }
        }
    }
    r = block_reduce(r);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        sc->v[blockIdx.x] = r.v;
        sc->i[blockIdx.x] = r.i;
        sc->n[blockIdx.x] = r.n;
        __threadfence();
        last = atomicAdd(&sc->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    Rec q{INFINITY, 0x7fffffff, 0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
        q = combine(q, Rec{((volatile double*)sc->v)[b], ((volatile int*)sc->i)[b], ((volatile int*)sc->n)[b]});
    q = block_reduce(q);
    if (threadIdx.x == 0) {
        *s_min = q.v;
        *argmin = q.n > 0 ? q.i : -1;
        *n_finite = q.n;
        sc->ticket = 0u;
    }
}

}  // namespace

extern "C" int mppi_argmin_noalloc(const double* d_S, int32_t K, double* d_s_min, int32_t* d_argmin,
                                   int32_t* d_n_finite, void* cuda_stream) {
    if (!d_S || !d_s_min || !d_argmin || !d_n_finite) return MPPI_ERR_ARG;
    if (K < 1) return MPPI_ERR_ARG;
    if (K > MPPI_NOALLOC_MAX_K) return MPPI_ERR_CAPACITY;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return MPPI_ERR_CUDA;
    void* addr = nullptr;
    {
        // one-time set-up per device: the device address of the scratch array (the array's
        // name is only a host-side stand-in and must not be passed to a kernel)
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_argmin_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return MPPI_ERR_CUDA;
            }
            g_scratch_addr[dev] = p;
        }
        addr = g_scratch_addr[dev];
    }
    ArgminScratch* sc = static_cast<ArgminScratch*>(addr);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // the ticket must start at zero whatever an earlier call left behind
    if (cudaMemsetAsync(&sc->ticket, 0, sizeof(unsigned int), st) != cudaSuccess) return MPPI_ERR_CUDA;
    const long long want = ((long long)K + NA_THREADS - 1) / NA_THREADS;
    const int blocks = (int)(want < NA_MAX_BLOCKS ? want : NA_MAX_BLOCKS);
    argmin_noalloc_kernel<<<blocks, NA_THREADS, 0, st>>>(d_S, K, sc, d_s_min, d_argmin, d_n_finite);
    if (cudaGetLastError() != cudaSuccess) return MPPI_ERR_CUDA;
    return MPPI_OK;
}
