// Shared device/host helpers of libpp (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#ifndef PP_NO_NVTX
#include <nvtx3/nvToolsExt.h>
#endif

#include "../../include/pagerank_pipeline.h"

// One device error word per translation unit (each .cu file gets its own
// copy); pp_last_device_error() reads and clears all of them.
static __device__ uint32_t pp_err_word;
static __device__ __forceinline__ void pp_set_error(uint32_t bits) { atomicOr(&pp_err_word, bits); }

// Index checks of the checked build (-DPP_CHECKED, libpp_checked.so).
// pp_idx(i, n) wraps every index that a kernel read from memory or computed
// from what it read, n being the length of the array addressed: it is i when
// i < n; otherwise it records PP_DEV_BOUNDS and gives 0, so that the access
// stays inside the array (the result is then invalid; nothing traps).  In the
// normal build it is i itself.
template <typename I, typename N>
static __device__ __forceinline__ I pp_idx(I i, N n) {
#ifdef PP_CHECKED
    if ((unsigned long long)i < (unsigned long long)n) return i;
    pp_set_error(PP_DEV_BOUNDS);
    return I(0);
#else
    (void)n;
    return i;
#endif
}
// pp_idx for an index that is only used when `on` holds (0 otherwise when checked).
template <typename I, typename N>
static __device__ __forceinline__ I pp_idx_if(bool on, I i, N n) {
#ifdef PP_CHECKED
    return on ? pp_idx(i, n) : I(0);
#else
    (void)on;
    (void)n;
    return i;
#endif
}
// A run of `len` items of `unit` elements from element `start` of an array
// of n: len when it fits; otherwise PP_DEV_BOUNDS and 0 (checked build).
template <typename L>
static __device__ __forceinline__ L pp_len(unsigned long long start, L len, unsigned long long n,
                                           unsigned long long unit = 1) {
#ifdef PP_CHECKED
    if (start <= n && (unsigned long long)len * unit <= n - start) return len;
    pp_set_error(PP_DEV_BOUNDS);
    return L(0);
#else
    (void)start;
    (void)n;
    (void)unit;
    return len;
#endif
}

namespace pp {

// ------------------------------------------------------------------ host side

// An NVTX range around one C-ABI call, named after the call: profilers show
// the call on their timeline and can select its kernels (ncu --nvtx
// --nvtx-include "pp_pagerank/").  Without an attached tool a push and a pop
// cost a few nanoseconds; -DPP_NO_NVTX leaves them out.
struct Range {
#ifndef PP_NO_NVTX
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
#else
    explicit Range(const char *) {}
#endif
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};
#define PP_RANGE(name) ::pp::Range pp_call_range_(name)

// Host-side fault injection (pp_inject_fault): true, with the status to
// return, when a failure is armed for the entry point `name`.  One relaxed
// load when nothing is armed.
extern std::atomic<int> g_faults_armed;
bool fault_hit(const char *name, pp_status *st);

// The first statement of every entry point that enqueues work: its NVTX
// range, then an armed failure returned before anything is checked or run.
#define PP_ENTRY(name)                                                                      \
    PP_RANGE(name);                                                                         \
    do {                                                                                    \
        pp_status pp_fault_st_;                                                             \
        if (::pp::g_faults_armed.load(std::memory_order_relaxed) && ::pp::fault_hit(name, &pp_fault_st_)) \
            return pp_fault_st_;                                                            \
    } while (0)

// Number of kernels enqueued by the library (pp_launch_count).
extern std::atomic<uint64_t> g_launches;

inline void count_launch(uint64_t n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Current value of a tuning knob (pp_set_tuning); defaults live in pp_api.cu.
int64_t tuning(const char *key);

constexpr int kMaxDevices = 64;

inline int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

// A launch setting computed once per device by f() (nonzero result): function
// attributes such as the shared-memory carveout are set per device, and the
// occupancy they give may differ between devices.  Threads that race compute
// the same value.
struct PerDevice {
    std::atomic<int64_t> v[kMaxDevices];
    template <typename F>
    int64_t get(F f) {
        const int d = current_device();
        if (d < 0 || d >= kMaxDevices) return f();
        int64_t x = v[d].load(std::memory_order_acquire);
        if (!x) {
            x = f();
            v[d].store(x, std::memory_order_release);
        }
        return x;
    }
};

inline int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

// Carves 256-byte aligned sub-buffers out of one workspace.  With base ==
// nullptr it only measures, so the size query and the carve share one layout.
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base(static_cast<char *>(b)) {}
    template <typename T>
    T *take(uint64_t count) {
        off = (off + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += size_t(count) * sizeof(T);
        return p;
    }
    size_t size() const { return (off + 255) & ~size_t(255); }
};

inline pp_status check_ws(void *ws, size_t have, size_t need) {
    if (need == 0) return PP_OK;
    if (!ws || have < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return PP_ERR_WORKSPACE;
    return PP_OK;
}

inline pp_status launch_status() {
    return cudaGetLastError() == cudaSuccess ? PP_OK : PP_ERR_CUDA;
}

// Longest poll of a cross-block wait before the kernel gives up and records
// PP_DEV_TIMEOUT (about a second at 2 GHz with the back-off below).
constexpr uint32_t kSpinLimit = 1u << 22;

// ---------------------------------------------------------------- device side

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// L2 eviction-priority policies (createpolicy) and loads/stores that carry
// them: streams read once are marked evict-first so they do not push out the
// data that is gathered over and over (marked evict-last).
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint32_t ld_stream_u32(const uint32_t *ptr, uint64_t pol) {
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ float ld_hint(const float *ptr, uint64_t pol) {
    float v;
    asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ double ld_hint(const double *ptr, uint64_t pol) {
    double v;
    asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ float4 ld_hint4(const float *ptr, uint64_t pol) {  // 16-byte aligned
    float4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ unsigned short ld_hint_b16(const void *ptr, uint64_t pol) {
    unsigned short v;
    asm volatile("ld.global.nc.L2::cache_hint.b16 %0, [%1], %2;" : "=h"(v) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_hint(float *ptr, float v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(ptr), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint(double *ptr, double v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(ptr), "d"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint_b16(void *ptr, unsigned short v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.b16 [%0], %1, %2;" ::"l"(ptr), "h"(v), "l"(pol) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ void backoff(uint32_t spin) {
    if (spin > 64) __nanosleep(spin > 4096 ? 256 : 32);
}

// Inclusive warp scan (sum).
template <typename T>
__device__ __forceinline__ T warp_inclusive_sum(T x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive block scan (sum) of one value per thread; returns the exclusive
// prefix and writes the block total to *total.  `scratch` holds >= 32 T.
template <typename T, int THREADS>
__device__ __forceinline__ T block_exclusive_sum(T x, T *scratch, T *total) {
    constexpr int W = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = warp_inclusive_sum(x);
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < W ? scratch[lane] : T(0);
        T wi = warp_inclusive_sum(w);
        if (lane < W) scratch[lane] = wi - w;
        if (lane == W - 1) scratch[W] = wi;
    }
    __syncthreads();
    T r = scratch[warp] + inc - x;
    *total = scratch[W];
    __syncthreads();
    return r;
}

// Block-wide sum with a fixed reduction tree (deterministic for floats).
template <typename T, int THREADS>
__device__ __forceinline__ T block_sum(T x, T *scratch) {
    constexpr int W = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) scratch[warp] = x;
    __syncthreads();
    T r = T(0);
    if (warp == 0) {
        r = lane < W ? scratch[lane] : T(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;  // valid in thread 0
}

// Decoupled look-back by one whole warp over 64-bit status words (flags in
// bits 63:62: 1 = aggregate of that tile only, 2 = inclusive prefix; the sum
// in bits 61:0).  Lane k reads the word of tile `tile - 1 - k`, so one round
// trip covers 32 predecessors; the walk stops at the nearest inclusive word.
// Returns the exclusive prefix of `tile` in every lane.  Waits are bounded:
// after kSpinLimit empty polls the device error word gets PP_DEV_TIMEOUT.
__device__ __forceinline__ uint64_t warp_lookback(const uint64_t *status, uint64_t tile) {
    constexpr uint64_t INC = 2ull << 62, ANY = 3ull << 62;
    const int lane = threadIdx.x & 31;
    uint64_t excl = 0;
    long long p = (long long)tile - 1;
    uint32_t spins = 0;
    while (p >= 0) {
        const long long q = p - lane;
        const uint64_t s = q >= 0 ? ld_relaxed_u64(status + q) : INC;  // tile 0 is always inclusive
        const uint32_t nready = __ballot_sync(0xffffffffu, (s & ANY) == 0);
        const uint32_t inc = __ballot_sync(0xffffffffu, (s & INC) != 0 && (s & ANY) != 0);
        const int first_nr = nready ? __ffs(nready) - 1 : 32;
        const int first_inc = inc ? __ffs(inc) - 1 : 32;
        const int take = first_inc < first_nr ? first_inc + 1 : first_nr;  // lanes 0 .. take-1
        uint64_t v = lane < take ? (s & ~ANY) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (first_inc < first_nr) break;
        p -= take;
        if (take == 0) {
            if (++spins > kSpinLimit) {
                if (lane == 0) pp_set_error(PP_DEV_TIMEOUT);
                break;
            }
            backoff(spins);
        }
    }
    return excl;
}

}  // namespace pp

// Host accessor of this translation unit's device error word.
#define PP_DEFINE_ERROR_WORD(fetch_fn)                                                  \
    namespace pp {                                                                      \
    uint32_t fetch_fn(cudaStream_t s) {                                                 \
        uint32_t v = 0, z = 0;                                                          \
        if (cudaMemcpyFromSymbolAsync(&v, pp_err_word, sizeof v, 0,                     \
                                      cudaMemcpyDeviceToHost, s) != cudaSuccess)        \
            return 0xffffffffu;                                                         \
        if (cudaMemcpyToSymbolAsync(pp_err_word, &z, sizeof z, 0,                       \
                                    cudaMemcpyHostToDevice, s) != cudaSuccess)          \
            return 0xffffffffu;                                                         \
        if (cudaStreamSynchronize(s) != cudaSuccess) return 0xffffffffu;                \
        return v;                                                                       \
    }                                                                                   \
    }
