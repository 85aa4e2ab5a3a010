// Stable LSD radix sort, one scatter pass per 8-bit digit.
//
// The scheme follows the published Onesweep method (Adinets & Merrill,
// "Onesweep: A Faster Least Significant Digit Radix Sort for GPUs", 2022):
// an up-front pass counts the digits of every pass at once; each scatter pass
// then takes tiles in the order blocks start, ranks the tile's keys with a
// warp-level multisplit into warp-private shared-memory counters, publishes
// the tile's per-digit counts, stages the keys in shared memory in digit
// order, and only then finds its global offset per digit by a decoupled
// look-back over earlier tiles' published counts, so the staging overlaps
// the wait; each digit's run is written to global memory with consecutive
// addresses.  The multisplit finds the lanes of a warp holding equal digits
// with one warp vote per digit bit (eight votes are cheaper on this GPU than
// one match.any).
//
// Look-back waits poll with a bound (kSpinLimit): a wait that expires records
// PP_DEV_TIMEOUT in the device error word and the kernel carries on, so no
// launch can hang.  A tile only ever waits for tiles that earlier-started
// blocks already own, so the bound is never reached in a correct run.
//
// Sources and sinks are small functors so that the same pass kernel packs
// (u, v) into a key on the first pass of Kernel 1 and unpacks on its last
// pass, or writes Kernel 2's permutation from its vertex keys.
#pragma once

#include <type_traits>

#include "pp_common.cuh"

namespace pp {
namespace os {

constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;
constexpr int ITEMS = 16;
constexpr int TILE = THREADS * ITEMS;
constexpr int RADIX = 256;
constexpr int MAX_PASSES = 8;
static_assert(THREADS == RADIX, "one thread per digit in the per-digit phases");

template <typename S>
struct Flags;
template <>
struct Flags<uint32_t> {
    static constexpr uint32_t AGG = 1u << 30, INC = 2u << 30, ANY = 3u << 30, VAL = (1u << 30) - 1;
};
template <>
struct Flags<uint64_t> {
    static constexpr uint64_t AGG = 1ull << 62, INC = 2ull << 62, ANY = 3ull << 62, VAL = (1ull << 62) - 1;
};

__device__ __forceinline__ uint32_t ld_status(const uint32_t *p) { return ld_relaxed_u32(p); }
__device__ __forceinline__ uint64_t ld_status(const uint64_t *p) { return ld_relaxed_u64(p); }
__device__ __forceinline__ void st_status(uint32_t *p, uint32_t v) { st_relaxed_u32(p, v); }
__device__ __forceinline__ void st_status(uint64_t *p, uint64_t v) { st_relaxed_u64(p, v); }

// Per-pass control block.
struct PassCtl {
    uint32_t shift;         // digit = (key >> shift) & 255
    const uint32_t *hist;   // [256] number of valid keys per digit in this pass
    void *status;           // [ntiles * 256] look-back words, zero on entry
    void *status_next;      // words the next pass uses, zeroed here (nullptr: none)
    uint32_t *tile_ctr;     // zero on entry
    const uint64_t *n_dev;  // element count on the device (nullptr: use n_host)
    uint64_t n_host;
    uint32_t spin_limit;    // empty polls before a look-back gives up
};

// A source with `load4(i4, k)` (four consecutive elements from i4, a multiple
// of 4) and a `vec` flag (its arrays are 16-byte aligned) is read with
// 16-byte loads where a whole tile is present.
template <class S, class = void>
struct has_load4 : std::false_type {};
template <class S>
struct has_load4<S, std::void_t<decltype(&S::load4)>> : std::true_type {};

// A source with `map(k)` has each loaded key passed through it once all of a
// thread's keys are loaded, so that a second, dependent load per key (a
// table lookup) is issued for all of them together.
template <class S, class = void>
struct has_map : std::false_type {};
template <class S>
struct has_map<S, std::void_t<decltype(&S::map)>> : std::true_type {};

// Status words are 32-bit while every count fits in 30 bits.
inline bool wide_status(uint64_t n_max) { return n_max >= (1ull << 30); }

// Blocks per SM the registers are budgeted for: four (64 registers, room for
// the digits held in registers) beat five (48 registers, the most the 42 KB of
// shared memory allows with 64-bit keys) on GB300.
constexpr int PASS_MINB = 4;

template <typename KeyT, typename StatT, class Src, class Dst>
__global__ void __launch_bounds__(THREADS, PASS_MINB) pass_kernel(Src src, Dst dst, PassCtl ctl) {
    using F = Flags<StatT>;
    __shared__ KeyT s_keys[TILE];               // the tile in input order, then in digit order
    __shared__ uint32_t s_whist[WARPS][RADIX];  // per-warp digit counters, then staging offsets
    __shared__ uint32_t s_gbase[RADIX];  // global index of the digit's first key minus its staging offset (mod 2^32)
    __shared__ uint32_t s_scan[40];
    __shared__ uint32_t s_tile;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(ctl.tile_ctr, 1u);
    for (int i = tid; i < WARPS * RADIX; i += THREADS) (&s_whist[0][0])[i] = 0;

    // Global start of each digit: exclusive scan of the pass histogram.
    uint32_t htotal;
    const uint32_t hexcl = block_exclusive_sum<uint32_t, THREADS>(ctl.hist[tid], s_scan, &htotal);

    const uint64_t n = ctl.n_dev ? *ctl.n_dev : ctl.n_host;
    const uint32_t tile = s_tile;
    const uint64_t ntiles = (n + TILE - 1) / TILE;
    if (tile >= ntiles) return;
    if (ctl.status_next) static_cast<StatT *>(ctl.status_next)[(uint64_t)tile * RADIX + tid] = 0;

    // Warp-striped load: warp w owns elements [w*ITEMS*32, (w+1)*ITEMS*32) of
    // the tile; item i of a lane is element i*32 + lane of that range, so the
    // order (warp, item, lane) is the input order.
    const uint32_t wbase = (uint32_t)warp * (ITEMS * 32);
    const uint64_t base = (uint64_t)tile * TILE + wbase;
    // valid items of this lane (the tile's tail may be short)
    const uint64_t first = base + lane;
    const uint64_t left = first < n ? (n - first + 31) / 32 : 0;
    const int nv = left < (uint64_t)ITEMS ? (int)left : ITEMS;
    // the digits stay in registers, four to a word; the keys wait in shared memory
    constexpr int DW = (ITEMS + 3) / 4;
    uint32_t dig[DW];
#pragma unroll
    for (int q = 0; q < DW; ++q) dig[q] = 0;
    {
        KeyT keys[ITEMS];
        uint32_t unused;
        bool loaded = false;
        if constexpr (has_load4<Src>::value) {
            // Only the first pass reads such a source, and the first pass may take
            // its input in any fixed order (the sort's result does not depend on
            // it): item 4q + j of a lane is element 128 q + 4 lane + j of the warp's
            // range, four ids per 16-byte load.  Whole warp ranges only, so that
            // every element of a range is read by exactly one of the two layouts.
            if (src.vec && base + (uint64_t)ITEMS * 32 <= n) {
#pragma unroll
                for (int q = 0; q < ITEMS / 4; ++q) src.load4(base + 128ull * q + 4ull * lane, &keys[4 * q]);
                loaded = true;
            }
        }
        if (!loaded) {
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                keys[i] = 0;
                if (i < nv) src.load(base + (uint64_t)i * 32 + lane, keys[i], unused);
            }
        }
        if constexpr (has_map<Src>::value) {
#pragma unroll
            for (int i = 0; i < ITEMS; ++i)
                if (i < nv) keys[i] = src.map(keys[i]);
        }
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            dig[i / 4] |= ((uint32_t)(keys[i] >> ctl.shift) & (RADIX - 1)) << (8 * (i % 4));
            s_keys[wbase + i * 32 + lane] = keys[i];
        }
    }

    // Warp-level multisplit: rank of each key among equal digits of its warp,
    // kept three 10-bit ranks to a register.  The lanes holding the same digit
    // (and the same validity) are the AND of one vote per digit bit; the lowest
    // of them adds the group to the warp's counter and hands the old count to
    // the others.  Item i + 1's add is issued after item i's result has been
    // handed on, so each counter sees the items in order.
    constexpr int RW = (ITEMS + 2) / 3;
    uint32_t rank[RW];
#pragma unroll
    for (int q = 0; q < RW; ++q) rank[q] = 0;
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const bool ok = i < nv;
        const uint32_t d = (dig[i / 4] >> (8 * (i % 4))) & (RADIX - 1);
        uint32_t peers = __ballot_sync(0xffffffffu, ok);
        if (!ok) peers = ~peers;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const uint32_t m = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? m : ~m;
        }
        const int leader = __ffs(peers) - 1;
        uint32_t before = 0;
        if (lane == leader && ok) before = atomicAdd(&s_whist[warp][d], (uint32_t)__popc(peers));
        before = __shfl_sync(0xffffffffu, before, leader);
        rank[i / 3] |= (before + __popc(peers & lt)) << (10 * (i % 3));
    }
    __syncthreads();

    // Per digit (thread tid): offsets of the warps within the tile's digit run.
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) {
        const uint32_t c = s_whist[w][tid];
        s_whist[w][tid] = run;
        run += c;
    }
    const uint32_t tcount = run;
    StatT *st = static_cast<StatT *>(ctl.status);
    StatT *mine = st + (uint64_t)tile * RADIX + tid;
    st_status(mine, (tile == 0 ? F::INC : F::AGG) | (StatT)tcount);

    uint32_t nvalid;
    const uint32_t bstart = block_exclusive_sum<uint32_t, THREADS>(tcount, s_scan, &nvalid);
    // staging offset of warp w's first key of digit tid (one lookup per key below)
#pragma unroll
    for (int w = 0; w < WARPS; ++w) s_whist[w][tid] += bstart;

    // Stage the tile in digit order, in place (every key is read before any is
    // written), while earlier tiles finish publishing.
    {
        KeyT keys[ITEMS];
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) keys[i] = s_keys[wbase + i * 32 + lane];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            if (i < nv) {
                const uint32_t d = (dig[i / 4] >> (8 * (i % 4))) & (RADIX - 1);
                s_keys[pp_idx(s_whist[warp][d] + ((rank[i / 3] >> (10 * (i % 3))) & 1023u), TILE)] = keys[i];
            }
        }
    }

    // Decoupled look-back for this digit, four predecessors per round trip.
    StatT excl = 0;
    if (tile > 0) {
        long long p = (long long)tile - 1;
        uint32_t spins = 0;
        while (true) {
            StatT s4[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) s4[q] = p - q >= 0 ? ld_status(st + (uint64_t)(p - q) * RADIX + tid) : StatT(0);
            int used = 0;
            bool done = false;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (done || used != q || (s4[q] & F::ANY) == 0) continue;
                excl += s4[q] & F::VAL;
                ++used;
                if (s4[q] & F::INC) done = true;
            }
            if (done) break;
            p -= used;  // tile 0 always publishes an inclusive word, so p stays >= 0
            if (used == 0) {
                if (++spins > ctl.spin_limit) {
                    pp_set_error(PP_DEV_TIMEOUT);
                    break;
                }
                backoff(spins);
            }
        }
        st_status(mine, F::INC | (excl + (StatT)tcount));
    }
    // every global index is below 2^31, so the offset arithmetic may wrap mod 2^32
    s_gbase[tid] = (uint32_t)((uint64_t)hexcl + (uint64_t)excl) - bstart;
    __syncthreads();

    // Write each digit run to its global position.
    for (uint32_t j = tid; j < nvalid; j += THREADS) {
        const KeyT k = s_keys[j];
        const uint32_t d = (uint32_t)(k >> ctl.shift) & (RADIX - 1);
        // htotal: the keys this pass places, the length of the output
        dst.store(pp_idx((uint64_t)(uint32_t)(s_gbase[d] + j), (uint64_t)htotal), k, 0u);
    }
}

// Up-front digit histogram of every pass, plus zeroing of pass 0's look-back
// words.  hist[p * 256 + d] must be zero on entry.
template <typename KeyT, class Src>
__global__ void __launch_bounds__(256) hist_kernel(Src src, const uint64_t *n_dev, uint64_t n_host,
                                                   int npasses, uint32_t *hist, uint32_t *status0,
                                                   uint64_t status0_words, uint32_t shift0 = 0) {
    __shared__ uint32_t sh[MAX_PASSES][RADIX];
    for (int i = threadIdx.x; i < MAX_PASSES * RADIX; i += blockDim.x) (&sh[0][0])[i] = 0;
    __syncthreads();
    const uint64_t n = n_dev ? *n_dev : n_host;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (has_load4<Src>::value) {
        if (src.vec) {  // whole groups of four with 16-byte loads, the rest below one by one
            for (; 4 * i0 + 4 <= n; i0 += stride) {
                KeyT k4[4];
                src.load4(4 * i0, k4);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    for (int p = 0; p < npasses; ++p)
                        atomicAdd(&sh[p][(uint32_t)(k4[j] >> (shift0 + 8 * p)) & (RADIX - 1)], 1u);
            }
            i0 = (n & ~3ull) + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;  // the tail, one by one
        }
    }
    for (uint64_t i = i0; i < n; i += stride) {
        KeyT k;
        uint32_t val;
        if (!src.load(i, k, val)) continue;
        for (int p = 0; p < npasses; ++p) atomicAdd(&sh[p][(uint32_t)(k >> (shift0 + 8 * p)) & (RADIX - 1)], 1u);
    }
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < status0_words; i += stride)
        status0[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < npasses * RADIX; i += blockDim.x) {
        const uint32_t c = (&sh[0][0])[i];
        if (c) atomicAdd(&hist[i], c);
    }
}

// Workspace of a sort of at most n_max elements in `npasses` passes.
struct SortWs {
    uint32_t *hist;      // [MAX_PASSES * 256]
    uint32_t *tile_ctr;  // [MAX_PASSES]
    void *status[2];     // look-back words, alternating between passes
    uint64_t ntiles_max;
    bool wide;
};

inline SortWs carve_sort_ws(Carver &c, uint64_t n_max) {
    SortWs w;
    w.hist = c.take<uint32_t>(MAX_PASSES * RADIX + MAX_PASSES);
    w.tile_ctr = w.hist ? w.hist + MAX_PASSES * RADIX : nullptr;
    w.ntiles_max = ceil_div(n_max ? n_max : 1, TILE);
    w.wide = wide_status(n_max);
    const size_t word = w.wide ? 8 : 4;
    for (int i = 0; i < 2; ++i) w.status[i] = c.take<char>(w.ntiles_max * RADIX * word);
    return w;
}

// Bytes of the control block (hist + tile counters) that must be zeroed
// before the histogram pass.
constexpr size_t kCtlBytes = (MAX_PASSES * RADIX + MAX_PASSES) * sizeof(uint32_t);

// Ask for the largest shared-memory carveout so that several 44 KB blocks fit per SM.
template <typename K>
inline bool prefer_shared(K kernel) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    return true;
}

// Launches pass `p` (of npasses) of a sort prepared in `w`.
template <typename KeyT, class Src, class Dst>
inline void launch_pass(const SortWs &w, int p, int npasses, Src src, Dst dst, const uint64_t *n_dev,
                        uint64_t n_max, cudaStream_t s, uint32_t shift0 = 0,
                        uint32_t spin_limit = kSpinLimit) {
    PassCtl ctl;
    ctl.shift = shift0 + 8u * (uint32_t)p;
    ctl.hist = w.hist + p * RADIX;
    ctl.status = w.status[p & 1];
    ctl.status_next = (p + 1 < npasses) ? w.status[(p + 1) & 1] : nullptr;
    ctl.tile_ctr = w.tile_ctr + p;
    ctl.n_dev = n_dev;
    ctl.n_host = n_max;
    ctl.spin_limit = spin_limit;
    const unsigned grid = (unsigned)ceil_div(n_max ? n_max : 1, TILE);
    if (w.wide) {
        static PerDevice carveout;
        carveout.get([] { return (int64_t)prefer_shared(pass_kernel<KeyT, uint64_t, Src, Dst>); });
        pass_kernel<KeyT, uint64_t, Src, Dst><<<grid, THREADS, 0, s>>>(src, dst, ctl);
    } else {
        static PerDevice carveout;
        carveout.get([] { return (int64_t)prefer_shared(pass_kernel<KeyT, uint32_t, Src, Dst>); });
        pass_kernel<KeyT, uint32_t, Src, Dst><<<grid, THREADS, 0, s>>>(src, dst, ctl);
    }
    count_launch();
}

}  // namespace os
}  // namespace pp
