// Kernel 3 (Sec. IV-D and the appendix): damped PageRank iterations
//
//     r(v) <- c * sum_u r(u) A(u,v) + ((1-c)/N) * sum(r)
//
// as a pull over Kernel 2's compressed columns.  With A(u,v) = count(u,v) /
// d_out(u), the sum over a column is sum_e count_e * x(u_e) for the vector
// x = r .* (1/d_out), which each iteration writes for the next one: the row
// normalisation is folded into the gathered vector and the matrix is read as
// packed (row position, count) words only.  Rows and columns are in Kernel
// 2's storage order (vertex iperm[p] at position p, grouped by degree), so x
// is written in the order it is gathered and the rows gathered most often
// share cache lines; r_out is written in vertex order.
//
// Work split by column length (a degree-bucketed pull SpMV), one warp per
// work item and no block-wide barriers, so each warp's gathers overlap other
// warps' arithmetic:
//   - a column longer than `shortmax` entries is cut into chunks of `chunk`
//     entries; a warp sums a chunk with coalesced index loads and a group of
//     gathers in flight per lane, reduces it in a fixed shuffle tree, and the
//     warp that finishes a column's last chunk adds the chunk sums in order;
//   - the other columns are summed one per lane, in slices of 32 columns
//     stored as a sliced ELLPACK copy of their entries (entry k of the
//     slice's lane j at word 32 * (slice base + k) + j): at each step the
//     warp reads 32 consecutive words, gathers 32 values of x and each lane
//     adds its own, so no shared memory and no reduction is needed.  Each
//     call builds the copy from the compressed columns: the positions are cut
//     into windows of 2^wbits consecutive columns, the short columns of a
//     window are sorted by decreasing length (counting sort) and dealt to
//     slices of 32, so a slice's lanes have nearly equal lengths and the
//     padding of a window is below 32 * shortmax words.
// shortmax and chunk are tuning knobs (k3_shortmax, k3_chunk).  The blocks
// keep almost no shared memory, so the SM's shared-memory / L1 array is
// nearly all L1, which the gathers of x need (the rows gathered most often
// are cached there).
// Items are dealt to warps round-robin.  Every column sum has a fixed order
// (a lane adds its column's entries in order; chunk sums in chunk order) and
// sum(r) is accumulated exactly in 128-bit fixed point, so results are
// bitwise reproducible whichever warp takes which item or lane.  With
// binary64 ranks the column sums are exact fixed-point sums as well (integer
// instructions, rounded once per column), which keeps the work off GB300's
// narrow FP64 pipe.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>

#include "fixedpoint.cuh"
#include "pp_common.cuh"

PP_DEFINE_ERROR_WORD(k3_fetch_error)

namespace pp {
namespace k3 {

constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;
constexpr int SHORTMAX_MAX = 512;  // largest long-column threshold (k3_shortmax)
constexpr int CHUNK_MIN = 256;     // smallest long-column chunk (small graphs; the k3_chunk knob is 2048 or 4096)
constexpr int SHORTMAX_MIN = 32;   // smallest long-column threshold (small graphs)
constexpr uint32_t NENT_BITS = 13; // a long chunk's item: entries | chunks of the column << NENT_BITS
constexpr uint32_t LONG_FLAG = 0x80000000u;
constexpr int SETUP_BLOCKS = 512;  // fixed, so the start-vector reduction is reproducible
constexpr int WIN_THREADS = 512;   // the window (slice planning) kernels
constexpr int SCAN_THREADS = 1024; // the one-block scan over windows
// A slice lane's slot word: length << SLOT_LEN_SHIFT | position within the
// window (at most 16 bits), or SLOT_NONE for a lane without a column.
constexpr uint32_t SLOT_LEN_SHIFT = 16;
constexpr uint32_t SLOT_NONE = 0xffffffffu;
// A slice's metadata: (base, window << META_LEN_BITS | length), where the
// slice's entry k of lane j is word 32 * (base + k) + j of the copy.
constexpr uint32_t META_LEN_BITS = 11;
constexpr uint32_t MAX_WIN_BITS = 16;
constexpr uint32_t EMPTY_PER_ITEM = 1024;  // empty columns per work item
// Exact sums (sum(r), and for the variants the dangling mass and the norm of
// the change) are spread over FX_SLOTS 128-bit accumulators per iterate, so
// that the warps' atomics do not all meet at one address; the readers add
// the slots (exactly: any order gives the same bits).
constexpr int FX_SLOTS = 32;

// log2 of the window width: about 1024 windows, each of 32 .. 65536 columns.
inline uint32_t win_bits(uint32_t scale) {
    const int b = std::min<int>(std::max<int>((int)scale - 10, 5), (int)MAX_WIN_BITS);
    return (uint32_t)std::min<int>(b, (int)scale);
}

__device__ __forceinline__ float to_acc(float x) { return x; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float to_acc(__half x) { return __half2float(x); }
__device__ __forceinline__ double to_acc(double x) { return x; }
template <typename TS>
__device__ __forceinline__ TS from_acc(float x);
template <>
__device__ __forceinline__ float from_acc<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half from_acc<__half>(float x) { return __float2half_rn(x); }

// binary16 keeps 5 exponent bits: the stored vector is x * 2^k (see xscale)
template <typename TS>
struct Scaled {
    static constexpr bool value = false;
};
template <>
struct Scaled<__half> {
    static constexpr bool value = true;
};
template <typename TS>
__device__ __forceinline__ TS from_acc(double x) { return x; }

// Control words in the workspace.
struct Ctl {
    uint32_t n_chunks;  // work items of the long columns (they come first)
    uint32_t n_slices;  // slices of 32 short columns (the next items)
    uint32_t sell_words32;  // words of the sliced copy / 32
    uint32_t n_empty;   // columns without entries (the last items, EMPTY_PER_ITEM each)
};

struct Args {
    uint32_t N, scale, cmax, iters;
    const uint32_t *colptr, *rowc;
    const uint32_t *iperm;  // vertex at position p
    const uint64_t *ovf_key;
    const uint32_t *ovf_cnt;
    const uint64_t *info;
    uint32_t wbits, nwin;     // windows of 2^wbits column positions, nwin of them
    uint4 *wcnt;              // [nwin] slices, sum of slice lengths, chunk items, empty columns of each window
    uint4 *woff;              // [nwin] exclusive prefix sums of the same
    uint32_t *slot;           // [32 * max slices] slot words (see SLOT_LEN_SHIFT)
    uint2 *meta;              // [max slices] slice metadata (see META_LEN_BITS)
    void *invs;               // [32 * max slices] 1/d_out of each slot's column (TA), 0 for empty slots
    uint32_t *elist;          // [N] positions of the columns without entries
    void *einv;               // [N] their 1/d_out (TA), in list order
    uint32_t *sell;           // the short columns' entries, sliced ELLPACK
    uint4 *item;              // [min(N, M/(SHORTMAX_MIN+1)) + M/CHUNK_MIN + 1] long-column chunks
    double *chunk_sum;        // [same] partial sums of long-column chunks
    uint32_t *ticket;         // [same] finished-chunk counters, at a column's first item
    unsigned long long *acc;  // [2 * FX_SLOTS * (iters + 1)] sum(r) per iterate, 128-bit fixed point
    int *fx_exp;              // [iters + 1] scale exponent of each accumulator
    double *ipart;            // [SETUP_BLOCKS]
    Ctl *ctl;
    double c;
    // The stored vector is x * xscale (a power of two): 2^min(scale - 9, 15)
    // for binary16, whose range (6e-8 .. 65504) would lose the small x = r /
    // d_out of a large graph (r is about 1/N); every r <= sum(r) <= 1, so the
    // stored values stay below 2^15.  1 for the other precisions.
    float xscale;
    uint32_t shortmax;    // columns longer than this are cut into chunks
    uint32_t chunk;       // entries of a long column per work item
    // variants (pp_pagerank_ex); zero / null for the plain iteration
    uint32_t flags;                  // PP_K3_DANGLING | PP_K3_CONVERGE
    double tol;                      // convergence threshold on norm(r_k - r_(k-1), 1)
    unsigned long long *dmass;       // [2 * FX_SLOTS * (iters + 1)] sum of r over dangling rows, per iterate
    unsigned long long *delta;       // [2 * FX_SLOTS * (iters + 1)] norm(r_k - r_(k-1), 1), per iterate
    uint32_t *state;                 // [0] converged, [1] iterations run
    // array lengths the checked build tests indices against
    uint32_t item_cap, slice_cap;    // entries of item / chunk_sum / ticket; of meta (slot: 32 per slice)
    uint64_t sell_cap;               // words of sell
};

__device__ __forceinline__ uint32_t ovf_lookup(const uint64_t *keys, const uint32_t *cnts, uint64_t n,
                                               uint64_t key) {
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (__ldg(keys + mid) < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < n && __ldg(keys + lo) == key) ? __ldg(cnts + lo) : 0u;
}

// The accumulator slots of iterate k.
__device__ __forceinline__ unsigned long long *fx_slot(unsigned long long *base, uint32_t k, uint32_t slot) {
    return base + 2ull * ((uint64_t)k * FX_SLOTS + slot % FX_SLOTS);
}

// Value of the exact sum of iterate k (every thread of the warp calls it;
// lane j reads slot j, the warp adds them in 128-bit fixed point).
__device__ __forceinline__ double fx_slots_value(const unsigned long long *base, uint32_t k, int E) {
    static_assert(FX_SLOTS == 32, "one slot per lane");
    const int lane = threadIdx.x & 31;
    const unsigned long long *p = base + 2ull * ((uint64_t)k * FX_SLOTS + lane);
    Fx128 t{p[0], p[1]};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t h = __shfl_xor_sync(0xffffffffu, t.hi, o);
        const uint64_t l = __shfl_xor_sync(0xffffffffu, t.lo, o);
        fx_add(t, h, l);
    }
    return fx_value(t.hi, t.lo, E);
}

// ------------------------------------------------------------------- planning
//
// Per window of 2^wbits column positions: the columns longer than shortmax
// become chunk items, the other non-empty ones are sorted by decreasing
// length and dealt to slices of 32 lanes, and the columns without entries
// (r = teleport only) go to a list processed EMPTY_PER_ITEM at a time.  Three launches: count (per window), scan (one
// block over the windows), fill (per window).  The placement of equal-length
// columns among lanes comes from shared-memory atomics and may differ from
// call to call; no result depends on it (each column is summed by one lane in
// entry order, and sum(r) is exact).

// Slices of a window whose non-empty short columns, by decreasing length,
// have the class counts hist[1..shortmax] (hist[L] columns of length L): the number
// of slices and the sum of their lengths (a slice is as long as its first,
// longest column).
__device__ __forceinline__ uint2 slice_totals(const uint32_t *hist, uint32_t shortmax) {
    uint32_t rank = 0, sum = 0;
    for (int L = (int)shortmax; L >= 1; --L) {
        const uint32_t n = hist[L];
        if (n) {
            sum += ((rank + n + 31) / 32 - (rank + 31) / 32) * (uint32_t)L;
            rank += n;
        }
    }
    return make_uint2((rank + 31) / 32, sum);
}

__global__ void __launch_bounds__(WIN_THREADS) window_count_kernel(Args a) {
    __shared__ uint32_t hist[SHORTMAX_MAX + 1];
    __shared__ uint32_t s_items;
    const uint32_t W = 1u << a.wbits, p0 = blockIdx.x << a.wbits;
    for (uint32_t i = threadIdx.x; i <= a.shortmax; i += blockDim.x) hist[i] = 0;
    if (threadIdx.x == 0) s_items = 0;
    __syncthreads();
    uint32_t items = 0;
    for (uint32_t i = threadIdx.x; i < W; i += blockDim.x) {
        const uint32_t p = p0 + i;
        const uint32_t len = __ldg(a.colptr + p + 1) - __ldg(a.colptr + p);
        if (len > a.shortmax)
            items += (len + a.chunk - 1) / a.chunk;
        else
            atomicAdd(&hist[len], 1u);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) items += __shfl_xor_sync(0xffffffffu, items, o);
    if ((threadIdx.x & 31) == 0 && items) atomicAdd(&s_items, items);
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint2 t = slice_totals(hist, a.shortmax);
        a.wcnt[blockIdx.x] = make_uint4(t.x, t.y, s_items, hist[0]);
    }
}

// Exclusive prefix sums of the windows' counts (one block); the totals go to ctl.
__global__ void __launch_bounds__(SCAN_THREADS) window_scan_kernel(Args a) {
    __shared__ uint32_t sc[40];
    uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
    for (uint32_t base = 0; base < a.nwin; base += SCAN_THREADS) {
        const uint32_t w = base + threadIdx.x;
        const uint4 c = w < a.nwin ? a.wcnt[w] : make_uint4(0u, 0u, 0u, 0u);
        uint32_t t0, t1, t2, t3;
        const uint32_t e0 = block_exclusive_sum<uint32_t, SCAN_THREADS>(c.x, sc, &t0);
        const uint32_t e1 = block_exclusive_sum<uint32_t, SCAN_THREADS>(c.y, sc, &t1);
        const uint32_t e2 = block_exclusive_sum<uint32_t, SCAN_THREADS>(c.z, sc, &t2);
        const uint32_t e3 = block_exclusive_sum<uint32_t, SCAN_THREADS>(c.w, sc, &t3);
        if (w < a.nwin) a.woff[w] = make_uint4(c0 + e0, c1 + e1, c2 + e2, c3 + e3);
        c0 += t0;
        c1 += t1;
        c2 += t2;
        c3 += t3;
    }
    if (threadIdx.x == 0) {
        a.ctl->n_slices = c0;
        a.ctl->sell_words32 = c1;
        a.ctl->n_chunks = c2;
        a.ctl->n_empty = c3;
    }
}

// Places a window's columns: chunk items for the long ones, slot words and
// slice metadata for the others, then copies the short columns' entries
// into their slices (one warp per slice; lane j copies its column's entries
// to words 32 * (base + k) + j, so the iteration reads them coalesced).
__global__ void __launch_bounds__(WIN_THREADS) window_fill_kernel(Args a) {
    __shared__ uint32_t next[SHORTMAX_MAX + 1];  // class counts, then the next free rank of each class
    __shared__ uint32_t first[SHORTMAX_MAX + 1]; // first rank of each class (classes by decreasing length)
    __shared__ uint32_t s_item, s_empty;
    __shared__ uint32_t sc[40];
    const uint32_t W = 1u << a.wbits, p0 = blockIdx.x << a.wbits;
    const uint4 off = a.woff[blockIdx.x];
    const uint32_t ns = pp_len(off.x, a.wcnt[blockIdx.x].x, a.slice_cap);
    const uint32_t L = a.shortmax;
    for (uint32_t i = threadIdx.x; i <= L; i += blockDim.x) next[i] = 0;
    if (threadIdx.x == 0) {
        s_item = off.z;
        s_empty = off.w;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < W; i += blockDim.x) {
        const uint32_t p = p0 + i;
        const uint32_t len = __ldg(a.colptr + p + 1) - __ldg(a.colptr + p);
        if (len <= L) atomicAdd(&next[len], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t r = 0;
        for (int c = (int)L; c >= 1; --c) {
            first[c] = r;
            r += next[c];
            next[c] = first[c];
        }
    }
    __syncthreads();
    uint32_t *slot = a.slot + 32ull * off.x;
    for (uint32_t i = threadIdx.x; i < W; i += blockDim.x) {
        const uint32_t p = p0 + i;
        const uint32_t s = __ldg(a.colptr + p), len = __ldg(a.colptr + p + 1) - s;
        if (len > L) {
            // a kept column has at most M/2 entries (the largest one is removed); the host picks
            // the chunk so that nc < 2^19 fits the item's high bits
            const uint32_t nc = (len + a.chunk - 1) / a.chunk;
            const uint32_t o = atomicAdd(&s_item, nc);
            for (uint32_t k = 0; k < nc; ++k) {
                const uint32_t cs = s + k * a.chunk;
                const uint32_t oi = pp_idx(o + k, a.item_cap);
                a.item[oi] = make_uint4(p | LONG_FLAG, o, cs, min(a.chunk, s + len - cs) | (nc << NENT_BITS));
                a.ticket[oi] = 0;
            }
        } else if (len == 0) {
            a.elist[pp_idx(atomicAdd(&s_empty, 1u), a.N)] = p;
        } else {
            const uint32_t rank = atomicAdd(&next[len], 1u);
            slot[pp_idx(rank, 32u * ns)] = (len << SLOT_LEN_SHIFT) | i;
        }
    }
    __syncthreads();
    // every class is placed, so the shortest one (length 1, the last) ends at the number of
    // non-empty short columns
    const uint32_t n_short = L >= 1 ? next[1] : 0u;
    for (uint32_t r = n_short + threadIdx.x; r < 32 * ns; r += blockDim.x) slot[r] = SLOT_NONE;
    // slice t starts at rank 32t and is as long as the class holding that rank: the first class
    // (from the longest) whose end rank next[c] exceeds 32t
    const uint32_t per = (ns + blockDim.x - 1) / blockDim.x;
    const uint32_t t0 = min(ns, threadIdx.x * per), t1 = min(ns, t0 + per);
    uint32_t mine = 0;
    for (uint32_t t = t0; t < t1; ++t) {
        uint32_t lo = 0, hi = L - 1;  // over j = L - c (c = L .. 1), where next[L - j] is nondecreasing in j
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (next[L - mid] > 32 * t)
                hi = mid;
            else
                lo = mid + 1;
        }
        mine += L - lo;
    }
    uint32_t tot;
    uint32_t base = off.y + block_exclusive_sum<uint32_t, WIN_THREADS>(mine, sc, &tot);
    for (uint32_t t = t0; t < t1; ++t) {
        uint32_t lo = 0, hi = L - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (next[L - mid] > 32 * t)
                hi = mid;
            else
                lo = mid + 1;
        }
        const uint32_t slen = L - lo;
        a.meta[off.x + t] = make_uint2(base, (blockIdx.x << META_LEN_BITS) | slen);
        base += slen;
    }
    __syncthreads();  // the slot words and metadata of this window are visible to the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t t = warp; t < ns; t += WIN_THREADS / 32) {
        const uint32_t o = slot[32 * t + lane];
        if (o == SLOT_NONE) continue;
        const uint32_t p = pp_idx(p0 + (o & ((1u << SLOT_LEN_SHIFT) - 1)), a.N);
        const uint32_t s0 = __ldg(a.colptr + p), sb = a.meta[off.x + t].x;
        const uint32_t len = pp_len(32ull * sb, pp_len(s0, o >> SLOT_LEN_SHIFT, a.info[PP_INFO_NNZ]), a.sell_cap, 32);
        const uint32_t *src = a.rowc + s0;
        uint32_t *dst = a.sell + 32ull * sb + lane;
        for (uint32_t k = 0; k < len; ++k) dst[32ull * k] = __ldg(src + k);
    }
}

// 1/d_out of each slot's column in slot order, and of each column without
// entries in list order (vertex-order input), so that the iteration reads
// them with the slot words instead of after them.
template <typename TA>
__global__ void __launch_bounds__(256) order_inv_kernel(Args a, const TA *inv) {
    const uint64_t nslots = 32ull * a.ctl->n_slices, nempty = a.ctl->n_empty;
    TA *invs = static_cast<TA *>(a.invs);
    TA *einv = static_cast<TA *>(a.einv);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nslots; q += stride) {
        const uint32_t o = a.slot[q];
        TA v = TA(0);
        if (o != SLOT_NONE) {
            const uint32_t win = a.meta[q / 32].y >> META_LEN_BITS;
            v = inv[pp_idx(a.iperm[pp_idx((win << a.wbits) + (o & ((1u << SLOT_LEN_SHIFT) - 1)), a.N)], a.N)];
        }
        invs[q] = v;
    }
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nempty; q += stride)
        einv[q] = inv[pp_idx(a.iperm[pp_idx(a.elist[q], a.N)], a.N)];
}

// Reset the per-call counters and sum |r0|.
__global__ void __launch_bounds__(256) setup_kernel(Args a, const double *r0) {
    __shared__ double s_red[32];
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = gtid; i < 2ull * FX_SLOTS * (a.iters + 1); i += stride) {
        a.acc[i] = 0;
        if (a.dmass) a.dmass[i] = 0;
        if (a.delta) a.delta[i] = 0;
    }
    if (gtid < 2 && a.state) a.state[gtid] = 0;
    if (gtid == 0) a.fx_exp[0] = 1;  // the normalised start vector has every entry <= 1 < 2^1
    double acc = 0.0;
    for (uint64_t i = gtid; i < a.N; i += stride) acc += fabs(r0[i]);
    const double bs = block_sum<double, 256>(acc, s_red);
    if (threadIdx.x == 0) a.ipart[blockIdx.x] = bs;
}

// r = r0 / norm(r0,1) rounded to the working precision; x = r / d_out; and
// sum(r) of that vector.  With iters == 0 the normalised r is the result.
// r0 is scaled by the binary64 reciprocal of the norm (within an ulp of the
// quotient; a division per element would occupy GB300's narrow FP64 pipe),
// and sum(r) is exact, so any grid gives the same bits.
template <typename TS, typename TA, typename TO>
__global__ void __launch_bounds__(256) normalize_kernel(Args a, const double *r0, const TA *inv, TA *invp, TS *x0,
                                                        TO *r_out, TA *rb0) {
    __shared__ double s_norm;
    __shared__ uint64_t s_fx[16];
    if (threadIdx.x == 0) {
        double n = 0.0;
        for (int b = 0; b < SETUP_BLOCKS; ++b) n += a.ipart[b];
        s_norm = n;
    }
    __syncthreads();
    const double rnorm = 1.0 / s_norm;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    Fx128 acc{0, 0}, dm{0, 0};
    // in storage order: position p holds vertex iperm[p]; 1/d_out is copied into that order too.
    // Four positions per round, so that their reads (iperm, then r0 and 1/d_out) are in flight together.
    constexpr int R = 4;
    for (uint64_t p0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p0 < a.N; p0 += R * stride) {
        uint32_t v[R];
        double q[R];
        TA iv[R];
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = p0 + k * stride < a.N ? pp_idx(a.iperm[p0 + k * stride], a.N) : 0u;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const bool in = p0 + k * stride < a.N;
            q[k] = in ? r0[v[k]] : 0.0;
            iv[k] = in ? inv[v[k]] : TA(0);
        }
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const uint64_t p = p0 + k * stride;
            if (p >= a.N) break;
            const TA r = (TA)(q[k] * rnorm);
            fx_add(acc, r, 1);
            invp[p] = iv[k];
            x0[p] = Scaled<TS>::value ? from_acc<TS>(r * iv[k] * (TA)a.xscale) : from_acc<TS>(r * iv[k]);
            if (a.iters == 0) r_out[v[k]] = (TO)r;
            if (rb0) rb0[p] = r;
            if ((a.flags & PP_K3_DANGLING) && iv[k] == TA(0)) fx_add(dm, r, 1);
        }
    }
    const Fx128 bt = fx_block_sum<256>(acc, s_fx);
    if (threadIdx.x == 0 && (bt.hi | bt.lo)) fx_atomic_add(fx_slot(a.acc, 0, blockIdx.x), bt);
    if (a.flags & PP_K3_DANGLING) {
        __syncthreads();
        const Fx128 bd = fx_block_sum<256>(dm, s_fx);
        if (threadIdx.x == 0 && (bd.hi | bd.lo)) fx_atomic_add(fx_slot(a.dmass, 0, blockIdx.x), bd);
    }
}

// ------------------------------------------------------------- the iteration

// Loads and stores of the iteration.  The gathered vector goes through L1
// (the rows gathered most often are cached there); the entries and the
// per-slice words are read once per iteration and bypass L1.  No L2
// eviction-policy operands: they would hold registers the gathers need.
__device__ __forceinline__ float ld_x(const float *p) { return __ldg(p); }
__device__ __forceinline__ double ld_x(const double *p) { return __ldg(p); }
__device__ __forceinline__ __nv_bfloat16 ld_x(const __nv_bfloat16 *p) {
    return __ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short *>(p)));
}
__device__ __forceinline__ void st_x(float *p, float v) { *p = v; }
__device__ __forceinline__ void st_x(double *p, double v) { *p = v; }
__device__ __forceinline__ void st_x(__nv_bfloat16 *p, __nv_bfloat16 v) { *p = v; }
__device__ __forceinline__ __half ld_x(const __half *p) {
    return __ushort_as_half(__ldg(reinterpret_cast<const unsigned short *>(p)));
}
__device__ __forceinline__ void st_x(__half *p, __half v) { *p = v; }
__device__ __forceinline__ uint32_t ld_once(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_once(const float *p) { return __uint_as_float(ld_once(reinterpret_cast<const uint32_t *>(p))); }
__device__ __forceinline__ double ld_once(const double *p) {
    double v;
    asm volatile("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}

// Per-thread exact accumulators: sum(r'), and for the variants the mass of
// the dangling rows and norm(r' - r, 1).
struct Sums {
    Fx128 s, dm, df;
};

// Finishes column `col` from its sum y: r = c*y + teleport, x' = r / d_out.
// EXT (the variants) also keeps r itself (rb_out) for the convergence test
// and the final result.
template <typename TS, typename TA, typename TO, bool LAST, bool EXT>
struct Epilogue {
    const TA *inv;
    TS *x_out;
    TO *r_out;
    TA cc, tele;  // cc = c / xscale: the column sums are of the stored (scaled) vector
    TA xscale;
    int E;
    const uint32_t *iperm;
    const TA *rb_in;
    TA *rb_out;
    uint32_t flags;
    uint32_t N;
    // col is a column position (vertex iperm[col])
    __device__ __forceinline__ void operator()(uint32_t col, TA y, TA inv_col, Sums &acc) const {
        col = pp_idx(col, N);
        const TA r = cc * y + tele;
        if (LAST && !EXT) r_out[pp_idx(__ldg(iperm + col), N)] = (TO)r;
        st_x(x_out + col, Scaled<TS>::value ? from_acc<TS>(r * inv_col * xscale) : from_acc<TS>(r * inv_col));
        fx_add(acc.s, r, E);
        if (EXT) {
            if (flags & PP_K3_CONVERGE) {
                const TA d = r - rb_in[col];
                fx_add(acc.df, d < TA(0) ? -d : d, E);
            }
            rb_out[col] = r;
            if ((flags & PP_K3_DANGLING) && inv_col == TA(0)) fx_add(acc.dm, r, E);
        }
    }
};

// count * x(u) of one packed entry of column `col` (the column is only needed,
// and only valid, when the count did not fit inline).
template <typename TA>
__device__ __forceinline__ TA entry_product(uint32_t w, TA xv, uint32_t col, const Args &a) {
    uint32_t cf = w >> a.scale;
    // most entries are one edge: x itself, without a conversion and a multiply
    // on the FP64 pipe (the narrowest one on GB300) for binary64 ranks
    if (cf == 1u) return xv;
    if (cf == a.cmax) {
        const uint32_t u = w & ((1u << a.scale) - 1u);
        cf = ovf_lookup(a.ovf_key, a.ovf_cnt, a.info[PP_INFO_NOVF],
                        ((uint64_t)__ldg(a.iperm + u) << 32) | __ldg(a.iperm + col));
    }
    return (TA)cf * xv;
}

template <typename TA>
__device__ __forceinline__ TA warp_sum(TA y) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xffffffffu, y, o);
    return y;  // in lane 0
}

// A column sum.  Binary32 (and bfloat16 or binary16 x): float additions in a fixed
// order.  Binary64: exact 128-bit fixed point scaled by the bound 2^E on
// sum(r) (every term cf * x(u) <= r(u) <= sum(r)), added with integer
// instructions and rounded once, because GB300's FP64 pipe is far narrower
// than its integer pipe; the sum then does not depend on the order either.
template <typename TA>
struct ColSum;
template <>
struct ColSum<float> {
    float v = 0.f;
    __device__ __forceinline__ void add(float x, int) { v += x; }
    __device__ __forceinline__ float value(int) const { return v; }
    __device__ __forceinline__ float warp_total(int) const { return warp_sum(v); }  // in lane 0
};
template <>
struct ColSum<double> {
    Fx128 v{0, 0};
    __device__ __forceinline__ void add(double x, int E) { fx_add_term(v, x, E); }
    __device__ __forceinline__ double value(int E) const { return fx_to_double(v, E); }
    __device__ __forceinline__ double warp_total(int E) const { return fx_to_double(fx_warp_sum(v), E); }
};

template <typename TS, typename TA, typename TO, bool LAST, int UNROLL, int MINB, bool EXT>
__global__ void __launch_bounds__(THREADS, MINB)
    iterate_kernel(Args a, const TA *inv, const TS *__restrict__ x_in, TS *__restrict__ x_out, TO *r_out,
                   uint32_t iter, const TA *rb_in, TA *rb_out) {
    constexpr int NW = WARPS;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double tele_extra = 0.0;
    if (EXT) {
        // the variants: stop once converged; the dangling rows' mass is spread evenly
        if (ld_relaxed_u32(a.state)) return;
        if ((a.flags & PP_K3_CONVERGE) && iter >= 1 &&
            fx_slots_value(a.delta, iter, a.fx_exp[iter]) < a.tol) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                a.state[1] = iter;
                st_relaxed_u32(a.state, 1u);
            }
            return;
        }
        if (a.flags & PP_K3_DANGLING)
            tele_extra = a.c / (double)a.N * fx_slots_value(a.dmass, iter, a.fx_exp[iter]);
    }
    const uint32_t n_chunks = a.ctl->n_chunks;
    const uint32_t n_cs = n_chunks + a.ctl->n_slices;  // chunks and slices; then the empty columns
    const uint32_t n_empty = a.ctl->n_empty;
    const uint32_t n_items = n_cs + (n_empty + EMPTY_PER_ITEM - 1) / EMPTY_PER_ITEM;
    const double S = fx_slots_value(a.acc, iter, a.fx_exp[iter]);
    const int E = fx_exponent(S);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.fx_exp[iter + 1] = E;
    const uint32_t umask = (1u << a.scale) - 1u;
    const Epilogue<TS, TA, TO, LAST, EXT> epi{inv,
                                              x_out,
                                              r_out,
                                              (TA)(a.c / (double)a.xscale),
                                              (TA)(((1.0 - a.c) / (double)a.N) * S + tele_extra),
                                              (TA)a.xscale,
                                              E,
                                              a.iperm,
                                              rb_in,
                                              rb_out,
                                              a.flags,
                                              a.N};
    Sums acc{{0, 0}, {0, 0}, {0, 0}};
    const uint32_t nwarps = gridDim.x * NW;

    // An item's descriptor: a chunk's (column | LONG_FLAG, first item, first
    // entry, entries | chunks << NENT_BITS), or a slice's (base, window <<
    // META_LEN_BITS | length, this lane's slot word, -) with this lane's
    // 1/d_out (stored in slot order, so it does not wait for the slot word).
    // The next one is fetched while this one is processed.
    struct Desc {
        uint4 d;
        TA iv;
    };
    auto descriptor = [&](uint32_t i) -> Desc {
        if (i >= n_cs) return Desc{make_uint4(0u, 0u, 0u, 0u), TA(0)};
        if (i < n_chunks) return Desc{__ldg(a.item + i), TA(0)};
        const uint32_t sl = i - n_chunks;
        const uint2 m = __ldg(a.meta + sl);
        return Desc{make_uint4(m.x, m.y, ld_once(a.slot + 32ull * sl + lane), 0u),
                    ld_once(static_cast<const TA *>(a.invs) + 32ull * sl + lane)};
    };
    uint32_t item = blockIdx.x * NW + warp;
    Desc cur = descriptor(item);
    while (item < n_items) {
        const uint32_t next = item + nwarps;
        const Desc nxt = descriptor(next);
        const uint4 it = cur.d;
        if (item < n_chunks) {
            // ---- one chunk of a long column: coalesced entries, a group of gathers in flight per lane
            const uint32_t col = pp_idx(it.x & ~LONG_FLAG, a.N), first = it.y, e0 = it.z;
            const uint32_t nent = pp_len(e0, it.w & ((1u << NENT_BITS) - 1), a.info[PP_INFO_NNZ]);
            // 0 (checked build) when the column's items leave the item arrays: then summed as one chunk
            const uint32_t nchunks = pp_len(first, it.w >> NENT_BITS, a.item_cap);
            ColSum<TA> part;
            // the entries of step s + 1 are loaded while the gathers of step s are in flight
            const uint32_t *rw = a.rowc + e0 + lane;
            uint32_t w[UNROLL];
#pragma unroll
            for (int m = 0; m < UNROLL; ++m) w[m] = (uint32_t)(m * 32 + lane) < nent ? ld_once(rw + m * 32) : 0u;
            for (uint32_t base = 0; base < nent; base += 32 * UNROLL) {
                TA xv[UNROLL];
#pragma unroll
                for (int m = 0; m < UNROLL; ++m) {
                    const uint32_t k = base + (uint32_t)(m * 32 + lane);
                    xv[m] = k < nent ? to_acc(ld_x(x_in + (w[m] & umask))) : TA(0);
                }
                uint32_t wn[UNROLL];
                const uint32_t nb = base + 32 * UNROLL;
#pragma unroll
                for (int m = 0; m < UNROLL; ++m) {
                    const uint32_t k = nb + (uint32_t)(m * 32 + lane);
                    wn[m] = k < nent ? ld_once(rw + nb + m * 32) : 0u;
                }
#pragma unroll
                for (int m = 0; m < UNROLL; ++m) {
                    const uint32_t k = base + (uint32_t)(m * 32 + lane);
                    if (k < nent) part.add(entry_product<TA>(w[m], xv[m], col, a), E);
                    w[m] = wn[m];
                }
            }
            const TA y = part.warp_total(E);
            if (lane == 0) {
                if (nchunks <= 1) {
                    epi(col, y, __ldg(inv + col), acc);
                } else {
                    // the warp finishing the column's last chunk adds the chunk sums in order
                    a.chunk_sum[item] = (double)y;
                    __threadfence();
                    const uint32_t t = atomicAdd(a.ticket + first, 1u);
                    if ((t + 1) % nchunks == 0) {
                        __threadfence();
                        TA tot = TA(0);
                        for (uint32_t q = 0; q < nchunks; ++q) tot += (TA)__ldcg(a.chunk_sum + first + q);
                        epi(col, tot, __ldg(inv + col), acc);
                    }
                }
            }
        } else if (item >= n_cs) {
            // ---- columns without entries: r = teleport, EMPTY_PER_ITEM of them, coalesced list reads
            const uint32_t q0 = (item - n_cs) * EMPTY_PER_ITEM;
            const uint32_t q1 = min(n_empty, q0 + EMPTY_PER_ITEM);
            const TA *einv = static_cast<const TA *>(a.einv);
            for (uint32_t q = q0 + lane; q < q1; q += 32) epi(ld_once(a.elist + q), TA(0), ld_once(einv + q), acc);
        } else {
            // ---- a slice of 32 short columns, one per lane: step k reads 32 consecutive words
            const uint32_t slen = it.y & ((1u << META_LEN_BITS) - 1), win = it.y >> META_LEN_BITS;
            const uint32_t o = it.z;
            const bool valid = o != SLOT_NONE;
            const uint32_t len = valid ? pp_len(32ull * it.x, o >> SLOT_LEN_SHIFT, a.sell_cap, 32) : 0u;
            const uint32_t col = pp_idx_if(valid, (win << a.wbits) + (o & ((1u << SLOT_LEN_SHIFT) - 1)), a.N);
            const TA myinv = cur.iv;
            const uint32_t *src = a.sell + 32ull * it.x + lane;
            ColSum<TA> y;
            uint32_t w[UNROLL];
#pragma unroll
            for (int m = 0; m < UNROLL; ++m) w[m] = (uint32_t)m < len ? ld_once(src + 32 * m) : 0u;
            for (uint32_t k = 0; k < slen; k += UNROLL) {
                TA xv[UNROLL];
#pragma unroll
                for (int m = 0; m < UNROLL; ++m)
                    xv[m] = k + m < len ? to_acc(ld_x(x_in + (w[m] & umask))) : TA(0);
                uint32_t wn[UNROLL];
#pragma unroll
                for (int m = 0; m < UNROLL; ++m)
                    wn[m] = k + UNROLL + m < len ? ld_once(src + 32ull * (k + UNROLL + m)) : 0u;
#pragma unroll
                for (int m = 0; m < UNROLL; ++m) {
                    if (k + m < len) y.add(entry_product<TA>(w[m], xv[m], col, a), E);
                    w[m] = wn[m];
                }
            }
            if (valid) epi(col, y.value(E), myinv, acc);
        }
        item = next;
        cur = nxt;
    }
    // exact sums per warp, added with one atomic pair per warp: the kernel
    // keeps no shared memory, so the driver leaves the whole array to L1
    const Fx128 bt = fx_warp_sum(acc.s);
    const uint32_t gw = blockIdx.x * NW + warp;
    if (lane == 0 && (bt.hi | bt.lo)) fx_atomic_add(fx_slot(a.acc, iter + 1, gw), bt);
    if (EXT && (a.flags & PP_K3_DANGLING)) {
        const Fx128 bd = fx_warp_sum(acc.dm);
        if (lane == 0 && (bd.hi | bd.lo)) fx_atomic_add(fx_slot(a.dmass, iter + 1, gw), bd);
    }
    if (EXT && (a.flags & PP_K3_CONVERGE)) {
        const Fx128 bf = fx_warp_sum(acc.df);
        if (lane == 0 && (bf.hi | bf.lo)) fx_atomic_add(fx_slot(a.delta, iter + 1, gw), bf);
    }
}

// The variants: r after the iterations that ran (storage order) into r_out
// (vertex order), and the number of iterations.
template <typename TA, typename TO>
__global__ void __launch_bounds__(256) finish_kernel(Args a, const TA *rb0, const TA *rb1, TO *r_out,
                                                     uint32_t *iters_done) {
    const uint32_t k = ld_relaxed_u32(a.state) ? a.state[1] : a.iters;
    const TA *rb = (k & 1) ? rb1 : rb0;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.N; p += (uint64_t)gridDim.x * blockDim.x)
        r_out[pp_idx(a.iperm[p], a.N)] = (TO)rb[p];
    if (iters_done && blockIdx.x == 0 && threadIdx.x == 0) *iters_done = k;
}

// r_l1 = r / norm(r,1) in binary64: sum, then scale.
template <typename TO>
__global__ void __launch_bounds__(256) l1_sum_kernel(const TO *r, uint32_t N, double *ipart) {
    __shared__ double s_red[32];
    double acc = 0.0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x)
        acc += fabs((double)r[i]);
    const double bs = block_sum<double, 256>(acc, s_red);
    if (threadIdx.x == 0) ipart[blockIdx.x] = bs;
}

template <typename TO>
__global__ void __launch_bounds__(256) l1_scale_kernel(const TO *r, uint32_t N, const double *ipart, double *out) {
    __shared__ double s_norm;
    if (threadIdx.x == 0) {
        double n = 0.0;
        for (int b = 0; b < SETUP_BLOCKS; ++b) n += ipart[b];
        s_norm = n;
    }
    __syncthreads();
    const double norm = s_norm;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = (double)r[i] / norm;
}

struct Layout {
    void *x[2];
    void *invp;  // 1/d_out in storage order (TA)
    uint4 *wcnt, *woff;
    uint32_t *slot;
    uint2 *meta;
    void *invs;
    uint32_t *elist;
    void *einv;
    uint32_t *sell;
    uint4 *item;
    double *chunk_sum;
    uint32_t *ticket;
    unsigned long long *acc;
    int *fx_exp;
    double *ipart;
    Ctl *ctl;
    // the variants only
    void *rb[2];  // r in storage order (TA), ping-pong
    unsigned long long *dmass, *delta;
    uint32_t *state;
    uint32_t wbits, nwin;
    uint64_t max_slices, max_items, sell_words;
    size_t bytes;
};

// The sliced copy holds each short column's entries plus padding; with the
// columns of a window sorted by decreasing length, a window pads fewer than
// 32 * shortmax words (slice t is as long as its first column, which is no
// longer than any column of slice t - 1), so M + windows * 32 * SHORTMAX_MAX
// words always suffice (nnz <= M).
inline Layout layout(void *ws, uint64_t M, uint32_t scale, uint32_t iters, pp_dtype dt, bool ext = false) {
    Carver c(ws);
    Layout L;
    const uint64_t N = 1ull << scale;
    L.wbits = win_bits(scale);
    L.nwin = (uint32_t)(N >> L.wbits);
    const uint64_t max_slices = (uint64_t)L.nwin * ceil_div(1ull << L.wbits, 32);
    L.max_slices = max_slices;
    // chunks: at most one per long column plus nnz/chunk, and a long column has
    // more than SHORTMAX_MIN of the nnz <= M entries
    const uint64_t max_items = std::min<uint64_t>(N, M / (SHORTMAX_MIN + 1)) + M / CHUNK_MIN + 1;
    const size_t xs = dt == PP_FP64 ? 8 : (dt == PP_FP32 ? 4 : 2);  // bfloat16, binary16: 2
    L.x[0] = c.take<char>(N * xs);
    L.x[1] = c.take<char>(N * xs);
    L.invp = c.take<char>(N * (dt == PP_FP64 ? 8 : 4));
    L.wcnt = c.take<uint4>(L.nwin);
    L.woff = c.take<uint4>(L.nwin);
    L.slot = c.take<uint32_t>(32 * max_slices);
    L.meta = c.take<uint2>(max_slices);
    L.invs = c.take<char>(32 * max_slices * (dt == PP_FP64 ? 8 : 4));
    L.elist = c.take<uint32_t>(N);
    L.einv = c.take<char>(N * (dt == PP_FP64 ? 8 : 4));
    L.max_items = max_items;
    L.sell_words = M + (uint64_t)L.nwin * 32 * SHORTMAX_MAX;
    L.sell = c.take<uint32_t>(L.sell_words);
    L.item = c.take<uint4>(max_items);
    L.chunk_sum = c.take<double>(max_items);
    L.ticket = c.take<uint32_t>(max_items);
    L.acc = c.take<unsigned long long>(2ull * FX_SLOTS * (iters + 1));
    L.fx_exp = c.take<int>((uint64_t)iters + 1);
    L.ipart = c.take<double>(SETUP_BLOCKS);
    L.ctl = c.take<Ctl>(1);
    L.rb[0] = L.rb[1] = nullptr;
    L.dmass = L.delta = nullptr;
    L.state = nullptr;
    if (ext) {
        const size_t ta = dt == PP_FP64 ? 8 : 4;
        L.rb[0] = c.take<char>(N * ta);
        L.rb[1] = c.take<char>(N * ta);
        L.dmass = c.take<unsigned long long>(2ull * FX_SLOTS * (iters + 1));
        L.delta = c.take<unsigned long long>(2ull * FX_SLOTS * (iters + 1));
        L.state = c.take<uint32_t>(2);
    }
    L.bytes = c.size();
    return L;
}

template <typename K>
inline int occupancy(K kernel, int threads, size_t smem) {
    int o = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kernel, threads, smem);
    return o > 0 ? o : 1;
}

inline int device_attr(cudaDeviceAttr attr) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, attr, dev);
    return v;
}

// Shared-memory carveout of `kernel` with `smem` dynamic bytes per block:
// the smallest of the SM's shared-memory sizes (0, 8, 16, 32, 64, 100, 132,
// 164, 196 or 228 KB; the rest of the 256 KB array is L1) that holds
// `blocks` blocks plus the 1 KB the system keeps per block.  The hint is a
// whole percentage of the largest size, which the driver rounds up to a
// supported size, so it is rounded down here: a percentage rounded up could
// land just past the wanted size and take the next one.
template <typename K>
inline void set_smem(K kernel, int blocks, size_t smem) {
    static const long kSizesKB[] = {0, 8, 16, 32, 64, 100, 132, 164, 196, 228};
    if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int pct = -1;  // cudaSharedmemCarveoutDefault
    const long per_sm = device_attr(cudaDevAttrMaxSharedMemoryPerMultiprocessor);
    const long need = (long)blocks * ((long)smem + 1024);
    for (long kb : kSizesKB)
        if (kb * 1024 >= need && kb * 1024 <= per_sm) {
            pct = (int)(100 * kb * 1024 / per_sm);
            break;
        }
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

// Variant options of pp_pagerank_ex (EXT kernels only).
struct Variant {
    uint32_t flags;
    double tol;
    uint32_t *iters_done;
};

template <typename TS, typename TA, typename TO, int UNROLL, int MINB, bool EXT>
pp_status run_unroll(const pp_graph *g, const double *r0, uint32_t iters, double c, pp_dtype dt, TO *r_out,
                     double *r_l1, const Layout &L, cudaStream_t s, const Variant &var) {
    const uint32_t N = 1u << g->scale;
    Args a;
    a.N = N;
    a.scale = g->scale;
    a.cmax = (uint32_t)((1ull << (32 - g->scale)) - 1);
    a.iters = iters;
    a.colptr = g->colptr;
    a.rowc = g->rowc;
    a.iperm = g->iperm;
    a.ovf_key = g->ovf_key;
    a.ovf_cnt = g->ovf_cnt;
    a.info = g->info;
    a.wbits = L.wbits;
    a.nwin = L.nwin;
    a.wcnt = L.wcnt;
    a.woff = L.woff;
    a.slot = L.slot;
    a.meta = L.meta;
    a.invs = L.invs;
    a.elist = L.elist;
    a.einv = L.einv;
    a.sell = L.sell;
    a.item = L.item;
    a.chunk_sum = L.chunk_sum;
    a.ticket = L.ticket;
    a.acc = L.acc;
    a.fx_exp = L.fx_exp;
    a.ipart = L.ipart;
    a.ctl = L.ctl;
    a.c = c;
    a.item_cap = (uint32_t)L.max_items;
    a.slice_cap = (uint32_t)L.max_slices;
    a.sell_cap = L.sell_words;
    auto *k_mid = iterate_kernel<TS, TA, TO, false, UNROLL, MINB, EXT>;
    auto *k_last = iterate_kernel<TS, TA, TO, !EXT, UNROLL, MINB, EXT>;
    constexpr int NT = THREADS;
    constexpr size_t smem = 0;
    // the carveout attributes and the occupancy, once per instantiation and device
    static PerDevice cached;  // o_mid << 16 | o_last
    const uint32_t cv = (uint32_t)cached.get([&] {
        set_smem(k_mid, MINB, 0);
        set_smem(k_last, MINB, 0);
        return (int64_t)(((uint32_t)occupancy(k_mid, NT, smem) << 16) | (uint32_t)occupancy(k_last, NT, smem));
    });
    const int o_mid = (int)(cv >> 16), o_last = (int)(cv & 0xffff);
    const int sms = sm_count();
    // A small graph gives each warp a few entries, and the iteration then
    // lasts as long as its longest item (a chain of dependent loads and
    // gathers in one warp): halve the long-column threshold and the chunk
    // while they exceed the entries per warp (resp. 8 times that).  A column
    // has at most M/2 entries (the largest one is removed), and its chunk
    // count must fit the item's 19-bit field.
    const uint64_t per_warp = g->M / ((uint64_t)sms * o_mid * WARPS);
    uint32_t shortmax = (uint32_t)tuning("k3_shortmax"), chunk = (uint32_t)tuning("k3_chunk");
    while (shortmax > (uint32_t)SHORTMAX_MIN && shortmax > per_warp) shortmax >>= 1;
    while (chunk > (uint32_t)CHUNK_MIN && chunk > 8 * per_warp) chunk >>= 1;
    while ((g->M / 2 + chunk - 1) / chunk >= (1ull << (32 - NENT_BITS))) chunk <<= 1;
    a.shortmax = shortmax;
    a.chunk = chunk;
    a.xscale = Scaled<TS>::value ? (float)(1u << std::min<int>(std::max<int>((int)g->scale - 9, 0), 15)) : 1.0f;
    a.flags = EXT ? var.flags : 0u;
    a.tol = var.tol;
    a.dmass = L.dmass;
    a.delta = L.delta;
    a.state = L.state;
    TA *rb0 = static_cast<TA *>(L.rb[0]), *rb1 = static_cast<TA *>(L.rb[1]);
    const TA *inv = dt == PP_FP64 ? reinterpret_cast<const TA *>(g->inv_dout64)
                                  : reinterpret_cast<const TA *>(g->inv_dout32);
    if (!inv) return PP_ERR_INVALID_ARG;
    TS *x0 = static_cast<TS *>(L.x[0]);
    TS *x1 = static_cast<TS *>(L.x[1]);
    setup_kernel<<<SETUP_BLOCKS, 256, 0, s>>>(a, r0);
    window_count_kernel<<<L.nwin, WIN_THREADS, 0, s>>>(a);
    window_scan_kernel<<<1, SCAN_THREADS, 0, s>>>(a);
    window_fill_kernel<<<L.nwin, WIN_THREADS, 0, s>>>(a);
    order_inv_kernel<TA><<<(unsigned)std::min<uint64_t>(ceil_div(32ull * L.max_slices + N, 256), 16ull * sm_count()),
                           256, 0, s>>>(a, inv);
    TA *invp = static_cast<TA *>(L.invp);  // 1/d_out in storage order
    // one wave of blocks (each sums the norm's partials once)
    const unsigned nblocks = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(ceil_div(N, 256), 8ull * sm_count()));
    normalize_kernel<TS, TA, TO><<<nblocks, 256, 0, s>>>(a, r0, inv, invp, x0, r_out, EXT ? rb0 : nullptr);
    count_launch(6);

    // no more blocks than the graph can give work to (warps take items
    // round-robin, so any grid is correct): an upper bound on the items --
    // slices, chunks (at most nnz/chunk plus one per long column, and a long
    // column has more than shortmax of the nnz <= M entries), runs of empty
    // columns -- over WARPS per block
    const uint64_t item_bound = L.max_slices + g->M / a.chunk + std::min<uint64_t>(N, g->M / (a.shortmax + 1)) +
                                N / EMPTY_PER_ITEM + 2;
    const unsigned blocks_cap = (unsigned)std::max<uint64_t>(1, ceil_div(item_bound, WARPS));
    const unsigned grid_mid = std::min<unsigned>(sms * o_mid, blocks_cap);
    const unsigned grid_last = std::min<unsigned>(sms * o_last, blocks_cap);
    for (uint32_t it = 0; it < iters; ++it) {
        const TS *xin = (it & 1) ? x1 : x0;
        TS *xout = (it & 1) ? x0 : x1;
        const TA *rin = (it & 1) ? rb1 : rb0;
        TA *rout = (it & 1) ? rb0 : rb1;
        // the variants write r every iteration and finish_kernel picks the last one
        if (it + 1 == iters && !EXT)
            k_last<<<grid_last, NT, smem, s>>>(a, invp, xin, xout, r_out, it, rin, rout);
        else
            k_mid<<<grid_mid, NT, smem, s>>>(a, invp, xin, xout, r_out, it, rin, rout);
        count_launch();
    }
    if (EXT) {
        finish_kernel<TA, TO><<<SETUP_BLOCKS, 256, 0, s>>>(a, rb0, rb1, r_out, var.iters_done);
        count_launch();
    }
    if (r_l1) {
        l1_sum_kernel<TO><<<SETUP_BLOCKS, 256, 0, s>>>(r_out, N, L.ipart);
        l1_scale_kernel<TO><<<SETUP_BLOCKS, 256, 0, s>>>(r_out, N, L.ipart, r_l1);
        count_launch(2);
    }
    return launch_status();
}

template <typename TS, typename TA, typename TO>
pp_status run(const pp_graph *g, const double *r0, uint32_t iters, double c, pp_dtype dt, TO *r_out,
              double *r_l1, const Layout &L, cudaStream_t s) {
    const Variant none{0u, 0.0, nullptr};
    const bool u4 = tuning(sizeof(TA) == 8 ? "k3_unroll_f64" : "k3_unroll_f32") == 4;
    switch (tuning("k3_minblocks")) {
        case 4:
            return u4 ? run_unroll<TS, TA, TO, 4, 4, false>(g, r0, iters, c, dt, r_out, r_l1, L, s, none)
                      : run_unroll<TS, TA, TO, 8, 4, false>(g, r0, iters, c, dt, r_out, r_l1, L, s, none);
        case 8:
            return u4 ? run_unroll<TS, TA, TO, 4, 8, false>(g, r0, iters, c, dt, r_out, r_l1, L, s, none)
                      : run_unroll<TS, TA, TO, 8, 8, false>(g, r0, iters, c, dt, r_out, r_l1, L, s, none);
        default:
            return u4 ? run_unroll<TS, TA, TO, 4, 6, false>(g, r0, iters, c, dt, r_out, r_l1, L, s, none)
                      : run_unroll<TS, TA, TO, 8, 6, false>(g, r0, iters, c, dt, r_out, r_l1, L, s, none);
    }
}

// The variants run one instantiation per precision (4 blocks per SM; unroll
// 8 for binary32 sums, 4 for the binary64 fixed-point sums).
template <typename TS, typename TA, typename TO>
pp_status run_ext(const pp_graph *g, const double *r0, uint32_t iters, double c, pp_dtype dt, TO *r_out,
                  double *r_l1, const Layout &L, cudaStream_t s, const Variant &var) {
    return run_unroll<TS, TA, TO, sizeof(TA) == 8 ? 4 : 8, 4, true>(g, r0, iters, c, dt, r_out, r_l1, L, s, var);
}

// The gather rate that bounds an iteration: the packed entries streamed once
// (coalesced, bypassing L1) and x gathered through L1 for each, with eight
// independent loads in flight per thread and nothing else; every thread's
// sum goes to *out (one atomic per warp) so that no load is dead.
constexpr int PROBE_UNROLL = 8;
__global__ void __launch_bounds__(256, 8) gather_probe_kernel(const uint32_t *rowc, uint64_t n, uint32_t umask,
                                                              const float *x, float *out) {
    float acc = 0.f;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t b = tid; b < n; b += PROBE_UNROLL * stride) {
        uint32_t w[PROBE_UNROLL];
        float xv[PROBE_UNROLL];
#pragma unroll
        for (int m = 0; m < PROBE_UNROLL; ++m) w[m] = b + m * stride < n ? ld_once(rowc + b + m * stride) : 0u;
#pragma unroll
        for (int m = 0; m < PROBE_UNROLL; ++m) xv[m] = b + m * stride < n ? __ldg(x + (w[m] & umask)) : 0.f;
#pragma unroll
        for (int m = 0; m < PROBE_UNROLL; ++m) acc += xv[m];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

}  // namespace k3
}  // namespace pp

using namespace pp;

extern "C" pp_status pp_gather_probe(const uint32_t *rowc, uint64_t n, uint32_t scale, const float *x, float *out,
                                     void *stream) {
    PP_ENTRY("pp_gather_probe");
    if (scale < 1 || scale > 27 || (n && (!rowc || !x)) || !out) return PP_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    static PerDevice occ_dev;
    const int occ = (int)occ_dev.get([] {
        // no shared memory at all: the whole array is L1, which the gathers need
        // (measured: 0.64 ms against 0.675 ms with an 8 KB carve-out at scale 24)
        cudaFuncSetAttribute(k3::gather_probe_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
        return (int64_t)k3::occupancy(k3::gather_probe_kernel, 256, 0);
    });
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sm_count() * occ,
                                                                             ceil_div(n, 256)));
    k3::gather_probe_kernel<<<grid, 256, 0, s>>>(rowc, n, (1u << scale) - 1u, x, out);
    count_launch();
    return launch_status();
}

extern "C" pp_status pp_pagerank_workspace(uint64_t M, uint32_t scale, uint32_t iters, pp_dtype dt,
                                           size_t *bytes) {
    if (!bytes || scale < 1 || scale > 27 || M > (1ull << 31) || (int)dt < 0 || (int)dt > 3)
        return PP_ERR_INVALID_ARG;
    *bytes = k3::layout(nullptr, M, scale, iters, dt).bytes;
    return PP_OK;
}

extern "C" pp_status pp_pagerank(const pp_graph *g, const double *r0, uint32_t iters, double c, pp_dtype dt,
                                 void *r_out, double *r_l1, void *ws, size_t ws_bytes, void *stream) {
    PP_ENTRY("pp_pagerank");
    if (!g || !r0 || !r_out || (int)dt < 0 || (int)dt > 3) return PP_ERR_INVALID_ARG;
    if (g->scale < 1 || g->scale > 27 || g->M > (1ull << 31) || !(c >= 0.0 && c <= 1.0)) return PP_ERR_INVALID_ARG;
    if (!g->colptr || !g->rowc || !g->ovf_key || !g->ovf_cnt || !g->info || !g->perm || !g->iperm)
        return PP_ERR_INVALID_ARG;
    const k3::Layout need = k3::layout(nullptr, g->M, g->scale, iters, dt);
    pp_status st = check_ws(ws, ws_bytes, need.bytes);
    if (st != PP_OK) return st;
    const k3::Layout L = k3::layout(ws, g->M, g->scale, iters, dt);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (dt) {
        case PP_FP64:
            return k3::run<double, double, double>(g, r0, iters, c, dt, static_cast<double *>(r_out), r_l1, L, s);
        case PP_FP32:
            return k3::run<float, float, float>(g, r0, iters, c, dt, static_cast<float *>(r_out), r_l1, L, s);
        case PP_BF16_FP32ACC:
            return k3::run<__nv_bfloat16, float, float>(g, r0, iters, c, dt, static_cast<float *>(r_out), r_l1, L,
                                                        s);
        default:
            return k3::run<__half, float, float>(g, r0, iters, c, dt, static_cast<float *>(r_out), r_l1, L, s);
    }
}

extern "C" pp_status pp_pagerank_ex_workspace(uint64_t M, uint32_t scale, uint32_t iters, pp_dtype dt,
                                              size_t *bytes) {
    if (!bytes || scale < 1 || scale > 27 || M > (1ull << 31) || (int)dt < 0 || (int)dt > 3)
        return PP_ERR_INVALID_ARG;
    *bytes = k3::layout(nullptr, M, scale, iters, dt, true).bytes;
    return PP_OK;
}

extern "C" pp_status pp_pagerank_ex(const pp_graph *g, const double *r0, uint32_t iters, double c, pp_dtype dt,
                                    uint32_t flags, double tol, void *r_out, double *r_l1, uint32_t *iters_done,
                                    void *ws, size_t ws_bytes, void *stream) {
    PP_ENTRY("pp_pagerank_ex");
    if (!g || !r0 || !r_out || (int)dt < 0 || (int)dt > 3) return PP_ERR_INVALID_ARG;
    if (g->scale < 1 || g->scale > 27 || g->M > (1ull << 31) || !(c >= 0.0 && c <= 1.0)) return PP_ERR_INVALID_ARG;
    if (flags & ~(uint32_t)(PP_K3_DANGLING | PP_K3_CONVERGE)) return PP_ERR_INVALID_ARG;
    if ((flags & PP_K3_CONVERGE) && !(tol > 0.0)) return PP_ERR_INVALID_ARG;
    if (!g->colptr || !g->rowc || !g->ovf_key || !g->ovf_cnt || !g->info || !g->perm || !g->iperm)
        return PP_ERR_INVALID_ARG;
    const k3::Layout need = k3::layout(nullptr, g->M, g->scale, iters, dt, true);
    pp_status st = check_ws(ws, ws_bytes, need.bytes);
    if (st != PP_OK) return st;
    const k3::Layout L = k3::layout(ws, g->M, g->scale, iters, dt, true);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const k3::Variant var{flags, (flags & PP_K3_CONVERGE) ? tol : 0.0, iters_done};
    switch (dt) {
        case PP_FP64:
            return k3::run_ext<double, double, double>(g, r0, iters, c, dt, static_cast<double *>(r_out), r_l1, L, s,
                                                       var);
        case PP_FP32:
            return k3::run_ext<float, float, float>(g, r0, iters, c, dt, static_cast<float *>(r_out), r_l1, L, s, var);
        case PP_BF16_FP32ACC:
            return k3::run_ext<__nv_bfloat16, float, float>(g, r0, iters, c, dt, static_cast<float *>(r_out), r_l1, L,
                                                            s, var);
        default:
            return k3::run_ext<__half, float, float>(g, r0, iters, c, dt, static_cast<float *>(r_out), r_l1, L, s,
                                                     var);
    }
}
