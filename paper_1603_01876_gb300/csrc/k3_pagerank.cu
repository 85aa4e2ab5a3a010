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
//   - the other columns form tiles of at most 32 consecutive columns and
//     2*shortmax entries; a warp gathers count * x(u) for the tile's entries
//     into its shared-memory slab, then each lane sums one short column (at
//     most `lane_short` entries) in order, and the whole warp takes each
//     medium column (lanes stride, fixed shuffle tree).
// shortmax, chunk and lane_short are tuning knobs (k3_shortmax, k3_chunk,
// k3_lane_short); for one setting every run gives the same bits.
// Blocks reserve no more shared memory than they use; the rest of the SM's
// shared-memory / L1 array is L1.
// Items are dealt to warps round-robin.  Every column sum has a fixed order
// and sum(r) is accumulated exactly in 128-bit fixed point, so results are
// bitwise reproducible whichever warp takes which item.  With binary64
// ranks the column sums are exact fixed-point sums as well (integer
// instructions, rounded once per column), which keeps the work off GB300's
// narrow FP64 pipe.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>

#include "fixedpoint.cuh"
#include "pp_common.cuh"

PP_DEFINE_ERROR_WORD(k3_fetch_error)

namespace pp {
namespace k3 {

constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;
constexpr int TILE_COLS = 32;      // one lane per column in a tile
constexpr int SHORTMAX_MAX = 256;  // largest long-column threshold (k3_shortmax)
constexpr int TILE_ENTRIES = 2 * SHORTMAX_MAX;
constexpr int CHUNK_MIN = 2048;    // smallest long-column chunk (k3_chunk)
constexpr uint32_t NENT_BITS = 13; // a long chunk's item: entries | chunks of the column << NENT_BITS
constexpr uint32_t LONG_FLAG = 0x80000000u;
constexpr int SETUP_BLOCKS = 512;  // fixed, so the start-vector reduction is reproducible
constexpr int PLAN_THREADS = 256;
constexpr int PLAN_ITEMS = 16;
constexpr int PLAN_TILE = PLAN_THREADS * PLAN_ITEMS;

__device__ __forceinline__ float to_acc(float x) { return x; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ double to_acc(double x) { return x; }
template <typename TS>
__device__ __forceinline__ TS from_acc(float x);
template <>
__device__ __forceinline__ float from_acc<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <typename TS>
__device__ __forceinline__ TS from_acc(double x) { return x; }

// Control words in the workspace.
struct Ctl {
    uint32_t n_items;  // work items (tiles and long-column chunks)
    uint32_t n_bound;  // columns that start a tile or a long column
    uint32_t pad[2];
};

struct Args {
    uint32_t N, scale, cmax, iters;
    const uint32_t *colptr, *rowc;
    const uint32_t *iperm;  // vertex at position p
    const uint64_t *ovf_key;
    const uint32_t *ovf_cnt;
    const uint64_t *info;
    uint32_t *bound;          // [N] boundary columns, ascending (plan)
    uint32_t *bound_item;     // [N] index of each boundary's first work item
    uint4 *item;              // [N + M/CHUNK_MIN + 1] work items, see plan_items_kernel
    double *chunk_sum;        // [same] partial sums of long-column chunks
    uint32_t *ticket;         // [same] finished-chunk counters, at a column's first item
    uint64_t *plan_status;    // [N / PLAN_TILE + 1] look-back words of the plan scan
    unsigned long long *acc;  // [2 * (iters + 1)] sum(r) per iterate, 128-bit fixed point
    int *fx_exp;              // [iters + 1] scale exponent of each accumulator
    double *ipart;            // [SETUP_BLOCKS]
    Ctl *ctl;
    uint32_t *ctr;            // [1] plan tile counter
    double c;
    uint32_t shortmax;    // columns longer than this are cut into chunks (power of two)
    uint32_t chunk;       // entries of a long column per work item
    uint32_t lane_short;  // tile columns up to this long are summed by one lane
    // variants (pp_pagerank_ex); zero / null for the plain iteration
    uint32_t flags;                  // PP_K3_DANGLING | PP_K3_CONVERGE
    double tol;                      // convergence threshold on norm(r_k - r_(k-1), 1)
    unsigned long long *dmass;       // [2 * (iters + 1)] sum of r over dangling rows, per iterate
    unsigned long long *delta;       // [2 * (iters + 1)] norm(r_k - r_(k-1), 1), per iterate
    uint32_t *state;                 // [0] converged, [1] iterations run
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

// ------------------------------------------------------------------- planning

constexpr uint64_t F_AGG = 1ull << 62, F_INC = 2ull << 62;

// Column v starts a work item if it is long, follows a long column, starts in
// a new shortmax-entry span of the entry array, or is a multiple of
// TILE_COLS.  So a tile holds at most TILE_COLS columns, all starting in one
// span, and its last column ends at most shortmax entries past that span:
// at most 2*shortmax entries.
__device__ __forceinline__ uint32_t item_count(const Args &a, uint32_t len) {
    return len > a.shortmax ? (len + a.chunk - 1) / a.chunk : 1u;
}

__device__ __forceinline__ void classify(const Args &a, uint32_t v, bool &bound, uint32_t &nitems) {
    const uint32_t s = __ldg(a.colptr + v), e = __ldg(a.colptr + v + 1);
    const bool is_long = e - s > a.shortmax;
    nitems = item_count(a, e - s);
    bound = true;
    if (v == 0 || is_long || v % TILE_COLS == 0) return;
    const uint32_t ps = __ldg(a.colptr + v - 1);
    if (s - ps > a.shortmax) return;  // the previous column is long
    bound = (s / a.shortmax) != (ps / a.shortmax);
}

// Compacts the boundary columns in order and numbers their work items (one
// look-back scan of two packed counters: boundaries, items).
__global__ void __launch_bounds__(PLAN_THREADS) plan_kernel(Args a) {
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_scan[40];
    __shared__ uint64_t s_excl;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(a.ctr, 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    const uint64_t ntiles = (a.N + PLAN_TILE - 1) / PLAN_TILE;
    if (tile >= ntiles) return;
    const uint64_t v0 = tile * PLAN_TILE + (uint64_t)tid * PLAN_ITEMS;
    uint32_t bmask = 0, nitems = 0;
#pragma unroll
    for (int j = 0; j < PLAN_ITEMS; ++j) {
        const uint64_t v = v0 + j;
        if (v < a.N) {
            bool b;
            uint32_t ni;
            classify(a, (uint32_t)v, b, ni);
            if (b) {
                bmask |= 1u << j;
                nitems += ni;
            }
        }
    }
    // bits 30:0 count boundaries, bits 61:31 work items
    const uint64_t mine = (uint64_t)__popc(bmask) | ((uint64_t)nitems << 31);
    uint64_t total;
    const uint64_t texcl = block_exclusive_sum<uint64_t, PLAN_THREADS>(mine, s_scan, &total);
    if (tid < 32) {
        // warp 0: publish this tile's counts and look back over earlier tiles
        uint64_t *st = a.plan_status + tile;
        uint64_t ex = 0;
        if (tile == 0) {
            if (tid == 0) st_relaxed_u64(st, F_INC | total);
        } else {
            if (tid == 0) st_relaxed_u64(st, F_AGG | total);
            ex = warp_lookback(a.plan_status, tile);
            if (tid == 0) st_relaxed_u64(st, F_INC | (ex + total));
        }
        if (tid == 0) {
            s_excl = ex;
            if (tile == ntiles - 1) {
                const uint64_t inc = ex + total;
                a.ctl->n_bound = (uint32_t)(inc & 0x7fffffffull);
                a.ctl->n_items = (uint32_t)(inc >> 31);
            }
        }
    }
    __syncthreads();
    const uint64_t g = s_excl + texcl;
    uint32_t bi = (uint32_t)(g & 0x7fffffffull), ii = (uint32_t)(g >> 31);
#pragma unroll
    for (int j = 0; j < PLAN_ITEMS; ++j) {
        if (!(bmask >> j & 1u)) continue;
        const uint32_t v = (uint32_t)(v0 + j);
        a.bound[bi] = v;
        a.bound_item[bi] = ii;
        const uint32_t s = __ldg(a.colptr + v), e = __ldg(a.colptr + v + 1);
        ii += item_count(a, e - s);
        ++bi;
    }
}

// Writes the work items of each boundary, so that a warp can start loading
// entries without reading the column pointers first:
//   tile:        (first column, number of columns, first entry, entries)
//   long chunk:  (column | LONG_FLAG, first item of the column, first entry,
//                 entries | chunks of the column << NENT_BITS)
// A tile runs to the next boundary; a long column gets one item per chunk.
__global__ void __launch_bounds__(256) plan_items_kernel(Args a) {
    const uint32_t nb = a.ctl->n_bound;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
        const uint32_t v = a.bound[i], o = a.bound_item[i];
        const uint32_t s = __ldg(a.colptr + v), e = __ldg(a.colptr + v + 1);
        if (e - s > a.shortmax) {
            // a kept column has at most M/2 <= 2^30 entries (the largest one is removed), so nc < 2^19
            const uint32_t nc = (e - s + a.chunk - 1) / a.chunk;
            for (uint32_t k = 0; k < nc; ++k) {
                const uint32_t cs = s + k * a.chunk;
                a.item[o + k] = make_uint4(v | LONG_FLAG, o, cs, min(a.chunk, e - cs) | (nc << NENT_BITS));
                a.ticket[o + k] = 0;
            }
        } else {
            const uint32_t c1 = i + 1 < nb ? a.bound[i + 1] : a.N;
            a.item[o] = make_uint4(v, c1 - v, s, __ldg(a.colptr + c1) - s);
        }
    }
}

// Reset the per-call counters and sum |r0|.
__global__ void __launch_bounds__(256) setup_kernel(Args a, const double *r0) {
    __shared__ double s_red[32];
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (gtid == 0) a.ctr[0] = 0;
    for (uint64_t i = gtid; i < 2ull * (a.iters + 1); i += stride) {
        a.acc[i] = 0;
        if (a.dmass) a.dmass[i] = 0;
        if (a.delta) a.delta[i] = 0;
    }
    if (gtid < 2 && a.state) a.state[gtid] = 0;
    for (uint64_t i = gtid; i < (a.N + PLAN_TILE - 1) / PLAN_TILE; i += stride) a.plan_status[i] = 0;
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
        for (int k = 0; k < R; ++k) v[k] = p0 + k * stride < a.N ? a.iperm[p0 + k * stride] : 0u;
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
            x0[p] = from_acc<TS>(r * iv[k]);
            if (a.iters == 0) r_out[v[k]] = (TO)r;
            if (rb0) rb0[p] = r;
            if ((a.flags & PP_K3_DANGLING) && iv[k] == TA(0)) fx_add(dm, r, 1);
        }
    }
    const Fx128 bt = fx_block_sum<256>(acc, s_fx);
    if (threadIdx.x == 0 && (bt.hi | bt.lo)) fx_atomic_add(a.acc, bt);
    if (a.flags & PP_K3_DANGLING) {
        __syncthreads();
        const Fx128 bd = fx_block_sum<256>(dm, s_fx);
        if (threadIdx.x == 0 && (bd.hi | bd.lo)) fx_atomic_add(a.dmass, bd);
    }
}

// ------------------------------------------------------------- the iteration

// Gathered-vector loads and stores, kept in L2 (evict-last).
__device__ __forceinline__ float ld_x(const float *p, uint64_t pol) { return ld_hint(p, pol); }
__device__ __forceinline__ double ld_x(const double *p, uint64_t pol) { return ld_hint(p, pol); }
__device__ __forceinline__ __nv_bfloat16 ld_x(const __nv_bfloat16 *p, uint64_t pol) {
    return __ushort_as_bfloat16(ld_hint_b16(p, pol));
}
__device__ __forceinline__ void st_x(float *p, float v, uint64_t pol) { st_hint(p, v, pol); }
__device__ __forceinline__ void st_x(double *p, double v, uint64_t pol) { st_hint(p, v, pol); }
__device__ __forceinline__ void st_x(__nv_bfloat16 *p, __nv_bfloat16 v, uint64_t pol) {
    st_hint_b16(p, __bfloat16_as_ushort(v), pol);
}
__device__ __forceinline__ float ld_inv(const float *p, uint64_t pol) { return ld_hint(p, pol); }
__device__ __forceinline__ double ld_inv(const double *p, uint64_t pol) { return ld_hint(p, pol); }

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
    TA cc, tele;
    uint64_t keep, stream;
    int E;
    const uint32_t *iperm;
    const TA *rb_in;
    TA *rb_out;
    uint32_t flags;
    // col is a column position (vertex iperm[col])
    __device__ __forceinline__ void operator()(uint32_t col, TA y, TA inv_col, Sums &acc) const {
        const TA r = cc * y + tele;
        if (LAST && !EXT) r_out[__ldg(iperm + col)] = (TO)r;
        st_x(x_out + col, from_acc<TS>(r * inv_col), keep);
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

// A column sum.  Binary32 (and bfloat16 x): float additions in a fixed
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

// Dynamic shared memory of iterate_kernel: the per-warp product slabs and
// column starts, then the block-sum scratch.
template <typename TA>
struct Smem {
    static constexpr size_t cp(int nw) { return (size_t)nw * TILE_ENTRIES * sizeof(TA); }
    static constexpr size_t fx(int nw) { return (cp(nw) + (size_t)nw * (TILE_COLS + 1) * 4 + 15) & ~(size_t)15; }
    static constexpr size_t total(int nw) { return fx(nw) + (size_t)nw * 2 * 8; }
};

template <typename TS, typename TA, typename TO, bool LAST, int UNROLL, int MINB, bool EXT>
__global__ void __launch_bounds__(THREADS, MINB)
    iterate_kernel(Args a, const TA *inv, const TS *__restrict__ x_in, TS *__restrict__ x_out, TO *r_out,
                   uint32_t iter, const TA *rb_in, TA *rb_out) {
    static_assert(TILE_ENTRIES % (32 * UNROLL) == 0, "unroll must divide the work");
    constexpr int NT = THREADS, NW = WARPS;
    extern __shared__ __align__(16) unsigned char k3_smem[];
    uint64_t *s_fx = reinterpret_cast<uint64_t *>(k3_smem + Smem<TA>::fx(NW));

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double tele_extra = 0.0;
    if (EXT) {
        // the variants: stop once converged; the dangling rows' mass is spread evenly
        if (ld_relaxed_u32(a.state)) return;
        if ((a.flags & PP_K3_CONVERGE) && iter >= 1 &&
            fx_value(a.delta[2 * iter], a.delta[2 * iter + 1], a.fx_exp[iter]) < a.tol) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                a.state[1] = iter;
                st_relaxed_u32(a.state, 1u);
            }
            return;
        }
        if (a.flags & PP_K3_DANGLING)
            tele_extra = a.c / (double)a.N * fx_value(a.dmass[2 * iter], a.dmass[2 * iter + 1], a.fx_exp[iter]);
    }
    const uint32_t n_items = a.ctl->n_items;
    const double S = fx_value(a.acc[2 * iter], a.acc[2 * iter + 1], a.fx_exp[iter]);
    const int E = fx_exponent(S);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.fx_exp[iter + 1] = E;
    const uint32_t umask = (1u << a.scale) - 1u;
    const uint64_t keep = policy_evict_last(), stream = policy_evict_first();
    const Epilogue<TS, TA, TO, LAST, EXT> epi{inv,
                                              x_out,
                                              r_out,
                                              (TA)a.c,
                                              (TA)(((1.0 - a.c) / (double)a.N) * S + tele_extra),
                                              keep,
                                              stream,
                                              E,
                                              a.iperm,
                                              rb_in,
                                              rb_out,
                                              a.flags};
    TA *prod = reinterpret_cast<TA *>(k3_smem) + warp * TILE_ENTRIES;
    uint32_t *cp = reinterpret_cast<uint32_t *>(k3_smem + Smem<TA>::cp(NW)) + warp * (TILE_COLS + 1);
    Sums acc{{0, 0}, {0, 0}, {0, 0}};
    const uint32_t nwarps = gridDim.x * NW;

    uint32_t item = blockIdx.x * NW + warp;
    uint4 it = item < n_items ? __ldg(a.item + item) : make_uint4(0, 0, 0, 0);
    while (item < n_items) {
        // the next item's descriptor is fetched while this one is processed
        const uint32_t next = item + nwarps;
        const uint4 nit = next < n_items ? __ldg(a.item + next) : make_uint4(0, 0, 0, 0);
        const uint32_t e0 = it.z;
        if (it.x & LONG_FLAG) {
            // ---- one chunk of a long column
            const uint32_t col = it.x & ~LONG_FLAG, first = it.y;
            const uint32_t nent = it.w & ((1u << NENT_BITS) - 1), nchunks = it.w >> NENT_BITS;
            ColSum<TA> part;
            for (uint32_t base = 0; base < nent; base += 32 * UNROLL) {
                uint32_t w[UNROLL];
                TA xv[UNROLL];
#pragma unroll
                for (int m = 0; m < UNROLL; ++m) {
                    const uint32_t k = base + (uint32_t)(m * 32 + lane);
                    w[m] = k < nent ? ld_stream_u32(a.rowc + e0 + k, stream) : 0u;
                }
#pragma unroll
                for (int m = 0; m < UNROLL; ++m) {
                    const uint32_t k = base + (uint32_t)(m * 32 + lane);
                    xv[m] = k < nent ? to_acc(ld_x(x_in + (w[m] & umask), keep)) : TA(0);
                }
#pragma unroll
                for (int m = 0; m < UNROLL; ++m) {
                    const uint32_t k = base + (uint32_t)(m * 32 + lane);
                    if (k < nent) part.add(entry_product<TA>(w[m], xv[m], col, a), E);
                }
            }
            const TA y = part.warp_total(E);
            if (lane == 0) {
                if (nchunks == 1) {
                    epi(col, y, ld_inv(inv + col, stream), acc);
                } else {
                    // the warp finishing the column's last chunk adds the chunk sums in order
                    a.chunk_sum[item] = (double)y;
                    __threadfence();
                    const uint32_t t = atomicAdd(a.ticket + first, 1u);
                    if ((t + 1) % nchunks == 0) {
                        __threadfence();
                        TA tot = TA(0);
                        for (uint32_t q = 0; q < nchunks; ++q) tot += (TA)__ldcg(a.chunk_sum + first + q);
                        epi(col, tot, ld_inv(inv + col, stream), acc);
                    }
                }
            }
        } else {
            // ---- a tile of up to 32 short columns
            const uint32_t c0 = it.x, ncol = it.y, nent = it.w;
            // column starts and 1/d_out of lane's column, in flight with the entries
            const uint32_t mycp = lane < (int)ncol ? ld_stream_u32(a.colptr + c0 + lane, stream) : 0u;
            const TA myinv = lane < (int)ncol ? ld_inv(inv + c0 + lane, stream) : TA(0);
#pragma unroll
            for (int g = 0; g < TILE_ENTRIES / 32; g += UNROLL) {
                if ((uint32_t)(g * 32) >= nent) break;
                uint32_t w[UNROLL];
                TA xv[UNROLL];
#pragma unroll
                for (int m = 0; m < UNROLL; ++m) {
                    const uint32_t k = (uint32_t)((g + m) * 32 + lane);
                    w[m] = k < nent ? ld_stream_u32(a.rowc + e0 + k, stream) : 0u;
                }
#pragma unroll
                for (int m = 0; m < UNROLL; ++m) {
                    const uint32_t k = (uint32_t)((g + m) * 32 + lane);
                    xv[m] = k < nent ? to_acc(ld_x(x_in + (w[m] & umask), keep)) : TA(0);
                }
                if (g == 0) {
                    if (lane < (int)ncol) cp[lane] = mycp - e0;
                    if (lane == 0) cp[ncol] = nent;
                    __syncwarp();
                }
#pragma unroll
                for (int m = 0; m < UNROLL; ++m) {
                    const uint32_t k = (uint32_t)((g + m) * 32 + lane);
                    if (k < nent) {
                        uint32_t col = 0;
                        if ((w[m] >> a.scale) == a.cmax) {
                            // the count did not fit inline: find this entry's column
                            uint32_t lo = 0, hi = ncol;
                            while (lo < hi) {
                                const uint32_t mid = (lo + hi) >> 1;
                                if (cp[mid + 1] <= k)
                                    lo = mid + 1;
                                else
                                    hi = mid;
                            }
                            col = c0 + lo;
                        }
                        prod[k] = entry_product<TA>(w[m], xv[m], col, a);
                    }
                }
            }
            if (nent == 0) {
                if (lane < (int)ncol) cp[lane] = mycp - e0;
                if (lane == 0) cp[ncol] = nent;
            }
            __syncwarp();
            // short columns: one lane each, entries in order
            uint32_t medium = 0;
            if (lane < (int)ncol) {
                const uint32_t s = cp[lane], e = cp[lane + 1];
                if (e - s <= a.lane_short) {
                    ColSum<TA> y;
                    for (uint32_t k = s; k < e; ++k) y.add(prod[k], E);
                    epi(c0 + lane, y.value(E), myinv, acc);
                } else {
                    medium = 1;
                }
            }
            // medium columns: the whole warp, lanes stride, fixed shuffle tree
            uint32_t mm = __ballot_sync(0xffffffffu, medium);
            while (mm) {
                const int j = __ffs(mm) - 1;
                mm &= mm - 1;
                const uint32_t s = cp[j], e = cp[j + 1];
                ColSum<TA> y;
                for (uint32_t k = s + lane; k < e; k += 32) y.add(prod[k], E);
                const TA yt = y.warp_total(E);
                const TA invj = __shfl_sync(0xffffffffu, myinv, j);
                if (lane == 0) epi(c0 + j, yt, invj, acc);
            }
            __syncwarp();
        }
        item = next;
        it = nit;
    }
    const Fx128 bt = fx_block_sum<NT>(acc.s, s_fx);
    if (threadIdx.x == 0 && (bt.hi | bt.lo)) fx_atomic_add(a.acc + 2 * (iter + 1), bt);
    if (EXT && (a.flags & PP_K3_DANGLING)) {
        __syncthreads();
        const Fx128 bd = fx_block_sum<NT>(acc.dm, s_fx);
        if (threadIdx.x == 0 && (bd.hi | bd.lo)) fx_atomic_add(a.dmass + 2 * (iter + 1), bd);
    }
    if (EXT && (a.flags & PP_K3_CONVERGE)) {
        __syncthreads();
        const Fx128 bf = fx_block_sum<NT>(acc.df, s_fx);
        if (threadIdx.x == 0 && (bf.hi | bf.lo)) fx_atomic_add(a.delta + 2 * (iter + 1), bf);
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
        r_out[a.iperm[p]] = (TO)rb[p];
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
    uint32_t *bound, *bound_item;
    uint4 *item;
    double *chunk_sum;
    uint32_t *ticket;
    uint64_t *plan_status;
    unsigned long long *acc;
    int *fx_exp;
    double *ipart;
    Ctl *ctl;
    uint32_t *ctr;
    // the variants only
    void *rb[2];  // r in storage order (TA), ping-pong
    unsigned long long *dmass, *delta;
    uint32_t *state;
    size_t bytes;
};

inline Layout layout(void *ws, uint64_t M, uint32_t scale, uint32_t iters, pp_dtype dt, bool ext = false) {
    Carver c(ws);
    Layout L;
    const uint64_t N = 1ull << scale;
    const uint64_t max_items = N + M / CHUNK_MIN + 1;
    const size_t xs = dt == PP_FP64 ? 8 : (dt == PP_FP32 ? 4 : 2);
    L.x[0] = c.take<char>(N * xs);
    L.x[1] = c.take<char>(N * xs);
    L.invp = c.take<char>(N * (dt == PP_FP64 ? 8 : 4));
    L.bound = c.take<uint32_t>(N);
    L.bound_item = c.take<uint32_t>(N);
    L.item = c.take<uint4>(max_items);
    L.chunk_sum = c.take<double>(max_items);
    L.ticket = c.take<uint32_t>(max_items);
    L.plan_status = c.take<uint64_t>(ceil_div(N, PLAN_TILE));
    L.acc = c.take<unsigned long long>(2ull * (iters + 1));
    L.fx_exp = c.take<int>((uint64_t)iters + 1);
    L.ipart = c.take<double>(SETUP_BLOCKS);
    L.ctl = c.take<Ctl>(1);
    L.ctr = c.take<uint32_t>(1);
    L.rb[0] = L.rb[1] = nullptr;
    L.dmass = L.delta = nullptr;
    L.state = nullptr;
    if (ext) {
        const size_t ta = dt == PP_FP64 ? 8 : 4;
        L.rb[0] = c.take<char>(N * ta);
        L.rb[1] = c.take<char>(N * ta);
        L.dmass = c.take<unsigned long long>(2ull * (iters + 1));
        L.delta = c.take<unsigned long long>(2ull * (iters + 1));
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
    a.bound = L.bound;
    a.bound_item = L.bound_item;
    a.item = L.item;
    a.chunk_sum = L.chunk_sum;
    a.ticket = L.ticket;
    a.plan_status = L.plan_status;
    a.acc = L.acc;
    a.fx_exp = L.fx_exp;
    a.ipart = L.ipart;
    a.ctl = L.ctl;
    a.ctr = L.ctr;
    a.c = c;
    a.shortmax = (uint32_t)tuning("k3_shortmax");
    a.chunk = (uint32_t)tuning("k3_chunk");
    a.lane_short = (uint32_t)tuning("k3_lane_short");
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
    plan_kernel<<<(unsigned)ceil_div(N, PLAN_TILE), PLAN_THREADS, 0, s>>>(a);
    plan_items_kernel<<<(unsigned)std::min<uint64_t>(ceil_div(N, 256), 4096), 256, 0, s>>>(a);
    TA *invp = static_cast<TA *>(L.invp);  // 1/d_out in storage order
    // one wave of blocks (each sums the norm's partials once)
    const unsigned nblocks = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(ceil_div(N, 256), 8ull * sm_count()));
    normalize_kernel<TS, TA, TO><<<nblocks, 256, 0, s>>>(a, r0, inv, invp, x0, r_out, EXT ? rb0 : nullptr);
    count_launch(4);

    auto *k_mid = iterate_kernel<TS, TA, TO, false, UNROLL, MINB, EXT>;
    auto *k_last = iterate_kernel<TS, TA, TO, !EXT, UNROLL, MINB, EXT>;
    constexpr int NT = THREADS;
    constexpr size_t smem = Smem<TA>::total(WARPS);
    // the carveout attributes and the occupancy, once per instantiation and device
    static PerDevice cached;  // o_mid << 16 | o_last
    const uint32_t cv = (uint32_t)cached.get([&] {
        set_smem(k_mid, MINB, smem);
        set_smem(k_last, MINB, smem);
        return (int64_t)(((uint32_t)occupancy(k_mid, NT, smem) << 16) | (uint32_t)occupancy(k_last, NT, smem));
    });
    const int o_mid = (int)(cv >> 16), o_last = (int)(cv & 0xffff);
    const int sms = sm_count();
    for (uint32_t it = 0; it < iters; ++it) {
        const TS *xin = (it & 1) ? x1 : x0;
        TS *xout = (it & 1) ? x0 : x1;
        const TA *rin = (it & 1) ? rb1 : rb0;
        TA *rout = (it & 1) ? rb0 : rb1;
        // the variants write r every iteration and finish_kernel picks the last one
        if (it + 1 == iters && !EXT)
            k_last<<<sms * o_last, NT, smem, s>>>(a, invp, xin, xout, r_out, it, rin, rout);
        else
            k_mid<<<sms * o_mid, NT, smem, s>>>(a, invp, xin, xout, r_out, it, rin, rout);
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
        case 5:
            return u4 ? run_unroll<TS, TA, TO, 4, 5, false>(g, r0, iters, c, dt, r_out, r_l1, L, s, none)
                      : run_unroll<TS, TA, TO, 8, 5, false>(g, r0, iters, c, dt, r_out, r_l1, L, s, none);
        case 6:
            return u4 ? run_unroll<TS, TA, TO, 4, 6, false>(g, r0, iters, c, dt, r_out, r_l1, L, s, none)
                      : run_unroll<TS, TA, TO, 8, 6, false>(g, r0, iters, c, dt, r_out, r_l1, L, s, none);
        default:
            return u4 ? run_unroll<TS, TA, TO, 4, 4, false>(g, r0, iters, c, dt, r_out, r_l1, L, s, none)
                      : run_unroll<TS, TA, TO, 8, 4, false>(g, r0, iters, c, dt, r_out, r_l1, L, s, none);
    }
}

// The variants run one instantiation (unroll 4, 4 blocks per SM).
template <typename TS, typename TA, typename TO>
pp_status run_ext(const pp_graph *g, const double *r0, uint32_t iters, double c, pp_dtype dt, TO *r_out,
                  double *r_l1, const Layout &L, cudaStream_t s, const Variant &var) {
    return run_unroll<TS, TA, TO, 4, 4, true>(g, r0, iters, c, dt, r_out, r_l1, L, s, var);
}

}  // namespace k3
}  // namespace pp

using namespace pp;

extern "C" pp_status pp_pagerank_workspace(uint64_t M, uint32_t scale, uint32_t iters, pp_dtype dt,
                                           size_t *bytes) {
    if (!bytes || scale < 1 || scale > 27 || M > (1ull << 31) || (int)dt < 0 || (int)dt > 2)
        return PP_ERR_INVALID_ARG;
    *bytes = k3::layout(nullptr, M, scale, iters, dt).bytes;
    return PP_OK;
}

extern "C" pp_status pp_pagerank(const pp_graph *g, const double *r0, uint32_t iters, double c, pp_dtype dt,
                                 void *r_out, double *r_l1, void *ws, size_t ws_bytes, void *stream) {
    if (!g || !r0 || !r_out || (int)dt < 0 || (int)dt > 2) return PP_ERR_INVALID_ARG;
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
        default:
            return k3::run<__nv_bfloat16, float, float>(g, r0, iters, c, dt, static_cast<float *>(r_out), r_l1, L,
                                                        s);
    }
}

extern "C" pp_status pp_pagerank_ex_workspace(uint64_t M, uint32_t scale, uint32_t iters, pp_dtype dt,
                                              size_t *bytes) {
    if (!bytes || scale < 1 || scale > 27 || M > (1ull << 31) || (int)dt < 0 || (int)dt > 2)
        return PP_ERR_INVALID_ARG;
    *bytes = k3::layout(nullptr, M, scale, iters, dt, true).bytes;
    return PP_OK;
}

extern "C" pp_status pp_pagerank_ex(const pp_graph *g, const double *r0, uint32_t iters, double c, pp_dtype dt,
                                    uint32_t flags, double tol, void *r_out, double *r_l1, uint32_t *iters_done,
                                    void *ws, size_t ws_bytes, void *stream) {
    if (!g || !r0 || !r_out || (int)dt < 0 || (int)dt > 2) return PP_ERR_INVALID_ARG;
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
        default:
            return k3::run_ext<__nv_bfloat16, float, float>(g, r0, iters, c, dt, static_cast<float *>(r_out), r_l1, L,
                                                            s, var);
    }
}
