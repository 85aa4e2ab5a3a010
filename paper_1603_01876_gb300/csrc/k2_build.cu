// Kernel 2 (Sec. IV-C): build, filter and normalise the adjacency matrix.
//
//   unique_kernel    step 1: run-lengths of equal (u, v) in Kernel 1's sorted
//                    output are the counts A(u,v); output offsets by a
//                    decoupled look-back over tiles.  Each entry is written
//                    as one 64-bit word (column << 32 | row | count << scale)
//                    in vertex order, its column digits go to the
//                    transpose's histograms, and each row's edges (the
//                    out-degree before filtering) and entries are counted.
//   relabel          rows ordered by decreasing floor(log2(out-degree)),
//                    vertex id breaking ties (a one-pass radix sort of the
//                    vertices): perm / iperm, the storage order of the rows
//                    and columns that Kernel 3 gathers from.
//   transpose        stable LSD radix sort of the entry words by column; the
//                    first pass puts each row's position in place of its
//                    vertex id (reading perm in ascending vertex order), and
//                    inside a column the rows stay in vertex order.
//   colscan_kernel   step 2: with the entries grouped by column, the entry
//                    count and d_in = sum(A,1) of each column, one atomic per
//                    run of a column inside a thread's stretch.
//   dmax_kernel      d_in out; max(d_in) and its lowest column.
//   mask_scan_kernel step 3: the supernode and leaf columns, and each
//                    column's first entry in the sorted words (look-back scan).
//   pos_scan_kernel  the column pointers of the kept entries with the
//                    columns in storage order (vertex iperm[p] at position p;
//                    look-back scan), so that Kernel 3 writes x in the order
//                    it gathers it.
//   compact_kernel   step 4: kept entries move to their column's place in
//                    storage order; a removed entry's count comes off its
//                    row's out-degree (d_out = sum(A,2) after the filter).
//   finalize_kernel  1/d_out in binary32 and binary64.
// Every pass after the unique pass streams the entries in column order, so
// the per-column lookups are nearly sequential and no atomic is issued per
// entry.
#include <algorithm>

#include "onesweep.cuh"

PP_DEFINE_ERROR_WORD(k2_fetch_error)

namespace pp {
namespace k2 {

constexpr int UQ_THREADS = 256;
constexpr int UQ_ITEMS = 16;
constexpr int UQ_TILE = UQ_THREADS * UQ_ITEMS;
constexpr int SC_THREADS = 256;
constexpr int SC_ITEMS = 16;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

constexpr uint64_t F_AGG = 1ull << 62, F_INC = 2ull << 62;

__device__ __forceinline__ uint64_t uq_tiles(uint64_t M) { return (M + UQ_TILE - 1) / UQ_TILE; }

__device__ __forceinline__ uint64_t edge_key(const uint32_t *us, const uint32_t *vs, uint64_t i) {
    return ((uint64_t)__ldg(us + i) << 32) | (uint64_t)__ldg(vs + i);
}

// Exclusive block max-scan of one int64 per thread (identity -1).
__device__ __forceinline__ long long block_exclusive_max(long long x, long long *scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc = max(inc, y);
    }
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    long long before = -1;
    for (int w = 0; w < warp; ++w) before = max(before, scratch[w]);
    long long ex = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) ex = -1;
    __syncthreads();
    return max(before, ex);
}

__device__ __forceinline__ uint32_t ovf_lookup(const uint64_t *keys, const uint32_t *cnts, uint64_t n,
                                               uint64_t key) {
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (keys[mid] < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < n && keys[lo] == key) ? cnts[lo] : 0u;
}

// Run by one whole warp: publishes a tile's aggregate, looks back over the
// earlier tiles and publishes the inclusive prefix; lane 0 stores the tile's
// exclusive prefix in *s_excl.
__device__ __forceinline__ void warp_tile_prefix(uint64_t *status, uint64_t tile, uint64_t total,
                                                 uint64_t *s_excl) {
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) {
            st_relaxed_u64(status, F_INC | total);
            *s_excl = 0;
        }
        return;
    }
    if (lane == 0) st_relaxed_u64(status + tile, F_AGG | total);
    const uint64_t ex = warp_lookback(status, tile);
    if (lane == 0) {
        st_relaxed_u64(status + tile, F_INC | (ex + total));
        *s_excl = ex;
    }
}

struct UniqueArgs {
    const uint32_t *us, *vs;
    uint64_t M;
    uint32_t scale, cmax;
    unsigned long long *ent;  // [nnz0] column << 32 | row | count field << scale
    uint64_t *ovf_key;
    uint32_t *ovf_cnt;
    uint32_t n_vert;          // N
    uint32_t *d_out;          // [N] edges of each row (the out-degree before the filters), zero on entry
    uint32_t *row_nent;       // [N] entries (distinct (u, v)) of each row, zero on entry (nullptr: not wanted)
    uint32_t *hist;           // [npasses * 256] column digits, for the transpose
    int npasses;
    int vec;                  // us and vs are 16-byte aligned: load 4 ids at a time
    uint64_t *status;
    uint32_t *tile_ctr;
    uint64_t *info;
};

// Persistent: each block claims tiles in order until none is left.
__global__ void __launch_bounds__(UQ_THREADS, 3) unique_kernel(UniqueArgs a) {
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_scan[40];
    __shared__ long long s_max[UQ_THREADS / 32];
    __shared__ uint64_t s_excl;
    __shared__ uint32_t s_hist[os::MAX_PASSES][os::RADIX];
    // the tile's entries, written out coalesced; one pad word per 16 so that
    // the threads' consecutive runs of stores hit different banks
    __shared__ unsigned long long s_out[UQ_TILE + UQ_TILE / 16];
    const int tid = threadIdx.x;
    for (int i = tid; i < os::MAX_PASSES * os::RADIX; i += UQ_THREADS) (&s_hist[0][0])[i] = 0;
    const uint64_t ntiles = uq_tiles(a.M);
    while (true) {
        if (tid == 0) s_tile = atomicAdd(a.tile_ctr, 1u);
        __syncthreads();
        const uint64_t tile = s_tile;
        if (tile >= ntiles) break;
        const uint64_t base = tile * UQ_TILE;
        const uint64_t my0 = base + (uint64_t)tid * UQ_ITEMS;

        uint64_t k[UQ_ITEMS];
        if (a.vec && my0 + UQ_ITEMS <= a.M) {
            const uint4 *pu = reinterpret_cast<const uint4 *>(a.us + my0);
            const uint4 *pv = reinterpret_cast<const uint4 *>(a.vs + my0);
#pragma unroll
            for (int q = 0; q < UQ_ITEMS / 4; ++q) {
                const uint4 x = __ldg(pu + q), y = __ldg(pv + q);
                k[4 * q + 0] = ((uint64_t)x.x << 32) | y.x;
                k[4 * q + 1] = ((uint64_t)x.y << 32) | y.y;
                k[4 * q + 2] = ((uint64_t)x.z << 32) | y.z;
                k[4 * q + 3] = ((uint64_t)x.w << 32) | y.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < UQ_ITEMS; ++j) k[j] = (my0 + j < a.M) ? edge_key(a.us, a.vs, my0 + j) : ~0ull;
        }
        const uint64_t knext = (my0 + UQ_ITEMS < a.M) ? edge_key(a.us, a.vs, my0 + UQ_ITEMS) : ~0ull;

        // each row's edges (the out-degree before the filters) and entries,
        // one atomic per array for each run of a row in this thread's edges;
        // an edge with an id >= N is no edge of any row (reported below)
        {
            uint32_t row = 0xffffffffu, edges = 0, entries = 0;
#pragma unroll
            for (int j = 0; j < UQ_ITEMS; ++j) {
                if (my0 + j >= a.M) break;
                if ((k[j] >> 32) >= (uint64_t)a.n_vert || (uint32_t)k[j] >= a.n_vert) continue;
                const uint32_t u = (uint32_t)(k[j] >> 32);
                if (u != row) {
                    if (edges) {
                        atomicAdd(&a.d_out[row], edges);
                        if (a.row_nent) atomicAdd(&a.row_nent[row], entries);
                    }
                    row = u;
                    edges = entries = 0;
                }
                ++edges;
                entries += k[j] != (j + 1 < UQ_ITEMS ? k[j + 1] : knext);  // a run of equal (u, v) ends here
            }
            if (edges) {
                atomicAdd(&a.d_out[row], edges);
                if (a.row_nent) atomicAdd(&a.row_nent[row], entries);
            }
        }

        // A run ends ("tail") where the next key differs.
        uint32_t tails = 0;
        int last_tail = -1;
#pragma unroll
        for (int j = 0; j < UQ_ITEMS; ++j) {
            const uint64_t nx = j + 1 < UQ_ITEMS ? k[j + 1] : knext;
            if (my0 + j < a.M && k[j] != nx) {
                tails |= 1u << j;
                last_tail = j;
            }
        }
        const long long prev_tail =
            block_exclusive_max(last_tail >= 0 ? (long long)(my0 + last_tail) : -1ll, s_max);

        // Start of the run of this thread's first tail.
        uint64_t start = (uint64_t)(prev_tail + 1);
        if (prev_tail < 0) {
            start = base;
            const int first = tails ? __ffs(tails) - 1 : -1;
            uint64_t K = 0;
#pragma unroll
            for (int j = 0; j < UQ_ITEMS; ++j)
                if (j == first) K = k[j];
            if (first >= 0 && base > 0 && edge_key(a.us, a.vs, base - 1) == K) {
                // The run began in an earlier tile: gallop back, then bisect.
                uint64_t hi = base - 1, step = 1;
                long long lo = -1;
                while (true) {
                    if (hi < step) break;
                    const uint64_t p = hi - step;
                    if (edge_key(a.us, a.vs, p) != K) {
                        lo = (long long)p;
                        break;
                    }
                    hi = p;
                    step <<= 1;
                }
                while ((long long)hi - lo > 1) {
                    const uint64_t mid = (uint64_t)((lo + (long long)hi) >> 1);
                    if (edge_key(a.us, a.vs, mid) == K)
                        hi = mid;
                    else
                        lo = (long long)mid;
                }
                start = hi;
            }
        }

        // Runs of an id >= N are not entries (reported; the stats pass skips them too,
        // so row counts and entries agree and every write stays in bounds).
        uint32_t valid = 0;
#pragma unroll
        for (int j = 0; j < UQ_ITEMS; ++j)
            if ((tails >> j & 1u) && !((k[j] >> 32) >= (uint64_t)a.n_vert || (uint32_t)k[j] >= a.n_vert))
                valid |= 1u << j;
        if (valid != tails) pp_set_error(PP_DEV_RANGE);
        const uint64_t start0 = start;
        uint32_t nt = 0, ne = 0;
#pragma unroll
        for (int j = 0; j < UQ_ITEMS; ++j) {
            if (tails >> j & 1u) {
                if (valid >> j & 1u) {
                    ne += (uint32_t)(my0 + j - start + 1) >= a.cmax;
                    ++nt;
                }
                start = my0 + j + 1;
            }
        }
        start = start0;

        // bits 61:32 count overflow entries, bits 31:0 entries
        uint64_t total;
        const uint64_t mine = ((uint64_t)ne << 32) | nt;
        const uint64_t texcl = block_exclusive_sum<uint64_t, UQ_THREADS>(mine, s_scan, &total);
        if (tid < 32) warp_tile_prefix(a.status, tile, total, &s_excl);
        __syncthreads();
        if (tid == 0 && tile == ntiles - 1) {
            const uint64_t inc = s_excl + total;
            a.info[PP_INFO_NNZ0] = inc & 0xffffffffull;
            a.info[PP_INFO_NOVF] = (inc >> 32) & 0x3fffffffull;
        }
        const uint64_t gex = s_excl + texcl;
        uint32_t lpos = (uint32_t)texcl;  // place inside the tile's output
        uint64_t epos = (gex >> 32) & 0x3fffffffull;

#pragma unroll
        for (int j = 0; j < UQ_ITEMS; ++j) {
            if (!(tails >> j & 1u)) continue;
            const uint32_t c = (uint32_t)(my0 + j - start + 1);
            start = my0 + j + 1;
            if (!(valid >> j & 1u)) continue;
            const uint32_t u = (uint32_t)(k[j] >> 32), v = (uint32_t)k[j];
            const uint32_t field = c >= a.cmax ? a.cmax : c;
            const uint32_t lp = pp_idx(lpos, (uint32_t)UQ_TILE);
            s_out[lp + lp / 16] = ((unsigned long long)v << 32) | (u | (field << a.scale));
            if (c >= a.cmax) {
                // the overflow table holds M / cmax + 1 entries
                const uint64_t eo = pp_idx(epos, a.M / a.cmax + 1);
                a.ovf_key[eo] = ((uint64_t)u << 32) | v;
                a.ovf_cnt[eo] = c;
                ++epos;
            }
            for (int p = 0; p < a.npasses; ++p) atomicAdd(&s_hist[p][(v >> (8 * p)) & (os::RADIX - 1)], 1u);
            ++lpos;
        }
        __syncthreads();
        {
            // the tile's entries in vertex order, one coalesced run
            const uint64_t first = s_excl & 0xffffffffull;
            const uint32_t n_out = (uint32_t)total;
            for (uint32_t i = tid; i < n_out; i += UQ_THREADS) a.ent[pp_idx(first + i, a.M)] = s_out[i + i / 16];
        }
        __syncthreads();  // shared scratch is reused by the next tile
    }
    __syncthreads();
    for (int i = tid; i < a.npasses * os::RADIX; i += UQ_THREADS) {
        const uint32_t c = (&s_hist[0][0])[i];
        if (c) atomicAdd(&a.hist[i], c);
    }
}

constexpr int CS_ITEMS = 8;
constexpr int CS_TILE = 256 * CS_ITEMS;

// In-degree and entry count of each column from the column-sorted entries.
// A block stages a tile through shared memory (coalesced reads), then each
// thread sums the runs of equal columns in its CS_ITEMS consecutive entries
// and adds each run with one atomic.
__global__ void __launch_bounds__(256) colscan_kernel(const unsigned long long *ent, const uint64_t *info,
                                                      uint32_t scale, uint32_t cmax, const uint64_t *ovf_key,
                                                      const uint32_t *ovf_cnt, const uint32_t *iperm,
                                                      unsigned long long *deg) {
    // row stride CS_ITEMS + 1 words: a half-warp's reads of its own rows hit distinct banks
    __shared__ unsigned long long s[256 * (CS_ITEMS + 1)];
    const int tid = threadIdx.x;
    const uint64_t n = info[PP_INFO_NNZ0];
    const uint64_t novf = info[PP_INFO_NOVF];
    const uint32_t umask = (1u << scale) - 1u;
    for (uint64_t t0 = (uint64_t)blockIdx.x * CS_TILE; t0 < n; t0 += (uint64_t)gridDim.x * CS_TILE) {
#pragma unroll
        for (int r = 0; r < CS_ITEMS; ++r) {
            const uint32_t k = tid + 256 * r;
            if (t0 + k < n) s[(k / CS_ITEMS) * (CS_ITEMS + 1) + k % CS_ITEMS] = ent[t0 + k];
        }
        __syncthreads();
        uint32_t col = 0xffffffffu;
        unsigned long long acc = 0;
        const uint64_t i0 = t0 + (uint64_t)tid * CS_ITEMS;
#pragma unroll
        for (int j = 0; j < CS_ITEMS; ++j) {
            if (i0 + j < n) {
                const unsigned long long e = s[tid * (CS_ITEMS + 1) + j];
                const uint32_t v = pp_idx((uint32_t)(e >> 32), umask + 1ull), w = (uint32_t)e;
                uint32_t c = w >> scale;
                if (c == cmax) c = ovf_lookup(ovf_key, ovf_cnt, novf, ((uint64_t)iperm[w & umask] << 32) | v);
                if (v != col) {
                    if (acc) atomicAdd(&deg[col], acc);
                    col = v;
                    acc = 0;
                }
                acc += (1ull << 32) | (unsigned long long)c;
            }
        }
        if (acc) atomicAdd(&deg[col], acc);
        __syncthreads();
    }
}

constexpr uint32_t KILL_BIT = 1u << 31;
constexpr int CP_ITEMS = 4;

// Step 4 over the column-sorted entries.  vstart[v] is column v's first entry
// in the sorted words, with the removal flag in bit 31; a kept entry moves to
// colptr[perm[v]] + its place inside the column; a removed entry's count
// leaves its row's out-degree.
__global__ void __launch_bounds__(256) compact_kernel(const unsigned long long *ent, const uint64_t *info,
                                                      uint32_t scale, uint32_t cmax, const uint64_t *ovf_key,
                                                      const uint32_t *ovf_cnt, const uint32_t *perm,
                                                      const uint32_t *iperm, const uint32_t *vstart,
                                                      const uint32_t *colptr, uint32_t *rowc, uint32_t *d_out) {
    const uint64_t n = info[PP_INFO_NNZ0];
    const uint64_t novf = info[PP_INFO_NOVF];
    const uint32_t umask = (1u << scale) - 1u;
    const uint64_t step = (uint64_t)gridDim.x * 256 * CP_ITEMS;
    for (uint64_t b = (uint64_t)blockIdx.x * 256 * CP_ITEMS + threadIdx.x; b < n; b += step) {
        unsigned long long e[CP_ITEMS];
        uint32_t sv[CP_ITEMS];
#pragma unroll
        for (int q = 0; q < CP_ITEMS; ++q) e[q] = (b + 256 * q < n) ? ent[b + 256 * q] : 0ull;
#pragma unroll
        for (int q = 0; q < CP_ITEMS; ++q)
            sv[q] = (b + 256 * q < n) ? vstart[pp_idx((uint32_t)(e[q] >> 32), umask + 1ull)] : 0u;
#pragma unroll
        for (int q = 0; q < CP_ITEMS; ++q) {
            const uint64_t i = b + 256 * q;
            if (i >= n) break;
            const uint32_t v = pp_idx((uint32_t)(e[q] >> 32), umask + 1ull), w = (uint32_t)e[q];
            if (sv[q] & KILL_BIT) {
                const uint32_t u = pp_idx(iperm[w & umask], umask + 1ull);
                uint32_t c = w >> scale;
                if (c == cmax) c = ovf_lookup(ovf_key, ovf_cnt, novf, ((uint64_t)u << 32) | v);
                atomicSub(&d_out[u], c);
            } else {
                // rowc holds nnz <= nnz0 = n words
                rowc[pp_idx(__ldg(colptr + pp_idx(__ldg(perm + v), umask + 1ull)) + ((uint32_t)i - sv[q]), n)] = w;
            }
        }
    }
}

// d_in out; max(d_in) with the lowest vertex attaining it.
__global__ void __launch_bounds__(256) dmax_kernel(const unsigned long long *deg, uint32_t N, uint32_t *d_in,
                                                   unsigned long long *dmaxkey) {
    unsigned long long best = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
        const uint32_t d = (uint32_t)deg[v];
        d_in[v] = d;
        const unsigned long long key = ((unsigned long long)d << 32) | (unsigned long long)(~v);
        best = key > best ? key : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_down_sync(0xffffffffu, best, o);
        best = y > best ? y : best;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(dmaxkey, best);
}

constexpr int MAX_G = PP_BATCH_MAX_GRAPHS;

// A batch's union vertex space: graph g owns union ids vbase[g] .. vbase[g+1]-1;
// ids from vbase[n] on belong to no graph (padding up to a power of two).
struct VBases {
    uint32_t n;
    uint32_t vbase[MAX_G + 1];
};

// graph owning union id v (n for the padding)
__device__ __forceinline__ uint32_t graph_of(const VBases &b, uint32_t v) {
    if (v >= b.vbase[b.n]) return b.n;
    uint32_t lo = 0, hi = b.n - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (b.vbase[mid] <= v)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// The batch's d_in out; per graph max(d_in) with its lowest vertex (one
// atomic per graph a thread's 16 consecutive vertices touch).
__global__ void __launch_bounds__(256) dmax_batched_kernel(const unsigned long long *deg, uint32_t N, VBases vb,
                                                           uint32_t *d_in, unsigned long long *dmaxkeys) {
    constexpr int ITEMS = 16;
    for (uint64_t v0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * ITEMS; v0 < N;
         v0 += (uint64_t)gridDim.x * blockDim.x * ITEMS) {
        uint32_t gr = graph_of(vb, (uint32_t)v0);
        unsigned long long best = 0;
        for (int j = 0; j < ITEMS && v0 + j < N; ++j) {
            const uint32_t v = (uint32_t)(v0 + j);
            const uint32_t d = (uint32_t)deg[v];
            d_in[v] = d;
            if (gr < vb.n && v >= vb.vbase[gr + 1]) {
                atomicMax(&dmaxkeys[gr], best);
                best = 0;
                gr = graph_of(vb, v);
            }
            const unsigned long long key = ((unsigned long long)d << 32) | (unsigned long long)(~v);
            best = key > best ? key : best;
        }
        if (gr < vb.n) atomicMax(&dmaxkeys[gr], best);
    }
}

struct ScanArgs {
    const unsigned long long *deg;  // entries << 32 | d_in, per vertex
    uint32_t N;
    int all_ties;
    const unsigned long long *dmaxkey;  // batch: one per graph
    uint32_t *vstart;  // first entry of each column in the sorted words | KILL_BIT
    uint64_t *status;
    uint32_t *tile_ctr;
    uint64_t *info;
    // a batch (union of graphs): each column is tested against its own
    // graph's maximum, and ties / supernodes are counted per graph
    int batched;
    unsigned long long *gcount;  // [2 * n]: ties, supernodes
    VBases vb;
};

__global__ void __launch_bounds__(SC_THREADS) mask_scan_kernel(ScanArgs a) {
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_scan[40];
    __shared__ uint64_t s_excl;
    __shared__ unsigned long long s_red[2][SC_THREADS / 32];
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(a.tile_ctr, 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    const uint64_t ntiles = (a.N + SC_TILE - 1) / SC_TILE;
    if (tile >= ntiles) return;
    const uint64_t v0 = tile * SC_TILE + (uint64_t)tid * SC_ITEMS;
    uint32_t gr = a.batched && v0 < a.N ? graph_of(a.vb, (uint32_t)v0) : 0u;
    unsigned long long key = a.dmaxkey[a.batched ? min(gr, a.vb.n - 1) : 0u];
    uint32_t dmax = (uint32_t)(key >> 32);
    uint32_t vmax = ~(uint32_t)key;
    uint32_t ent[SC_ITEMS], killed = 0;
    uint64_t sum = 0;
    unsigned long long ties = 0, sup = 0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        const uint64_t v = v0 + j;
        ent[j] = 0;
        if (v < a.N) {
            const unsigned long long w = a.deg[v];
            const uint32_t din = (uint32_t)w;
            ent[j] = (uint32_t)(w >> 32);
            if (a.batched) {
                while (gr < a.vb.n && (uint32_t)v >= a.vb.vbase[gr + 1]) {
                    ++gr;
                    if (gr < a.vb.n) {
                        key = a.dmaxkey[gr];
                        dmax = (uint32_t)(key >> 32);
                        vmax = ~(uint32_t)key;
                    }
                }
                if (gr >= a.vb.n) {  // padding: no graph, no entries
                    sum += ent[j];
                    continue;
                }
            }
            const bool is_max = din == dmax && (a.all_ties || (uint32_t)v == vmax);
            if (a.batched) {
                if (din == dmax) atomicAdd(&a.gcount[2 * gr], 1ull);
                if (is_max) atomicAdd(&a.gcount[2 * gr + 1], 1ull);
            }
            ties += din == dmax;
            sup += is_max;
            killed |= (uint32_t)(is_max || din == 1) << j;
            sum += ent[j];
        }
    }
    uint64_t total;
    const uint64_t ex = block_exclusive_sum<uint64_t, SC_THREADS>(sum, s_scan, &total);
    if (tid < 32) warp_tile_prefix(a.status, tile, total, &s_excl);
    __syncthreads();
    if (tid == 0 && tile == ntiles - 1 && !a.batched) {
        a.info[PP_INFO_DMAX] = dmax;
        a.info[PP_INFO_VMAX] = vmax;
    }
    uint64_t run = s_excl + ex;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        // every start is below nnz0 <= 2^31, so bit 31 is free for the flag
        if (v0 + j < a.N) a.vstart[v0 + j] = (uint32_t)run | ((killed >> j & 1u) ? KILL_BIT : 0u);
        run += ent[j];
    }
    // tie and supernode counts
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ties += __shfl_down_sync(0xffffffffu, ties, o);
        sup += __shfl_down_sync(0xffffffffu, sup, o);
    }
    if ((tid & 31) == 0) {
        s_red[0][tid >> 5] = ties;
        s_red[1][tid >> 5] = sup;
    }
    __syncthreads();
    if (tid == 0 && !a.batched) {
        unsigned long long t = 0, s = 0;
        for (int w = 0; w < SC_THREADS / 32; ++w) {
            t += s_red[0][w];
            s += s_red[1][w];
        }
        if (t) atomicAdd((unsigned long long *)&a.info[PP_INFO_TIES], t);
        if (s) atomicAdd((unsigned long long *)&a.info[PP_INFO_SUPERNODES], s);
    }
}

// Column pointers of the kept entries, columns in storage order.
struct PosArgs {
    const unsigned long long *deg;
    const uint32_t *iperm, *vstart;
    uint32_t N;
    uint32_t *colptr;
    uint64_t *status;
    uint32_t *tile_ctr;
    uint64_t *info;
};

__global__ void __launch_bounds__(SC_THREADS) pos_scan_kernel(PosArgs a) {
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_scan[40];
    __shared__ uint64_t s_excl;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(a.tile_ctr, 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    const uint64_t ntiles = (a.N + SC_TILE - 1) / SC_TILE;
    if (tile >= ntiles) return;
    const uint64_t p0 = tile * SC_TILE + (uint64_t)tid * SC_ITEMS;
    uint32_t kept[SC_ITEMS];
    uint64_t sum = 0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        kept[j] = 0;
        if (p0 + j < a.N) {
            const uint32_t v = pp_idx(a.iperm[p0 + j], a.N);
            kept[j] = (a.vstart[v] & KILL_BIT) ? 0u : (uint32_t)(a.deg[v] >> 32);
        }
        sum += kept[j];
    }
    uint64_t total;
    const uint64_t ex = block_exclusive_sum<uint64_t, SC_THREADS>(sum, s_scan, &total);
    if (tid < 32) warp_tile_prefix(a.status, tile, total, &s_excl);
    __syncthreads();
    if (tid == 0 && tile == ntiles - 1) {
        a.colptr[a.N] = (uint32_t)(s_excl + total);
        a.info[PP_INFO_NNZ] = s_excl + total;
    }
    uint64_t run = s_excl + ex;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        if (p0 + j < a.N) a.colptr[p0 + j] = (uint32_t)run;
        run += kept[j];
    }
}

__global__ void __launch_bounds__(256) finalize_kernel(const uint32_t *d_out, uint32_t N, float *inv32,
                                                       double *inv64) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
        const uint32_t d = d_out[v];
        if (inv32) inv32[v] = d ? 1.0f / (float)d : 0.0f;
        if (inv64) inv64[v] = d ? 1.0 / (double)d : 0.0;
    }
}

// ----------------------------------------------------------------- relabel
// A row's bucket is clz(d | 1) = 31 - floor(log2(max(d, 1))) of its
// out-degree d before the filter: ascending buckets = descending degrees.
__device__ __forceinline__ uint32_t row_bucket(uint32_t d) { return (uint32_t)__clz(d | 1u); }

constexpr uint32_t VKEY_SHIFT = 27;  // vertex key: bucket << 27 | u (u < 2^27)

// Histogram of the row buckets over the vertices (for the vertex pass), and
// that pass's look-back words cleared.
__global__ void __launch_bounds__(256) relabel_hist_kernel(const uint32_t *d_out, uint32_t N, uint32_t *vhist,
                                                           uint32_t *vstatus0, uint64_t vstatus_words) {
    __shared__ uint32_t sv[32];
    if (threadIdx.x < 32) sv[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < N; u += stride) atomicAdd(&sv[row_bucket(d_out[u])], 1u);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < vstatus_words; i += stride) vstatus0[i] = 0;
    __syncthreads();
    if (threadIdx.x < 32 && sv[threadIdx.x]) atomicAdd(&vhist[threadIdx.x], sv[threadIdx.x]);
}

// Vertex keys for the relabel pass and the permutation it writes.
struct VertexSrc {
    const uint32_t *d_out;
    __device__ __forceinline__ bool load(uint64_t i, uint32_t &k, uint32_t &) const {
        k = (row_bucket(d_out[i]) << VKEY_SHIFT) | (uint32_t)i;
        return true;
    }
};
struct PermDst {
    uint32_t *perm, *iperm;
    uint32_t N;
    __device__ __forceinline__ void store(uint64_t pos, uint32_t k, uint32_t) const {
        const uint32_t u = k & ((1u << VKEY_SHIFT) - 1u);
        iperm[pos] = u;
        perm[pp_idx(u, N)] = (uint32_t)pos;
    }
};

// A batch's storage order is graph-major: graph, then row bucket, then id,
// so that every graph's rows and columns keep one range of positions (its
// union ids) and, inside it, the order a single-graph call gives.  Key:
// (graph << 5 | bucket) << 32 | union id, sorted on bits 32..47 (two passes).
__global__ void __launch_bounds__(256) vkey_kernel(const uint32_t *d_out, uint32_t N, VBases vb,
                                                   unsigned long long *vkey) {
    constexpr int ITEMS = 16;
    for (uint64_t v0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * ITEMS; v0 < N;
         v0 += (uint64_t)gridDim.x * blockDim.x * ITEMS) {
        uint32_t gr = graph_of(vb, (uint32_t)v0);
        for (int j = 0; j < ITEMS && v0 + j < N; ++j) {
            const uint32_t v = (uint32_t)(v0 + j);
            while (gr < vb.n && v >= vb.vbase[gr + 1]) ++gr;
            vkey[v] = ((unsigned long long)((gr << 5) | row_bucket(d_out[v])) << 32) | v;
        }
    }
}
struct VKeySrc {
    const unsigned long long *k;
    __device__ __forceinline__ bool load(uint64_t i, unsigned long long &key, uint32_t &) const {
        key = k[i];
        return true;
    }
};
struct VKeyDst {
    unsigned long long *k;
    __device__ __forceinline__ void store(uint64_t pos, unsigned long long key, uint32_t) const { k[pos] = key; }
};
struct PermDst64 {
    uint32_t *perm, *iperm;
    uint32_t N;
    __device__ __forceinline__ void store(uint64_t pos, unsigned long long key, uint32_t) const {
        const uint32_t u = (uint32_t)key;
        iperm[pos] = u;
        perm[pp_idx(u, N)] = (uint32_t)pos;
    }
};

// The transpose sorts the 64-bit entry words by their column (bits 63:32).
struct EntSrc {
    const unsigned long long *e;
    __device__ __forceinline__ bool load(uint64_t i, unsigned long long &k, uint32_t &) const {
        k = e[i];
        return true;
    }
};
// The first transpose pass reads the words in vertex order (as the unique
// pass wrote them) and puts each row's position in place of its vertex id;
// the reads of perm follow the ascending vertex ids.
struct EntSrcPerm {
    const unsigned long long *e;
    const uint32_t *perm;
    uint32_t umask;
    __device__ __forceinline__ bool load(uint64_t i, unsigned long long &k, uint32_t &) const {
        k = e[i];
        return true;
    }
    __device__ __forceinline__ unsigned long long map(unsigned long long w) const {
        return (w & ~(unsigned long long)umask) | __ldg(perm + pp_idx((uint32_t)w & umask, umask + 1ull));
    }
};
struct EntDst {
    unsigned long long *e;
    __device__ __forceinline__ void store(uint64_t pos, unsigned long long k, uint32_t) const { e[pos] = k; }
};

struct Layout {
    unsigned long long *ent[2];  // entry words, ping-pong
    unsigned long long *deg;
    uint32_t *shift;  // vstart: each column's first entry in the sorted words | KILL_BIT
    uint32_t *row_nent;
    uint64_t *uq_status, *sc_status;
    uint32_t *ctr;                // tile counters: [0] unique, [1] mask scan, [5] column pointers
    unsigned long long *dmaxkey;  // follows ctr in one control block
    os::SortWs sort;   // the entry words: bucket pass + column passes
    os::SortWs vsort;  // the vertices by bucket
    size_t bytes;
};

inline int num_passes(uint32_t scale) { return (int)ceil_div(scale, 8u); }
constexpr int CTR_WORDS = 8;  // tile counters [0], [1], [5]; the 8-byte max key at [6..7]

inline Layout layout(void *ws, uint64_t M, uint32_t scale) {
    Carver c(ws);
    Layout L;
    const uint64_t N = 1ull << scale;
    const uint64_t cap = M ? M : 1;
    L.ent[0] = c.take<unsigned long long>(cap);
    L.ent[1] = c.take<unsigned long long>(cap);
    L.deg = c.take<unsigned long long>(N);
    L.shift = c.take<uint32_t>(N);
    L.row_nent = c.take<uint32_t>(N);
    L.uq_status = c.take<uint64_t>(ceil_div(cap, UQ_TILE));
    L.sc_status = c.take<uint64_t>(2 * ceil_div(N, SC_TILE));
    L.ctr = c.take<uint32_t>(CTR_WORDS);
    L.dmaxkey = L.ctr ? reinterpret_cast<unsigned long long *>(L.ctr + 6) : nullptr;
    L.sort = os::carve_sort_ws(c, cap);
    L.vsort = os::carve_sort_ws(c, N);
    L.bytes = c.size();
    return L;
}

}  // namespace k2
}  // namespace pp

using namespace pp;

extern "C" pp_status pp_graph_lengths(uint64_t M, uint32_t scale, uint64_t out[PP_GRAPH_ARRAYS]) {
    if (!out || scale < 1 || scale > 27 || M > (1ull << 31)) return PP_ERR_INVALID_ARG;
    const uint64_t N = 1ull << scale;
    const uint64_t cmax = (1ull << (32 - scale)) - 1;
    out[0] = N + 1;
    out[1] = M ? M : 1;
    out[2] = M / cmax + 1;
    out[3] = M / cmax + 1;
    out[4] = N;
    out[5] = N;
    out[6] = N;
    out[7] = N;
    out[8] = PP_INFO_LEN;
    out[9] = N;
    out[10] = N;
    return PP_OK;
}

extern "C" pp_status pp_build_filter_normalize_workspace(uint64_t M, uint32_t scale, size_t *bytes) {
    if (!bytes || scale < 1 || scale > 27 || M > (1ull << 31)) return PP_ERR_INVALID_ARG;
    *bytes = k2::layout(nullptr, M, scale).bytes;
    return PP_OK;
}

namespace pp {
namespace k2 {

// What a batch changes in the sequence below: the relabel (graph-major
// storage order), max(d_in) and the supernode test per graph.
struct BatchCtx {
    VBases vb;
    unsigned long long *vkey[2];  // [N] vertex keys of the relabel, ping-pong
    unsigned long long *dmaxkeys; // [n] zeroed by the caller
    unsigned long long *gcount;   // [2 n] zeroed by the caller
};

// Kernel 2 on sorted (us, vs) into g; a batch runs it on the union of its graphs.
// The in-degree the column filters test: the graph's own, or (d_in_all) one
// supplied for every column when this call holds only some rows of a graph.
__global__ void __launch_bounds__(256) set_d_in_kernel(unsigned long long *deg, const uint32_t *d_in_all, uint32_t N) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x)
        deg[v] = (deg[v] & 0xffffffff00000000ull) | d_in_all[v];
}

inline pp_status run(const uint32_t *us, const uint32_t *vs, uint64_t M, uint32_t scale, pp_supernode_rule rule,
                     const pp_graph *g, const Layout &L, cudaStream_t s, const BatchCtx *bc,
                     const uint32_t *d_in_all = nullptr) {
    const uint32_t N = 1u << scale;
    const uint32_t cmax = (uint32_t)((1ull << (32 - scale)) - 1);
    const int P = k2::num_passes(scale);
    const int sms = sm_count();
    const uint64_t sc_tiles = ceil_div(N, k2::SC_TILE);

    const size_t word = L.sort.wide ? 8 : 4;
    cudaMemsetAsync(g->info, 0, PP_INFO_LEN * sizeof(uint64_t), s);
    cudaMemsetAsync(L.ctr, 0, k2::CTR_WORDS * sizeof(uint32_t), s);
    cudaMemsetAsync(L.deg, 0, (size_t)N * sizeof(unsigned long long), s);
    cudaMemsetAsync(g->d_out, 0, (size_t)N * sizeof(uint32_t), s);
    if (bc) cudaMemsetAsync(L.row_nent, 0, (size_t)N * sizeof(uint32_t), s);  // a batch's per-graph nnz0
    cudaMemsetAsync(L.sort.hist, 0, os::kCtlBytes, s);
    cudaMemsetAsync(L.vsort.hist, 0, os::kCtlBytes, s);
    cudaMemsetAsync(L.uq_status, 0, ceil_div(M ? M : 1, k2::UQ_TILE) * sizeof(uint64_t), s);
    cudaMemsetAsync(L.sc_status, 0, 2 * sc_tiles * sizeof(uint64_t), s);
    cudaMemsetAsync(L.sort.status[0], 0, ceil_div(M ? M : 1, os::TILE) * os::RADIX * word, s);

    const unsigned ngrid = (unsigned)std::min<uint64_t>(ceil_div(N, 256), (uint64_t)sms * 8);
    unsigned long long *sorted = L.ent[0];
    if (M) {
        // step 1, entries in vertex order, with each row's edges and entries
        static PerDevice uq_occ_dev;
        const int uq_occ = (int)uq_occ_dev.get([] {
            int o = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k2::unique_kernel, k2::UQ_THREADS, 0);
            return (int64_t)(o < 1 ? 1 : o);
        });
        const unsigned ugrid = (unsigned)std::min<uint64_t>(ceil_div(M, k2::UQ_TILE), (uint64_t)sms * uq_occ);
        const int vec = (((uintptr_t)us | (uintptr_t)vs) & 15u) == 0;
        k2::UniqueArgs ua{us,          vs,         M,  scale, cmax, L.ent[0],    g->ovf_key, g->ovf_cnt, N,
                          g->d_out, bc ? L.row_nent : nullptr, L.sort.hist, P,   vec,  L.uq_status, L.ctr,      g->info};
        k2::unique_kernel<<<ugrid, k2::UQ_THREADS, 0, s>>>(ua);
        count_launch();
    }
    // relabel: the vertices by row bucket (one pass), giving perm and iperm
    const uint64_t vtiles = ceil_div(N, os::TILE);
    const size_t vword = L.vsort.wide ? 8 : 4;
    if (!bc) {
        k2::relabel_hist_kernel<<<ngrid, 256, 0, s>>>(g->d_out, N, L.vsort.hist,
                                                      static_cast<uint32_t *>(L.vsort.status[0]),
                                                      vtiles * os::RADIX * vword / 4);
        count_launch();
        os::launch_pass<uint32_t>(L.vsort, 0, 1, k2::VertexSrc{g->d_out}, k2::PermDst{g->perm, g->iperm, N}, nullptr, N,
                                  s, k2::VKEY_SHIFT);
    } else {
        // graph-major: (graph, bucket) in two 8-bit passes over bits 32..47 of the vertex keys
        k2::vkey_kernel<<<ngrid, 256, 0, s>>>(g->d_out, N, bc->vb, bc->vkey[0]);
        os::hist_kernel<unsigned long long, k2::VKeySrc><<<ngrid, 256, 0, s>>>(
            k2::VKeySrc{bc->vkey[0]}, nullptr, N, 2, L.vsort.hist, static_cast<uint32_t *>(L.vsort.status[0]),
            vtiles * os::RADIX * vword / 4, 32u);
        count_launch(2);
        os::launch_pass<unsigned long long>(L.vsort, 0, 2, k2::VKeySrc{bc->vkey[0]}, k2::VKeyDst{bc->vkey[1]}, nullptr,
                                            N, s, 32u);
        os::launch_pass<unsigned long long>(L.vsort, 1, 2, k2::VKeySrc{bc->vkey[1]},
                                            k2::PermDst64{g->perm, g->iperm, N}, nullptr, N, s, 32u);
    }
    if (M) {
        // transpose: every entry sorted by column, P passes over bits 32 .. 32+scale
        const uint64_t *n_dev = g->info + PP_INFO_NNZ0;
        os::launch_pass<unsigned long long>(L.sort, 0, P, k2::EntSrcPerm{L.ent[0], g->perm, N - 1},
                                            k2::EntDst{L.ent[1]}, n_dev, M, s, 32);
        for (int p = 1; p < P; ++p) {
            os::launch_pass<unsigned long long>(L.sort, p, P, k2::EntSrc{L.ent[p & 1]},
                                                k2::EntDst{L.ent[(p + 1) & 1]}, n_dev, M, s, 32);
        }
        sorted = L.ent[P & 1];
        const unsigned cgrid = (unsigned)std::min<uint64_t>(ceil_div(M, k2::CS_TILE), (uint64_t)sms * 8);
        k2::colscan_kernel<<<cgrid, 256, 0, s>>>(sorted, g->info, scale, cmax, g->ovf_key, g->ovf_cnt, g->iperm,
                                                 L.deg);
        count_launch();
    }
    if (d_in_all) {
        k2::set_d_in_kernel<<<ngrid, 256, 0, s>>>(L.deg, d_in_all, N);
        count_launch();
    }
    if (!bc)
        k2::dmax_kernel<<<ngrid, 256, 0, s>>>(L.deg, N, g->d_in, L.dmaxkey);
    else
        k2::dmax_batched_kernel<<<ngrid, 256, 0, s>>>(L.deg, N, bc->vb, g->d_in, bc->dmaxkeys);
    k2::ScanArgs sa;
    sa.deg = L.deg;
    sa.N = N;
    sa.all_ties = rule == PP_SUPERNODE_ALL_TIES;
    sa.dmaxkey = bc ? bc->dmaxkeys : L.dmaxkey;
    sa.vstart = L.shift;
    sa.status = L.sc_status;
    sa.tile_ctr = L.ctr + 1;
    sa.info = g->info;
    sa.batched = bc != nullptr;
    sa.gcount = bc ? bc->gcount : nullptr;
    sa.vb.n = 0;
    if (bc) sa.vb = bc->vb;
    k2::mask_scan_kernel<<<(unsigned)sc_tiles, k2::SC_THREADS, 0, s>>>(sa);
    k2::PosArgs pa{L.deg, g->iperm, L.shift, N, g->colptr, L.sc_status + sc_tiles, L.ctr + 5, g->info};
    k2::pos_scan_kernel<<<(unsigned)sc_tiles, k2::SC_THREADS, 0, s>>>(pa);
    count_launch(3);
    if (M) {
        const unsigned pgrid = (unsigned)std::min<uint64_t>(ceil_div(M, 256 * k2::CP_ITEMS), (uint64_t)sms * 8);
        k2::compact_kernel<<<pgrid, 256, 0, s>>>(sorted, g->info, scale, cmax, g->ovf_key, g->ovf_cnt, g->perm,
                                                 g->iperm, L.shift, g->colptr, g->rowc, g->d_out);
        count_launch();
    }
    k2::finalize_kernel<<<ngrid, 256, 0, s>>>(g->d_out, N, g->inv_dout32, g->inv_dout64);
    count_launch();
    return launch_status();
}

}  // namespace k2
}  // namespace pp

extern "C" pp_status pp_build_filter_normalize(const uint32_t *us, const uint32_t *vs, uint64_t M,
                                               uint32_t scale, pp_supernode_rule rule, const pp_graph *g,
                                               void *ws, size_t ws_bytes, void *stream) {
    PP_ENTRY("pp_build_filter_normalize");
    if (scale < 1 || scale > 27 || M > (1ull << 31) || !g) return PP_ERR_INVALID_ARG;
    if (rule != PP_SUPERNODE_LOWEST && rule != PP_SUPERNODE_ALL_TIES) return PP_ERR_INVALID_ARG;
    if (g->scale != scale || g->M != M) return PP_ERR_INVALID_ARG;
    if (!g->colptr || !g->rowc || !g->ovf_key || !g->ovf_cnt || !g->d_in || !g->d_out || !g->info || !g->perm ||
        !g->iperm)
        return PP_ERR_INVALID_ARG;
    if (M && (!us || !vs)) return PP_ERR_INVALID_ARG;
    const k2::Layout need = k2::layout(nullptr, M, scale);
    pp_status st = check_ws(ws, ws_bytes, need.bytes);
    if (st != PP_OK) return st;
    const k2::Layout L = k2::layout(ws, M, scale);
    return k2::run(us, vs, M, scale, rule, g, L, static_cast<cudaStream_t>(stream), nullptr);
}

extern "C" pp_status pp_build_filter_normalize_rows(const uint32_t *us, const uint32_t *vs, uint64_t M,
                                                    uint32_t scale, pp_supernode_rule rule, const uint32_t *d_in_all,
                                                    const pp_graph *g, void *ws, size_t ws_bytes, void *stream) {
    PP_ENTRY("pp_build_filter_normalize_rows");
    if (scale < 1 || scale > 27 || M > (1ull << 31) || !g || !d_in_all) return PP_ERR_INVALID_ARG;
    if (rule != PP_SUPERNODE_LOWEST && rule != PP_SUPERNODE_ALL_TIES) return PP_ERR_INVALID_ARG;
    if (g->scale != scale || g->M != M) return PP_ERR_INVALID_ARG;
    if (!g->colptr || !g->rowc || !g->ovf_key || !g->ovf_cnt || !g->d_in || !g->d_out || !g->info || !g->perm ||
        !g->iperm)
        return PP_ERR_INVALID_ARG;
    if (M && (!us || !vs)) return PP_ERR_INVALID_ARG;
    const k2::Layout need = k2::layout(nullptr, M, scale);
    pp_status st = check_ws(ws, ws_bytes, need.bytes);
    if (st != PP_OK) return st;
    const k2::Layout L = k2::layout(ws, M, scale);
    return k2::run(us, vs, M, scale, rule, g, L, static_cast<cudaStream_t>(stream), nullptr, d_in_all);
}

// ---------------------------------------------------------------------------
// Kernel 2 for a batch of graphs (pp_build_filter_normalize_batched).  The
// graphs' sorted edges are gathered into one union graph (graph g's vertex u
// becomes union id vbase[g] + u; the union stays sorted by (u, v) because
// the id ranges follow the graph order), Kernel 2 runs once on it with a
// graph-major storage order and per-graph supernodes, and split passes write
// each graph's own outputs: local ids and positions, counts repacked into
// the graph's count field (32 - scale bits) with its own overflow table,
// and its scalars.  Every output equals that of a single-graph call.

namespace pp {
namespace k2b {

constexpr int MAX_G = PP_BATCH_MAX_GRAPHS;
constexpr int TILE = 4096;

struct Shape {
    uint32_t n, S;        // graphs, union scale
    uint64_t Mtot;
    uint32_t nvert;       // sum of N_g
};

// The union's inputs: graph g's sorted edges and where they go.
struct GatherArgs {
    uint32_t n;
    const uint32_t *us[MAX_G], *vs[MAX_G];
    uint64_t eoff[MAX_G + 1];
    uint32_t vbase[MAX_G + 1];
    uint64_t toff[MAX_G + 1];  // first tile of graph g
    uint32_t scale[MAX_G];
};

__device__ __forceinline__ uint32_t tile_graph(const uint64_t *toff, uint32_t n, uint64_t t) {
    uint32_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (toff[mid] <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) gather_kernel(GatherArgs a, uint32_t *U, uint32_t *V) {
    const uint32_t g = tile_graph(a.toff, a.n, blockIdx.x);
    const uint64_t e0 = (blockIdx.x - a.toff[g]) * (uint64_t)TILE, M = a.eoff[g + 1] - a.eoff[g];
    const uint32_t base = a.vbase[g], sc = a.scale[g];
    for (uint64_t i = e0 + threadIdx.x; i < min(M, e0 + TILE); i += blockDim.x) {
        uint32_t x = __ldg(a.us[g] + i), y = __ldg(a.vs[g] + i);
        if ((x | y) >> sc) {  // an id >= N_g: reported, kept inside the graph's own range
            pp_set_error(PP_DEV_RANGE);
            x &= (1u << sc) - 1u;
            y &= (1u << sc) - 1u;
        }
        U[a.eoff[g] + i] = base + x;
        V[a.eoff[g] + i] = base + y;
    }
}

// The union's outputs and each graph's.
struct SplitArgs {
    uint32_t n, S, cmaxU;
    uint32_t vbase[MAX_G + 1];
    uint64_t vtoff[MAX_G + 1];  // first vertex tile of graph g
    const uint32_t *colptr, *rowc, *ovf_cnt, *d_in, *d_out, *perm, *iperm, *row_nent;
    const uint64_t *ovf_key, *info;
    const float *inv32;
    const double *inv64;
    const unsigned long long *dmaxkeys, *gcount;
    pp_graph out[MAX_G];
};

// Per vertex of every graph: degrees, 1/d_out, the storage order and the column pointers, local.
__global__ void __launch_bounds__(256) split_vertex_kernel(SplitArgs a) {
    const uint32_t g = tile_graph(a.vtoff, a.n, blockIdx.x);
    const uint32_t base = a.vbase[g], Ng = a.vbase[g + 1] - base;
    const pp_graph &o = a.out[g];
    const uint32_t c0 = a.colptr[base];
    const uint64_t l0 = (blockIdx.x - a.vtoff[g]) * (uint64_t)TILE;
    for (uint64_t l = l0 + threadIdx.x; l < min((uint64_t)Ng, l0 + TILE); l += blockDim.x) {
        const uint32_t u = base + (uint32_t)l;
        o.d_in[l] = a.d_in[u];
        o.d_out[l] = a.d_out[u];
        if (o.inv_dout32) o.inv_dout32[l] = a.inv32[u];
        if (o.inv_dout64) o.inv_dout64[l] = a.inv64[u];
        o.perm[l] = a.perm[u] - base;
        o.iperm[l] = a.iperm[u] - base;
        o.colptr[l] = a.colptr[u] - c0;
        if (l + 1 == Ng) o.colptr[Ng] = a.colptr[base + Ng] - c0;
    }
}

__device__ __forceinline__ uint32_t ovf_find(const uint64_t *keys, const uint32_t *cnts, uint64_t n, uint64_t key) {
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (keys[mid] < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < n && keys[lo] == key) ? cnts[lo] : 0u;
}

// One warp per union column position: its kept entries as the graph's words
// (local row position, count in the graph's field, escaped past its maximum).
__global__ void __launch_bounds__(256) split_entry_kernel(SplitArgs a) {
    const int lane = threadIdx.x & 31;
    const uint32_t nvert = a.vbase[a.n], umaskU = (1u << a.S) - 1u;
    const uint64_t novf = a.info[PP_INFO_NOVF];
    const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t q = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); q < nvert; q += nw) {
        uint32_t g = 0, lo = 0, hi = a.n - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (a.vbase[mid] <= q)
                lo = mid;
            else
                hi = mid - 1;
        }
        g = lo;
        const uint32_t base = a.vbase[g], sg = a.out[g].scale;
        const uint32_t cmaxg = (uint32_t)((1ull << (32 - sg)) - 1);
        const uint32_t s = a.colptr[q], e = a.colptr[q + 1], d0 = s - a.colptr[base];
        uint32_t *dst = a.out[g].rowc;
        const uint64_t mg = a.out[g].M ? a.out[g].M : 1, mu = a.info[PP_INFO_NNZ];
        for (uint32_t k = lane; k < e - s; k += 32) {
            const uint32_t w = a.rowc[pp_idx(s + k, mu)];
            const uint32_t pos = w & umaskU;
            uint32_t c = w >> a.S;
            if (c == a.cmaxU) c = ovf_find(a.ovf_key, a.ovf_cnt, novf, ((uint64_t)a.iperm[pos] << 32) | a.iperm[q]);
            dst[pp_idx(d0 + k, mg)] = ((c >= cmaxg ? cmaxg : c) << sg) | (pos - base);
        }
    }
}

// One thread per graph: its overflow table (the union table's entries of the
// graph whose count reaches the graph's own escape value, in key order).
__global__ void __launch_bounds__(128) split_ovf_kernel(SplitArgs a) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.n) return;
    const uint64_t novf = a.info[PP_INFO_NOVF];
    const uint32_t base = a.vbase[g], end = a.vbase[g + 1], sg = a.out[g].scale;
    const uint32_t cmaxg = (uint32_t)((1ull << (32 - sg)) - 1);
    uint64_t lo = 0, hi = novf;
    const uint64_t first_key = (uint64_t)base << 32;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (a.ovf_key[mid] < first_key)
            lo = mid + 1;
        else
            hi = mid;
    }
    uint64_t k = 0;
    for (uint64_t i = lo; i < novf && (uint32_t)(a.ovf_key[i] >> 32) < end; ++i) {
        if (a.ovf_cnt[i] < cmaxg) continue;
        const uint64_t key = a.ovf_key[i];
        const uint64_t ko = pp_idx(k, a.out[g].M / cmaxg + 1);  // the graph's table length
        a.out[g].ovf_key[ko] = ((uint64_t)((uint32_t)(key >> 32) - base) << 32) | (uint32_t)((uint32_t)key - base);
        a.out[g].ovf_cnt[ko] = a.ovf_cnt[i];
        ++k;
    }
    a.out[g].info[PP_INFO_NOVF] = k;
}

// One block per graph: its scalars.
__global__ void __launch_bounds__(256) split_info_kernel(SplitArgs a) {
    __shared__ unsigned long long s_red[8];
    const uint32_t g = blockIdx.x;
    const uint32_t base = a.vbase[g], Ng = a.vbase[g + 1] - base;
    unsigned long long nnz0 = 0;
    for (uint32_t l = threadIdx.x; l < Ng; l += blockDim.x) nnz0 += a.row_nent[base + l];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nnz0 += __shfl_down_sync(0xffffffffu, nnz0, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = nnz0;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < 8; ++w) t += s_red[w];
        uint64_t *info = a.out[g].info;
        const unsigned long long key = a.dmaxkeys[g];
        info[PP_INFO_NNZ0] = t;
        info[PP_INFO_NNZ] = a.colptr[base + Ng] - a.colptr[base];
        info[PP_INFO_DMAX] = key >> 32;
        info[PP_INFO_VMAX] = ~(uint32_t)key - base;
        info[PP_INFO_TIES] = a.gcount[2 * g];
        info[PP_INFO_SUPERNODES] = a.gcount[2 * g + 1];
        info[7] = 0;
    }
}

struct Layout {
    uint32_t *U, *V;
    pp_graph ug;  // the union graph
    unsigned long long *vkey[2], *dmaxkeys, *gcount;
    k2::Layout k2;
    size_t bytes;
};

inline Layout layout(void *ws, const Shape &sh) {
    Carver c(ws);
    Layout L;
    const uint64_t N = 1ull << sh.S, cap = sh.Mtot ? sh.Mtot : 1;
    uint64_t len[PP_GRAPH_ARRAYS];
    pp_graph_lengths(sh.Mtot, sh.S, len);
    L.U = c.take<uint32_t>(cap);
    L.V = c.take<uint32_t>(cap);
    L.ug.scale = sh.S;
    L.ug.reserved = 0;
    L.ug.M = sh.Mtot;
    L.ug.colptr = c.take<uint32_t>(len[0]);
    L.ug.rowc = c.take<uint32_t>(len[1]);
    L.ug.ovf_key = c.take<uint64_t>(len[2]);
    L.ug.ovf_cnt = c.take<uint32_t>(len[3]);
    L.ug.d_in = c.take<uint32_t>(len[4]);
    L.ug.d_out = c.take<uint32_t>(len[5]);
    L.ug.inv_dout32 = c.take<float>(len[6]);
    L.ug.inv_dout64 = c.take<double>(len[7]);
    L.ug.info = c.take<uint64_t>(len[8]);
    L.ug.perm = c.take<uint32_t>(len[9]);
    L.ug.iperm = c.take<uint32_t>(len[10]);
    L.vkey[0] = c.take<unsigned long long>(N);
    L.vkey[1] = c.take<unsigned long long>(N);
    L.dmaxkeys = c.take<unsigned long long>(MAX_G);
    L.gcount = c.take<unsigned long long>(2 * MAX_G);
    const size_t head = c.size();
    L.k2 = k2::layout(ws ? static_cast<char *>(ws) + head : nullptr, sh.Mtot, sh.S);
    L.bytes = head + L.k2.bytes;
    return L;
}

inline bool shape(uint32_t n, const uint64_t *M, const uint32_t *scale, Shape *sh) {
    if (n < 1 || n > (uint32_t)MAX_G || !M || !scale) return false;
    uint64_t nv = 0, me = 0;
    for (uint32_t g = 0; g < n; ++g) {
        if (scale[g] < 1 || scale[g] > 27 || M[g] > (1ull << 31)) return false;
        nv += 1ull << scale[g];
        me += M[g];
    }
    if (nv > (1ull << 27) || me > (1ull << 31)) return false;
    uint32_t s = 1;
    while ((1ull << s) < nv) ++s;
    sh->n = n;
    sh->S = s;
    sh->Mtot = me;
    sh->nvert = (uint32_t)nv;
    return true;
}

}  // namespace k2b
}  // namespace pp

extern "C" pp_status pp_build_filter_normalize_batched_workspace(uint32_t n_graphs, const uint64_t *M,
                                                                 const uint32_t *scale, size_t *bytes) {
    k2b::Shape sh;
    if (!bytes || !k2b::shape(n_graphs, M, scale, &sh)) return PP_ERR_INVALID_ARG;
    *bytes = k2b::layout(nullptr, sh).bytes;
    return PP_OK;
}

extern "C" pp_status pp_build_filter_normalize_batched(uint32_t n_graphs, const uint32_t *const *u_sorted,
                                                       const uint32_t *const *v_sorted, pp_supernode_rule rule,
                                                       const pp_graph *gs, void *ws, size_t ws_bytes,
                                                       void *stream) {
    PP_ENTRY("pp_build_filter_normalize_batched");
    if (!gs || !u_sorted || !v_sorted || n_graphs < 1 || n_graphs > (uint32_t)k2b::MAX_G) return PP_ERR_INVALID_ARG;
    if (rule != PP_SUPERNODE_LOWEST && rule != PP_SUPERNODE_ALL_TIES) return PP_ERR_INVALID_ARG;
    uint64_t M[k2b::MAX_G];
    uint32_t scale[k2b::MAX_G];
    for (uint32_t g = 0; g < n_graphs; ++g) {
        const pp_graph &o = gs[g];
        M[g] = o.M;
        scale[g] = o.scale;
        if (!o.colptr || !o.rowc || !o.ovf_key || !o.ovf_cnt || !o.d_in || !o.d_out || !o.info || !o.perm ||
            !o.iperm)
            return PP_ERR_INVALID_ARG;
        if (o.M && (!u_sorted[g] || !v_sorted[g])) return PP_ERR_INVALID_ARG;
    }
    k2b::Shape sh;
    if (!k2b::shape(n_graphs, M, scale, &sh)) return PP_ERR_INVALID_ARG;
    const k2b::Layout need = k2b::layout(nullptr, sh);
    pp_status st = check_ws(ws, ws_bytes, need.bytes);
    if (st != PP_OK) return st;
    const k2b::Layout L = k2b::layout(ws, sh);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // the union's edges
    k2b::GatherArgs ga;
    ga.n = n_graphs;
    uint64_t eo = 0, to = 0;
    uint32_t vb = 0;
    k2::BatchCtx bc;
    bc.vb.n = n_graphs;
    for (uint32_t g = 0; g < n_graphs; ++g) {
        ga.us[g] = u_sorted[g];
        ga.vs[g] = v_sorted[g];
        ga.eoff[g] = eo;
        ga.vbase[g] = vb;
        ga.toff[g] = to;
        ga.scale[g] = scale[g];
        bc.vb.vbase[g] = vb;
        eo += M[g];
        to += ceil_div(M[g], k2b::TILE);
        vb += 1u << scale[g];
    }
    ga.eoff[n_graphs] = eo;
    ga.vbase[n_graphs] = vb;
    ga.toff[n_graphs] = to;
    bc.vb.vbase[n_graphs] = vb;
    if (to) {
        k2b::gather_kernel<<<(unsigned)to, 256, 0, s>>>(ga, L.U, L.V);
        count_launch();
    }
    // Kernel 2 on the union
    bc.vkey[0] = L.vkey[0];
    bc.vkey[1] = L.vkey[1];
    bc.dmaxkeys = L.dmaxkeys;
    bc.gcount = L.gcount;
    cudaMemsetAsync(L.dmaxkeys, 0, k2b::MAX_G * sizeof(unsigned long long), s);
    cudaMemsetAsync(L.gcount, 0, 2 * k2b::MAX_G * sizeof(unsigned long long), s);
    st = k2::run(L.U, L.V, sh.Mtot, sh.S, rule, &L.ug, L.k2, s, &bc);
    if (st != PP_OK) return st;
    // each graph's outputs
    k2b::SplitArgs sa;
    sa.n = n_graphs;
    sa.S = sh.S;
    sa.cmaxU = (uint32_t)((1ull << (32 - sh.S)) - 1);
    uint64_t vt = 0;
    for (uint32_t g = 0; g <= n_graphs; ++g) {
        sa.vbase[g] = bc.vb.vbase[g];
        sa.vtoff[g] = vt;
        if (g < n_graphs) {
            vt += ceil_div(1ull << scale[g], k2b::TILE);
            sa.out[g] = gs[g];
        }
    }
    sa.colptr = L.ug.colptr;
    sa.rowc = L.ug.rowc;
    sa.ovf_key = L.ug.ovf_key;
    sa.ovf_cnt = L.ug.ovf_cnt;
    sa.d_in = L.ug.d_in;
    sa.d_out = L.ug.d_out;
    sa.inv32 = L.ug.inv_dout32;
    sa.inv64 = L.ug.inv_dout64;
    sa.info = L.ug.info;
    sa.perm = L.ug.perm;
    sa.iperm = L.ug.iperm;
    sa.row_nent = L.k2.row_nent;
    sa.dmaxkeys = L.dmaxkeys;
    sa.gcount = L.gcount;
    const int sms = sm_count();
    k2b::split_vertex_kernel<<<(unsigned)vt, 256, 0, s>>>(sa);
    k2b::split_entry_kernel<<<(unsigned)std::max<uint64_t>(1, std::min<uint64_t>(ceil_div(sh.nvert, 8), 32ull * sms)),
                              256, 0, s>>>(sa);
    k2b::split_ovf_kernel<<<(unsigned)ceil_div(n_graphs, 128), 128, 0, s>>>(sa);
    k2b::split_info_kernel<<<n_graphs, 256, 0, s>>>(sa);
    count_launch(4);
    return launch_status();
}
