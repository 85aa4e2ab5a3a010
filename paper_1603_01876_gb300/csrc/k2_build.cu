// Kernel 2 (Sec. IV-C): build, filter and normalise the adjacency matrix.
//
//   unique_kernel    step 1: run-lengths of equal (u, v) in Kernel 1's sorted
//                    output are the counts A(u,v); one thread block per tile,
//                    output offsets by decoupled look-back; each entry adds
//                    (1, count) to a packed per-column (entries, d_in) word.
//   dmax_kernel      step 2 done: d_in out; max(d_in) and its lowest column.
//   mask_scan_kernel step 3: the supernode and leaf columns; the CSC column
//                    pointer of what survives by a look-back scan over N.
//   prepass_kernel   step 4: d_out = row sums of the kept counts (entries are
//                    in row order, so a warp aggregates a row before its
//                    atomic); digit histograms for the transpose.
//   onesweep passes  stable sort of the kept entries by column: rows stay
//                    ascending inside every column (the CSC layout).
//   finalize_kernel  1/d_out in binary32 and binary64.
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

constexpr uint64_t F_AGG = 1ull << 62, F_INC = 2ull << 62, F_ANY = 3ull << 62, F_VAL = F_AGG - 1;

__device__ __forceinline__ uint64_t uq_tiles(uint64_t M) { return (M + UQ_TILE - 1) / UQ_TILE; }

__device__ __forceinline__ uint64_t edge_key(const uint32_t *us, const uint32_t *vs, uint64_t i) {
    return ((uint64_t)__ldg(us + i) << 32) | (uint64_t)__ldg(vs + i);
}

// Exclusive prefix of the tiles before `tile` in a chained scan whose status
// words carry flags in bits 63:62 and a sum in bits 61:0.
__device__ __forceinline__ uint64_t lookback(uint64_t *status, uint64_t tile) {
    uint64_t excl = 0;
    uint64_t p = tile - 1;
    uint32_t spins = 0;
    while (true) {
        const uint64_t s = ld_relaxed_u64(status + p);
        if ((s & F_ANY) == 0) {
            if (++spins > kSpinLimit) {
                pp_set_error(PP_DEV_TIMEOUT);
                return excl;
            }
            backoff(spins);
            continue;
        }
        excl += s & F_VAL;
        if (s & F_INC) return excl;
        --p;
    }
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

struct UniqueArgs {
    const uint32_t *us, *vs;
    uint64_t M;
    uint32_t scale, cmax;
    uint32_t *out_v, *out_rowc;
    uint64_t *ovf_key;
    uint32_t *ovf_cnt;
    unsigned long long *deg;  // [N]: entries << 32 | d_in
    uint64_t *status;
    uint32_t *tile_ctr;
    uint64_t *info;
};

__global__ void __launch_bounds__(UQ_THREADS) unique_kernel(UniqueArgs a) {
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_scan[40];
    __shared__ long long s_max[UQ_THREADS / 32];
    __shared__ uint64_t s_excl;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(a.tile_ctr, 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= uq_tiles(a.M)) return;
    const uint64_t base = tile * UQ_TILE;
    const uint64_t my0 = base + (uint64_t)tid * UQ_ITEMS;

    uint64_t k[UQ_ITEMS];
#pragma unroll
    for (int j = 0; j < UQ_ITEMS; ++j) k[j] = (my0 + j < a.M) ? edge_key(a.us, a.vs, my0 + j) : ~0ull;
    const uint64_t knext = (my0 + UQ_ITEMS < a.M) ? edge_key(a.us, a.vs, my0 + UQ_ITEMS) : ~0ull;

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
    const long long prev_tail = block_exclusive_max(last_tail >= 0 ? (long long)(my0 + last_tail) : -1ll, s_max);

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

    uint32_t cnt[UQ_ITEMS];
    uint32_t nt = 0, ne = 0;
#pragma unroll
    for (int j = 0; j < UQ_ITEMS; ++j) {
        cnt[j] = 0;
        if (tails >> j & 1u) {
            cnt[j] = (uint32_t)(my0 + j - start + 1);
            start = my0 + j + 1;
            ++nt;
            ne += cnt[j] >= a.cmax;
        }
    }

    uint64_t total;
    const uint64_t mine = ((uint64_t)ne << 32) | nt;
    const uint64_t texcl = block_exclusive_sum<uint64_t, UQ_THREADS>(mine, s_scan, &total);
    if (tid == 0) {
        uint64_t *st = a.status + tile;
        if (tile == 0) {
            st_relaxed_u64(st, F_INC | total);
            s_excl = 0;
        } else {
            st_relaxed_u64(st, F_AGG | total);
            const uint64_t ex = lookback(a.status, tile);
            st_relaxed_u64(st, F_INC | (ex + total));
            s_excl = ex;
        }
        if (tile == uq_tiles(a.M) - 1) {
            const uint64_t inc = s_excl + total;
            a.info[PP_INFO_NNZ0] = inc & 0xffffffffull;
            a.info[PP_INFO_NOVF] = (inc >> 32) & 0x3fffffffull;
        }
    }
    __syncthreads();
    const uint64_t gex = s_excl + texcl;
    uint64_t pos = gex & 0xffffffffull;
    uint64_t epos = (gex >> 32) & 0x3fffffffull;
    const uint32_t umask = (a.scale >= 32) ? 0xffffffffu : ((1u << a.scale) - 1u);
#pragma unroll
    for (int j = 0; j < UQ_ITEMS; ++j) {
        if (!(tails >> j & 1u)) continue;
        uint32_t u = (uint32_t)(k[j] >> 32), v = (uint32_t)k[j];
        if ((u | v) & ~umask) {
            // an id >= N: report it and keep every later access in bounds
            pp_set_error(PP_DEV_RANGE);
            u &= umask;
            v &= umask;
        }
        const uint32_t c = cnt[j];
        const uint32_t field = c >= a.cmax ? a.cmax : c;
        a.out_v[pos] = v;
        a.out_rowc[pos] = u | (field << a.scale);
        if (c >= a.cmax) {
            a.ovf_key[epos] = k[j];
            a.ovf_cnt[epos] = c;
            ++epos;
        }
        atomicAdd(&a.deg[v], (1ull << 32) | (unsigned long long)c);
        ++pos;
    }
}

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

struct ScanArgs {
    const unsigned long long *deg;
    uint32_t N;
    int all_ties;
    const unsigned long long *dmaxkey;
    uint8_t *kill;
    uint32_t *colptr;
    uint32_t *d_out;
    uint64_t *status;
    uint32_t *tile_ctr;
    uint64_t *info;
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
    const unsigned long long key = *a.dmaxkey;
    const uint32_t dmax = (uint32_t)(key >> 32);
    const uint32_t vmax = ~(uint32_t)key;
    const uint64_t v0 = tile * SC_TILE + (uint64_t)tid * SC_ITEMS;
    uint32_t cnt[SC_ITEMS];
    uint64_t sum = 0;
    unsigned long long ties = 0, sup = 0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        const uint64_t v = v0 + j;
        cnt[j] = 0;
        if (v < a.N) {
            const unsigned long long w = a.deg[v];
            const uint32_t din = (uint32_t)w, entries = (uint32_t)(w >> 32);
            const bool is_max = din == dmax && (a.all_ties || (uint32_t)v == vmax);
            const bool kill = is_max || din == 1;
            ties += din == dmax;
            sup += is_max;
            a.kill[v] = kill;
            a.d_out[v] = 0;
            cnt[j] = kill ? 0u : entries;
            sum += cnt[j];
        }
    }
    uint64_t total;
    const uint64_t texcl = block_exclusive_sum<uint64_t, SC_THREADS>(sum, s_scan, &total);
    if (tid == 0) {
        uint64_t *st = a.status + tile;
        if (tile == 0) {
            st_relaxed_u64(st, F_INC | total);
            s_excl = 0;
        } else {
            st_relaxed_u64(st, F_AGG | total);
            const uint64_t ex = lookback(a.status, tile);
            st_relaxed_u64(st, F_INC | (ex + total));
            s_excl = ex;
        }
        if (tile == ntiles - 1) {
            a.colptr[a.N] = (uint32_t)(s_excl + total);
            a.info[PP_INFO_NNZ] = s_excl + total;
            a.info[PP_INFO_DMAX] = dmax;
            a.info[PP_INFO_VMAX] = vmax;
        }
    }
    __syncthreads();
    uint64_t run = s_excl + texcl;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        const uint64_t v = v0 + j;
        if (v < a.N) a.colptr[v] = (uint32_t)run;
        run += cnt[j];
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
    if (tid == 0) {
        unsigned long long t = 0, s = 0;
        for (int w = 0; w < SC_THREADS / 32; ++w) {
            t += s_red[0][w];
            s += s_red[1][w];
        }
        if (t) atomicAdd((unsigned long long *)&a.info[PP_INFO_TIES], t);
        if (s) atomicAdd((unsigned long long *)&a.info[PP_INFO_SUPERNODES], s);
    }
}

struct PrepassArgs {
    const uint32_t *uv_v, *uv_rowc;
    const uint64_t *info;
    uint32_t scale, cmax;
    const uint8_t *kill;
    const uint64_t *ovf_key;
    const uint32_t *ovf_cnt;
    uint32_t *d_out;
    int npasses;
    uint32_t *hist;
    uint32_t *status0;
    uint64_t status0_words;
};

__global__ void __launch_bounds__(256) prepass_kernel(PrepassArgs a) {
    __shared__ uint32_t sh[os::MAX_PASSES][os::RADIX];
    for (int i = threadIdx.x; i < os::MAX_PASSES * os::RADIX; i += blockDim.x) (&sh[0][0])[i] = 0;
    __syncthreads();
    const uint64_t n = a.info[PP_INFO_NNZ0];
    const uint64_t novf = a.info[PP_INFO_NOVF];
    const uint32_t umask = (1u << a.scale) - 1u;
    const int lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); b < n; b += stride) {
        const uint64_t i = b + lane;
        uint32_t u = 0xffffffffu, c = 0;
        if (i < n) {
            const uint32_t v = a.uv_v[i];
            const uint32_t w = a.uv_rowc[i];
            u = w & umask;
            if (!a.kill[v]) {
                for (int p = 0; p < a.npasses; ++p) atomicAdd(&sh[p][(v >> (8 * p)) & (os::RADIX - 1)], 1u);
                c = w >> a.scale;
                if (c == a.cmax) c = ovf_lookup(a.ovf_key, a.ovf_cnt, novf, ((uint64_t)u << 32) | v);
            }
        }
        // rows are contiguous: sum each row's kept counts across the warp first
        const uint32_t peers = __match_any_sync(0xffffffffu, u);
        const uint32_t rowsum = __reduce_add_sync(peers, c);
        if (i < n && rowsum && lane == __ffs(peers) - 1) atomicAdd(&a.d_out[u], rowsum);
    }
    const uint64_t gs = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.status0_words; i += gs) a.status0[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < a.npasses * os::RADIX; i += blockDim.x) {
        const uint32_t c = (&sh[0][0])[i];
        if (c) atomicAdd(&a.hist[i], c);
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

// Sources and sinks of the transpose sort (key = column v, value = packed row/count).
struct FilterSrc {
    const uint32_t *v, *rowc;
    const uint8_t *kill;
    __device__ __forceinline__ bool load(uint64_t i, uint32_t &k, uint32_t &val) const {
        k = v[i];
        val = rowc[i];
        return !kill[k];
    }
};
struct KVSrc {
    const uint32_t *k, *val;
    __device__ __forceinline__ bool load(uint64_t i, uint32_t &kk, uint32_t &vv) const {
        kk = k[i];
        vv = val[i];
        return true;
    }
};
struct KVDst {
    uint32_t *k, *val;
    __device__ __forceinline__ void store(uint64_t pos, uint32_t kk, uint32_t vv) const {
        k[pos] = kk;
        val[pos] = vv;
    }
};
struct ValDst {
    uint32_t *val;
    __device__ __forceinline__ void store(uint64_t pos, uint32_t, uint32_t vv) const { val[pos] = vv; }
};

struct Layout {
    uint32_t *uv_v, *uv_rowc, *a_key, *a_val;
    unsigned long long *deg;
    uint8_t *kill;
    uint64_t *uq_status, *sc_status;
    uint32_t *ctr;                 // [0] unique tiles, [1] scan tiles
    unsigned long long *dmaxkey;   // follows ctr in one control block
    os::SortWs sort;
    size_t bytes;
};

inline int num_passes(uint32_t scale) { return (int)ceil_div(scale, 8u); }

inline Layout layout(void *ws, uint64_t M, uint32_t scale) {
    Carver c(ws);
    Layout L;
    const uint64_t N = 1ull << scale;
    const uint64_t cap = M ? M : 1;
    L.uv_v = c.take<uint32_t>(cap);
    L.uv_rowc = c.take<uint32_t>(cap);
    const bool two = num_passes(scale) >= 2;
    L.a_key = two ? c.take<uint32_t>(cap) : nullptr;
    L.a_val = two ? c.take<uint32_t>(cap) : nullptr;
    L.deg = c.take<unsigned long long>(N);
    L.kill = c.take<uint8_t>(N);
    L.uq_status = c.take<uint64_t>(ceil_div(cap, UQ_TILE));
    L.sc_status = c.take<uint64_t>(ceil_div(N, SC_TILE));
    L.ctr = c.take<uint32_t>(4);  // two counters + the 8-byte max key
    L.dmaxkey = L.ctr ? reinterpret_cast<unsigned long long *>(L.ctr + 2) : nullptr;
    L.sort = os::carve_sort_ws(c, cap);
    L.bytes = c.size();
    return L;
}

}  // namespace k2
}  // namespace pp

using namespace pp;

extern "C" pp_status pp_graph_lengths(uint64_t M, uint32_t scale, uint64_t out[9]) {
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
    return PP_OK;
}

extern "C" pp_status pp_build_filter_normalize_workspace(uint64_t M, uint32_t scale, size_t *bytes) {
    if (!bytes || scale < 1 || scale > 27 || M > (1ull << 31)) return PP_ERR_INVALID_ARG;
    *bytes = k2::layout(nullptr, M, scale).bytes;
    return PP_OK;
}

extern "C" pp_status pp_build_filter_normalize(const uint32_t *us, const uint32_t *vs, uint64_t M,
                                               uint32_t scale, pp_supernode_rule rule, const pp_graph *g,
                                               void *ws, size_t ws_bytes, void *stream) {
    if (scale < 1 || scale > 27 || M > (1ull << 31) || !g) return PP_ERR_INVALID_ARG;
    if (rule != PP_SUPERNODE_LOWEST && rule != PP_SUPERNODE_ALL_TIES) return PP_ERR_INVALID_ARG;
    if (g->scale != scale || g->M != M) return PP_ERR_INVALID_ARG;
    if (!g->colptr || !g->rowc || !g->ovf_key || !g->ovf_cnt || !g->d_in || !g->d_out || !g->info)
        return PP_ERR_INVALID_ARG;
    if (M && (!us || !vs)) return PP_ERR_INVALID_ARG;
    const k2::Layout need = k2::layout(nullptr, M, scale);
    pp_status st = check_ws(ws, ws_bytes, need.bytes);
    if (st != PP_OK) return st;
    const k2::Layout L = k2::layout(ws, M, scale);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t N = 1u << scale;
    const uint32_t cmax = (uint32_t)((1ull << (32 - scale)) - 1);
    const int P = k2::num_passes(scale);
    const int sms = sm_count();

    cudaMemsetAsync(g->info, 0, PP_INFO_LEN * sizeof(uint64_t), s);
    cudaMemsetAsync(L.ctr, 0, 4 * sizeof(uint32_t), s);
    cudaMemsetAsync(L.deg, 0, (size_t)N * sizeof(unsigned long long), s);
    cudaMemsetAsync(L.sort.hist, 0, os::kCtlBytes, s);
    cudaMemsetAsync(L.uq_status, 0, ceil_div(M ? M : 1, k2::UQ_TILE) * sizeof(uint64_t), s);
    cudaMemsetAsync(L.sc_status, 0, ceil_div(N, k2::SC_TILE) * sizeof(uint64_t), s);

    if (M) {
        k2::UniqueArgs ua{us, vs, M, scale, cmax, L.uv_v, L.uv_rowc, g->ovf_key, g->ovf_cnt, L.deg,
                          L.uq_status, L.ctr, g->info};
        k2::unique_kernel<<<(unsigned)ceil_div(M, k2::UQ_TILE), k2::UQ_THREADS, 0, s>>>(ua);
        count_launch();
    }
    const unsigned ngrid = (unsigned)std::min<uint64_t>(ceil_div(N, 256), (uint64_t)sms * 8);
    k2::dmax_kernel<<<ngrid, 256, 0, s>>>(L.deg, N, g->d_in, L.dmaxkey);
    k2::ScanArgs sa{L.deg, N, rule == PP_SUPERNODE_ALL_TIES, L.dmaxkey, L.kill, g->colptr, g->d_out,
                    L.sc_status, L.ctr + 1, g->info};
    k2::mask_scan_kernel<<<(unsigned)ceil_div(N, k2::SC_TILE), k2::SC_THREADS, 0, s>>>(sa);
    count_launch(2);
    if (M) {
        const size_t word = L.sort.wide ? 8 : 4;
        k2::PrepassArgs pa{L.uv_v, L.uv_rowc, g->info, scale, cmax, L.kill, g->ovf_key, g->ovf_cnt, g->d_out, P,
                           L.sort.hist, static_cast<uint32_t *>(L.sort.status[0]),
                           ceil_div(M, os::TILE) * os::RADIX * word / 4};
        const unsigned pgrid = (unsigned)std::min<uint64_t>(ceil_div(M, 256 * 4), (uint64_t)sms * 8);
        k2::prepass_kernel<<<pgrid, 256, 0, s>>>(pa);
        count_launch();
        // pass 0 reads every unique entry and drops the zeroed columns; later
        // passes see only the nnz entries that survived
        const uint64_t *n_dev = g->info + PP_INFO_NNZ0;
        const uint64_t *n_kept = g->info + PP_INFO_NNZ;
        const k2::FilterSrc fsrc{L.uv_v, L.uv_rowc, L.kill};
        const k2::ValDst out{g->rowc};
        if (P == 1) {
            os::launch_pass<uint32_t, true>(L.sort, 0, P, fsrc, out, n_dev, M, s);
        } else {
            // ping-pong between A and the (by then consumed) unique-pass arrays
            uint32_t *bk = L.uv_v, *bv = L.uv_rowc;
            os::launch_pass<uint32_t, true>(L.sort, 0, P, fsrc, k2::KVDst{L.a_key, L.a_val}, n_dev, M, s);
            for (int p = 1; p < P - 1; ++p) {
                const bool odd = p & 1;
                os::launch_pass<uint32_t, true>(L.sort, p, P, k2::KVSrc{odd ? L.a_key : bk, odd ? L.a_val : bv},
                                                k2::KVDst{odd ? bk : L.a_key, odd ? bv : L.a_val}, n_kept, M, s);
            }
            const bool odd = (P - 1) & 1;
            os::launch_pass<uint32_t, true>(L.sort, P - 1, P, k2::KVSrc{odd ? L.a_key : bk, odd ? L.a_val : bv},
                                            out, n_kept, M, s);
        }
    }
    k2::finalize_kernel<<<ngrid, 256, 0, s>>>(g->d_out, N, g->inv_dout32, g->inv_dout64);
    count_launch();
    return launch_status();
}
