// Kernel 3 for a batch: several graphs, each with several start vectors.
//
// Every (graph, start vector) pair is one PageRank run of Sec. IV-D:
//     r(v) <- c * sum_u r(u) A(u,v) + ((1-c)/N) * sum(r),
// r0 normalised to unit L1 norm first.  The runs of one graph share its
// matrix, so the iteration is a sparse-matrix times dense-matrix product
// (SpMM): X holds one row per vertex and one column per start vector
// (x = r / d_out as in the single-vector kernel), and lane j of a warp owns
// start vector j, so gathering row X[u] is one coalesced 128-byte access.
//
// One persistent launch per iteration covers every graph of the batch.  The
// columns of all graphs are planned together into warp work items (tiles of
// up to 32 short columns; chunks of `chunk` entries of long columns), dealt to
// warps round-robin so that the warps work on neighbouring items of the same
// graph at any moment and that graph's X stays in L2.  Each column is summed
// in entry order (a long column's chunk sums are added in chunk order by the
// warp that finishes it), and sum(r) of every (graph, vector) pair is
// accumulated exactly in 128-bit fixed point, so results do not depend on
// which warp took which item.
//
// With 32 start vectors (k3b_vec), 8 lanes share an entry, each with 4
// vectors (one 16-byte piece of the gathered row), so a warp takes 4
// entries per step and the per-entry work (the packed word, the row
// address, the count) is shared by 4 times as many products.  Entry k of a
// column goes to slot k mod 4; each slot keeps a compensated sum per vector
// and the 4 slot sums are added in a fixed shuffle tree.
#include <algorithm>
#include <cstring>

#include "fixedpoint.cuh"
#include "pp_common.cuh"

PP_DEFINE_ERROR_WORD(k3b_fetch_error)

namespace pp {
namespace k3b {

constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;
constexpr int TILE_COLS = 32;
constexpr int SHORTMAX_MAX = 256;  // largest long-column threshold (k3b_shortmax)
constexpr int SHORTMAX_MIN = 128;
constexpr int TILE_ENTRIES = 2 * SHORTMAX_MAX;
constexpr int CHUNK_MIN = 256;     // smallest long-column chunk (k3b_chunk)
constexpr int GATHERS = 8;     // gathers in flight per lane
constexpr int MAXG = PP_BATCH_MAX_GRAPHS;
constexpr int NORM_ROWS = 2048;  // rows per block of the start-vector passes
constexpr uint32_t LONG_FLAG = 0x80000000u;
constexpr int PLAN_THREADS = 256;
constexpr int PLAN_ITEMS = 16;
constexpr int PLAN_TILE = PLAN_THREADS * PLAN_ITEMS;
constexpr uint64_t F_AGG = 1ull << 62, F_INC = 2ull << 62;

// One graph of the batch, as the kernels see it.
struct BG {
    const uint32_t *colptr, *rowc;
    const uint32_t *iperm;  // vertex at storage position p (Kernel 2's order of rows and columns)
    const uint64_t *ovf_key;
    const uint32_t *ovf_cnt;
    const uint64_t *info;
    const float *inv;
    uint32_t N, scale, cmax, nblk;  // nblk: NORM_ROWS-row blocks of this graph
    uint64_t row0;                  // first row of this graph in X, r0 and r_out
    uint32_t blk0, pad;             // first start-vector block of this graph
};

struct Desc {
    BG g[MAXG];
    uint32_t ng, nrhs, iters;
    uint32_t item_cap;  // entries of the item arrays (bounds of the checked build)
    uint32_t shortmax;  // columns longer than this are cut into chunks (power of two)
    uint32_t chunk;     // entries of a long column per work item
    uint64_t rows;  // rows of all graphs together
    double c;
};

struct Ws {
    float *x[2];               // [rows * nrhs], rows in storage order
    float *invp;               // [rows] 1/d_out in storage order
    uint32_t *bound;           // [rows] global columns that start a work item
    uint32_t *bound_item;      // [rows] first work item of each
    uint4 *item;               // [max_items] (col | LONG_FLAG, first item, first entry, entries | chunks<<12)
                               //             or (first col, cols, first entry, entries)
    uint8_t *item_g;           // [max_items] graph of each item
    float *chunk_sum;          // [max_items * nrhs]
    uint32_t *ticket;          // [max_items]
    uint32_t *first_item;      // [ng]
    uint64_t *plan_status;     // [rows / PLAN_TILE + 1]
    unsigned long long *acc;   // [(iters + 1) * ng * 32 * 2] sum(r) per (iterate, graph, vector)
    int *fx_exp;               // [(iters + 1) * ng * 32]
    double *norm_part;         // [blocks * 32]
    double *norm;              // [ng * 32]
    uint32_t *ctl;             // [0] items, [1] boundaries, [2] plan tile counter
};

__device__ __forceinline__ int graph_of(const Desc &d, uint64_t row) {
    int lo = 0, hi = (int)d.ng - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d.g[mid].row0 <= row)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

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

__device__ __forceinline__ uint32_t item_count(const Desc &d, uint32_t len) {
    return len > d.shortmax ? (len + d.chunk - 1) / d.chunk : 1u;
}

// ------------------------------------------------------------------ set-up

__global__ void __launch_bounds__(256) setup_kernel(const __grid_constant__ Desc d, Ws w) {
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (gtid < 3) w.ctl[gtid] = 0;
    const uint64_t nacc = 2ull * (d.iters + 1) * d.ng * 32;
    for (uint64_t i = gtid; i < nacc; i += stride) w.acc[i] = 0;
    for (uint64_t i = gtid; i < (uint64_t)d.ng * 32; i += stride) w.fx_exp[i] = 1;  // normalised r0 <= 1 < 2^1
    for (uint64_t i = gtid; i < (d.rows + PLAN_TILE - 1) / PLAN_TILE; i += stride) w.plan_status[i] = 0;
}

// Partial sums of |r0| over NORM_ROWS rows of one graph, per start vector.
__global__ void __launch_bounds__(256) norm_part_kernel(const __grid_constant__ Desc d, Ws w, const double *r0) {
    __shared__ double s_part[WARPS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t b = blockIdx.x;
    int g = 0;
    while (g + 1 < (int)d.ng && d.g[g + 1].blk0 <= b) ++g;
    const BG &G = d.g[g];
    const uint64_t r_begin = (uint64_t)(b - G.blk0) * NORM_ROWS;
    const uint64_t r_end = std::min<uint64_t>(r_begin + NORM_ROWS, G.N);
    double acc = 0.0;
    if (lane < (int)d.nrhs)
        for (uint64_t i = r_begin + warp; i < r_end; i += WARPS) acc += fabs(r0[(G.row0 + i) * d.nrhs + lane]);
    s_part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
        double t = 0.0;
        for (int q = 0; q < WARPS; ++q) t += s_part[q][lane];
        w.norm_part[(uint64_t)b * 32 + lane] = t;
    }
}

// norm(r0,1) per (graph, vector): the block partials added in block order.
__global__ void norm_finish_kernel(const __grid_constant__ Desc d, Ws w) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= d.ng * 32u) return;
    const uint32_t g = t / 32, j = t % 32;
    double s = 0.0;
    for (uint32_t b = 0; b < d.g[g].nblk; ++b) s += w.norm_part[(uint64_t)(d.g[g].blk0 + b) * 32 + j];
    w.norm[t] = s;
}

// x0 = (r0 / norm) / d_out, and sum(r) of each normalised start vector.
__global__ void __launch_bounds__(256) normalize_kernel(const __grid_constant__ Desc d, Ws w, const double *r0,
                                                        float *r_out) {
    __shared__ uint64_t s_fx[WARPS][32][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t b = blockIdx.x;
    int g = 0;
    while (g + 1 < (int)d.ng && d.g[g + 1].blk0 <= b) ++g;
    const BG &G = d.g[g];
    const uint64_t r_begin = (uint64_t)(b - G.blk0) * NORM_ROWS;
    const uint64_t r_end = std::min<uint64_t>(r_begin + NORM_ROWS, G.N);
    Fx128 acc{0, 0};
    if (lane < (int)d.nrhs) {
        const double rnorm = 1.0 / w.norm[g * 32 + lane];  // a multiply per element, not a division
        for (uint64_t p = r_begin + warp; p < r_end; p += WARPS) {
            // storage position p holds vertex v; r0 and r_out are in vertex order
            const uint32_t v = pp_idx(__ldg(G.iperm + p), G.N);
            const uint64_t at = (G.row0 + v) * d.nrhs + lane;
            const float r = (float)(r0[at] * rnorm);
            fx_add(acc, r, 1);
            const float iv = G.inv[v];
            if (lane == 0) w.invp[G.row0 + p] = iv;
            w.x[0][(G.row0 + p) * d.nrhs + lane] = r * iv;
            if (d.iters == 0) r_out[at] = r;
        }
    }
    s_fx[warp][lane][0] = acc.hi;
    s_fx[warp][lane][1] = acc.lo;
    __syncthreads();
    if (warp == 0 && lane < (int)d.nrhs) {
        Fx128 t{0, 0};
        for (int q = 0; q < WARPS; ++q) fx_add(t, s_fx[q][lane][0], s_fx[q][lane][1]);
        if (t.hi | t.lo) fx_atomic_add(w.acc + 2ull * (g * 32 + lane), t);
    }
}

// Column gc (global numbering) starts a work item if it starts its graph, is
// long, follows a long column, starts in a new shortmax-entry span of its
// graph's entry array, or is a multiple of TILE_COLS within its graph.
__device__ __forceinline__ void classify(const Desc &d, uint64_t gc, bool &bound, uint32_t &nitems) {
    const int g = graph_of(d, gc);
    const BG &G = d.g[g];
    const uint32_t v = (uint32_t)(gc - G.row0);
    const uint32_t s = __ldg(G.colptr + v), e = __ldg(G.colptr + v + 1);
    nitems = item_count(d, e - s);
    bound = true;
    if (v == 0 || e - s > d.shortmax || v % TILE_COLS == 0) return;
    const uint32_t ps = __ldg(G.colptr + v - 1);
    if (s - ps > d.shortmax) return;
    bound = (s / d.shortmax) != (ps / d.shortmax);
}

__global__ void __launch_bounds__(PLAN_THREADS) plan_kernel(const __grid_constant__ Desc d, Ws w) {
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_scan[40];
    __shared__ uint64_t s_excl;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(w.ctl + 2, 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    const uint64_t ntiles = (d.rows + PLAN_TILE - 1) / PLAN_TILE;
    if (tile >= ntiles) return;
    const uint64_t c0 = tile * PLAN_TILE + (uint64_t)tid * PLAN_ITEMS;
    uint32_t bmask = 0, nitems = 0;
#pragma unroll
    for (int j = 0; j < PLAN_ITEMS; ++j) {
        if (c0 + j < d.rows) {
            bool b;
            uint32_t ni;
            classify(d, c0 + j, b, ni);
            if (b) {
                bmask |= 1u << j;
                nitems += ni;
            }
        }
    }
    const uint64_t mine = (uint64_t)__popc(bmask) | ((uint64_t)nitems << 31);
    uint64_t total;
    const uint64_t texcl = block_exclusive_sum<uint64_t, PLAN_THREADS>(mine, s_scan, &total);
    if (tid < 32) {
        // warp 0: publish this tile's counts and look back over earlier tiles
        uint64_t *st = w.plan_status + tile;
        uint64_t ex = 0;
        if (tile == 0) {
            if (tid == 0) st_relaxed_u64(st, F_INC | total);
        } else {
            if (tid == 0) st_relaxed_u64(st, F_AGG | total);
            ex = warp_lookback(w.plan_status, tile);
            if (tid == 0) st_relaxed_u64(st, F_INC | (ex + total));
        }
        if (tid == 0) {
            s_excl = ex;
            if (tile == ntiles - 1) {
                const uint64_t inc = ex + total;
                w.ctl[1] = (uint32_t)(inc & 0x7fffffffull);
                w.ctl[0] = (uint32_t)(inc >> 31);
            }
        }
    }
    __syncthreads();
    const uint64_t gsum = s_excl + texcl;
    uint32_t bi = (uint32_t)(gsum & 0x7fffffffull), ii = (uint32_t)(gsum >> 31);
#pragma unroll
    for (int j = 0; j < PLAN_ITEMS; ++j) {
        if (!(bmask >> j & 1u)) continue;
        const uint64_t gc = c0 + j;
        const uint32_t bo = pp_idx(bi, d.rows);
        w.bound[bo] = (uint32_t)gc;
        w.bound_item[bo] = ii;
        const int g = graph_of(d, gc);
        const uint32_t v = (uint32_t)(gc - d.g[g].row0);
        if (v == 0) w.first_item[g] = ii;
        ii += item_count(d, __ldg(d.g[g].colptr + v + 1) - __ldg(d.g[g].colptr + v));
        ++bi;
    }
}

__global__ void __launch_bounds__(256) plan_items_kernel(const __grid_constant__ Desc d, Ws w) {
    const uint32_t nb = w.ctl[1];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
        const uint64_t gc = w.bound[i];
        const int g = graph_of(d, gc);
        const BG &G = d.g[g];
        const uint32_t v = (uint32_t)(gc - G.row0), o = w.bound_item[i];
        const uint32_t s = __ldg(G.colptr + v), e = __ldg(G.colptr + v + 1);
        if (e - s > d.shortmax) {
            // graphs here have scale <= 24: a kept column has < 2^27 entries, so nc < 2^20
            const uint32_t nc = (e - s + d.chunk - 1) / d.chunk;
            for (uint32_t k = 0; k < nc; ++k) {
                const uint32_t cs = s + k * d.chunk;
                const uint32_t oi = pp_idx(o + k, d.item_cap);
                w.item[oi] = make_uint4(v | LONG_FLAG, o, cs, min(d.chunk, e - cs) | (nc << 12));
                w.item_g[oi] = (uint8_t)g;
                w.ticket[oi] = 0;
            }
        } else {
            // the tile runs to the next boundary of the same graph, or to the graph's end
            uint32_t c1 = G.N;
            if (i + 1 < nb && w.bound[i + 1] < G.row0 + G.N) c1 = (uint32_t)(w.bound[i + 1] - G.row0);
            const uint32_t oi = pp_idx(o, d.item_cap);
            w.item[oi] = make_uint4(v, c1 - v, s, __ldg(G.colptr + c1) - s);
            w.item_g[oi] = (uint8_t)g;
        }
    }
}

// --------------------------------------------------------------- iteration

// Compensated (Kahan) running sum: each column and vector is summed in entry
// order in binary32 with a correction term, so the error does not grow with
// the column length.
struct KSum {
    float s, comp;
    __device__ __forceinline__ void add(float x) {
        const float y = x - comp;
        const float t = s + y;
        comp = (t - s) - y;
        s = t;
    }
};

template <bool LAST>
__global__ void __launch_bounds__(THREADS) iterate_kernel(const __grid_constant__ Desc d, Ws w, const float *x_in,
                                                          float *x_out, float *r_out, uint32_t iter) {
    __shared__ uint32_t s_rowc[WARPS][TILE_ENTRIES];
    __shared__ uint32_t s_cp[WARPS][TILE_COLS + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool active = lane < (int)d.nrhs;
    const uint32_t nrhs = d.nrhs;
    const uint32_t n_items = pp_len(0, w.ctl[0], d.item_cap);
    const uint32_t nwarps = gridDim.x * WARPS;
    const float cc = (float)d.c;
    const uint64_t keep = policy_evict_last(), stream = policy_evict_first();
    uint32_t *rowc_s = s_rowc[warp];
    uint32_t *cp = s_cp[warp];
    unsigned long long *acc_now = w.acc + 2ull * iter * d.ng * 32;
    unsigned long long *acc_next = w.acc + 2ull * (iter + 1) * d.ng * 32;

    int cur = -1;
    Fx128 acc{0, 0};
    float tele = 0.f;
    int E = 1;
    for (uint32_t item = blockIdx.x * WARPS + warp; item < n_items; item += nwarps) {
        const uint4 it = __ldg(w.item + item);
        const int g = pp_idx((int)__ldg(w.item_g + item), (int)d.ng);
        if (g != cur) {
            if (cur >= 0 && active && (acc.hi | acc.lo)) fx_atomic_add(acc_next + 2 * (cur * 32 + lane), acc);
            acc = Fx128{0, 0};
            cur = g;
            const int slot = g * 32 + (active ? lane : 0);
            const double S = fx_value(acc_now[2 * slot], acc_now[2 * slot + 1], w.fx_exp[iter * d.ng * 32 + slot]);
            E = fx_exponent(S);
            tele = (float)(((1.0 - d.c) / (double)d.g[g].N) * S);
            if (item == w.first_item[g] && active) w.fx_exp[(iter + 1) * d.ng * 32 + slot] = E;
        }
        const BG &G = d.g[g];
        const float *xg = x_in + G.row0 * nrhs;
        float *xo = x_out + G.row0 * nrhs;
        float *ro = r_out + G.row0 * nrhs;
        const uint32_t umask = (1u << G.scale) - 1u;
        const float *invp = w.invp + G.row0;
        // col is a column position (vertex iperm[col]); r_out is in vertex order
        auto epi = [&](uint32_t col, float y, float invc) {
            if (!active) return;
            col = pp_idx(col, G.N);
            const float r = cc * y + tele;
            if (LAST) ro[(uint64_t)pp_idx(__ldg(G.iperm + col), G.N) * nrhs + lane] = r;
            st_hint(xo + (uint64_t)col * nrhs + lane, r * invc, keep);
            fx_add(acc, r, E);
        };
        const uint32_t e0 = it.z;
        if (it.x & LONG_FLAG) {
            const uint32_t col = pp_idx(it.x & ~LONG_FLAG, G.N), first = it.y;
            const uint32_t nent = pp_len(e0, it.w & 0xfffu, G.info[PP_INFO_NNZ]);
            // 0 (checked build) when the column's items leave the item arrays: then summed as one chunk
            const uint32_t nchunks = pp_len(first, it.w >> 12, d.item_cap);
            KSum y{0.f, 0.f};
            for (uint32_t b = 0; b < nent; b += 32) {
                const uint32_t mine = b + lane < nent ? ld_stream_u32(G.rowc + e0 + b + lane, stream) : 0u;
                const uint32_t n = min(32u, nent - b);
                for (uint32_t k = 0; k < n; k += GATHERS) {
                    float xv[GATHERS];
                    uint32_t wk[GATHERS];
#pragma unroll
                    for (int m = 0; m < GATHERS; ++m) {
                        wk[m] = __shfl_sync(0xffffffffu, mine, (k + m) & 31);
                        xv[m] = (k + m < n && active) ? ld_hint(xg + (uint64_t)(wk[m] & umask) * nrhs + lane, keep)
                                                      : 0.f;
                    }
#pragma unroll
                    for (int m = 0; m < GATHERS; ++m) {
                        if (k + m < n) {
                            uint32_t cf = wk[m] >> G.scale;
                            if (cf == G.cmax)
                                cf = ovf_lookup(G.ovf_key, G.ovf_cnt, G.info[PP_INFO_NOVF],
                                                ((uint64_t)__ldg(G.iperm + (wk[m] & umask)) << 32) |
                                                    __ldg(G.iperm + col));
                            y.add((float)cf * xv[m]);
                        }
                    }
                }
            }
            if (nchunks <= 1) {
                epi(col, y.s, invp[col]);
            } else {
                // the warp finishing the column's last chunk adds the chunk sums in order
                if (active) w.chunk_sum[(uint64_t)item * nrhs + lane] = y.s;
                __threadfence();
                __syncwarp();
                uint32_t t = 0;
                if (lane == 0) t = atomicAdd(w.ticket + first, 1u);
                t = __shfl_sync(0xffffffffu, t, 0);
                if ((t + 1) % nchunks == 0) {
                    __threadfence();
                    KSum tot{0.f, 0.f};
                    if (active)
                        for (uint32_t q = 0; q < nchunks; ++q)
                            tot.add(__ldcg(w.chunk_sum + (uint64_t)(first + q) * nrhs + lane));
                    epi(col, tot.s, invp[col]);
                }
            }
        } else {
            const uint32_t c0 = it.x, ncol = pp_len(c0, pp_len(0, it.y, TILE_COLS), G.N);
            const uint32_t nent = pp_len(e0, pp_len(0, it.w, TILE_ENTRIES), G.info[PP_INFO_NNZ]);
            if (lane < (int)ncol) cp[lane] = ld_stream_u32(G.colptr + c0 + lane, stream) - e0;
            if (lane == 0) cp[ncol] = nent;
            const float myinv = lane < (int)ncol ? invp[c0 + lane] : 0.f;
            for (uint32_t k = lane; k < nent; k += 32) rowc_s[k] = ld_stream_u32(G.rowc + e0 + k, stream);
            __syncwarp();
            // entries in order; a column is finished when its last entry has been added
            uint32_t ci = 0, next_end = cp[1];
            KSum y{0.f, 0.f};
            for (uint32_t k = 0; k < nent; k += GATHERS) {
                float xv[GATHERS];
                uint32_t wk[GATHERS];
#pragma unroll
                for (int m = 0; m < GATHERS; ++m) {
                    wk[m] = k + m < nent ? rowc_s[k + m] : 0u;
                    xv[m] = (k + m < nent && active) ? ld_hint(xg + (uint64_t)(wk[m] & umask) * nrhs + lane, keep)
                                                     : 0.f;
                }
#pragma unroll
                for (int m = 0; m < GATHERS; ++m) {
                    if (k + m < nent) {
                        while (k + m >= next_end) {
                            epi(c0 + ci, y.s, __shfl_sync(0xffffffffu, myinv, ci));
                            y = KSum{0.f, 0.f};
                            ++ci;
                            next_end = cp[pp_idx(ci + 1, ncol + 1)];
                        }
                        uint32_t cf = wk[m] >> G.scale;
                        if (cf == G.cmax)
                            cf = ovf_lookup(G.ovf_key, G.ovf_cnt, G.info[PP_INFO_NOVF],
                                            ((uint64_t)__ldg(G.iperm + (wk[m] & umask)) << 32) |
                                                __ldg(G.iperm + pp_idx(c0 + ci, G.N)));
                        y.add((float)cf * xv[m]);
                    }
                }
            }
            while (ci < ncol) {  // the last column, and empty columns at the end
                epi(c0 + ci, y.s, __shfl_sync(0xffffffffu, myinv, ci));
                y = KSum{0.f, 0.f};
                ++ci;
            }
            __syncwarp();
        }
    }
    if (cur >= 0 && active && (acc.hi | acc.lo)) fx_atomic_add(acc_next + 2 * (cur * 32 + lane), acc);
}

// ------------------------------------------------ iteration, 32 start vectors

constexpr int VEC_UNROLL = 2;  // steps of 4 entries in flight per warp

// Compensated sums of the 4 vectors of one lane, for one slot of a column.
struct KSum4 {
    KSum v[4];
    __device__ __forceinline__ void add(float cf, float4 x) {
        v[0].add(cf * x.x);
        v[1].add(cf * x.y);
        v[2].add(cf * x.z);
        v[3].add(cf * x.w);
    }
};

// The slot sums of entries [lo, hi) of the staged words ws (a column's
// entries, or a chunk of one), slot = entry index mod 4 counted from lo.
// `col` is the column position, for a count that did not fit inline.
__device__ __forceinline__ void vec_accumulate(const BG &G, const uint32_t *ws, uint32_t lo, uint32_t hi,
                                               const float *xg, uint32_t col, int slot, int quad, uint64_t keep,
                                               KSum4 &ks) {
    const uint32_t umask = (1u << G.scale) - 1u;
    for (uint32_t k = lo + slot; k < hi; k += 4 * VEC_UNROLL) {
        uint32_t wk[VEC_UNROLL];
        float4 xv[VEC_UNROLL];
#pragma unroll
        for (int m = 0; m < VEC_UNROLL; ++m) {
            const uint32_t kk = k + 4 * m;
            wk[m] = kk < hi ? ws[kk] : 0u;
            xv[m] = kk < hi ? ld_hint4(xg + (uint64_t)(wk[m] & umask) * 32u + 4 * quad, keep)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int m = 0; m < VEC_UNROLL; ++m) {
            if (k + 4 * m < hi) {
                uint32_t cf = wk[m] >> G.scale;
                if (cf == G.cmax)
                    cf = ovf_lookup(G.ovf_key, G.ovf_cnt, G.info[PP_INFO_NOVF],
                                    ((uint64_t)__ldg(G.iperm + (wk[m] & umask)) << 32) | __ldg(G.iperm + col));
                ks.add((float)cf, xv[m]);
            }
        }
    }
}

// The column total of vector `lane` from the slot sums: the 4 slots added in
// a fixed tree (all lanes of a quad then hold its 4 totals), then each lane
// takes its own vector from the quad that holds it.
__device__ __forceinline__ float vec_total(const KSum4 &ks, int lane) {
    float t[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        t[j] = ks.v[j].s;
        t[j] += __shfl_xor_sync(0xffffffffu, t[j], 8);
        t[j] += __shfl_xor_sync(0xffffffffu, t[j], 16);
    }
    const int src = lane >> 2;  // slot 0, quad lane / 4
    const float y0 = __shfl_sync(0xffffffffu, t[0], src), y1 = __shfl_sync(0xffffffffu, t[1], src);
    const float y2 = __shfl_sync(0xffffffffu, t[2], src), y3 = __shfl_sync(0xffffffffu, t[3], src);
    const int j = lane & 3;
    return j == 0 ? y0 : (j == 1 ? y1 : (j == 2 ? y2 : y3));
}

template <bool LAST>
__global__ void __launch_bounds__(THREADS) iterate_vec_kernel(const __grid_constant__ Desc d, Ws w,
                                                              const float *x_in, float *x_out, float *r_out,
                                                              uint32_t iter) {
    __shared__ uint32_t s_rowc[WARPS][TILE_ENTRIES];
    __shared__ uint32_t s_cp[WARPS][TILE_COLS + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int quad = lane & 7, slot = lane >> 3;
    const uint32_t n_items = pp_len(0, w.ctl[0], d.item_cap);
    const uint32_t nwarps = gridDim.x * WARPS;
    const float cc = (float)d.c;
    const uint64_t keep = policy_evict_last(), stream = policy_evict_first();
    uint32_t *rowc_s = s_rowc[warp];
    uint32_t *cp = s_cp[warp];
    unsigned long long *acc_now = w.acc + 2ull * iter * d.ng * 32;
    unsigned long long *acc_next = w.acc + 2ull * (iter + 1) * d.ng * 32;

    int cur = -1;
    Fx128 acc{0, 0};
    float tele = 0.f;
    int E = 1;
    for (uint32_t item = blockIdx.x * WARPS + warp; item < n_items; item += nwarps) {
        const uint4 it = __ldg(w.item + item);
        const int g = pp_idx((int)__ldg(w.item_g + item), (int)d.ng);
        if (g != cur) {
            if (cur >= 0 && (acc.hi | acc.lo)) fx_atomic_add(acc_next + 2 * (cur * 32 + lane), acc);
            acc = Fx128{0, 0};
            cur = g;
            const int sl = g * 32 + lane;
            const double S = fx_value(acc_now[2 * sl], acc_now[2 * sl + 1], w.fx_exp[iter * d.ng * 32 + sl]);
            E = fx_exponent(S);
            tele = (float)(((1.0 - d.c) / (double)d.g[g].N) * S);
            if (item == w.first_item[g]) w.fx_exp[(iter + 1) * d.ng * 32 + sl] = E;
        }
        const BG &G = d.g[g];
        const float *xg = x_in + G.row0 * 32u;
        float *xo = x_out + G.row0 * 32u;
        float *ro = r_out + G.row0 * 32u;
        const float *invp = w.invp + G.row0;
        // col is a column position (vertex iperm[col]); r_out is in vertex order; lane = vector
        auto epi = [&](uint32_t col, float y, float invc) {
            col = pp_idx(col, G.N);
            const float r = cc * y + tele;
            if (LAST) ro[(uint64_t)pp_idx(__ldg(G.iperm + col), G.N) * 32u + lane] = r;
            st_hint(xo + (uint64_t)col * 32u + lane, r * invc, keep);
            fx_add(acc, r, E);
        };
        const uint32_t e0 = it.z;
        if (it.x & LONG_FLAG) {
            const uint32_t col = pp_idx(it.x & ~LONG_FLAG, G.N), first = it.y;
            const uint32_t nent = pp_len(e0, it.w & 0xfffu, G.info[PP_INFO_NNZ]);
            // 0 (checked build) when the column's items leave the item arrays: then summed as one chunk
            const uint32_t nchunks = pp_len(first, it.w >> 12, d.item_cap);
            KSum4 ks{};
            for (uint32_t b = 0; b < nent; b += TILE_ENTRIES) {
                const uint32_t n = min((uint32_t)TILE_ENTRIES, nent - b);
                for (uint32_t k = lane; k < n; k += 32) rowc_s[k] = ld_stream_u32(G.rowc + e0 + b + k, stream);
                __syncwarp();
                vec_accumulate(G, rowc_s, 0, n, xg, col, slot, quad, keep, ks);
                __syncwarp();
            }
            const float y = vec_total(ks, lane);
            if (nchunks <= 1) {
                epi(col, y, invp[col]);
            } else {
                // the warp finishing the column's last chunk adds the chunk sums in order
                w.chunk_sum[(uint64_t)item * 32u + lane] = y;
                __threadfence();
                __syncwarp();
                uint32_t t = 0;
                if (lane == 0) t = atomicAdd(w.ticket + first, 1u);
                t = __shfl_sync(0xffffffffu, t, 0);
                if ((t + 1) % nchunks == 0) {
                    __threadfence();
                    KSum tot{0.f, 0.f};
                    for (uint32_t q = 0; q < nchunks; ++q)
                        tot.add(__ldcg(w.chunk_sum + (uint64_t)(first + q) * 32u + lane));
                    epi(col, tot.s, invp[col]);
                }
            }
        } else {
            const uint32_t c0 = it.x, ncol = pp_len(c0, pp_len(0, it.y, TILE_COLS), G.N);
            const uint32_t nent = pp_len(e0, pp_len(0, it.w, TILE_ENTRIES), G.info[PP_INFO_NNZ]);
            if (lane < (int)ncol) cp[lane] = ld_stream_u32(G.colptr + c0 + lane, stream) - e0;
            if (lane == 0) cp[ncol] = nent;
            const float myinv = lane < (int)ncol ? invp[c0 + lane] : 0.f;
            for (uint32_t k = lane; k < nent; k += 32) rowc_s[k] = ld_stream_u32(G.rowc + e0 + k, stream);
            __syncwarp();
            for (uint32_t ci = 0; ci < ncol; ++ci) {
                const uint32_t lo = cp[ci], hi = lo + pp_len(lo, cp[ci + 1] - lo, nent);
                const float invc = __shfl_sync(0xffffffffu, myinv, ci);
                if (lo == hi) {  // a column without entries (most of them): y = 0, no reduction
                    epi(c0 + ci, 0.f, invc);
                    continue;
                }
                KSum4 ks{};
                vec_accumulate(G, rowc_s, lo, hi, xg, c0 + ci, slot, quad, keep, ks);
                epi(c0 + ci, vec_total(ks, lane), invc);
            }
            __syncwarp();
        }
    }
    if (cur >= 0 && (acc.hi | acc.lo)) fx_atomic_add(acc_next + 2 * (cur * 32 + lane), acc);
}

// ------------------------------------------------------------------- host

struct Layout {
    Ws w;
    size_t bytes;
};

inline bool batch_sizes(const pp_graph *gs, uint32_t ng, uint64_t &rows, uint64_t &edges) {
    rows = 0;
    edges = 0;
    for (uint32_t g = 0; g < ng; ++g) {
        if (gs[g].scale < 1 || gs[g].scale > 24 || gs[g].M > (1ull << 31)) return false;
        rows += 1ull << gs[g].scale;
        edges += gs[g].M;
    }
    return rows < (1ull << 31) && edges < (1ull << 40);
}

inline uint64_t max_items(uint32_t ng, uint64_t rows, uint64_t edges) {
    // boundaries: graph starts, multiples of TILE_COLS, long columns, columns after
    // them, and shortmax-entry span starts; plus up to one chunk per chunk entries
    return 3ull * ng + rows / TILE_COLS + 4 * (edges / SHORTMAX_MIN) + edges / CHUNK_MIN + 64;
}

inline Layout layout(void *ws, uint32_t ng, uint64_t rows, uint64_t edges, uint32_t nrhs, uint32_t iters,
                     uint32_t nblocks) {
    Carver c(ws);
    Layout L;
    const uint64_t mi = max_items(ng, rows, edges);
    L.w.x[0] = c.take<float>(rows * nrhs);
    L.w.x[1] = c.take<float>(rows * nrhs);
    L.w.invp = c.take<float>(rows);
    L.w.bound = c.take<uint32_t>(rows);
    L.w.bound_item = c.take<uint32_t>(rows);
    L.w.item = c.take<uint4>(mi);
    L.w.item_g = c.take<uint8_t>(mi);
    L.w.chunk_sum = c.take<float>(mi * nrhs);
    L.w.ticket = c.take<uint32_t>(mi);
    L.w.first_item = c.take<uint32_t>(ng);
    L.w.plan_status = c.take<uint64_t>(ceil_div(rows, PLAN_TILE));
    L.w.acc = c.take<unsigned long long>(2ull * (iters + 1) * ng * 32);
    L.w.fx_exp = c.take<int>((uint64_t)(iters + 1) * ng * 32);
    L.w.norm_part = c.take<double>((uint64_t)nblocks * 32);
    L.w.norm = c.take<double>((uint64_t)ng * 32);
    L.w.ctl = c.take<uint32_t>(4);
    L.bytes = c.size();
    return L;
}

inline uint32_t norm_blocks(const pp_graph *gs, uint32_t ng) {
    uint64_t b = 0;
    for (uint32_t g = 0; g < ng; ++g) b += ceil_div(1ull << gs[g].scale, NORM_ROWS);
    return (uint32_t)b;
}

}  // namespace k3b
}  // namespace pp

using namespace pp;

static bool batch_args_ok(const pp_graph *gs, uint32_t ng, uint32_t nrhs) {
    if (!gs || ng == 0 || ng > PP_BATCH_MAX_GRAPHS || nrhs == 0 || nrhs > PP_BATCH_MAX_RHS) return false;
    for (uint32_t g = 0; g < ng; ++g)
        if (!gs[g].colptr || !gs[g].rowc || !gs[g].ovf_key || !gs[g].ovf_cnt || !gs[g].info || !gs[g].inv_dout32 ||
            !gs[g].perm || !gs[g].iperm)
            return false;
    return true;
}

extern "C" pp_status pp_pagerank_batched_workspace(const pp_graph *gs, uint32_t n_graphs, uint32_t nrhs,
                                                   uint32_t iters, size_t *bytes) {
    uint64_t rows, edges;
    if (!bytes || !batch_args_ok(gs, n_graphs, nrhs) || !k3b::batch_sizes(gs, n_graphs, rows, edges))
        return PP_ERR_INVALID_ARG;
    *bytes = k3b::layout(nullptr, n_graphs, rows, edges, nrhs, iters, k3b::norm_blocks(gs, n_graphs)).bytes;
    return PP_OK;
}

extern "C" pp_status pp_pagerank_batched(const pp_graph *gs, uint32_t n_graphs, const double *r0, uint32_t nrhs,
                                         uint32_t iters, double c, float *r_out, void *ws, size_t ws_bytes,
                                         void *stream) {
    PP_ENTRY("pp_pagerank_batched");
    uint64_t rows, edges;
    if (!batch_args_ok(gs, n_graphs, nrhs) || !k3b::batch_sizes(gs, n_graphs, rows, edges) || !r0 || !r_out ||
        !(c >= 0.0 && c <= 1.0))
        return PP_ERR_INVALID_ARG;
    const uint32_t nblocks = k3b::norm_blocks(gs, n_graphs);
    const k3b::Layout need = k3b::layout(nullptr, n_graphs, rows, edges, nrhs, iters, nblocks);
    pp_status st = check_ws(ws, ws_bytes, need.bytes);
    if (st != PP_OK) return st;
    const k3b::Layout L = k3b::layout(ws, n_graphs, rows, edges, nrhs, iters, nblocks);
    k3b::Desc d;
    std::memset(&d, 0, sizeof d);
    uint64_t row0 = 0;
    uint32_t blk0 = 0;
    for (uint32_t g = 0; g < n_graphs; ++g) {
        k3b::BG &G = d.g[g];
        G.colptr = gs[g].colptr;
        G.rowc = gs[g].rowc;
        G.iperm = gs[g].iperm;
        G.ovf_key = gs[g].ovf_key;
        G.ovf_cnt = gs[g].ovf_cnt;
        G.info = gs[g].info;
        G.inv = gs[g].inv_dout32;
        G.N = 1u << gs[g].scale;
        G.scale = gs[g].scale;
        G.cmax = (uint32_t)((1ull << (32 - gs[g].scale)) - 1);
        G.nblk = (uint32_t)ceil_div(G.N, k3b::NORM_ROWS);
        G.row0 = row0;
        G.blk0 = blk0;
        row0 += G.N;
        blk0 += G.nblk;
    }
    d.ng = n_graphs;
    d.item_cap = (uint32_t)k3b::max_items(n_graphs, rows, edges);
    d.nrhs = nrhs;
    d.iters = iters;
    d.rows = rows;
    d.c = c;
    d.shortmax = (uint32_t)tuning("k3b_shortmax");
    d.chunk = (uint32_t)tuning("k3b_chunk");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const k3b::Ws &w = L.w;
    k3b::setup_kernel<<<512, 256, 0, s>>>(d, w);
    k3b::norm_part_kernel<<<nblocks, 256, 0, s>>>(d, w, r0);
    k3b::norm_finish_kernel<<<(unsigned)ceil_div(n_graphs * 32ull, 256), 256, 0, s>>>(d, w);
    k3b::normalize_kernel<<<nblocks, 256, 0, s>>>(d, w, r0, r_out);
    k3b::plan_kernel<<<(unsigned)ceil_div(rows, k3b::PLAN_TILE), k3b::PLAN_THREADS, 0, s>>>(d, w);
    k3b::plan_items_kernel<<<(unsigned)std::min<uint64_t>(ceil_div(rows, 256), 4096), 256, 0, s>>>(d, w);
    count_launch(6);
    static PerDevice occ_dev;  // four 16-bit occupancies
    const uint64_t occs = (uint64_t)occ_dev.get([] {
        auto occ = [](auto kernel) {
            int o = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kernel, k3b::THREADS, 0);
            return (uint64_t)(o > 0 ? o : 1);
        };
        return (int64_t)(occ(k3b::iterate_kernel<false>) | occ(k3b::iterate_kernel<true>) << 16 |
                         occ(k3b::iterate_vec_kernel<false>) << 32 | occ(k3b::iterate_vec_kernel<true>) << 48);
    });
    const int o_mid = (int)(occs & 0xffff), o_last = (int)(occs >> 16 & 0xffff);
    const int v_mid = (int)(occs >> 32 & 0xffff), v_last = (int)(occs >> 48 & 0xffff);
    const bool vec = nrhs == 32 && tuning("k3b_vec") != 0;
    const int sms = sm_count();
    for (uint32_t it = 0; it < iters; ++it) {
        const float *xin = w.x[it & 1];
        float *xout = w.x[(it + 1) & 1];
        const bool last = it + 1 == iters;
        if (vec && last)
            k3b::iterate_vec_kernel<true><<<sms * v_last, k3b::THREADS, 0, s>>>(d, w, xin, xout, r_out, it);
        else if (vec)
            k3b::iterate_vec_kernel<false><<<sms * v_mid, k3b::THREADS, 0, s>>>(d, w, xin, xout, r_out, it);
        else if (last)
            k3b::iterate_kernel<true><<<sms * o_last, k3b::THREADS, 0, s>>>(d, w, xin, xout, r_out, it);
        else
            k3b::iterate_kernel<false><<<sms * o_mid, k3b::THREADS, 0, s>>>(d, w, xin, xout, r_out, it);
        count_launch();
    }
    return launch_status();
}
