// Kernel 3 (Sec. IV-D and the appendix): damped PageRank iterations
//
//     r(v) <- c * sum_u r(u) A(u,v) + ((1-c)/N) * sum(r)
//
// as a pull over Kernel 2's compressed columns.  With A(u,v) = count(u,v) /
// d_out(u), the sum over a column is sum_e count_e * x(u_e) for the vector
// x = r .* (1/d_out), which each iteration writes for the next one; so the
// row normalisation is folded into the gathered vector and the matrix is
// read as packed (row, count) words only.
//
// Work split: a merge path over the sequence of column ends and entries
// (Merrill & Garland, "Merge-based parallel sparse matrix-vector
// multiplication", SC'16) cuts the columns + entries into equal tiles, so
// empty, short and very long columns all cost the same per item.  A tile
// stages its column ends in shared memory, gathers count * x(u) for its
// entries with coalesced index loads, reduces each column by a segmented
// scan, and finishes the columns that end inside it: r = c*y + teleport,
// x' = r / d_out(v), and its share of sum(r) in binary64.  A column that
// started in earlier tiles adds their published partial sums in a fixed
// order.  The sum(r) of the next iteration is reduced in a fixed two-level
// tree, so results are bitwise reproducible.
#include <cuda_bf16.h>

#include <algorithm>

#include "pp_common.cuh"

PP_DEFINE_ERROR_WORD(k3_fetch_error)

namespace pp {
namespace k3 {

constexpr int THREADS = 256;
constexpr int ITEMS = 8;
constexpr int D = THREADS * ITEMS;  // merge items (column ends + entries) per tile
constexpr int GROUP = 256;          // tiles whose partial sums are reduced together
constexpr int SETUP_BLOCKS = 512;   // fixed, so the start-vector reductions are reproducible

struct Carry {
    double val;
    uint32_t col;
    uint32_t epoch;
};

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
    uint32_t ntiles;
    uint32_t ngroups;
    uint32_t init_ticket;
    uint32_t pad;
};

struct Args {
    uint32_t N, scale, cmax, iters;
    const uint32_t *colptr, *rowc;
    const uint64_t *ovf_key;
    const uint32_t *ovf_cnt;
    const uint64_t *info;
    uint2 *coord;       // [max_tiles + 1] (column, entry) at each tile's start
    Carry *carry;       // [max_tiles]
    double *partial;    // [max_tiles]
    double *gpartial;   // [max_groups]
    double *shist;      // [iters + 1]: sum(r) before each iteration, then of the result
    double *ipart;      // [2 * SETUP_BLOCKS]
    Ctl *ctl;
    uint32_t *tile_ctr; // [iters]
    uint32_t *ticket;   // [iters]
    uint32_t *gticket;  // [iters * max_groups]
    uint32_t max_groups;
    double c;
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

// Plan the tiles, reset the per-call counters and sum |r0|.
__global__ void __launch_bounds__(256) setup_kernel(Args a, const double *r0) {
    __shared__ double s_red[32];
    const uint64_t nnz = a.info[PP_INFO_NNZ];
    const uint64_t total = (uint64_t)a.N + nnz;
    const uint32_t ntiles = (uint32_t)((total + D - 1) / D);
    const uint32_t ngroups = (ntiles + GROUP - 1) / GROUP;
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (gtid == 0) {
        a.ctl->ntiles = ntiles;
        a.ctl->ngroups = ngroups;
        a.ctl->init_ticket = 0;
    }
    for (uint64_t t = gtid; t <= ntiles; t += stride) {
        const uint64_t diag = std::min<uint64_t>(t * D, total);
        // merge path: column end i (= colptr[i+1]) comes before entry j iff colptr[i+1] <= j
        uint64_t lo = diag > nnz ? diag - nnz : 0, hi = std::min<uint64_t>(diag, a.N);
        while (lo < hi) {
            const uint64_t pivot = (lo + hi) >> 1;
            if ((uint64_t)__ldg(a.colptr + pivot + 1) + pivot + 1 <= diag)
                lo = pivot + 1;
            else
                hi = pivot;
        }
        a.coord[t] = make_uint2((uint32_t)lo, (uint32_t)(diag - lo));
    }
    for (uint64_t t = gtid; t < ntiles; t += stride) a.carry[t].epoch = 0;
    for (uint64_t i = gtid; i < a.iters; i += stride) {
        a.tile_ctr[i] = 0;
        a.ticket[i] = 0;
    }
    for (uint64_t i = gtid; i < (uint64_t)a.iters * a.max_groups; i += stride) a.gticket[i] = 0;
    double acc = 0.0;
    for (uint64_t i = gtid; i < a.N; i += stride) acc += fabs(r0[i]);
    const double bs = block_sum<double, 256>(acc, s_red);
    if (threadIdx.x == 0) a.ipart[blockIdx.x] = bs;
}

// r = r0 / norm(r0,1) rounded to the working precision; x = r / d_out; and
// sum(r) of that vector.  With iters == 0 the normalised r is the result.
template <typename TS, typename TA, typename TO>
__global__ void __launch_bounds__(256) normalize_kernel(Args a, const double *r0, const TA *inv, TS *x0,
                                                        TO *r_out) {
    __shared__ double s_red[32];
    __shared__ double s_norm;
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        double n = 0.0;
        for (int b = 0; b < SETUP_BLOCKS; ++b) n += __ldcg(a.ipart + b);
        s_norm = n;
    }
    __syncthreads();
    const double norm = s_norm;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    double acc = 0.0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += stride) {
        const TA r = (TA)(r0[i] / norm);
        acc += (double)r;
        x0[i] = from_acc<TS>(r * inv[i]);
        if (a.iters == 0) r_out[i] = (TO)r;
    }
    const double bs = block_sum<double, 256>(acc, s_red);
    if (threadIdx.x == 0) {
        a.ipart[SETUP_BLOCKS + blockIdx.x] = bs;
        __threadfence();
        s_last = atomicAdd(&a.ctl->init_ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        double s = 0.0;
        for (int b = 0; b < SETUP_BLOCKS; ++b) s += __ldcg(a.ipart + SETUP_BLOCKS + b);
        a.shist[0] = s;
    }
}

// One iteration.  Persistent: each block takes tiles in order from a counter.
template <typename TS, typename TA, typename TO, bool LAST>
__global__ void __launch_bounds__(THREADS) iterate_kernel(Args a, const TA *inv, const TS *__restrict__ x_in,
                                                          TS *__restrict__ x_out, TO *r_out, uint32_t iter) {
    __shared__ uint32_t s_colend[D];
    __shared__ TA s_prod[D];
    __shared__ TA s_out[D];
    __shared__ TA s_wv[THREADS / 32];
    __shared__ int s_wf[THREADS / 32];
    __shared__ double s_red[32];
    __shared__ uint32_t s_tile;
    __shared__ int s_flag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t ntiles = a.ctl->ntiles;
    const uint32_t ngroups = a.ctl->ngroups;
    const double S = a.shist[iter];
    const TA tele = (TA)(((1.0 - a.c) / (double)a.N) * S);
    const TA cc = (TA)a.c;
    const uint32_t umask = (1u << a.scale) - 1u;
    const uint64_t novf = a.info[PP_INFO_NOVF];
    const uint32_t epoch = iter + 1;

    while (true) {
        if (tid == 0) s_tile = atomicAdd(a.tile_ctr + iter, 1u);
        __syncthreads();
        const uint32_t t = s_tile;
        if (t >= ntiles) break;
        const uint2 c0 = a.coord[t], c1 = a.coord[t + 1];
        const uint32_t i0 = c0.x, j0 = c0.y;
        const int ncol = (int)(c1.x - c0.x), nent = (int)(c1.y - c0.y);

        for (int k = tid; k < ncol; k += THREADS) s_colend[k] = __ldg(a.colptr + i0 + 1 + k);
        __syncthreads();

        // Gather count * x(u) for the tile's entries (coalesced index loads).
#pragma unroll
        for (int m = 0; m < ITEMS; ++m) {
            const int k = tid + m * THREADS;
            if (k < nent) {
                const uint32_t w = __ldg(a.rowc + j0 + k);
                const uint32_t u = w & umask;
                uint32_t cf = w >> a.scale;
                const TA xv = to_acc(x_in[u]);
                if (cf == a.cmax) {
                    // the count did not fit inline: find the column, then the overflow entry
                    int lo = 0, hi = ncol;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (s_colend[mid] <= j0 + (uint32_t)k)
                            lo = mid + 1;
                        else
                            hi = mid;
                    }
                    const uint32_t v = i0 + (uint32_t)lo;
                    cf = ovf_lookup(a.ovf_key, a.ovf_cnt, novf, ((uint64_t)u << 32) | v);
                }
                s_prod[k] = (TA)cf * xv;
            }
        }
        __syncthreads();

        // This thread's stretch of the tile's merge path.
        const int total = ncol + nent;
        const int d0 = min(tid * ITEMS, total), d1 = min(d0 + ITEMS, total);
        int lo = max(d0 - nent, 0), hi = min(d0, ncol);
        while (lo < hi) {
            const int pivot = (lo + hi) >> 1;
            if ((int)(s_colend[pivot] - j0) <= d0 - pivot - 1)
                lo = pivot + 1;
            else
                hi = pivot;
        }
        int ci = lo, ej = d0 - lo;
        TA running = TA(0);
        int first = -1;
        for (int it = d0; it < d1; ++it) {
            if (ci < ncol && (int)(s_colend[ci] - j0) <= ej) {
                s_out[ci] = running;
                if (first < 0) first = ci;
                running = TA(0);
                ++ci;
            } else {
                running += s_prod[ej];
                ++ej;
            }
        }

        // Segmented scan of the threads' open partial sums, in thread order.
        int f = first >= 0;
        TA v = running;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const TA vu = __shfl_up_sync(0xffffffffu, v, o);
            const int fu = __shfl_up_sync(0xffffffffu, f, o);
            if (lane >= o) {
                if (!f) v = vu + v;
                f |= fu;
            }
        }
        if (lane == 31) {
            s_wv[warp] = v;
            s_wf[warp] = f;
        }
        __syncthreads();
        // carry into this warp from the warps before it
        TA wc = TA(0);
        for (int w = 0; w < warp; ++w) wc = s_wf[w] ? s_wv[w] : wc + s_wv[w];
        TA ev = __shfl_up_sync(0xffffffffu, v, 1);
        int ef = __shfl_up_sync(0xffffffffu, f, 1);
        if (lane == 0) {
            ev = TA(0);
            ef = 0;
        }
        const TA cin = ef ? ev : wc + ev;
        if (first >= 0) s_out[first] += cin;
        if (tid == THREADS - 1) {
            // this tile's partial sum of column c1.x, which continues in later tiles
            const TA cout = f ? v : wc + v;
            a.carry[t].val = (double)cout;
            a.carry[t].col = c1.x;
            __threadfence();
            st_release_u32(&a.carry[t].epoch, epoch);
        }
        __syncthreads();

        // A first column that began before this tile collects the earlier tiles' partials.
        if (tid == 0 && ncol > 0) {
            const uint32_t start = __ldg(a.colptr + i0);
            if (start < j0) {
                TA acc = TA(0);
                uint32_t p = t - 1;
                while (true) {
                    uint32_t spins = 0;
                    while (ld_acquire_u32(&a.carry[p].epoch) != epoch) {
                        if (++spins > kSpinLimit) {
                            pp_set_error(PP_DEV_TIMEOUT);
                            break;
                        }
                        backoff(spins);
                    }
                    acc += (TA)__ldcg(&a.carry[p].val);
                    if (a.coord[p].y <= start || p == 0) break;
                    --p;
                }
                s_out[0] += acc;
            }
        }
        __syncthreads();

        // Finish the columns that end in this tile.
        double part = 0.0;
        for (int k = tid; k < ncol; k += THREADS) {
            const uint32_t col = i0 + (uint32_t)k;
            const TA r = cc * s_out[k] + tele;
            if (LAST) r_out[col] = (TO)r;
            x_out[col] = from_acc<TS>(r * inv[col]);
            part += (double)r;
        }
        const double bs = block_sum<double, THREADS>(part, s_red);
        if (tid == 0) {
            a.partial[t] = bs;
            __threadfence();
            const uint32_t g = t / GROUP;
            const uint32_t gsize = min((uint32_t)GROUP, ntiles - g * GROUP);
            int last = 0;
            if (atomicAdd(a.gticket + (uint64_t)iter * a.max_groups + g, 1u) == gsize - 1) {
                __threadfence();
                double gs = 0.0;
                for (uint32_t q = 0; q < gsize; ++q) gs += __ldcg(a.partial + g * GROUP + q);
                a.gpartial[g] = gs;
                __threadfence();
                last = atomicAdd(a.ticket + iter, 1u) == ngroups - 1;
            }
            s_flag = last;
        }
        __syncthreads();
        if (s_flag) {
            __threadfence();
            double acc = 0.0;
            for (uint32_t q = tid; q < ngroups; q += THREADS) acc += __ldcg(a.gpartial + q);
            const double tot = block_sum<double, THREADS>(acc, s_red);
            if (tid == 0) a.shist[iter + 1] = tot;
        }
        __syncthreads();
    }
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
    uint2 *coord;
    Carry *carry;
    double *partial, *gpartial, *shist, *ipart;
    Ctl *ctl;
    uint32_t *tile_ctr, *ticket, *gticket;
    uint32_t max_tiles, max_groups;
    size_t bytes;
};

inline Layout layout(void *ws, uint64_t M, uint32_t scale, uint32_t iters, pp_dtype dt) {
    Carver c(ws);
    Layout L;
    const uint64_t N = 1ull << scale;
    const size_t xs = dt == PP_FP64 ? 8 : (dt == PP_FP32 ? 4 : 2);
    L.max_tiles = (uint32_t)ceil_div(N + M, D) + 1;
    L.max_groups = (uint32_t)ceil_div(L.max_tiles, GROUP) + 1;
    L.x[0] = c.take<char>(N * xs);
    L.x[1] = c.take<char>(N * xs);
    L.coord = c.take<uint2>((uint64_t)L.max_tiles + 1);
    L.carry = c.take<Carry>(L.max_tiles);
    L.partial = c.take<double>(L.max_tiles);
    L.gpartial = c.take<double>(L.max_groups);
    L.shist = c.take<double>((uint64_t)iters + 1);
    L.ipart = c.take<double>(2 * SETUP_BLOCKS);
    L.ctl = c.take<Ctl>(1);
    L.tile_ctr = c.take<uint32_t>(iters ? iters : 1);
    L.ticket = c.take<uint32_t>(iters ? iters : 1);
    L.gticket = c.take<uint32_t>((uint64_t)(iters ? iters : 1) * L.max_groups);
    L.bytes = c.size();
    return L;
}

template <typename TS, typename TA, typename TO>
pp_status run(const pp_graph *g, const double *r0, uint32_t iters, double c, pp_dtype dt, TO *r_out,
              double *r_l1, const Layout &L, cudaStream_t s) {
    const uint32_t N = 1u << g->scale;
    Args a;
    a.N = N;
    a.scale = g->scale;
    a.cmax = (uint32_t)((1ull << (32 - g->scale)) - 1);
    a.iters = iters;
    a.colptr = g->colptr;
    a.rowc = g->rowc;
    a.ovf_key = g->ovf_key;
    a.ovf_cnt = g->ovf_cnt;
    a.info = g->info;
    a.coord = L.coord;
    a.carry = L.carry;
    a.partial = L.partial;
    a.gpartial = L.gpartial;
    a.shist = L.shist;
    a.ipart = L.ipart;
    a.ctl = L.ctl;
    a.tile_ctr = L.tile_ctr;
    a.ticket = L.ticket;
    a.gticket = L.gticket;
    a.max_groups = L.max_groups;
    a.c = c;
    const TA *inv = dt == PP_FP64 ? reinterpret_cast<const TA *>(g->inv_dout64)
                                  : reinterpret_cast<const TA *>(g->inv_dout32);
    if (!inv) return PP_ERR_INVALID_ARG;
    TS *x0 = static_cast<TS *>(L.x[0]);
    TS *x1 = static_cast<TS *>(L.x[1]);
    setup_kernel<<<SETUP_BLOCKS, 256, 0, s>>>(a, r0);
    normalize_kernel<TS, TA, TO><<<SETUP_BLOCKS, 256, 0, s>>>(a, r0, inv, x0, r_out);
    count_launch(2);

    static int occ[2][3] = {{0, 0, 0}, {0, 0, 0}};
    int &o_mid = occ[0][(int)dt], &o_last = occ[1][(int)dt];
    if (!o_mid) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o_mid, iterate_kernel<TS, TA, TO, false>, THREADS, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o_last, iterate_kernel<TS, TA, TO, true>, THREADS, 0);
        if (o_mid < 1) o_mid = 1;
        if (o_last < 1) o_last = 1;
    }
    const int sms = sm_count();
    for (uint32_t it = 0; it < iters; ++it) {
        const TS *xin = (it & 1) ? x1 : x0;
        TS *xout = (it & 1) ? x0 : x1;
        if (it + 1 == iters)
            iterate_kernel<TS, TA, TO, true><<<sms * o_last, THREADS, 0, s>>>(a, inv, xin, xout, r_out, it);
        else
            iterate_kernel<TS, TA, TO, false><<<sms * o_mid, THREADS, 0, s>>>(a, inv, xin, xout, r_out, it);
        count_launch();
    }
    if (r_l1) {
        l1_sum_kernel<TO><<<SETUP_BLOCKS, 256, 0, s>>>(r_out, N, L.ipart);
        l1_scale_kernel<TO><<<SETUP_BLOCKS, 256, 0, s>>>(r_out, N, L.ipart, r_l1);
        count_launch(2);
    }
    return launch_status();
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
    if (!g->colptr || !g->rowc || !g->ovf_key || !g->ovf_cnt || !g->info) return PP_ERR_INVALID_ARG;
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
