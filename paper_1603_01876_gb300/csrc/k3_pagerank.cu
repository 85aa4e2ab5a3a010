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
// scan, and finishes the columns that end inside it: r = c*y + teleport and
// x' = r / d_out(v).  A column that started in earlier tiles adds their
// published partial sums in a fixed order.  sum(r) for the next iteration is
// accumulated exactly in 128-bit fixed point, so it does not depend on which
// block took which tile and results are bitwise reproducible.
#include <cuda_bf16.h>

#include <algorithm>

#include "pp_common.cuh"

PP_DEFINE_ERROR_WORD(k3_fetch_error)

namespace pp {
namespace k3 {

constexpr int THREADS = 256;
constexpr int ITEMS_F32 = 12;       // merge items per thread: binary32 / bfloat16 ranks
constexpr int ITEMS_F64 = 8;        // binary64 ranks (twice the shared memory per item)
constexpr int D_MIN = THREADS * ITEMS_F64;
constexpr int SETUP_BLOCKS = 512;   // fixed, so the start-vector reduction is reproducible

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
    uint32_t pad[3];
};

struct Args {
    uint32_t N, scale, cmax, iters;
    uint32_t D;         // merge items per tile
    const uint32_t *colptr, *rowc;
    const uint64_t *ovf_key;
    const uint32_t *ovf_cnt;
    const uint64_t *info;
    uint2 *coord;       // [max_tiles + 1] (column, entry) at each tile's start
    Carry *carry;       // [max_tiles]
    unsigned long long *acc;  // [2 * (iters + 1)]: sum(r) before each iteration (and of
                              // the result) in 128-bit fixed point, hi then lo
    int *fx_exp;              // [iters + 1]: the scale exponent E of each accumulator
    double *ipart;      // [SETUP_BLOCKS]
    Ctl *ctl;
    uint32_t *tile_ctr; // [iters]
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
    const uint64_t D = a.D;
    const uint32_t ntiles = (uint32_t)((total + D - 1) / D);
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (gtid == 0) a.ctl->ntiles = ntiles;
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
    for (uint64_t i = gtid; i < a.iters; i += stride) a.tile_ctr[i] = 0;
    for (uint64_t i = gtid; i < 2ull * (a.iters + 1); i += stride) a.acc[i] = 0;
    if (gtid == 0) a.fx_exp[0] = 1;  // the normalised start vector has every entry <= 1 < 2^1
    double acc = 0.0;
    for (uint64_t i = gtid; i < a.N; i += stride) acc += fabs(r0[i]);
    const double bs = block_sum<double, 256>(acc, s_red);
    if (threadIdx.x == 0) a.ipart[blockIdx.x] = bs;
}

// Exact, order-independent accumulation of non-negative doubles in 128-bit
// fixed point whose last bit is worth 2^(E-100), where 2^E bounds every term
// (E is derived from the previous sum(r), which bounds every new rank because
// the update never increases the total).  Any grouping of the same terms
// gives the same bits, so sum(r) does not depend on which block took which
// tile, and terms below 2^(E-100) are the only ones truncated.
struct Fx128 {
    uint64_t hi, lo;
};

__device__ __forceinline__ void fx_add(Fx128 &a, uint64_t h, uint64_t l) {
    a.lo += l;
    a.hi += h + (a.lo < l ? 1ull : 0ull);
}

__device__ __forceinline__ void fx_add(Fx128 &a, double x, int E) {
    if (!(x > 0.0)) return;
    const uint64_t bits = (uint64_t)__double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7ff);
    const uint64_t m = (bits & ((1ull << 52) - 1)) | (e ? (1ull << 52) : 0ull);
    const int sh = (e ? e : 1) - 1075 + 100 - E;  // x = m * 2^(sh + E - 100)
    uint64_t h = 0, l = 0;
    if (sh <= -64) {
        return;
    } else if (sh < 0) {
        l = m >> (-sh);
    } else if (sh == 0) {
        l = m;
    } else if (sh < 64) {
        l = m << sh;
        h = m >> (64 - sh);
    } else if (sh < 75) {
        h = m << (sh - 64);
    } else {
        h = ~0ull;  // cannot happen for terms below 2^(E+11); saturate rather than wrap
    }
    fx_add(a, h, l);
}

__device__ __forceinline__ double fx_value(uint64_t hi, uint64_t lo, int E) {
    return ldexp((double)hi, E - 36) + ldexp((double)lo, E - 100);
}

// Exponent for the next accumulator: 2^E > S >= any rank of the next iterate.
__device__ __forceinline__ int fx_exponent(double S) {
    int e = 0;
    frexp(S, &e);
    return e + 1;
}

template <int THREADS_>
__device__ __forceinline__ Fx128 fx_block_sum(Fx128 a, uint64_t *scratch /* 2 * warps */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t h = __shfl_down_sync(0xffffffffu, a.hi, o);
        const uint64_t l = __shfl_down_sync(0xffffffffu, a.lo, o);
        fx_add(a, h, l);
    }
    if (lane == 0) {
        scratch[2 * warp] = a.hi;
        scratch[2 * warp + 1] = a.lo;
    }
    __syncthreads();
    Fx128 t{0, 0};
    if (threadIdx.x == 0)
        for (int w = 0; w < THREADS_ / 32; ++w) fx_add(t, scratch[2 * w], scratch[2 * w + 1]);
    __syncthreads();
    return t;
}

__device__ __forceinline__ void fx_atomic_add(unsigned long long *acc /* [hi, lo] */, Fx128 v) {
    const unsigned long long old = atomicAdd(acc + 1, (unsigned long long)v.lo);
    const unsigned long long carry = (old + v.lo < old) ? 1ull : 0ull;
    if (v.hi + carry) atomicAdd(acc, (unsigned long long)(v.hi + carry));
}

template <typename TS>
__device__ __forceinline__ TS ldg_x(const TS *p) { return __ldg(p); }

// r = r0 / norm(r0,1) rounded to the working precision; x = r / d_out; and
// sum(r) of that vector.  With iters == 0 the normalised r is the result.
template <typename TS, typename TA, typename TO>
__global__ void __launch_bounds__(256) normalize_kernel(Args a, const double *r0, const TA *inv, TS *x0,
                                                        TO *r_out) {
    __shared__ double s_norm;
    __shared__ uint64_t s_fx[16];
    if (threadIdx.x == 0) {
        double n = 0.0;
        for (int b = 0; b < SETUP_BLOCKS; ++b) n += a.ipart[b];
        s_norm = n;
    }
    __syncthreads();
    const double norm = s_norm;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    Fx128 acc{0, 0};
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += stride) {
        const TA r = (TA)(r0[i] / norm);
        fx_add(acc, (double)r, 1);
        x0[i] = from_acc<TS>(r * inv[i]);
        if (a.iters == 0) r_out[i] = (TO)r;
    }
    const Fx128 bt = fx_block_sum<256>(acc, s_fx);
    if (threadIdx.x == 0 && (bt.hi | bt.lo)) fx_atomic_add(a.acc, bt);
}

// One iteration.  Persistent: each block claims tiles in order from a counter
// (the next claim is issued while the current tile is processed).
template <typename TS, typename TA, typename TO, bool LAST, int ITEMS>
__global__ void __launch_bounds__(THREADS) iterate_kernel(Args a, const TA *inv, const TS *__restrict__ x_in,
                                                          TS *__restrict__ x_out, TO *r_out, uint32_t iter) {
    constexpr int DT = THREADS * ITEMS;
    constexpr int W = THREADS / 32;
    __shared__ uint32_t s_colend[DT];
    __shared__ TA s_prod[DT];
    __shared__ TA s_y[DT];
    __shared__ TA s_wv[W];
    __shared__ int s_wf[W];
    __shared__ uint64_t s_fx[2 * W];
    __shared__ TA s_tcin;
    __shared__ uint32_t s_next;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t ntiles = a.ctl->ntiles;
    const double S = fx_value(a.acc[2 * iter], a.acc[2 * iter + 1], a.fx_exp[iter]);
    const int E = fx_exponent(S);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.fx_exp[iter + 1] = E;
    const TA tele = (TA)(((1.0 - a.c) / (double)a.N) * S);
    const TA cc = (TA)a.c;
    const uint32_t umask = (1u << a.scale) - 1u;
    const uint32_t epoch = iter + 1;
    uint32_t *ctr = a.tile_ctr + iter;
    Fx128 acc{0, 0};

    if (tid == 0) s_next = atomicAdd(ctr, 1u);
    __syncthreads();
    while (true) {
        const uint32_t t = s_next;
        if (t >= ntiles) break;
        uint32_t nxt = 0;
        if (tid == 0) nxt = atomicAdd(ctr, 1u);
        const uint2 c0 = a.coord[t], c1 = a.coord[t + 1];
        const uint32_t i0 = c0.x, j0 = c0.y;
        const int ncol = (int)(c1.x - c0.x), nent = (int)(c1.y - c0.y);

        for (int k = tid; k < ncol; k += THREADS) s_colend[k] = __ldg(a.colptr + i0 + 1 + k);

        // Gather count * x(u): all index loads first, then all gathers.
        uint32_t w[ITEMS];
#pragma unroll
        for (int m = 0; m < ITEMS; ++m) {
            const int k = tid + m * THREADS;
            w[m] = k < nent ? __ldg(a.rowc + j0 + k) : 0u;
        }
        TA xv[ITEMS];
#pragma unroll
        for (int m = 0; m < ITEMS; ++m) {
            const int k = tid + m * THREADS;
            xv[m] = k < nent ? to_acc(ldg_x(x_in + (w[m] & umask))) : TA(0);
        }
        int esc = 0;
#pragma unroll
        for (int m = 0; m < ITEMS; ++m) {
            const int k = tid + m * THREADS;
            if (k < nent) {
                const uint32_t cf = w[m] >> a.scale;
                esc |= cf == a.cmax;
                s_prod[k] = (TA)cf * xv[m];
            }
        }
        if (__syncthreads_or(esc)) {
            // a count that did not fit inline: find its column, then the overflow entry
#pragma unroll
            for (int m = 0; m < ITEMS; ++m) {
                const int k = tid + m * THREADS;
                if (k < nent && (w[m] >> a.scale) == a.cmax) {
                    int lo = 0, hi = ncol;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (s_colend[mid] <= j0 + (uint32_t)k)
                            lo = mid + 1;
                        else
                            hi = mid;
                    }
                    const uint32_t u = w[m] & umask, v = i0 + (uint32_t)lo;
                    s_prod[k] = (TA)ovf_lookup(a.ovf_key, a.ovf_cnt, a.info[PP_INFO_NOVF], ((uint64_t)u << 32) | v) * xv[m];
                }
            }
            __syncthreads();
        }

        // This thread's stretch of the merge path: first walk finds where its
        // first column ends and its open partial sum.
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
        const int ci0 = lo, ej0 = d0 - lo;
        TA running = TA(0);
        int f = 0;
        {
            int ci = ci0, ej = ej0;
            for (int it = d0; it < d1; ++it) {
                if (ci < ncol && (int)(s_colend[ci] - j0) <= ej) {
                    f = 1;
                    running = TA(0);
                    ++ci;
                } else {
                    running += s_prod[ej];
                    ++ej;
                }
            }
        }
        // Segmented scan of the open partial sums in thread order.
        TA v = running;
        int fl = f;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const TA vu = __shfl_up_sync(0xffffffffu, v, o);
            const int fu = __shfl_up_sync(0xffffffffu, fl, o);
            if (lane >= o) {
                if (!fl) v = vu + v;
                fl |= fu;
            }
        }
        if (lane == 31) {
            s_wv[warp] = v;
            s_wf[warp] = fl;
        }
        TA ev = __shfl_up_sync(0xffffffffu, v, 1);
        int ef = __shfl_up_sync(0xffffffffu, fl, 1);
        if (lane == 0) {
            ev = TA(0);
            ef = 0;
        }
        if (tid == 0) s_tcin = TA(0);
        __syncthreads();
        TA wc = TA(0);
        for (int q = 0; q < warp; ++q) wc = s_wf[q] ? s_wv[q] : wc + s_wv[q];
        const TA cin = ef ? ev : wc + ev;
        if (tid == THREADS - 1) {
            // this tile's own partial sum of column c1.x, which ends in a later tile
            a.carry[t].val = (double)(fl ? v : wc + v);
            a.carry[t].col = c1.x;
            st_release_u32(&a.carry[t].epoch, epoch);
        }
        if (tid == 0 && ncol > 0) {
            // the first column began in earlier tiles: add their partials, nearest first
            const uint32_t start = __ldg(a.colptr + i0);
            if (start < j0) {
                TA tacc = TA(0);
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
                    tacc += (TA)__ldcg(&a.carry[p].val);
                    if (a.coord[p].y <= start || p == 0) break;
                    --p;
                }
                s_tcin = tacc;
            }
        }
        // Second walk: the sums of the columns that end here, carry-in first.
        {
            int ci = ci0, ej = ej0;
            TA run = cin;
            for (int it = d0; it < d1; ++it) {
                if (ci < ncol && (int)(s_colend[ci] - j0) <= ej) {
                    s_y[ci] = run;
                    run = TA(0);
                    ++ci;
                } else {
                    run += s_prod[ej];
                    ++ej;
                }
            }
        }
        if (tid == 0) s_next = nxt;
        __syncthreads();

        // Finish the columns that end in this tile.
        for (int k = tid; k < ncol; k += THREADS) {
            const uint32_t col = i0 + (uint32_t)k;
            const TA y = k == 0 ? s_y[0] + s_tcin : s_y[k];
            const TA r = cc * y + tele;
            if (LAST) r_out[col] = (TO)r;
            x_out[col] = from_acc<TS>(r * inv[col]);
            fx_add(acc, (double)r, E);
        }
    }
    const Fx128 bt = fx_block_sum<THREADS>(acc, s_fx);
    if (tid == 0 && (bt.hi | bt.lo)) fx_atomic_add(a.acc + 2 * (iter + 1), bt);
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
    unsigned long long *acc;
    int *fx_exp;
    double *ipart;
    Ctl *ctl;
    uint32_t *tile_ctr;
    uint32_t max_tiles;
    size_t bytes;
};

inline Layout layout(void *ws, uint64_t M, uint32_t scale, uint32_t iters, pp_dtype dt) {
    Carver c(ws);
    Layout L;
    const uint64_t N = 1ull << scale;
    const size_t xs = dt == PP_FP64 ? 8 : (dt == PP_FP32 ? 4 : 2);
    L.max_tiles = (uint32_t)ceil_div(N + M, D_MIN) + 1;
    L.x[0] = c.take<char>(N * xs);
    L.x[1] = c.take<char>(N * xs);
    L.coord = c.take<uint2>((uint64_t)L.max_tiles + 1);
    L.carry = c.take<Carry>(L.max_tiles);
    L.acc = c.take<unsigned long long>(2ull * (iters + 1));
    L.fx_exp = c.take<int>((uint64_t)iters + 1);
    L.ipart = c.take<double>(SETUP_BLOCKS);
    L.ctl = c.take<Ctl>(1);
    L.tile_ctr = c.take<uint32_t>(iters ? iters : 1);
    L.bytes = c.size();
    return L;
}

template <typename K>
inline int occupancy(K kernel) {
    int o = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kernel, THREADS, 0);
    return o > 0 ? o : 1;
}

template <typename TS, typename TA, typename TO, int ITEMS>
pp_status run(const pp_graph *g, const double *r0, uint32_t iters, double c, pp_dtype dt, TO *r_out,
              double *r_l1, const Layout &L, cudaStream_t s) {
    const uint32_t N = 1u << g->scale;
    Args a;
    a.N = N;
    a.scale = g->scale;
    a.cmax = (uint32_t)((1ull << (32 - g->scale)) - 1);
    a.iters = iters;
    a.D = THREADS * ITEMS;
    a.colptr = g->colptr;
    a.rowc = g->rowc;
    a.ovf_key = g->ovf_key;
    a.ovf_cnt = g->ovf_cnt;
    a.info = g->info;
    a.coord = L.coord;
    a.carry = L.carry;
    a.acc = L.acc;
    a.fx_exp = L.fx_exp;
    a.ipart = L.ipart;
    a.ctl = L.ctl;
    a.tile_ctr = L.tile_ctr;
    a.c = c;
    const TA *inv = dt == PP_FP64 ? reinterpret_cast<const TA *>(g->inv_dout64)
                                  : reinterpret_cast<const TA *>(g->inv_dout32);
    if (!inv) return PP_ERR_INVALID_ARG;
    TS *x0 = static_cast<TS *>(L.x[0]);
    TS *x1 = static_cast<TS *>(L.x[1]);
    setup_kernel<<<SETUP_BLOCKS, 256, 0, s>>>(a, r0);
    normalize_kernel<TS, TA, TO><<<SETUP_BLOCKS, 256, 0, s>>>(a, r0, inv, x0, r_out);
    count_launch(2);

    static const int o_mid = occupancy(iterate_kernel<TS, TA, TO, false, ITEMS>);
    static const int o_last = occupancy(iterate_kernel<TS, TA, TO, true, ITEMS>);
    const int sms = sm_count();
    for (uint32_t it = 0; it < iters; ++it) {
        const TS *xin = (it & 1) ? x1 : x0;
        TS *xout = (it & 1) ? x0 : x1;
        if (it + 1 == iters)
            iterate_kernel<TS, TA, TO, true, ITEMS><<<sms * o_last, THREADS, 0, s>>>(a, inv, xin, xout, r_out, it);
        else
            iterate_kernel<TS, TA, TO, false, ITEMS><<<sms * o_mid, THREADS, 0, s>>>(a, inv, xin, xout, r_out, it);
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
            return k3::run<double, double, double, k3::ITEMS_F64>(g, r0, iters, c, dt, static_cast<double *>(r_out),
                                                                  r_l1, L, s);
        case PP_FP32:
            return k3::run<float, float, float, k3::ITEMS_F32>(g, r0, iters, c, dt, static_cast<float *>(r_out), r_l1,
                                                               L, s);
        default:
            return k3::run<__nv_bfloat16, float, float, k3::ITEMS_F32>(g, r0, iters, c, dt, static_cast<float *>(r_out),
                                                                       r_l1, L, s);
    }
}
