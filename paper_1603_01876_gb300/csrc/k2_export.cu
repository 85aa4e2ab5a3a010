// The filtered matrix A of Kernel 2 (Sec. IV-C step 4) exported in
// compressed-row form, in vertex order: row pointers, columns ascending
// within each row, counts, and the normalised values count / d_out(u) in
// binary64 and binary32.
//
// Kernel 2 keeps A as compressed columns in its storage order with the
// counts packed into the row words (the layout Kernel 3 reads).  The export
// lists every kept entry once as a 64-bit word (u << 32 | count field <<
// scale | v) with the columns taken in vertex order, so that a stable LSD
// radix sort on the bits of u (ceil(scale/8) passes of the Onesweep pass
// used by Kernels 1 and 2) leaves the entries ordered by (u, v); a last pass
// decodes them, resolves counts that did not fit their packed field through
// the overflow table, divides, and writes the row pointers from the row
// boundaries.
#include <algorithm>

#include "onesweep.cuh"

PP_DEFINE_ERROR_WORD(kx_fetch_error)

namespace pp {
namespace kx {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr int TOP_THREADS = 1024;

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

// Entries of each vertex's column (vertex order) into len[v]; per-tile sums.
__global__ void __launch_bounds__(SCAN_THREADS) col_len_kernel(const uint32_t *colptr, const uint32_t *perm,
                                                               uint32_t N, uint32_t *len, uint32_t *tile_sum) {
    __shared__ uint32_t sc[40];
    const uint64_t v0 = (uint64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        const uint64_t v = v0 + j;
        if (v < N) {
            const uint32_t p = pp_idx(__ldg(perm + v), N);
            const uint32_t l = __ldg(colptr + p + 1) - __ldg(colptr + p);
            len[v] = l;
            sum += l;
        }
    }
    uint32_t tot;
    block_exclusive_sum<uint32_t, SCAN_THREADS>(sum, sc, &tot);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

// Exclusive prefix sums of the tile sums (one block).
__global__ void __launch_bounds__(TOP_THREADS) tile_scan_kernel(uint32_t *tile_sum, uint32_t ntiles) {
    __shared__ uint32_t sc[40];
    uint32_t carry = 0;
    for (uint32_t base = 0; base < ntiles; base += TOP_THREADS) {
        const uint32_t t = base + threadIdx.x;
        const uint32_t x = t < ntiles ? tile_sum[t] : 0u;
        uint32_t tot;
        const uint32_t e = block_exclusive_sum<uint32_t, TOP_THREADS>(x, sc, &tot);
        if (t < ntiles) tile_sum[t] = carry + e;
        carry += tot;
    }
}

// Each vertex's first word: len[v] becomes the exclusive prefix sum over v.
__global__ void __launch_bounds__(SCAN_THREADS) col_off_kernel(uint32_t *len, uint32_t N, const uint32_t *tile_off) {
    __shared__ uint32_t sc[40];
    const uint64_t v0 = (uint64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    uint32_t l[SCAN_ITEMS], sum = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        l[j] = v0 + j < N ? len[v0 + j] : 0u;
        sum += l[j];
    }
    uint32_t tot;
    uint32_t run = tile_off[blockIdx.x] + block_exclusive_sum<uint32_t, SCAN_THREADS>(sum, sc, &tot);
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        if (v0 + j < N) len[v0 + j] = run;
        run += l[j];
    }
}

// One warp per vertex v: its column's entries as words (u << 32 | count
// field << scale | v), written from the vertex's first word on.
__global__ void __launch_bounds__(256) emit_kernel(const uint32_t *colptr, const uint32_t *rowc, const uint32_t *perm,
                                                   const uint32_t *iperm, uint32_t N, uint32_t scale,
                                                   const uint32_t *voff, const uint64_t *info, uint64_t *words) {
    const int lane = threadIdx.x & 31;
    const uint32_t umask = (1u << scale) - 1u;
    const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t v = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); v < N; v += nw) {
        const uint32_t p = pp_idx(__ldg(perm + v), N);
        const uint32_t s = __ldg(colptr + p);
        const uint64_t o = __ldg(voff + v);
        // rowc and words both hold nnz entries
        const uint32_t len = pp_len(o, pp_len(s, __ldg(colptr + p + 1) - s, info[PP_INFO_NNZ]), info[PP_INFO_NNZ]);
        for (uint32_t k = lane; k < len; k += 32) {
            const uint32_t w = __ldg(rowc + s + k);
            const uint32_t u = __ldg(iperm + (w & umask));
            words[o + k] = ((uint64_t)u << 32) | (w & ~umask) | (uint32_t)v;
        }
    }
}

struct WordSrc {
    const uint64_t *w;
    __device__ __forceinline__ bool load(uint64_t i, uint64_t &k, uint32_t &) const {
        k = w[i];
        return true;
    }
};
struct WordDst {
    uint64_t *w;
    __device__ __forceinline__ void store(uint64_t pos, uint64_t k, uint32_t) const { w[pos] = k; }
};

struct FinishArgs {
    const uint64_t *words;  // sorted by (u, v)
    const uint64_t *info;
    const uint64_t *ovf_key;
    const uint32_t *ovf_cnt;
    const uint32_t *d_out;
    uint32_t N, scale, cmax;
    uint64_t cap;
    uint64_t *rowptr;
    uint32_t *col, *cnt;
    double *val64;
    float *val32;
};

// Decode, divide, and write the row pointers at the row boundaries: entry i
// starts every row after the previous entry's row up to its own.
__global__ void __launch_bounds__(256) finish_kernel(FinishArgs a) {
    const uint64_t nnz = a.info[PP_INFO_NNZ], novf = a.info[PP_INFO_NOVF];
    const bool room = nnz <= a.cap;
    const uint32_t umask = (1u << a.scale) - 1u;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gtid == 0 && !room) pp_set_error(PP_DEV_CAPACITY);
    if (nnz == 0)
        for (uint64_t u = gtid; u <= a.N; u += stride) a.rowptr[u] = 0;
    for (uint64_t i = gtid; i < nnz; i += stride) {
        const uint64_t w = a.words[i];
        const uint32_t u = pp_idx((uint32_t)(w >> 32), a.N), lo = (uint32_t)w;
        const uint32_t v = lo & umask;
        if (room) {
            uint32_t c = lo >> a.scale;
            if (c == a.cmax) c = ovf_lookup(a.ovf_key, a.ovf_cnt, novf, ((uint64_t)u << 32) | v);
            const uint32_t d = __ldg(a.d_out + u);  // >= c >= 1: the row keeps this entry
            a.col[i] = v;
            a.cnt[i] = c;
            if (a.val64) a.val64[i] = (double)c / (double)d;
            if (a.val32) a.val32[i] = (float)c / (float)d;
        }
        const uint64_t prev = i == 0 ? 0 : (a.words[i - 1] >> 32) + 1;  // first row this entry starts
        for (uint64_t r = prev; r <= u; ++r) a.rowptr[r] = i;
        if (i + 1 == nnz)
            for (uint64_t r = (uint64_t)u + 1; r <= a.N; ++r) a.rowptr[r] = nnz;
    }
}

struct Layout {
    uint32_t *voff, *tile_sum;
    uint64_t *words[2];
    os::SortWs sort;
    size_t bytes;
};

inline int num_passes(uint32_t scale) { return (int)ceil_div(scale, 8u); }

inline Layout layout(void *ws, uint64_t M, uint32_t scale) {
    Carver c(ws);
    Layout L;
    const uint64_t N = 1ull << scale;
    const uint64_t cap = M ? M : 1;
    L.voff = c.take<uint32_t>(N);
    L.tile_sum = c.take<uint32_t>(ceil_div(N, SCAN_TILE));
    L.words[0] = c.take<uint64_t>(cap);
    L.words[1] = c.take<uint64_t>(cap);
    L.sort = os::carve_sort_ws(c, cap);
    L.bytes = c.size();
    return L;
}

}  // namespace kx
}  // namespace pp

using namespace pp;

extern "C" pp_status pp_export_csr_workspace(uint64_t M, uint32_t scale, size_t *bytes) {
    if (!bytes || scale < 1 || scale > 27 || M > (1ull << 31)) return PP_ERR_INVALID_ARG;
    *bytes = kx::layout(nullptr, M, scale).bytes;
    return PP_OK;
}

extern "C" pp_status pp_export_csr(const pp_graph *g, uint64_t *rowptr, uint32_t *col, uint32_t *cnt,
                                   double *val64, float *val32, uint64_t cap, void *ws, size_t ws_bytes,
                                   void *stream) {
    PP_ENTRY("pp_export_csr");
    if (!g || !rowptr || (cap > 0 && (!col || !cnt))) return PP_ERR_INVALID_ARG;
    if (g->scale < 1 || g->scale > 27 || g->M > (1ull << 31)) return PP_ERR_INVALID_ARG;
    if (!g->colptr || !g->rowc || !g->ovf_key || !g->ovf_cnt || !g->d_out || !g->info || !g->perm || !g->iperm)
        return PP_ERR_INVALID_ARG;
    const kx::Layout need = kx::layout(nullptr, g->M, g->scale);
    pp_status st = check_ws(ws, ws_bytes, need.bytes);
    if (st != PP_OK) return st;
    const kx::Layout L = kx::layout(ws, g->M, g->scale);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t N = 1u << g->scale;
    const uint32_t ntiles = (uint32_t)ceil_div(N, kx::SCAN_TILE);
    kx::col_len_kernel<<<ntiles, kx::SCAN_THREADS, 0, s>>>(g->colptr, g->perm, N, L.voff, L.tile_sum);
    kx::tile_scan_kernel<<<1, kx::TOP_THREADS, 0, s>>>(L.tile_sum, ntiles);
    kx::col_off_kernel<<<ntiles, kx::SCAN_THREADS, 0, s>>>(L.voff, N, L.tile_sum);
    const unsigned egrid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(ceil_div(N, 8), 64ull * sm_count()));
    kx::emit_kernel<<<egrid, 256, 0, s>>>(g->colptr, g->rowc, g->perm, g->iperm, N, g->scale, L.voff, g->info, L.words[0]);
    count_launch(4);
    // stable sort of the words by u (bits 32 .. 32 + scale), nnz of them
    const uint64_t *n_dev = g->info + PP_INFO_NNZ;
    const int P = kx::num_passes(g->scale);
    const size_t word = L.sort.wide ? 8 : 4;
    cudaMemsetAsync(L.sort.hist, 0, os::kCtlBytes, s);
    const unsigned hgrid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(ceil_div(g->M, 256 * 8), 8ull * sm_count()));
    os::hist_kernel<uint64_t, kx::WordSrc><<<hgrid, 256, 0, s>>>(
        kx::WordSrc{L.words[0]}, n_dev, g->M, P, L.sort.hist, static_cast<uint32_t *>(L.sort.status[0]),
        L.sort.ntiles_max * os::RADIX * word / 4, 32u);
    count_launch();
    for (int p = 0; p < P; ++p)
        os::launch_pass<uint64_t>(L.sort, p, P, kx::WordSrc{L.words[p & 1]}, kx::WordDst{L.words[(p + 1) & 1]},
                                  n_dev, g->M, s, 32u);
    kx::FinishArgs fa{L.words[P & 1], g->info, g->ovf_key, g->ovf_cnt, g->d_out, N, g->scale,
                      (uint32_t)((1ull << (32 - g->scale)) - 1), cap, rowptr, col, cnt, val64, val32};
    const unsigned fgrid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(ceil_div(g->M, 256), 16ull * sm_count()));
    kx::finish_kernel<<<fgrid, 256, 0, s>>>(fa);
    count_launch();
    return launch_status();
}
