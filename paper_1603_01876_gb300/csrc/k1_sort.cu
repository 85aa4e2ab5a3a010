// Kernel 1 (Sec. IV-B): sort the edge list by start vertex.
//
// Each edge becomes the key (u << scale | v) (32-bit when 2*scale <= 32,
// 64-bit otherwise); an LSD radix sort over its 2*scale bits, 8 bits per
// pass, orders the edges by u and, within equal u, by v.  The pack into keys
// happens while the first pass loads, and the unpack into (u_out, v_out) while
// the last pass stores, so the edge list is read and written once per pass.
#include <algorithm>

#include "onesweep.cuh"

PP_DEFINE_ERROR_WORD(k1_fetch_error)

namespace pp {
namespace k1 {

template <typename KeyT, bool CHECK>
struct PackSrc {
    const uint32_t *u, *v;
    uint32_t scale;
    bool vec;  // u and v are 16-byte aligned: four ids per load (see has_load4)
    __device__ __forceinline__ bool load(uint64_t i, KeyT &k, uint32_t &) const {
        const uint32_t a = __ldg(u + i), b = __ldg(v + i);
        if (CHECK && ((a | b) >> scale)) pp_set_error(PP_DEV_RANGE);
        k = ((KeyT)a << scale) | (KeyT)b;
        return true;
    }
    __device__ __forceinline__ void load4(uint64_t i4, KeyT *k) const {
        const uint4 a = __ldg(reinterpret_cast<const uint4 *>(u + i4));
        const uint4 b = __ldg(reinterpret_cast<const uint4 *>(v + i4));
        if (CHECK && ((a.x | a.y | a.z | a.w | b.x | b.y | b.z | b.w) >> scale)) pp_set_error(PP_DEV_RANGE);
        k[0] = ((KeyT)a.x << scale) | (KeyT)b.x;
        k[1] = ((KeyT)a.y << scale) | (KeyT)b.y;
        k[2] = ((KeyT)a.z << scale) | (KeyT)b.z;
        k[3] = ((KeyT)a.w << scale) | (KeyT)b.w;
    }
};

inline bool aligned16(const void *a, const void *b) { return (((uintptr_t)a | (uintptr_t)b) & 15u) == 0; }

template <typename KeyT>
struct KeySrc {
    const KeyT *keys;
    __device__ __forceinline__ bool load(uint64_t i, KeyT &k, uint32_t &) const {
        k = keys[i];
        return true;
    }
};

template <typename KeyT>
struct KeyDst {
    KeyT *keys;
    __device__ __forceinline__ void store(uint64_t pos, KeyT k, uint32_t) const { keys[pos] = k; }
};

template <typename KeyT>
struct UnpackDst {
    uint32_t *u, *v;
    uint32_t scale;
    __device__ __forceinline__ void store(uint64_t pos, KeyT k, uint32_t) const {
        u[pos] = (uint32_t)(k >> scale);
        v[pos] = (uint32_t)(k & (((KeyT)1 << scale) - 1));
    }
};

struct Layout {
    void *keys[2];
    os::SortWs sort;
    size_t bytes;
};

inline int num_passes(uint32_t scale) { return (int)ceil_div(2u * scale, 8u); }

inline Layout layout(void *ws, uint64_t M, uint32_t scale) {
    Carver c(ws);
    Layout L;
    const int P = num_passes(scale);
    const size_t kb = (2 * scale <= 32) ? 4 : 8;
    L.keys[0] = P >= 2 ? c.take<char>(M * kb) : nullptr;
    L.keys[1] = P >= 3 ? c.take<char>(M * kb) : nullptr;
    L.sort = os::carve_sort_ws(c, M);
    L.bytes = c.size();
    return L;
}

// keys_out == nullptr: the last pass unpacks into (u_out, v_out); otherwise it
// writes the sorted packed keys there (the chunked sort of the host-buffer
// pipeline merges them afterwards).
template <typename KeyT>
void run(const uint32_t *u, const uint32_t *v, uint64_t M, uint32_t scale, uint32_t *u_out,
         uint32_t *v_out, const Layout &L, cudaStream_t s, KeyT *keys_out = nullptr) {
    const int P = num_passes(scale);
    const size_t word = L.sort.wide ? 8 : 4;
    const uint64_t ntiles = ceil_div(M, os::TILE);
    cudaMemsetAsync(L.sort.hist, 0, os::kCtlBytes, s);
    const unsigned hgrid = (unsigned)std::min<uint64_t>(ceil_div(M, 256 * 8), (uint64_t)sm_count() * 8);
    const bool vec = aligned16(u, v);
    os::hist_kernel<KeyT, PackSrc<KeyT, true>><<<hgrid ? hgrid : 1, 256, 0, s>>>(
        PackSrc<KeyT, true>{u, v, scale, vec}, nullptr, M, P, L.sort.hist,
        static_cast<uint32_t *>(L.sort.status[0]), ntiles * os::RADIX * word / 4);
    count_launch();
    KeyT *A = static_cast<KeyT *>(L.keys[0]);
    KeyT *B = static_cast<KeyT *>(L.keys[1]);
    const PackSrc<KeyT, false> pack{u, v, scale, vec};
    const UnpackDst<KeyT> unpack{u_out, v_out, scale};
    if (P == 1) {
        if (keys_out)
            os::launch_pass<KeyT>(L.sort, 0, P, pack, KeyDst<KeyT>{keys_out}, nullptr, M, s);
        else
            os::launch_pass<KeyT>(L.sort, 0, P, pack, unpack, nullptr, M, s);
        return;
    }
    os::launch_pass<KeyT>(L.sort, 0, P, pack, KeyDst<KeyT>{A}, nullptr, M, s);
    for (int p = 1; p < P - 1; ++p) {
        KeyT *in = (p & 1) ? A : B;
        KeyT *out = (p & 1) ? B : A;
        os::launch_pass<KeyT>(L.sort, p, P, KeySrc<KeyT>{in}, KeyDst<KeyT>{out}, nullptr, M, s);
    }
    KeyT *last_in = ((P - 1) & 1) ? A : B;
    if (keys_out)
        os::launch_pass<KeyT>(L.sort, P - 1, P, KeySrc<KeyT>{last_in}, KeyDst<KeyT>{keys_out}, nullptr, M, s);
    else
        os::launch_pass<KeyT>(L.sort, P - 1, P, KeySrc<KeyT>{last_in}, unpack, nullptr, M, s);
}

}  // namespace k1

// ---------------------------------------------------------------------------
// Kernel 1 in chunks, for the host-buffer pipeline: each chunk of the edge
// list is sorted into packed 64-bit keys as soon as its copy has arrived
// (while the next chunk is still crossing the host link), and the sorted
// chunks are merged pairwise.  The merged keys are the keys the single sort
// produces (the order of equal keys cannot be told apart), so the output is
// the same.  A merge follows the merge-path scheme (Green, McColl & Bader,
// "GPU merge path", 2012): the output is cut into tiles, the split of each
// tile boundary between the two inputs is found by a binary search along
// the cross diagonal, and each tile is merged in shared memory.

namespace k1m {

constexpr int THREADS = 256;
constexpr int ITEMS = 16;
constexpr int TILE = THREADS * ITEMS;

// Elements of a among the first k of the merge of a and b (a first on ties).
__device__ __forceinline__ uint64_t corank(uint64_t k, const uint64_t *a, uint64_t na, const uint64_t *b,
                                           uint64_t nb) {
    uint64_t lo = k > nb ? k - nb : 0, hi = k < na ? k : na;
    while (lo < hi) {
        const uint64_t i = (lo + hi) >> 1;
        if (__ldg(a + i) <= __ldg(b + (k - 1 - i)))
            lo = i + 1;
        else
            hi = i;
    }
    return lo;
}

// split[t] = corank of output index min(t * TILE, na + nb), t = 0 .. tiles.
__global__ void __launch_bounds__(256) split_kernel(const uint64_t *a, uint64_t na, const uint64_t *b, uint64_t nb,
                                                    uint64_t tiles, uint64_t *split) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t > tiles) return;
    const uint64_t k = t * TILE < na + nb ? t * TILE : na + nb;
    split[t] = corank(k, a, na, b, nb);
}

struct KeyOut {
    uint64_t *k;
    __device__ __forceinline__ void store(uint64_t i, uint64_t key) const { k[i] = key; }
};
struct UnpackOut {
    uint32_t *u, *v;
    uint32_t scale;
    __device__ __forceinline__ void store(uint64_t i, uint64_t key) const {
        u[i] = (uint32_t)(key >> scale);
        v[i] = (uint32_t)(key & ((1ull << scale) - 1));
    }
};

template <class Out>
__global__ void __launch_bounds__(THREADS) merge_kernel(const uint64_t *a, uint64_t na, const uint64_t *b, uint64_t nb,
                                                        const uint64_t *split, Out out) {
    __shared__ uint64_t s[TILE];
    const uint64_t n = na + nb;
    const uint64_t k0 = (uint64_t)blockIdx.x * TILE, k1 = k0 + TILE < n ? k0 + TILE : n;
    const uint64_t a0 = split[blockIdx.x], a1 = split[blockIdx.x + 1];
    const uint64_t b0 = k0 - a0;
    // la + lb = k1 - k0 <= TILE
    const uint32_t la = (uint32_t)pp_len(0, a1 - a0, (uint64_t)TILE), total = (uint32_t)(k1 - k0);
    const uint32_t lb = total - la;
    for (uint32_t i = threadIdx.x; i < la; i += THREADS) s[i] = __ldg(a + a0 + i);
    for (uint32_t i = threadIdx.x; i < lb; i += THREADS) s[pp_idx(la + i, (uint32_t)TILE)] = __ldg(b + b0 + i);
    __syncthreads();
    // thread t merges outputs [t * ITEMS, (t + 1) * ITEMS) of the tile
    const uint32_t t0 = threadIdx.x * ITEMS;
    uint64_t val[ITEMS];
    if (t0 < total) {
        uint32_t lo = t0 > lb ? t0 - lb : 0, hi = t0 < la ? t0 : la;
        while (lo < hi) {
            const uint32_t i = (lo + hi) >> 1;
            if (s[i] <= s[la + (t0 - 1 - i)])
                lo = i + 1;
            else
                hi = i;
        }
        uint32_t i = lo, j = t0 - lo;
#pragma unroll
        for (int q = 0; q < ITEMS; ++q) {
            if (t0 + q < total) {
                const bool take_a = j >= lb || (i < la && s[i] <= s[la + j]);
                val[q] = take_a ? s[i++] : s[la + j++];
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < ITEMS; ++q)
        if (t0 + q < total) s[t0 + q] = val[q];
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < total; i += THREADS) out.store(k0 + i, s[i]);
}

template <class Out>
pp_status merge(const uint64_t *a, uint64_t na, const uint64_t *b, uint64_t nb, uint64_t *split, Out out,
                cudaStream_t s) {
    const uint64_t tiles = ceil_div(na + nb, TILE);
    if (!tiles) return PP_OK;
    split_kernel<<<(unsigned)ceil_div(tiles + 1, 256), 256, 0, s>>>(a, na, b, nb, tiles, split);
    merge_kernel<Out><<<(unsigned)tiles, THREADS, 0, s>>>(a, na, b, nb, split, out);
    count_launch(2);
    return launch_status();
}

}  // namespace k1m

size_t k1_chunk_workspace(uint64_t Mc, uint32_t scale) { return k1::layout(nullptr, Mc, scale).bytes; }

size_t k1_merge_split_words(uint64_t n) { return ceil_div(n, k1m::TILE) + 1; }

pp_status k1_sort_chunk_keys(const uint32_t *u, const uint32_t *v, uint64_t Mc, uint32_t scale, uint64_t *keys,
                             void *ws, size_t ws_bytes, cudaStream_t s) {
    if (2 * scale <= 32 || scale > 27) return PP_ERR_INVALID_ARG;  // 64-bit keys only
    if (Mc == 0) return PP_OK;
    const k1::Layout need = k1::layout(nullptr, Mc, scale);
    pp_status st = check_ws(ws, ws_bytes, need.bytes);
    if (st != PP_OK) return st;
    k1::run<uint64_t>(u, v, Mc, scale, nullptr, nullptr, k1::layout(ws, Mc, scale), s, keys);
    return launch_status();
}

pp_status k1_merge_keys(const uint64_t *a, uint64_t na, const uint64_t *b, uint64_t nb, uint64_t *out,
                        uint64_t *split, cudaStream_t s) {
    return k1m::merge(a, na, b, nb, split, k1m::KeyOut{out}, s);
}

pp_status k1_merge_unpack(const uint64_t *a, uint64_t na, const uint64_t *b, uint64_t nb, uint32_t scale,
                          uint32_t *u_out, uint32_t *v_out, uint64_t *split, cudaStream_t s) {
    return k1m::merge(a, na, b, nb, split, k1m::UnpackOut{u_out, v_out, scale}, s);
}

}  // namespace pp

using namespace pp;

static bool k1_args_ok(uint64_t M, uint32_t scale) {
    return scale >= 1 && scale <= 27 && M <= (1ull << 31);
}

extern "C" pp_status pp_sort_edges_workspace(uint64_t M, uint32_t scale, size_t *bytes) {
    if (!bytes || !k1_args_ok(M, scale)) return PP_ERR_INVALID_ARG;
    *bytes = k1::layout(nullptr, M, scale).bytes;
    return PP_OK;
}

extern "C" pp_status pp_sort_edges(const uint32_t *u, const uint32_t *v, uint64_t M, uint32_t scale,
                                   uint32_t *u_out, uint32_t *v_out, void *ws, size_t ws_bytes,
                                   void *stream) {
    PP_ENTRY("pp_sort_edges");
    if (!k1_args_ok(M, scale)) return PP_ERR_INVALID_ARG;
    if (M == 0) return PP_OK;
    if (!u || !v || !u_out || !v_out) return PP_ERR_INVALID_ARG;
    const k1::Layout need = k1::layout(nullptr, M, scale);
    pp_status st = check_ws(ws, ws_bytes, need.bytes);
    if (st != PP_OK) return st;
    const k1::Layout L = k1::layout(ws, M, scale);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (2 * scale <= 32)
        k1::run<uint32_t>(u, v, M, scale, u_out, v_out, L, s);
    else
        k1::run<uint64_t>(u, v, M, scale, u_out, v_out, L, s);
    return launch_status();
}

// ---------------------------------------------------------------------------
// Kernel 1 for a batch of graphs (pp_sort_edges_batched): one sort of every
// graph's edges at once.  Graph g's vertices get the ids base_g .. base_g +
// N_g - 1 of a union vertex space (base_g = N_0 + ... + N_(g-1)); its edges
// become the keys (U << S | V) of that union (S = ceil(log2(sum N_g))), one
// gather launch over all graphs writes them, the radix passes sort them
// together, and one unpack launch writes each graph's output.  The union ids
// of a graph form one range, so sorting by (U, V) leaves every graph's edges
// in its own segment, ordered by (u, v).  The batch table travels as a
// kernel parameter (no host-to-device copy), so the call can be captured in
// a CUDA graph.

namespace pp {
namespace k1b {

constexpr int MAX_G = PP_BATCH_MAX_GRAPHS;
constexpr int TILE = 4096;

struct Batch {
    uint32_t n, S;  // graphs, union scale
    const uint32_t *u[MAX_G], *v[MAX_G];
    uint32_t *uo[MAX_G], *vo[MAX_G];
    uint64_t eoff[MAX_G + 1];   // union index of graph g's first edge
    uint32_t vbase[MAX_G + 1];  // union id of graph g's vertex 0
    uint64_t toff[MAX_G + 1];   // first tile of graph g in the gather / unpack grids
    uint32_t scale[MAX_G];
};

// graph of tile t: the last g with toff[g] <= t (same for every thread of a block)
__device__ __forceinline__ uint32_t tile_graph(const Batch &b, uint64_t t) {
    uint32_t lo = 0, hi = b.n - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (b.toff[mid] <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <typename KeyT>
__global__ void __launch_bounds__(256) gather_kernel(Batch b, KeyT *keys) {
    const uint32_t g = tile_graph(b, blockIdx.x);
    const uint64_t e0 = (blockIdx.x - b.toff[g]) * (uint64_t)TILE, M = b.eoff[g + 1] - b.eoff[g];
    const uint32_t base = b.vbase[g], sc = b.scale[g];
    KeyT *out = keys + b.eoff[g];
    for (uint64_t i = e0 + threadIdx.x; i < min(M, e0 + TILE); i += blockDim.x) {
        uint32_t a = __ldg(b.u[g] + i), c = __ldg(b.v[g] + i);
        if ((a | c) >> sc) {
            pp_set_error(PP_DEV_RANGE);
            a &= (1u << sc) - 1u;
            c &= (1u << sc) - 1u;
        }
        out[i] = ((KeyT)(base + a) << b.S) | (KeyT)(base + c);
    }
}

template <typename KeyT>
__global__ void __launch_bounds__(256) unpack_kernel(Batch b, const KeyT *keys) {
    const uint32_t g = tile_graph(b, blockIdx.x);
    const uint64_t e0 = (blockIdx.x - b.toff[g]) * (uint64_t)TILE, M = b.eoff[g + 1] - b.eoff[g];
    const uint32_t base = b.vbase[g];
    const KeyT *in = keys + b.eoff[g];
    const KeyT mask = ((KeyT)1 << b.S) - 1;
    for (uint64_t i = e0 + threadIdx.x; i < min(M, e0 + TILE); i += blockDim.x) {
        const KeyT k = in[i];
        b.uo[g][i] = (uint32_t)(k >> b.S) - base;
        b.vo[g][i] = (uint32_t)(k & mask) - base;
    }
}

struct Layout {
    void *keys[2];
    os::SortWs sort;
    size_t bytes;
};

inline Layout layout(void *ws, uint64_t Mtot, uint32_t S) {
    Carver c(ws);
    Layout L;
    const size_t kb = (2 * S <= 32) ? 4 : 8;
    const uint64_t cap = Mtot ? Mtot : 1;
    L.keys[0] = c.take<char>(cap * kb);
    L.keys[1] = c.take<char>(cap * kb);
    L.sort = os::carve_sort_ws(c, cap);
    L.bytes = c.size();
    return L;
}

// Union scale and totals of a batch; false if it does not fit the limits.
inline bool batch_shape(uint32_t n, const uint64_t *M, const uint32_t *scale, uint64_t *Mtot, uint32_t *S) {
    if (n < 1 || n > (uint32_t)MAX_G || !M || !scale) return false;
    uint64_t nv = 0, me = 0;
    for (uint32_t g = 0; g < n; ++g) {
        if (scale[g] < 1 || scale[g] > 27) return false;
        nv += 1ull << scale[g];
        me += M[g];
    }
    if (nv > (1ull << 27) || me > (1ull << 31)) return false;
    uint32_t s = 1;
    while ((1ull << s) < nv) ++s;
    *Mtot = me;
    *S = s;
    return true;
}

template <typename KeyT>
void run(const Batch &b, uint64_t Mtot, uint64_t ntiles_g, const Layout &L, cudaStream_t s) {
    const int P = (int)ceil_div(2u * b.S, 8u);
    const size_t word = L.sort.wide ? 8 : 4;
    KeyT *A = static_cast<KeyT *>(L.keys[0]), *B = static_cast<KeyT *>(L.keys[1]);
    gather_kernel<KeyT><<<(unsigned)ntiles_g, 256, 0, s>>>(b, A);
    cudaMemsetAsync(L.sort.hist, 0, os::kCtlBytes, s);
    const unsigned hgrid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(ceil_div(Mtot, 256 * 8), (uint64_t)sm_count() * 8));
    os::hist_kernel<KeyT, k1::KeySrc<KeyT>><<<hgrid, 256, 0, s>>>(
        k1::KeySrc<KeyT>{A}, nullptr, Mtot, P, L.sort.hist, static_cast<uint32_t *>(L.sort.status[0]),
        ceil_div(Mtot, os::TILE) * os::RADIX * word / 4);
    count_launch(2);
    for (int p = 0; p < P; ++p) {
        KeyT *in = (p & 1) ? B : A;
        KeyT *out = (p & 1) ? A : B;
        os::launch_pass<KeyT>(L.sort, p, P, k1::KeySrc<KeyT>{in}, k1::KeyDst<KeyT>{out}, nullptr, Mtot, s);
    }
    unpack_kernel<KeyT><<<(unsigned)ntiles_g, 256, 0, s>>>(b, (P & 1) ? B : A);
    count_launch();
}

}  // namespace k1b
}  // namespace pp

extern "C" pp_status pp_sort_edges_batched_workspace(uint32_t n_graphs, const uint64_t *M, const uint32_t *scale,
                                                     size_t *bytes) {
    uint64_t Mtot;
    uint32_t S;
    if (!bytes || !k1b::batch_shape(n_graphs, M, scale, &Mtot, &S)) return PP_ERR_INVALID_ARG;
    *bytes = k1b::layout(nullptr, Mtot, S).bytes;
    return PP_OK;
}

extern "C" pp_status pp_sort_edges_batched(uint32_t n_graphs, const uint32_t *const *u, const uint32_t *const *v,
                                           const uint64_t *M, const uint32_t *scale, uint32_t *const *u_out,
                                           uint32_t *const *v_out, void *ws, size_t ws_bytes, void *stream) {
    PP_ENTRY("pp_sort_edges_batched");
    uint64_t Mtot;
    uint32_t S;
    if (!k1b::batch_shape(n_graphs, M, scale, &Mtot, &S) || !u || !v || !u_out || !v_out) return PP_ERR_INVALID_ARG;
    k1b::Batch b;
    b.n = n_graphs;
    b.S = S;
    uint64_t eo = 0, to = 0;
    uint32_t vb = 0;
    for (uint32_t g = 0; g < n_graphs; ++g) {
        if (M[g] && (!u[g] || !v[g] || !u_out[g] || !v_out[g])) return PP_ERR_INVALID_ARG;
        b.u[g] = u[g];
        b.v[g] = v[g];
        b.uo[g] = u_out[g];
        b.vo[g] = v_out[g];
        b.scale[g] = scale[g];
        b.eoff[g] = eo;
        b.vbase[g] = vb;
        b.toff[g] = to;
        eo += M[g];
        vb += 1u << scale[g];
        to += ceil_div(M[g], k1b::TILE);
    }
    b.eoff[n_graphs] = eo;
    b.vbase[n_graphs] = vb;
    b.toff[n_graphs] = to;
    if (Mtot == 0) return PP_OK;
    const k1b::Layout need = k1b::layout(nullptr, Mtot, S);
    pp_status st = check_ws(ws, ws_bytes, need.bytes);
    if (st != PP_OK) return st;
    const k1b::Layout L = k1b::layout(ws, Mtot, S);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (2 * S <= 32)
        k1b::run<uint32_t>(b, Mtot, to, L, s);
    else
        k1b::run<uint64_t>(b, Mtot, to, L, s);
    return launch_status();
}

// ---------------------------------------------------------------------------
// Kernel 1 without allocation (pp_sort_edges_static).  Some callers cannot
// allocate device memory at all: their GPU memory belongs to another
// allocator (a framework's caching pool, a fixed real-time budget) or
// cudaMalloc's implicit device synchronisation would stall their other
// streams.  For them this entry point keeps its scratch space in a
// fixed-size array in device memory, which every GPU that loads the library
// holds until the process exits.  Its device address is looked up
// (cudaGetSymbolAddress) on the first call made in each CUDA context, i.e.
// once per device, and again after cudaDeviceReset or any other replacement
// of the device's context (the module is then loaded anew and the array may
// sit elsewhere); make those first calls outside any stream capture.  The
// cache is keyed by the driver's context id, which is never reused within a
// process.  All calls share
// the array and it keeps the last call's contents: the sort clears its
// counters and look-back words itself, and calls whose work overlaps on the
// GPU (concurrent streams, several host threads) race on it.

#include <cuda.h>

#include <mutex>

namespace {
constexpr uint64_t kStaticMaxEdges = PP_SORT_STATIC_MAX_EDGES;
// Largest layout the sort needs for kStaticMaxEdges edges: two 64-bit key
// buffers, the digit histograms and two sets of 32-bit look-back words.
constexpr size_t kStaticBytes = (size_t)17 << 20;
static __device__ __align__(256) unsigned char k1_static_scratch[kStaticBytes];

// The driver's cuCtxGetCurrent and cuCtxGetId, fetched through the runtime
// so that the library does not link libcuda itself.
typedef CUresult (*ctx_current_fn)(CUcontext *);
typedef CUresult (*ctx_id_fn)(CUcontext, unsigned long long *);

struct StaticAddr {
    unsigned long long ctx_id;  // context the address was looked up in (0 = none yet)
    void *addr;
};

std::mutex g_static_mutex;
StaticAddr g_static_addr[kMaxDevices] = {};
ctx_current_fn g_ctx_current = nullptr;
ctx_id_fn g_ctx_id = nullptr;

// Id of the calling thread's current context, 0 if there is none.
bool current_ctx_id(unsigned long long *id) {
    *id = 0;
    if (!g_ctx_current || !g_ctx_id) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return false;
        g_ctx_current = reinterpret_cast<ctx_current_fn>(f1);
        g_ctx_id = reinterpret_cast<ctx_id_fn>(f2);
    }
    CUcontext ctx = nullptr;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS) return false;
    if (ctx && g_ctx_id(ctx, id) != CUDA_SUCCESS) return false;
    return true;
}

// Device address of the scratch array in the current context.
pp_status static_scratch(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    unsigned long long id = 0;
    if (!current_ctx_id(&id)) return PP_ERR_CUDA;
    StaticAddr &c = g_static_addr[dev];
    if (id == 0 || c.ctx_id != id || !c.addr) {
        void *p = nullptr;
        // creates the device's primary context if the thread has none yet
        if (cudaGetSymbolAddress(&p, k1_static_scratch) != cudaSuccess || !p) return PP_ERR_CUDA;
        if (!current_ctx_id(&id)) return PP_ERR_CUDA;
        c.ctx_id = id;  // an id of 0 is never reused: the next call looks the address up again
        c.addr = p;
    }
    *out = c.addr;
    return PP_OK;
}
}  // namespace

extern "C" pp_status pp_sort_edges_static(const uint32_t *u, const uint32_t *v, uint64_t M, uint32_t scale,
                                          uint32_t *u_out, uint32_t *v_out, void *stream) {
    PP_ENTRY("pp_sort_edges_static");
    if (!k1_args_ok(M, scale) || M > kStaticMaxEdges) return PP_ERR_INVALID_ARG;
    if (M == 0) return PP_OK;
    if (!u || !v || !u_out || !v_out) return PP_ERR_INVALID_ARG;
    const k1::Layout need = k1::layout(nullptr, M, scale);
    if (need.bytes > kStaticBytes) return PP_ERR_INVALID_ARG;
    void *base = nullptr;
    const pp_status sa = static_scratch(&base);
    if (sa != PP_OK) return sa;
    const k1::Layout L = k1::layout(base, M, scale);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (2 * scale <= 32)
        k1::run<uint32_t>(u, v, M, scale, u_out, v_out, L, s);
    else
        k1::run<uint64_t>(u, v, M, scale, u_out, v_out, L, s);
    return launch_status();
}

// ---------------------------------------------------------------------------
// Self-test of the bounded look-back wait (no counterpart in the paper).  A
// two-tile scatter pass starts with its tile counter at 1, so tile 0 is never
// processed and tile 1 waits for a status word that nothing writes.  After
// spin_limit empty polls the wait gives up, PP_DEV_TIMEOUT lands in the
// device error word, and the kernel finishes (its output is meaningless).

namespace {
__global__ void k1_set_u32(uint32_t *p, uint32_t v) { *p = v; }
constexpr uint64_t kSelftestEdges = 2 * os::TILE;
constexpr uint32_t kSelftestScale = 8;

struct SelftestLayout {
    uint32_t *u, *v;
    k1::Layout k1;
    size_t bytes;
};

SelftestLayout selftest_layout(void *ws) {
    Carver c(ws);
    SelftestLayout L;
    L.u = c.take<uint32_t>(kSelftestEdges);
    L.v = c.take<uint32_t>(kSelftestEdges);
    const size_t head = c.size();
    L.k1 = k1::layout(ws ? static_cast<char *>(ws) + head : nullptr, kSelftestEdges, kSelftestScale);
    L.bytes = head + L.k1.bytes;
    return L;
}
}  // namespace

extern "C" pp_status pp_selftest_lookback_timeout(uint32_t spin_limit, void *ws, size_t ws_bytes,
                                                  size_t *bytes_needed, void *stream) {
    PP_ENTRY("pp_selftest_lookback_timeout");
    const size_t need = selftest_layout(nullptr).bytes;
    if (bytes_needed) *bytes_needed = need;
    if (!ws) return bytes_needed ? PP_OK : PP_ERR_INVALID_ARG;
    if (spin_limit == 0) return PP_ERR_INVALID_ARG;
    pp_status st = check_ws(ws, ws_bytes, need);
    if (st != PP_OK) return st;
    const SelftestLayout L = selftest_layout(ws);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t M = kSelftestEdges;
    const uint32_t scale = kSelftestScale;
    const int P = k1::num_passes(scale);
    const size_t word = L.k1.sort.wide ? 8 : 4;
    cudaMemsetAsync(L.u, 0, M * sizeof(uint32_t), s);
    cudaMemsetAsync(L.v, 0, M * sizeof(uint32_t), s);
    cudaMemsetAsync(L.k1.sort.hist, 0, os::kCtlBytes, s);
    os::hist_kernel<uint32_t, k1::PackSrc<uint32_t, true>><<<2, 256, 0, s>>>(
        k1::PackSrc<uint32_t, true>{L.u, L.v, scale}, nullptr, M, P, L.k1.sort.hist,
        static_cast<uint32_t *>(L.k1.sort.status[0]), ceil_div(M, os::TILE) * os::RADIX * word / 4);
    k1_set_u32<<<1, 1, 0, s>>>(L.k1.sort.tile_ctr, 1u);
    count_launch(2);
    os::launch_pass<uint32_t>(L.k1.sort, 0, P, k1::PackSrc<uint32_t, false>{L.u, L.v, scale},
                                     k1::KeyDst<uint32_t>{static_cast<uint32_t *>(L.k1.keys[0])}, nullptr, M, s, 0,
                                     spin_limit);
    return launch_status();
}
