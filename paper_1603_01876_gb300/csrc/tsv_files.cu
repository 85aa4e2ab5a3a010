// The benchmark's edge files (Sec. IV-A and IV-B): one edge per line, the
// start and end vertex in decimal separated by a tab, "u\tv\n".  Kernel 0
// writes them, Kernel 1 reads them, sorts and writes them again, Kernel 2
// reads them.  Here the text is formatted and parsed on the GPU; moving the
// text between host memory (or storage) and the device is the caller's.
//
// Formatting: each line's length is known from its digits, so a tile of
// edges gets its output offset from a decoupled look-back over the earlier
// tiles' byte counts, builds its text in shared memory and copies it out
// contiguously.  Parsing: each thread reads 32 bytes, a look-back over the
// tiles' newline counts numbers the lines, and every line is parsed by the
// thread holding its newline (a line never exceeds PP_TSV_MAX_LINE bytes, so
// its start is at most that far back).  Malformed text sets PP_DEV_PARSE
// and the offending line is stored as (0, 0); every access stays in bounds.
#include "pp_common.cuh"

PP_DEFINE_ERROR_WORD(tsv_fetch_error)

namespace pp {
namespace tsv {

constexpr int THREADS = 256;
constexpr int FMT_ITEMS = 4;  // edges per thread
constexpr int FMT_TILE = THREADS * FMT_ITEMS;
constexpr int MAX_LINE = PP_TSV_MAX_LINE;
constexpr int PARSE_BYTES = 32;  // bytes per thread
constexpr int PARSE_TILE = THREADS * PARSE_BYTES;
constexpr uint64_t F_AGG = 1ull << 62, F_INC = 2ull << 62;

__device__ __forceinline__ int ndigits(uint32_t x) {
    int n = 1;
    while (x >= 10u) {
        x /= 10u;
        ++n;
    }
    return n;
}

__device__ __forceinline__ void put_decimal(char *p, uint32_t x, int n) {
    for (int i = n - 1; i >= 0; --i) {
        p[i] = (char)('0' + x % 10u);
        x /= 10u;
    }
}

// One warp: publishes the tile's total, looks back, publishes the inclusive
// prefix; returns the tile's exclusive prefix (all lanes).
__device__ __forceinline__ uint64_t tile_prefix(uint64_t *status, uint64_t tile, uint64_t total) {
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) st_relaxed_u64(status, F_INC | total);
        return 0;
    }
    if (lane == 0) st_relaxed_u64(status + tile, F_AGG | total);
    const uint64_t ex = warp_lookback(status, tile);
    if (lane == 0) st_relaxed_u64(status + tile, F_INC | (ex + total));
    return ex;
}

struct FormatArgs {
    const uint32_t *u, *v;
    uint64_t M;
    char *text;
    uint64_t *text_len;
    uint64_t *status;
    uint32_t *tile_ctr;
};

__global__ void __launch_bounds__(THREADS) format_kernel(FormatArgs a) {
    __shared__ char s_text[FMT_TILE * MAX_LINE];
    __shared__ uint64_t s_scan[40];
    __shared__ uint64_t s_excl;
    __shared__ uint32_t s_tile;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(a.tile_ctr, 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    const uint64_t ntiles = (a.M + FMT_TILE - 1) / FMT_TILE;
    if (tile >= ntiles) return;
    const uint64_t e0 = tile * FMT_TILE + (uint64_t)tid * FMT_ITEMS;
    uint32_t us[FMT_ITEMS], vs[FMT_ITEMS];
    int du[FMT_ITEMS], dv[FMT_ITEMS];
    uint64_t mine = 0;
#pragma unroll
    for (int j = 0; j < FMT_ITEMS; ++j) {
        const bool ok = e0 + j < a.M;
        us[j] = ok ? a.u[e0 + j] : 0u;
        vs[j] = ok ? a.v[e0 + j] : 0u;
        du[j] = ok ? ndigits(us[j]) : 0;
        dv[j] = ok ? ndigits(vs[j]) : 0;
        mine += ok ? (uint64_t)(du[j] + dv[j] + 2) : 0u;
    }
    uint64_t total;
    const uint64_t ex = block_exclusive_sum<uint64_t, THREADS>(mine, s_scan, &total);
    if (tid < 32) {
        const uint64_t e = tile_prefix(a.status, tile, total);
        if (tid == 0) s_excl = e;
    }
    uint32_t at = (uint32_t)ex;  // < FMT_TILE * MAX_LINE
#pragma unroll
    for (int j = 0; j < FMT_ITEMS; ++j) {
        if (e0 + j >= a.M) break;
        put_decimal(s_text + at, us[j], du[j]);
        at += du[j];
        s_text[at++] = '\t';
        put_decimal(s_text + at, vs[j], dv[j]);
        at += dv[j];
        s_text[at++] = '\n';
    }
    __syncthreads();
    const uint64_t base = s_excl;
    char *dst = a.text + base;
    for (uint32_t i = tid; i < (uint32_t)total; i += THREADS) dst[i] = s_text[i];
    if (tid == 0 && tile == ntiles - 1) *a.text_len = base + total;
}

struct ParseArgs {
    const char *text;
    uint64_t len;
    int vec;  // text is 16-byte aligned
    uint32_t *u, *v;
    uint64_t m_cap;
    uint64_t *m_out;
    uint64_t *status;
    uint32_t *tile_ctr;
};

// Parses text[s, q) as "digits\tdigits" (q is the newline); false if malformed.
__device__ __forceinline__ bool parse_line(const char *text, uint64_t s, uint64_t q, uint32_t &a, uint32_t &b) {
    uint64_t x = 0, y = 0;
    int nx = 0, ny = 0, tabs = 0;
    for (uint64_t i = s; i < q; ++i) {
        const char ch = __ldg(text + i);
        if (ch == '\t') {
            if (++tabs > 1) return false;
        } else if (ch >= '0' && ch <= '9') {
            if (tabs == 0) {
                x = x * 10u + (uint64_t)(ch - '0');
                ++nx;
            } else {
                y = y * 10u + (uint64_t)(ch - '0');
                ++ny;
            }
        } else {
            return false;
        }
    }
    if (tabs != 1 || nx == 0 || ny == 0 || nx > 10 || ny > 10 || x > 0xffffffffull || y > 0xffffffffull) return false;
    a = (uint32_t)x;
    b = (uint32_t)y;
    return true;
}

__global__ void __launch_bounds__(THREADS) parse_kernel(ParseArgs a) {
    __shared__ uint64_t s_scan[40];
    __shared__ uint64_t s_excl;
    __shared__ uint32_t s_tile;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(a.tile_ctr, 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    const uint64_t ntiles = (a.len + PARSE_TILE - 1) / PARSE_TILE;
    if (tile >= ntiles) return;
    const uint64_t c0 = tile * PARSE_TILE + (uint64_t)tid * PARSE_BYTES;
    // this thread's bytes; newlines marked in a bit mask
    char b[PARSE_BYTES];
    if (a.vec && c0 + PARSE_BYTES <= a.len) {
        const uint4 *p = reinterpret_cast<const uint4 *>(a.text + c0);
#pragma unroll
        for (int q = 0; q < PARSE_BYTES / 16; ++q) {
            const uint4 w = __ldg(p + q);
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int k = 0; k < 16; ++k) b[16 * q + k] = (char)(ws[k >> 2] >> (8 * (k & 3)));
        }
    } else {
#pragma unroll
        for (int k = 0; k < PARSE_BYTES; ++k) b[k] = c0 + k < a.len ? __ldg(a.text + c0 + k) : '\0';
    }
    uint32_t nl = 0;
#pragma unroll
    for (int k = 0; k < PARSE_BYTES; ++k)
        if (b[k] == '\n') nl |= 1u << k;
    uint64_t total;
    const uint64_t ex = block_exclusive_sum<uint64_t, THREADS>((uint64_t)__popc(nl), s_scan, &total);
    if (tid < 32) {
        const uint64_t e = tile_prefix(a.status, tile, total);
        if (tid == 0) s_excl = e;
    }
    __syncthreads();
    uint64_t line = s_excl + ex;
    if (tid == 0 && tile == ntiles - 1) {
        *a.m_out = s_excl + total;
        if (a.len && a.text[a.len - 1] != '\n') pp_set_error(PP_DEV_PARSE);  // a last line without newline
        if (s_excl + total > a.m_cap) pp_set_error(PP_DEV_PARSE);
    }
    int prev = -1;  // last newline seen in this chunk
    while (nl) {
        const int k = __ffs(nl) - 1;
        nl &= nl - 1;
        const uint64_t q = c0 + (uint64_t)k;
        uint64_t s = c0 + (uint64_t)(prev + 1);
        bool ok = true;
        if (prev < 0) {
            // the line began before this chunk: walk back to the previous newline
            s = c0;
            int steps = 0;
            while (s > 0 && __ldg(a.text + s - 1) != '\n') {
                --s;
                if (++steps > MAX_LINE) {
                    ok = false;
                    break;
                }
            }
        }
        prev = k;
        uint32_t x = 0, y = 0;
        if (!ok || q - s + 1 > (uint64_t)MAX_LINE || !parse_line(a.text, s, q, x, y)) {
            pp_set_error(PP_DEV_PARSE);
            x = y = 0;
        }
        if (line < a.m_cap) {
            a.u[line] = x;
            a.v[line] = y;
        }
        ++line;
    }
}

inline uint64_t format_tiles(uint64_t M) { return ceil_div(M ? M : 1, FMT_TILE); }
inline uint64_t parse_tiles(uint64_t L) { return ceil_div(L ? L : 1, PARSE_TILE); }

// Workspace: the look-back words and one tile counter.
inline size_t ws_bytes(uint64_t tiles) { return (size_t)(tiles * 8 + 256); }

}  // namespace tsv
}  // namespace pp

using namespace pp;

extern "C" pp_status pp_format_tsv_workspace(uint64_t M, size_t *bytes) {
    if (!bytes || M > (1ull << 31)) return PP_ERR_INVALID_ARG;
    *bytes = tsv::ws_bytes(tsv::format_tiles(M));
    return PP_OK;
}

extern "C" pp_status pp_format_tsv(const uint32_t *u, const uint32_t *v, uint64_t M, char *text, uint64_t text_cap,
                                   uint64_t *text_len, void *ws, size_t ws_bytes, void *stream) {
    if (M > (1ull << 31) || !text_len || (M && (!u || !v || !text))) return PP_ERR_INVALID_ARG;
    if (text_cap < M * (uint64_t)PP_TSV_MAX_LINE) return PP_ERR_INVALID_ARG;
    const uint64_t tiles = tsv::format_tiles(M);
    pp_status st = check_ws(ws, ws_bytes, tsv::ws_bytes(tiles));
    if (st != PP_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t *status = static_cast<uint64_t *>(ws);
    uint32_t *ctr = reinterpret_cast<uint32_t *>(status + tiles);
    cudaMemsetAsync(ws, 0, tsv::ws_bytes(tiles), s);
    cudaMemsetAsync(text_len, 0, sizeof(uint64_t), s);
    if (M) {
        tsv::format_kernel<<<(unsigned)tiles, tsv::THREADS, 0, s>>>(tsv::FormatArgs{u, v, M, text, text_len, status, ctr});
        count_launch();
    }
    return launch_status();
}

extern "C" pp_status pp_parse_tsv_workspace(uint64_t text_len, size_t *bytes) {
    if (!bytes || text_len > (1ull << 31) * (uint64_t)PP_TSV_MAX_LINE) return PP_ERR_INVALID_ARG;
    *bytes = tsv::ws_bytes(tsv::parse_tiles(text_len));
    return PP_OK;
}

extern "C" pp_status pp_parse_tsv(const char *text, uint64_t text_len, uint32_t *u, uint32_t *v, uint64_t m_cap,
                                  uint64_t *m_out, void *ws, size_t ws_bytes, void *stream) {
    if (text_len > (1ull << 31) * (uint64_t)PP_TSV_MAX_LINE || !m_out || (text_len && !text) ||
        (m_cap && (!u || !v)))
        return PP_ERR_INVALID_ARG;
    const uint64_t tiles = tsv::parse_tiles(text_len);
    pp_status st = check_ws(ws, ws_bytes, tsv::ws_bytes(tiles));
    if (st != PP_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t *status = static_cast<uint64_t *>(ws);
    uint32_t *ctr = reinterpret_cast<uint32_t *>(status + tiles);
    cudaMemsetAsync(ws, 0, tsv::ws_bytes(tiles), s);
    cudaMemsetAsync(m_out, 0, sizeof(uint64_t), s);
    if (text_len) {
        const int vec = (reinterpret_cast<uintptr_t>(text) & 15u) == 0;
        tsv::parse_kernel<<<(unsigned)tiles, tsv::THREADS, 0, s>>>(
            tsv::ParseArgs{text, text_len, vec, u, v, m_cap, m_out, status, ctr});
        count_launch();
    }
    return launch_status();
}
