// The benchmark's edge files (Sec. IV-A and IV-B): one edge per line, the
// start and end vertex in decimal separated by a tab, "u\tv\n".  Kernel 0
// writes them, Kernel 1 reads them, sorts and writes them again, Kernel 2
// reads them.  Here the text is formatted and parsed on the GPU; moving the
// text between host memory (or storage) and the device is the caller's.
//
// Both directions run in three launches with no waits between blocks: a
// streaming pass counts each tile's output (bytes of text, or lines), one
// block scans the counts into tile offsets, and the main pass processes
// every tile at its offset.
// Formatting: each line's length is known from its digits; a tile of edges
// builds its text in shared memory and copies it out with aligned 16-byte
// stores.  Parsing: a tile of text (and the bytes just before it) is
// loaded into shared memory and every line is parsed there by the thread
// holding its newline (a line never exceeds PP_TSV_MAX_LINE bytes, so its
// start is at most that far back); the tile's (u, v) are staged and written
// out coalesced.  Malformed text sets PP_DEV_PARSE and the offending line is
// stored as (0, 0); every access stays in bounds.
#include "pp_common.cuh"

PP_DEFINE_ERROR_WORD(tsv_fetch_error)

namespace pp {
namespace tsv {

constexpr int THREADS = 256;
constexpr int FMT_ITEMS = 4;  // edges per thread
constexpr int FMT_TILE = THREADS * FMT_ITEMS;
constexpr int MAX_LINE = PP_TSV_MAX_LINE;
constexpr int SCAN_THREADS = 1024;
constexpr int PARSE_BYTES = 32;  // bytes per thread
constexpr int PARSE_TILE = THREADS * PARSE_BYTES;
constexpr int HALO = 32;  // bytes kept before a parse tile: >= MAX_LINE, a multiple of 16
constexpr int STAGE_LINES = PARSE_TILE / 4;  // a well-formed line has at least 4 bytes
static_assert(HALO >= MAX_LINE && HALO % 16 == 0, "the halo holds a line's start");
static_assert(PARSE_BYTES == 32 && HALO == 32, "a thread's newlines fit one mask word; the halo is one chunk");
constexpr int TAIL = 48;  // zero bytes after a parse tile: line windows may read past its end

__device__ __forceinline__ int ndigits(uint32_t x) {
    return 1 + (x >= 10u) + (x >= 100u) + (x >= 1000u) + (x >= 10000u) + (x >= 100000u) + (x >= 1000000u) +
           (x >= 10000000u) + (x >= 100000000u) + (x >= 1000000000u);
}

// Byte classes of a little-endian word, exact per byte: bit 7 of each byte
// of the result is set where the class holds.
__device__ __forceinline__ uint32_t bytes_equal(uint32_t w, uint32_t pattern) {
    const uint32_t x = w ^ pattern;  // zero where equal
    return ~(((x & 0x7f7f7f7fu) + 0x7f7f7f7fu) | x) & 0x80808080u;
}
__device__ __forceinline__ uint32_t bytes_nondigit(uint32_t w) {
    const uint32_t x = w ^ 0x30303030u;  // '0'..'9' become 0..9
    return (((x & 0x7f7f7f7fu) + 0x76767676u) | x) & 0x80808080u;
}
// The four flag bits (bit 7 of each byte) as a nibble, byte 0 lowest.
__device__ __forceinline__ uint32_t nibble(uint32_t flags) { return (flags * 0x00204081u) >> 28; }

// The value of 8 ASCII digits, the first (most significant) in the lowest
// byte: adjacent digits, then pairs, then quads combined by multiplication
// (the SWAR method of Lemire and Langdale's simdjson, "parse eight digits").
__device__ __forceinline__ uint32_t eight_digits(uint64_t w) {
    w -= 0x3030303030303030ull;
    w = w * 10u + (w >> 8);
    w = ((w & 0x000000ff000000ffull) * (100ull + (1000000ull << 32)) +
         ((w >> 16) & 0x000000ff000000ffull) * (1ull + (10000ull << 32))) >> 32;
    return (uint32_t)w;
}

// The decimal digits of x < 10^8 as 8 ASCII bytes with leading zeros, the
// most significant in the lowest byte: the quotients by 10^4, 10^2 and 10
// are taken in parallel in the lanes of one 64-bit word, each by a
// multiply-shift reciprocal that is exact for the lane's range.
__device__ __forceinline__ uint64_t eight_ascii(uint32_t x) {
    const uint32_t hi = x / 10000u, lo = x - hi * 10000u;
    uint64_t v = hi | ((uint64_t)lo << 32);                 // two 4-digit lanes
    const uint64_t q = ((v * 5243u) >> 19) & 0x0000007f0000007full;
    v = q | ((v - q * 100u) << 16);                          // four 2-digit lanes
    const uint64_t t = ((v * 103u) >> 10) & 0x000f000f000f000full;
    v = t | ((v - t * 10u) << 8);                            // eight digits
    return v + 0x3030303030303030ull;
}

// Writes the n-digit decimal x (n = ndigits(x)) at p.
__device__ __forceinline__ void put_decimal(char *p, uint32_t x, int n) {
    int nlo = n;
    if (n > 8) {
        const uint32_t hi = x / 100000000u;  // one or two digits
        x -= hi * 100000000u;
        if (n == 10) *p++ = (char)('0' + hi / 10u);
        *p++ = (char)('0' + hi % 10u);
        nlo = 8;
    }
    const uint64_t d = eight_ascii(x) >> (8 * (8 - nlo));
#pragma unroll
    for (int i = 0; i < 8; ++i)
        if (i < nlo) p[i] = (char)(d >> (8 * i));
}

// Exclusive scan of c[0, n) in place, c[n] = the total, also stored in
// *total_out (one block; each thread takes a contiguous run of counts).
__global__ void __launch_bounds__(SCAN_THREADS) scan_kernel(uint64_t *c, uint64_t n, uint64_t *total_out) {
    __shared__ uint64_t s_scan[40];
    const uint64_t per = (n + SCAN_THREADS - 1) / SCAN_THREADS;
    const uint64_t lo = min(n, (uint64_t)threadIdx.x * per), hi = min(n, lo + per);
    uint64_t sum = 0;
    for (uint64_t i = lo; i < hi; ++i) sum += c[i];
    uint64_t total;
    uint64_t run = block_exclusive_sum<uint64_t, SCAN_THREADS>(sum, s_scan, &total);
    for (uint64_t i = lo; i < hi; ++i) {
        const uint64_t t = c[i];
        c[i] = run;
        run += t;
    }
    if (threadIdx.x == 0) {
        c[n] = total;
        *total_out = total;
    }
}

struct FormatArgs {
    const uint32_t *u, *v;
    uint64_t M;
    int vec;  // u and v are 16-byte aligned
    char *text;
    uint64_t *offs;  // [tiles + 1] bytes of text before each tile (after the scan)
};

// This thread's edges (FMT_ITEMS from e0, zero past M) and their digits.
__device__ __forceinline__ uint32_t load_edges(const FormatArgs &a, uint64_t e0, uint32_t (&us)[FMT_ITEMS],
                                               uint32_t (&vs)[FMT_ITEMS], int (&du)[FMT_ITEMS],
                                               int (&dv)[FMT_ITEMS]) {
    static_assert(FMT_ITEMS == 4, "one 16-byte load per thread");
    if (a.vec && e0 + FMT_ITEMS <= a.M) {
        const uint4 pu = __ldg(reinterpret_cast<const uint4 *>(a.u + e0));
        const uint4 pv = __ldg(reinterpret_cast<const uint4 *>(a.v + e0));
        us[0] = pu.x, us[1] = pu.y, us[2] = pu.z, us[3] = pu.w;
        vs[0] = pv.x, vs[1] = pv.y, vs[2] = pv.z, vs[3] = pv.w;
    } else {
#pragma unroll
        for (int j = 0; j < FMT_ITEMS; ++j) {
            us[j] = e0 + j < a.M ? a.u[e0 + j] : 0u;
            vs[j] = e0 + j < a.M ? a.v[e0 + j] : 0u;
        }
    }
    uint32_t bytes = 0;
#pragma unroll
    for (int j = 0; j < FMT_ITEMS; ++j) {
        const bool ok = e0 + j < a.M;
        du[j] = ok ? ndigits(us[j]) : 0;
        dv[j] = ok ? ndigits(vs[j]) : 0;
        bytes += ok ? (uint32_t)(du[j] + dv[j] + 2) : 0u;
    }
    return bytes;
}

// Bytes of text of each tile of edges.
__global__ void __launch_bounds__(THREADS) format_count_kernel(FormatArgs a) {
    __shared__ uint64_t s_scan[40];
    const uint64_t tile = blockIdx.x;
    uint32_t us[FMT_ITEMS], vs[FMT_ITEMS];
    int du[FMT_ITEMS], dv[FMT_ITEMS];
    const uint32_t mine = load_edges(a, tile * FMT_TILE + (uint64_t)threadIdx.x * FMT_ITEMS, us, vs, du, dv);
    uint64_t total;
    block_exclusive_sum<uint64_t, THREADS>((uint64_t)mine, s_scan, &total);
    if (threadIdx.x == 0) a.offs[tile] = total;
}

__global__ void __launch_bounds__(THREADS) format_kernel(FormatArgs a) {
    __shared__ __align__(16) char s_text[16 + FMT_TILE * MAX_LINE];  // placed at the destination's alignment
    __shared__ uint64_t s_scan[40];
    const int tid = threadIdx.x;
    const uint64_t tile = blockIdx.x;
    const uint64_t e0 = tile * FMT_TILE + (uint64_t)tid * FMT_ITEMS;
    uint32_t us[FMT_ITEMS], vs[FMT_ITEMS];
    int du[FMT_ITEMS], dv[FMT_ITEMS];
    const uint32_t mine = load_edges(a, e0, us, vs, du, dv);
    uint64_t total;
    const uint64_t ex = block_exclusive_sum<uint64_t, THREADS>((uint64_t)mine, s_scan, &total);
    // the text sits in shared memory at its destination's offset modulo 16
    char *dst = a.text + a.offs[tile];
    const uint32_t sh = (uint32_t)(reinterpret_cast<uintptr_t>(dst) & 15u);
    uint32_t at = sh + (uint32_t)ex;  // < 16 + FMT_TILE * MAX_LINE
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
    // 16-byte pieces of the aligned span around [dst, dst + total): whole
    // pieces as one 16-byte copy, the partial first and last bytewise
    char *abase = dst - sh;
    const uint32_t end = sh + (uint32_t)total, npieces = (end + 15u) / 16u;
    for (uint32_t k = tid; k < npieces; k += THREADS) {
        const uint32_t lo = max(16u * k, sh), hi = min(16u * k + 16u, end);
        if (lo == 16u * k && hi == 16u * k + 16u) {
            *reinterpret_cast<uint4 *>(abase + lo) = *reinterpret_cast<const uint4 *>(s_text + lo);
        } else {
            for (uint32_t b = lo; b < hi; ++b) abase[b] = s_text[b];
        }
    }
}

struct ParseArgs {
    const char *text;
    uint64_t len;
    int vec;  // text is 16-byte aligned
    uint32_t *u, *v;
    uint64_t m_cap;
    uint64_t *offs;  // [tiles + 1] lines before each tile (after the scan)
};

// Newlines of a tile of text, one launch over all tiles.
__global__ void __launch_bounds__(THREADS) parse_count_kernel(ParseArgs a) {
    __shared__ uint64_t s_scan[40];
    const uint64_t c0 = (uint64_t)blockIdx.x * PARSE_TILE + (uint64_t)threadIdx.x * PARSE_BYTES;
    uint32_t n = 0;
    if (a.vec && c0 + PARSE_BYTES <= a.len) {
        const uint4 *p = reinterpret_cast<const uint4 *>(a.text + c0);
#pragma unroll
        for (int k = 0; k < PARSE_BYTES / 16; ++k) {
            const uint4 w = __ldg(p + k);
            n += __popc(bytes_equal(w.x, 0x0a0a0a0au)) + __popc(bytes_equal(w.y, 0x0a0a0a0au)) +
                 __popc(bytes_equal(w.z, 0x0a0a0a0au)) + __popc(bytes_equal(w.w, 0x0a0a0a0au));
        }
    } else {
        for (int k = 0; k < PARSE_BYTES; ++k) n += (c0 + k < a.len && __ldg(a.text + c0 + k) == '\n') ? 1u : 0u;
    }
    uint64_t total;
    block_exclusive_sum<uint64_t, THREADS>((uint64_t)n, s_scan, &total);
    if (threadIdx.x == 0) a.offs[blockIdx.x] = total;
}

// Eight bytes of shared memory from byte a (a + 11 within the buffer).
__device__ __forceinline__ uint64_t load8(const char *b, int a) {
    const uint32_t *w = reinterpret_cast<const uint32_t *>(b + (a & ~3));
    const uint32_t sh = 8u * (uint32_t)(a & 3);
    const uint32_t w0 = w[0], w1 = w[1], w2 = w[2];
    return (uint64_t)__funnelshift_r(w0, w1, sh) | ((uint64_t)__funnelshift_r(w1, w2, sh) << 32);
}

// The n decimal digits (1 <= n <= 10, already checked to be digits) at b[a]:
// false if the value exceeds 2^32 - 1.
__device__ __forceinline__ bool field_value(const char *b, int a, int n, uint32_t &out) {
    if (n <= 8) {
        // the digits to the top of the word, '0' below them
        const uint64_t w = (load8(b, a) << (8 * (8 - n))) | ((0x3030303030303030ull >> (8 * n - 1)) >> 1);
        out = eight_digits(w);
        return true;
    }
    uint32_t hi = (uint32_t)(b[a] - '0');
    if (n == 10) hi = hi * 10u + (uint32_t)(b[a + 1] - '0');
    const uint64_t v = (uint64_t)hi * 100000000ull + eight_digits(load8(b, a + n - 8));
    out = (uint32_t)v;
    return v <= 0xffffffffull;
}

// Parses the line b[s, q) ("digits\tdigits"; b[q] is its newline); false if
// malformed.  The line is classified word by word: a well-formed line has
// exactly one non-digit byte, a tab, with 1 to 10 digits on each side.
__device__ __forceinline__ bool parse_line(const char *b, int s, int q, uint32_t &x, uint32_t &y) {
    const int len = q - s;
    if (len < 3 || len > MAX_LINE - 1) return false;
    const uint32_t *w = reinterpret_cast<const uint32_t *>(b + (s & ~3));
    const uint32_t sh = 8u * (uint32_t)(s & 3);
    uint32_t nd = 0;  // non-digit bytes of the 24 from s, one bit each
    uint32_t lo = w[0];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const uint32_t hi = w[i + 1];
        nd |= nibble(bytes_nondigit(__funnelshift_r(lo, hi, sh))) << (4 * i);
        lo = hi;
    }
    nd &= (1u << len) - 1u;
    if (__popc(nd) != 1) return false;
    const int t = __ffs(nd) - 1;
    const int nx = t, ny = len - t - 1;
    if (b[s + t] != '\t' || nx < 1 || nx > 10 || ny < 1 || ny > 10) return false;
    const bool okx = field_value(b, s, nx, x);
    const bool oky = field_value(b, s + t + 1, ny, y);
    return okx && oky;
}

__global__ void __launch_bounds__(THREADS) parse_kernel(ParseArgs a) {
    // s_b[HALO + i] = text[c0 + i]; s_b[HALO - j] = text[c0 - j] (a newline
    // before the text's start); TAIL zero bytes after the tile
    __shared__ __align__(16) char s_b[HALO + PARSE_TILE + TAIL];
    __shared__ uint32_t s_nl[THREADS + 1];  // newline masks: [0] the halo, [1 + t] thread t's bytes
    __shared__ uint32_t s_u[STAGE_LINES], s_v[STAGE_LINES];
    __shared__ uint64_t s_scan[40];
    const int tid = threadIdx.x;
    const uint64_t tile = blockIdx.x;
    const uint64_t ntiles = (a.len + PARSE_TILE - 1) / PARSE_TILE;
    const uint64_t c0 = tile * PARSE_TILE;
    const int my0 = HALO + tid * PARSE_BYTES;
    uint32_t *mine = reinterpret_cast<uint32_t *>(s_b + my0);
    if (a.vec && c0 + PARSE_TILE <= a.len) {
        const uint4 *p = reinterpret_cast<const uint4 *>(a.text + c0) + tid * (PARSE_BYTES / 16);
#pragma unroll
        for (int k = 0; k < PARSE_BYTES / 16; ++k) reinterpret_cast<uint4 *>(mine)[k] = __ldg(p + k);
    } else {
        for (int i = tid; i < PARSE_TILE; i += THREADS) s_b[HALO + i] = c0 + i < a.len ? __ldg(a.text + c0 + i) : '\0';
    }
    if (tid < HALO) s_b[tid] = c0 >= (uint64_t)(HALO - tid) ? __ldg(a.text + c0 - (HALO - tid)) : '\n';
    if (tid < TAIL / 4) reinterpret_cast<uint32_t *>(s_b + HALO + PARSE_TILE)[tid] = 0u;
    __syncthreads();
    // newline masks of this thread's bytes and (thread 0) of the halo; bytes
    // past the text's end were loaded as 0
    uint32_t nl = 0;
#pragma unroll
    for (int q = 0; q < PARSE_BYTES / 4; ++q) nl |= nibble(bytes_equal(mine[q], 0x0a0a0a0au)) << (4 * q);
    s_nl[1 + tid] = nl;
    if (tid == 0) {
        uint32_t h = 0;
#pragma unroll
        for (int q = 0; q < HALO / 4; ++q)
            h |= nibble(bytes_equal(reinterpret_cast<const uint32_t *>(s_b)[q], 0x0a0a0a0au)) << (4 * q);
        s_nl[0] = h;
    }
    uint64_t total;  // the block scan's barriers also publish s_nl
    const uint64_t ex = block_exclusive_sum<uint64_t, THREADS>((uint64_t)__popc(nl), s_scan, &total);
    const uint64_t first_line = a.offs[tile];
    if (tid == 0 && tile == ntiles - 1) {
        if (a.text[a.len - 1] != '\n') pp_set_error(PP_DEV_PARSE);  // a last line without newline
        if (first_line + total > a.m_cap) pp_set_error(PP_DEV_PARSE);
    }
    // the first line starts after the last newline of the 32 bytes before this
    // thread's; without one it is longer than any well-formed line
    const uint32_t prev = s_nl[tid];
    int start = prev ? my0 - 32 + (32 - __clz(prev)) : -1;
    uint32_t li = (uint32_t)ex;  // index of this thread's next line within the tile
    while (nl) {
        const int k = __ffs(nl) - 1;
        nl &= nl - 1;
        const int pos = my0 + k;  // the newline
        uint32_t x = 0, y = 0;
        if (start < 0 || !parse_line(s_b, start, pos, x, y)) {
            pp_set_error(PP_DEV_PARSE);  // too long, or not "digits\tdigits"
            x = y = 0;
        }
        start = pos + 1;
        if (li < (uint32_t)STAGE_LINES) {
            s_u[li] = x;
            s_v[li] = y;
        } else if (first_line + li < a.m_cap) {
            a.u[first_line + li] = x;  // only malformed text has this many lines
            a.v[first_line + li] = y;
        }
        ++li;
    }
    __syncthreads();
    const uint32_t staged = total < (uint64_t)STAGE_LINES ? (uint32_t)total : (uint32_t)STAGE_LINES;
    for (uint32_t i = tid; i < staged; i += THREADS) {
        if (first_line + i < a.m_cap) {
            a.u[first_line + i] = s_u[i];
            a.v[first_line + i] = s_v[i];
        }
    }
}

inline uint64_t format_tiles(uint64_t M) { return ceil_div(M ? M : 1, FMT_TILE); }
inline uint64_t parse_tiles(uint64_t L) { return ceil_div(L ? L : 1, PARSE_TILE); }

// Workspace: the tile counts / offsets (tiles + 1 words).
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
    PP_ENTRY("pp_format_tsv");
    if (M > (1ull << 31) || !text_len || (M && (!u || !v || !text))) return PP_ERR_INVALID_ARG;
    if (text_cap < M * (uint64_t)PP_TSV_MAX_LINE) return PP_ERR_INVALID_ARG;
    const uint64_t tiles = tsv::format_tiles(M);
    pp_status st = check_ws(ws, ws_bytes, tsv::ws_bytes(tiles));
    if (st != PP_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t *offs = static_cast<uint64_t *>(ws);
    cudaMemsetAsync(text_len, 0, sizeof(uint64_t), s);
    if (M) {
        const int vec = ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(v)) & 15u) == 0;
        const tsv::FormatArgs fa{u, v, M, vec, text, offs};
        tsv::format_count_kernel<<<(unsigned)tiles, tsv::THREADS, 0, s>>>(fa);
        tsv::scan_kernel<<<1, tsv::SCAN_THREADS, 0, s>>>(offs, tiles, text_len);
        tsv::format_kernel<<<(unsigned)tiles, tsv::THREADS, 0, s>>>(fa);
        count_launch(3);
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
    PP_ENTRY("pp_parse_tsv");
    if (text_len > (1ull << 31) * (uint64_t)PP_TSV_MAX_LINE || !m_out || (text_len && !text) ||
        (m_cap && (!u || !v)))
        return PP_ERR_INVALID_ARG;
    const uint64_t tiles = tsv::parse_tiles(text_len);
    pp_status st = check_ws(ws, ws_bytes, tsv::ws_bytes(tiles));
    if (st != PP_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t *offs = static_cast<uint64_t *>(ws);
    cudaMemsetAsync(m_out, 0, sizeof(uint64_t), s);
    if (text_len) {
        const int vec = (reinterpret_cast<uintptr_t>(text) & 15u) == 0;
        const tsv::ParseArgs pa{text, text_len, vec, u, v, m_cap, offs};
        tsv::parse_count_kernel<<<(unsigned)tiles, tsv::THREADS, 0, s>>>(pa);
        tsv::scan_kernel<<<1, tsv::SCAN_THREADS, 0, s>>>(offs, tiles, m_out);
        tsv::parse_kernel<<<(unsigned)tiles, tsv::THREADS, 0, s>>>(pa);
        count_launch(3);
    }
    return launch_status();
}
