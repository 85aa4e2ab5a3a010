// Library-wide entry points: status strings, the device error word, the
// launch counter, and the host-buffer pipeline (Kernels 1-3 back to back).
#include <algorithm>
#include <cstring>
#include <mutex>

#include "pp_common.cuh"

namespace pp {
std::atomic<uint64_t> g_launches{0};
uint32_t k1_fetch_error(cudaStream_t s);
uint32_t k2_fetch_error(cudaStream_t s);
uint32_t k3_fetch_error(cudaStream_t s);
uint32_t k3b_fetch_error(cudaStream_t s);
uint32_t tsv_fetch_error(cudaStream_t s);
uint32_t kx_fetch_error(cudaStream_t s);
uint32_t kr_fetch_error(cudaStream_t s);
}  // namespace pp

namespace pp {
namespace {
struct Knob {
    const char *key;
    std::atomic<int64_t> value;
    int n_allowed;
    int64_t allowed[5];
};
Knob g_knobs[] = {
    {"k3_unroll_f32", {8}, 2, {4, 8}},
    {"k3_unroll_f64", {4}, 2, {4, 8}},
    {"k3_minblocks", {4}, 3, {4, 6, 8}},
    {"k3_shortmax", {256}, 3, {128, 256, 512}},
    {"k3_chunk", {4096}, 2, {2048, 4096}},
    {"k3b_shortmax", {256}, 2, {128, 256}},
    {"k3b_chunk", {512}, 3, {256, 512, 1024}},
    {"k3b_vec", {1}, 2, {0, 1}},
};
Knob *find_knob(const char *key) {
    if (!key) return nullptr;
    for (Knob &k : g_knobs)
        if (std::strcmp(k.key, key) == 0) return &k;
    return nullptr;
}
}  // namespace

int64_t tuning(const char *key) {
    Knob *k = find_knob(key);
    return k ? k->value.load() : 0;
}

// Armed failures: the next `left` calls of entry point `name` ("*": any)
// return `status`.
namespace {
struct Fault {
    char name[64];
    pp_status status;
    uint32_t left;
};
constexpr int kMaxFaults = 16;
Fault g_faults[kMaxFaults];
std::mutex g_fault_mu;
}  // namespace
std::atomic<int> g_faults_armed{0};

bool fault_hit(const char *name, pp_status *st) {
    std::lock_guard<std::mutex> lock(g_fault_mu);
    for (Fault &f : g_faults) {
        if (f.left && (std::strcmp(f.name, name) == 0 || std::strcmp(f.name, "*") == 0)) {
            *st = f.status;
            if (--f.left == 0) g_faults_armed.fetch_sub(1, std::memory_order_relaxed);
            return true;
        }
    }
    return false;
}
}  // namespace pp

using namespace pp;

extern "C" pp_status pp_set_tuning(const char *key, int64_t value) {
    Knob *k = find_knob(key);
    if (!k) return PP_ERR_INVALID_ARG;
    for (int i = 0; i < k->n_allowed; ++i)
        if (k->allowed[i] == value) {
            k->value.store(value);
            return PP_OK;
        }
    return PP_ERR_INVALID_ARG;
}

extern "C" pp_status pp_get_tuning(const char *key, int64_t *value) {
    Knob *k = find_knob(key);
    if (!k || !value) return PP_ERR_INVALID_ARG;
    *value = k->value.load();
    return PP_OK;
}

extern "C" uint64_t pp_launch_count(void) { return g_launches.load(); }

extern "C" pp_status pp_inject_fault(const char *call, pp_status status, uint32_t count) {
    if (!call || std::strlen(call) >= sizeof(((Fault *)nullptr)->name)) return PP_ERR_INVALID_ARG;
    if (count && (status == PP_OK || (int)status < 0 || (int)status > PP_ERR_DEVICE)) return PP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_fault_mu);
    Fault *slot = nullptr;
    for (Fault &f : g_faults)
        if (f.left && std::strcmp(f.name, call) == 0) slot = &f;
    if (!slot && count)
        for (Fault &f : g_faults)
            if (!f.left) {
                slot = &f;
                break;
            }
    if (!slot) return count ? PP_ERR_INVALID_ARG : PP_OK;  // table full / nothing to clear
    if (slot->left) g_faults_armed.fetch_sub(1, std::memory_order_relaxed);
    std::strcpy(slot->name, call);
    slot->status = status;
    slot->left = count;
    if (count) g_faults_armed.fetch_add(1, std::memory_order_relaxed);
    return PP_OK;
}

extern "C" uint32_t pp_build_flags(void) {
    uint32_t f = 0;
#ifdef PP_CHECKED
    f |= PP_BUILD_CHECKED;
#endif
#ifndef PP_NO_NVTX
    f |= PP_BUILD_NVTX;
#endif
    return f;
}

extern "C" const char *pp_status_string(pp_status st) {
    switch (st) {
        case PP_OK: return "ok";
        case PP_ERR_INVALID_ARG: return "invalid argument";
        case PP_ERR_WORKSPACE: return "workspace missing, too small or not 256-byte aligned";
        case PP_ERR_CUDA: return "CUDA runtime error";
        case PP_ERR_DEVICE: return "the device recorded an error (see pp_last_device_error)";
    }
    return "unknown status";
}

extern "C" pp_status pp_last_device_error(void *stream, uint32_t *code) {
    PP_ENTRY("pp_last_device_error");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return PP_ERR_CUDA;
    uint32_t w = 0;
    const uint32_t parts[7] = {k1_fetch_error(s), k2_fetch_error(s), k3_fetch_error(s), k3b_fetch_error(s),
                               tsv_fetch_error(s), kx_fetch_error(s), kr_fetch_error(s)};
    for (uint32_t p : parts) {
        if (p == 0xffffffffu) return PP_ERR_CUDA;
        w |= p;
    }
    if (code) *code = w;
    return w ? PP_ERR_DEVICE : PP_OK;
}

namespace pp {
// Kernel 1 in chunks (k1_sort.cu), for the host-buffer pipeline.
size_t k1_chunk_workspace(uint64_t Mc, uint32_t scale);
size_t k1_merge_split_words(uint64_t n);
pp_status k1_sort_chunk_keys(const uint32_t *u, const uint32_t *v, uint64_t Mc, uint32_t scale, uint64_t *keys,
                             void *ws, size_t ws_bytes, cudaStream_t s);
pp_status k1_merge_keys(const uint64_t *a, uint64_t na, const uint64_t *b, uint64_t nb, uint64_t *out,
                        uint64_t *split, cudaStream_t s);
pp_status k1_merge_unpack(const uint64_t *a, uint64_t na, const uint64_t *b, uint64_t nb, uint32_t scale,
                          uint32_t *u_out, uint32_t *v_out, uint64_t *split, cudaStream_t s);
}  // namespace pp

namespace {

// The host-buffer pipeline sorts the edge list in CHUNKS pieces while it
// crosses the host link (64-bit keys, at least CHUNK_MIN_M edges).
constexpr int CHUNKS = 4;
constexpr uint64_t CHUNK_MIN_M = 1ull << 20;
inline bool chunked(uint64_t M, uint32_t scale) { return 2 * scale > 32 && M >= CHUNK_MIN_M; }
// chunk boundaries on multiples of 4 ids, so that every chunk starts 16-byte aligned
inline uint64_t chunk_begin(uint64_t M, int c) { return c >= CHUNKS ? M : (M * (uint64_t)c / CHUNKS) & ~3ull; }

struct PipeLayout {
    uint32_t *u, *v, *us, *vs;
    pp_graph g;
    double *r0;
    void *r_out;
    void *scratch;
    size_t scratch_bytes;
    // the chunked sort, inside the scratch region (Kernels 2 and 3 reuse it after)
    uint64_t *keys[2], *split;
    void *chunk_ws;
    size_t chunk_ws_bytes;
    size_t bytes;
};

PipeLayout pipe_layout(void *ws, uint64_t M, uint32_t scale, uint32_t iters, pp_dtype dt) {
    Carver c(ws);
    PipeLayout L;
    const uint64_t N = 1ull << scale;
    const uint64_t cap = M ? M : 1;
    uint64_t len[PP_GRAPH_ARRAYS];
    pp_graph_lengths(M, scale, len);
    L.u = c.take<uint32_t>(cap);
    L.v = c.take<uint32_t>(cap);
    L.us = c.take<uint32_t>(cap);
    L.vs = c.take<uint32_t>(cap);
    L.g.scale = scale;
    L.g.reserved = 0;
    L.g.M = M;
    L.g.colptr = c.take<uint32_t>(len[0]);
    L.g.rowc = c.take<uint32_t>(len[1]);
    L.g.ovf_key = c.take<uint64_t>(len[2]);
    L.g.ovf_cnt = c.take<uint32_t>(len[3]);
    L.g.d_in = c.take<uint32_t>(len[4]);
    L.g.d_out = c.take<uint32_t>(len[5]);
    L.g.inv_dout32 = c.take<float>(len[6]);
    L.g.inv_dout64 = c.take<double>(len[7]);
    L.g.info = c.take<uint64_t>(len[8]);
    L.g.perm = c.take<uint32_t>(len[9]);
    L.g.iperm = c.take<uint32_t>(len[10]);
    L.r0 = c.take<double>(N);
    L.r_out = c.take<char>(N * (dt == PP_FP64 ? 8 : 4));
    size_t b1 = 0, b2 = 0, b3 = 0;
    pp_sort_edges_workspace(M, scale, &b1);
    pp_build_filter_normalize_workspace(M, scale, &b2);
    pp_pagerank_workspace(M, scale, iters, dt, &b3);
    // the chunked sort's buffers, carved from the start of the scratch region
    Carver k(nullptr);
    L.keys[0] = L.keys[1] = L.split = nullptr;
    L.chunk_ws = nullptr;
    L.chunk_ws_bytes = 0;
    if (chunked(M, scale)) {
        k.take<uint64_t>(M);
        k.take<uint64_t>(M);
        k.take<uint64_t>(k1_merge_split_words(M));
        L.chunk_ws_bytes = k1_chunk_workspace(M / CHUNKS + 4, scale);  // the largest chunk (boundaries rounded to 4)
        k.take<char>(L.chunk_ws_bytes);
    }
    L.scratch_bytes = std::max(std::max(b1, k.size()), std::max(b2, b3));
    L.scratch = c.take<char>(L.scratch_bytes);
    if (L.scratch && chunked(M, scale)) {
        Carver kc(L.scratch);
        L.keys[0] = kc.take<uint64_t>(M);
        L.keys[1] = kc.take<uint64_t>(M);
        L.split = kc.take<uint64_t>(k1_merge_split_words(M));
        L.chunk_ws = kc.take<char>(L.chunk_ws_bytes);
    }
    L.bytes = c.size();
    return L;
}

}  // namespace

extern "C" pp_status pp_pipeline_workspace(uint64_t M, uint32_t scale, uint32_t iters, pp_dtype dt,
                                           size_t *bytes) {
    if (!bytes || scale < 1 || scale > 27 || M > (1ull << 31) || (int)dt < 0 || (int)dt > 3)
        return PP_ERR_INVALID_ARG;
    *bytes = pipe_layout(nullptr, M, scale, iters, dt).bytes;
    return PP_OK;
}

// A side stream that starts after the work already enqueued on `s`, and an
// event marking the end of what is enqueued on it.  Destroying them while
// their work is pending is allowed: the runtime releases them when it ends.
struct SideCopy {
    static constexpr int EVENTS = CHUNKS + 1;
    cudaStream_t stream = nullptr;
    cudaEvent_t start = nullptr, done[EVENTS] = {};
    bool open(cudaStream_t s) {
        bool ok = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&start, cudaEventDisableTiming) == cudaSuccess;
        for (int e = 0; e < EVENTS && ok; ++e) ok = cudaEventCreateWithFlags(&done[e], cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaEventRecord(start, s) == cudaSuccess && cudaStreamWaitEvent(stream, start, 0) == cudaSuccess;
        if (!ok) {
            close();
            cudaGetLastError();
        }
        return ok;
    }
    void close() {
        if (start) cudaEventDestroy(start);
        for (cudaEvent_t &e : done) {
            if (e) cudaEventDestroy(e);
            e = nullptr;
        }
        if (stream) cudaStreamDestroy(stream);
        start = nullptr;
        stream = nullptr;
    }
    ~SideCopy() { close(); }
};

// Kernel 1 of the host-buffer pipeline in chunks: chunk c's ids are copied
// on the side stream (event done[c]); the main stream sorts each chunk into
// packed keys once it has arrived, then merges the four sorted chunks in two
// rounds, the last one writing the sorted (u, v).
static pp_status sort_chunked(const PipeLayout &L, const uint32_t *u_host, const uint32_t *v_host, uint64_t M,
                              uint32_t scale, SideCopy &side, cudaStream_t s) {
    for (int c = 0; c < CHUNKS; ++c) {
        const uint64_t b = chunk_begin(M, c), n = chunk_begin(M, c + 1) - b;
        if (cudaMemcpyAsync(L.u + b, u_host + b, n * 4, cudaMemcpyHostToDevice, side.stream) != cudaSuccess ||
            cudaMemcpyAsync(L.v + b, v_host + b, n * 4, cudaMemcpyHostToDevice, side.stream) != cudaSuccess ||
            cudaEventRecord(side.done[c], side.stream) != cudaSuccess)
            return PP_ERR_CUDA;
    }
    for (int c = 0; c < CHUNKS; ++c) {
        const uint64_t b = chunk_begin(M, c), n = chunk_begin(M, c + 1) - b;
        if (cudaStreamWaitEvent(s, side.done[c], 0) != cudaSuccess) return PP_ERR_CUDA;
        pp_status st = k1_sort_chunk_keys(L.u + b, L.v + b, n, scale, L.keys[0] + b, L.chunk_ws, L.chunk_ws_bytes, s);
        if (st != PP_OK) return st;
    }
    static_assert(CHUNKS == 4, "two merge rounds");
    const uint64_t q1 = chunk_begin(M, 1), q2 = chunk_begin(M, 2), q3 = chunk_begin(M, 3);
    pp_status st = k1_merge_keys(L.keys[0], q1, L.keys[0] + q1, q2 - q1, L.keys[1], L.split, s);
    if (st == PP_OK) st = k1_merge_keys(L.keys[0] + q2, q3 - q2, L.keys[0] + q3, M - q3, L.keys[1] + q2, L.split, s);
    if (st == PP_OK) st = k1_merge_unpack(L.keys[1], q2, L.keys[1] + q2, M - q2, scale, L.us, L.vs, L.split, s);
    return st;
}

extern "C" pp_status pp_pipeline_host(const uint32_t *u_host, const uint32_t *v_host, uint64_t M,
                                      uint32_t scale, const double *r0_host, uint32_t iters, double c,
                                      pp_dtype dt, pp_supernode_rule rule, void *r_out_host,
                                      uint64_t *info_host, void *ws, size_t ws_bytes, void *stream) {
    PP_ENTRY("pp_pipeline_host");
    if (scale < 1 || scale > 27 || M > (1ull << 31) || (int)dt < 0 || (int)dt > 3) return PP_ERR_INVALID_ARG;
    if ((M && (!u_host || !v_host)) || !r0_host || !r_out_host) return PP_ERR_INVALID_ARG;
    const PipeLayout need = pipe_layout(nullptr, M, scale, iters, dt);
    pp_status st = check_ws(ws, ws_bytes, need.bytes);
    if (st != PP_OK) return st;
    const PipeLayout L = pipe_layout(ws, M, scale, iters, dt);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t N = 1ull << scale;
    // The copies run on a side stream where one can be had: the edge list in
    // chunks that Kernel 1 sorts as they arrive (large graphs), then r0, which
    // only Kernel 3 reads, while Kernels 1 and 2 compute.  The side stream and
    // its events are released once their work is done.
    SideCopy side;
    const pp_status result = [&]() -> pp_status {
        const bool split_copy = chunked(M, scale) && side.open(s);
        if (split_copy) {
            st = sort_chunked(L, u_host, v_host, M, scale, side, s);
            if (st != PP_OK) return st;
        } else {
            if (M) {
                if (cudaMemcpyAsync(L.u, u_host, M * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) return PP_ERR_CUDA;
                if (cudaMemcpyAsync(L.v, v_host, M * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) return PP_ERR_CUDA;
            }
            side.open(s);  // after the edge copies, which the r0 copy would only slow down on the host link
        }
        const cudaEvent_t r0_done = side.stream ? side.done[CHUNKS] : nullptr;
        if (r0_done) {
            if (cudaMemcpyAsync(L.r0, r0_host, N * 8, cudaMemcpyHostToDevice, side.stream) != cudaSuccess)
                return PP_ERR_CUDA;
            if (cudaEventRecord(r0_done, side.stream) != cudaSuccess) return PP_ERR_CUDA;
        } else if (cudaMemcpyAsync(L.r0, r0_host, N * 8, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            return PP_ERR_CUDA;
        }
        if (!split_copy) {
            st = pp_sort_edges(L.u, L.v, M, scale, L.us, L.vs, L.scratch, L.scratch_bytes, stream);
            if (st != PP_OK) return st;
        }
        st = pp_build_filter_normalize(L.us, L.vs, M, scale, rule, &L.g, L.scratch, L.scratch_bytes, stream);
        if (st != PP_OK) return st;
        if (r0_done && cudaStreamWaitEvent(s, r0_done, 0) != cudaSuccess) return PP_ERR_CUDA;
        st = pp_pagerank(&L.g, L.r0, iters, c, dt, L.r_out, nullptr, L.scratch, L.scratch_bytes, stream);
        if (st != PP_OK) return st;
        if (cudaMemcpyAsync(r_out_host, L.r_out, N * (dt == PP_FP64 ? 8 : 4), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return PP_ERR_CUDA;
        if (info_host &&
            cudaMemcpyAsync(info_host, L.g.info, PP_INFO_LEN * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return PP_ERR_CUDA;
        return PP_OK;
    }();
    if (result != PP_OK && side.stream) {
        // On an error the main stream may not have waited for every copy on
        // the side stream; those copies write into the caller's workspace, so
        // they are ordered before whatever the caller enqueues on `stream` next.
        if (cudaEventRecord(side.start, side.stream) == cudaSuccess) cudaStreamWaitEvent(s, side.start, 0);
        cudaGetLastError();
    }
    return result;
}

// ---------------------------------------------------------------------------
// CUDA-graph capture of the batched Kernel 3 stage.

struct pp_exec {
    cudaGraphExec_t exec;
    uint64_t kernels;  // kernels in the graph, for pp_launch_count
};

extern "C" pp_status pp_pagerank_batched_capture(const pp_graph *gs, uint32_t n_graphs, const double *r0,
                                                 uint32_t nrhs, uint32_t iters, double c, float *r_out, void *ws,
                                                 size_t ws_bytes, void *stream, pp_exec **exec) {
    PP_ENTRY("pp_pagerank_batched_capture");
    if (!exec) return PP_ERR_INVALID_ARG;
    *exec = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool own = s == nullptr;  // the legacy default stream cannot be captured
    if (own && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return PP_ERR_CUDA;
    pp_status st = PP_ERR_CUDA;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
        const uint64_t before = g_launches.load();
        st = pp_pagerank_batched(gs, n_graphs, r0, nrhs, iters, c, r_out, ws, ws_bytes, s);
        const uint64_t kernels = g_launches.load() - before;
        g_launches.fetch_sub(kernels);  // recorded, not launched
        const cudaError_t e = cudaStreamEndCapture(s, &graph);
        if (st == PP_OK && (e != cudaSuccess || !graph)) st = PP_ERR_CUDA;
        if (st == PP_OK) {
            cudaGraphExec_t ge = nullptr;
            if (cudaGraphInstantiate(&ge, graph, 0) == cudaSuccess) {
                *exec = new pp_exec{ge, kernels};
            } else {
                st = PP_ERR_CUDA;
            }
        }
    }
    if (graph) cudaGraphDestroy(graph);
    if (st != PP_OK) cudaGetLastError();
    if (own) cudaStreamDestroy(s);
    return st;
}

namespace {
bool batch_sizes(uint32_t n, const pp_graph *gs, uint64_t *M, uint32_t *scale) {
    if (!gs || n < 1 || n > PP_BATCH_MAX_GRAPHS) return false;
    for (uint32_t g = 0; g < n; ++g) {
        M[g] = gs[g].M;
        scale[g] = gs[g].scale;
    }
    return true;
}
}  // namespace

extern "C" pp_status pp_pipeline_batched_workspace(uint32_t n_graphs, const pp_graph *gs, uint32_t nrhs,
                                                   uint32_t iters, size_t *bytes) {
    uint64_t M[PP_BATCH_MAX_GRAPHS];
    uint32_t scale[PP_BATCH_MAX_GRAPHS];
    if (!bytes || !batch_sizes(n_graphs, gs, M, scale)) return PP_ERR_INVALID_ARG;
    size_t b1 = 0, b2 = 0, b3 = 0;
    pp_status st = pp_sort_edges_batched_workspace(n_graphs, M, scale, &b1);
    if (st == PP_OK) st = pp_build_filter_normalize_batched_workspace(n_graphs, M, scale, &b2);
    if (st == PP_OK) st = pp_pagerank_batched_workspace(gs, n_graphs, nrhs, iters, &b3);
    if (st != PP_OK) return st;
    *bytes = std::max(b1, std::max(b2, b3));
    return PP_OK;
}

extern "C" pp_status pp_pipeline_batched_capture(uint32_t n_graphs, const uint32_t *const *u,
                                                 const uint32_t *const *v, uint32_t *const *u_sorted,
                                                 uint32_t *const *v_sorted, pp_supernode_rule rule, const pp_graph *gs,
                                                 const double *r0, uint32_t nrhs, uint32_t iters, double c,
                                                 float *r_out, void *ws, size_t ws_bytes, void *stream,
                                                 pp_exec **exec) {
    PP_ENTRY("pp_pipeline_batched_capture");
    if (!exec) return PP_ERR_INVALID_ARG;
    *exec = nullptr;
    uint64_t M[PP_BATCH_MAX_GRAPHS];
    uint32_t scale[PP_BATCH_MAX_GRAPHS];
    if (!batch_sizes(n_graphs, gs, M, scale) || !u_sorted || !v_sorted) return PP_ERR_INVALID_ARG;
    size_t need = 0;
    pp_status st = pp_pipeline_batched_workspace(n_graphs, gs, nrhs, iters, &need);
    if (st != PP_OK) return st;
    st = check_ws(ws, ws_bytes, need);
    if (st != PP_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool own = s == nullptr;
    if (own && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return PP_ERR_CUDA;
    st = PP_ERR_CUDA;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
        const uint64_t before = g_launches.load();
        st = pp_sort_edges_batched(n_graphs, u, v, M, scale, u_sorted, v_sorted, ws, ws_bytes, s);
        if (st == PP_OK)
            st = pp_build_filter_normalize_batched(n_graphs, u_sorted, v_sorted, rule, gs, ws, ws_bytes, s);
        if (st == PP_OK) st = pp_pagerank_batched(gs, n_graphs, r0, nrhs, iters, c, r_out, ws, ws_bytes, s);
        const uint64_t kernels = g_launches.load() - before;
        g_launches.fetch_sub(kernels);  // recorded, not launched
        const cudaError_t e = cudaStreamEndCapture(s, &graph);
        if (st == PP_OK && (e != cudaSuccess || !graph)) st = PP_ERR_CUDA;
        if (st == PP_OK) {
            cudaGraphExec_t ge = nullptr;
            if (cudaGraphInstantiate(&ge, graph, 0) == cudaSuccess)
                *exec = new pp_exec{ge, kernels};
            else
                st = PP_ERR_CUDA;
        }
    }
    if (graph) cudaGraphDestroy(graph);
    if (st != PP_OK) cudaGetLastError();
    if (own) cudaStreamDestroy(s);
    return st;
}

extern "C" pp_status pp_exec_launch(pp_exec *exec, void *stream) {
    PP_ENTRY("pp_exec_launch");
    if (!exec) return PP_ERR_INVALID_ARG;
    if (cudaGraphLaunch(exec->exec, static_cast<cudaStream_t>(stream)) != cudaSuccess) return PP_ERR_CUDA;
    count_launch(exec->kernels);
    return PP_OK;
}

extern "C" pp_status pp_exec_destroy(pp_exec *exec) {
    if (!exec) return PP_OK;
    const cudaError_t e = cudaGraphExecDestroy(exec->exec);
    delete exec;
    return e == cudaSuccess ? PP_OK : PP_ERR_CUDA;
}
