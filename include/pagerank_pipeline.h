/*
 * libpp — GB300 (sm_103a) CUDA implementation of the data-parallel hot path
 * of the PageRank Pipeline Benchmark (Dreher et al., arXiv:1603.01876):
 *
 *   Kernel 1 (Sec. IV-B)  sort the edge list by start vertex,
 *   Kernel 2 (Sec. IV-C)  build the count matrix A = sparse(u,v,1,N,N), take
 *                         the in-degree, zero the supernode and leaf columns,
 *                         take the out-degree and normalise the rows,
 *   Kernel 3 (Sec. IV-D)  run damped PageRank iterations
 *                         r = ((c.*r)*A) + ((1-c)/N).*sum(r).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Vertex ids are 0-based uint32 in [0, N), N = 2^scale, 1 <= scale <= 27.
 *    (The paper's Matlab statements are 1-based.)  Edge counts M <= 2^31.
 *  - Every array argument is DEVICE memory owned by the caller unless its
 *    name ends in _host.  The library never allocates device memory: scratch
 *    space ("workspace") is passed in, its size given by the matching
 *    *_workspace query.  Workspace must be 256-byte aligned.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    asynchronous: they enqueue kernels and return.  Argument errors found on
 *    the host are returned at once and nothing is enqueued.  Errors found on
 *    the device (an out-of-range vertex id, an expired bounded wait) are
 *    recorded in a device error word that pp_last_device_error() returns.
 *  - Calls on one stream are ordered; two calls may run concurrently on
 *    different streams only if they share no output and no workspace.
 *  - No call launches anything that waits without bound: every cross-block
 *    wait gives up after a fixed number of polls and records PP_DEV_TIMEOUT.
 */
#ifndef PAGERANK_PIPELINE_H
#define PAGERANK_PIPELINE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PP_OK = 0,
    PP_ERR_INVALID_ARG = 1, /* a size, pointer or enum is out of range */
    PP_ERR_WORKSPACE = 2,   /* workspace missing, too small or misaligned */
    PP_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed */
    PP_ERR_DEVICE = 4       /* pp_last_device_error: the device recorded an error */
} pp_status;

/* Arithmetic of Kernel 3's rank vector. */
typedef enum {
    PP_FP64 = 0,          /* stored and accumulated in binary64 */
    PP_FP32 = 1,          /* stored and accumulated in binary32 */
    PP_BF16_FP32ACC = 2,  /* the gathered vector stored in bfloat16, sums in binary32 */
    PP_FP16_FP32ACC = 3   /* the gathered vector stored in binary16 (scaled by a power of
                             two into its range), sums in binary32 */
} pp_dtype;

/* Which columns the supernode statement A(:, d_in == max(d_in)) = 0 zeroes. */
typedef enum {
    PP_SUPERNODE_LOWEST = 0,  /* only the lowest-numbered column attaining the maximum */
    PP_SUPERNODE_ALL_TIES = 1 /* every column attaining the maximum (the literal statement) */
} pp_supernode_rule;

/* Device error word bits (pp_last_device_error). */
#define PP_DEV_RANGE 1u   /* an input vertex id was >= N */
#define PP_DEV_TIMEOUT 2u /* a bounded cross-block wait expired; outputs are invalid */
#define PP_DEV_PARSE 4u   /* edge-file text was malformed (pp_parse_tsv) */
#define PP_DEV_CAPACITY 8u /* an output array was too short for the result (pp_export_csr) */
#define PP_DEV_BOUNDS 16u  /* checked build only: an index read or computed by a kernel
                              was outside the array it addresses; outputs are invalid */

/* Slots of pp_graph.info (device uint64[PP_INFO_LEN]), written by Kernel 2. */
#define PP_INFO_NNZ0 0       /* nonzeros of A before the column filters */
#define PP_INFO_NNZ 1        /* nonzeros of A after them */
#define PP_INFO_DMAX 2       /* max(d_in) */
#define PP_INFO_VMAX 3       /* lowest column attaining max(d_in) */
#define PP_INFO_TIES 4       /* number of columns attaining max(d_in) */
#define PP_INFO_NOVF 5       /* entries whose count does not fit inline (see rowc) */
#define PP_INFO_SUPERNODES 6 /* supernode columns zeroed under the chosen rule */
#define PP_INFO_LEN 8

/*
 * Kernel 2's output: the filtered matrix A in compressed-column form (the
 * layout Kernel 3's pull iteration reads), plus the degree vectors.  All
 * pointers are device arrays allocated by the caller with the lengths that
 * pp_graph_lengths() returns.  Kernel 3 only reads it.
 *
 *   colptr[N+1]  the column of vertex v is at position p = perm[v] and holds
 *                entries colptr[p] .. colptr[p+1]-1; colptr[N] = nnz.
 *   rowc[M]      entry e (e < nnz) packs the position perm[u] of its row u
 *                (= start vertex) in its low `scale` bits and the count
 *                A(u,v) in the high 32-scale bits; within a column the
 *                rows' vertex ids u ascend.  A count >= 2^(32-scale)-1 is stored as the
 *                all-ones field and found in the overflow table.
 *   perm[N], iperm[N]  the storage order of rows and columns: vertices by
 *                decreasing floor(log2(out-degree before the column
 *                filters)), ties by vertex id; perm[v] is the position of
 *                vertex v and iperm[p] the vertex at position p.  Kernel 3
 *                keeps x in this order, so the rows gathered most often sit
 *                together and a warp's gathers share cache lines.  (A storage
 *                order only: d_in, d_out, 1/d_out, the overflow keys and the
 *                ranks are indexed by vertex id.)
 *   ovf_key[n], ovf_cnt[n]  the overflow table: key (u << 32 | v) ascending,
 *                count; n = info[PP_INFO_NOVF] <= pp_graph_lengths()[2].
 *   d_in[N]      sum(A,1) before the column filters (Sec. IV-C step 2).
 *   d_out[N]     sum(A,2) after them (step 4).
 *   inv_dout32[N], inv_dout64[N]  1/d_out (IEEE round-to-nearest division),
 *                0 where d_out = 0; A(u,v) = count * inv_dout[u] (step 4).
 *   info[PP_INFO_LEN]  the scalars listed above.
 */
typedef struct {
    uint32_t scale;
    uint32_t reserved;
    uint64_t M; /* number of edges the graph was built from */
    uint32_t *colptr;
    uint32_t *rowc;
    uint64_t *ovf_key;
    uint32_t *ovf_cnt;
    uint32_t *d_in;
    uint32_t *d_out;
    float *inv_dout32;
    double *inv_dout64;
    uint64_t *info;
    uint32_t *perm;
    uint32_t *iperm;
} pp_graph;

/* Element counts of the pp_graph arrays for M edges at this scale, in the
 * order colptr, rowc, ovf_key, ovf_cnt, d_in, d_out, inv_dout32, inv_dout64,
 * info, perm, iperm.  out[] must hold 11 values. */
#define PP_GRAPH_ARRAYS 11
pp_status pp_graph_lengths(uint64_t M, uint32_t scale, uint64_t out[PP_GRAPH_ARRAYS]);

/*
 * Kernel 1 (Sec. IV-B): sort the edges so that u_out is nondecreasing,
 * u(i-1) <= u(i) <= u(i+1); edges with equal start vertex are ordered by end
 * vertex, which makes the result unique.  u, v: M input ids; u_out, v_out:
 * M outputs, which must not overlap the inputs.  The sort is an LSD radix
 * sort over the key (u << scale | v), ceil(2*scale/8) passes of 8 bits.
 * An id >= N sets PP_DEV_RANGE and leaves the output unspecified.
 */
pp_status pp_sort_edges_workspace(uint64_t M, uint32_t scale, size_t *bytes);
pp_status pp_sort_edges(const uint32_t *u, const uint32_t *v, uint64_t M, uint32_t scale,
                        uint32_t *u_out, uint32_t *v_out, void *workspace, size_t workspace_bytes,
                        void *stream);

/*
 * Kernel 1 for callers that cannot allocate device memory (the paper has no
 * counterpart; this is a deployment variant of pp_sort_edges).  Callers whose
 * GPU memory is owned by another allocator, or who must not trigger
 * cudaMalloc's implicit device synchronisation, pass only inputs and
 * outputs; the scratch space is a fixed array in device memory
 * (about 17 MiB, held by every GPU that loads the library until the process
 * exits).  M must not exceed PP_SORT_STATIC_MAX_EDGES, otherwise
 * PP_ERR_INVALID_ARG is returned and nothing is enqueued.  The call
 * allocates nothing (no cudaMalloc or cudaFree).  Its first call on a device
 * looks up the array's device address with that device current; make that
 * first call outside any stream capture.  A device reset (cudaDeviceReset, or
 * anything else that replaces the device's context) invalidates that lookup:
 * the next call in the new context looks the address up again, so make it
 * outside stream capture too.  Calls share the array, which keeps
 * the last call's contents: each call clears what it needs zeroed, and calls
 * that overlap on the GPU (other streams, other host threads) race on it.
 * Results are identical to pp_sort_edges.
 */
#define PP_SORT_STATIC_MAX_EDGES (1u << 20)
pp_status pp_sort_edges_static(const uint32_t *u, const uint32_t *v, uint64_t M, uint32_t scale,
                               uint32_t *u_out, uint32_t *v_out, void *stream);

/*
 * Self-test of the bounded cross-block wait (no counterpart in the paper;
 * failure detection).  Runs one Kernel 1 scatter pass over a built-in
 * two-tile input whose first tile is never processed, so the second tile's
 * look-back polls a status word that nothing writes.  After `spin_limit`
 * empty polls (each followed by a short sleep once the count passes 64) the
 * wait gives up, PP_DEV_TIMEOUT is recorded in the device error word (read it
 * with pp_last_device_error) and the kernel returns; the context stays usable.
 * With ws == NULL the call only stores the workspace size in *bytes_needed.
 * spin_limit == 0 gives PP_ERR_INVALID_ARG.
 */
pp_status pp_selftest_lookback_timeout(uint32_t spin_limit, void *workspace, size_t workspace_bytes,
                                       size_t *bytes_needed, void *stream);

/*
 * Kernel 2 (Sec. IV-C), from Kernel 1's output (u_sorted, v_sorted; M edges
 * sorted by (u, v)):
 *   step 1  A = sparse(u,v,1,N,N)           duplicate edges become counts
 *   step 2  d_in = sum(A,1)
 *   step 3  A(:, d_in == max(d_in)) = 0     per `rule`
 *           A(:, d_in == 1) = 0             (same d_in as the line above)
 *   step 4  d_out = sum(A,2); A(i,:) = A(i,:) ./ d_out(i) for d_out(i) > 0
 * Rows with d_out = 0 stay zero: no dangling-node correction (Sec. IV-C).
 * g->scale and g->M must equal scale and M; g's arrays are overwritten.
 */
pp_status pp_build_filter_normalize_workspace(uint64_t M, uint32_t scale, size_t *bytes);
pp_status pp_build_filter_normalize(const uint32_t *u_sorted, const uint32_t *v_sorted, uint64_t M,
                                    uint32_t scale, pp_supernode_rule rule, const pp_graph *g,
                                    void *workspace, size_t workspace_bytes, void *stream);

/*
 * Kernels 1 and 2 for a batch of graphs of uneven scale (the batched
 * configuration), each stage one set of launches over every graph at once.
 * The graphs are laid side by side in one union vertex space (graph g's
 * vertex u is union vertex N_0 + ... + N_(g-1) + u), sorted and filtered
 * together, and split again; every output equals that of the single-graph
 * call on the same graph (pp_sort_edges, pp_build_filter_normalize).
 *   n_graphs     1 .. PP_BATCH_MAX_GRAPHS; sum of 2^scale[g] <= 2^27 and of
 *                M[g] <= 2^31.
 *   u, v         host arrays of n_graphs device pointers (graph g's M[g] ids).
 *   u_out, v_out host arrays of device pointers, M[g] each, not overlapping
 *                the inputs: graph g's edges sorted by (u, v).
 *   gs           host array of n_graphs graphs (device arrays inside, sized
 *                by pp_graph_lengths(gs[g].M, gs[g].scale)); graph g is built
 *                from u_sorted[g], v_sorted[g] (gs[g].M edges, ids below
 *                2^gs[g].scale).
 * An id >= N of its graph sets PP_DEV_RANGE; the outputs are then
 * unspecified.  Workspace from the matching *_workspace query.  The batch
 * tables travel as kernel parameters, so the calls can be stream-captured.
 */
pp_status pp_sort_edges_batched_workspace(uint32_t n_graphs, const uint64_t *M, const uint32_t *scale,
                                          size_t *bytes);
pp_status pp_sort_edges_batched(uint32_t n_graphs, const uint32_t *const *u, const uint32_t *const *v,
                                const uint64_t *M, const uint32_t *scale, uint32_t *const *u_out,
                                uint32_t *const *v_out, void *workspace, size_t workspace_bytes, void *stream);
pp_status pp_build_filter_normalize_batched_workspace(uint32_t n_graphs, const uint64_t *M, const uint32_t *scale,
                                                      size_t *bytes);
pp_status pp_build_filter_normalize_batched(uint32_t n_graphs, const uint32_t *const *u_sorted,
                                            const uint32_t *const *v_sorted, pp_supernode_rule rule,
                                            const pp_graph *gs, void *workspace, size_t workspace_bytes,
                                            void *stream);

/*
 * The local steps of the row-decomposed form of Kernels 1-3 (the paper's
 * parallel implementations, Sec. IV-B to IV-D: each process owns a range of
 * start vertices, i.e. of rows); the collectives between the steps are the
 * caller's.
 *
 * pp_range_counts: counts[p] = the edges of u_sorted (M start vertices in
 *   nondecreasing order) that lie in [bounds[p], bounds[p+1]), p < parts
 *   (bounds: device uint32[parts+1]; counts: device uint64[parts]) -- the
 *   split sizes of Kernel 1's exchange by start vertex range.
 * pp_in_degree: d_in[v] = number of the M edges ending in v (device
 *   uint32[2^scale], overwritten) -- the part of d_in = sum(A,1) that a
 *   share of the rows contributes (Sec. IV-C step 2); an end vertex >= N
 *   sets PP_DEV_RANGE and is skipped.
 * pp_build_filter_normalize_rows: Kernel 2 on edges that hold every edge of
 *   their start vertices (a share of the rows), with the in-degree of every
 *   column of the whole graph supplied (d_in_all, device uint32[2^scale]):
 *   the supernode and leaf filters and g->d_in use it, d_out and the matrix
 *   are this share's.  Otherwise as pp_build_filter_normalize (same
 *   workspace).
 * pp_rank_update: r[i] = a * y[i] + b for i < n (binary64 or binary32 by
 *   dtype), and *r_sum (device double) = the sum of the new r[i] in binary64
 *   (a fixed order); r may equal y.  Workspace: 2048 bytes.
 */
pp_status pp_range_counts(const uint32_t *u_sorted, uint64_t M, const uint32_t *bounds, uint32_t parts,
                          uint64_t *counts, void *stream);
pp_status pp_in_degree(const uint32_t *v, uint64_t M, uint32_t scale, uint32_t *d_in, void *stream);
pp_status pp_build_filter_normalize_rows(const uint32_t *u_sorted, const uint32_t *v_sorted, uint64_t M,
                                         uint32_t scale, pp_supernode_rule rule, const uint32_t *d_in_all,
                                         const pp_graph *g, void *workspace, size_t workspace_bytes,
                                         void *stream);
pp_status pp_rank_update(const void *y, uint64_t n, double a, double b, void *r, double *r_sum, pp_dtype dtype,
                         void *workspace, size_t workspace_bytes, void *stream);

/*
 * Kernel 2's filtered matrix A (Sec. IV-C step 4, A(i,:) = A(i,:) ./ d_out(i))
 * in compressed-row form, in vertex order: row u holds the entries of start
 * vertex u with their end vertices ascending.
 *   rowptr[N+1]  (uint64) row u is entries rowptr[u] .. rowptr[u+1]-1;
 *                rowptr[N] = nnz = g->info[PP_INFO_NNZ]
 *   col[nnz]     end vertex v of each entry
 *   cnt[nnz]     count(u,v), the number of edges from u to v (sparse(u,v,1))
 *   val64[nnz]   cnt / d_out(u), IEEE binary64 division (NULL: not written)
 *   val32[nnz]   (float)cnt / (float)d_out(u), IEEE binary32 division (NULL:
 *                not written)
 * All device arrays owned by the caller.  cap is the room (entries) in col,
 * cnt, val64 and val32; nnz <= g->M, so cap = g->M always suffices.  If nnz
 * exceeds cap, those four are left untouched, rowptr is still written and
 * PP_DEV_CAPACITY is recorded in the device error word.  The graph is only
 * read; workspace from pp_export_csr_workspace(g->M, g->scale).
 */
pp_status pp_export_csr_workspace(uint64_t M, uint32_t scale, size_t *bytes);
pp_status pp_export_csr(const pp_graph *g, uint64_t *rowptr, uint32_t *col, uint32_t *cnt, double *val64,
                        float *val32, uint64_t cap, void *workspace, size_t workspace_bytes, void *stream);

/*
 * Kernel 3 (Sec. IV-D and the appendix): from the start vector r0 (device
 * binary64[N], any positive values; the call divides by norm(r0,1) first),
 * run `iters` iterations of
 *     r(v) = c * sum_u r(u) A(u,v) + ((1-c)/N) * sum(r)
 * with A from Kernel 2.  sum(r) is reduced in binary64 for every dtype.
 * r_out receives the final r: double[N] for PP_FP64, float[N] otherwise.
 * r_l1 (nullable, double[N]) receives r / norm(r,1) in binary64.
 * The result is deterministic: the same inputs give the same bits.
 */
pp_status pp_pagerank_workspace(uint64_t M, uint32_t scale, uint32_t iters, pp_dtype dtype,
                                size_t *bytes);
pp_status pp_pagerank(const pp_graph *g, const double *r0, uint32_t iters, double c, pp_dtype dtype,
                      void *r_out, double *r_l1, void *workspace, size_t workspace_bytes,
                      void *stream);

/*
 * Kernel 3 variants the paper describes but leaves out of the benchmark
 * (Sec. IV-C and IV-D), as flags:
 *   PP_K3_DANGLING  the rows without entries (dangling nodes) pass their mass
 *                   on evenly: with D = sum of r over those rows, each
 *                   iteration is r(v) = c*(sum_u r(u) A(u,v) + D/N) +
 *                   ((1-c)/N)*sum(r), so sum(r) stays 1.
 *   PP_K3_CONVERGE  stop after the first iteration k with
 *                   norm(r_k - r_(k-1), 1) < tol (tol > 0 required), at
 *                   most `iters` iterations.
 * flags = 0 gives pp_pagerank's result up to rounding.  iters_done (device
 * uint32, may be NULL) receives the number of iterations run.  D and the
 * norms are reduced exactly (fixed point), so the stopping iteration does not
 * depend on scheduling.  Workspace from pp_pagerank_ex_workspace (larger than
 * pp_pagerank's: r itself is kept each iteration).  Other arguments and
 * errors as pp_pagerank; unknown flags give PP_ERR_INVALID_ARG.
 */
#define PP_K3_DANGLING 1u
#define PP_K3_CONVERGE 2u
pp_status pp_pagerank_ex_workspace(uint64_t M, uint32_t scale, uint32_t iters, pp_dtype dtype, size_t *bytes);
pp_status pp_pagerank_ex(const pp_graph *g, const double *r0, uint32_t iters, double c, pp_dtype dtype,
                         uint32_t flags, double tol, void *r_out, double *r_l1, uint32_t *iters_done,
                         void *workspace, size_t workspace_bytes, void *stream);

/*
 * Kernel 3 for a batch of graphs with several start vectors each (a sparse
 * matrix times dense matrix product; every (graph, vector) pair is one run of
 * the iteration above, in binary32 with sum(r) reduced exactly).
 *   gs[n_graphs]   host array of Kernel 2 outputs (device arrays inside);
 *                  1 <= n_graphs <= PP_BATCH_MAX_GRAPHS, scales 1..24.
 *   nrhs           start vectors per graph, 1 <= nrhs <= PP_BATCH_MAX_RHS.
 *   r0             device binary64, the start vectors of all graphs as one
 *                  row-major (sum of N_g) x nrhs matrix: graph g's rows come
 *                  after graph g-1's, row i holds the nrhs values of vertex i.
 *   r_out          device binary32, the final ranks in the same layout.
 * Deterministic; one persistent kernel per iteration covers every graph.
 */
#define PP_BATCH_MAX_GRAPHS 128
#define PP_BATCH_MAX_RHS 32
pp_status pp_pagerank_batched_workspace(const pp_graph *gs, uint32_t n_graphs, uint32_t nrhs, uint32_t iters,
                                        size_t *bytes);
pp_status pp_pagerank_batched(const pp_graph *gs, uint32_t n_graphs, const double *r0, uint32_t nrhs,
                              uint32_t iters, double c, float *r_out, void *workspace, size_t workspace_bytes,
                              void *stream);

/*
 * The same batched Kernel 3 captured once as a CUDA graph and replayed.
 * pp_pagerank_batched_capture records the kernels that pp_pagerank_batched
 * would enqueue with these exact arguments (stream capture on `stream`, or
 * on a private stream when stream is NULL) and instantiates them; nothing
 * runs.  pp_exec_launch replays the whole stage on `stream` with one call:
 * it reads r0 and the graphs and writes r_out at launch time, so the caller
 * may refill r0 (and rebuild the graphs in the same buffers) between
 * launches.  The buffers, the workspace and the graphs' arrays must stay
 * allocated until pp_exec_destroy; two launches of one exec must not
 * overlap.  Argument errors are those of pp_pagerank_batched and leave
 * *exec NULL.
 */
typedef struct pp_exec pp_exec;
pp_status pp_pagerank_batched_capture(const pp_graph *gs, uint32_t n_graphs, const double *r0, uint32_t nrhs,
                                      uint32_t iters, double c, float *r_out, void *workspace,
                                      size_t workspace_bytes, void *stream, pp_exec **exec);
/*
 * The whole batched pipeline recorded as one CUDA graph: Kernel 1 on every
 * graph's edges (u, v into u_sorted, v_sorted), Kernel 2 into gs, Kernel 3
 * on r0 into r_out (binary32, nrhs start vectors per graph), each stage as
 * pp_sort_edges_batched, pp_build_filter_normalize_batched and
 * pp_pagerank_batched would enqueue it.  The three stages run one after the
 * other in the same workspace (size from pp_pipeline_batched_workspace).
 * Replay with pp_exec_launch; buffers as for the three calls.
 */
pp_status pp_pipeline_batched_workspace(uint32_t n_graphs, const pp_graph *gs, uint32_t nrhs, uint32_t iters,
                                        size_t *bytes);
pp_status pp_pipeline_batched_capture(uint32_t n_graphs, const uint32_t *const *u, const uint32_t *const *v,
                                      uint32_t *const *u_sorted, uint32_t *const *v_sorted, pp_supernode_rule rule,
                                      const pp_graph *gs, const double *r0, uint32_t nrhs, uint32_t iters,
                                      double c, float *r_out, void *workspace, size_t workspace_bytes,
                                      void *stream, pp_exec **exec);
pp_status pp_exec_launch(pp_exec *exec, void *stream);
pp_status pp_exec_destroy(pp_exec *exec);

/*
 * The edge files of Kernels 0-2 (Sec. IV-A, IV-B): one edge per line, the
 * start and end vertex in decimal separated by a tab and ended by a newline,
 * "u\tv\n" (0-based ids, no signs or spaces; at most PP_TSV_MAX_LINE bytes
 * a line).  The text is formatted and parsed on the device; reading and
 * writing the files (and the host/device copies) is the caller's.
 *
 * pp_format_tsv writes the M edges (u[i], v[i]) as text[0 .. *text_len)
 * (text_len: device uint64); text_cap must be at least
 * M * PP_TSV_MAX_LINE, else PP_ERR_INVALID_ARG.
 *
 * pp_parse_tsv reads text[0 .. text_len) (device) into u[], v[] (device, room
 * for m_cap edges) and stores the number of lines in *m_out (device uint64).
 * Malformed text (a field that is not 1..10 digits or exceeds 2^32-1, not
 * exactly one tab, an empty or over-long line, no newline at the end) or more
 * than m_cap lines sets PP_DEV_PARSE in the device error word; a malformed
 * line is stored as (0, 0) and lines beyond m_cap are dropped.
 */
#define PP_TSV_MAX_LINE 22
pp_status pp_format_tsv_workspace(uint64_t M, size_t *bytes);
pp_status pp_format_tsv(const uint32_t *u, const uint32_t *v, uint64_t M, char *text, uint64_t text_cap,
                        uint64_t *text_len, void *workspace, size_t workspace_bytes, void *stream);
pp_status pp_parse_tsv_workspace(uint64_t text_len, size_t *bytes);
pp_status pp_parse_tsv(const char *text, uint64_t text_len, uint32_t *u, uint32_t *v, uint64_t m_cap,
                       uint64_t *m_out, void *workspace, size_t workspace_bytes, void *stream);

/*
 * Kernels 1-3 back to back from HOST buffers: copies u_host, v_host (M ids
 * each) and r0_host (N values) to the device, runs the three kernels, each
 * complete before the next starts, and copies the final r into r_out_host
 * (double[N] for PP_FP64, float[N] otherwise) and, if info_host is not NULL,
 * Kernel 2's scalars into info_host[PP_INFO_LEN].  Every device buffer is
 * carved from `workspace` (size from pp_pipeline_workspace).  Host buffers
 * should be page-locked for the copies to be asynchronous; the results are
 * valid after the stream has been synchronised.  The copies run on a
 * short-lived side stream (the call creates and releases it and its events
 * itself, so it cannot be recorded into a CUDA graph): with 2*scale > 32 and
 * M >= 2^20 the edge list crosses in four chunks and Kernel 1 sorts each
 * chunk as soon as it has arrived, then merges the sorted chunks (the result
 * is the sort pp_sort_edges gives); r0, which only Kernel 3 reads, is copied
 * while Kernels 1 and 2 compute.  On an error return, the copies already
 * enqueued on the side stream are ordered before later work on `stream`, so
 * the workspace may be reused on `stream` (or freed) right away.
 */
pp_status pp_pipeline_workspace(uint64_t M, uint32_t scale, uint32_t iters, pp_dtype dtype,
                                size_t *bytes);
pp_status pp_pipeline_host(const uint32_t *u_host, const uint32_t *v_host, uint64_t M, uint32_t scale,
                           const double *r0_host, uint32_t iters, double c, pp_dtype dtype,
                           pp_supernode_rule rule, void *r_out_host, uint64_t *info_host,
                           void *workspace, size_t workspace_bytes, void *stream);

/*
 * Measurement aid (no counterpart in the paper): the gather rate that bounds
 * a Kernel 3 iteration.  Reads rowc[0 .. n) once (Kernel 2's packed entries:
 * a row position in the low `scale` bits) and, for each, gathers
 * x[rowc[e] mod 2^scale] (x: device float[2^scale]) with nothing else to do
 * per entry; the sum of the gathered values is added to *out (device float,
 * caller-initialised).  Timing this call on a graph's first nnz entries gives
 * the time an iteration over those entries cannot beat with these loads.
 */
pp_status pp_gather_probe(const uint32_t *rowc, uint64_t n, uint32_t scale, const float *x, float *out,
                          void *stream);

/* Synchronise `stream`, then return and clear the device error word (a
 * PP_DEV_* bit set) of the current device in *code.  Returns PP_ERR_DEVICE if
 * the word was non-zero, PP_ERR_CUDA if synchronisation failed, else PP_OK. */
pp_status pp_last_device_error(void *stream, uint32_t *code);

/* Host-side fault injection, for testing how callers handle failures without
 * making a GPU fail: the next `count` calls of the entry point named `call`
 * (for example "pp_sort_edges"; "*" matches every entry point that enqueues
 * work, and pp_last_device_error) return `status` at once, before checking
 * their arguments, enqueueing anything or touching their outputs.  count 0
 * disarms `call`.  Up to 16 names may be armed; process-wide, thread-safe.
 * Returns PP_ERR_INVALID_ARG for a NULL or over-long name, for status PP_OK
 * or out of range with count > 0, or when the table is full. */
pp_status pp_inject_fault(const char *call, pp_status status, uint32_t count);

/* How this library was compiled: PP_BUILD_CHECKED is set in the bounds-checked
 * build (libpp_checked.so), whose kernels compare every index they read from
 * memory, or compute from what they read, with the length of the array it
 * addresses; an index out of range records PP_DEV_BOUNDS and the access goes
 * to element 0 of that array instead (no trap).  Same entry points and
 * results as libpp.so, somewhat slower.  Every call also opens an NVTX range
 * named after it unless the library was built with -DPP_NO_NVTX
 * (PP_BUILD_NVTX). */
#define PP_BUILD_CHECKED 1u
#define PP_BUILD_NVTX 2u
uint32_t pp_build_flags(void);

/* A short English description of a status code (static storage). */
const char *pp_status_string(pp_status status);

/* Number of kernels this library has enqueued in this process so far. */
uint64_t pp_launch_count(void);

/*
 * Tuning knobs (process-wide, read when a call is made).  The unroll
 * and block knobs change speed only; the thresholds also
 * change the order in which some column sums are added, so results move
 * within rounding (every setting meets the stated tolerances, and one
 * setting always gives the same bits):
 *   "k3_unroll_f32"  entries each Kernel 3 lane loads and gathers before
 *                    using any, binary32 and bfloat16 ranks: 4 or 8 (default 8)
 *   "k3_unroll_f64"  the same for binary64 ranks: 4 or 8 (default 4)
 *   "k3_minblocks"   Kernel 3 blocks per SM the registers are budgeted for:
 *                    4, 6 or 8 (default 4)
 *   "k3_shortmax"    Kernel 3 columns longer than this are cut into chunks
 *                    summed by whole warps, the others are summed one per
 *                    lane in 32-column slices: 128, 256 or 512 (default 256)
 *   "k3_chunk"       entries per chunk of a long column: 2048 or 4096 (default 4096)
 *   "k3b_shortmax"   the long-column threshold of the batched Kernel 3:
 *                    128 or 256 (default 256)
 *   "k3b_chunk"      its entries per chunk: 256, 512 or 1024 (default 512)
 *   "k3b_vec"        1: with 32 start vectors, 8 lanes of the batched Kernel
 *                    3 share an entry, 4 vectors each (4 entries per warp
 *                    step); 0: one entry per warp step, a vector per lane
 *                    (default 1).  The two sum each column in a different
 *                    (fixed) order.
 * pp_set_tuning returns PP_ERR_INVALID_ARG for an unknown key or value.
 * The autotuner (paper_1603_01876_gb300/tune.py) measures the choices and
 * stores the fastest per device and scale.
 */
pp_status pp_set_tuning(const char *key, int64_t value);
pp_status pp_get_tuning(const char *key, int64_t *value);

#ifdef __cplusplus
}
#endif

#endif /* PAGERANK_PIPELINE_H */
