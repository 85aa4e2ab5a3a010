// The pieces the row-decomposed form of Kernels 1-3 needs beside the
// single-graph kernels (Sec. IV-B to IV-D, where each process owns a range
// of rows): the edge counts per destination range of a sorted edge list
// (Kernel 1's exchange), the in-degree of an edge list (Kernel 2's partial
// column sums, added across ranks), and the update of a rank's own ranks from
// the column sums added across ranks, with the sum of the new ranks
// (Kernel 3).
#include <algorithm>

#include "pp_common.cuh"

PP_DEFINE_ERROR_WORD(kr_fetch_error)

namespace pp {
namespace kr {

constexpr int SUM_BLOCKS = 256;  // fixed, so the sum is reproducible

// counts[p] = edges of the sorted list whose start vertex lies in
// [bounds[p], bounds[p+1]) (a binary search per bound, one thread each).
__global__ void __launch_bounds__(128) range_counts_kernel(const uint32_t *us, uint64_t M, const uint32_t *bounds,
                                                           uint32_t parts, uint64_t *counts) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= parts) return;
    auto lower = [&](uint32_t key) {
        uint64_t lo = 0, hi = M;
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            if (us[mid] < key)
                lo = mid + 1;
            else
                hi = mid;
        }
        return lo;
    };
    counts[p] = lower(bounds[p + 1]) - lower(bounds[p]);
}

// d_in[v] += edges into v (one atomic per run of equal v in a thread's 16 edges).
__global__ void __launch_bounds__(256) in_degree_kernel(const uint32_t *vs, uint64_t M, uint32_t N, uint32_t *d_in) {
    constexpr int ITEMS = 16;
    for (uint64_t i0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * ITEMS; i0 < M;
         i0 += (uint64_t)gridDim.x * blockDim.x * ITEMS) {
        uint32_t cur = 0xffffffffu, run = 0;
        for (int j = 0; j < ITEMS && i0 + j < M; ++j) {
            const uint32_t v = vs[i0 + j];
            if (v >= N) {
                pp_set_error(PP_DEV_RANGE);
                continue;
            }
            if (v != cur) {
                if (run) atomicAdd(&d_in[cur], run);
                cur = v;
                run = 0;
            }
            ++run;
        }
        if (run) atomicAdd(&d_in[cur], run);
    }
}

// r[i] = a * y[i] + b for the rank's n vertices; per-block partial sums of r.
template <typename T>
__global__ void __launch_bounds__(256) update_kernel(const T *y, uint64_t n, double a, double b, T *r, double *part) {
    __shared__ double s_red[32];
    double acc = 0.0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const T v = (T)(a * (double)y[i] + b);
        r[i] = v;
        acc += (double)v;
    }
    const double bs = block_sum<double, 256>(acc, s_red);
    if (threadIdx.x == 0) part[blockIdx.x] = bs;
}

__global__ void sum_parts_kernel(const double *part, double *sum) {
    double s = 0.0;
    for (int i = 0; i < SUM_BLOCKS; ++i) s += part[i];
    *sum = s;
}

}  // namespace kr
}  // namespace pp

using namespace pp;

extern "C" pp_status pp_range_counts(const uint32_t *u_sorted, uint64_t M, const uint32_t *bounds, uint32_t parts,
                                     uint64_t *counts, void *stream) {
    PP_ENTRY("pp_range_counts");
    if (parts < 1 || !bounds || !counts || (M && !u_sorted)) return PP_ERR_INVALID_ARG;
    kr::range_counts_kernel<<<(parts + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(u_sorted, M, bounds,
                                                                                                parts, counts);
    count_launch();
    return launch_status();
}

extern "C" pp_status pp_in_degree(const uint32_t *v, uint64_t M, uint32_t scale, uint32_t *d_in, void *stream) {
    PP_ENTRY("pp_in_degree");
    if (scale < 1 || scale > 27 || !d_in || (M && !v)) return PP_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t N = 1u << scale;
    if (cudaMemsetAsync(d_in, 0, (size_t)N * sizeof(uint32_t), s) != cudaSuccess) return PP_ERR_CUDA;
    if (M) {
        const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(ceil_div(M, 256 * 16), 8ull * sm_count()));
        kr::in_degree_kernel<<<grid, 256, 0, s>>>(v, M, N, d_in);
        count_launch();
    }
    return launch_status();
}

extern "C" pp_status pp_rank_update(const void *y, uint64_t n, double a, double b, void *r, double *r_sum,
                                    pp_dtype dtype, void *workspace, size_t workspace_bytes, void *stream) {
    PP_ENTRY("pp_rank_update");
    if ((n && (!y || !r)) || !r_sum || (dtype != PP_FP64 && dtype != PP_FP32)) return PP_ERR_INVALID_ARG;
    pp_status st = check_ws(workspace, workspace_bytes, kr::SUM_BLOCKS * sizeof(double));
    if (st != PP_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *part = static_cast<double *>(workspace);
    if (dtype == PP_FP64)
        kr::update_kernel<double><<<kr::SUM_BLOCKS, 256, 0, s>>>(static_cast<const double *>(y), n, a, b,
                                                                 static_cast<double *>(r), part);
    else
        kr::update_kernel<float><<<kr::SUM_BLOCKS, 256, 0, s>>>(static_cast<const float *>(y), n, a, b,
                                                                static_cast<float *>(r), part);
    kr::sum_parts_kernel<<<1, 1, 0, s>>>(part, r_sum);
    count_launch(2);
    return launch_status();
}
