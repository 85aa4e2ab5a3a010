// Device side of libkernel0: the Kronecker edge process, one thread per edge.
#include "../../include/kernel0.h"
#include "k0_core.h"

#include <cuda_runtime.h>
#include <cstring>

static_assert(sizeof(k0_params_t) == sizeof(k0_params), "k0 parameter layouts differ");

__global__ void k0_edges_kernel(k0_params p, uint64_t e0, uint64_t count, uint32_t *__restrict__ u,
                                uint32_t *__restrict__ v) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        uint32_t a, b;
        k0_edge(&p, e0 + i, &a, &b);
        u[i] = a;
        v[i] = b;
    }
}

extern "C" int k0_gen_edges_device(const k0_params_t *p, uint64_t e0, uint64_t count, uint32_t *u,
                                   uint32_t *v, void *stream) {
    if (!p || (count && (!u || !v))) return -1;
    if (!count) return 0;
    k0_params q;
    memcpy(&q, p, sizeof q);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    uint64_t want = (count + 255) / 256;
    uint64_t cap = (uint64_t)sms * 16;
    unsigned grid = (unsigned)(want < cap ? want : cap);
    k0_edges_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(q, e0, count, u, v);
    cudaError_t err = cudaGetLastError();
    return err == cudaSuccess ? 0 : (int)err;
}
