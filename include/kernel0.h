/*
 * libkernel0 — seeded synthetic inputs for the PageRank pipeline.
 *
 * Kernel 0 of the pipeline (Sec. IV-A) generates the edge list that the
 * timed kernels consume; its run time is not part of the benchmark.  This
 * library makes that input twice, on the host and on the device, bit for bit
 * the same, so that the CPU oracle and the GPU path can be fed identical data
 * without either one producing the other's input.  It also draws the random
 * start vector r = rand(1,N) of Kernel 3 (Sec. IV-D), which is an input of
 * the method, not part of it.
 *
 * Conventions: vertex ids are 0-based uint32; N = 2^scale; edges are stored
 * as two separate arrays u (start vertex) and v (end vertex).  All functions
 * return 0 on success and a negative value on a bad argument; the device
 * function returns a positive CUDA error code if the launch fails.
 */
#ifndef KERNEL0_H
#define KERNEL0_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    uint32_t key0, key1;
    uint32_t graph;
    uint32_t scale;
    uint32_t t_a, t_ab, t_abc;
    uint32_t mul[3];
    uint32_t add[3];
    uint32_t shift;
} k0_params_t;

/* Fill *p for a graph of the given scale (1..31) drawn with initiator
 * probabilities a, b, c, d (non-negative, summing to 1 within 1e-9), seed and
 * graph id (< 2^24).  Host only; touches nothing but *p. */
int k0_params_init(k0_params_t *p, uint32_t scale, uint64_t seed, uint32_t graph,
                   double a, double b, double c, double d);

/* Edges e0 .. e0+count-1 into host arrays u[count], v[count], using up to
 * nthreads host threads (nthreads <= 0: one per online core). */
int k0_gen_edges_host(const k0_params_t *p, uint64_t e0, uint64_t count, uint32_t *u,
                      uint32_t *v, int nthreads);

/* The same edges into device arrays u[count], v[count], launched on the CUDA
 * stream `stream` (a cudaStream_t; NULL = legacy default stream).  Asynchronous. */
int k0_gen_edges_device(const k0_params_t *p, uint64_t e0, uint64_t count, uint32_t *u,
                        uint32_t *v, void *stream);

/* Start values r0[i] for i < n, uniform in (0, 1), into a host array
 * (binary64).  Each (seed, graph, rhs) triple gives an independent vector. */
int k0_gen_r0_host(uint64_t seed, uint32_t graph, uint32_t rhs, uint64_t n, double *r0,
                   int nthreads);

/* Test hooks: one Philox4x32-10 block (out = philox(ctr, key)) and the
 * relabel bijection applied to x[0..n) in place. */
int k0_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
int k0_relabel_host(const k0_params_t *p, uint32_t *x, uint64_t n);

#ifdef __cplusplus
}
#endif

#endif /* KERNEL0_H */
