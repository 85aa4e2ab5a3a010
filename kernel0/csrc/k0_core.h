/*
 * Kernel 0 core: the seeded Kronecker (Graph500-shaped) edge process and the
 * rank-vector start values, written once and compiled by both the host (C)
 * and the device (CUDA) generator so that the two produce identical bits.
 *
 * Kernel 0 is the untimed graph generator of the pipeline (Sec. IV-A): S is
 * the scale factor, N = 2^S vertices, M = k*N edges with k = 16; each edge is
 * a (start, end) pair stored in the M-element vectors u and v.  The paper
 * names the Graph500 generator but prints no code for it; what is built here
 * is a generator of the same shape (see kernel0/__init__.py for the recipe):
 *
 *   per edge e, per bit level l = 0..S-1, one 32-bit uniform draw w_l picks a
 *   quadrant of the 2x2 initiator [[A, B], [C, D]] by comparing w_l with the
 *   integer thresholds floor(A*2^32), floor((A+B)*2^32), floor((A+B+C)*2^32);
 *   the quadrant's (row, column) bits become bit l of u and of v.  Both ids
 *   then pass through one seeded bijection of [0, 2^S) so that vertex labels
 *   carry no locality.
 *
 * Random bits come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11), implemented here
 * from that paper's definition: 10 rounds of two 32x32->64 multiplications
 * with multipliers 0xD2511F53 / 0xCD9E8D57 and a Weyl key schedule with
 * increments 0x9E3779B9 / 0xBB67AE85.
 *
 * Only integer arithmetic appears in the edge process, so host and device
 * agree bit for bit.
 */
#ifndef K0_CORE_H
#define K0_CORE_H

#include <stdint.h>

#ifdef __CUDACC__
#define K0_HD __host__ __device__ __forceinline__
#else
#define K0_HD static inline
#endif

/* Counter word 3 carries a purpose tag (high 8 bits) and the graph id (low 24). */
#define K0_PURPOSE_EDGE 1u
#define K0_PURPOSE_RELABEL 2u
#define K0_PURPOSE_R0 3u

typedef struct {
    uint32_t x[4];
} k0_u32x4;

K0_HD k0_u32x4 k0_philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                uint32_t k0, uint32_t k1) {
    k0_u32x4 r;
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    r.x[0] = c0;
    r.x[1] = c1;
    r.x[2] = c2;
    r.x[3] = c3;
    return r;
}

/* Everything a generator launch needs; filled on the host by k0_params_init. */
typedef struct {
    uint32_t key0, key1;   /* Philox key = the 64-bit seed */
    uint32_t graph;        /* graph id (< 2^24), separates the graphs of a batch */
    uint32_t scale;        /* S, 1..31 */
    uint32_t t_a, t_ab, t_abc; /* cumulative initiator thresholds in units of 2^-32 */
    uint32_t mul[3];       /* odd multipliers of the relabel bijection */
    uint32_t add[3];       /* additive constants of the relabel bijection */
    uint32_t shift;        /* xorshift distance of the relabel bijection */
} k0_params;

/* Seeded bijection of [0, 2^S): affine maps with odd multipliers and
 * right-xorshifts, each of which is invertible modulo 2^S. */
K0_HD uint32_t k0_relabel(const k0_params *p, uint32_t x) {
    uint32_t mask = p->scale >= 32 ? 0xffffffffu : ((1u << p->scale) - 1u);
    x = (x * p->mul[0] + p->add[0]) & mask;
    x ^= x >> p->shift;
    x = (x * p->mul[1] + p->add[1]) & mask;
    x ^= x >> p->shift;
    x = (x * p->mul[2] + p->add[2]) & mask;
    return x;
}

/* Edge e of the graph: S quadrant choices, then the relabel. */
K0_HD void k0_edge(const k0_params *p, uint64_t e, uint32_t *u_out, uint32_t *v_out) {
    uint32_t u = 0, v = 0;
    uint32_t c0 = (uint32_t)e, c1 = (uint32_t)(e >> 32);
    uint32_t c3 = (K0_PURPOSE_EDGE << 24) | (p->graph & 0xffffffu);
    for (uint32_t blk = 0; blk * 4 < p->scale; ++blk) {
        k0_u32x4 w = k0_philox4x32_10(c0, c1, blk, c3, p->key0, p->key1);
        for (uint32_t j = 0; j < 4; ++j) {
            uint32_t level = blk * 4 + j;
            if (level >= p->scale) break;
            uint32_t x = w.x[j];
            uint32_t ib, jb;
            if (x < p->t_a) {
                ib = 0; jb = 0;          /* A: top-left */
            } else if (x < p->t_ab) {
                ib = 0; jb = 1;          /* B: top-right */
            } else if (x < p->t_abc) {
                ib = 1; jb = 0;          /* C: bottom-left */
            } else {
                ib = 1; jb = 1;          /* D: bottom-right */
            }
            u |= ib << level;
            v |= jb << level;
        }
    }
    *u_out = k0_relabel(p, u);
    *v_out = k0_relabel(p, v);
}

/* Start value i of rank vector `rhs` of graph `graph`: a uniform draw in
 * (0, 1) built from 52 random bits as (x + 1/2) * 2^-52, exact in binary64. */
K0_HD double k0_r0_value(uint32_t key0, uint32_t key1, uint32_t graph, uint32_t rhs,
                         uint64_t i) {
    k0_u32x4 w = k0_philox4x32_10((uint32_t)i, (uint32_t)(i >> 32), rhs,
                                  (K0_PURPOSE_R0 << 24) | (graph & 0xffffffu), key0, key1);
    uint64_t x = ((uint64_t)(w.x[0] >> 12) << 32) | (uint64_t)w.x[1]; /* 20 + 32 bits */
    return ((double)x + 0.5) * (1.0 / 4503599627370496.0);             /* 2^-52 */
}

#endif /* K0_CORE_H */
