/* Host side of libkernel0: parameter set-up and the threaded host generator. */
#include "../../include/kernel0.h"
#include "k0_core.h"

#include <math.h>
#include <pthread.h>
#include <string.h>
#include <unistd.h>

_Static_assert(sizeof(k0_params_t) == sizeof(k0_params), "k0 parameter layouts differ");

static uint32_t k0_threshold(double cum) {
    double t = floor(cum * 4294967296.0);
    if (t < 0.0) t = 0.0;
    if (t > 4294967295.0) t = 4294967295.0;
    return (uint32_t)t;
}

int k0_params_init(k0_params_t *out, uint32_t scale, uint64_t seed, uint32_t graph,
                   double a, double b, double c, double d) {
    if (!out || scale < 1 || scale > 31 || graph >= (1u << 24)) return -1;
    if (!(a >= 0 && b >= 0 && c >= 0 && d >= 0)) return -1;
    if (fabs(a + b + c + d - 1.0) > 1e-9) return -1;
    k0_params p;
    memset(&p, 0, sizeof p);
    p.key0 = (uint32_t)seed;
    p.key1 = (uint32_t)(seed >> 32);
    p.graph = graph;
    p.scale = scale;
    p.t_a = k0_threshold(a);
    p.t_ab = k0_threshold(a + b);
    p.t_abc = k0_threshold(a + b + c);
    uint32_t c3 = (K0_PURPOSE_RELABEL << 24) | graph;
    k0_u32x4 w0 = k0_philox4x32_10(0, 0, 0, c3, p.key0, p.key1);
    k0_u32x4 w1 = k0_philox4x32_10(1, 0, 0, c3, p.key0, p.key1);
    p.mul[0] = w0.x[0] | 1u;
    p.add[0] = w0.x[1];
    p.mul[1] = w0.x[2] | 1u;
    p.add[1] = w0.x[3];
    p.mul[2] = w1.x[0] | 1u;
    p.add[2] = w1.x[1];
    p.shift = (scale + 1) / 2;
    if (p.shift < 1) p.shift = 1;
    memcpy(out, &p, sizeof p);
    return 0;
}

typedef struct {
    const k0_params *p;
    uint64_t e0, count;
    uint32_t *u, *v;
    uint64_t seed;
    uint32_t graph, rhs;
    double *r0;
} k0_job;

static void *k0_edges_worker(void *arg) {
    k0_job *j = (k0_job *)arg;
    for (uint64_t i = 0; i < j->count; ++i) k0_edge(j->p, j->e0 + i, &j->u[i], &j->v[i]);
    return NULL;
}

static void *k0_r0_worker(void *arg) {
    k0_job *j = (k0_job *)arg;
    uint32_t key0 = (uint32_t)j->seed, key1 = (uint32_t)(j->seed >> 32);
    for (uint64_t i = 0; i < j->count; ++i)
        j->r0[i] = k0_r0_value(key0, key1, j->graph, j->rhs, j->e0 + i);
    return NULL;
}

static int k0_threads(int nthreads, uint64_t work) {
    if (nthreads <= 0) {
        long n = sysconf(_SC_NPROCESSORS_ONLN);
        nthreads = n > 0 ? (int)n : 1;
    }
    if (nthreads > 256) nthreads = 256;
    if ((uint64_t)nthreads > work / 65536 + 1) nthreads = (int)(work / 65536 + 1);
    return nthreads;
}

static int k0_run(k0_job *base, uint64_t count, int nthreads, void *(*fn)(void *), int is_r0) {
    int nt = k0_threads(nthreads, count);
    pthread_t tid[256];
    k0_job jobs[256];
    uint64_t per = (count + (uint64_t)nt - 1) / (uint64_t)nt;
    int started = 0;
    for (int t = 0; t < nt; ++t) {
        uint64_t lo = (uint64_t)t * per;
        if (lo >= count) break;
        uint64_t hi = lo + per < count ? lo + per : count;
        jobs[t] = *base;
        jobs[t].e0 = base->e0 + lo;
        jobs[t].count = hi - lo;
        if (is_r0) {
            jobs[t].r0 = base->r0 + lo;
        } else {
            jobs[t].u = base->u + lo;
            jobs[t].v = base->v + lo;
        }
        if (nt == 1) {
            fn(&jobs[t]);
            continue;
        }
        if (pthread_create(&tid[t], NULL, fn, &jobs[t]) != 0) {
            fn(&jobs[t]); /* fall back to running the slice inline */
            tid[t] = 0;
        }
        started = t + 1;
    }
    for (int t = 0; t < started; ++t)
        if (tid[t]) pthread_join(tid[t], NULL);
    return 0;
}

int k0_gen_edges_host(const k0_params_t *p, uint64_t e0, uint64_t count, uint32_t *u,
                      uint32_t *v, int nthreads) {
    if (!p || (count && (!u || !v))) return -1;
    if (!count) return 0;
    k0_job job;
    memset(&job, 0, sizeof job);
    job.p = (const k0_params *)p;
    job.e0 = e0;
    job.u = u;
    job.v = v;
    return k0_run(&job, count, nthreads, k0_edges_worker, 0);
}

int k0_gen_r0_host(uint64_t seed, uint32_t graph, uint32_t rhs, uint64_t n, double *r0,
                   int nthreads) {
    if ((n && !r0) || graph >= (1u << 24)) return -1;
    if (!n) return 0;
    k0_job job;
    memset(&job, 0, sizeof job);
    job.seed = seed;
    job.graph = graph;
    job.rhs = rhs;
    job.r0 = r0;
    job.e0 = 0;
    return k0_run(&job, n, nthreads, k0_r0_worker, 1);
}

int k0_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    if (!ctr || !key || !out) return -1;
    k0_u32x4 w = k0_philox4x32_10(ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1]);
    for (int i = 0; i < 4; ++i) out[i] = w.x[i];
    return 0;
}

int k0_relabel_host(const k0_params_t *p, uint32_t *x, uint64_t n) {
    if (!p || (n && !x)) return -1;
    for (uint64_t i = 0; i < n; ++i) x[i] = k0_relabel((const k0_params *)p, x[i]);
    return 0;
}
