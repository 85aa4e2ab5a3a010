/*
 * CPU oracle for the PageRank pipeline — TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * call this code.  It is a plain, single-threaded, binary64 restatement of
 * Kernels 1-3 of the PageRank Pipeline Benchmark (Dreher et al., "PageRank
 * Pipeline Benchmark: Proposal for a Holistic System Benchmark for Big-Data
 * Platforms", Sec. IV), written so that each step can be checked against the
 * paper by eye.  It shares no code with the GPU path.
 *
 * Readings of the paper taken here (each one is also pinned by a test):
 *  - Kernel 1 sorts by start vertex u; ties are ordered by end vertex v so
 *    that the sorted list is unique (the paper asks whether v should be
 *    sorted too, Sec. V).
 *  - Kernel 2 follows its four Matlab statements literally: counts summed
 *    into A, in-degree = column sums of those counts, both column filters use
 *    the same unfiltered in-degree, out-degree = row sums of the kept counts,
 *    rows with out-degree 0 stay zero (no dangling-node correction).
 *    The supernode rule is selectable: every column whose in-degree equals
 *    the maximum (the literal statement) or only the lowest-numbered one.
 *  - Kernel 3 keeps the 1/N of the teleport term: the update is
 *    r <- (c r) A + ((1-c)/N) sum(r), as in its first form and the appendix;
 *    the "simplified" form printed without the /N is read as a misprint.
 *  - The edge files (Sec. IV-A, IV-B) hold 0-based ids as decimal strings,
 *    "u\tv\n" per edge (the paper's Matlab files count from 1).
 *  - The variants (oracle_k3_pagerank_ex): the dangling-node term the paper
 *    omits spreads the mass of rows without entries evenly, scaled by c
 *    (the usual uniform correction); the convergence test is the L1 norm of
 *    the difference of consecutive iterates against an absolute tolerance.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_RULE_LOWEST 0
#define ORACLE_RULE_ALL_TIES 1

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* Neumaier's compensated sum (Neumaier 1974) of x[0..n). */
static double sum_compensated(const double *x, uint64_t n) {
    double s = 0.0, comp = 0.0;
    for (uint64_t i = 0; i < n; ++i) {
        double t = s + x[i];
        if ((s >= 0 ? s : -s) >= (x[i] >= 0 ? x[i] : -x[i]))
            comp += (s - t) + x[i];
        else
            comp += (x[i] - t) + s;
        s = t;
    }
    return s + comp;
}

static double abs_d(double x) { return x < 0 ? -x : x; }

/*
 * Kernel 1 (Sec. IV-B): sort the M edges by start vertex, so that
 * u(i-1) <= u(i) <= u(i+1); equal start vertices are ordered by end vertex.
 * The sort itself is the C library's qsort on the pair (u, v) packed into one
 * 64-bit key with u in the high half.
 */
int oracle_k1_sort(const uint32_t *u, const uint32_t *v, uint64_t M, uint32_t *u_out,
                   uint32_t *v_out) {
    if (M == 0) return 0;
    uint64_t *key = (uint64_t *)malloc(M * sizeof(uint64_t));
    if (!key) return -1;
    for (uint64_t i = 0; i < M; ++i) key[i] = ((uint64_t)u[i] << 32) | v[i];
    qsort(key, M, sizeof(uint64_t), cmp_u64);
    for (uint64_t i = 0; i < M; ++i) {
        u_out[i] = (uint32_t)(key[i] >> 32);
        v_out[i] = (uint32_t)key[i];
    }
    free(key);
    return 0;
}

/*
 * Kernel 2 (Sec. IV-C), from any edge list u, v of length M over N vertices.
 *
 *  step 1  A = sparse(u,v,1,N,N): A(u,v) = number of edges (u,v).
 *  step 2  d_in = sum(A,1): column sums of A.
 *  step 3  A(:, d_in == max(d_in)) = 0;  A(:, d_in == 1) = 0.
 *  step 4  d_out = sum(A,2);  A(i,:) = A(i,:) ./ d_out(i) for d_out(i) > 0.
 *
 * Output: the filtered, row-normalised A as compressed rows (row u holds
 * entries rowptr[u] .. rowptr[u+1]-1, columns ascending), with both the
 * integer count cnt and the normalised value val = cnt / d_out(u) of each
 * entry; the unfiltered in-degree d_in[N]; the filtered out-degree d_out[N].
 * col/cnt/val need room for M entries.
 * stats[0] = nnz of A before the filters, stats[1] = nnz after them,
 * stats[2] = max(d_in), stats[3] = number of columns attaining it,
 * stats[4] = the lowest column attaining it, stats[5] = number of supernode
 * columns zeroed by step 3's first statement under the chosen rule.
 */
int oracle_k2_filter(const uint32_t *u, const uint32_t *v, uint64_t M, uint32_t N, int rule,
                     uint64_t *rowptr, uint32_t *col, uint32_t *cnt, double *val, uint32_t *d_in,
                     uint32_t *d_out, uint64_t *stats) {
    if (N == 0) return -1;
    if (rule != ORACLE_RULE_LOWEST && rule != ORACLE_RULE_ALL_TIES) return -1;
    for (uint64_t i = 0; i < M; ++i)
        if (u[i] >= N || v[i] >= N) return -2;

    /* step 1: A(u,v) = count of (u,v); built as (u,v)-ordered triples */
    uint64_t *key = (uint64_t *)malloc((M ? M : 1) * sizeof(uint64_t));
    uint32_t *tu = (uint32_t *)malloc((M ? M : 1) * sizeof(uint32_t));
    uint32_t *tv = (uint32_t *)malloc((M ? M : 1) * sizeof(uint32_t));
    uint32_t *tc = (uint32_t *)malloc((M ? M : 1) * sizeof(uint32_t));
    unsigned char *zero_col = (unsigned char *)calloc(N, 1);
    if (!key || !tu || !tv || !tc || !zero_col) {
        free(key); free(tu); free(tv); free(tc); free(zero_col);
        return -1;
    }
    for (uint64_t i = 0; i < M; ++i) key[i] = ((uint64_t)u[i] << 32) | v[i];
    qsort(key, M, sizeof(uint64_t), cmp_u64);
    uint64_t nnz0 = 0;
    for (uint64_t i = 0; i < M; ++i) {
        if (nnz0 > 0 && key[i] == (((uint64_t)tu[nnz0 - 1] << 32) | tv[nnz0 - 1])) {
            tc[nnz0 - 1] += 1;
        } else {
            tu[nnz0] = (uint32_t)(key[i] >> 32);
            tv[nnz0] = (uint32_t)key[i];
            tc[nnz0] = 1;
            nnz0++;
        }
    }
    free(key);

    /* step 2: d_in = sum(A,1), the sum of each column */
    memset(d_in, 0, (size_t)N * sizeof(uint32_t));
    for (uint64_t e = 0; e < nnz0; ++e) d_in[tv[e]] += tc[e];

    /* step 3: zero the supernode column(s), then the leaf columns, both
       chosen from the d_in of step 2 */
    uint32_t dmax = 0;
    for (uint32_t j = 0; j < N; ++j)
        if (d_in[j] > dmax) dmax = d_in[j];
    uint64_t ties = 0, supernodes = 0;
    uint32_t lowest = N;
    for (uint32_t j = 0; j < N; ++j) {
        if (d_in[j] == dmax) {
            ties++;
            if (lowest == N) lowest = j;
        }
    }
    for (uint32_t j = 0; j < N; ++j) {
        int is_max = d_in[j] == dmax && (rule == ORACLE_RULE_ALL_TIES || j == lowest);
        if (is_max) supernodes++;
        if (is_max || d_in[j] == 1) zero_col[j] = 1;
    }

    /* step 4: d_out = sum(A,2) over what is left; divide each row by it */
    memset(d_out, 0, (size_t)N * sizeof(uint32_t));
    for (uint64_t e = 0; e < nnz0; ++e)
        if (!zero_col[tv[e]]) d_out[tu[e]] += tc[e];
    memset(rowptr, 0, ((size_t)N + 1) * sizeof(uint64_t));
    uint64_t nnz = 0;
    for (uint64_t e = 0; e < nnz0; ++e) {
        if (zero_col[tv[e]]) continue;
        col[nnz] = tv[e];
        cnt[nnz] = tc[e];
        val[nnz] = (double)tc[e] / (double)d_out[tu[e]];
        rowptr[tu[e] + 1]++;
        nnz++;
    }
    for (uint32_t i = 0; i < N; ++i) rowptr[i + 1] += rowptr[i];

    stats[0] = nnz0;
    stats[1] = nnz;
    stats[2] = dmax;
    stats[3] = ties;
    stats[4] = lowest;
    stats[5] = supernodes;
    free(tu); free(tv); free(tc); free(zero_col);
    return 0;
}

/*
 * Kernel 3 (Sec. IV-D and the appendix).
 *
 *   r = rand(1,N)                     -> given as r0 (an input)
 *   r = r ./ norm(r,1)
 *   a = ones(1,N) .* (1-c) ./ N
 *   repeat `iters` times:  r = ((c .* r) * A) + (a .* sum(r,2))
 *
 * r is a row vector, so (r A)(v) = sum over u of r(u) A(u,v); A is the
 * normalised matrix of Kernel 2 given by rows (rowptr, col, val).
 * sums, if not NULL, receives sum(r) before iteration 1 .. iters and, in
 * sums[iters], the sum of the returned vector.
 */
int oracle_k3_pagerank(uint32_t N, const uint64_t *rowptr, const uint32_t *col, const double *val,
                       const double *r0, uint32_t iters, double c, double *r_out, double *sums) {
    if (N == 0) return -1;
    double *r = r_out;
    double *y = (double *)malloc((size_t)N * sizeof(double));
    double *absr = (double *)malloc((size_t)N * sizeof(double));
    if (!y || !absr) {
        free(y); free(absr);
        return -1;
    }
    for (uint32_t i = 0; i < N; ++i) absr[i] = abs_d(r0[i]);
    double norm1 = sum_compensated(absr, N);
    for (uint32_t i = 0; i < N; ++i) r[i] = r0[i] / norm1;
    free(absr);

    double a = (1.0 - c) / (double)N;
    for (uint32_t it = 0; it < iters; ++it) {
        double s = sum_compensated(r, N);
        if (sums) sums[it] = s;
        memset(y, 0, (size_t)N * sizeof(double));
        for (uint32_t uu = 0; uu < N; ++uu) {
            double cr = c * r[uu];
            for (uint64_t e = rowptr[uu]; e < rowptr[uu + 1]; ++e) y[col[e]] += cr * val[e];
        }
        for (uint32_t vv = 0; vv < N; ++vv) r[vv] = y[vv] + a * s;
    }
    if (sums) sums[iters] = sum_compensated(r, N);
    free(y);
    return 0;
}

/* Kernel 3 variants beyond the paper's fixed iteration count (Sec. IV-D):
 *   dangling != 0  the mass of the rows without entries (the dangling nodes
 *                  Sec. IV-C and IV-D leave out) is spread evenly over all
 *                  vertices: with D = sum of r over those rows,
 *                  r' = c*(r*A) + c*D/N + (1-c)*sum(r)/N;
 *   tol > 0        stop after the first iteration k with
 *                  norm(r_k - r_(k-1), 1) < tol (the convergence test Sec.
 *                  IV-D describes), running at most `iters` iterations.
 * With dangling == 0 and tol <= 0 this is oracle_k3_pagerank.  *iters_done
 * receives the number of iterations run. */
int oracle_k3_pagerank_ex(uint32_t N, const uint64_t *rowptr, const uint32_t *col, const double *val,
                          const double *r0, uint32_t iters, double c, int dangling, double tol, double *r_out,
                          uint32_t *iters_done) {
    if (N == 0 || !iters_done) return -1;
    double *r = r_out;
    double *y = (double *)malloc((size_t)N * sizeof(double));
    double *tmp = (double *)malloc((size_t)N * sizeof(double));
    if (!y || !tmp) {
        free(y); free(tmp);
        return -1;
    }
    for (uint32_t i = 0; i < N; ++i) tmp[i] = abs_d(r0[i]);
    double norm1 = sum_compensated(tmp, N);
    for (uint32_t i = 0; i < N; ++i) r[i] = r0[i] / norm1;

    double a = (1.0 - c) / (double)N;
    uint32_t done = iters;
    for (uint32_t it = 0; it < iters; ++it) {
        double s = sum_compensated(r, N);
        double dmass = 0.0;
        if (dangling) {
            uint32_t n = 0;
            for (uint32_t uu = 0; uu < N; ++uu)
                if (rowptr[uu] == rowptr[uu + 1]) tmp[n++] = r[uu];
            dmass = sum_compensated(tmp, n);
        }
        memset(y, 0, (size_t)N * sizeof(double));
        for (uint32_t uu = 0; uu < N; ++uu) {
            double cr = c * r[uu];
            for (uint64_t e = rowptr[uu]; e < rowptr[uu + 1]; ++e) y[col[e]] += cr * val[e];
        }
        double spread = c * dmass / (double)N;
        for (uint32_t vv = 0; vv < N; ++vv) {
            double rn = y[vv] + spread + a * s;
            tmp[vv] = abs_d(rn - r[vv]);
            r[vv] = rn;
        }
        if (tol > 0.0 && sum_compensated(tmp, N) < tol) {
            done = it + 1;
            break;
        }
    }
    *iters_done = done;
    free(y);
    free(tmp);
    return 0;
}

/* The edge files of Kernels 0-2 (Sec. IV-A, IV-B): one edge per line, start
 * and end vertex in decimal separated by a tab, "u\tv\n".  Formats M edges
 * into out (room for cap bytes); returns the length, or -1 if out is too
 * small. */
int64_t oracle_format_tsv(const uint32_t *u, const uint32_t *v, uint64_t M, char *out, uint64_t cap) {
    uint64_t n = 0;
    char line[32];
    for (uint64_t i = 0; i < M; ++i) {
        int k = snprintf(line, sizeof line, "%u\t%u\n", (unsigned)u[i], (unsigned)v[i]);
        if (k < 0 || n + (uint64_t)k > cap) return -1;
        memcpy(out + n, line, (size_t)k);
        n += (uint64_t)k;
    }
    return (int64_t)n;
}

/* One field: 1 to 10 decimal digits, value below 2^32. */
static int parse_field(const char *p, const char *end, uint32_t *out) {
    uint64_t x = 0;
    if (p == end || end - p > 10) return 0;
    for (; p < end; ++p) {
        if (*p < '0' || *p > '9') return 0;
        x = x * 10 + (uint64_t)(*p - '0');
    }
    if (x > 0xffffffffull) return 0;
    *out = (uint32_t)x;
    return 1;
}

/* Parses text[0 .. len) line by line.  Stores at most cap edges, the number
 * of lines in *m, and 1 in *bad if any line is malformed (not "digits\tdigits",
 * a field of more than 10 digits or above 2^32-1, longer than 22 bytes), if
 * the text does not end with a newline, or if there are more than cap lines;
 * a malformed line is stored as (0, 0). */
int oracle_parse_tsv(const char *text, uint64_t len, uint32_t *u, uint32_t *v, uint64_t cap, uint64_t *m, int *bad) {
    uint64_t line = 0, start = 0;
    *bad = 0;
    for (uint64_t i = 0; i < len; ++i) {
        if (text[i] != '\n') continue;
        const char *s = text + start, *e = text + i;
        const char *tab = memchr(s, '\t', (size_t)(e - s));
        uint32_t a = 0, b = 0;
        int ok = tab != NULL && (e - s) + 1 <= 22 && memchr(tab + 1, '\t', (size_t)(e - tab - 1)) == NULL &&
                 parse_field(s, tab, &a) && parse_field(tab + 1, e, &b);
        if (!ok) {
            *bad = 1;
            a = b = 0;
        }
        if (line < cap) {
            u[line] = a;
            v[line] = b;
        }
        ++line;
        start = i + 1;
    }
    if (start != len) *bad = 1; /* text after the last newline */
    if (line > cap) *bad = 1;
    *m = line;
    return 0;
}
