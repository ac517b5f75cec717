/*
 * FP64 CPU oracle for S^3TTVc on the blowup tensor -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this file's library.  It shares no code, header or table with the
 * CUDA path.
 *
 * It evaluates Algorithm 2 (AAY, Sec. II-A) exactly as stated: for every node
 * v and every edge e that contains v,
 *
 *     y_v += w(e)/|beta(e)| * (N-1)! * ( E_N(x_v) * conv_{u in e minus v} Ebar_N(x_u) )[N-1]
 *
 * with E_N(c) = [1, c, c^2/2!, ..., c^(N-1)/(N-1)!], Ebar_N(c) the same list
 * with slot 0 set to 0, and (a*b)[k] = sum_{i<=k} a_i b_{k-i} truncated to
 * k < N.  The factor w(e)/|beta(e)| * (N-1)! for each edge size s is passed in
 * as ``scale[s]`` (the caller computes it from exact integers).  Every
 * convolution is the plain O(N^2) double loop; nothing is shared between
 * pairs (e, v).  The only parallelism is an optional split of the node loop
 * over OpenMP threads, which leaves every node's own summation order intact.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* E_N(c) (bar = 0) or Ebar_N(c) (bar = 1). */
static void egf_list(double c, int N, int bar, double *out)
{
    double t = 1.0;
    out[0] = bar ? 0.0 : 1.0;
    for (int k = 1; k < N; ++k) {
        t = t * c / (double)k;
        out[k] = t;
    }
}

/* out = (a * b) truncated to N entries; out may not alias a or b. */
static void conv_trunc(const double *a, const double *b, int N, double *out)
{
    for (int k = 0; k < N; ++k) {
        double acc = 0.0;
        for (int i = 0; i <= k; ++i)
            acc += a[i] * b[k - i];
        out[k] = acc;
    }
}

/* One node: Algorithm 2's inner loop over the edges that contain v. */
static double node_value(int64_t v, const int64_t *inc_ptr, const int64_t *inc_edge,
                         const int64_t *edge_ptr, const int32_t *members, int N,
                         const double *scale, const double *x,
                         double *coefs, double *tmp, double *bar)
{
    double c = 0.0;
    for (int64_t k = inc_ptr[v]; k < inc_ptr[v + 1]; ++k) {
        int64_t e = inc_edge[k];
        int64_t b = edge_ptr[e], t = edge_ptr[e + 1];
        int s = (int)(t - b);
        egf_list(x[v], N, 0, coefs);
        for (int64_t j = b; j < t; ++j) {
            int64_t u = members[j];
            if (u == v)
                continue;
            egf_list(x[u], N, 1, bar);
            conv_trunc(coefs, bar, N, tmp);
            memcpy(coefs, tmp, sizeof(double) * (size_t)N);
        }
        c += scale[s] * coefs[N - 1];
    }
    return c;
}

/*
 * y_out[i] = [B x^(N-1)]_{nodes[i]} for i < count (nodes == NULL: all n nodes,
 * count ignored).  Returns 0 on success, 1 on bad input, 2 on allocation
 * failure.  nthreads <= 0 uses the OpenMP default.
 */
int s3o_ttsv1(int64_t n, int64_t m, const int64_t *edge_ptr, const int32_t *members,
              int N, const double *scale, const double *x, const int64_t *nodes,
              int64_t count, double *y_out, int nthreads)
{
    if (n < 0 || m < 0 || N < 1)
        return 1;
    int64_t nnz = edge_ptr[m];
    for (int64_t j = 0; j < nnz; ++j)
        if (members[j] < 0 || members[j] >= n)
            return 1;
    for (int64_t e = 0; e < m; ++e)
        if (edge_ptr[e + 1] - edge_ptr[e] > N)
            return 1;
    /* node -> edges incidence by counting sort */
    int64_t *inc_ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *inc_edge = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!inc_ptr || !inc_edge || !fill) {
        free(inc_ptr); free(inc_edge); free(fill);
        return 2;
    }
    for (int64_t j = 0; j < nnz; ++j)
        inc_ptr[members[j] + 1]++;
    for (int64_t v = 0; v < n; ++v)
        inc_ptr[v + 1] += inc_ptr[v];
    memcpy(fill, inc_ptr, sizeof(int64_t) * (size_t)n);
    for (int64_t e = 0; e < m; ++e)
        for (int64_t j = edge_ptr[e]; j < edge_ptr[e + 1]; ++j)
            inc_edge[fill[members[j]]++] = e;
    free(fill);

    int64_t total = nodes ? count : n;
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double *work = (double *)malloc(sizeof(double) * 3 * (size_t)N);
        if (!work) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            err = 2;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
            for (int64_t i = 0; i < total; ++i) {
                int64_t v = nodes ? nodes[i] : i;
                if (v < 0 || v >= n) {
                    y_out[i] = 0.0;
                    continue;
                }
                y_out[i] = node_value(v, inc_ptr, inc_edge, edge_ptr, members, N, scale, x,
                                      work, work + N, work + 2 * N);
            }
            free(work);
        }
    }
    free(inc_ptr);
    free(inc_edge);
    return err;
}

/* Number of threads an OpenMP parallel region would use (1 without OpenMP). */
int s3o_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
