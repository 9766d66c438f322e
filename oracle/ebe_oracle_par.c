/*
 * All-core timing build of the FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * This file compiles the single-thread oracle (ebe_oracle.c, included below,
 * unchanged) together with OpenMP versions of the parts the CPU baseline
 * times: the element matrices (independent per element), the element-based
 * residual and operator of Sec. 2 (Eq. residual) and Jacobi-PCG.  It is used
 * only by the benchmark's CPU-baseline leg, to report the oracle's
 * throughput on every host core beside the single-thread checker, and by the
 * tests that compare it with the single-thread oracle.  It is not a checker:
 * the tests judge with the single-thread functions.
 *
 * The element loop of the residual runs colour by colour: a greedy colouring
 * (computed once per mesh, before any timing) puts elements that share a
 * node in different colours, so within a colour the threads add into
 * distinct nodes and need no atomics.  Only the order of the additions into
 * a node differs from the single-thread loop (by colour, then by element),
 * so results agree to rounding.  Dot products are OpenMP reductions.
 */
#include "ebe_oracle.c"

#include <omp.h>

/* Number of threads OpenMP uses here (the caller's OMP_NUM_THREADS or all cores). */
int orcp_threads(void) { return omp_get_max_threads(); }

/* Greedy colouring of the elements: colour[e] is the smallest colour not used
 * by an earlier element sharing a node.  order receives the elements grouped
 * by colour (ascending within a colour), col_ptr[c] the start of colour c;
 * returns the number of colours (< 0 if more than max_col are needed). */
int orcp_colour(int nb, int64_t n_n, int64_t n_e, const int32_t *elems, int32_t *order, int64_t *col_ptr,
                int max_col)
{
    uint64_t *used = calloc((size_t)n_n, sizeof(uint64_t));   /* colour bitmask per node (<= 64 colours) */
    int32_t *colour = malloc(sizeof(int32_t) * (size_t)(n_e > 0 ? n_e : 1));
    if (!used || !colour || max_col > 64) { free(used); free(colour); return -1; }
    int n_col = 0;
    for (int64_t e = 0; e < n_e; ++e) {
        uint64_t busy = 0;
        for (int i = 0; i < nb; ++i) busy |= used[elems[e * nb + i]];
        int c = 0;
        while (c < 64 && (busy >> c) & 1u) ++c;
        if (c >= max_col) { free(used); free(colour); return -1; }
        colour[e] = c;
        for (int i = 0; i < nb; ++i) used[elems[e * nb + i]] |= (uint64_t)1 << c;
        if (c + 1 > n_col) n_col = c + 1;
    }
    for (int c = 0; c <= n_col; ++c) col_ptr[c] = 0;
    for (int64_t e = 0; e < n_e; ++e) ++col_ptr[colour[e] + 1];
    for (int c = 0; c < n_col; ++c) col_ptr[c + 1] += col_ptr[c];
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)(n_col > 0 ? n_col : 1));
    if (!fill) { free(used); free(colour); return -1; }
    for (int c = 0; c < n_col; ++c) fill[c] = col_ptr[c];
    for (int64_t e = 0; e < n_e; ++e) order[fill[colour[e]]++] = (int32_t)e;
    free(fill); free(used); free(colour);
    return n_col;
}

/* Element matrices of Eq. matrices_K_M, the elements split across threads
 * (the single-thread function applied to contiguous element ranges). */
int orcp_element_matrices(int dim, int64_t n_n, int64_t n_e, const double *coords, const int32_t *elems,
                          double *K, double *M)
{
    const int nb = dim + 1;
    int status = ORC_OK;
#pragma omp parallel
    {
        const int t = omp_get_thread_num(), nt = omp_get_num_threads();
        const int64_t lo = n_e * t / nt, hi = n_e * (t + 1) / nt;
        int64_t bad = -1;
        const int s = orc_element_matrices(dim, n_n, hi - lo, coords, elems + lo * nb, K + lo * nb * nb,
                                           M + lo * nb * nb, NULL, &bad);
        if (s != ORC_OK) {
#pragma omp critical
            status = s;
        }
    }
    return status;
}

/* A_e = K_e + nu M_e and b_e = M_e f_e (Sec. 2), elements split across threads. */
void orcp_local_system(int nb, int64_t n_e, double nu, const double *K, const double *M, const int32_t *elems,
                       const double *f_nodal, double *A, double *be)
{
#pragma omp parallel
    {
        const int t = omp_get_thread_num(), nt = omp_get_num_threads();
        const int64_t lo = n_e * t / nt, hi = n_e * (t + 1) / nt;
        orc_local_system(nb, hi - lo, nu, K + lo * nb * nb, M + lo * nb * nb, elems + lo * nb, f_nodal,
                         A + lo * nb * nb, be ? be + lo * nb : NULL);
    }
}

/* sum_e C_e^T (sgn b_e + A_e R_e x) colour by colour (Eq. residual with
 * sgn = -1 and the sign folded in by the caller; the operator with be NULL). */
static void colour_sum(int nb, int64_t n_n, const int32_t *elems, const double *A, const double *be,
                       const double *x, const int32_t *order, const int64_t *col_ptr, int n_col, double sgn,
                       double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n_n; ++i) out[i] = 0.0;
    for (int c = 0; c < n_col; ++c) {
#pragma omp parallel for schedule(static)
        for (int64_t k = col_ptr[c]; k < col_ptr[c + 1]; ++k) {
            const int64_t e = order[k];
            const int32_t *idx = elems + e * nb;
            const double *Ae = A + (int64_t)nb * nb * e;
            double xe[4];
            for (int i = 0; i < nb; ++i) xe[i] = x[idx[i]];
            for (int i = 0; i < nb; ++i) {
                double s = 0.0;
                for (int j = 0; j < nb; ++j) s += Ae[i + nb * j] * xe[j];
                out[idx[i]] += (be ? be[e * nb + i] : 0.0) + sgn * s;
            }
        }
    }
}

/* r = mask(b - A x), element-based (Eq. residual), colour-parallel. */
void orcp_residual(int nb, int64_t n_n, const int32_t *elems, const double *A, const double *be, const double *x,
                   const int32_t *nd, int64_t n_d, const int32_t *order, const int64_t *col_ptr, int n_col,
                   double *r)
{
    colour_sum(nb, n_n, elems, A, be, x, order, col_ptr, n_col, -1.0, r);
    zero_rows(r, nd, n_d);
}

static double pdot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Jacobi-PCG as orc_pcg (Saad, Alg. 9.1; same stopping rule), each step on
 * all threads.  info = {iterations, true rel. residual, residual evals}. */
int orcp_pcg(int nb, int64_t n_n, int64_t n_e, const int32_t *elems, const double *A, const double *be,
             const int32_t *nd, int64_t n_d, const double *g, const int32_t *order, const int64_t *col_ptr,
             int n_col, double *x, double rtol, int64_t maxit, double *info)
{
    double *r = malloc(sizeof(double) * n_n), *z = malloc(sizeof(double) * n_n);
    double *p = malloc(sizeof(double) * n_n), *q = malloc(sizeof(double) * n_n);
    double *dinv = malloc(sizeof(double) * n_n), *rt = malloc(sizeof(double) * n_n);
    if (!r || !z || !p || !q || !dinv || !rt) {
        free(r); free(z); free(p); free(q); free(dinv); free(rt);
        return ORC_BAD_ARG;
    }
    set_dirichlet(x, nd, g, n_d);
    orc_jacobi_diag(nb, n_n, n_e, elems, A, dinv);
    for (int64_t i = 0; i < n_n; ++i) dinv[i] = (dinv[i] != 0.0) ? 1.0 / dinv[i] : 0.0;
    zero_rows(dinv, nd, n_d);
    orcp_residual(nb, n_n, elems, A, be, x, nd, n_d, order, col_ptr, n_col, r);
    const double r0 = sqrt(pdot(n_n, r, r));
    double rel = 1.0;
    int64_t it = 0, evals = 1;
    int status = ORC_OK;
    if (r0 == 0.0) { rel = 0.0; goto done; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n_n; ++i) { z[i] = dinv[i] * r[i]; p[i] = z[i]; }
    double rho = pdot(n_n, r, z);
    for (;;) {
        if (it >= maxit) { status = ORC_MAXIT; break; }
        colour_sum(nb, n_n, elems, A, NULL, p, order, col_ptr, n_col, 1.0, q);
        zero_rows(q, nd, n_d);
        const double pq = pdot(n_n, p, q);
        if (!(pq > 0.0) || !isfinite(pq)) { status = ORC_BREAKDOWN; break; }
        const double alpha = rho / pq;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n_n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        ++it;
        if (sqrt(pdot(n_n, r, r)) / r0 <= rtol) {
            orcp_residual(nb, n_n, elems, A, be, x, nd, n_d, order, col_ptr, n_col, rt);
            ++evals;
            rel = sqrt(pdot(n_n, rt, rt)) / r0;
            if (rel <= rtol) break;
        }
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n_n; ++i) z[i] = dinv[i] * r[i];
        const double rho_new = pdot(n_n, r, z);
        const double beta = rho_new / rho;
        rho = rho_new;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n_n; ++i) p[i] = z[i] + beta * p[i];
    }
    if (status != ORC_OK) {
        orcp_residual(nb, n_n, elems, A, be, x, nd, n_d, order, col_ptr, n_col, rt);
        ++evals;
        rel = sqrt(pdot(n_n, rt, rt)) / r0;
    }
done:
    info[0] = (double)it; info[1] = rel; info[2] = (double)evals;
    free(r); free(z); free(p); free(q); free(dinv); free(rt);
    return status;
}
