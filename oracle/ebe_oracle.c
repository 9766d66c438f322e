/*
 * FP64 CPU oracle for the element-by-element (EbE) finite-element path of
 * Marcinkowski & Valdman, "MATLAB Implementation of Element-based Solvers".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is plain, slow, single-threaded C that
 * states what the method computes, one paper passage per function.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Layout: element arrays use the paper's n_b x n_b x n_e storage (Sec. 1,
 * Fig. 2), column-major as in MATLAB, so entry (i, j) of element e sits at
 * [i + n_b*j + n_b*n_b*e]: each element's block is contiguous.
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   - the load vector uses f interpolated at the nodes: b_e = M_e f_e
 *     (Eq. matrices_K_M defines b_j as the integral of f*Phi_j);
 *   - Dirichlet rows are handled as in the Sec. 2 listings: after every
 *     residual the Dirichlet entries are set to zero, and the iterate carries
 *     the Dirichlet values g;
 *   - the first three-level Chebyshev step uses 2/(lambda_1+lambda_2) (the
 *     Richardson optimum it is said to equal), not the 2/(lambda_2-lambda_1)
 *     printed in Eq. Czebyshev3lev.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_INDEX_RANGE (-1)
#define ORC_DEGENERATE (-2)
#define ORC_BAD_ARG (-3)
#define ORC_MAXIT (1)
#define ORC_BREAKDOWN (2)

/* ------------------------------------------------------------------------ */
/* P1 basis on one simplex (Sec. 1: nodal linear elements, n_b = dim + 1).   */
/* lambda_i(x) = c_i + g_i . x with lambda_i(v_k) = delta_ik, i.e. the       */
/* columns of inv(V), V[k] = [1, v_k].  Gauss-Jordan with partial pivoting.  */
/* Returns the simplex measure |det V| / dim! in *meas, 0 when singular.     */
/* ------------------------------------------------------------------------ */
static int simplex_basis(int dim, const double *v, double *grad, double *meas)
{
    const int nb = dim + 1;
    double V[4][8];
    for (int k = 0; k < nb; ++k) {
        V[k][0] = 1.0;
        for (int d = 0; d < dim; ++d) V[k][1 + d] = v[k * dim + d];
        for (int c = 0; c < nb; ++c) V[k][nb + c] = (k == c) ? 1.0 : 0.0;
    }
    double det = 1.0;
    for (int col = 0; col < nb; ++col) {
        int piv = col;
        for (int k = col + 1; k < nb; ++k)
            if (fabs(V[k][col]) > fabs(V[piv][col])) piv = k;
        if (V[piv][col] == 0.0) { *meas = 0.0; return ORC_DEGENERATE; }
        if (piv != col) {
            for (int c = 0; c < 2 * nb; ++c) { double t = V[col][c]; V[col][c] = V[piv][c]; V[piv][c] = t; }
            det = -det;
        }
        det *= V[col][col];
        double inv = 1.0 / V[col][col];
        for (int c = 0; c < 2 * nb; ++c) V[col][c] *= inv;
        for (int k = 0; k < nb; ++k) {
            if (k == col) continue;
            double fac = V[k][col];
            if (fac != 0.0)
                for (int c = 0; c < 2 * nb; ++c) V[k][c] -= fac * V[col][c];
        }
    }
    double fact = (dim == 2) ? 2.0 : 6.0;
    *meas = fabs(det) / fact;
    /* inv(V) sits in the right half; column i of inv(V) holds (c_i, g_i). */
    for (int i = 0; i < nb; ++i)
        for (int d = 0; d < dim; ++d) grad[i * dim + d] = V[1 + d][nb + i];
    return (*meas > 0.0) ? ORC_OK : ORC_DEGENERATE;
}

/* ------------------------------------------------------------------------ */
/* Element stiffness and mass matrices, Eq. matrices_K_M restricted to one    */
/* element: K_ij = int grad Phi_i . grad Phi_j,  M_ij = int Phi_i Phi_j.     */
/* K uses the constant P1 gradients; M uses a quadrature rule exact for      */
/* quadratics (2D: the three edge midpoints, weight |T|/3; 3D: the 4-point   */
/* rule with barycentric (a,b,b,b), a = (5+3 sqrt5)/20, b = (5-sqrt5)/20,    */
/* weight |T|/4).  Output layout n_b x n_b x n_e (Fig. 2).                   */
/* ------------------------------------------------------------------------ */
int orc_element_matrices(int dim, int64_t n_n, int64_t n_e, const double *coords,
                         const int32_t *elems, double *K, double *M, double *meas,
                         int64_t *bad_element)
{
    if (dim != 2 && dim != 3) return ORC_BAD_ARG;
    const int nb = dim + 1;
    /* quadrature points in barycentric coordinates */
    double qp[4][4];
    int nq;
    if (dim == 2) {
        nq = 3;
        for (int q = 0; q < 3; ++q)
            for (int i = 0; i < 3; ++i) qp[q][i] = (i == q) ? 0.0 : 0.5;
    } else {
        nq = 4;
        double a = (5.0 + 3.0 * sqrt(5.0)) / 20.0, b = (5.0 - sqrt(5.0)) / 20.0;
        for (int q = 0; q < 4; ++q)
            for (int i = 0; i < 4; ++i) qp[q][i] = (i == q) ? a : b;
    }
    for (int64_t e = 0; e < n_e; ++e) {
        double v[4 * 3], g[4 * 3], vol;
        for (int k = 0; k < nb; ++k) {
            int32_t node = elems[e * nb + k];
            if (node < 0 || node >= n_n) { if (bad_element) *bad_element = e; return ORC_INDEX_RANGE; }
            for (int d = 0; d < dim; ++d) v[k * dim + d] = coords[(int64_t)node * dim + d];
        }
        if (simplex_basis(dim, v, g, &vol) != ORC_OK) { if (bad_element) *bad_element = e; return ORC_DEGENERATE; }
        if (meas) meas[e] = vol;
        double *Ke = K + (int64_t)nb * nb * e, *Me = M + (int64_t)nb * nb * e;
        for (int j = 0; j < nb; ++j)
            for (int i = 0; i < nb; ++i) {
                double s = 0.0;
                for (int d = 0; d < dim; ++d) s += g[i * dim + d] * g[j * dim + d];
                Ke[i + nb * j] = vol * s;
                double m = 0.0;
                for (int q = 0; q < nq; ++q) m += qp[q][i] * qp[q][j];
                Me[i + nb * j] = vol / nq * m;
            }
    }
    return ORC_OK;
}

/* Local systems of Sec. 2: A_e := K_e + nu M_e, and the local load vectors  */
/* b_e = M_e f_e with f taken at the element's nodes (reading of b_j).       */
void orc_local_system(int nb, int64_t n_e, double nu, const double *K, const double *M,
                      const int32_t *elems, const double *f_nodal, double *A, double *be)
{
    for (int64_t e = 0; e < n_e; ++e) {
        const double *Ke = K + (int64_t)nb * nb * e, *Me = M + (int64_t)nb * nb * e;
        double *Ae = A + (int64_t)nb * nb * e;
        for (int t = 0; t < nb * nb; ++t) Ae[t] = Ke[t] + nu * Me[t];
        if (be) {
            for (int i = 0; i < nb; ++i) {
                double s = 0.0;
                for (int j = 0; j < nb; ++j) s += Me[i + nb * j] * f_nodal[elems[e * nb + j]];
                be[e * nb + i] = s;
            }
        }
    }
}

/* Dirichlet condition of the Sec. 2 listings: r(nd) = 0. */
static void zero_rows(double *r, const int32_t *nd, int64_t n_d)
{
    for (int64_t k = 0; k < n_d; ++k) r[nd[k]] = 0.0;
}

/* ------------------------------------------------------------------------ */
/* The element-based residual of Sec. 2, Eq. residual,                       */
/*   r = sum_e C_e^T (b_e - A_e R_e x),  then r(nd) = 0,                     */
/* evaluated element by element in ascending element order.                 */
/* ------------------------------------------------------------------------ */
void orc_residual(int nb, int64_t n_n, int64_t n_e, const int32_t *elems, const double *A,
                  const double *be, const double *x, const int32_t *nd, int64_t n_d, double *r)
{
    memset(r, 0, sizeof(double) * (size_t)n_n);
    for (int64_t e = 0; e < n_e; ++e) {
        const int32_t *idx = elems + e * nb;
        const double *Ae = A + (int64_t)nb * nb * e;
        double xe[4], re[4];
        for (int i = 0; i < nb; ++i) xe[i] = x[idx[i]];
        for (int i = 0; i < nb; ++i) {
            double s = 0.0;
            for (int j = 0; j < nb; ++j) s += Ae[i + nb * j] * xe[j];
            re[i] = (be ? be[e * nb + i] : 0.0) - s;
        }
        for (int i = 0; i < nb; ++i) r[idx[i]] += re[i];
    }
    zero_rows(r, nd, n_d);
}

/* Operator application y = mask(sum_e C_e^T A_e C_e x): the residual's sum  */
/* with the local loads left out and the sign of the local term dropped.     */
void orc_apply(int nb, int64_t n_n, int64_t n_e, const int32_t *elems, const double *A,
               const double *x, const int32_t *nd, int64_t n_d, double *y)
{
    memset(y, 0, sizeof(double) * (size_t)n_n);
    for (int64_t e = 0; e < n_e; ++e) {
        const int32_t *idx = elems + e * nb;
        const double *Ae = A + (int64_t)nb * nb * e;
        double xe[4];
        for (int i = 0; i < nb; ++i) xe[i] = x[idx[i]];
        for (int i = 0; i < nb; ++i) {
            double s = 0.0;
            for (int j = 0; j < nb; ++j) s += Ae[i + nb * j] * xe[j];
            y[idx[i]] += s;
        }
    }
    zero_rows(y, nd, n_d);
}

/* Assembled right-hand side b = sum_e C_e^T b_e (Sec. 1, the assembly rule */
/* applied to the local load vectors).                                       */
void orc_assemble_vector(int nb, int64_t n_n, int64_t n_e, const int32_t *elems,
                         const double *be, double *b)
{
    memset(b, 0, sizeof(double) * (size_t)n_n);
    for (int64_t e = 0; e < n_e; ++e)
        for (int i = 0; i < nb; ++i) b[elems[e * nb + i]] += be[e * nb + i];
}

/* Diagonal of A without assembling A: d = sum_e C_e^T diag(A_e). */
void orc_jacobi_diag(int nb, int64_t n_n, int64_t n_e, const int32_t *elems, const double *A, double *d)
{
    memset(d, 0, sizeof(double) * (size_t)n_n);
    for (int64_t e = 0; e < n_e; ++e)
        for (int i = 0; i < nb; ++i)
            d[elems[e * nb + i]] += A[(int64_t)nb * nb * e + i + nb * i];
}

/* Dense assembly A = sum_e C_e^T A_e C_e (Sec. 1), row-major n_n x n_n.     */
/* Only for tiny meshes: it exists to check the element-based path.          */
void orc_assemble_dense(int nb, int64_t n_n, int64_t n_e, const int32_t *elems, const double *A,
                        double *dense)
{
    memset(dense, 0, sizeof(double) * (size_t)(n_n * n_n));
    for (int64_t e = 0; e < n_e; ++e) {
        const int32_t *idx = elems + e * nb;
        const double *Ae = A + (int64_t)nb * nb * e;
        for (int i = 0; i < nb; ++i)
            for (int j = 0; j < nb; ++j) dense[(int64_t)idx[i] * n_n + idx[j]] += Ae[i + nb * j];
    }
}

static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* x(nd) = g(nd): the iterate carries the Dirichlet values. */
static void set_dirichlet(double *x, const int32_t *nd, const double *g, int64_t n_d)
{
    for (int64_t k = 0; k < n_d; ++k) x[nd[k]] = g ? g[k] : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Jacobi-preconditioned conjugate gradients (Saad, Iterative Methods for     */
/* Sparse Linear Systems, Alg. 9.1) on the system of Eq. linear_system with   */
/* the Dirichlet rows removed by r(nd) = 0.  The preconditioner is           */
/* diag(A)^{-1} on free nodes, 0 on Dirichlet nodes.  Stops when the true     */
/* relative residual |mask(b - A x)| / |mask(b - A x0)| <= rtol; the true     */
/* residual is recomputed by Algorithm 1 whenever the recurrence residual     */
/* has reached rtol.  Stops with a breakdown status when p.Ap <= 0 or is not */
/* finite.  On return info = {iterations, true rel. residual, residual evals}. */
/* ------------------------------------------------------------------------ */
int orc_pcg(int nb, int64_t n_n, int64_t n_e, const int32_t *elems, const double *A,
            const double *be, const int32_t *nd, int64_t n_d, const double *g, double *x,
            double rtol, int64_t maxit, double *info)
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
    orc_residual(nb, n_n, n_e, elems, A, be, x, nd, n_d, r);
    double r0 = sqrt(dot(n_n, r, r));
    double rel = 1.0;
    int64_t it = 0, evals = 1;
    int status = ORC_OK;
    if (r0 == 0.0) { rel = 0.0; goto done; }
    for (int64_t i = 0; i < n_n; ++i) { z[i] = dinv[i] * r[i]; p[i] = z[i]; }
    double rho = dot(n_n, r, z);
    for (;;) {
        if (it >= maxit) { status = ORC_MAXIT; break; }
        orc_apply(nb, n_n, n_e, elems, A, p, nd, n_d, q);
        double pq = dot(n_n, p, q);
        if (!(pq > 0.0) || !isfinite(pq)) { status = ORC_BREAKDOWN; break; }   /* A not SPD on p, or p = 0 */
        double alpha = rho / pq;
        for (int64_t i = 0; i < n_n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        ++it;
        double rec = sqrt(dot(n_n, r, r)) / r0;
        if (rec <= rtol) {
            orc_residual(nb, n_n, n_e, elems, A, be, x, nd, n_d, rt);
            ++evals;
            rel = sqrt(dot(n_n, rt, rt)) / r0;
            if (rel <= rtol) break;
        }
        for (int64_t i = 0; i < n_n; ++i) z[i] = dinv[i] * r[i];
        double rho_new = dot(n_n, r, z);
        double beta = rho_new / rho;
        rho = rho_new;
        for (int64_t i = 0; i < n_n; ++i) p[i] = z[i] + beta * p[i];
    }
    if (status != ORC_OK) {
        orc_residual(nb, n_n, n_e, elems, A, be, x, nd, n_d, rt);
        ++evals;
        rel = sqrt(dot(n_n, rt, rt)) / r0;
    }
done:
    info[0] = (double)it; info[1] = rel; info[2] = (double)evals;
    free(r); free(z); free(p); free(q); free(dinv); free(rt);
    return status;
}

/* True relative residual of a given x: |mask(b - A x)| / |mask(b - A x0)|. */
double orc_rel_residual(int nb, int64_t n_n, int64_t n_e, const int32_t *elems, const double *A,
                        const double *be, const int32_t *nd, int64_t n_d, const double *x,
                        const double *x0)
{
    double *r = malloc(sizeof(double) * n_n);
    if (!r) return -1.0;
    orc_residual(nb, n_n, n_e, elems, A, be, x0, nd, n_d, r);
    double den = sqrt(dot(n_n, r, r));
    orc_residual(nb, n_n, n_e, elems, A, be, x, nd, n_d, r);
    double num = sqrt(dot(n_n, r, r));
    free(r);
    return den > 0.0 ? num / den : num;
}

/* ------------------------------------------------------------------------ */
/* Richardson iteration, Eq. richardson with Dirichlet rows zeroed:           */
/*   r^k = b - A x^k,  x^{k+1} = x^k + omega r^k.                             */
/* ------------------------------------------------------------------------ */
void orc_richardson(int nb, int64_t n_n, int64_t n_e, const int32_t *elems, const double *A,
                    const double *be, const int32_t *nd, int64_t n_d, double *x, int64_t iters,
                    double omega)
{
    double *r = malloc(sizeof(double) * n_n);
    if (!r) return;
    for (int64_t k = 0; k < iters; ++k) {
        orc_residual(nb, n_n, n_e, elems, A, be, x, nd, n_d, r);
        for (int64_t i = 0; i < n_n; ++i) x[i] += omega * r[i];
    }
    free(r);
}

/* Two-level cyclic Chebyshev iteration, Eq. Czebyshev2lev:                   */
/*   x^{k+1} = x^k + r^k / alpha_{k mod N},                                   */
/* with the roots alpha_k of the shifted and scaled polynomial P_N taken in   */
/* the given order (the caller passes them).                                  */
void orc_chebyshev2(int nb, int64_t n_n, int64_t n_e, const int32_t *elems, const double *A,
                    const double *be, const int32_t *nd, int64_t n_d, double *x, int64_t iters,
                    const double *alphas, int64_t N)
{
    double *r = malloc(sizeof(double) * n_n);
    if (!r) return;
    for (int64_t k = 0; k < iters; ++k) {
        orc_residual(nb, n_n, n_e, elems, A, be, x, nd, n_d, r);
        double a = alphas[k % N];
        for (int64_t i = 0; i < n_n; ++i) x[i] += r[i] / a;
    }
    free(r);
}

/* Three-level Chebyshev iteration, Eq. Czebyshev3lev with the scaling        */
/* factors C_k of Eq. recrCk (C_0 = 1, C_1 = (l1+l2)/(l2-l1),                 */
/* C_{k+1} = 2 (l1+l2)/(l2-l1) C_k - C_{k-1}):                               */
/*   x^1     = x^0 + 2/(l1+l2) r_0,                                           */
/*   x^{k+1} = x^k + C_{k-1}/C_{k+1} (x^k - x^{k-1}) + 4/(l2-l1) C_k/C_{k+1} r_k. */
/* The C_k grow geometrically; they are carried as ratios C_{k-1}/C_k to     */
/* stay finite (the recurrence divided by C_k).                               */
void orc_chebyshev3(int nb, int64_t n_n, int64_t n_e, const int32_t *elems, const double *A,
                    const double *be, const int32_t *nd, int64_t n_d, double *x, int64_t iters,
                    double l1, double l2)
{
    double *r = malloc(sizeof(double) * n_n), *xprev = malloc(sizeof(double) * n_n);
    if (!r || !xprev) { free(r); free(xprev); return; }
    if (iters <= 0) { free(r); free(xprev); return; }
    const double s = (l1 + l2) / (l2 - l1);
    orc_residual(nb, n_n, n_e, elems, A, be, x, nd, n_d, r);
    for (int64_t i = 0; i < n_n; ++i) { xprev[i] = x[i]; x[i] += 2.0 / (l1 + l2) * r[i]; }
    /* rho_k = C_{k-1}/C_k; rho_1 = C_0/C_1 = 1/s */
    double rho = 1.0 / s;
    for (int64_t k = 1; k < iters; ++k) {
        /* C_{k+1}/C_k = 2 s - C_{k-1}/C_k */
        double ratio_next = 2.0 * s - rho;               /* C_{k+1} / C_k   */
        double c_km1_over_c_kp1 = rho / ratio_next;      /* C_{k-1}/C_{k+1} */
        double c_k_over_c_kp1 = 1.0 / ratio_next;        /* C_k / C_{k+1}   */
        orc_residual(nb, n_n, n_e, elems, A, be, x, nd, n_d, r);
        for (int64_t i = 0; i < n_n; ++i) {
            double xk = x[i];
            x[i] = xk + c_km1_over_c_kp1 * (xk - xprev[i]) + 4.0 / (l2 - l1) * c_k_over_c_kp1 * r[i];
            xprev[i] = xk;
        }
        rho = c_k_over_c_kp1;                            /* C_k / C_{k+1} becomes the next C_{k-1}/C_k */
    }
    free(r); free(xprev);
}

/* Discrete L2 error sqrt(e^T M e), M = sum_e C_e^T M_e C_e, without assembly. */
double orc_mass_norm(int nb, int64_t n_e, const int32_t *elems, const double *M, const double *err)
{
    double s = 0.0;
    for (int64_t e = 0; e < n_e; ++e) {
        const int32_t *idx = elems + e * nb;
        const double *Me = M + (int64_t)nb * nb * e;
        for (int i = 0; i < nb; ++i)
            for (int j = 0; j < nb; ++j) s += err[idx[i]] * Me[i + nb * j] * err[idx[j]];
    }
    return sqrt(s);
}
