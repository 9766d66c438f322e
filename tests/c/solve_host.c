/* The whole path from C with host buffers only: the 33 x 33 unit square in
 * SW-NE triangles, nu = 1, f = 1, Dirichlet 0 on the whole boundary (the
 * small configuration), solved by Jacobi-PCG to 1e-8 in FP64 and in mixed
 * precision through ebe_create / ebe_set_problem / ebe_assemble /
 * ebe_solve_host.  Writes both solutions (raw doubles, FP64 first) to the
 * file named by argv[1] and prints one line per solve. */
#include <stdio.h>
#include <stdlib.h>

#include "ebe.h"

int main(int argc, char** argv) {
    if (argc < 2) return 2;
    const int n = 33;
    const int64_t n_n = (int64_t)n * n, n_e = 2 * (int64_t)(n - 1) * (n - 1);
    double* coords = malloc(sizeof(double) * 2 * (size_t)n_n);
    int32_t* elems = malloc(sizeof(int32_t) * 3 * (size_t)n_e);
    double* f = malloc(sizeof(double) * (size_t)n_n);
    int32_t* bnd = malloc(sizeof(int32_t) * 4 * (size_t)n);
    double* x = malloc(sizeof(double) * 2 * (size_t)n_n);
    if (!coords || !elems || !f || !bnd || !x) return 3;
    int64_t nb = 0, e = 0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            const int64_t k = (int64_t)j * n + i;
            coords[2 * k] = (double)i / (n - 1);
            coords[2 * k + 1] = (double)j / (n - 1);
            f[k] = 1.0;
            if (i == 0 || j == 0 || i == n - 1 || j == n - 1) bnd[nb++] = (int32_t)k;
        }
    for (int j = 0; j < n - 1; ++j)
        for (int i = 0; i < n - 1; ++i) {
            const int32_t a = j * n + i, b = a + 1, c = a + n, d = c + 1;   /* SW-NE diagonal a-d */
            elems[3 * e] = a; elems[3 * e + 1] = b; elems[3 * e + 2] = d; ++e;
            elems[3 * e] = a; elems[3 * e + 1] = d; elems[3 * e + 2] = c; ++e;
        }
    ebe_mesh m = {2, 3, n_n, n_e, coords, elems};
    ebe_handle* h = NULL;
    if (ebe_create(&h, &m, NULL, NULL) != EBE_OK) { fprintf(stderr, "create: %s\n", ebe_last_error(NULL)); return 4; }
    if (ebe_set_problem(h, 1.0, f, bnd, nb, NULL, NULL, 0) != EBE_OK ||
        ebe_assemble(h, EBE_STORE_MIXED) != EBE_OK) {
        fprintf(stderr, "setup: %s\n", ebe_last_error(h));
        return 5;
    }
    for (int pass = 0; pass < 2; ++pass) {
        ebe_solve_opts o;
        ebe_solve_opts_default(&o);
        o.precision = pass == 0 ? EBE_PREC_FP64 : EBE_PREC_MIXED;
        ebe_solve_info info;
        double* xp = x + pass * n_n;
        for (int64_t k = 0; k < n_n; ++k) xp[k] = 0.0;
        const ebe_status s = ebe_solve_host(h, xp, &o, &info);
        printf("%s %s %lld %.3e\n", pass == 0 ? "fp64" : "mixed", ebe_status_string(s), (long long)info.iterations,
               info.rel_residual);
        if (s != EBE_OK) { fprintf(stderr, "solve: %s\n", ebe_last_error(h)); return 6; }
    }
    ebe_destroy(h);
    FILE* out = fopen(argv[1], "wb");
    if (!out || fwrite(x, sizeof(double), 2 * (size_t)n_n, out) != 2 * (size_t)n_n) return 7;
    fclose(out);
    free(coords); free(elems); free(f); free(bnd); free(x);
    return 0;
}
