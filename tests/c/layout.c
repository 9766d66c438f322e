/* Prints the size and the field offsets of every struct in include/ebe.h, one
 * "name size off0 off1 ..." line per struct, so that the ctypes binding's
 * declarations can be compared with the C compiler's layout (no GPU needed). */
#include <stddef.h>
#include <stdio.h>

#include "ebe.h"


int main(void) {
    printf("ebe_mesh %zu %zu %zu %zu %zu %zu %zu\n", sizeof(ebe_mesh), offsetof(ebe_mesh, dim), offsetof(ebe_mesh, n_b),
           offsetof(ebe_mesh, n_n), offsetof(ebe_mesh, n_e), offsetof(ebe_mesh, coords), offsetof(ebe_mesh, elems));
    printf("ebe_create_opts %zu %zu %zu\n", sizeof(ebe_create_opts), offsetof(ebe_create_opts, device),
           offsetof(ebe_create_opts, patch_elems));
    printf("ebe_solve_opts %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(ebe_solve_opts), offsetof(ebe_solve_opts, rtol),
           offsetof(ebe_solve_opts, maxit), offsetof(ebe_solve_opts, precision), offsetof(ebe_solve_opts, chunk),
           offsetof(ebe_solve_opts, delta), offsetof(ebe_solve_opts, stall_updates), offsetof(ebe_solve_opts, use_graph),
           offsetof(ebe_solve_opts, race_iters));
    printf("ebe_solve_info %zu %zu %zu %zu %zu %zu %zu\n", sizeof(ebe_solve_info), offsetof(ebe_solve_info, status),
           offsetof(ebe_solve_info, iterations), offsetof(ebe_solve_info, true_residuals),
           offsetof(ebe_solve_info, rel_residual), offsetof(ebe_solve_info, r0_norm), offsetof(ebe_solve_info, solve_ms));
    printf("ebe_stats %zu %zu %zu\n", sizeof(ebe_stats), offsetof(ebe_stats, kernel_launches),
           offsetof(ebe_stats, device_error));
    printf("ebe_batch_config %zu %zu %zu %zu\n", sizeof(ebe_batch_config), offsetof(ebe_batch_config, ctas_per_sm),
           offsetof(ebe_batch_config, tile_nodes), offsetof(ebe_batch_config, barrier_ns));
    printf("ebe_batch_info %zu %zu %zu %zu %zu %zu %zu\n", sizeof(ebe_batch_info), offsetof(ebe_batch_info, loops),
           offsetof(ebe_batch_info, launches), offsetof(ebe_batch_info, n_converged), offsetof(ebe_batch_info, solve_ms),
           offsetof(ebe_batch_info, config), offsetof(ebe_batch_info, phase_ms));
    printf("ebe_partition_sizes %zu %zu %zu\n", sizeof(ebe_partition_sizes), offsetof(ebe_partition_sizes, n_patches),
           offsetof(ebe_partition_sizes, patch_elems));
    return 0;
}
