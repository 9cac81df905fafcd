/* A plain C program against the public C ABI: one context, a field from the
 * library's generator, a two-right-hand-side solve, the observables and one
 * HMC trajectory.  The CPU tests compile and link it against libhubhmc.so (it
 * needs a GPU to run).  Device buffers come from the CUDA runtime's C API. */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "hubhmc.h"

#define CHECK(call)                                                             \
    do {                                                                        \
        int rc_ = (call);                                                       \
        if (rc_ != HH_OK) {                                                     \
            fprintf(stderr, "%s: %s\n", #call, hh_strerror(rc_));               \
            return 1;                                                           \
        }                                                                       \
    } while (0)

int main(void)
{
    hh_lattice lat = {1, 32, 64};
    hh_params p;
    hh_default_params(&p);
    p.seed = 1007;
    hh_ctx *ctx = NULL;
    CHECK(hh_create(&ctx, &lat, &p, NULL));
    CHECK(hh_init_field_random(ctx, 1007));
    const long long n = hh_nsites(ctx);
    double *b = NULL, *x = NULL;
    if (cudaMalloc((void **)&b, 2 * n * sizeof(double)) != cudaSuccess) return 1;
    if (cudaMalloc((void **)&x, 2 * n * sizeof(double)) != cudaSuccess) return 1;
    double *hb = (double *)malloc(2 * n * sizeof(double));
    for (long long i = 0; i < 2 * n; ++i) hb[i] = (double)((i * 7919) % 23) - 11.0;
    cudaMemcpy(b, hb, 2 * n * sizeof(double), cudaMemcpyHostToDevice);
    hh_solve_info si;
    CHECK(hh_solve(ctx, b, x, 2, &si));
    hh_obs_info oi;
    CHECK(hh_observables(ctx, 4, 0, &oi));
    hh_traj_info ti;
    CHECK(hh_trajectory(ctx, 10, 0.1, 0, &ti));
    printf("solve: %d iterations, true relres %.2e; tr M^-1 / N = %.6f +- %.6f; dH = %.4g, accepted %d\n",
           si.iterations, si.true_relres, oi.trace_Minv, oi.trace_err, ti.dH, ti.accepted);
    free(hb);
    cudaFree(b);
    cudaFree(x);
    CHECK(hh_destroy(ctx));
    return 0;
}
