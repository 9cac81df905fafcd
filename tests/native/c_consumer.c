/* A plain C program against the public C ABI: one context, a field from the
 * library's generator, a two-right-hand-side solve, a Q apply of both
 * right-hand sides in one call, the observables and one HMC trajectory (5
 * leapfrog steps of dt = 0.04, a stable step on this hot field).
 * Device buffers come from the CUDA runtime's C API.  The CPU tests compile
 * and link it; the GPU tests run it with an output path and check what it
 * writes there against the oracle: N (int64), then doubles: the initial field
 * (N), the right-hand sides b (2N), the solutions x (2N), Q b (2N), the
 * trajectory's H0, H1, dH, u and accept flag (5), and the final field (N). */
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

static int dump(FILE *f, const double *d, long long n)
{
    return fwrite(d, sizeof(double), (size_t)n, f) == (size_t)n ? 0 : 1;
}

int main(int argc, char **argv)
{
    hh_lattice lat = {1, 32, 64};
    hh_params p;
    hh_default_params(&p);
    p.seed = 1007;
    hh_ctx *ctx = NULL;
    CHECK(hh_create(&ctx, &lat, &p, NULL));
    CHECK(hh_init_field_random(ctx, 1007));
    const long long n = hh_nsites(ctx);
    double *b = NULL, *x = NULL, *qb = NULL;
    if (cudaMalloc((void **)&b, 2 * n * sizeof(double)) != cudaSuccess) return 1;
    if (cudaMalloc((void **)&x, 2 * n * sizeof(double)) != cudaSuccess) return 1;
    if (cudaMalloc((void **)&qb, 2 * n * sizeof(double)) != cudaSuccess) return 1;
    double *hb = (double *)malloc(2 * n * sizeof(double));
    double *hx = (double *)malloc(2 * n * sizeof(double));
    double *hq = (double *)malloc(2 * n * sizeof(double));
    double *s0 = (double *)malloc(n * sizeof(double));
    double *s1 = (double *)malloc(n * sizeof(double));
    if (!hb || !hx || !hq || !s0 || !s1) return 1;
    for (long long i = 0; i < 2 * n; ++i) hb[i] = (double)((i * 7919) % 23) - 11.0;
    cudaMemcpy(b, hb, 2 * n * sizeof(double), cudaMemcpyHostToDevice);
    CHECK(hh_get_field(ctx, s0, 0));
    hh_solve_info si;
    CHECK(hh_solve(ctx, b, x, 2, &si));
    CHECK(hh_apply_multi(ctx, HH_OP_MTM, b, qb, 2, HH_DTYPE_F64));
    cudaMemcpy(hx, x, 2 * n * sizeof(double), cudaMemcpyDeviceToHost);
    cudaMemcpy(hq, qb, 2 * n * sizeof(double), cudaMemcpyDeviceToHost);
    hh_obs_info oi;
    CHECK(hh_observables(ctx, 4, 0, &oi));
    hh_traj_info ti;
    CHECK(hh_trajectory(ctx, 5, 0.04, 0, &ti));
    CHECK(hh_get_field(ctx, s1, 0));
    printf("solve: %d iterations, true relres %.2e; tr M^-1 / N = %.6f +- %.6f; dH = %.4g, accepted %d\n",
           si.iterations, si.true_relres, oi.trace_Minv, oi.trace_err, ti.dH, ti.accepted);
    if (argc > 1) {
        FILE *f = fopen(argv[1], "wb");
        if (!f) return 1;
        const double tr[5] = {ti.H0, ti.H1, ti.dH, ti.u, (double)ti.accepted};
        int bad = fwrite(&n, sizeof(n), 1, f) != 1;
        bad |= dump(f, s0, n) | dump(f, hb, 2 * n) | dump(f, hx, 2 * n) | dump(f, hq, 2 * n) | dump(f, tr, 5) |
               dump(f, s1, n);
        if (fclose(f) != 0 || bad) return 1;
    }
    free(hb);
    free(hx);
    free(hq);
    free(s0);
    free(s1);
    cudaFree(b);
    cudaFree(x);
    cudaFree(qb);
    CHECK(hh_destroy(ctx));
    return 0;
}
