// Host-only checks of the library's inline host logic: the engine's tiling
// rule and the molecular-dynamics schedules (leapfrog, Sec. 4.1; Omelyan's
// second-order minimum-norm scheme).  Prints the first failure and exits 1.
#include <cmath>
#include <cstdio>

#include "../../paper_1007_3432_gb300/csrc/hh_engine.cuh"
#include "../../paper_1007_3432_gb300/csrc/hh_kernels.cuh"

static int fail(const char *what, long long a, long long b)
{
    std::printf("FAIL %s: %lld %lld\n", what, a, b);
    return 1;
}

int main()
{
    // Tiling: tiles of 'chunk' contiguous sites (a multiple of 32) cover the
    // N sites exactly once, the last one possibly shorter, with at most one
    // tile per block per system and at most one tile per 512 sites.
    const int Ns[] = {1, 31, 32, 33, 512, 513, 2048, 6144, 100003, 524288, 4194304, 3538944};
    for (int N : Ns)
        for (int nsys : {1, 2, 3, 4, 64})
            for (int grid : {1, 76, 152, 304}) {
                hh::Tiling t = hh::engine_tiling(N, nsys, grid);
                if (t.chunk % 32 != 0) return fail("chunk multiple of 32", t.chunk, N);
                if ((long long)t.tiles * t.chunk < N) return fail("tiles cover N", t.tiles, N);
                if ((long long)(t.tiles - 1) * t.chunk >= N) return fail("no empty tile", t.tiles, N);
                const int want = (grid + nsys - 1) / nsys;
                if (t.tiles > (want > 1 ? want : 1) && t.tiles > 1) return fail("tiles per system", t.tiles, want);
                if (t.tiles > (N + hh::ENGINE_MIN_TILE - 1) / hh::ENGINE_MIN_TILE)
                    return fail("sites per tile", t.tiles, N);
            }
    // Group widths divide N_x.
    for (int nx = 1; nx < 200; ++nx) {
        const int w = hh::engine_group_width(nx);
        if (nx % w != 0 || (nx % 4 == 0 && w != 4)) return fail("group width", nx, w);
    }
    // MD schedules: total kick n_md dt, total drift n_md dt, and the force
    // counts; Omelyan's lambda (Omelyan, Mryglod, Folk, Comput. Phys. Commun.
    // 151 (2003) 272) is 1/2 - c/12 + 1/(6c), c = (2 sqrt(326) + 36)^(1/3),
    // = 0.1931833275037836 (evaluated independently in double precision).
    for (int integ : {0, 1})
        for (int n_md : {1, 2, 5, 20})
            for (double dt : {0.002, 0.05, 0.25}) {
                double kick, drift, ksum = 0.0, dsum = 0.0;
                const int forces = hh::md_schedule(integ, n_md, dt, 0, &kick, &drift);
                if (forces != (integ ? 2 * n_md + 1 : n_md + 1)) return fail("force count", forces, n_md);
                for (int j = 0; j < forces; ++j) {
                    hh::md_schedule(integ, n_md, dt, j, &kick, &drift);
                    ksum += kick;
                    if (j + 1 < forces) dsum += drift;
                }
                if (std::fabs(ksum - n_md * dt) > 1e-12 || std::fabs(dsum - n_md * dt) > 1e-12)
                    return fail("schedule sums", integ, n_md);
                if (integ == 1) {
                    hh::md_schedule(1, n_md, dt, 0, &kick, &drift);
                    if (std::fabs(kick / dt - 0.1931833275037836) > 1e-15) return fail("omelyan lambda", 0, 0);
                }
            }
    std::printf("ok\n");
    return 0;
}
