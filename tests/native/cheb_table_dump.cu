// Host-only: evaluates the library's Chebyshev preconditioner table (built by
// engine_cheb_table) as the polynomial the engine applies,
//   P(x) = (1/m) prod_k ((x - a_k)^2 + b_k^2) / q_k   (x = eigenvalue / lam),
// factor by factor in the stored order, at the points given on the command
// line after (n, eps); prints one value per line.  Built with the engine's
// host-side translation unit (hh_engine_host.cu) alone.
#include <cstdio>
#include <cstdlib>

#include "../../paper_1007_3432_gb300/csrc/hh_engine.cuh"

int main(int argc, char **argv)
{
    if (argc < 4) return 2;
    const int n = atoi(argv[1]);
    const double eps = atof(argv[2]);
    double tab[2 + 3 * hh::CHEB_MAX_DEGREE];
    hh::engine_cheb_table(1, 0.05, 0.5, n, eps, tab);
    for (int i = 3; i < argc; ++i) {
        const double x = atof(argv[i]);
        double p = tab[1];
        for (int k = 0; k < n; ++k) {
            const double a = tab[2 + 3 * k], b2 = tab[3 + 3 * k], invq = tab[4 + 3 * k];
            p *= ((x - a) * (x - a) + b2) * invq;
        }
        std::printf("%.17g\n", p);
    }
    return 0;
}
