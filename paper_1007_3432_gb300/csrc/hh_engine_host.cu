// Host-side policies of the persistent CG engine: the Chebyshev
// preconditioner's coefficient table (Sec. 4.2), the control-warp count, the
// L2 prefetch distance, the overlapped layout and the iteration form.  No CUDA
// call: they depend only on their arguments and the environment.
#include <cmath>
#include <cstdlib>

#include "hh_engine.cuh"

namespace hh {

void engine_cheb_table(int d, double h, double A, int n, double eps, double *tab)
{
    // Sec. 4.2: roots z_k = m (1 - cos th_k) - i sqrt(eps) sin th_k,
    // th_k = 2 pi k / (2n + 1), m = (1 + eps)/2, for Q / lam with lam the
    // Gershgorin bound of its spectrum: each row of M has the unit diagonal,
    // 2d hops of h and one link of size <= 1 + A.  The conjugate pair k,
    // 2n + 1 - k forms the real factor ((z - a_k)^2 + b_k^2) / q_k with q_k its
    // value at m.  Order of the factors: each one's rounding is relative to the
    // whole vector, and the factors after it amplify it by the spread
    // max / min over [0, 1] of their product (1e31 at n = 32 in the order
    // k = 1..n).  They are stored, and applied, in the Leja order of their
    // centres a_k (Reichel 1990): the largest first, then each next one
    // maximising the product of its distances to those before (ties: the
    // smallest k), which keeps the spread below 1e8 up to n = 64.
    const double pi = 3.14159265358979323846;
    const double m = 0.5 * (1.0 + eps);
    const double rowsum = 2.0 + 2.0 * d * fabs(h) + fabs(A);
    const double lam = rowsum * rowsum;
    for (int i = 0; i < 2 + 3 * CHEB_MAX_DEGREE; ++i) tab[i] = 0.0;
    tab[0] = 1.0 / lam;
    tab[1] = 1.0 / m;
    double ak[CHEB_MAX_DEGREE], bk[CHEB_MAX_DEGREE];
    bool taken[CHEB_MAX_DEGREE];
    for (int k = 0; k < n; ++k) {
        const double th = 2.0 * pi * (k + 1) / (2.0 * n + 1.0);
        ak[k] = m * (1.0 - cos(th));
        bk[k] = sqrt(eps) * sin(th);
        taken[k] = false;
    }
    int seq[CHEB_MAX_DEGREE];
    for (int j = 0; j < n; ++j) {
        int pick = -1;
        double score = 0.0;
        for (int k = 0; k < n; ++k) {
            if (taken[k]) continue;
            double v = 0.0;
            if (j == 0)
                v = fabs(ak[k]);
            else
                for (int i = 0; i < j; ++i) v += log(fabs(ak[k] - ak[seq[i]]));
            if (pick < 0 || v > score) {
                pick = k;
                score = v;
            }
        }
        seq[j] = pick;
        taken[pick] = true;
        const double a = ak[pick], b = bk[pick];
        tab[2 + 3 * j] = a;
        tab[3 + 3 * j] = b * b;
        tab[4 + 3 * j] = 1.0 / ((m - a) * (m - a) + b * b);
    }
}

int engine_ctl_warps(int dflt)
{
    const char *env = getenv("HH_ENGINE_CTL_WARPS");
    if (!env) return dflt;
    const int v = atoi(env);
    return v < 0 ? 0 : (v > 2 ? 2 : v);
}

int engine_prefetch(long long bytes, int d)
{
    int pf = (d == 3 && bytes > (64LL << 20)) ? 1 : 0;
    if (const char *env = getenv("HH_ENGINE_PREFETCH")) pf = atoi(env);
    return pf < 0 ? 0 : (pf > 8 ? 8 : pf);
}

bool engine_overlap(int nsys, long long sites, bool mixed)
{
    const char *env = getenv("HH_ENGINE_OVERLAP");
    if (nsys < 2) return false;
    if (env) return atoi(env) != 0;
    return sites >= (mixed ? (1LL << 21) : (1LL << 18));
}

int engine_two_slot(int kind)
{
    const char *env = getenv("HH_ENGINE_SLOTS");
    if (env && atoi(env) == 3) return 0;
    if (env && atoi(env) == 2) return 1;
    // Measured on GB300: the fused form is faster for d = 1 (its neighbour
    // recomputation is two x-halo sites and one earlier row), slower for
    // d = 3, where it re-reads both operands of p at six neighbour rows.
    return (kind == ENGINE_D1 || kind == ENGINE_D1_L16) ? 1 : 0;
}

}  // namespace hh
