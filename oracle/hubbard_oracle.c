/*
 * Hubbard-model HMC oracle: a plain, slow, obviously correct FP64 CPU
 * restatement of the method of arXiv:1007.3432 (Wendt, Drut, Laehde).
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may build, load and call this file;
 * nothing on the product path does, and it shares no code, header, table or
 * helper with the CUDA library.  It is single-threaded and untuned on purpose:
 * every function is written for a reader checking it against the paper, with
 * loops over lattice sites and explicit coordinates.
 *
 * Readings of passages the paper leaves open (each is listed with its
 * justification in the design notes of the repository):
 *   R1 (Eq. (10), coefficients A-D unspecified): the diagonal block is the
 *      linearised 1 + dtau*K, i.e. 1 on the site and -h = -t*dtau on each of
 *      the 2d spatial neighbours; the time link into slice tau carries
 *      L(n, tau-1) = -(1 + A sin sigma(n, tau-1)).
 *   R2 (Eq. (6), HS transform unspecified): compact form 1 + A sin(sigma),
 *      flat measure, S_g = 0.
 *   R3 (Eq. (7)): the link from slice tau' to tau'+1 carries the source slice's
 *      field; its sign is -1 except on the wrap link N_tau-1 -> 0, which is +1
 *      (the +B_{N_tau} corner block: antiperiodic in time).
 *   R4 (Eqs. (11)-(12)): n_pf real Gaussian pseudofermion components,
 *      chi_a = M^T xi_a, S_pf = 1/2 sum_a chi_a^T Q^{-1} chi_a.  Two components
 *      give the weight det Q = (det M)^2 of Eq. (6).
 *   R5 (Sec. 4.1, CG): x0 = 0; stop on the recursive residual, then confirm
 *      with the true residual; if the check fails, the residual is replaced by
 *      the true one and the iteration continues.
 *   R6 (Sec. 4.1, MD): leapfrog with step dt; Metropolis accepts iff
 *      u < exp(-dH).
 *   R7 (random numbers, not specified by the paper): Philox4x64-10 with
 *      counter (block, tag | a<<8, traj, chain) and key (seed, 0);
 *      tags 0 sigma init, 1 momenta, 2 pseudofermion sources, 3 Metropolis,
 *      6 observable noise.
 *   R8 (Eq. (9)): with N_x = 2 both neighbours along an axis are one site and
 *      both count (coefficient -2h).
 *   R10 (Sec. 4.2, root ordering referenced but not given): the n conjugate
 *      root pairs form real quadratic factors applied in the Leja order of
 *      their centres.
 *   R11 (Eq. (7), exact blocks): B = e^{-dtau K} e^{-dtau V} with e^{-dtau K}
 *      = e^{hH} expanded to first or second order (link_order 1, 2).
 *   R12 (MD beyond leapfrog): Omelyan's second-order minimum-norm scheme;
 *      chronological initial guesses of the MD solves.
 *   R13 (observables, none named by the paper): noise estimators of
 *      diag(M^{-1}), whose diagonal blocks are the equal-time Green's
 *      functions (1 + B_tau ... B_{tau+1})^{-1} of the block form of Eq. (7).
 */
#include "hubbard_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Lattice geometry.                                                         */
/* ------------------------------------------------------------------------ */

static long spatial_volume(const oracle_lattice *lat)
{
    long v = 1;
    for (int j = 0; j < lat->d; ++j) v *= lat->nx;
    return v;
}

long oracle_nsites(const oracle_lattice *lat)
{
    return spatial_volume(lat) * lat->ntau;
}

/* Index of site (n, tau) with n = (c[0], ..., c[d-1]), c[0] = x fastest. */
static long site_index(const oracle_lattice *lat, const int *c, int tau)
{
    long s = 0;
    for (int j = lat->d - 1; j >= 0; --j) s = s * lat->nx + c[j];
    return s + (long)tau * spatial_volume(lat);
}

/* Inverse of site_index. */
static void site_coords(const oracle_lattice *lat, long i, int *c, int *tau)
{
    long v = spatial_volume(lat);
    *tau = (int)(i / v);
    long s = i % v;
    for (int j = 0; j < lat->d; ++j) {
        c[j] = (int)(s % lat->nx);
        s /= lat->nx;
    }
}

/* Sum of x over the 2d spatial nearest neighbours of (c, tau), periodic in
 * every spatial direction (Sec. 2: "periodic in the spatial directions").
 * For N_x = 2 the two neighbours along a direction coincide and both count,
 * exactly as the Kronecker deltas of Eq. (9) do. */
static double neighbour_sum(const oracle_lattice *lat, const double *x, const int *c, int tau)
{
    int cc[3];
    double s = 0.0;
    for (int j = 0; j < lat->d; ++j) {
        for (int k = 0; k < lat->d; ++k) cc[k] = c[k];
        cc[j] = (c[j] + 1) % lat->nx;
        s += x[site_index(lat, cc, tau)];
        cc[j] = (c[j] + lat->nx - 1) % lat->nx;
        s += x[site_index(lat, cc, tau)];
    }
    return s;
}

/* ------------------------------------------------------------------------ */
/* Fermion matrix, Sec. 2 Eqs. (7)-(10).                                      */
/* ------------------------------------------------------------------------ */

/* L(n,tau) for the link from slice tau to slice tau+1 (reading R1-R3):
 * -(1 + A sin sigma(n,tau)) for tau < N_tau-1 (the -B_j blocks of Eq. (7)) and
 * +(1 + A sin sigma(n,N_tau-1)) on the wrap link (the +B_{N_tau} corner). */
void oracle_links(const oracle_lattice *lat, double A, const double *sigma, double *L)
{
    long n = oracle_nsites(lat);
    int c[3], tau;
    for (long i = 0; i < n; ++i) {
        site_coords(lat, i, c, &tau);
        double link = 1.0 + A * sin(sigma[i]);
        L[i] = (tau == lat->ntau - 1) ? link : -link;
    }
}

/* (M x)(n,tau) = x(n,tau) - h sum_{+-j} x(n +- e_j, tau) + L(n,tau-1) x(n,tau-1),
 * tau-1 taken modulo N_tau (Eq. (10): one temporal link, the site itself and
 * 2d spatial neighbours; the wrap term is the corner block of Eq. (7)). */
void oracle_apply_M(const oracle_lattice *lat, double h, const double *L,
                    const double *x, double *y)
{
    long n = oracle_nsites(lat);
    int c[3], tau;
    for (long i = 0; i < n; ++i) {
        site_coords(lat, i, c, &tau);
        int tprev = (tau + lat->ntau - 1) % lat->ntau;
        long iprev = site_index(lat, c, tprev);
        y[i] = x[i] - h * neighbour_sum(lat, x, c, tau) + L[iprev] * x[iprev];
    }
}

/* (M^T y)(n,tau) = y(n,tau) - h sum_{+-j} y(n +- e_j, tau) + L(n,tau) y(n,tau+1):
 * the transpose of Eq. (10); the spatial hopping of Eq. (9) is symmetric. */
void oracle_apply_MT(const oracle_lattice *lat, double h, const double *L,
                     const double *x, double *y)
{
    long n = oracle_nsites(lat);
    int c[3], tau;
    for (long i = 0; i < n; ++i) {
        site_coords(lat, i, c, &tau);
        int tnext = (tau + 1) % lat->ntau;
        long inext = site_index(lat, c, tnext);
        y[i] = x[i] - h * neighbour_sum(lat, x, c, tau) + L[i] * x[inext];
    }
}

/* Q x = M^T (M x), applied as two successive sweeps (Sec. 4.3). */
void oracle_apply_MTM(const oracle_lattice *lat, double h, const double *L,
                      const double *x, double *y)
{
    long n = oracle_nsites(lat);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)n);
    oracle_apply_M(lat, h, L, x, tmp);
    oracle_apply_MT(lat, h, L, tmp, y);
    free(tmp);
}

/* E v on every time slice: E = 1 + h H (order 1) or 1 + h H + h^2 H^2 / 2
 * (order 2), (H v)(n,tau) the sum of v over the 2d spatial neighbours: the
 * expansion of e^{-dtau K} = e^{h H} (K = -t H, Sec. 2, Eqs. (8)-(9)). */
static void hop_factor(const oracle_lattice *lat, double h, int order, const double *v, double *out)
{
    long n = oracle_nsites(lat);
    int c[3], tau;
    double *hv = (double *)malloc(sizeof(double) * (size_t)n);
    for (long i = 0; i < n; ++i) {
        site_coords(lat, i, c, &tau);
        hv[i] = neighbour_sum(lat, v, c, tau);
    }
    for (long i = 0; i < n; ++i) out[i] = v[i] + h * hv[i];
    if (order == 2)
        for (long i = 0; i < n; ++i) {
            site_coords(lat, i, c, &tau);
            out[i] += 0.5 * h * h * neighbour_sum(lat, hv, c, tau);
        }
    free(hv);
}

/* Exact-block form of M: the blocks of Eq. (7) with B = e^{-dtau K} e^{-dtau V},
 * e^{-dtau K} expanded to order 1 or 2 (E above), e^{-dtau V} = 1 + A sin sigma
 * (reading R2), and the diagonal blocks 1:
 *   (M x)(n,tau) = x(n,tau) + [E w](n,tau-1),  w(m,tau') = L(m,tau') x(m,tau'),
 * with L = -(1 + A sin sigma) and + on the wrap link as in oracle_links.
 * order 0 is the form of oracle_apply_M (reading R1). */
void oracle_apply_M_ex(const oracle_lattice *lat, double h, const double *L, int order,
                       const double *x, double *y)
{
    if (order == 0) {
        oracle_apply_M(lat, h, L, x, y);
        return;
    }
    long n = oracle_nsites(lat);
    int c[3], tau;
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    double *ew = (double *)malloc(sizeof(double) * (size_t)n);
    for (long i = 0; i < n; ++i) w[i] = L[i] * x[i];
    hop_factor(lat, h, order, w, ew);
    for (long i = 0; i < n; ++i) {
        site_coords(lat, i, c, &tau);
        long iprev = site_index(lat, c, (tau + lat->ntau - 1) % lat->ntau);
        y[i] = x[i] + ew[iprev];
    }
    free(w);
    free(ew);
}

/* (M^T y)(m,tau) = y(m,tau) + L(m,tau) [E y](m,tau+1): E is symmetric. */
void oracle_apply_MT_ex(const oracle_lattice *lat, double h, const double *L, int order,
                        const double *x, double *y)
{
    if (order == 0) {
        oracle_apply_MT(lat, h, L, x, y);
        return;
    }
    long n = oracle_nsites(lat);
    int c[3], tau;
    double *ex = (double *)malloc(sizeof(double) * (size_t)n);
    hop_factor(lat, h, order, x, ex);
    for (long i = 0; i < n; ++i) {
        site_coords(lat, i, c, &tau);
        long inext = site_index(lat, c, (tau + 1) % lat->ntau);
        y[i] = x[i] + L[i] * ex[inext];
    }
    free(ex);
}

void oracle_apply_MTM_ex(const oracle_lattice *lat, double h, const double *L, int order,
                         const double *x, double *y)
{
    long n = oracle_nsites(lat);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)n);
    oracle_apply_M_ex(lat, h, L, order, x, tmp);
    oracle_apply_MT_ex(lat, h, L, order, tmp, y);
    free(tmp);
}

/* ------------------------------------------------------------------------ */
/* Conjugate gradient for Q x = b (Sec. 4.1).                               */
/* ------------------------------------------------------------------------ */

static double dot(long n, const double *a, const double *b)
{
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* CG for Q x = b from x0 = 0, or from the x passed in when guess != 0
 * (r0 = b - Q x0, stopping at once if that already meets tol; b = 0 gives
 * x = 0 either way). */
static int cg_from(const oracle_lattice *lat, double h, const double *L, int order, const double *b,
                   double *x, int guess, double tol, int maxit, int *iterations, double *true_relres)
{
    long n = oracle_nsites(lat);
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    int status = -4, k = 0;
    double bnorm = sqrt(dot(n, b, b));

    if (!guess || bnorm == 0.0) {
        for (long i = 0; i < n; ++i) {
            x[i] = 0.0;
            r[i] = b[i];
        }
    } else {
        oracle_apply_MTM_ex(lat, h, L, order, x, q);
        for (long i = 0; i < n; ++i) r[i] = b[i] - q[i];
    }
    for (long i = 0; i < n; ++i) p[i] = r[i];
    *true_relres = 0.0;
    if (bnorm == 0.0) {
        status = 0;
        goto done;
    }
    double rr = dot(n, r, r);
    *true_relres = sqrt(rr) / bnorm;
    if (guess && sqrt(rr) <= tol * bnorm) {
        status = 0;
        goto done;
    }
    for (k = 1; k <= maxit; ++k) {
        oracle_apply_MTM_ex(lat, h, L, order, p, q);
        double alpha = rr / dot(n, p, q);
        for (long i = 0; i < n; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
        }
        double rr_new = dot(n, r, r);
        if (sqrt(rr_new) <= tol * bnorm) {
            /* Confirm with the true residual b - Q x (reading R5). */
            oracle_apply_MTM_ex(lat, h, L, order, x, q);
            for (long i = 0; i < n; ++i) r[i] = b[i] - q[i];
            rr_new = dot(n, r, r);
            *true_relres = sqrt(rr_new) / bnorm;
            if (sqrt(rr_new) <= tol * bnorm) {
                status = 0;
                break;
            }
        }
        double beta = rr_new / rr;
        rr = rr_new;
        for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    }
    if (status != 0) {
        oracle_apply_MTM_ex(lat, h, L, order, x, q);
        for (long i = 0; i < n; ++i) r[i] = b[i] - q[i];
        *true_relres = sqrt(dot(n, r, r)) / bnorm;
        k = maxit;
    }
done:
    *iterations = k;
    free(r);
    free(p);
    free(q);
    return status;
}

int oracle_cg(const oracle_lattice *lat, double h, const double *L, const double *b,
              double *x, double tol, int maxit, int *iterations, double *true_relres)
{
    return cg_from(lat, h, L, 0, b, x, 0, tol, maxit, iterations, true_relres);
}

int oracle_cg_guess(const oracle_lattice *lat, double h, const double *L, const double *b,
                    double *x, double tol, int maxit, int *iterations, double *true_relres)
{
    return cg_from(lat, h, L, 0, b, x, 1, tol, maxit, iterations, true_relres);
}

int oracle_cg_ex(const oracle_lattice *lat, double h, const double *L, int order, const double *b,
                 double *x, int guess, double tol, int maxit, int *iterations, double *true_relres)
{
    return cg_from(lat, h, L, order, b, x, guess, tol, maxit, iterations, true_relres);
}

/* ------------------------------------------------------------------------ */
/* Chebyshev polynomial preconditioner, Sec. 4.2 Eqs. (13)-(17).            */
/* ------------------------------------------------------------------------ */

/* Root z_k of Eq. (15), as (re, im). */
static void cheb_root(int n, double eps, int k, double *re, double *im)
{
    const double pi = 3.14159265358979323846264338328;
    double m = 0.5 * (1.0 + eps);
    double th = 2.0 * pi * (double)k / (double)(2 * n + 1);
    *re = m * (1.0 - cos(th));
    *im = -sqrt(eps) * sin(th);
}

/* P(z) = c_2n prod_k (z - z_k) with c_2n^{-1} = m prod_k (m - z_k) (Eqs. (13)-(14)).
 * The roots come in conjugate pairs (k and 2n+1-k), so the product is real;
 * it is evaluated as a complex product of the 2n factors, each divided by its
 * value at z = m, in the order k = 1..2n. */
double oracle_cheb_poly(int n, double eps, double z)
{
    double m = 0.5 * (1.0 + eps);
    double pr = 1.0 / m, pi_ = 0.0;
    for (int k = 1; k <= 2 * n; ++k) {
        double re, im;
        cheb_root(n, eps, k, &re, &im);
        /* (z - z_k) / (m - z_k) */
        double ar = z - re, ai = -im;
        double br = m - re, bi = -im;
        double den = br * br + bi * bi;
        double qr = (ar * br + ai * bi) / den, qi = (ai * br - ar * bi) / den;
        double nr = pr * qr - pi_ * qi, ni = pr * qi + pi_ * qr;
        pr = nr;
        pi_ = ni;
    }
    return pr;
}

/* Order of the real factors.  Sec. 4.2 leaves the ordering of the roots open
 * (it points to an optimised one without giving it).  Applied to a vector,
 * each factor's rounding error is relative to the whole vector, and the
 * factors after it amplify it by the spread max_z / min_z of their product on
 * [0, 1]; in the order k = 1..n that spread reaches 1e31 at n = 32.  Reading:
 * Leja order of the real parts a_k (Reichel, BIT 30 (1990) 332): start with
 * the largest a_k, then repeatedly take the a_k that maximises the product of
 * its distances to those already taken (ties: the smallest k).  The spread
 * then stays below 1e8 up to n = 64. */
static void cheb_order(int n, double eps, int *order)
{
    double a[64], im;
    int used[64];
    for (int k = 1; k <= n; ++k) {
        cheb_root(n, eps, k, &a[k - 1], &im);
        used[k - 1] = 0;
    }
    int first = 0;
    for (int k = 1; k < n; ++k)
        if (fabs(a[k]) > fabs(a[first])) first = k;
    order[0] = first + 1;
    used[first] = 1;
    for (int j = 1; j < n; ++j) {
        int best = -1;
        double bv = 0.0;
        for (int k = 0; k < n; ++k) {
            if (used[k]) continue;
            double v = 0.0;
            for (int i = 0; i < j; ++i) v += log(fabs(a[k] - a[order[i] - 1]));
            if (best < 0 || v > bv) {
                best = k;
                bv = v;
            }
        }
        order[j] = best + 1;
        used[best] = 1;
    }
}

/* y = P(Q/lam) x: the conjugate pair k, 2n+1-k gives the real factor
 * ((Q/lam - a)^2 + b^2) / ((m - a)^2 + b^2) with a = Re z_k, b = Im z_k;
 * factors applied in the order of cheb_order(), then the overall 1/m
 * (n <= 64). */
void oracle_cheb_apply(const oracle_lattice *lat, double h, const double *L, int n, double eps,
                       double lam, const double *x, double *y)
{
    long N = oracle_nsites(lat);
    double m = 0.5 * (1.0 + eps);
    double *v = (double *)malloc(sizeof(double) * (size_t)N);
    double *u = (double *)malloc(sizeof(double) * (size_t)N);
    double *w = (double *)malloc(sizeof(double) * (size_t)N);
    for (long i = 0; i < N; ++i) v[i] = x[i];
    int order[64];
    cheb_order(n, eps, order);
    for (int j = 0; j < n; ++j) {
        double a, b;
        cheb_root(n, eps, order[j], &a, &b);
        double qm = (m - a) * (m - a) + b * b;
        /* u = (Q/lam - a) v */
        oracle_apply_MTM(lat, h, L, v, w);
        for (long i = 0; i < N; ++i) u[i] = w[i] / lam - a * v[i];
        /* v = ((Q/lam - a) u + b^2 v) / qm */
        oracle_apply_MTM(lat, h, L, u, w);
        for (long i = 0; i < N; ++i) v[i] = (w[i] / lam - a * u[i] + b * b * v[i]) / qm;
    }
    for (long i = 0; i < N; ++i) y[i] = v[i] / m;
    free(v);
    free(u);
    free(w);
}

/* Preconditioned CG (Sec. 4.2: CG on Q with the preconditioner P(Q/lam)),
 * x0 = 0, same stopping rule as oracle_cg. */
int oracle_pcg(const oracle_lattice *lat, double h, const double *L, int n, double eps, double lam,
               const double *b, double *x, double tol, int maxit, int *iterations, double *true_relres)
{
    long N = oracle_nsites(lat);
    double *r = (double *)malloc(sizeof(double) * (size_t)N);
    double *z = (double *)malloc(sizeof(double) * (size_t)N);
    double *p = (double *)malloc(sizeof(double) * (size_t)N);
    double *q = (double *)malloc(sizeof(double) * (size_t)N);
    int status = -4, k = 0;
    double bnorm = sqrt(dot(N, b, b));
    for (long i = 0; i < N; ++i) {
        x[i] = 0.0;
        r[i] = b[i];
    }
    *true_relres = 0.0;
    if (bnorm == 0.0) {
        status = 0;
        goto done;
    }
    *true_relres = 1.0;
    oracle_cheb_apply(lat, h, L, n, eps, lam, r, z);
    for (long i = 0; i < N; ++i) p[i] = z[i];
    double rz = dot(N, r, z);
    for (k = 1; k <= maxit; ++k) {
        oracle_apply_MTM(lat, h, L, p, q);
        double alpha = rz / dot(N, p, q);
        for (long i = 0; i < N; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
        }
        if (sqrt(dot(N, r, r)) <= tol * bnorm) {
            oracle_apply_MTM(lat, h, L, x, q);
            for (long i = 0; i < N; ++i) r[i] = b[i] - q[i];
            *true_relres = sqrt(dot(N, r, r)) / bnorm;
            if (*true_relres <= tol) {
                status = 0;
                break;
            }
        }
        oracle_cheb_apply(lat, h, L, n, eps, lam, r, z);
        double rz_new = dot(N, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
        for (long i = 0; i < N; ++i) p[i] = z[i] + beta * p[i];
    }
    if (status != 0) {
        oracle_apply_MTM(lat, h, L, x, q);
        for (long i = 0; i < N; ++i) r[i] = b[i] - q[i];
        *true_relres = sqrt(dot(N, r, r)) / bnorm;
        k = maxit;
    }
done:
    *iterations = k;
    free(r);
    free(z);
    free(p);
    free(q);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw,        */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11).                    */
/* ------------------------------------------------------------------------ */

void oracle_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t mult0 = 0xD2E7470EE14C6C93ULL, mult1 = 0xCA5A826395121157ULL;
    const uint64_t weyl0 = 0x9E3779B97F4A7C15ULL, weyl1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += weyl0;
            k1 += weyl1;
        }
        unsigned __int128 prod0 = (unsigned __int128)mult0 * c0;
        unsigned __int128 prod1 = (unsigned __int128)mult1 * c2;
        uint64_t hi0 = (uint64_t)(prod0 >> 64), lo0 = (uint64_t)prod0;
        uint64_t hi1 = (uint64_t)(prod1 >> 64), lo1 = (uint64_t)prod1;
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* 53-bit uniform in [0, 1) from the top bits of a 64-bit word. */
static double unit_uniform(uint64_t w)
{
    return (double)(w >> 11) * (1.0 / 9007199254740992.0);
}

static void philox_block(uint64_t seed, int tag, int a, uint64_t traj, uint64_t chain,
                         uint64_t block, uint64_t w[4])
{
    uint64_t ctr[4] = {block, (uint64_t)tag | ((uint64_t)a << 8), traj, chain};
    uint64_t key[2] = {seed, 0};
    oracle_philox4x64(ctr, key, w);
}

/* Element i: Box-Muller on the word pair (2j, 2j+1), j = (i >> 1) & 1, of
 * block i >> 2; even i takes the cosine branch, odd i the sine branch. */
void oracle_gaussian(uint64_t seed, int tag, int a, uint64_t traj, uint64_t chain,
                     long n, double *out)
{
    const double two_pi = 6.283185307179586476925286766559;
    for (long i = 0; i < n; ++i) {
        uint64_t w[4];
        philox_block(seed, tag, a, traj, chain, (uint64_t)i >> 2, w);
        int j = (int)((i >> 1) & 1);
        double u1 = unit_uniform(w[2 * j]);
        double u2 = unit_uniform(w[2 * j + 1]);
        double rad = sqrt(-2.0 * log(1.0 - u1));
        out[i] = (i & 1) ? rad * sin(two_pi * u2) : rad * cos(two_pi * u2);
    }
}

double oracle_uniform(uint64_t seed, int tag, uint64_t traj, uint64_t chain, long i)
{
    uint64_t w[4];
    philox_block(seed, tag, 0, traj, chain, (uint64_t)i >> 2, w);
    return unit_uniform(w[i & 3]);
}

/* sigma ~ U[-pi, pi) (reading R2), tag 0, trajectory word 0. */
void oracle_init_field(uint64_t seed, uint64_t chain, long n, double *sigma)
{
    const double pi = 3.14159265358979323846264338328;
    for (long i = 0; i < n; ++i)
        sigma[i] = -pi + 2.0 * pi * oracle_uniform(seed, 0, 0, chain, i);
}

/* ------------------------------------------------------------------------ */
/* HMC phi-algorithm, Sec. 4.1.                                              */
/* ------------------------------------------------------------------------ */

/* Pseudofermion heatbath (Eqs. (11)-(12), reading R4): chi_a = M^T xi_a with
 * xi_a ~ N(0,1), so chi_a has covariance Q and S_pf(sigma) = 1/2 |xi|^2. */
void oracle_heatbath(const oracle_lattice *lat, const oracle_params *p,
                     const double *sigma, uint64_t traj, double *chi)
{
    long n = oracle_nsites(lat);
    double *L = (double *)malloc(sizeof(double) * (size_t)n);
    double *xi = (double *)malloc(sizeof(double) * (size_t)n);
    oracle_links(lat, p->A, sigma, L);
    for (int a = 0; a < p->n_pf; ++a) {
        oracle_gaussian(p->seed, 2, a, traj, p->chain, n, xi);
        oracle_apply_MT_ex(lat, p->t * p->dtau, L, p->link_order, xi, chi + (long)a * n);
    }
    free(L);
    free(xi);
}

/* S_pf = 1/2 sum_a chi_a^T Q^{-1} chi_a (Eq. (12) with real components). */
double oracle_action(const oracle_lattice *lat, const oracle_params *p,
                     const double *sigma, const double *chi, int *iters, double *relres,
                     int *status)
{
    long n = oracle_nsites(lat);
    double h = p->t * p->dtau;
    double *L = (double *)malloc(sizeof(double) * (size_t)n);
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    double S = 0.0;
    oracle_links(lat, p->A, sigma, L);
    for (int a = 0; a < p->n_pf; ++a) {
        int it;
        double rr;
        int st = oracle_cg_ex(lat, h, L, p->link_order, chi + (long)a * n, x, 0, p->cg_tol, p->cg_maxit,
                              &it, &rr);
        if (st != 0) *status = st;
        *iters += it;
        if (rr > *relres) *relres = rr;
        S += 0.5 * dot(n, chi + (long)a * n, x);
    }
    free(L);
    free(x);
    return S;
}

/* F(n,tau) = dS_pf / dsigma(n,tau).  With x_a = Q^{-1} chi_a and y_a = M x_a,
 * dS/dsigma = -sum_a y_a^T (dM/dsigma) x_a, and sigma(n,tau) enters M only
 * through the link L(n,tau) at row (n,tau+1), column (n,tau), whose derivative
 * is s(tau) A cos sigma(n,tau) with s = -1, or +1 on the wrap link. */
/* The force with the solutions x_a kept in xs (n_pf * N); guess != 0 starts
 * each solve from the xs passed in. */
static void force_from(const oracle_lattice *lat, const oracle_params *p, const double *sigma,
                       const double *chi, double *F, double *xs, int guess, int *iters,
                       double *relres, int *status)
{
    long n = oracle_nsites(lat);
    double h = p->t * p->dtau;
    double *L = (double *)malloc(sizeof(double) * (size_t)n);
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    double *ey = (double *)malloc(sizeof(double) * (size_t)n);
    int c[3], tau;
    oracle_links(lat, p->A, sigma, L);
    for (long i = 0; i < n; ++i) F[i] = 0.0;
    for (int a = 0; a < p->n_pf; ++a) {
        int it;
        double rr;
        double *x = xs + (long)a * n;
        int st = oracle_cg_ex(lat, h, L, p->link_order, chi + (long)a * n, x, guess, p->cg_tol, p->cg_maxit,
                              &it, &rr);
        if (st != 0) *status = st;
        *iters += it;
        if (rr > *relres) *relres = rr;
        oracle_apply_M_ex(lat, h, L, p->link_order, x, y);
        /* Exact-block form: sigma(n,tau) enters through w(n,tau) = L x, seen by
         * row (., tau+1) through E, so the factor of y is (E y)(n, tau+1). */
        if (p->link_order != 0) {
            hop_factor(lat, h, p->link_order, y, ey);
            for (long i = 0; i < n; ++i) y[i] = ey[i];
        }
        for (long i = 0; i < n; ++i) {
            site_coords(lat, i, c, &tau);
            long inext = site_index(lat, c, (tau + 1) % lat->ntau);
            double s = (tau == lat->ntau - 1) ? 1.0 : -1.0;
            F[i] -= y[inext] * s * p->A * cos(sigma[i]) * x[i];
        }
    }
    free(L);
    free(y);
    free(ey);
}

void oracle_force(const oracle_lattice *lat, const oracle_params *p, const double *sigma,
                  const double *chi, double *F, int *iters, double *relres, int *status)
{
    double *xs = (double *)malloc(sizeof(double) * (size_t)oracle_nsites(lat) * (size_t)p->n_pf);
    force_from(lat, p, sigma, chi, F, xs, 0, iters, relres, status);
    free(xs);
}

/* Leapfrog integration of d sigma/dt = pi, d pi/dt = -F (reading R6):
 * half momentum step, n_md full sigma steps with full momentum steps between
 * them, half momentum step at the end; n_md + 1 force evaluations. */
/* Solutions of the molecular dynamics' solves, for chronological initial
 * guesses: xs the latest, xp the one before; j counts the solves so far. */
typedef struct {
    double *xs, *xp;
    int j;
} md_solutions;

/* pi -= eps F(sigma).  Initial guess of its solves (p->chrono): 0 none;
 * 1 the previous force's solutions; 2 their linear extrapolation
 * 2 x_{j-1} - x_{j-2} (1 at the second force). */
static void kick(const oracle_lattice *lat, const oracle_params *p, const double *sigma,
                 double *pi, const double *chi, double eps, double *F, md_solutions *ms,
                 int *iters, double *relres, int *status)
{
    long n = oracle_nsites(lat), m = n * (long)p->n_pf;
    int guess = p->chrono != 0 && ms->j >= 1;
    if (p->chrono == 2 && ms->j >= 2)
        for (long i = 0; i < m; ++i) {
            double t = ms->xs[i];
            ms->xs[i] = 2.0 * t - ms->xp[i];
            ms->xp[i] = t;
        }
    else
        for (long i = 0; i < m; ++i) ms->xp[i] = ms->xs[i];
    force_from(lat, p, sigma, chi, F, ms->xs, guess, iters, relres, status);
    ms->j += 1;
    for (long i = 0; i < n; ++i) pi[i] -= eps * F[i];
}

/* sigma += eps pi */
static void drift(long n, double *sigma, const double *pi, double eps)
{
    for (long i = 0; i < n; ++i) sigma[i] += eps * pi[i];
}

/* The parameter of Omelyan's second-order minimum-norm scheme, the root
 * 1/2 - c/12 + 1/(6c), c = (2 sqrt(326) + 36)^(1/3), of its error norm. */
static double omelyan_lambda(void)
{
    double c = cbrt(2.0 * sqrt(326.0) + 36.0);
    return 0.5 - c / 12.0 + 1.0 / (6.0 * c);
}

void oracle_leapfrog(const oracle_lattice *lat, const oracle_params *p, double *sigma,
                     double *pi, const double *chi, int n_md, double dt, int *iters,
                     double *relres, int *status)
{
    long n = oracle_nsites(lat);
    double *F = (double *)malloc(sizeof(double) * (size_t)n);
    md_solutions ms;
    ms.xs = (double *)calloc((size_t)n * (size_t)p->n_pf, sizeof(double));
    ms.xp = (double *)calloc((size_t)n * (size_t)p->n_pf, sizeof(double));
    ms.j = 0;
    if (p->integrator == 1) {
        /* Per step: kick lambda dt, drift dt/2, kick (1 - 2 lambda) dt, drift
         * dt/2, kick lambda dt; the end kick of a step and the first of the
         * next merge into one of 2 lambda dt. */
        double lam = omelyan_lambda();
        kick(lat, p, sigma, pi, chi, lam * dt, F, &ms, iters, relres, status);
        for (int k = 1; k <= n_md; ++k) {
            drift(n, sigma, pi, 0.5 * dt);
            kick(lat, p, sigma, pi, chi, (1.0 - 2.0 * lam) * dt, F, &ms, iters, relres, status);
            drift(n, sigma, pi, 0.5 * dt);
            kick(lat, p, sigma, pi, chi, (k == n_md ? lam : 2.0 * lam) * dt, F, &ms, iters, relres, status);
        }
    } else {
        kick(lat, p, sigma, pi, chi, 0.5 * dt, F, &ms, iters, relres, status);
        for (int k = 1; k <= n_md; ++k) {
            drift(n, sigma, pi, dt);
            kick(lat, p, sigma, pi, chi, (k == n_md) ? 0.5 * dt : dt, F, &ms, iters, relres, status);
        }
    }
    free(F);
    free(ms.xs);
    free(ms.xp);
}

/* One HMC trajectory (Sec. 4.1): momenta and pseudofermion heatbath,
 * H0 = 1/2 |pi|^2 + S_pf, leapfrog, H1, Metropolis accept/reject. */
int oracle_trajectory(const oracle_lattice *lat, const oracle_params *p, double *sigma,
                      int n_md, double dt, uint64_t traj, oracle_traj_info *info)
{
    long n = oracle_nsites(lat);
    double *pi = (double *)malloc(sizeof(double) * (size_t)n);
    double *chi = (double *)malloc(sizeof(double) * (size_t)n * (size_t)p->n_pf);
    double *sigma0 = (double *)malloc(sizeof(double) * (size_t)n);
    int iters = 0, status = 0;
    double relres = 0.0;

    memcpy(sigma0, sigma, sizeof(double) * (size_t)n);
    oracle_gaussian(p->seed, 1, 0, traj, p->chain, n, pi);
    oracle_heatbath(lat, p, sigma, traj, chi);

    double H0 = 0.5 * dot(n, pi, pi) + oracle_action(lat, p, sigma, chi, &iters, &relres, &status);
    oracle_leapfrog(lat, p, sigma, pi, chi, n_md, dt, &iters, &relres, &status);
    double H1 = 0.5 * dot(n, pi, pi) + oracle_action(lat, p, sigma, chi, &iters, &relres, &status);

    double dH = H1 - H0;
    double u = oracle_uniform(p->seed, 3, traj, p->chain, 0);
    int accepted = u < exp(-dH);
    if (!accepted) memcpy(sigma, sigma0, sizeof(double) * (size_t)n);

    info->H0 = H0;
    info->H1 = H1;
    info->dH = dH;
    info->u = u;
    info->accepted = accepted;
    info->cg_iterations = iters;
    info->n_solves = p->n_pf * ((p->integrator == 1 ? 2 * n_md + 1 : n_md + 1) + 2);
    info->max_relres = relres;
    info->status = status;
    free(pi);
    free(chi);
    free(sigma0);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Observables (reading R13).                                                */
/* ------------------------------------------------------------------------ */

/* Z2 noise vector k: element i is +1 if the top bit of word i & 3 of Philox
 * block i >> 2 (tag 6, a = k) is set, else -1. */
void oracle_z2_noise(uint64_t seed, int k, uint64_t traj, uint64_t chain, long n, double *eta)
{
    for (long i = 0; i < n; ++i) {
        uint64_t w[4];
        philox_block(seed, 6, k, traj, chain, (uint64_t)i >> 2, w);
        eta[i] = (w[i & 3] >> 63) ? 1.0 : -1.0;
    }
}

/* With n_noise Z2 vectors eta_k and y_k = M^{-1} eta_k = Q^{-1} (M^T eta_k)
 * (a CG solve on Q, the form of M given by p->link_order):
 *   t_k = (1/N) eta_k . y_k  estimates (1/N) tr M^{-1} without bias;
 *   g_A(i), g_B(i) = the means of eta_k(i) y_k(i) over the first and the
 *   second half of the vectors estimate M^{-1}_ii independently, so
 *   (1/N) sum_i (1 - g_A(i)) (1 - g_B(i)) estimates (1/N) sum_i (1 - M^{-1}_ii)^2.
 * out[0] = mean of t_k, out[1] = its standard error (sample deviation over
 * sqrt(n_noise)), out[2] = the product estimate, out[3] = (1/N) sum sin sigma,
 * out[4] = (1/N) sum sin^2 sigma.  n_noise must be even and >= 2. */
int oracle_observables(const oracle_lattice *lat, const oracle_params *p, const double *sigma,
                       int n_noise, uint64_t traj, double *out, int *iters, double *relres)
{
    long n = oracle_nsites(lat);
    int half = n_noise / 2, status = 0;
    double h = p->t * p->dtau;
    double *L = (double *)malloc(sizeof(double) * (size_t)n);
    double *eta = (double *)malloc(sizeof(double) * (size_t)n);
    double *rhs = (double *)malloc(sizeof(double) * (size_t)n);
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    double *gA = (double *)calloc((size_t)n, sizeof(double));
    double *gB = (double *)calloc((size_t)n, sizeof(double));
    double *t = (double *)malloc(sizeof(double) * (size_t)n_noise);
    oracle_links(lat, p->A, sigma, L);
    for (int k = 0; k < n_noise; ++k) {
        int it;
        double rr;
        oracle_z2_noise(p->seed, k, traj, p->chain, n, eta);
        oracle_apply_MT_ex(lat, h, L, p->link_order, eta, rhs);
        int st = oracle_cg_ex(lat, h, L, p->link_order, rhs, y, 0, p->cg_tol, p->cg_maxit, &it, &rr);
        if (st != 0) status = st;
        *iters += it;
        if (rr > *relres) *relres = rr;
        t[k] = dot(n, eta, y) / (double)n;
        double *g = k < half ? gA : gB;
        for (long i = 0; i < n; ++i) g[i] += eta[i] * y[i] / (double)half;
    }
    double mean = 0.0, var = 0.0, prod = 0.0, s1 = 0.0, s2 = 0.0;
    for (int k = 0; k < n_noise; ++k) mean += t[k];
    mean /= (double)n_noise;
    for (int k = 0; k < n_noise; ++k) var += (t[k] - mean) * (t[k] - mean);
    var /= (double)(n_noise - 1);
    for (long i = 0; i < n; ++i) {
        prod += (1.0 - gA[i]) * (1.0 - gB[i]);
        s1 += sin(sigma[i]);
        s2 += sin(sigma[i]) * sin(sigma[i]);
    }
    out[0] = mean;
    out[1] = sqrt(var / (double)n_noise);
    out[2] = prod / (double)n;
    out[3] = s1 / (double)n;
    out[4] = s2 / (double)n;
    free(L);
    free(eta);
    free(rhs);
    free(y);
    free(gA);
    free(gB);
    free(t);
    return status;
}
