/*
 * Hubbard-model HMC oracle: declarations.
 *
 * TEST INFRASTRUCTURE ONLY.  This header belongs to the plain FP64 CPU oracle
 * in this directory.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may include, link or call it.  The CUDA library does not
 * include this file and shares no code with it.
 *
 * Method: K. A. Wendt, J. E. Drut, T. A. Laehde, "Toward large-scale Hybrid
 * Monte Carlo simulations of the Hubbard model on graphics processing units",
 * arXiv:1007.3432.  Section 2 defines the fermion matrix M (Eqs. (7)-(10));
 * Sec. 4.1 defines the HMC phi-algorithm with pseudofermions (Eqs. (11)-(12))
 * and the linear problem Q x = b with Q = M^T M solved by conjugate gradient.
 *
 * Site index of (n, tau) on the (d+1)-dimensional lattice, x fastest:
 *   d = 1: i = x + Nx * tau
 *   d = 3: i = x + Nx * (y + Nx * (z + Nx * tau))
 */
#ifndef HUBBARD_ORACLE_H
#define HUBBARD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int d;      /* spatial dimension, 1 or 3 */
    int nx;     /* spatial extent N_x (periodic), >= 2 */
    int ntau;   /* time slices N_tau (antiperiodic), >= 2 */
} oracle_lattice;

typedef struct {
    double t;         /* hopping amplitude */
    double dtau;      /* Trotter step (the paper's tau in Eq. (8)) */
    double A;         /* auxiliary-field coupling: link factor 1 + A sin(sigma) */
    double cg_tol;    /* stop when ||b - Q x|| <= cg_tol * ||b|| */
    int cg_maxit;     /* CG iteration cap */
    int n_pf;         /* real pseudofermion components (2 = one complex field) */
    uint64_t seed;    /* Philox key */
    uint64_t chain;   /* Philox counter word 3 */
    int integrator;   /* 0: leapfrog (Sec. 4.1); 1: Omelyan's second-order
                         minimum-norm scheme (Omelyan, Mryglod, Folk, Comput.
                         Phys. Commun. 151 (2003) 272) */
    int chrono;       /* initial guess of the MD's solves: 0 zero (reversible);
                         1 the previous force's solution; 2 linear extrapolation
                         of the last two.  Not part of the paper's method: it
                         makes the MD reversible only to the CG tolerance. */
    int link_order;   /* form of M: 0 reading R1 (oracle_apply_M); 1, 2 the
                         exact-block form (oracle_apply_M_ex) */
} oracle_params;

typedef struct {
    double H0, H1, dH;   /* Hamiltonian before/after the MD trajectory */
    double u;            /* Metropolis uniform */
    int accepted;        /* 1 if u < exp(-dH) */
    int cg_iterations;   /* CG iterations summed over all solves */
    int n_solves;        /* CG solves performed */
    double max_relres;   /* largest true relative residual over the solves */
    int status;          /* 0, or -4 if a solve did not converge */
} oracle_traj_info;

long oracle_nsites(const oracle_lattice *lat);

/* Link coefficients L(n,tau), Sec. 2 Eqs. (7)-(10). */
void oracle_links(const oracle_lattice *lat, double A, const double *sigma, double *L);

/* y = M x, y = M^T x, y = M^T M x (Eq. (10) with the Eq. (7) boundary). */
void oracle_apply_M(const oracle_lattice *lat, double h, const double *L,
                    const double *x, double *y);
void oracle_apply_MT(const oracle_lattice *lat, double h, const double *L,
                     const double *x, double *y);
void oracle_apply_MTM(const oracle_lattice *lat, double h, const double *L,
                      const double *x, double *y);

/* Exact-block form of M (Eq. (7) with B = e^{-dtau K} e^{-dtau V}, the hopping
 * factor expanded to order 1 or 2 in dtau K; order 0 is the R1 form above):
 * (M x)(n,tau) = x(n,tau) + [E (L x)](n,tau-1), E = 1 + h H (+ h^2 H^2 / 2),
 * H the sum over the 2d spatial neighbours; M^T and M^T M likewise. */
void oracle_apply_M_ex(const oracle_lattice *lat, double h, const double *L, int order,
                       const double *x, double *y);
void oracle_apply_MT_ex(const oracle_lattice *lat, double h, const double *L, int order,
                        const double *x, double *y);
void oracle_apply_MTM_ex(const oracle_lattice *lat, double h, const double *L, int order,
                         const double *x, double *y);

/* Plain CG for Q x = b, x0 = 0 (Sec. 4.1).  Returns 0 or -4 (no convergence). */
int oracle_cg(const oracle_lattice *lat, double h, const double *L, const double *b,
              double *x, double tol, int maxit, int *iterations, double *true_relres);
/* The same from the initial guess x0 held in x: r0 = b - Q x0 (0 iterations
 * if that already meets tol; b = 0 gives x = 0). */
int oracle_cg_guess(const oracle_lattice *lat, double h, const double *L, const double *b,
                    double *x, double tol, int maxit, int *iterations, double *true_relres);
/* CG for the M of the given order, from zero or (guess != 0) from x. */
int oracle_cg_ex(const oracle_lattice *lat, double h, const double *L, int order, const double *b,
                 double *x, int guess, double tol, int maxit, int *iterations, double *true_relres);

/* Chebyshev polynomial preconditioner of Sec. 4.2, Eqs. (13)-(17).
 * Roots z_k = m (1 - cos(2 pi k/(2n+1))) - i sqrt(eps) sin(2 pi k/(2n+1)),
 * m = (1 + eps)/2, k = 1..2n, for Q normalised to eigenvalues in [0, 1]. */
double oracle_cheb_poly(int n, double eps, double z);
/* y = P(Q/lam) x (normalisation lam >= lambda_max(Q); n <= 64), as n real
 * quadratic factors in the Leja order of their centres (a reading: the paper
 * leaves the ordering open). */
void oracle_cheb_apply(const oracle_lattice *lat, double h, const double *L, int n, double eps,
                       double lam, const double *x, double *y);
/* Preconditioned CG with preconditioner P(Q/lam); x0 = 0; stop on the true
 * residual as oracle_cg.  *iterations counts PCG steps. */
int oracle_pcg(const oracle_lattice *lat, double h, const double *L, int n, double eps, double lam,
               const double *b, double *x, double tol, int maxit, int *iterations, double *true_relres);

/* Philox4x64-10 block cipher (Salmon et al., SC'11). */
void oracle_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
void oracle_gaussian(uint64_t seed, int tag, int a, uint64_t traj, uint64_t chain,
                     long n, double *out);
double oracle_uniform(uint64_t seed, int tag, uint64_t traj, uint64_t chain, long i);
void oracle_init_field(uint64_t seed, uint64_t chain, long n, double *sigma);

/* HMC pieces (Sec. 4.1). */
void oracle_heatbath(const oracle_lattice *lat, const oracle_params *p,
                     const double *sigma, uint64_t traj, double *chi);
double oracle_action(const oracle_lattice *lat, const oracle_params *p,
                     const double *sigma, const double *chi, int *iters, double *relres,
                     int *status);
void oracle_force(const oracle_lattice *lat, const oracle_params *p, const double *sigma,
                  const double *chi, double *F, int *iters, double *relres, int *status);
/* n_md molecular-dynamics steps of size dt with the integrator of p:
 * leapfrog (n_md + 1 forces) or Omelyan (2 n_md + 1 forces). */
void oracle_leapfrog(const oracle_lattice *lat, const oracle_params *p, double *sigma,
                     double *pi, const double *chi, int n_md, double dt, int *iters,
                     double *relres, int *status);
int oracle_trajectory(const oracle_lattice *lat, const oracle_params *p, double *sigma,
                      int n_md, double dt, uint64_t traj, oracle_traj_info *info);

/* Z2 noise vector k (Philox tag 6) and the noise estimators of (1/N) tr M^{-1}
 * and (1/N) sum_i (1 - M^{-1}_ii)^2 with the field moments (reading R13). */
void oracle_z2_noise(uint64_t seed, int k, uint64_t traj, uint64_t chain, long n, double *eta);
int oracle_observables(const oracle_lattice *lat, const oracle_params *p, const double *sigma,
                       int n_noise, uint64_t traj, double *out, int *iters, double *relres);

#ifdef __cplusplus
}
#endif

#endif
