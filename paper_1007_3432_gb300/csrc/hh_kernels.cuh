// Launchers of the non-persistent kernels of the library (links, stencil
// applies, random draws, HMC updates).  All launch on the given stream and
// return the launch's cudaError_t.
#pragma once

#include <cmath>

#include "hh_device.cuh"

namespace hh {

// Device scalars of one HMC context (one slot each, written by kernels).
struct HmcScalars {
    double H0, H1, dH, u;
    double S_pf;            // last action evaluated
    int accepted;
    int pad;
    double part_scratch;    // unused padding to keep doubles aligned
};

// L64(i) = s(tau) (1 + A sin sigma_i), s = -1 except +1 at tau = N_tau - 1;
// L32 = (float)L64.
cudaError_t launch_links(const Geo &g, double A, const double *sigma, double *L64, float *L32,
                         cudaStream_t st);

// sigma += dt * pi, then the links.
cudaError_t launch_sigma_step(const Geo &g, double A, double dt, double *sigma, const double *pi,
                              double *L64, float *L32, cudaStream_t st);

// y = M x or y = M^T x (op 0 / 1), FP64 or FP32; order 0 is the form of
// reading R1, 1 and 2 the exact-block form (stencil_M_ex).
cudaError_t launch_apply_f64(const Geo &g, int op, double h, const double *L, const double *x,
                             double *y, cudaStream_t st, int order = 0);
cudaError_t launch_apply_f32(const Geo &g, int op, float h, const float *L, const float *x, float *y,
                             cudaStream_t st, int order = 0);

// out[i] = N(0,1) Philox/Box-Muller draw for element i (tag, a, traj, chain).
cudaError_t launch_gaussian(double *out, int n, uint64_t seed, int tag, int a, uint64_t traj,
                            uint64_t chain, cudaStream_t st);
// sigma[i] = -pi + 2 pi u_i (tag 0).
cudaError_t launch_init_field(double *sigma, int n, uint64_t seed, uint64_t chain, cudaStream_t st);

// Force F = dS/dsigma from solutions x_a (n_rhs of them, at x + a*N); if pi is
// non-null, pi -= eps * F; if F_out is non-null, F is stored.
cudaError_t launch_force(const Geo &g, double h, double A, const double *sigma, const double *L64,
                         const double *x, int n_rhs, double *pi, double eps, double *F_out,
                         cudaStream_t st);

// Energy partials: block b writes part[b] = sum over its sites of
// 1/2 pi^2 (if pi) + 1/2 sum_a chi_a x_a.  'nblocks' is returned by
// energy_blocks(N).  Then energy_finish sums part[0..nblocks) in order into
// *out (device double).
int energy_blocks(int n);
cudaError_t launch_energy(int n, const double *pi, const double *chi, const double *x, int n_rhs,
                          double *part, double *out, cudaStream_t st);

// dH = H1 - H0, u = Philox uniform (tag 3, index 0), accepted = u < exp(-dH).
cudaError_t launch_metropolis(HmcScalars *sc, uint64_t seed, uint64_t traj, uint64_t chain,
                              cudaStream_t st);
// If !sc->accepted: sigma = sigma0 and the links are recomputed.
cudaError_t launch_restore(const Geo &g, double A, const HmcScalars *sc, double *sigma,
                           const double *sigma0, double *L64, float *L32, cudaStream_t st);

// 16-bit links of the FP32 steps (mode 1 bfloat16, mode 2 fixed point with
// value = code * scale) from the FP64 links.
cudaError_t launch_links16(int n, const double *L64, unsigned short *L16, int mode, double scale, cudaStream_t st);

// Observables (noise estimators of diag M^{-1}; see hh_observables).
// nvec Z2 noise vectors (Philox tag 6, vector k at out + k n).
constexpr int kObsMaxNoise = 64;
cudaError_t launch_z2_noise(double *out, int n, int nvec, uint64_t seed, uint64_t traj, uint64_t chain,
                            cudaStream_t st);
// From eta_k and y_k = M^{-1} eta_k (k < nvec, even): out[0] = mean of
// (1/n) eta_k . y_k, out[1] its standard error, out[2] = (1/n) sum_i
// (1 - gA_i)(1 - gB_i) with gA, gB the half-set means of eta_k y_k, out[3],
// out[4] = (1/n) sum sin sigma, sin^2 sigma.  part: (nvec + 3) *
// energy_blocks(n) doubles of scratch.
cudaError_t launch_observables(int n, int nvec, const double *eta, const double *y, const double *sigma,
                               double *part, double *out, cudaStream_t st);

// Chronological initial guess by linear extrapolation: x <- 2 x - xp and
// xp <- the old x, over n elements.
cudaError_t launch_extrapolate(double *x, double *xp, long long n, cudaStream_t st);

// The force of the exact-block form of M (order 1 or 2): per right-hand side
// y = M x_a into ytmp, then F accumulated in Facc (N doubles); pi -= eps F and
// F_out (may be NULL) as launch_force.  2 n_rhs launches.
cudaError_t launch_force_ex(const Geo &g, double h, double A, int order, const double *sigma,
                            const double *L64, const double *x, int n_rhs, double *ytmp, double *Facc,
                            double *pi, double eps, double *F_out, cudaStream_t st);

// Molecular-dynamics schedule of one trajectory as a sequence of forces:
// after force j (j = 0 .. forces - 1, each computed from a fresh solve at the
// current sigma) the momenta take a kick pi -= kick F, then, except after the
// last force, sigma drifts by drift * pi.  Leapfrog (Sec. 4.1): kicks dt/2,
// dt, ..., dt, dt/2 and drifts dt (n_md + 1 forces).  Omelyan's second-order
// minimum-norm scheme (Comput. Phys. Commun. 151 (2003) 272): kicks lambda dt,
// (1 - 2 lambda) dt, 2 lambda dt, ..., (1 - 2 lambda) dt, lambda dt and drifts
// dt/2 (2 n_md + 1 forces), lambda = 1/2 - c/12 + 1/(6c), c = (2 sqrt(326) +
// 36)^(1/3).  Returns the number of forces.
inline int md_schedule(int integrator, int n_md, double dt, int j, double *kick, double *drift)
{
    if (integrator == 1) {
        const double c = cbrt(2.0 * sqrt(326.0) + 36.0);
        const double lam = 0.5 - c / 12.0 + 1.0 / (6.0 * c);
        const int forces = 2 * n_md + 1;
        if (j == 0 || j == forces - 1)
            *kick = lam * dt;
        else
            *kick = (j % 2 == 1) ? (1.0 - 2.0 * lam) * dt : 2.0 * lam * dt;
        *drift = 0.5 * dt;
        return forces;
    }
    const int forces = n_md + 1;
    *kick = (j == 0 || j == forces - 1) ? 0.5 * dt : dt;
    *drift = dt;
    return forces;
}

}  // namespace hh
