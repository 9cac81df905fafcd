// Non-persistent kernels of the HMC path (Sec. 4.1): links, stencil applies,
// Philox draws, the pseudofermion force with the fused momentum update, the
// sigma step, energy reductions and the Metropolis test.
#include <cuda_bf16.h>

#include "hh_kernels.cuh"

namespace hh {

namespace {

constexpr int kBlock = 256;

inline int grid_for(long long n, int per_thread = 1)
{
    long long b = (n + (long long)kBlock * per_thread - 1) / ((long long)kBlock * per_thread);
    if (b < 1) b = 1;
    if (b > 65535LL * 16) b = 65535LL * 16;
    return (int)b;
}

__device__ __forceinline__ double link_value(const Geo &g, double A, double sigma, int i)
{
    uint32_t tau = fd_div((uint32_t)i, g.f_V);
    double c = 1.0 + A * sin(sigma);
    return ((int)tau == g.ntau - 1) ? c : -c;
}

__global__ void k_links(Geo g, double A, const double *__restrict__ sigma, double *__restrict__ L64,
                        float *__restrict__ L32)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += gridDim.x * blockDim.x) {
        double l = link_value(g, A, sigma[i], i);
        L64[i] = l;
        L32[i] = (float)l;
    }
}

__global__ void k_sigma_step(Geo g, double A, double dt, double *__restrict__ sigma,
                             const double *__restrict__ pi, double *__restrict__ L64,
                             float *__restrict__ L32)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += gridDim.x * blockDim.x) {
        double s = fma(dt, pi[i], sigma[i]);
        sigma[i] = s;
        double l = link_value(g, A, s, i);
        L64[i] = l;
        L32[i] = (float)l;
    }
}

template <typename T>
__global__ void k_apply(Geo g, int op, T h, const T *__restrict__ L, const T *__restrict__ x,
                        T *__restrict__ y, int order)
{
    Nbr nb;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += gridDim.x * blockDim.x) {
        neighbours(g, i, nb);
        if (order == 0)
            y[i] = (op == 0) ? stencil_M<T>(g, h, L, x, i, nb) : stencil_MT<T>(g, h, L, x, i, nb);
        else
            y[i] = (op == 0) ? stencil_M_ex<T>(g, h, L, x, i, nb, order)
                             : stencil_MT_ex<T>(g, h, L, x, i, nb, order);
    }
}

// One thread per Philox block of four elements.
__global__ void k_gaussian(double *__restrict__ out, int n, uint64_t seed, uint64_t ctr1,
                           uint64_t traj, uint64_t chain)
{
    const double two_pi = 6.283185307179586476925286766559;
    int nblk = (n + 3) >> 2;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        U64x4 w = philox4x64_10((uint64_t)b, ctr1, traj, chain, seed, 0);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            double u1 = u53(w.v[2 * j]), u2 = u53(w.v[2 * j + 1]);
            double rad = sqrt(-2.0 * log(1.0 - u1));
            double th = two_pi * u2;
            int i0 = 4 * b + 2 * j;
            if (i0 < n) out[i0] = rad * cos(th);
            if (i0 + 1 < n) out[i0 + 1] = rad * sin(th);
        }
    }
}

__global__ void k_init_field(double *__restrict__ sigma, int n, uint64_t seed, uint64_t chain)
{
    const double pi = 3.14159265358979323846264338328;
    int nblk = (n + 3) >> 2;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        U64x4 w = philox4x64_10((uint64_t)b, 0, 0, chain, seed, 0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int i = 4 * b + j;
            // Explicit roundings: (-pi) + (2 pi) u with no fused multiply-add.
            if (i < n) sigma[i] = __dadd_rn(-pi, __dmul_rn(2.0 * pi, u53(w.v[j])));
        }
    }
}

// F_i = -sum_a (M x_a)(next(i)) s(tau_i) A cos(sigma_i) x_a(i).
__global__ void k_force(Geo g, double h, double A, const double *__restrict__ sigma,
                        const double *__restrict__ L64, const double *__restrict__ x, int n_rhs,
                        double *__restrict__ pi, double eps, double *__restrict__ F_out)
{
    Nbr nb, nn;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += gridDim.x * blockDim.x) {
        neighbours(g, i, nb);
        const int j = nb.next;
        neighbours(g, j, nn);
        uint32_t tau = fd_div((uint32_t)i, g.f_V);
        double s = ((int)tau == g.ntau - 1) ? 1.0 : -1.0;
        double coef = s * A * cos(sigma[i]);
        double F = 0.0;
        for (int a = 0; a < n_rhs; ++a) {
            const double *xa = x + (size_t)a * g.N;
            double y = stencil_M<double>(g, h, L64, xa, j, nn);
            F -= y * coef * xa[i];
        }
        if (F_out) F_out[i] = F;
        if (pi) pi[i] = fma(-eps, F, pi[i]);
    }
}

// Exact-block form: sigma(n,tau) enters through w = L x at (n,tau), which row
// (., tau+1) sees through E, so y's factor is (E y)(n, tau+1) with y = M x_a
// (ya, precomputed).  Accumulates over right-hand sides in Facc; the last one
// writes F_out and updates pi.
__global__ void k_force_ex(Geo g, double h, double A, int order, const double *__restrict__ sigma,
                           const double *__restrict__ L64, const double *__restrict__ xa,
                           const double *__restrict__ ya, double *__restrict__ Facc, int first, int last,
                           double *__restrict__ pi, double eps, double *__restrict__ F_out)
{
    Nbr nb;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += gridDim.x * blockDim.x) {
        neighbours(g, i, nb);
        uint32_t tau = fd_div((uint32_t)i, g.f_V);
        double s = ((int)tau == g.ntau - 1) ? 1.0 : -1.0;
        double coef = s * A * cos(sigma[i]);
        double e = e_factor<double, false>(g, h, L64, ya, nb.next, order);
        double F = (first ? 0.0 : Facc[i]) - e * coef * xa[i];
        if (last) {
            if (F_out) F_out[i] = F;
            if (pi) pi[i] = fma(-eps, F, pi[i]);
        } else {
            Facc[i] = F;
        }
    }
}

constexpr int kEnergyMaxBlocks = 1024;

__global__ void k_energy(int n, const double *__restrict__ pi, const double *__restrict__ chi,
                         const double *__restrict__ x, int n_rhs, double *__restrict__ part)
{
    __shared__ double red[kBlock / 32];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double e = 0.0;
        if (pi) e = pi[i] * pi[i];
        for (int a = 0; a < n_rhs; ++a) e = fma(chi[(size_t)a * n + i], x[(size_t)a * n + i], e);
        acc += 0.5 * e;
    }
    double tot = block_sum(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void k_sum_partials(const double *__restrict__ part, int nb, double *__restrict__ out)
{
    double v = 0.0;
    for (int j = threadIdx.x; j < nb; j += 32) v += part[j];
    v = warp_sum(v);
    if (threadIdx.x == 0) *out = v;
}

// 16-bit links of the FP32 steps from the FP64 links: mode 1 the bfloat16
// rounding (to nearest even) of the FP32 value, mode 2 the fixed-point code
// rint(L / scale) (|L| / scale < 2^15 by the choice of scale).
__global__ void k_links16(int n, const double *__restrict__ L64, unsigned short *__restrict__ L16, int mode,
                          double inv_scale)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = L64[i];
        unsigned short u;
        if (mode == 1)
            u = __bfloat16_as_ushort(__float2bfloat16_rn(__double2float_rn(v)));
        else
            u = (unsigned short)(short)__double2int_rn(v * inv_scale);
        L16[i] = u;
    }
}

// Z2 noise of the observables: vector k = blockIdx.y (+ gridDim.y steps) at
// out + k n; element i is +1 when the top bit of word i & 3 of Philox block
// i >> 2 (tag 6, a = k) is set, else -1.
__global__ void k_z2_noise(double *__restrict__ out, int n, int nvec, uint64_t seed, uint64_t traj,
                           uint64_t chain)
{
    const int nblk = (n + 3) >> 2;
    for (int k = blockIdx.y; k < nvec; k += gridDim.y) {
        const uint64_t ctr1 = 6u | ((uint64_t)k << 8);
        double *o = out + (size_t)k * n;
        for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
            U64x4 w = philox4x64_10((uint64_t)b, ctr1, traj, chain, seed, 0);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = 4 * b + j;
                if (i < n) o[i] = (w.v[j] >> 63) ? 1.0 : -1.0;
            }
        }
    }
}

// Block partials of the observables: for blockIdx.y = k < nvec the dot
// eta_k . y_k into part[k nb + b]; for blockIdx.y = nvec the site sums of
// (1 - gA)(1 - gB), sin sigma and sin^2 sigma into part[(nvec + j) nb + b],
// gA and gB being the means of eta_k y_k over the first and second halves of
// the vectors.
__global__ void k_obs_partials(int n, int nvec, const double *__restrict__ eta, const double *__restrict__ y,
                               const double *__restrict__ sigma, double *__restrict__ part)
{
    __shared__ double red[kBlock / 32];
    const int nb = gridDim.x, k = blockIdx.y;
    if (k < nvec) {
        const double *e = eta + (size_t)k * n, *v = y + (size_t)k * n;
        double acc = 0.0;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += nb * blockDim.x) acc = fma(e[i], v[i], acc);
        const double tot = block_sum(acc, red);
        if (threadIdx.x == 0) part[(size_t)k * nb + blockIdx.x] = tot;
        return;
    }
    const int half = nvec / 2;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += nb * blockDim.x) {
        double gA = 0.0, gB = 0.0;
        for (int q = 0; q < half; ++q) gA = fma(eta[(size_t)q * n + i], y[(size_t)q * n + i], gA);
        for (int q = half; q < nvec; ++q) gB = fma(eta[(size_t)q * n + i], y[(size_t)q * n + i], gB);
        gA /= half;
        gB /= half;
        a0 = fma(1.0 - gA, 1.0 - gB, a0);
        const double sn = sin(sigma[i]);
        a1 += sn;
        a2 = fma(sn, sn, a2);
    }
    double tot = block_sum(a0, red);
    if (threadIdx.x == 0) part[(size_t)nvec * nb + blockIdx.x] = tot;
    __syncthreads();
    tot = block_sum(a1, red);
    if (threadIdx.x == 0) part[(size_t)(nvec + 1) * nb + blockIdx.x] = tot;
    __syncthreads();
    tot = block_sum(a2, red);
    if (threadIdx.x == 0) part[(size_t)(nvec + 2) * nb + blockIdx.x] = tot;
}

// One warp: sums each quantity's nb partials in a fixed order and writes
// out[0] = mean over k of t_k = dot_k / n, out[1] = its standard error,
// out[2..4] = the three site sums over n.
__global__ void k_obs_finish(const double *__restrict__ part, int nb, int nvec, int n, double *__restrict__ out)
{
    __shared__ double q[kObsMaxNoise + 3];
    for (int j = 0; j < nvec + 3; ++j) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nb; b += 32) v += part[(size_t)j * nb + b];
        v = warp_sum(v);
        if (threadIdx.x == 0) q[j] = v / (double)n;
    }
    if (threadIdx.x != 0) return;
    double mean = 0.0, var = 0.0;
    for (int k = 0; k < nvec; ++k) mean += q[k];
    mean /= nvec;
    for (int k = 0; k < nvec; ++k) var += (q[k] - mean) * (q[k] - mean);
    var /= (nvec - 1);
    out[0] = mean;
    out[1] = sqrt(var / nvec);
    out[2] = q[nvec];
    out[3] = q[nvec + 1];
    out[4] = q[nvec + 2];
}

__global__ void k_metropolis(HmcScalars *sc, uint64_t seed, uint64_t traj, uint64_t chain)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double dH = sc->H1 - sc->H0;
    U64x4 w = philox4x64_10(0, 3, traj, chain, seed, 0);
    double u = u53(w.v[0]);
    sc->dH = dH;
    sc->u = u;
    sc->accepted = (u < exp(-dH)) ? 1 : 0;
}

__global__ void k_restore(Geo g, double A, const HmcScalars *__restrict__ sc, double *__restrict__ sigma,
                          const double *__restrict__ sigma0, double *__restrict__ L64,
                          float *__restrict__ L32)
{
    if (sc->accepted) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += gridDim.x * blockDim.x) {
        double s = sigma0[i];
        sigma[i] = s;
        double l = link_value(g, A, s, i);
        L64[i] = l;
        L32[i] = (float)l;
    }
}

}  // namespace

cudaError_t launch_links(const Geo &g, double A, const double *sigma, double *L64, float *L32,
                         cudaStream_t st)
{
    k_links<<<grid_for(g.N), kBlock, 0, st>>>(g, A, sigma, L64, L32);
    return cudaGetLastError();
}

cudaError_t launch_sigma_step(const Geo &g, double A, double dt, double *sigma, const double *pi,
                              double *L64, float *L32, cudaStream_t st)
{
    k_sigma_step<<<grid_for(g.N), kBlock, 0, st>>>(g, A, dt, sigma, pi, L64, L32);
    return cudaGetLastError();
}

cudaError_t launch_apply_f64(const Geo &g, int op, double h, const double *L, const double *x,
                             double *y, cudaStream_t st, int order)
{
    k_apply<double><<<grid_for(g.N), kBlock, 0, st>>>(g, op, h, L, x, y, order);
    return cudaGetLastError();
}

cudaError_t launch_apply_f32(const Geo &g, int op, float h, const float *L, const float *x, float *y,
                             cudaStream_t st, int order)
{
    k_apply<float><<<grid_for(g.N), kBlock, 0, st>>>(g, op, h, L, x, y, order);
    return cudaGetLastError();
}

cudaError_t launch_gaussian(double *out, int n, uint64_t seed, int tag, int a, uint64_t traj,
                            uint64_t chain, cudaStream_t st)
{
    uint64_t ctr1 = (uint64_t)tag | ((uint64_t)a << 8);
    k_gaussian<<<grid_for((n + 3) / 4), kBlock, 0, st>>>(out, n, seed, ctr1, traj, chain);
    return cudaGetLastError();
}

cudaError_t launch_init_field(double *sigma, int n, uint64_t seed, uint64_t chain, cudaStream_t st)
{
    k_init_field<<<grid_for((n + 3) / 4), kBlock, 0, st>>>(sigma, n, seed, chain);
    return cudaGetLastError();
}

cudaError_t launch_force(const Geo &g, double h, double A, const double *sigma, const double *L64,
                         const double *x, int n_rhs, double *pi, double eps, double *F_out,
                         cudaStream_t st)
{
    k_force<<<grid_for(g.N), kBlock, 0, st>>>(g, h, A, sigma, L64, x, n_rhs, pi, eps, F_out);
    return cudaGetLastError();
}

cudaError_t launch_force_ex(const Geo &g, double h, double A, int order, const double *sigma,
                            const double *L64, const double *x, int n_rhs, double *ytmp, double *Facc,
                            double *pi, double eps, double *F_out, cudaStream_t st)
{
    for (int a = 0; a < n_rhs; ++a) {
        const double *xa = x + (size_t)a * g.N;
        cudaError_t e = launch_apply_f64(g, 0, h, L64, xa, ytmp, st, order);
        if (e != cudaSuccess) return e;
        k_force_ex<<<grid_for(g.N), kBlock, 0, st>>>(g, h, A, order, sigma, L64, xa, ytmp, Facc, a == 0,
                                                      a == n_rhs - 1, pi, eps, F_out);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int energy_blocks(int n)
{
    int b = (n + kBlock - 1) / kBlock;
    if (b > kEnergyMaxBlocks) b = kEnergyMaxBlocks;
    if (b < 1) b = 1;
    return b;
}

cudaError_t launch_energy(int n, const double *pi, const double *chi, const double *x, int n_rhs,
                          double *part, double *out, cudaStream_t st)
{
    int nb = energy_blocks(n);
    k_energy<<<nb, kBlock, 0, st>>>(n, pi, chi, x, n_rhs, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sum_partials<<<1, 32, 0, st>>>(part, nb, out);
    return cudaGetLastError();
}

cudaError_t launch_links16(int n, const double *L64, unsigned short *L16, int mode, double scale, cudaStream_t st)
{
    k_links16<<<grid_for(n), kBlock, 0, st>>>(n, L64, L16, mode, 1.0 / scale);
    return cudaGetLastError();
}

cudaError_t launch_z2_noise(double *out, int n, int nvec, uint64_t seed, uint64_t traj, uint64_t chain,
                            cudaStream_t st)
{
    dim3 grid(grid_for((n + 3) / 4), nvec);
    k_z2_noise<<<grid, kBlock, 0, st>>>(out, n, nvec, seed, traj, chain);
    return cudaGetLastError();
}

cudaError_t launch_observables(int n, int nvec, const double *eta, const double *y, const double *sigma,
                               double *part, double *out, cudaStream_t st)
{
    if (nvec < 2 || nvec > kObsMaxNoise || (nvec & 1)) return cudaErrorInvalidValue;
    const int nb = energy_blocks(n);
    k_obs_partials<<<dim3(nb, nvec + 1), kBlock, 0, st>>>(n, nvec, eta, y, sigma, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_obs_finish<<<1, 32, 0, st>>>(part, nb, nvec, n, out);
    return cudaGetLastError();
}

cudaError_t launch_metropolis(HmcScalars *sc, uint64_t seed, uint64_t traj, uint64_t chain,
                              cudaStream_t st)
{
    k_metropolis<<<1, 32, 0, st>>>(sc, seed, traj, chain);
    return cudaGetLastError();
}

cudaError_t launch_restore(const Geo &g, double A, const HmcScalars *sc, double *sigma,
                           const double *sigma0, double *L64, float *L32, cudaStream_t st)
{
    k_restore<<<grid_for(g.N), kBlock, 0, st>>>(g, A, sc, sigma, sigma0, L64, L32);
    return cudaGetLastError();
}

namespace {

__global__ void k_extrapolate(double *__restrict__ x, double *__restrict__ xp, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double t = x[i];
        x[i] = fma(2.0, t, -xp[i]);
        xp[i] = t;
    }
}

}  // namespace

cudaError_t launch_extrapolate(double *x, double *xp, long long n, cudaStream_t st)
{
    long long blocks = (n + kBlock - 1) / kBlock;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_extrapolate<<<(int)blocks, kBlock, 0, st>>>(x, xp, n);
    return cudaGetLastError();
}

}  // namespace hh
