// Standalone applies of M, M^T and Q = M^T M (Eq. (10); Q as in Sec. 4.3).
//
// M and M^T are one sweep each over x-contiguous groups of W sites with
// 16-byte loads.  For Q in FP32 on d = 3 lattices whose x-y plane fits in
// shared memory, one fused kernel replaces the two sweeps: a block owns a
// slab of TZ z-planes (all x, y) and marches through a chunk of time slices.
// At each slice it holds in shared memory x(tau+1) on the slab plus two halo
// planes, x(tau) and L(tau) on the slab plus one, t(tau) and t(tau+1) = (M x)
// on the slab plus one halo plane, and writes q(tau) = (M^T t)(tau) for the
// slab.  The slices are brought in by 1-D TMA bulk copies that complete on
// mbarriers, two slices ahead of use, so HBM is read once per site (halo
// re-reads hit L2) and q is written once: 12 bytes per site in FP32.
#include "hh_apply.cuh"

namespace hh {

namespace {

// ---------------------------------------------------------------------------
// Two-sweep path: y = M x (TRANS = false) or y = M^T x (TRANS = true).
// ---------------------------------------------------------------------------
template <int D, typename T, int W, bool TRANS>
__global__ void __launch_bounds__(256) k_apply_group(const Geo g, const T h, const T *__restrict__ L,
                                                     const T *__restrict__ x, T *__restrict__ y)
{
    const int stride = W * gridDim.x * blockDim.x;
    for (int i = W * (blockIdx.x * blockDim.x + threadIdx.x); i < g.N; i += stride) {
        GroupNbr nb;
        group_nbrs<D, W>(g, i, nb);
        Vec<T, W> self = vldg<T, W>(x + i);
        Vec<T, W> hs = group_hop<D, T, W>(x, nb, self);
        Vec<T, W> lk = vldg<T, W>(L + (TRANS ? i : nb.prev));
        Vec<T, W> ov = vldg<T, W>(x + (TRANS ? nb.next : nb.prev));
        Vec<T, W> out;
#pragma unroll
        for (int u = 0; u < W; ++u) out.a[u] = fma(lk.a[u], ov.a[u], fma(-h, hs.a[u], self.a[u]));
        vst<T, W>(y + i, out);
    }
}

template <typename T, bool TRANS>
cudaError_t launch_sweep(const Geo &g, T h, const T *L, const T *x, T *y, cudaStream_t st)
{
    const int w = engine_group_width(g.nx);
    long long groups = g.N / w;
    int blocks = (int)((groups + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
#define HH_SWEEP(D, W) k_apply_group<D, T, W, TRANS><<<blocks, 256, 0, st>>>(g, h, L, x, y)
    if (g.d == 3) {
        if (w == 4) HH_SWEEP(3, 4);
        else if (w == 2) HH_SWEEP(3, 2);
        else HH_SWEEP(3, 1);
    } else {
        if (w == 4) HH_SWEEP(1, 4);
        else if (w == 2) HH_SWEEP(1, 2);
        else HH_SWEEP(1, 1);
    }
#undef HH_SWEEP
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fused FP32 Q = M^T M for d = 3.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Returns true when the phase with the given parity has completed.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// 1-D bulk copy global -> shared completing on an mbarrier (16-byte aligned,
// size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

struct FusedCfg {
    Geo g;
    float h;
    int tz;        // core z-planes per block
    int nslab;     // Nx / tz
    int tc;        // time slices per block
    int P;         // Nx * Nx sites per plane
};

// Planes [z_first, z_first + count) of time slice tau (z periodic) into dst:
// one bulk copy per contiguous run.  Returns the bytes requested.
__device__ __forceinline__ unsigned load_planes(const FusedCfg &c, const float *src, int tau, int z_first,
                                                int count, float *dst, uint64_t *bar)
{
    const int nx = c.g.nx;
    int z = ((z_first % nx) + nx) % nx;
    int done = 0;
    unsigned bytes = 0;
    while (done < count) {
        int run = count - done;
        if (z + run > nx) run = nx - z;
        const float *s = src + (size_t)tau * c.g.V + (size_t)z * c.P;
        unsigned nb = (unsigned)(run * c.P * sizeof(float));
        bulk_g2s(dst + (size_t)done * c.P, s, nb, bar);
        bytes += nb;
        done += run;
        z = 0;
    }
    return bytes;
}

constexpr long long kSpinLimit = 1LL << 26;

// Bounded wait on an mbarrier phase; on timeout sets *err and returns false.
__device__ __forceinline__ bool wait_phase(uint64_t *bar, unsigned parity, int *err)
{
    long long spins = 0;
    while (!mbar_try_wait(bar, parity)) {
        if (++spins > kSpinLimit) {
            atomicCAS(err, 0, -6);
            return false;
        }
    }
    return true;
}

__global__ void __launch_bounds__(512, 1) k_mtm_fused_d3(const FusedCfg c, const float *__restrict__ L,
                                                         const float *__restrict__ x, float *__restrict__ y,
                                                         int *err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bars[2];
    const int P = c.P, tz = c.tz, nx = c.g.nx, ntau = c.g.ntau;
    const int xpl = tz + 4, tpl = tz + 2;  // planes held for x and for t / L
    float *XB = (float *)smem_raw;                     // 3 slices of x
    float *LB = XB + 3 * (size_t)xpl * P;              // 2 slices of L
    float *TB = LB + 2 * (size_t)tpl * P;              // 2 slices of t

    const int slab = blockIdx.x % c.nslab;
    const int chunk = blockIdx.x / c.nslab;
    const int z0 = slab * tz;
    const int tau0 = chunk * c.tc;
    int tau1 = tau0 + c.tc;
    if (tau1 > ntau) tau1 = ntau;
    if (tau0 >= tau1) return;
    const float h = c.h;

    // x slices live in XB slot (tau - tau0 + 1) % 3; L and t slices in slot tau % 2.
    auto xslot = [&](int tau) { return XB + (size_t)(((tau - tau0 + 1) % 3 + 3) % 3) * xpl * P; };
    auto lslot = [&](int tau) { return LB + (size_t)(((tau % 2) + 2) % 2) * tpl * P; };
    auto tslot = [&](int tau) { return TB + (size_t)(((tau % 2) + 2) % 2) * tpl * P; };
    auto wrap_tau = [&](int tau) { return ((tau % ntau) + ntau) % ntau; };

    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    unsigned phase[2] = {0u, 0u};

    // Stage 0: x(tau0-1), x(tau0), L(tau0-1).  Stage 1: x(tau0+1), L(tau0).
    if (threadIdx.x == 0) {
        unsigned bytes = (unsigned)(2 * xpl + tpl) * P * sizeof(float);
        mbar_expect_tx(&bars[0], bytes);
        load_planes(c, x, wrap_tau(tau0 - 1), z0 - 2, xpl, xslot(tau0 - 1), &bars[0]);
        load_planes(c, x, wrap_tau(tau0), z0 - 2, xpl, xslot(tau0), &bars[0]);
        load_planes(c, L, wrap_tau(tau0 - 1), z0 - 1, tpl, lslot(tau0 - 1), &bars[0]);
        bytes = (unsigned)(xpl + tpl) * P * sizeof(float);
        mbar_expect_tx(&bars[1], bytes);
        load_planes(c, x, wrap_tau(tau0 + 1), z0 - 2, xpl, xslot(tau0 + 1), &bars[1]);
        load_planes(c, L, wrap_tau(tau0), z0 - 1, tpl, lslot(tau0), &bars[1]);
    }

    // t(tau) on the slab plus one halo plane from x(tau) (xs) and x(tau-1)
    // (xp, site term) with L(tau-1) (ls).  A thread owns in-plane sites s and
    // walks them through the planes, so the in-plane neighbour offsets are
    // computed once per site and step.
    auto compute_t = [&](const float *xs, const float *xp, const float *ls, float *ts) {
        for (int s = threadIdx.x; s < P; s += blockDim.x) {
            const int yy = s / nx, xx = s - yy * nx;
            const int oxp = yy * nx + (xx + 1 == nx ? 0 : xx + 1), oxm = yy * nx + (xx == 0 ? nx - 1 : xx - 1);
            const int oyp = (yy + 1 == nx ? 0 : yy + 1) * nx + xx, oym = (yy == 0 ? nx - 1 : yy - 1) * nx + xx;
            // x planes q = pz + 1 - 1 .. pz + 1 + 1 around t plane pz; keep a
            // sliding window of the site value along z.
            float below = xs[s], here = xs[(size_t)P + s];
            for (int pz = 0; pz < tpl; ++pz) {
                const float *xc = xs + (size_t)(pz + 1) * P;
                const float above = xc[(size_t)P + s];
                float hop = (xc[oxp] + xc[oxm]) + (xc[oyp] + xc[oym]) + (above + below);
                float v = fmaf(-h, hop, here);
                ts[(size_t)pz * P + s] = fmaf(ls[(size_t)pz * P + s], xp[(size_t)(pz + 1) * P + s], v);
                below = here;
                here = above;
            }
        }
    };

    int stage = 0;
    // Prologue: wait for stage 0, build t(tau0).
    if (!wait_phase(&bars[0], phase[0], err)) return;
    phase[0] ^= 1u;
    compute_t(xslot(tau0), xslot(tau0 - 1), lslot(tau0 - 1), tslot(tau0));
    __syncthreads();

    for (int tau = tau0; tau < tau1; ++tau) {
        stage = (tau - tau0 + 1) & 1;
        // Wait for x(tau+1) and L(tau).
        if (!wait_phase(&bars[stage], phase[stage], err)) return;
        phase[stage] ^= 1u;
        // Prefetch x(tau+2), L(tau+1) into the buffers freed by the last step.
        if (tau + 1 < tau1 && threadIdx.x == 0) {
            const int nb = stage ^ 1;
            unsigned bytes = (unsigned)(xpl + tpl) * P * sizeof(float);
            mbar_expect_tx(&bars[nb], bytes);
            load_planes(c, x, wrap_tau(tau + 2), z0 - 2, xpl, xslot(tau + 2), &bars[nb]);
            load_planes(c, L, wrap_tau(tau + 1), z0 - 1, tpl, lslot(tau + 1), &bars[nb]);
        }
        // t(tau+1) = (M x)(tau+1): site term x(tau) with L(tau).
        compute_t(xslot(tau + 1), xslot(tau), lslot(tau), tslot(tau + 1));
        __syncthreads();
        // q(tau) = t(tau) - h hop(t(tau)) + L(tau) t(tau+1) on the core planes.
        const float *t0 = tslot(tau), *t1 = tslot(tau + 1), *lc = lslot(tau);
        float *yo = y + (size_t)wrap_tau(tau) * c.g.V + (size_t)z0 * P;
        for (int s = threadIdx.x; s < P; s += blockDim.x) {
            const int yy = s / nx, xx = s - yy * nx;
            const int oxp = yy * nx + (xx + 1 == nx ? 0 : xx + 1), oxm = yy * nx + (xx == 0 ? nx - 1 : xx - 1);
            const int oyp = (yy + 1 == nx ? 0 : yy + 1) * nx + xx, oym = (yy == 0 ? nx - 1 : yy - 1) * nx + xx;
            float below = t0[s], here = t0[(size_t)P + s];
            for (int pz = 0; pz < tz; ++pz) {
                const float *tc = t0 + (size_t)(pz + 1) * P;
                const float above = tc[(size_t)P + s];
                float hop = (tc[oxp] + tc[oxm]) + (tc[oyp] + tc[oym]) + (above + below);
                const size_t k = (size_t)(pz + 1) * P + s;
                float v = fmaf(-h, hop, here);
                yo[(size_t)pz * P + s] = fmaf(lc[k], t1[k], v);
                below = here;
                here = above;
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t fused_mtm_smem(int nx, int tz)
{
    size_t P = (size_t)nx * nx;
    return (3 * (size_t)(tz + 4) + 2 * (size_t)(tz + 2) * 2) * P * sizeof(float);
}

bool fused_mtm_ok(const Geo &g, const void *L, const void *x, const void *y)
{
    if (g.d != 3) return false;
    size_t P = (size_t)g.nx * g.nx;
    if ((P * sizeof(float)) % 16) return false;
    if (((uintptr_t)L | (uintptr_t)x) & 15u) return false;
    if (g.nx < 4 || g.ntau < 3) return false;
    int tz = (g.nx % 4 == 0) ? 4 : (g.nx % 2 == 0 ? 2 : 1);
    return fused_mtm_smem(g.nx, tz) <= 200 * 1024;
}

cudaError_t launch_mtm_fused_f32(const Geo &g, float h, const float *L, const float *x, float *y, int *err,
                                 int nsm, cudaStream_t st)
{
    FusedCfg c;
    c.g = g;
    c.h = h;
    c.tz = (g.nx % 4 == 0) ? 4 : (g.nx % 2 == 0 ? 2 : 1);
    c.nslab = g.nx / c.tz;
    c.P = g.nx * g.nx;
    int chunks = (nsm + c.nslab - 1) / c.nslab;
    if (chunks > g.ntau) chunks = g.ntau;
    c.tc = (g.ntau + chunks - 1) / chunks;
    chunks = (g.ntau + c.tc - 1) / c.tc;
    size_t smem = fused_mtm_smem(g.nx, c.tz);
    cudaError_t e = cudaFuncSetAttribute(k_mtm_fused_d3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_mtm_fused_d3<<<c.nslab * chunks, 512, smem, st>>>(c, L, x, y, err);
    return cudaGetLastError();
}

cudaError_t launch_sweep_f64(const Geo &g, bool trans, double h, const double *L, const double *x, double *y,
                             cudaStream_t st)
{
    return trans ? launch_sweep<double, true>(g, h, L, x, y, st) : launch_sweep<double, false>(g, h, L, x, y, st);
}

cudaError_t launch_sweep_f32(const Geo &g, bool trans, float h, const float *L, const float *x, float *y,
                             cudaStream_t st)
{
    return trans ? launch_sweep<float, true>(g, h, L, x, y, st) : launch_sweep<float, false>(g, h, L, x, y, st);
}

}  // namespace hh
