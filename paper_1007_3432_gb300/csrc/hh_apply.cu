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
#include <cstdlib>

#include "hh_apply.cuh"
#include "hh_slab.cuh"

namespace hh {

namespace {

// ---------------------------------------------------------------------------
// Two-sweep path: y = M x (TRANS = false) or y = M^T x (TRANS = true).
// ---------------------------------------------------------------------------
template <int D, typename T, int W, bool TRANS>
__global__ void __launch_bounds__(256) k_apply_group(const Geo g, const T h, const T *__restrict__ L,
                                                     const T *__restrict__ x, T *__restrict__ y)
{
    // Programmatic dependent launch: a sweep launched after this one with
    // programmatic stream serialization may start its blocks once every block
    // here has started; it waits below, until this grid has completed and
    // its writes are visible, before reading.  Without that launch attribute
    // both instructions return at once.
    asm volatile("griddepcontrol.launch_dependents;");
    asm volatile("griddepcontrol.wait;" ::: "memory");
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

template <typename K, typename T>
cudaError_t launch_group_kernel(K kern, int blocks, bool pdl, cudaStream_t st, const Geo &g, T h, const T *L,
                                const T *x, T *y)
{
    if (!pdl) {
        kern<<<blocks, 256, 0, st>>>(g, h, L, x, y);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, g, h, L, x, y);
}

template <typename T, bool TRANS>
cudaError_t launch_sweep(const Geo &g, T h, const T *L, const T *x, T *y, cudaStream_t st, bool pdl)
{
    const int w = engine_group_width(g.nx);
    long long groups = g.N / w;
    int blocks = (int)((groups + 255) / 256);
    // Grid cap: 16 blocks per SM of the 152 (HH_APPLY_SWEEP_BLOCKS overrides
    // it, 0 removes it; measured on GB300 the same or slower either way).
    static const int cap = [] {
        const char *env = getenv("HH_APPLY_SWEEP_BLOCKS");
        return env ? atoi(env) : 152 * 16;
    }();
    if (cap > 0 && blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
#define HH_SWEEP(D, W) \
    return launch_group_kernel(k_apply_group<D, T, W, TRANS>, blocks, pdl, st, g, h, L, x, y)
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
struct FusedCfg {
    Geo g;
    float h;
    int tz;        // core z-planes per block
    int nslab;     // Nx / tz
    int tc;        // time slices per block
    int P;         // Nx * Nx sites per plane
};

constexpr int kFusedThreads = 512;

template <int TZ>
__global__ void __launch_bounds__(kFusedThreads, 1) k_mtm_fused_d3(const FusedCfg c, const float *__restrict__ L,
                                                         const float *__restrict__ x, float *__restrict__ y,
                                                         int *err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bars[2];
    constexpr int XPL = TZ + 4, TPL = TZ + 2;  // planes held for x and for t / L
    const int P = c.P, nx = c.g.nx, ntau = c.g.ntau, V = c.g.V;
    float *XB = (float *)smem_raw;                     // 3 slices of x
    float *LB = XB + 3 * XPL * P;                      // 2 slices of L
    float *TB = LB + 2 * TPL * P;                      // 2 slices of t

    const int slab = blockIdx.x % c.nslab;
    const int chunk = blockIdx.x / c.nslab;
    const int z0 = slab * TZ;
    const int tau0 = chunk * c.tc;
    int tau1 = tau0 + c.tc;
    if (tau1 > ntau) tau1 = ntau;
    if (tau0 >= tau1) return;
    const float h = c.h;

    // Thread -> (float4 group in the plane, range of planes).
    const int G = P / 4;
    const int R = (int)blockDim.x / G > 0 ? (int)blockDim.x / G : 1;
    const int g = threadIdx.x % G, r = threadIdx.x / G;
    const bool worker = r < R && (int)threadIdx.x < R * G;
    const PlaneGroup q = plane_group(g, nx);
    const int t_per = (TPL + R - 1) / R, t_lo = r * t_per, t_hi = min(TPL, t_lo + t_per);
    const int c_per = (TZ + R - 1) / R, c_lo = r * c_per, c_hi = min(TZ, c_lo + c_per);
    // Shuffles for the x halo when the groups of a row are consecutive lanes
    // of one warp and every lane of the warp is a worker on the same planes.
    const int gpr = nx / 4, lane = threadIdx.x & 31, j = lane % gpr;
    const bool shfl = (32 % gpr == 0) && (G % 32 == 0) && (R * G == (int)blockDim.x);
    const int src_m = (j == 0) ? lane + gpr - 1 : lane - 1;
    const int src_p = (j == gpr - 1) ? lane - gpr + 1 : lane + 1;

    auto xslot = [&](int tau) { return XB + (((tau - tau0 + 1) % 3 + 3) % 3) * XPL * P; };
    auto lslot = [&](int tau) { return LB + (((tau % 2) + 2) % 2) * TPL * P; };
    auto tslot = [&](int tau) { return TB + (((tau % 2) + 2) % 2) * TPL * P; };
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
        unsigned bytes = (unsigned)(2 * XPL + TPL) * P * sizeof(float);
        mbar_expect_tx(&bars[0], bytes);
        load_planes(c.g, c.P, x, wrap_tau(tau0 - 1), z0 - 2, XPL, xslot(tau0 - 1), &bars[0]);
        load_planes(c.g, c.P, x, wrap_tau(tau0), z0 - 2, XPL, xslot(tau0), &bars[0]);
        load_planes(c.g, c.P, L, wrap_tau(tau0 - 1), z0 - 1, TPL, lslot(tau0 - 1), &bars[0]);
        bytes = (unsigned)(XPL + TPL) * P * sizeof(float);
        mbar_expect_tx(&bars[1], bytes);
        load_planes(c.g, c.P, x, wrap_tau(tau0 + 1), z0 - 2, XPL, xslot(tau0 + 1), &bars[1]);
        load_planes(c.g, c.P, L, wrap_tau(tau0), z0 - 1, TPL, lslot(tau0), &bars[1]);
        // Keep HBM streaming ahead of the shared-memory stages.
        for (int a = 2; a <= 4 && tau0 + a - 1 < tau1; ++a) {
            prefetch_planes(c.g, c.P, x, wrap_tau(tau0 + a), z0 - 2, XPL);
            prefetch_planes(c.g, c.P, L, wrap_tau(tau0 + a - 1), z0 - 1, TPL);
        }
    }

    // t(tau) on planes [t_lo, t_hi) of the slab plus one halo plane: x plane
    // pz + 1 of xs is aligned with t plane pz; xp is x(tau-1), ls is L(tau-1).
    auto compute_t = [&](const float *xs, const float *xp, const float *ls, float *ts) {
        if (!worker || t_lo >= t_hi) return;
        float4 below = ld4(xs + t_lo * P + q.s), here = ld4(xs + (t_lo + 1) * P + q.s);
        for (int pz = t_lo; pz < t_hi; ++pz) {
            const float *xc = xs + (pz + 1) * P;
            const float4 above = ld4(xc + P + q.s);
            const float4 l = ld4(ls + pz * P + q.s), o = ld4(xp + (pz + 1) * P + q.s);
            float hm, hp;
            x_halo(xc, q, here, shfl, src_m, src_p, hm, hp);
            *reinterpret_cast<float4 *>(ts + pz * P + q.s) = plane_stencil(xc, q, here, below, above, l, o, h, hm, hp);
            below = here;
            here = above;
        }
    };

    // Prologue: wait for stage 0, build t(tau0).
    if (!wait_phase(&bars[0], phase[0], err)) return;
    phase[0] ^= 1u;
    compute_t(xslot(tau0), xslot(tau0 - 1), lslot(tau0 - 1), tslot(tau0));
    __syncthreads();

    for (int tau = tau0; tau < tau1; ++tau) {
        const int stage = (tau - tau0 + 1) & 1;
        // Wait for x(tau+1) and L(tau).
        if (!wait_phase(&bars[stage], phase[stage], err)) return;
        phase[stage] ^= 1u;
        // Prefetch x(tau+2), L(tau+1) into the buffers freed by the last step.
        if (tau + 1 < tau1 && threadIdx.x == 0) {
            const int nb = stage ^ 1;
            unsigned bytes = (unsigned)(XPL + TPL) * P * sizeof(float);
            mbar_expect_tx(&bars[nb], bytes);
            load_planes(c.g, c.P, x, wrap_tau(tau + 2), z0 - 2, XPL, xslot(tau + 2), &bars[nb]);
            load_planes(c.g, c.P, L, wrap_tau(tau + 1), z0 - 1, TPL, lslot(tau + 1), &bars[nb]);
            if (tau + 4 < tau1) {
                prefetch_planes(c.g, c.P, x, wrap_tau(tau + 5), z0 - 2, XPL);
                prefetch_planes(c.g, c.P, L, wrap_tau(tau + 4), z0 - 1, TPL);
            }
        }
        // t(tau+1) = (M x)(tau+1): site term x(tau) with L(tau).
        compute_t(xslot(tau + 1), xslot(tau), lslot(tau), tslot(tau + 1));
        __syncthreads();
        // q(tau) = t(tau) - h hop(t(tau)) + L(tau) t(tau+1) on core planes [c_lo, c_hi).
        if (worker && c_lo < c_hi) {
            const float *t0 = tslot(tau), *t1 = tslot(tau + 1), *lc = lslot(tau);
            float *yo = y + wrap_tau(tau) * V + z0 * P;
            float4 below = ld4(t0 + c_lo * P + q.s), here = ld4(t0 + (c_lo + 1) * P + q.s);
            for (int pz = c_lo; pz < c_hi; ++pz) {
                const float *tc = t0 + (pz + 1) * P;
                const float4 above = ld4(tc + P + q.s);
                const int k = (pz + 1) * P + q.s;
                const float4 l = ld4(lc + k), o = ld4(t1 + k);
                float hm, hp;
                x_halo(tc, q, here, shfl, src_m, src_p, hm, hp);
                *reinterpret_cast<float4 *>(yo + pz * P + q.s) =
                    plane_stencil(tc, q, here, below, above, l, o, h, hm, hp);
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

static int fused_tz(int nx)
{
    return (nx % 4 == 0 && nx >= 8) ? 4 : 2;
}

bool fused_mtm_ok(const Geo &g, const void *L, const void *x, const void *y)
{
    if (g.d != 3 || g.nx % 4 != 0 || g.nx < 4 || g.ntau < 3) return false;
    if (((uintptr_t)L | (uintptr_t)x | (uintptr_t)y) & 15u) return false;
    if ((size_t)g.nx * g.nx / 4 > 1024) return false;   // one float4 group per thread at least
    return fused_mtm_smem(g.nx, fused_tz(g.nx)) <= 200 * 1024;
}

cudaError_t launch_mtm_fused_f32(const Geo &g, float h, const float *L, const float *x, float *y, int *err,
                                 int nsm, cudaStream_t st)
{
    FusedCfg c;
    c.g = g;
    c.h = h;
    c.tz = fused_tz(g.nx);
    c.nslab = g.nx / c.tz;
    c.P = g.nx * g.nx;
    int chunks = (nsm + c.nslab - 1) / c.nslab;
    if (chunks > g.ntau) chunks = g.ntau;
    c.tc = (g.ntau + chunks - 1) / chunks;
    chunks = (g.ntau + c.tc - 1) / c.tc;
    size_t smem = fused_mtm_smem(g.nx, c.tz);
    cudaError_t e;
    if (c.tz == 4) {
        e = cudaFuncSetAttribute(k_mtm_fused_d3<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_mtm_fused_d3<4><<<c.nslab * chunks, kFusedThreads, smem, st>>>(c, L, x, y, err);
    } else {
        e = cudaFuncSetAttribute(k_mtm_fused_d3<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_mtm_fused_d3<2><<<c.nslab * chunks, kFusedThreads, smem, st>>>(c, L, x, y, err);
    }
    return cudaGetLastError();
}

cudaError_t launch_sweep_f64(const Geo &g, bool trans, double h, const double *L, const double *x, double *y,
                             cudaStream_t st, bool pdl)
{
    return trans ? launch_sweep<double, true>(g, h, L, x, y, st, pdl)
                 : launch_sweep<double, false>(g, h, L, x, y, st, pdl);
}

cudaError_t launch_sweep_f32(const Geo &g, bool trans, float h, const float *L, const float *x, float *y,
                             cudaStream_t st, bool pdl)
{
    return trans ? launch_sweep<float, true>(g, h, L, x, y, st, pdl)
                 : launch_sweep<float, false>(g, h, L, x, y, st, pdl);
}

}  // namespace hh
