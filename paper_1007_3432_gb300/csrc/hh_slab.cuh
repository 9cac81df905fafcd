// Device helpers of the shared-memory slab kernels (the fused and the
// multi-vector FP32 Q = M^T M applies for d = 3): 1-D TMA bulk copies into
// shared memory completing on mbarriers, L2 bulk prefetches, and the in-plane
// stencil of one float4 group of x sites.  A slab holds whole x-y planes
// (P = Nx * Nx sites each) of consecutive z, periodic in z.
#pragma once

#include "hh_device.cuh"

namespace hh {

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

// Bulk prefetch of [src, src + bytes) into L2 (16-byte aligned, multiple of 16).
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Planes [z_first, z_first + count) of time slice tau (z periodic) into dst:
// one bulk copy per contiguous run.  Returns the bytes requested.
__device__ __forceinline__ unsigned load_planes(const Geo &g, int P, const float *src, int tau, int z_first,
                                                int count, float *dst, uint64_t *bar)
{
    const int nx = g.nx;
    int z = ((z_first % nx) + nx) % nx;
    int done = 0;
    unsigned bytes = 0;
    while (done < count) {
        int run = count - done;
        if (z + run > nx) run = nx - z;
        const float *s = src + (size_t)tau * g.V + (size_t)z * P;
        unsigned nb = (unsigned)(run * P * sizeof(float));
        bulk_g2s(dst + (size_t)done * P, s, nb, bar);
        bytes += nb;
        done += run;
        z = 0;
    }
    return bytes;
}

// Planes [z_first, z_first + count) of slice tau into L2, one request per run.
__device__ __forceinline__ void prefetch_planes(const Geo &g, int P, const float *src, int tau, int z_first,
                                                int count)
{
    const int nx = g.nx;
    int z = ((z_first % nx) + nx) % nx;
    int done = 0;
    while (done < count) {
        int run = count - done;
        if (z + run > nx) run = nx - z;
        bulk_prefetch_l2(src + (size_t)tau * g.V + (size_t)z * P, (unsigned)(run * P * sizeof(float)));
        done += run;
        z = 0;
    }
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

// In-plane geometry of one thread's float4 group: 4 consecutive x sites at
// in-plane offset s (x0 = s mod Nx is a multiple of 4), the single sites just
// before and after the group along x, and the groups one row up / down in y.
struct PlaneGroup {
    int s, xm, xp, yp, ym;
};

__device__ __forceinline__ PlaneGroup plane_group(int g, int nx)
{
    PlaneGroup q;
    const int s = 4 * g;
    const int yy = s / nx, x0 = s - yy * nx;
    q.s = s;
    q.xm = yy * nx + (x0 == 0 ? nx - 1 : x0 - 1);
    q.xp = yy * nx + (x0 + 4 == nx ? 0 : x0 + 4);
    q.yp = (yy + 1 == nx ? 0 : yy + 1) * nx + x0;
    q.ym = (yy == 0 ? nx - 1 : yy - 1) * nx + x0;
    return q;
}

__device__ __forceinline__ float4 ld4(const float *p)
{
    return *reinterpret_cast<const float4 *>(p);
}

// One plane of the stencil for a float4 group: out = c - h hop(c) + l * o,
// with the z neighbours 'below' and 'above' already loaded.
// The x neighbours outside the group come from the adjacent lanes' groups
// when a row of groups lies inside one warp (shfl), else from shared memory.
__device__ __forceinline__ void x_halo(const float *c, const PlaneGroup &q, const float4 &self, bool shfl,
                                       int src_m, int src_p, float &xm, float &xp)
{
    if (shfl) {
        xm = __shfl_sync(0xffffffffu, self.w, src_m);
        xp = __shfl_sync(0xffffffffu, self.x, src_p);
    } else {
        xm = c[q.xm];
        xp = c[q.xp];
    }
}

__device__ __forceinline__ float4 plane_stencil(const float *c, const PlaneGroup &q, float4 self, float4 below,
                                                float4 above, float4 l, float4 o, float h, float xm, float xp)
{
    const float4 yp = ld4(c + q.yp), ym = ld4(c + q.ym);
    float4 r;
    r.x = fmaf(l.x, o.x, fmaf(-h, (xm + self.y) + (yp.x + ym.x) + (above.x + below.x), self.x));
    r.y = fmaf(l.y, o.y, fmaf(-h, (self.x + self.z) + (yp.y + ym.y) + (above.y + below.y), self.y));
    r.z = fmaf(l.z, o.z, fmaf(-h, (self.y + self.w) + (yp.z + ym.z) + (above.z + below.z), self.z));
    r.w = fmaf(l.w, o.w, fmaf(-h, (self.z + xp) + (yp.w + ym.w) + (above.w + below.w), self.w));
    return r;
}

__device__ __forceinline__ void st4(float *p, const float4 &v)
{
    *reinterpret_cast<float4 *>(p) = v;
}

// L2 eviction policies for the cache-hint forms below: evict_last for data
// that other CTAs read again during the kernel, evict_first for data written
// once and not read again.
__device__ __forceinline__ uint64_t l2_policy_evict_last()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ uint64_t l2_policy_evict_first()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// bulk_g2s with an L2 cache policy.
__device__ __forceinline__ void bulk_g2s_hint(void *dst, const void *src, unsigned bytes, uint64_t *bar,
                                              uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

// load_planes with an L2 cache policy on the copies.
__device__ __forceinline__ unsigned load_planes_hint(const Geo &g, int P, const float *src, int tau, int z_first,
                                                     int count, float *dst, uint64_t *bar, uint64_t pol)
{
    const int nx = g.nx;
    int z = ((z_first % nx) + nx) % nx;
    int done = 0;
    unsigned bytes = 0;
    while (done < count) {
        int run = count - done;
        if (z + run > nx) run = nx - z;
        const float *s = src + (size_t)tau * g.V + (size_t)z * P;
        unsigned nb = (unsigned)(run * P * sizeof(float));
        bulk_g2s_hint(dst + (size_t)done * P, s, nb, bar, pol);
        bytes += nb;
        done += run;
        z = 0;
    }
    return bytes;
}

// 16-byte read-only global load that does not allocate in L1, with an L2
// cache policy.
// Not volatile: the compiler may schedule it like any load of read-only data.
__device__ __forceinline__ float4 ldg4_hint(const float *p, uint64_t pol)
{
    float4 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p), "l"(pol));
    return v;
}

// 16-byte global store with an L2 cache policy.  No memory clobber: it is
// meant for output that the kernel does not read back, so the compiler may
// move other memory operations across it.
__device__ __forceinline__ void st4_global_hint(float *p, const float4 &v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w), "l"(pol));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

}  // namespace hh
