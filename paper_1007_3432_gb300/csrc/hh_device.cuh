// Device-side building blocks of the GB300 Hubbard HMC library: lattice
// geometry with division by invariant integers, the stencil of the fermion
// matrix, the Philox counter generator, deterministic block reductions and the
// signal slots of the persistent engine, whose waits are bounded in time.
#pragma once

#include <type_traits>

#include <cuda_runtime.h>
#include <stdint.h>

namespace hh {

// ---------------------------------------------------------------------------
// Index checks of the debug build (compiled with -DHH_BOUNDS_CHECK): an index
// outside [lo, hi) is recorded in a device error word (the first one per
// translation unit: check code << 32 | index, top bit set) and replaced by lo,
// so the access stays in bounds and nothing traps.  hh_bounds_check_status
// reads and clears the words of every translation unit.  In the default
// build the checks compile to nothing.
// ---------------------------------------------------------------------------
enum BoundsCode : int {
    BC_NEIGHBOUR = 1,   // a neighbour site of the scalar stencil
    BC_GROUP = 2,       // a neighbour row of a W-site group
    BC_ROW = 3,         // a site shifted by one time slice
    BC_TILE = 4,        // a tile range of the CG engine
    BC_COPY = 5,        // a bulk copy of the multi-vector apply (source plane range)
    BC_SELFTEST = 15,   // the self-test kernel
};

#ifdef HH_BOUNDS_CHECK
namespace bounds {
static __device__ unsigned long long word;   // one per translation unit
using Reader = unsigned long long (*)();
void register_reader(Reader r);               // in hh_capi.cu
static unsigned long long read_and_clear()
{
    unsigned long long v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, word, sizeof(v)) != cudaSuccess) return 0;
    cudaMemcpyToSymbol(word, &z, sizeof(z));
    return v;
}
static struct Registrar {
    Registrar() { register_reader(&read_and_clear); }
} registrar;
}  // namespace bounds

__device__ __forceinline__ int check_index(int idx, int lo, int hi, int code)
{
    if (idx < lo || idx >= hi) {
        atomicCAS(&bounds::word, 0ull,
                  (1ull << 63) | ((unsigned long long)(unsigned)code << 32) | (unsigned long long)(unsigned)idx);
        return lo;
    }
    return idx;
}
#define HH_CHECK(idx, lo, hi, code) ((idx) = ::hh::check_index((idx), (lo), (hi), (code)))
#else
#define HH_CHECK(idx, lo, hi, code) ((void)0)
#endif

// ---------------------------------------------------------------------------
// Division by a run-time invariant 32-bit divisor (Granlund & Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994, round-up
// variant with a 33-bit multiplier): q = (umulhi(n, m) + n) >> s.
// ---------------------------------------------------------------------------
struct FastDiv {
    uint32_t d, m, s;
};

inline FastDiv make_fastdiv(uint32_t d)
{
    FastDiv f;
    f.d = d;
    uint32_t s = 0;
    while ((1ull << s) < d) ++s;
    f.s = s;
    // m = floor(2^32 (2^s - d) / d) + 1 ; zero when d is a power of two.
    uint64_t num = ((1ull << s) - d) << 32;
    f.m = (uint32_t)(num / d + 1ull);
    if (d == 1) f.m = 0;
    if ((1ull << s) == d) f.m = 0;
    return f;
}

__host__ __device__ inline uint32_t fd_div(uint32_t n, const FastDiv &f)
{
#ifdef __CUDA_ARCH__
    uint32_t hi = __umulhi(n, f.m);
#else
    uint32_t hi = (uint32_t)(((uint64_t)n * f.m) >> 32);
#endif
    return (uint32_t)(((uint64_t)hi + n) >> f.s);
}

// ---------------------------------------------------------------------------
// Lattice geometry.  Site index i = s + V * tau with the spatial index
// s = x + Nx (y + Nx z) (d = 3) or s = x (d = 1); x runs fastest.
// ---------------------------------------------------------------------------
struct Geo {
    int d, nx, ntau, V;
    int N;               // V * ntau
    FastDiv f_nx, f_V;
};

inline Geo make_geo(int d, int nx, int ntau)
{
    Geo g;
    g.d = d;
    g.nx = nx;
    g.ntau = ntau;
    g.V = (d == 1) ? nx : nx * nx * nx;
    g.N = g.V * ntau;
    g.f_nx = make_fastdiv((uint32_t)nx);
    g.f_V = make_fastdiv((uint32_t)g.V);
    return g;
}

// Neighbour indices of site i: 2d spatial neighbours (periodic) and the
// previous / next time slice (the antiperiodic sign lives in the links).
struct Nbr {
    int sp[6];
    int prev, next;
};

__device__ __forceinline__ void neighbours(const Geo &g, int i, Nbr &nb)
{
    uint32_t tau = fd_div((uint32_t)i, g.f_V);
    int s = i - (int)tau * g.V;
    uint32_t yz = fd_div((uint32_t)s, g.f_nx);
    int x = s - (int)yz * g.nx;
    nb.sp[0] = (x == g.nx - 1) ? i - (g.nx - 1) : i + 1;
    nb.sp[1] = (x == 0) ? i + (g.nx - 1) : i - 1;
    if (g.d == 3) {
        uint32_t z = fd_div(yz, g.f_nx);
        int y = (int)yz - (int)z * g.nx;
        int sy = g.nx, sz = g.nx * g.nx;
        nb.sp[2] = (y == g.nx - 1) ? i - (g.nx - 1) * sy : i + sy;
        nb.sp[3] = (y == 0) ? i + (g.nx - 1) * sy : i - sy;
        nb.sp[4] = ((int)z == g.nx - 1) ? i - (g.nx - 1) * sz : i + sz;
        nb.sp[5] = (z == 0) ? i + (g.nx - 1) * sz : i - sz;
    }
    nb.prev = (tau == 0) ? i + (g.ntau - 1) * g.V : i - g.V;
    nb.next = ((int)tau == g.ntau - 1) ? i - (g.ntau - 1) * g.V : i + g.V;
#ifdef HH_BOUNDS_CHECK
    for (int k = 0; k < 2 * g.d; ++k) HH_CHECK(nb.sp[k], 0, g.N, BC_NEIGHBOUR);
    HH_CHECK(nb.prev, 0, g.N, BC_NEIGHBOUR);
    HH_CHECK(nb.next, 0, g.N, BC_NEIGHBOUR);
#endif
}

// Sum of the 2d spatial neighbours in a fixed order.
template <typename T>
__device__ __forceinline__ T hop_sum(const Geo &g, const T *v, const Nbr &nb)
{
    T s = v[nb.sp[0]] + v[nb.sp[1]];
    if (g.d == 3) s += (v[nb.sp[2]] + v[nb.sp[3]]) + (v[nb.sp[4]] + v[nb.sp[5]]);
    return s;
}

// (M v)_i = v_i - h sum_nbr v + L(prev) v(prev)        (Eq. (10))
template <typename T>
__device__ __forceinline__ T stencil_M(const Geo &g, T h, const T *__restrict__ L, const T *v, int i,
                                       const Nbr &nb)
{
    T acc = fma(-h, hop_sum(g, v, nb), v[i]);
    return fma(__ldg(L + nb.prev), v[nb.prev], acc);
}

// (M^T v)_i = v_i - h sum_nbr v + L(i) v(next)
template <typename T>
__device__ __forceinline__ T stencil_MT(const Geo &g, T h, const T *__restrict__ L, const T *v, int i,
                                        const Nbr &nb)
{
    T acc = fma(-h, hop_sum(g, v, nb), v[i]);
    return fma(__ldg(L + i), v[nb.next], acc);
}

// Exact-block form of M (the blocks of Eq. (7) with B = e^{-dtau K} e^{-dtau V},
// e^{-dtau K} = e^{h H} expanded to order 1 or 2): E = 1 + h H (+ h^2 H^2 / 2)
// applied at site p of one time slice to w = L v (WL) or to v, with H the
// sum over the 2d spatial neighbours, summed in the neighbour order of
// hop_sum (the H^2 term as a sum over neighbours of neighbour sums).
template <typename T, bool WL>
__device__ __forceinline__ T e_factor(const Geo &g, T h, const T *__restrict__ L, const T *v, int p,
                                      int order)
{
    Nbr nb;
    neighbours(g, p, nb);
    const int nn = 2 * g.d;
    T s1 = T(0), s2 = T(0);
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        if (a >= nn) break;
        const int q = nb.sp[a];
        s1 += WL ? __ldg(L + q) * v[q] : v[q];
        if (order == 2) {
            Nbr nq;
            neighbours(g, q, nq);
            T t = T(0);
#pragma unroll
            for (int b = 0; b < 6; ++b) {
                if (b >= nn) break;
                const int r = nq.sp[b];
                t += WL ? __ldg(L + r) * v[r] : v[r];
            }
            s2 += t;
        }
    }
    T e = fma(h, s1, WL ? __ldg(L + p) * v[p] : v[p]);
    if (order == 2) e = fma(T(0.5) * h * h, s2, e);
    return e;
}

// Exact-block form: (M v)_i = v_i + [E (L v)](prev)
template <typename T>
__device__ __forceinline__ T stencil_M_ex(const Geo &g, T h, const T *__restrict__ L, const T *v, int i,
                                          const Nbr &nb, int order)
{
    return v[i] + e_factor<T, true>(g, h, L, v, nb.prev, order);
}

// Exact-block form: (M^T v)_i = v_i + L(i) [E v](next)
template <typename T>
__device__ __forceinline__ T stencil_MT_ex(const Geo &g, T h, const T *__restrict__ L, const T *v, int i,
                                           const Nbr &nb, int order)
{
    return fma(__ldg(L + i), e_factor<T, false>(g, h, L, v, nb.next, order), v[i]);
}

// ---------------------------------------------------------------------------
// Short vectors of W consecutive elements (W = 1, 2, 4), loaded and stored
// with 8- or 16-byte accesses.  The address must be aligned to the access.
// 'vld' uses the coherent path (data written earlier in the same kernel);
// 'vldg' the read-only path (links, right-hand sides).
// ---------------------------------------------------------------------------
template <typename T, int W>
struct Vec {
    T a[W];
};

// Hint to bring the line holding *p into L2 ahead of a demand load.  p must
// point into an allocation (callers keep it inside the vector they stream).
__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Site j shifted one slice earlier / later (cyclic in tau).
__device__ __forceinline__ int row_prev(const Geo &g, int j)
{
    int r = j >= g.V ? j - g.V : j + (g.ntau - 1) * g.V;
    HH_CHECK(r, 0, g.N, BC_ROW);
    return r;
}
__device__ __forceinline__ int row_next(const Geo &g, int j)
{
    int r = j < g.N - g.V ? j + g.V : j - (g.ntau - 1) * g.V;
    HH_CHECK(r, 0, g.N, BC_ROW);
    return r;
}

template <typename T, int W>
__device__ __forceinline__ Vec<T, W> vld(const T *p)
{
    Vec<T, W> r;
    if constexpr (sizeof(T) == 8 && W >= 2) {
#pragma unroll
        for (int j = 0; j < W; j += 2) {
            double2 q = *reinterpret_cast<const double2 *>(p + j);
            r.a[j] = q.x;
            r.a[j + 1] = q.y;
        }
    } else if constexpr (sizeof(T) == 4 && W == 4) {
        float4 q = *reinterpret_cast<const float4 *>(p);
        r.a[0] = q.x; r.a[1] = q.y; r.a[2] = q.z; r.a[3] = q.w;
    } else if constexpr (sizeof(T) == 4 && W == 2) {
        float2 q = *reinterpret_cast<const float2 *>(p);
        r.a[0] = q.x; r.a[1] = q.y;
    } else {
#pragma unroll
        for (int j = 0; j < W; ++j) r.a[j] = p[j];
    }
    return r;
}

template <typename T, int W>
__device__ __forceinline__ Vec<T, W> vldg(const T *p)
{
    Vec<T, W> r;
    if constexpr (sizeof(T) == 8 && W >= 2) {
#pragma unroll
        for (int j = 0; j < W; j += 2) {
            double2 q = __ldg(reinterpret_cast<const double2 *>(p + j));
            r.a[j] = q.x;
            r.a[j + 1] = q.y;
        }
    } else if constexpr (sizeof(T) == 4 && W == 4) {
        float4 q = __ldg(reinterpret_cast<const float4 *>(p));
        r.a[0] = q.x; r.a[1] = q.y; r.a[2] = q.z; r.a[3] = q.w;
    } else if constexpr (sizeof(T) == 4 && W == 2) {
        float2 q = __ldg(reinterpret_cast<const float2 *>(p));
        r.a[0] = q.x; r.a[1] = q.y;
    } else {
#pragma unroll
        for (int j = 0; j < W; ++j) r.a[j] = __ldg(p + j);
    }
    return r;
}

// 16-bit links of an FP32 inner iteration (mode 1: the upper half of the FP32
// bit pattern, bfloat16 rounded to nearest even; mode 2: fixed point, value =
// (signed code) * scale).  FP32 links are passed as a plain pointer instead.
struct LinkSrc {
    const unsigned short *L16;
    int mode;
    float scale;
};

__device__ __forceinline__ float link16_value(unsigned u, int mode, float scale)
{
    return mode == 1 ? __uint_as_float(u << 16) : (float)(short)(unsigned short)u * scale;
}

// W consecutive links from site i (i a multiple of W): a vector load of the
// FP32 or FP64 links, or of the 16-bit codes (8, 4 or 2 bytes, aligned as the
// site index).
template <typename T, int W, typename LK>
__device__ __forceinline__ Vec<T, W> link_row(const LK &L, int i)
{
    if constexpr (std::is_same<LK, LinkSrc>::value) {
        Vec<T, W> r;
        if constexpr (W == 4) {
            const uint2 q = __ldg(reinterpret_cast<const uint2 *>(L.L16 + i));
            r.a[0] = link16_value(q.x & 0xffffu, L.mode, L.scale);
            r.a[1] = link16_value(q.x >> 16, L.mode, L.scale);
            r.a[2] = link16_value(q.y & 0xffffu, L.mode, L.scale);
            r.a[3] = link16_value(q.y >> 16, L.mode, L.scale);
        } else if constexpr (W == 2) {
            const unsigned q = __ldg(reinterpret_cast<const unsigned *>(L.L16 + i));
            r.a[0] = link16_value(q & 0xffffu, L.mode, L.scale);
            r.a[1] = link16_value(q >> 16, L.mode, L.scale);
        } else {
            r.a[0] = link16_value(__ldg(L.L16 + i), L.mode, L.scale);
        }
        return r;
    } else {
        return vldg<T, W>(L + i);
    }
}

// Address of the link storage of site i (for prefetches).
template <typename LK>
__device__ __forceinline__ const void *link_addr(const LK &L, int i)
{
    if constexpr (std::is_same<LK, LinkSrc>::value)
        return (const void *)(L.L16 + i);
    else
        return (const void *)(L + i);
}


template <typename T, int W>
__device__ __forceinline__ void vst(T *p, const Vec<T, W> &v)
{
    if constexpr (sizeof(T) == 8 && W >= 2) {
#pragma unroll
        for (int j = 0; j < W; j += 2) *reinterpret_cast<double2 *>(p + j) = make_double2(v.a[j], v.a[j + 1]);
    } else if constexpr (sizeof(T) == 4 && W == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v.a[0], v.a[1], v.a[2], v.a[3]);
    } else if constexpr (sizeof(T) == 4 && W == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(v.a[0], v.a[1]);
    } else {
#pragma unroll
        for (int j = 0; j < W; ++j) p[j] = v.a[j];
    }
}

// Neighbour rows of a group of W consecutive x sites starting at site i
// (x0 = i mod Nx, W divides Nx, so the group stays inside one x row).
struct GroupNbr {
    int left, right;     // site before the group / after it along x (periodic)
    int yp, ym, zp, zm;  // the group's start shifted by +-1 in y and z (periodic)
    int prev, next;      // the group's start one slice earlier / later (cyclic)
};

template <int D, int W>
__device__ __forceinline__ void group_nbrs(const Geo &g, int i, GroupNbr &nb)
{
    uint32_t tau = fd_div((uint32_t)i, g.f_V);
    int s = i - (int)tau * g.V;
    uint32_t yz = fd_div((uint32_t)s, g.f_nx);
    int x0 = s - (int)yz * g.nx;
    nb.left = (x0 == 0) ? i + (g.nx - 1) : i - 1;
    nb.right = (x0 + W == g.nx) ? i + W - g.nx : i + W;
    if (D == 3) {
        uint32_t z = fd_div(yz, g.f_nx);
        int y = (int)yz - (int)z * g.nx;
        int sy = g.nx, sz = g.nx * g.nx;
        nb.yp = (y == g.nx - 1) ? i - (g.nx - 1) * sy : i + sy;
        nb.ym = (y == 0) ? i + (g.nx - 1) * sy : i - sy;
        nb.zp = ((int)z == g.nx - 1) ? i - (g.nx - 1) * sz : i + sz;
        nb.zm = (z == 0) ? i + (g.nx - 1) * sz : i - sz;
    }
    nb.prev = (tau == 0) ? i + (g.ntau - 1) * g.V : i - g.V;
    nb.next = ((int)tau == g.ntau - 1) ? i - (g.ntau - 1) * g.V : i + g.V;
#ifdef HH_BOUNDS_CHECK
    // single sites x - 1 and x + W; W-site rows elsewhere
    HH_CHECK(nb.left, 0, g.N, BC_GROUP);
    HH_CHECK(nb.right, 0, g.N, BC_GROUP);
    if (D == 3) {
        HH_CHECK(nb.yp, 0, g.N - W + 1, BC_GROUP);
        HH_CHECK(nb.ym, 0, g.N - W + 1, BC_GROUP);
        HH_CHECK(nb.zp, 0, g.N - W + 1, BC_GROUP);
        HH_CHECK(nb.zm, 0, g.N - W + 1, BC_GROUP);
    }
    HH_CHECK(nb.prev, 0, g.N - W + 1, BC_GROUP);
    HH_CHECK(nb.next, 0, g.N - W + 1, BC_GROUP);
#endif
}

// Spatial hopping sums of a group: for site u the x neighbours are the
// group's own elements except at the two ends.
template <int D, typename T, int W>
__device__ __forceinline__ Vec<T, W> group_hop(const T *v, const GroupNbr &nb, const Vec<T, W> &self)
{
    T vl = v[nb.left], vr = v[nb.right];
    Vec<T, W> out;
    Vec<T, W> yp, ym, zp, zm;
    if (D == 3) {
        yp = vld<T, W>(v + nb.yp);
        ym = vld<T, W>(v + nb.ym);
        zp = vld<T, W>(v + nb.zp);
        zm = vld<T, W>(v + nb.zm);
    }
#pragma unroll
    for (int u = 0; u < W; ++u) {
        T xr = (u == W - 1) ? vr : self.a[u + 1 < W ? u + 1 : u];
        T xl = (u == 0) ? vl : self.a[u > 0 ? u - 1 : 0];
        T hsum = xr + xl;
        if (D == 3) hsum += (yp.a[u] + ym.a[u]) + (zp.a[u] + zm.a[u]);
        out.a[u] = hsum;
    }
    return out;
}

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Counter layout of the
// library: (block, tag | a << 8, trajectory, chain), key (seed, 0).
// ---------------------------------------------------------------------------
struct U64x4 {
    uint64_t v[4];
};

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                               uint64_t k0, uint64_t k1)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    U64x4 o;
    o.v[0] = c0;
    o.v[1] = c1;
    o.v[2] = c2;
    o.v[3] = c3;
    return o;
}

__device__ __forceinline__ double u53(uint64_t w)
{
    return (double)(w >> 11) * (1.0 / 9007199254740992.0);
}

// ---------------------------------------------------------------------------
// Deterministic reductions: a fixed tree inside the warp, then warps in order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;  // valid in lane 0
}

// Block-wide sum; every thread must call it; the result is valid in thread 0.
// 'red' must hold blockDim.x / 32 doubles.
__device__ __forceinline__ double block_sum(double v, double *red)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        int nw = blockDim.x >> 5;
        for (int j = 0; j < nw; ++j) s += red[j];
    }
    return s;
}

// ---------------------------------------------------------------------------
// Control block of a cooperative engine launch, and the signal slots through
// which its blocks exchange per-tile partial sums.
//
// A tile publishes the partial of each phase it runs into a slot of a
// parity-indexed pair (iteration k writes slot k & 1) with a release store,
// after emptying the slot of the other parity.  A block that needs the phase
// complete (its neighbour data written, its partial sums known) polls the
// slots of every tile of that system with relaxed loads until none is empty,
// then fences: one round trip both synchronises and delivers the values, and
// a block waits only for the tiles of its own systems.  Every wait is bounded
// by a wall-clock budget read from the global timer, after which it records
// HH_ETIMEOUT (-6) and the kernel leaves.
// ---------------------------------------------------------------------------
struct EngCtl {
    int error;              // 0, or a negative library error code (first one wins)
    int drop_sig;           // fault injection for tests: j + 1 makes the launch never publish
                            // tile partial j, so every wait for it runs out; 0: none
    long long k;            // engine iteration counter when the launch starts
    long long k_end;        // engine iteration counter after it (max over blocks)
    long long timeout_ns;   // bound of every wait
};

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_volatile_i32(const int *p)
{
    return *(const volatile int *)p;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Empty slot: a NaN bit pattern no published value has (a NaN partial is
// published as the canonical quiet NaN).
constexpr unsigned long long kSigEmpty = ~0ull;
constexpr unsigned long long kSigNaN = 0x7FF8000000000000ull;

// Called by one thread after a __syncthreads() that follows all of the block's
// writes of the phase: empties 'next' (the slot the tile writes next
// iteration), then release-stores v into 'now'.
__device__ __forceinline__ void sig_publish(unsigned long long *now, unsigned long long *next, double v)
{
    unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    if (v != v) bits = kSigNaN;
    *next = kSigEmpty;
    asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(now), "l"(bits) : "memory");
}

// Called by all 32 lanes of one warp: waits until the n slots sig[0, n) are
// published and returns their sum in lane 0 (lane-strided sums over
// j = lane, lane + 32, ... in order, then a fixed shuffle tree; the same bits
// in every block).  Returns false in every lane on a timeout or a recorded
// error.
__device__ __forceinline__ bool poll_sum(const unsigned long long *sig, int n, EngCtl *ctl, double &sum)
{
    constexpr int U = 8;
    const int lane = (int)(threadIdx.x & 31u);
    double v = 0.0;
    bool ok = true;
    unsigned spins = 0;
    uint64_t t0 = 0;
    for (int j0 = 0; j0 < n && ok; j0 += 32 * U) {
        unsigned long long a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = j0 + 32 * u + lane;
            a[u] = j < n ? ld_relaxed_u64(sig + j) : 0ull;
        }
        while (true) {
            bool ready = true;
#pragma unroll
            for (int u = 0; u < U; ++u) ready = ready && (a[u] != kSigEmpty);
            if (ready) break;
            if ((++spins & 63u) == 0) {
                if (t0 == 0) t0 = global_ns();
                if (ld_volatile_i32(&ctl->error) != 0) {
                    ok = false;
                    break;
                }
                if ((long long)(global_ns() - t0) > ctl->timeout_ns) {
                    atomicCAS(&ctl->error, 0, -6);
                    ok = false;
                    break;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (a[u] == kSigEmpty) a[u] = ld_relaxed_u64(sig + j0 + 32 * u + lane);
        }
        if (ok) {
#pragma unroll
            for (int u = 0; u < U; ++u) v += __longlong_as_double((long long)a[u]);
        }
    }
    // Acquire side: the relaxed loads above observed the publishers' release
    // stores; the fence orders this block's later reads after their writes.
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    ok = __all_sync(0xffffffffu, ok);
    sum = warp_sum(v);
    return ok;
}

}  // namespace hh
