// Q = M^T M (Eq. (10); Q applied as M then M^T, Sec. 4.3) on k FP32 vectors
// that share one field, d = 3: y_v = Q x_v for v = 0 .. k-1 in one persistent
// launch.
//
// Work split.  The lattice is cut into z-slabs of TZ planes (all x, y); CTA b
// owns slab b % nslab and, in that slab, a contiguous range of the k N_tau
// (vector, time slice) pairs u = v N_tau + tau, range b / nslab of m equal
// ranges.  All slabs use the same m ranges, so the CTAs of neighbouring slabs
// work on the same (vector, slice) at about the same time and the halo planes
// one CTA copies are the core planes its neighbours have just brought into L2.
// The links are read with an L2 evict-last policy (every vector reads them;
// they stay in L2 for the launch) and q is stored with evict-first (written
// once), so HBM sees every x_v and the links once and every y_v once:
// (8 k + 4) bytes per site.
//
// A CTA marches its range in time slices with the paper's thread blocking
// (Sec. 4.3: shared-memory tiles with a boundary layer), laid out as a TMA
// pipeline:
//  * per step, x(tau + 1) on the slab plus two halo planes arrives in one of
//    NS shared-memory stages by 1-D TMA bulk copies completing on an mbarrier.
//    Thread 0 issues them: the first NS stages up front, then the stage NS
//    ahead right after each step's barrier (the barrier proves the slot's
//    previous stage has been read); it also prefetches later stages (x and
//    the links) into L2;
//  * the threads build t(tau + 1) = (M x)(tau + 1) on the slab plus one halo
//    plane.  A thread owns one float4 group of one (x, y) row in one part of
//    the slab's planes and streams z with the z neighbours in registers; the
//    x(tau) of the link term is carried in registers from the previous step,
//    and the links L(tau) of its planes are loaded into registers at the start
//    of the step, so that their L2 round trip overlaps the wait for the stage.
//    As soon as t(tau + 1) is known on a core plane, the thread writes q(tau)
//    = t(tau) - h hop t(tau) + L(tau) t(tau + 1) there, from the shared-memory
//    copy of t(tau) (written in the previous step) and the registers holding
//    L(tau) and t(tau + 1).  Two t buffers alternate, so one barrier per step
//    orders the writes of t(tau + 1) against the reads of t(tau).  The
//    stencil sums run in packed FP32 pairs (two sites per instruction).
// A segment of a range (one vector, slices [ta, tb)) takes tb - ta + 2 steps:
// x(ta - 1) into the carry registers, t(ta), then one step per q slice.
//
// Every wait is bounded in time; on expiry the CTA records HH_ETIMEOUT, thread
// 0 waits (bounded) for the copies in flight, and the CTA leaves.
//
// What bounds it (GB300, 32^3 x 128, 16 vectors).  The one-row form (a
// thread owns one float4 group of one row) is bound by the shared-memory
// datapath: per site and vector it moves about 50 bytes through it (the x
// and t rows of the y neighbours, the t planes, the links and q through L1)
// against 8.5 bytes of HBM traffic, and ncu shows the pipe 67-74% busy.  The
// row-pair form (below) halves the y-neighbour reads and keeps t in
// registers: the pipe drops to 43% and the kernel is then bound by latency,
// with 8 warps per SM held to one block barrier per step (its register
// count, 255, leaves no room for more warps).
#include <cstdlib>

#include "hh_apply.cuh"
#include "hh_slab.cuh"

namespace hh {

namespace {

struct MultiCfg {
    Geo g;
    float h;
    int nslab;          // Nx / TZ
    int P;              // Nx * Nx
    int k;              // vectors
    int m;              // ranges (CTAs per slab)
    int shfl;           // x halo by warp shuffles (else from shared memory)
    int pf_ahead;       // L2 prefetch of the stage this many after the one being copied
    int drop_tx;        // fault injection for tests: the first stage expects 16 bytes more than
                        // it copies, so its waits run out
    long long timeout_ns;
};

constexpr int kPartThreads = 256;  // threads per part (one float4 group of each x-y row per thread)
constexpr int kPrefetchAhead = 1;  // default L2 prefetch distance, in stages after the one being copied
constexpr int kMaxRuns = 4;        // contiguous z runs of a slab's planes (periodic z, Nx >= 4)

enum StageKind : int { STAGE_PRE = 0, STAGE_TFIRST = 1, STAGE_FULL = 2, STAGE_END = 3 };

// A CTA's range [w, w1) of u = v * Ntau + tau as the sequence of its
// pipeline stages (kind, v, tau'); the stage of tau' holds x_v(tau' + 1) and
// works with L(tau').  A segment of slices [ta, tb) of one vector gives
// tau' = ta - 2 (STAGE_PRE: x_v(ta - 1) for the carry), ta - 1 (STAGE_TFIRST:
// t(ta)), then ta .. tb - 1 (STAGE_FULL: t(tau' + 1) and q(tau')).
struct StageIter {
    long long w, w1;
    int ntau, vec, tau, ta, tb;
    bool in_seg;

    __device__ void init(long long a, long long b, int nt)
    {
        w = a;
        w1 = b;
        ntau = nt;
        in_seg = false;
    }

    __device__ int next(int &v, int &tp)
    {
        if (!in_seg || tau >= tb) {
            if (w >= w1) return STAGE_END;
            vec = (int)(w / ntau);
            ta = (int)(w - (long long)vec * ntau);
            const long long rem = w1 - w;
            tb = (rem < (long long)(ntau - ta)) ? ta + (int)rem : ntau;
            w = (long long)vec * ntau + tb;
            tau = ta - 2;
            in_seg = true;
        }
        v = vec;
        tp = tau;
        const int kind = (tau == ta - 2) ? STAGE_PRE : (tau == ta - 1) ? STAGE_TFIRST : STAGE_FULL;
        ++tau;
        return kind;
    }
};

// tau in [-ntau, 2 ntau) to [0, ntau).
__device__ __forceinline__ int wrap_once(int t, int ntau)
{
    return t < 0 ? t + ntau : (t >= ntau ? t - ntau : t);
}

// Bounded wait on an mbarrier phase: false once budget_ns has passed or the
// CTA has been told to abort.
__device__ __forceinline__ bool wait_bounded(uint64_t *bar, unsigned parity, long long budget_ns,
                                             const volatile int *abort)
{
    uint64_t t0 = 0;
    unsigned spins = 0;
    while (!mbar_try_wait(bar, parity)) {
        if ((++spins & 31u) == 0) {
            if (*abort) return false;
            const uint64_t now = global_ns();
            if (t0 == 0)
                t0 = now;
            else if ((long long)(now - t0) > budget_ns)
                return false;
        }
    }
    return true;
}

// Block-wide barrier that also ORs a flag over the block.  The two halves of
// the block reach it from different code (one instantiation each), so it is
// the non-.aligned form of the barrier, on its own id.
constexpr int kBarBlock = 1;
template <int NTHREADS>
__device__ __forceinline__ int block_sync_or(int flag)
{
    int out;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.s32 q, %1, 0;\n\t"
        "barrier.red.or.pred p, %2, %3, q;\n\t"
        "selp.s32 %0, 1, 0, p;\n\t}"
        : "=r"(out)
        : "r"(flag), "r"(kBarBlock), "r"(NTHREADS)
        : "memory");
    return out;
}

template <int TZ, int NS>
struct MultiLayout {
    static constexpr int XPL = TZ + 4;   // x planes per stage
    static constexpr int TPL = TZ + 2;   // t planes
    static constexpr int TBUF = 2;
    static size_t smem(int P)
    {
        return ((size_t)NS * XPL + (size_t)TBUF * TPL) * (size_t)P * sizeof(float);
    }
};

// Contiguous runs of the periodic z range [z_first, z_first + count):
// run r covers planes off[r] .. off[r] + n[r] - 1 of the range, starting at z[r].
struct ZRuns {
    int nr;
    int z[kMaxRuns], off[kMaxRuns], n[kMaxRuns];

    // Unrolled over the run index, so that the arrays can live in registers.
    __device__ void init(int z_first, int count, int nx)
    {
        int zz = ((z_first % nx) + nx) % nx, done = 0;
        nr = 0;
#pragma unroll
        for (int r = 0; r < kMaxRuns; ++r) {
            int run = count - done;
            if (zz + run > nx) run = nx - zz;
            z[r] = zz;
            off[r] = done;
            n[r] = run > 0 ? run : 0;
            if (run > 0) nr = r + 1;
            done += run > 0 ? run : 0;
            zz = 0;
        }
    }
};

// L2 prefetch of the next stage of 'pf': its x planes and, after the first
// stage of a segment, its link planes.
__device__ __forceinline__ void prefetch_stage(StageIter &pf, const ZRuns &xr, const ZRuns &lr, const MultiCfg &c,
                                               const float *x, const float *L)
{
    int v, tp;
    const int kind = pf.next(v, tp);
    if (kind == STAGE_END) return;
    const int P = c.P;
    const float *xb = x + (size_t)v * c.g.N + (size_t)wrap_once(tp + 1, c.g.ntau) * c.g.V;
#pragma unroll
    for (int r = 0; r < kMaxRuns; ++r)
        if (r < xr.nr) bulk_prefetch_l2(xb + (size_t)xr.z[r] * P, (unsigned)(xr.n[r] * P * sizeof(float)));
    if (kind != STAGE_PRE) {
        const float *lb = L + (size_t)wrap_once(tp, c.g.ntau) * c.g.V;
#pragma unroll
        for (int r = 0; r < kMaxRuns; ++r)
            if (r < lr.nr) bulk_prefetch_l2(lb + (size_t)lr.z[r] * P, (unsigned)(lr.n[r] * P * sizeof(float)));
    }
}

// Issues the copies of the stages of a CTA's range in order (thread 0 only;
// the state lives in shared memory): stage j goes to slot j % NS, whose
// previous stage j - NS must have been read.
template <int TZ, int NS>
struct Issuer {
    StageIter it, pf;
    ZRuns xr, lr;        // runs of the x planes and of the link planes of the slab
    long long issued;
    int done;

    __device__ void init(long long w0, long long w1, const MultiCfg &c, const float *x, const float *L, int z0)
    {
        it.init(w0, w1, c.g.ntau);
        pf.init(w0, w1, c.g.ntau);
        xr.init(z0 - 2, TZ + 4, c.g.nx);
        lr.init(z0 - 1, TZ + 2, c.g.nx);
        issued = 0;
        done = 0;
        // the prefetch iterator runs kPrefetchAhead stages ahead of the copies
        int v, tp;
        pf.next(v, tp);
        for (int a = 1; a <= c.pf_ahead; ++a) prefetch_next(c, x, L);
    }

    __device__ void prefetch_next(const MultiCfg &c, const float *x, const float *L)
    {
        prefetch_stage(pf, xr, lr, c, x, L);
    }

    // Issue every stage j <= upto that has not been issued yet.
    __device__ void issue_upto(long long upto, const MultiCfg &c, float *XS, uint64_t *full, const float *x,
                               const float *L)
    {
        constexpr int XPL = TZ + 4;
        const int P = c.P;
        const unsigned stage_bytes = (unsigned)XPL * (unsigned)P * (unsigned)sizeof(float);
        const unsigned extra0 = (c.drop_tx && issued == 0) ? 16u : 0u;
        while (!done && issued <= upto) {
            int v, tau;
            if (it.next(v, tau) == STAGE_END) {
                done = 1;
                break;
            }
            const int slot = (int)(issued % NS);
#ifdef HH_BOUNDS_CHECK
            {
                // The copy's vector and slice, and each run's planes, inside x.
                int vv = v, ts = wrap_once(tau + 1, c.g.ntau);
                HH_CHECK(vv, 0, c.k, BC_COPY);
                HH_CHECK(ts, 0, c.g.ntau, BC_COPY);
                v = vv;
                tau = ts - 1;
                for (int r = 0; r < kMaxRuns; ++r)
                    if (r < xr.nr) {
                        int zend = xr.z[r] + xr.n[r], oend = xr.off[r] + xr.n[r];
                        HH_CHECK(zend, 1, c.g.nx + 1, BC_COPY);
                        HH_CHECK(oend, 1, XPL + 1, BC_COPY);
                        if (zend != xr.z[r] + xr.n[r] || oend != xr.off[r] + xr.n[r]) xr.n[r] = 0;
                    }
            }
#endif
            const float *xb = x + (size_t)v * c.g.N + (size_t)wrap_once(tau + 1, c.g.ntau) * c.g.V;
            float *dst = XS + (size_t)slot * XPL * P;
            mbar_expect_tx(&full[slot], stage_bytes + (issued == 0 ? extra0 : 0u));
#pragma unroll
            for (int r = 0; r < kMaxRuns; ++r)
                if (r < xr.nr && xr.n[r] > 0) bulk_g2s(dst + (size_t)xr.off[r] * P, xb + (size_t)xr.z[r] * P,
                         (unsigned)(xr.n[r] * P * sizeof(float)), &full[slot]);
            ++issued;
            prefetch_next(c, x, L);
        }
    }
};

// One plane of the stencil c - h hop(c) + l o for a float4 group of x sites
// in packed FP32 pairs (sites 0, 1 and 2, 3): the x neighbours are the
// group's own lanes plus xm, xp, the y neighbours yp, ym, the z neighbours
// a(bove), b(elow).  The sums are taken in the order
// ((x- + x+) + (y+ + y-)) + (z+ + z-), each lane rounded as in FP32.
__device__ __forceinline__ float4 stencil_x2(const float4 &c, const float4 &b, const float4 &a, const float4 &yp,
                                             const float4 &ym, float xm, float xp, const float4 &l,
                                             const float4 &o, const float2 mh)
{
    const float2 mid = make_float2(c.y, c.z);
    float2 s0 = __fadd2_rn(make_float2(xm, c.x), mid);
    float2 s1 = __fadd2_rn(mid, make_float2(c.w, xp));
    s0 = __fadd2_rn(s0, __fadd2_rn(make_float2(yp.x, yp.y), make_float2(ym.x, ym.y)));
    s1 = __fadd2_rn(s1, __fadd2_rn(make_float2(yp.z, yp.w), make_float2(ym.z, ym.w)));
    s0 = __fadd2_rn(s0, __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y)));
    s1 = __fadd2_rn(s1, __fadd2_rn(make_float2(a.z, a.w), make_float2(b.z, b.w)));
    const float2 r0 = __ffma2_rn(make_float2(l.x, l.y), make_float2(o.x, o.y),
                                 __ffma2_rn(mh, s0, make_float2(c.x, c.y)));
    const float2 r1 = __ffma2_rn(make_float2(l.z, l.w), make_float2(o.z, o.w),
                                 __ffma2_rn(mh, s1, make_float2(c.z, c.w)));
    return make_float4(r0.x, r0.y, r1.x, r1.y);
}

// The per-thread part of the march for one of PARTS parts of the slab's
// planes (PARTS = 2: PART 0 has t planes [0, TPL/2) and core planes
// [0, TZ/2), PART 1 the rest; PARTS = 1: all), compiled per part so that
// every register array is indexed by constants.  NX > 0 fixes N_x at compile
// time (plane offsets become immediates); NX = 0 reads it from c.
template <int NX, int TZ, int NS, int PARTS, int PART>
__device__ __forceinline__ void multi_consumer(const MultiCfg &c, float *XS, float *TS, uint64_t *full,
                                               volatile int *abort, void *issuer_mem, long long w0, long long w1,
                                               const float *__restrict__ x, const float *__restrict__ L,
                                               float *__restrict__ y, int slab, int *err)
{
    constexpr int TPL = TZ + 2, XPL = TZ + 4, TH = TPL / PARTS, CH = TZ / PARTS;
    constexpr int NTHREADS = kPartThreads * PARTS;
    constexpr int TLO = PART * TH;   // first t plane of this part
    constexpr int CLO = PART * CH;   // first core plane (core plane cc is t plane cc + 1)
    constexpr int PC0 = CLO + 1, PC1 = CLO + CH;   // core t planes of this part
    const int nx = NX ? NX : c.g.nx;
    const int P = nx * nx, ntau = c.g.ntau, V = NX ? NX * NX * NX : c.g.V;
    const size_t N = (size_t)c.g.N;
    const int lane = (int)threadIdx.x & 31;
    const int col = (int)threadIdx.x - PART * kPartThreads;
    const int G = P / 4;
    const bool active = col < G;     // Nx <= 32: at most one group per thread
    const PlaneGroup q = plane_group(active ? col : 0, nx);
    const int gpr = nx / 4, jx = lane % gpr;
    const bool shfl = NX ? ((32 % (NX / 4) == 0) && ((NX * NX / 4) % 32 == 0)) : (c.shfl != 0);
    const int src_m = (jx == 0) ? lane + gpr - 1 : lane - 1;
    const int src_p = (jx == gpr - 1) ? lane - gpr + 1 : lane + 1;
    const float2 mh = make_float2(-c.h, -c.h);
    const int z0 = slab * TZ;
    const uint64_t pol_y = l2_policy_evict_first();
    const uint64_t pol_l = l2_policy_evict_last();
    // In-slice offsets of this thread's group in each of its part's t planes
    // (t plane p is z = z0 - 1 + p, periodic).
    int loff[TH];
#pragma unroll
    for (int pp = 0; pp < TH; ++pp) {
        int z = z0 - 1 + TLO + pp;
        z = z < 0 ? z + nx : (z >= nx ? z - nx : z);
        loff[pp] = z * P + q.s;
    }
    auto halo = [&](const float *pl, const float4 &self, float &hm, float &hp) {
        if (shfl) {
            hm = __shfl_sync(0xffffffffu, self.w, src_m);
            hp = __shfl_sync(0xffffffffu, self.x, src_p);
        } else {
            hm = pl[q.xm];
            hp = pl[q.xp];
        }
    };

    // Thread 0 issues the copies: the first NS stages now.
    const bool issuer = PART == 0 && threadIdx.x == 0;
    Issuer<TZ, NS> &is = *static_cast<Issuer<TZ, NS> *>(issuer_mem);
    if (issuer) {
        is.init(w0, w1, c, x, L, z0);
        is.issue_upto(NS - 1, c, XS, full, x, L);
    }

    float4 xc[TH];   // x(tau) at this thread's group of each of the part's t planes (link term)
    float4 lc[TH];   // L(tau') of the current stage at the part's t planes
    StageIter it;
    it.init(w0, w1, ntau);
    int slot = 0;
    unsigned phase = 0;   // parity of the slot's current use
    long long j = 0;      // stage index
    int cb = 0;           // t buffer holding t(tau)
    int failed = 0;       // warp-uniform: a wait of this warp ran out
    bool aborted = false; // block-uniform: some warp's wait ran out
    for (;;) {
        int v, tau;
        const int kind = it.next(v, tau);
        if (kind == STAGE_END) break;
        // The links of this stage: their L2 round trip overlaps the wait.
        if (kind != STAGE_PRE && active) {
            const float *lb = L + (size_t)wrap_once(tau, ntau) * V;
#pragma unroll
            for (int pp = 0; pp < TH; ++pp) lc[pp] = ldg4_hint(lb + loff[pp], pol_l);
        }
        if (!failed) {
            const bool ok = wait_bounded(&full[slot], phase, c.timeout_ns, abort);
            failed = __all_sync(0xffffffffu, ok) ? 0 : 1;
            if (failed && lane == 0) {
                *abort = 1;
                atomicCAS(err, 0, -6);
            }
        }
        const float *X = XS + (size_t)slot * XPL * P;
        if (!failed && active) {
            const float *xs = X + q.s, *xyp = X + q.yp, *xym = X + q.ym;
            if (kind == STAGE_PRE) {
#pragma unroll
                for (int pp = 0; pp < TH; ++pp) xc[pp] = ld4(xs + (TLO + pp + 1) * P);
            } else {
                // t(tau + 1) on the part's t planes (t plane p is the slab's
                // z0 - 1 + p; x planes p, p + 1, p + 2 are z - 1, z, z + 1) and,
                // on a full step, q(tau) on each core plane p - 1 as soon as
                // t(tau + 1) at p is known: q needs t(tau) at t planes p - 1,
                // p, p + 1 (buffer cb, written last step) and, at the site
                // itself, t(tau + 1) and L(tau).
                const bool full_step = kind == STAGE_FULL;
                float *tn = TS + (size_t)(cb ^ 1) * TPL * P + q.s;
                const float *T0 = TS + (size_t)cb * TPL * P;
                const float *ts = T0 + q.s, *typ = T0 + q.yp, *tym = T0 + q.ym;
                float *yo = y + (size_t)v * N + (size_t)(tau < 0 ? 0 : tau) * V + (size_t)z0 * P + q.s;
                float4 below = ld4(xs + TLO * P), here = ld4(xs + (TLO + 1) * P);
                float4 tb = make_float4(0.f, 0.f, 0.f, 0.f), th = tb;
                if (full_step) {
                    tb = ld4(ts + (PC0 - 1) * P);
                    th = ld4(ts + PC0 * P);
                }
#pragma unroll
                for (int pp = 0; pp < TH; ++pp) {
                    const int p = TLO + pp;
                    const float4 above = ld4(xs + (p + 2) * P);
                    const float4 yp = ld4(xyp + (p + 1) * P), ym = ld4(xym + (p + 1) * P);
                    float hm, hp;
                    halo(X + (p + 1) * P, here, hm, hp);
                    const float4 t = stencil_x2(here, below, above, yp, ym, hm, hp, lc[pp], xc[pp], mh);
                    st4(tn + p * P, t);
                    xc[pp] = here;
                    below = here;
                    here = above;
                    if (p >= PC0 && p <= PC1 && full_step) {
                        const float4 ta = ld4(ts + (p + 1) * P);
                        const float4 gp = ld4(typ + p * P), gm = ld4(tym + p * P);
                        float em, ep;
                        halo(T0 + p * P, th, em, ep);
                        st4_global_hint(yo + (p - 1) * P, stencil_x2(th, tb, ta, gp, gm, em, ep, lc[pp], t, mh),
                                        pol_y);
                        tb = th;
                        th = ta;
                    }
                }
            }
        }
        if (kind != STAGE_PRE) {
            // Every stage up to j has now been read and t(tau + 1) written:
            // stage j's slot can take stage j + NS.
            if (block_sync_or<NTHREADS>(failed)) {
                aborted = true;
                break;
            }
            if (issuer) is.issue_upto(j + NS, c, XS, full, x, L);
            cb ^= 1;
        }
        ++j;
        if (++slot == NS) {
            slot = 0;
            phase ^= 1u;
        }
    }
    if (issuer && aborted) {
        // Copies in flight must land before the CTA ends (bounded wait, at
        // least a second whatever the caller's budget; a phase that has
        // already completed returns at once).
        const int never = 0;
        const long long drain_ns = c.timeout_ns > 1000000000LL ? c.timeout_ns : 1000000000LL;
        for (long long jj = j; jj < is.issued; ++jj)
            wait_bounded(&full[(int)(jj % NS)], (unsigned)((jj / NS) & 1), drain_ns, &never);
    }
}

// Row-pair form of the march (N_x = 32).  A thread owns one float4 group in
// each of two adjacent rows y0, y0 + 1 of one part of the slab's planes, so
// the y neighbour between the two rows comes from registers and only rows
// y0 - 1 and y0 + 2 are read from shared memory: two 16-byte loads per plane
// and row pair for the y neighbours instead of four.  The thread also keeps
// its own t(tau) (written by itself in the previous step) in registers, so q
// reads from shared memory only the y neighbours of t, plus one plane at a
// part boundary.  Measured at 32^3 x 128 with 16 vectors: 14.8M shared-
// memory wavefronts per launch against 28.1M for the one-row form, about 28
// bytes per site and vector against 54.
constexpr int kPairThreads = 128;  // threads per part: (32 x 32 / 4) groups / 2 rows
template <int TZ, int NS, int PARTS, int PART>
__device__ __forceinline__ void multi_consumer_rp(const MultiCfg &c, float *XS, float *TS, uint64_t *full,
                                                  volatile int *abort, long long w0, long long w1,
                                                  const float *__restrict__ x, const float *__restrict__ L,
                                                  float *__restrict__ y, int slab, int *err)
{
    constexpr int NX = 32, P = NX * NX, V = NX * NX * NX, GPR = NX / 4;
    constexpr int TPL = TZ + 2, XPL = TZ + 4, TH = TPL / PARTS, CH = TZ / PARTS;
    constexpr int NTHREADS = kPairThreads * PARTS;
    constexpr int TLO = PART * TH;   // first t plane of this part
    constexpr int CLO = PART * CH;   // first core plane (core plane cc is t plane cc + 1)
    constexpr int PC0 = CLO + 1, PC1 = CLO + CH;   // core t planes of this part
    static_assert(TPL % PARTS == 0 && TZ % PARTS == 0, "parts split the planes evenly");
    static_assert(PC0 - TLO >= 0 && PC1 - TLO < TH, "a part holds t(tau) of its own core planes");
    const int ntau = c.g.ntau;
    const size_t N = (size_t)c.g.N;
    const int lane = (int)threadIdx.x & 31;
    const int col = (int)threadIdx.x - PART * kPairThreads;   // 0 .. 127, all active for N_x = 32
    const int jx = col % GPR, y0 = 2 * (col / GPR);
    const int sA = y0 * NX + 4 * jx, sB = sA + NX;                       // rows y0, y0 + 1
    const int sM = (y0 == 0 ? NX - 1 : y0 - 1) * NX + 4 * jx;            // row y0 - 1
    const int sP = (y0 + 2 == NX ? 0 : y0 + 2) * NX + 4 * jx;            // row y0 + 2
    const int src_m = (jx == 0) ? lane + GPR - 1 : lane - 1;
    const int src_p = (jx == GPR - 1) ? lane - GPR + 1 : lane + 1;
    const float2 mh = make_float2(-c.h, -c.h);
    const int z0 = slab * TZ;
    const uint64_t pol_y = l2_policy_evict_first();
    const uint64_t pol_l = l2_policy_evict_last();
    int zoff[TH];   // in-slice offset of each of the part's t planes (t plane p is z = z0 - 1 + p)
#pragma unroll
    for (int pp = 0; pp < TH; ++pp) {
        int z = z0 - 1 + TLO + pp;
        z = z < 0 ? z + NX : (z >= NX ? z - NX : z);
        zoff[pp] = z * P;
    }
    auto halo = [&](const float4 &self, float &hm, float &hp) {
        hm = __shfl_sync(0xffffffffu, self.w, src_m);
        hp = __shfl_sync(0xffffffffu, self.x, src_p);
    };

    // Thread 0 issues the copies, its issuer state in registers (this form
    // has the registers to spare; a thread holds 2 TH float4 of each of x,
    // t and L).
    const bool issuer = PART == 0 && threadIdx.x == 0;
    Issuer<TZ, NS> is;
    if (issuer) {
        is.init(w0, w1, c, x, L, z0);
        is.issue_upto(NS - 1, c, XS, full, x, L);
    }

    float4 xcA[TH], xcB[TH];   // x(tau) of the two rows at the part's t planes (link term)
    float4 tcA[TH], tcB[TH];   // t(tau), computed by this thread in the previous step
    float4 lcA[TH], lcB[TH];   // L(tau') of the current stage
    StageIter it;
    it.init(w0, w1, ntau);
    int slot = 0;
    unsigned phase = 0;
    long long j = 0;
    int cb = 0;
    int failed = 0;
    bool aborted = false;
    for (;;) {
        int v, tau;
        const int kind = it.next(v, tau);
        if (kind == STAGE_END) break;
        if (kind != STAGE_PRE) {
            const float *lb = L + (size_t)wrap_once(tau, ntau) * V;
#pragma unroll
            for (int pp = 0; pp < TH; ++pp) {
                lcA[pp] = ldg4_hint(lb + zoff[pp] + sA, pol_l);
                lcB[pp] = ldg4_hint(lb + zoff[pp] + sB, pol_l);
            }
        }
        if (!failed) {
            const bool ok = wait_bounded(&full[slot], phase, c.timeout_ns, abort);
            failed = __all_sync(0xffffffffu, ok) ? 0 : 1;
            if (failed && lane == 0) {
                *abort = 1;
                atomicCAS(err, 0, -6);
            }
        }
        const float *X = XS + (size_t)slot * XPL * P;
        if (!failed) {
            if (kind == STAGE_PRE) {
#pragma unroll
                for (int pp = 0; pp < TH; ++pp) {
                    xcA[pp] = ld4(X + (TLO + pp + 1) * P + sA);
                    xcB[pp] = ld4(X + (TLO + pp + 1) * P + sB);
                }
            } else {
                const bool full_step = kind == STAGE_FULL;
                float *tn = TS + (size_t)(cb ^ 1) * TPL * P;
                const float *T0 = TS + (size_t)cb * TPL * P;
                float *yo = y + (size_t)v * N + (size_t)(tau < 0 ? 0 : tau) * V + (size_t)z0 * P;
                float4 belowA = ld4(X + TLO * P + sA), hereA = ld4(X + (TLO + 1) * P + sA);
                float4 belowB = ld4(X + TLO * P + sB), hereB = ld4(X + (TLO + 1) * P + sB);
                // t(tau) at planes p - 1 and p of the q march (rolling)
                float4 tbA = make_float4(0.f, 0.f, 0.f, 0.f), tbB = tbA, thA = tbA, thB = tbA;
                if (full_step) {
                    if (PC0 - 1 >= TLO) {
                        tbA = tcA[PC0 - 1 >= TLO ? PC0 - 1 - TLO : 0];
                        tbB = tcB[PC0 - 1 >= TLO ? PC0 - 1 - TLO : 0];
                    } else {   // the plane below is the other part's
                        tbA = ld4(T0 + (PC0 - 1) * P + sA);
                        tbB = ld4(T0 + (PC0 - 1) * P + sB);
                    }
                    thA = tcA[PC0 - TLO];
                    thB = tcB[PC0 - TLO];
                }
#pragma unroll
                for (int pp = 0; pp < TH; ++pp) {
                    const int p = TLO + pp;
                    const float *Xp = X + (p + 1) * P;
                    const float4 aboveA = ld4(X + (p + 2) * P + sA), aboveB = ld4(X + (p + 2) * P + sB);
                    const float4 ymA = ld4(Xp + sM), ypB = ld4(Xp + sP);
                    const float4 lA = lcA[pp], lB = lcB[pp];
                    float hmA, hpA, hmB, hpB;
                    halo(hereA, hmA, hpA);
                    halo(hereB, hmB, hpB);
                    const float4 tA = stencil_x2(hereA, belowA, aboveA, hereB, ymA, hmA, hpA, lA, xcA[pp], mh);
                    const float4 tB = stencil_x2(hereB, belowB, aboveB, ypB, hereA, hmB, hpB, lB, xcB[pp], mh);
                    xcA[pp] = hereA;
                    xcB[pp] = hereB;
                    belowA = hereA;
                    belowB = hereB;
                    hereA = aboveA;
                    hereB = aboveB;
                    if (p >= PC0 && p <= PC1 && full_step) {
                        float4 taA, taB;
                        if (pp + 1 < TH) {
                            taA = tcA[pp + 1 < TH ? pp + 1 : 0];
                            taB = tcB[pp + 1 < TH ? pp + 1 : 0];
                        } else {   // the plane above is the other part's
                            taA = ld4(T0 + (p + 1) * P + sA);
                            taB = ld4(T0 + (p + 1) * P + sB);
                        }
                        const float4 gmA = ld4(T0 + p * P + sM), gpB = ld4(T0 + p * P + sP);
                        float emA, epA, emB, epB;
                        halo(thA, emA, epA);
                        halo(thB, emB, epB);
                        float *yq = yo + (p - 1) * P;
                        st4_global_hint(yq + sA, stencil_x2(thA, tbA, taA, thB, gmA, emA, epA, lA, tA, mh), pol_y);
                        st4_global_hint(yq + sB, stencil_x2(thB, tbB, taB, gpB, thA, emB, epB, lB, tB, mh), pol_y);
                        tbA = thA;
                        tbB = thB;
                        thA = taA;
                        thB = taB;
                    }
                    tcA[pp] = tA;
                    tcB[pp] = tB;
                }
                // The shared-memory copy of t(tau + 1) (the other threads' y
                // neighbours) is written after the march, so that no store
                // sits between the loads of the march.
#pragma unroll
                for (int pp = 0; pp < TH; ++pp) {
                    st4(tn + (TLO + pp) * P + sA, tcA[pp]);
                    st4(tn + (TLO + pp) * P + sB, tcB[pp]);
                }
            }
        }
        if (kind != STAGE_PRE) {
            if (block_sync_or<NTHREADS>(failed)) {
                aborted = true;
                break;
            }
            // Every stage up to j has been read and t(tau + 1) written:
            // stage j's slot can take stage j + NS.
            if (issuer) is.issue_upto(j + NS, c, XS, full, x, L);
            cb ^= 1;
        }
        ++j;
        if (++slot == NS) {
            slot = 0;
            phase ^= 1u;
        }
    }
    if (issuer && aborted) {
        const int never = 0;
        const long long drain_ns = c.timeout_ns > 1000000000LL ? c.timeout_ns : 1000000000LL;
        for (long long jj = j; jj < is.issued; ++jj)
            wait_bounded(&full[(int)(jj % NS)], (unsigned)((jj / NS) & 1), drain_ns, &never);
    }
}

template <int TZ, int NS, int PARTS, int MINB>
__global__ void __launch_bounds__(kPairThreads * PARTS, MINB)
    k_mtm_multi_rp_d3(const MultiCfg c, const float *__restrict__ L, const float *__restrict__ x,
                      float *__restrict__ y, int *err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[NS];
    __shared__ int s_abort;
    using Lay = MultiLayout<TZ, NS>;
    float *XS = (float *)smem_raw;
    float *TS = XS + (size_t)NS * Lay::XPL * c.P;

    const int slab = (int)blockIdx.x % c.nslab;
    const int ci = (int)blockIdx.x / c.nslab;
    const long long K = (long long)c.k * c.g.ntau;
    const long long w0 = (long long)ci * K / c.m, w1 = (long long)(ci + 1) * K / c.m;

    if (threadIdx.x == 0) {
        for (int b = 0; b < NS; ++b) mbar_init(&full[b], 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (PARTS == 1 || (int)threadIdx.x < kPairThreads)
        multi_consumer_rp<TZ, NS, PARTS, 0>(c, XS, TS, full, &s_abort, w0, w1, x, L, y, slab, err);
    else
        multi_consumer_rp<TZ, NS, PARTS, (PARTS > 1 ? 1 : 0)>(c, XS, TS, full, &s_abort, w0, w1, x, L, y, slab, err);
}

template <int TZ, int NS, int PARTS, int MINB>
cudaError_t launch_multi_rp(MultiCfg c, int nsm, const float *L, const float *x, float *y, int *err,
                            cudaStream_t st)
{
    const size_t smem = MultiLayout<TZ, NS>::smem(c.P);
    auto kern = k_mtm_multi_rp_d3<TZ, NS, PARTS, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    c.nslab = c.g.nx / TZ;
    const int ctas = nsm * MINB;
    c.m = ctas / c.nslab > 0 ? ctas / c.nslab : 1;
    kern<<<c.m * c.nslab, kPairThreads * PARTS, smem, st>>>(c, L, x, y, err);
    return cudaGetLastError();
}

// TZ: core z planes of a slab; NS: pipeline stages; PARTS: parts of the
// slab's planes (256 threads each); MINB: CTAs per SM.
template <int NX, int TZ, int NS, int PARTS, int MINB>
__global__ void __launch_bounds__(kPartThreads * PARTS, MINB)
    k_mtm_multi_d3(const MultiCfg c, const float *__restrict__ L, const float *__restrict__ x,
                   float *__restrict__ y, int *err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[NS];
    __shared__ int s_abort;
    __shared__ Issuer<TZ, NS> s_issuer;
    using Lay = MultiLayout<TZ, NS>;
    float *XS = (float *)smem_raw;                       // NS stages of x (XPL planes each)
    float *TS = XS + (size_t)NS * Lay::XPL * c.P;        // two t buffers (TPL planes each)

    const int slab = (int)blockIdx.x % c.nslab;
    const int ci = (int)blockIdx.x / c.nslab;
    const long long K = (long long)c.k * c.g.ntau;
    const long long w0 = (long long)ci * K / c.m, w1 = (long long)(ci + 1) * K / c.m;

    if (threadIdx.x == 0) {
        for (int b = 0; b < NS; ++b) mbar_init(&full[b], 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (PARTS == 1 || (int)threadIdx.x < kPartThreads)
        multi_consumer<NX, TZ, NS, PARTS, 0>(c, XS, TS, full, &s_abort, &s_issuer, w0, w1, x, L, y, slab, err);
    else
        multi_consumer<NX, TZ, NS, PARTS, (PARTS > 1 ? 1 : 0)>(c, XS, TS, full, &s_abort, &s_issuer, w0, w1, x,
                                                               L, y, slab, err);
}

template <int NX, int TZ, int NS, int PARTS, int MINB>
cudaError_t launch_multi(MultiCfg c, int nsm, const float *L, const float *x, float *y, int *err, cudaStream_t st)
{
    const size_t smem = MultiLayout<TZ, NS>::smem(c.P);
    auto kern = k_mtm_multi_d3<NX, TZ, NS, PARTS, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    c.nslab = c.g.nx / TZ;
    const int ctas = nsm * MINB;
    c.m = ctas / c.nslab > 0 ? ctas / c.nslab : 1;
    kern<<<c.m * c.nslab, kPartThreads * PARTS, smem, st>>>(c, L, x, y, err);
    return cudaGetLastError();
}

// Pipeline forms (HH_APPLY_MULTI_FORM selects one):
//   5 (default for N_x = 32): row pairs, 8-plane slabs, two stages, two parts
//      of 128 threads, one CTA per SM (176 KB of shared memory);
//   2 (default otherwise): one float4 group per thread, 4-plane slabs, two
//      stages, one part of 256 threads, two CTAs per SM (112 KB each);
//   1: one group per thread, 8-plane slabs, three stages, two parts, one CTA
//      per SM (8 | N_x);
//   3: one group per thread, 4-plane slabs, four stages, two parts, one CTA
//      per SM;
//   4 (N_x = 32): row pairs, 4-plane slabs, two stages, one part of 128
//      threads, two CTAs per SM.
// Measured on GB300 (32^3 x 128, 16 vectors per launch, cold L2, fraction of
// the measured HBM bandwidth on (8 k + 4) bytes per site): 5: 0.52-0.535;
// 2: 0.47-0.48; 1: 0.47; 4: 0.40-0.49; 3: 0.34.  Variants with more warps
// per SM (two parts of row pairs in two CTAs per SM) or with a producer warp
// of their own ran out of registers (at most 128 and 168 per thread) and
// were slower.
int multi_form(int nx)
{
    const char *e = getenv("HH_APPLY_MULTI_FORM");
    const int forced = e ? atoi(e) : 0;
    if (forced == 1 && nx % 8 == 0) return 1;
    if (forced == 2 || forced == 3) return forced;
    if ((forced == 4 || forced == 5) && nx == 32) return forced;
    return nx == 32 ? 5 : 2;
}

size_t multi_smem(int nx, int form)
{
    const int P = nx * nx;
    switch (form) {
    case 1: return MultiLayout<8, 3>::smem(P);
    case 2: return MultiLayout<4, 2>::smem(P);
    case 4: return MultiLayout<4, 2>::smem(P);
    case 5: return MultiLayout<8, 2>::smem(P);
    default: return MultiLayout<4, 4>::smem(P);
    }
}

}  // namespace

bool multi_mtm_ok(const Geo &g, const void *L, const void *x, const void *y)
{
    if (g.d != 3 || g.nx % 4 != 0 || g.nx < 4 || g.nx > 32 || g.ntau < 2) return false;
    if (((uintptr_t)L | (uintptr_t)x | (uintptr_t)y) & 15u) return false;
    // dynamic shared memory, leaving 1 KB of the 227 KB for the static part
    // (two CTAs per SM: half of it each)
    const int form = multi_form(g.nx);
    return multi_smem(g.nx, form) <= (form == 2 || form == 4 ? 112 : 226) * 1024;
}

cudaError_t launch_mtm_multi_f32(const Geo &g, float h, const float *L, const float *x, float *y, int k, int *err,
                                 int nsm, long long timeout_ns, cudaStream_t st)
{
    if (k < 1) return cudaSuccess;
    MultiCfg c;
    c.g = g;
    c.h = h;
    c.P = g.nx * g.nx;
    c.k = k;
    const int G = c.P / 4, gpr = g.nx / 4;
    c.shfl = (32 % gpr == 0) && (G % 32 == 0);
    c.timeout_ns = timeout_ns;
    const char *pfe = getenv("HH_APPLY_MULTI_PF");
    c.pf_ahead = pfe ? atoi(pfe) : kPrefetchAhead;
    // Fault injection for the failure-detection tests (HH_APPLY_MULTI_DROP_TX=1).
    const char *dte = getenv("HH_APPLY_MULTI_DROP_TX");
    c.drop_tx = dte ? atoi(dte) : 0;
    const bool n32 = g.nx == 32;
    switch (multi_form(g.nx)) {
    case 1: return n32 ? launch_multi<32, 8, 3, 2, 1>(c, nsm, L, x, y, err, st)
                       : launch_multi<0, 8, 3, 2, 1>(c, nsm, L, x, y, err, st);
    case 2: return n32 ? launch_multi<32, 4, 2, 1, 2>(c, nsm, L, x, y, err, st)
                       : launch_multi<0, 4, 2, 1, 2>(c, nsm, L, x, y, err, st);
    case 4: return launch_multi_rp<4, 2, 1, 2>(c, nsm, L, x, y, err, st);
    case 5: return launch_multi_rp<8, 2, 2, 1>(c, nsm, L, x, y, err, st);
    default: return n32 ? launch_multi<32, 4, 4, 2, 1>(c, nsm, L, x, y, err, st)
                        : launch_multi<0, 4, 4, 2, 1>(c, nsm, L, x, y, err, st);
    }
}

}  // namespace hh
