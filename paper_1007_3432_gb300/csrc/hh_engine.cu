// Persistent conjugate-gradient engine (Sec. 4.1: CG on Q = M^T M).
// The slot/mode structure is described in hh_engine.cuh; the host-side
// policies (tiling, layouts, prefetch distance, the Chebyshev table) are in
// hh_engine_host.cu.
//
// GB300 layout of the work: one 512-thread block per SM, every block owning
// fixed tiles of contiguous sites; a thread handles groups of W consecutive x
// sites, issuing all their loads (the group, its 2d spatial neighbour rows,
// the time neighbour row and the links) before any arithmetic, so that each
// thread has several independent L2/HBM requests in flight.  The lattice
// dimension is a compile-time parameter of the site loops.
#include <cstdlib>

#include "hh_engine.cuh"

namespace hh {

namespace {

constexpr int kNumericErr = -5;
constexpr int kNoConv = -4;

// ---------------------------------------------------------------------------
// Site loops over [b, e) of one system, in groups of W consecutive x sites per
// thread (b and e are multiples of W).  Each returns this thread's partial
// sum (|t|^2 or |r|^2), accumulated in T.
// ---------------------------------------------------------------------------

// t = M v; acc += t^2.                                      (Eq. (10))
// The engine block's compute threads: all of its threads in a flat launch,
// warps 1 .. 15 when warp 0 is the control warp (see the kernel).
constexpr int kCtlThreads = 32;
__shared__ int s_ctl_threads;
__device__ __forceinline__ int ctid()
{
    return (int)threadIdx.x - s_ctl_threads;
}
__device__ __forceinline__ int cnth()
{
    return (int)blockDim.x - s_ctl_threads;
}

template <int D, typename T, int W, typename LK>
__device__ double gloop_M(const Geo g, const T h, const LK L, const T *v, T *t, int b, int e, int pf = 0)
{
    T acc = T(0);
    const int step = W * cnth(), ahead = pf * step;
    for (int i = b + W * ctid(); i < e; i += step) {
        if (ahead && i + ahead < e) {
            const int j = i + ahead, jp = row_prev(g, j);
            prefetch_l2(v + j);
            prefetch_l2(v + jp);
            prefetch_l2(link_addr(L, jp));
        }
        GroupNbr nb;
        group_nbrs<D, W>(g, i, nb);
        Vec<T, W> self = vld<T, W>(v + i);
        Vec<T, W> hs = group_hop<D, T, W>(v, nb, self);
        Vec<T, W> lk = link_row<T, W>(L, nb.prev);
        Vec<T, W> pv = vld<T, W>(v + nb.prev);
        Vec<T, W> out;
#pragma unroll
        for (int u = 0; u < W; ++u) {
            out.a[u] = fma(lk.a[u], pv.a[u], fma(-h, hs.a[u], self.a[u]));
            acc = fma(out.a[u], out.a[u], acc);
        }
        vst<T, W>(t + i, out);
    }
    return (double)acc;
}

// CG slot 3: q = M^T t, x += alpha p, r -= alpha q; acc += r^2.
template <int D, typename T, int W, typename LK>
__device__ double gloop_update(const Geo g, const T h, const LK L, const T *t, T *x, const T *p, T *r,
                               const T alpha, int b, int e, int pf = 0)
{
    T acc = T(0);
    const int step = W * cnth(), ahead = pf * step;
    for (int i = b + W * ctid(); i < e; i += step) {
        if (ahead && i + ahead < e) {
            const int j = i + ahead;
            prefetch_l2(t + j);
            prefetch_l2(t + row_next(g, j));
            prefetch_l2(link_addr(L, j));
            prefetch_l2(x + j);
            prefetch_l2(p + j);
            prefetch_l2(r + j);
        }
        GroupNbr nb;
        group_nbrs<D, W>(g, i, nb);
        Vec<T, W> self = vld<T, W>(t + i);
        Vec<T, W> hs = group_hop<D, T, W>(t, nb, self);
        Vec<T, W> lk = link_row<T, W>(L, i);
        Vec<T, W> nv = vld<T, W>(t + nb.next);
        Vec<T, W> xv = vld<T, W>(x + i);
        Vec<T, W> pv = vld<T, W>(p + i);
        Vec<T, W> rv = vld<T, W>(r + i);
#pragma unroll
        for (int u = 0; u < W; ++u) {
            T q = fma(lk.a[u], nv.a[u], fma(-h, hs.a[u], self.a[u]));
            xv.a[u] = fma(alpha, pv.a[u], xv.a[u]);
            rv.a[u] = fma(-alpha, q, rv.a[u]);
            acc = fma(rv.a[u], rv.a[u], acc);
        }
        vst<T, W>(x + i, xv);
        vst<T, W>(r + i, rv);
    }
    return (double)acc;
}

// RU slot 3 (FP64): res = b - M^T t64; r64 = res and, for a mixed system,
// r32 = (float)res; acc += res^2.
template <int D, int W>
__device__ double gloop_residual(const Geo g, const double h, const double *__restrict__ L,
                                 const double *t, const double *__restrict__ bvec, double *r, float *r32,
                                 int b, int e)
{
    double acc = 0.0;
    for (int i = b + W * ctid(); i < e; i += W * cnth()) {
        GroupNbr nb;
        group_nbrs<D, W>(g, i, nb);
        Vec<double, W> self = vld<double, W>(t + i);
        Vec<double, W> hs = group_hop<D, double, W>(t, nb, self);
        Vec<double, W> lk = vldg<double, W>(L + i);
        Vec<double, W> nv = vld<double, W>(t + nb.next);
        Vec<double, W> bv = vldg<double, W>(bvec + i);
        Vec<float, W> r32v;
#pragma unroll
        for (int u = 0; u < W; ++u) {
            double q = fma(lk.a[u], nv.a[u], fma(-h, hs.a[u], self.a[u]));
            bv.a[u] = bv.a[u] - q;
            r32v.a[u] = (float)bv.a[u];
            acc = fma(bv.a[u], bv.a[u], acc);
        }
        vst<double, W>(r + i, bv);
        if (r32) vst<float, W>(r32 + i, r32v);
    }
    return acc;
}

// Preconditioner sub-step of an even index: u = (Q/lam) z - a z, from t = M z.
template <int D, int W>
__device__ void gloop_cheb_u(const Geo g, const double h, const double *__restrict__ L, const double *t,
                             const double *z, double *u, const double invlam, const double a, int b, int e,
                             int pf = 0)
{
    const int step = W * cnth(), ahead = pf * step;
    for (int i = b + W * ctid(); i < e; i += step) {
        if (ahead && i + ahead < e) {
            const int j = i + ahead;
            prefetch_l2(t + j);
            prefetch_l2(t + row_next(g, j));
            prefetch_l2(L + j);
            prefetch_l2(z + j);
        }
        GroupNbr nb;
        group_nbrs<D, W>(g, i, nb);
        Vec<double, W> self = vld<double, W>(t + i);
        Vec<double, W> hs = group_hop<D, double, W>(t, nb, self);
        Vec<double, W> lk = vldg<double, W>(L + i);
        Vec<double, W> nv = vld<double, W>(t + nb.next);
        Vec<double, W> zv = vld<double, W>(z + i);
#pragma unroll
        for (int k = 0; k < W; ++k) {
            double q = fma(lk.a[k], nv.a[k], fma(-h, hs.a[k], self.a[k]));
            zv.a[k] = fma(q, invlam, -a * zv.a[k]);
        }
        vst<double, W>(u + i, zv);
    }
}

// Odd index: z = ((Q/lam) u - a u + b2 z) * invq, from t = M u; after the last
// factor also z *= scale and acc += r . z.
template <int D, int W>
__device__ double gloop_cheb_z(const Geo g, const double h, const double *__restrict__ L, const double *t,
                               const double *u, double *z, const double *r, const double invlam,
                               const double a, const double b2, const double invq, const double scale,
                               bool dot, int b, int e, int pf = 0)
{
    double acc = 0.0;
    const int step = W * cnth(), ahead = pf * step;
    for (int i = b + W * ctid(); i < e; i += step) {
        if (ahead && i + ahead < e) {
            const int j = i + ahead;
            prefetch_l2(t + j);
            prefetch_l2(t + row_next(g, j));
            prefetch_l2(L + j);
            prefetch_l2(u + j);
            prefetch_l2(z + j);
            if (dot) prefetch_l2(r + j);
        }
        GroupNbr nb;
        group_nbrs<D, W>(g, i, nb);
        Vec<double, W> self = vld<double, W>(t + i);
        Vec<double, W> hs = group_hop<D, double, W>(t, nb, self);
        Vec<double, W> lk = vldg<double, W>(L + i);
        Vec<double, W> nv = vld<double, W>(t + nb.next);
        Vec<double, W> uv = vld<double, W>(u + i);
        Vec<double, W> zv = vld<double, W>(z + i);
        Vec<double, W> rv;
        if (dot) rv = vld<double, W>(r + i);
#pragma unroll
        for (int k = 0; k < W; ++k) {
            double q = fma(lk.a[k], nv.a[k], fma(-h, hs.a[k], self.a[k]));
            double v = fma(q, invlam, fma(-a, uv.a[k], b2 * zv.a[k]));
            zv.a[k] = v * invq * scale;
            if (dot) acc = fma(rv.a[k], zv.a[k], acc);
        }
        vst<double, W>(z + i, zv);
    }
    return acc;
}

// Exact-block form of M (link_order 1, 2): scalar site loops with the stencils
// of hh_device.cuh.  t = M p, acc += t^2.
template <typename T>
__device__ double gloop_M_ex(const Geo g, const T h, const T *__restrict__ L, const T *v, T *t, int order,
                             int b, int e)
{
    T acc = T(0);
    Nbr nb;
    for (int i = b + ctid(); i < e; i += cnth()) {
        neighbours(g, i, nb);
        const T y = stencil_M_ex<T>(g, h, L, v, i, nb, order);
        t[i] = y;
        acc = fma(y, y, acc);
    }
    return (double)acc;
}

// q = M^T t, x += alpha p, r -= alpha q; acc += r^2.
template <typename T>
__device__ double gloop_update_ex(const Geo g, const T h, const T *__restrict__ L, const T *t, T *x,
                                  const T *p, T *r, const T alpha, int order, int b, int e)
{
    T acc = T(0);
    Nbr nb;
    for (int i = b + ctid(); i < e; i += cnth()) {
        neighbours(g, i, nb);
        const T q = stencil_MT_ex<T>(g, h, L, t, i, nb, order);
        x[i] = fma(alpha, p[i], x[i]);
        const T rv = fma(-alpha, q, r[i]);
        r[i] = rv;
        acc = fma(rv, rv, acc);
    }
    return (double)acc;
}

// res = b - M^T t64 in FP64; r64 = res, r32 = (float)res (mixed); acc += res^2.
__device__ double gloop_residual_ex(const Geo g, const double h, const double *__restrict__ L,
                                    const double *t, const double *__restrict__ bvec, double *r, float *r32,
                                    int order, int b, int e)
{
    double acc = 0.0;
    Nbr nb;
    for (int i = b + ctid(); i < e; i += cnth()) {
        neighbours(g, i, nb);
        const double res = __ldg(bvec + i) - stencil_MT_ex<double>(g, h, L, t, i, nb, order);
        r[i] = res;
        if (r32) r32[i] = (float)res;
        acc = fma(res, res, acc);
    }
    return acc;
}

// Two-slot CG step: p_new = src + beta p_old on the tile's sites (stored), and
// t = M p_new with p_new recomputed at the neighbour sites from src and p_old,
// which are final there; acc += t^2.  The recomputed values are bitwise the
// ones their owners store (the same fma on the same inputs).
template <int D, typename T, int W, typename LK>
__device__ double gloop_pM(const Geo g, const T h, const LK L, const T *src, const T *pold, T *pnew, T *t,
                           const T beta, bool restart, int b, int e, int pf = 0)
{
    T acc = T(0);
    const int step = W * cnth(), ahead = pf * step;
    for (int i = b + W * ctid(); i < e; i += step) {
        if (ahead && i + ahead < e) {
            const int j = i + ahead, jp = row_prev(g, j);
            prefetch_l2(src + j);
            prefetch_l2(src + jp);
            prefetch_l2(link_addr(L, jp));
            if (!restart) {
                prefetch_l2(pold + j);
                prefetch_l2(pold + jp);
            }
        }
        GroupNbr nb;
        group_nbrs<D, W>(g, i, nb);
        auto pn_at = [&](int j) -> T {
            const T sv = src[j];
            return restart ? sv : fma(beta, pold[j], sv);
        };
        auto pn_row = [&](int j) -> Vec<T, W> {
            Vec<T, W> sv = vld<T, W>(src + j);
            if (!restart) {
                const Vec<T, W> q = vld<T, W>(pold + j);
#pragma unroll
                for (int u = 0; u < W; ++u) sv.a[u] = fma(beta, q.a[u], sv.a[u]);
            }
            return sv;
        };
        const Vec<T, W> self = pn_row(i);
        vst<T, W>(pnew + i, self);
        const T vl = pn_at(nb.left), vr = pn_at(nb.right);
        Vec<T, W> yp, ym, zp, zm;
        if (D == 3) {
            yp = pn_row(nb.yp);
            ym = pn_row(nb.ym);
            zp = pn_row(nb.zp);
            zm = pn_row(nb.zm);
        }
        const Vec<T, W> pv = pn_row(nb.prev);
        const Vec<T, W> lk = link_row<T, W>(L, nb.prev);
        Vec<T, W> out;
#pragma unroll
        for (int u = 0; u < W; ++u) {
            T xr = (u == W - 1) ? vr : self.a[u + 1 < W ? u + 1 : u];
            T xl = (u == 0) ? vl : self.a[u > 0 ? u - 1 : 0];
            T hsum = xr + xl;
            if (D == 3) hsum += (yp.a[u] + ym.a[u]) + (zp.a[u] + zm.a[u]);
            out.a[u] = fma(lk.a[u], pv.a[u], fma(-h, hsum, self.a[u]));
            acc = fma(out.a[u], out.a[u], acc);
        }
        vst<T, W>(t + i, out);
    }
    return (double)acc;
}

// Two-slot reliable update, first half: t64 = M (x64 + x32) with the sum
// formed at every site read (x64 and x32 are only written in slot 3).
template <int D, int W>
__device__ void gloop_accM(const Geo g, const double h, const double *__restrict__ L, const double *x,
                           const float *x32, double *t, int b, int e)
{
    for (int i = b + W * ctid(); i < e; i += W * cnth()) {
        GroupNbr nb;
        group_nbrs<D, W>(g, i, nb);
        auto xs_at = [&](int j) -> double { return x[j] + (double)x32[j]; };
        auto xs_row = [&](int j) -> Vec<double, W> {
            Vec<double, W> a = vld<double, W>(x + j);
            const Vec<float, W> c = vld<float, W>(x32 + j);
#pragma unroll
            for (int u = 0; u < W; ++u) a.a[u] += (double)c.a[u];
            return a;
        };
        const Vec<double, W> self = xs_row(i);
        const double vl = xs_at(nb.left), vr = xs_at(nb.right);
        Vec<double, W> yp, ym, zp, zm;
        if (D == 3) {
            yp = xs_row(nb.yp);
            ym = xs_row(nb.ym);
            zp = xs_row(nb.zp);
            zm = xs_row(nb.zm);
        }
        const Vec<double, W> pv = xs_row(nb.prev);
        const Vec<double, W> lk = vldg<double, W>(L + nb.prev);
        Vec<double, W> out;
#pragma unroll
        for (int u = 0; u < W; ++u) {
            double xr = (u == W - 1) ? vr : self.a[u + 1 < W ? u + 1 : u];
            double xl = (u == 0) ? vl : self.a[u > 0 ? u - 1 : 0];
            double hsum = xr + xl;
            if (D == 3) hsum += (yp.a[u] + ym.a[u]) + (zp.a[u] + zm.a[u]);
            out.a[u] = fma(lk.a[u], pv.a[u], fma(-h, hsum, self.a[u]));
        }
        vst<double, W>(t + i, out);
    }
}

// p = r + beta p (restart: p = r).
template <typename T, int W>
__device__ void gloop_direction(const T *r, T *p, const T beta, bool restart, int b, int e, int pf = 0)
{
    const int step = W * cnth(), ahead = pf * step;
    for (int i = b + W * ctid(); i < e; i += step) {
        if (ahead && i + ahead < e) {
            prefetch_l2(r + i + ahead);
            if (!restart) prefetch_l2(p + i + ahead);
        }
        Vec<T, W> rv = vld<T, W>(r + i);
        if (!restart) {
            Vec<T, W> pv = vld<T, W>(p + i);
#pragma unroll
            for (int u = 0; u < W; ++u) rv.a[u] = fma(beta, pv.a[u], rv.a[u]);
        }
        vst<T, W>(p + i, rv);
    }
}

// x64 += x32, x32 = 0 (reliable update of a mixed system).
template <int W>
__device__ void gloop_accumulate(double *x, float *x32, int b, int e)
{
    for (int i = b + W * ctid(); i < e; i += W * cnth()) {
        Vec<double, W> xv = vld<double, W>(x + i);
        Vec<float, W> yv = vld<float, W>(x32 + i), z;
#pragma unroll
        for (int u = 0; u < W; ++u) {
            xv.a[u] += (double)yv.a[u];
            z.a[u] = 0.0f;
        }
        vst<double, W>(x + i, xv);
        vst<float, W>(x32 + i, z);
    }
}

// ---------------------------------------------------------------------------
// Per-system decisions.
// ---------------------------------------------------------------------------

// Next mode of a system from its previous state and the |r|^2 (or, after the
// last preconditioner sub-step, <r, z>) reduced from the previous iteration's
// slot 3.  Pure function of its inputs: all blocks agree.
__device__ EngState decide(const EngSystem &Y, const EngState &P, double rr)
{
    EngState S = P;
    switch (P.mode) {
    case MODE_DONE:
        return S;
    case MODE_NEW:
        S.mode = MODE_INIT;
        S.cg_steps = 0;
        S.n_ru = 0;
        S.status = 0;
        S.final_ru = 0;
        S.true_relres = 1.0;
        S.prec = Y.precision;
        S.stall = 0;
        S.fp64_steps = 0;
        S.since_ru = 0;
        S.pre_j = 0;
        S.no_guess = 0;
        return S;
    case MODE_INIT:
        S.bb = rr;
        S.rr_last = rr;
        S.rr_ru = rr;
        if (!isfinite(rr)) {
            S.mode = MODE_DONE;
            S.status = kNumericErr;
            return S;
        }
        if (Y.x0_given && !P.no_guess) {
            if (rr == 0.0) {
                // b = 0: the solution is x = 0 whatever the guess; one more
                // INIT zeroes x.
                S.no_guess = 1;
                return S;
            }
            // Initial guess: the true residual b - Q x0 first (an RU step),
            // then CG from it (beta = rr / inf = 0 restarts).  The guess's
            // residual is not a stall of the mixed iteration.
            S.mode = MODE_RU;
            S.rr_alpha = INFINITY;
            S.rr_ru = INFINITY;
            S.rr_last = INFINITY;
            S.maxr2 = rr;
            return S;
        }
        if (rr == 0.0) {
            S.mode = MODE_DONE;
            S.true_relres = 0.0;
            return S;
        }
        S.mode = MODE_CG;
        S.beta = 0.0;
        S.rr_alpha = rr;
        S.maxr2 = rr;
        if (Y.cheb_n > 0) {
            // PCG: first precondition r = b; beta = 0 marks the first step.
            S.mode = MODE_PRE;
            S.pre_j = 0;
            S.rr_alpha = 0.0;
        }
        return S;
    case MODE_PRE: {
        // rr is <r, z> after the last sub-step (published in slot 3).
        if (P.pre_j + 1 < 2 * Y.cheb_n) {
            S.pre_j = P.pre_j + 1;
            return S;
        }
        if (!isfinite(rr) || rr <= 0.0) {
            S.mode = MODE_DONE;
            S.status = kNumericErr;
            return S;
        }
        S.mode = MODE_CG;
        S.beta = (P.rr_alpha > 0.0) ? rr / P.rr_alpha : 0.0;
        S.rr_alpha = rr;
        return S;
    }
    case MODE_CG: {
        S.cg_steps = P.cg_steps + 1;
        if (P.prec == PREC_FP64) S.fp64_steps = P.fp64_steps + 1;
        S.rr_last = rr;
        if (!isfinite(rr)) {
            S.mode = MODE_DONE;
            S.status = kNumericErr;
            return S;
        }
        S.since_ru = P.since_ru + 1;
        bool need = rr <= Y.tol2 * P.bb;
        if (P.prec == PREC_MIXED && rr < Y.delta2 * P.maxr2) need = true;
        if (P.prec == PREC_MIXED && S.since_ru >= Y.stall_window) need = true;
        if (S.cg_steps >= Y.maxit) {
            need = true;
            S.final_ru = 1;
        }
        if (need) {
            S.mode = MODE_RU;
            return S;
        }
        if (Y.cheb_n > 0) {
            S.mode = MODE_PRE;
            S.pre_j = 0;
            return S;
        }
        S.mode = MODE_CG;
        S.beta = rr / P.rr_alpha;
        S.rr_alpha = rr;
        S.maxr2 = fmax(P.maxr2, rr);
        return S;
    }
    case MODE_RU:
    default: {
        S.n_ru = P.n_ru + 1;
        S.rr_last = rr;
        S.true_relres = sqrt(rr / P.bb);
        if (!isfinite(rr)) {
            S.mode = MODE_DONE;
            S.status = kNumericErr;
            return S;
        }
        if (rr <= Y.tol2 * P.bb) {
            S.mode = MODE_DONE;
            S.status = 0;
            return S;
        }
        if (P.final_ru) {
            S.mode = MODE_DONE;
            S.status = kNoConv;
            return S;
        }
        S.mode = MODE_CG;
        S.beta = rr / P.rr_alpha;
        S.rr_alpha = rr;
        S.maxr2 = rr;
        S.since_ru = 0;
        if (Y.cheb_n > 0) {
            // PCG after residual replacement: precondition the new r; beta
            // comes from <r, z> at the end of the sub-steps.
            S.mode = MODE_PRE;
            S.pre_j = 0;
            S.rr_alpha = P.rr_alpha;
            S.rr_ru = rr;
            return S;
        }
        if (P.prec == PREC_MIXED) {
            // A reliable update that did not halve the true residual norm
            // since the previous one (whether the FP32 residual fell below
            // delta or the stall window ran out) means the FP32 steps have
            // stopped making progress (eps_32 * cond(Q) >~ 1).  After two
            // stalls in a row the system continues with FP64 CG steps from a
            // restart at the FP64 residual.
            // Also a stall: the true residual is more than 4x (in norm) the
            // FP32 recursive residual that triggered this update, i.e. the
            // FP32 recursion no longer tracks b - Q x.
            const bool no_progress = rr > 0.25 * P.rr_ru;
            const bool drifted = rr > 16.0 * P.rr_last;
            S.stall = (no_progress || drifted) ? P.stall + 1 : 0;
            if (S.stall >= 2) {
                S.prec = PREC_FP64;
                S.beta = 0.0;
            }
        }
        S.rr_ru = rr;
        return S;
    }
    }
}

// ---------------------------------------------------------------------------
// Slot bodies for one tile (D and W fixed; mode and precision from the state).
// ---------------------------------------------------------------------------
struct TileCtl {
    int mode, prec, pre_j, two;    // two: the launch runs the two-slot form
    int pold, pnew;                // p buffers holding the previous / new direction
    int zero_x, pad1;              // INIT: x starts at 0 (else x holds the guess)
    double beta, alpha;
};

// Tile controls of a system in state S.  Three-slot form: the direction is
// updated in place in buffer S.pbuf.  Two-slot form: each CG step writes the
// new direction to S.pbuf and reads the previous one from the other buffer.
__device__ __forceinline__ TileCtl make_ctl(const EngState &S, int two, int x0_given)
{
    TileCtl c;
    c.mode = S.mode;
    c.prec = S.prec;
    c.pre_j = S.pre_j;
    c.two = two;
    c.pnew = S.pbuf;
    c.pold = two ? (S.pbuf ^ 1) : S.pbuf;
    c.zero_x = (x0_given && !S.no_guess) ? 0 : 1;
    c.pad1 = 0;
    c.beta = S.beta;
    c.alpha = 0.0;
    return c;
}

__device__ __forceinline__ LinkSrc link_src(const EngSystem &Y)
{
    return LinkSrc{Y.L16, Y.link16, Y.l16_scale};
}

__device__ __forceinline__ double *pbuf64(const EngSystem &Y, int k)
{
    return k ? Y.p2 : Y.p;
}

__device__ __forceinline__ float *pbuf32(const EngSystem &Y, int k)
{
    return k ? Y.p32b : Y.p32;
}

// r = b (and r32 = b for a mixed system); returns this thread's |b|^2.
__device__ double init_residual(const EngSystem &Y, const EngTile &T)
{
    double acc = 0.0;
    for (int i = T.begin + ctid(); i < T.end; i += cnth()) {
        double bi = __ldg(Y.b + i);
        Y.r[i] = bi;
        if (Y.precision == PREC_MIXED) Y.r32[i] = (float)bi;
        acc = fma(bi, bi, acc);
    }
    return acc;
}

template <int D, int W, bool PF = true>
__device__ void slot1(const EngSystem &Y, const TileCtl &c, const EngTile &T)
{
    const int pf = PF ? Y.pf : 0;
    if (c.mode == MODE_PRE) {
        if (c.pre_j == 0) gloop_direction<double, W>(Y.r, Y.z, 0.0, true, T.begin, T.end);
    } else if (c.mode == MODE_CG) {
        bool restart = (c.beta == 0.0);
        if (Y.cheb_n > 0)
            gloop_direction<double, W>(Y.z, pbuf64(Y, c.pnew), c.beta, restart, T.begin, T.end, pf);
        else if (c.prec == PREC_FP64)
            gloop_direction<double, W>(Y.r, pbuf64(Y, c.pnew), c.beta, restart, T.begin, T.end, pf);
        else
            gloop_direction<float, W>(Y.r32, pbuf32(Y, c.pnew), (float)c.beta, restart, T.begin, T.end, pf);
    } else if (c.mode == MODE_RU) {
        if (c.prec == PREC_MIXED && !c.two) gloop_accumulate<W>(Y.x, Y.x32, T.begin, T.end);
    } else if (c.mode == MODE_INIT) {
        if (c.zero_x)
            for (int i = T.begin + ctid(); i < T.end; i += cnth()) Y.x[i] = 0.0;
        if (Y.precision == PREC_MIXED)
            for (int i = T.begin + ctid(); i < T.end; i += cnth()) Y.x32[i] = 0.0f;
    }
}

template <int D, int W, bool PF = true, bool L16 = false>
__device__ double slot2(const EngSystem &Y, const TileCtl &c, const EngTile &T)
{
    const int pf = PF ? Y.pf : 0;
    if (c.mode == MODE_CG) {
        if (c.prec == PREC_FP64)
            return gloop_M<D, double, W>(Y.g, Y.h, Y.L64, pbuf64(Y, c.pnew), Y.t, T.begin, T.end, pf);
        if constexpr (L16)
            return gloop_M<D, float, W>(Y.g, (float)Y.h, link_src(Y), pbuf32(Y, c.pnew), Y.t32, T.begin, T.end,
                                        pf);
        else
            return gloop_M<D, float, W>(Y.g, (float)Y.h, Y.L32, pbuf32(Y, c.pnew), Y.t32, T.begin, T.end, pf);
    }
    if (c.mode == MODE_RU) gloop_M<D, double, W>(Y.g, Y.h, Y.L64, Y.x, Y.t, T.begin, T.end);
    if (c.mode == MODE_PRE)
        gloop_M<D, double, W>(Y.g, Y.h, Y.L64, (c.pre_j & 1) ? Y.u : Y.z, Y.t, T.begin, T.end, pf);
    return 0.0;
}

template <int D, int W, bool PF = true, bool L16 = false>
__device__ double slot3(const EngSystem &Y, const TileCtl &c, const EngTile &T)
{
    const int pf = PF ? Y.pf : 0;
    if (c.mode == MODE_CG) {
        if (c.prec == PREC_FP64)
            return gloop_update<D, double, W>(Y.g, Y.h, Y.L64, Y.t, Y.x, pbuf64(Y, c.pnew), Y.r, c.alpha,
                                              T.begin, T.end, pf);
        if constexpr (L16)
            return gloop_update<D, float, W>(Y.g, (float)Y.h, link_src(Y), Y.t32, Y.x32, pbuf32(Y, c.pnew),
                                             Y.r32, (float)c.alpha, T.begin, T.end, pf);
        else
            return gloop_update<D, float, W>(Y.g, (float)Y.h, Y.L32, Y.t32, Y.x32, pbuf32(Y, c.pnew), Y.r32,
                                             (float)c.alpha, T.begin, T.end, pf);
    }
    if (c.mode == MODE_RU) {
        // Two-slot form: the mixed reliable update accumulates here, after
        // every block has read x64 + x32 for t64 in the previous slot.
        if (c.two && c.prec == PREC_MIXED) gloop_accumulate<W>(Y.x, Y.x32, T.begin, T.end);
        return gloop_residual<D, W>(Y.g, Y.h, Y.L64, Y.t, Y.b, Y.r,
                                    Y.precision == PREC_MIXED ? Y.r32 : nullptr, T.begin, T.end);
    }
    if (c.mode == MODE_PRE) {
        const int k = c.pre_j >> 1;
        const double invlam = __ldg(Y.cheb), a = __ldg(Y.cheb + 2 + 3 * k);
        if ((c.pre_j & 1) == 0) {
            gloop_cheb_u<D, W>(Y.g, Y.h, Y.L64, Y.t, Y.z, Y.u, invlam, a, T.begin, T.end, pf);
            return 0.0;
        }
        const bool last = (c.pre_j == 2 * Y.cheb_n - 1);
        const double b2 = __ldg(Y.cheb + 3 + 3 * k), invq = __ldg(Y.cheb + 4 + 3 * k);
        return gloop_cheb_z<D, W>(Y.g, Y.h, Y.L64, Y.t, Y.u, Y.z, Y.r, invlam, a, b2, invq,
                                  last ? __ldg(Y.cheb + 1) : 1.0, last, T.begin, T.end, pf);
    }
    if (c.mode == MODE_INIT) return init_residual(Y, T);
    return 0.0;
}

// Slots 2 and 3 of a system with the exact-block form of M (three-slot
// form; CG, RU and INIT modes).
__device__ double slot2_ex(const EngSystem &Y, const TileCtl &c, const EngTile &T)
{
    if (c.mode == MODE_CG) {
        if (c.prec == PREC_FP64)
            return gloop_M_ex<double>(Y.g, Y.h, Y.L64, pbuf64(Y, c.pnew), Y.t, Y.link_order, T.begin, T.end);
        return gloop_M_ex<float>(Y.g, (float)Y.h, Y.L32, pbuf32(Y, c.pnew), Y.t32, Y.link_order, T.begin, T.end);
    }
    if (c.mode == MODE_RU) gloop_M_ex<double>(Y.g, Y.h, Y.L64, Y.x, Y.t, Y.link_order, T.begin, T.end);
    return 0.0;
}

__device__ double slot3_ex(const EngSystem &Y, const TileCtl &c, const EngTile &T)
{
    if (c.mode == MODE_CG) {
        if (c.prec == PREC_FP64)
            return gloop_update_ex<double>(Y.g, Y.h, Y.L64, Y.t, Y.x, pbuf64(Y, c.pnew), Y.r, c.alpha,
                                           Y.link_order, T.begin, T.end);
        return gloop_update_ex<float>(Y.g, (float)Y.h, Y.L32, Y.t32, Y.x32, pbuf32(Y, c.pnew), Y.r32,
                                      (float)c.alpha, Y.link_order, T.begin, T.end);
    }
    if (c.mode == MODE_RU)
        return gloop_residual_ex(Y.g, Y.h, Y.L64, Y.t, Y.b, Y.r, Y.precision == PREC_MIXED ? Y.r32 : nullptr,
                                 Y.link_order, T.begin, T.end);
    if (c.mode == MODE_INIT) return init_residual(Y, T);
    return 0.0;
}

// Two-slot first slot: slot 1 folded into slot 2.  Returns this thread's
// |t|^2 partial for a CG step (0 otherwise).
template <int D, int W, bool PF = true, bool L16 = false>
__device__ double slotA(const EngSystem &Y, const TileCtl &c, const EngTile &T)
{
    const int pf = PF ? Y.pf : 0;
    if (c.mode == MODE_CG) {
        const bool restart = (c.beta == 0.0);
        if (Y.cheb_n > 0)
            return gloop_pM<D, double, W>(Y.g, Y.h, Y.L64, Y.z, pbuf64(Y, c.pold), pbuf64(Y, c.pnew), Y.t,
                                          c.beta, restart, T.begin, T.end, pf);
        if (c.prec == PREC_FP64)
            return gloop_pM<D, double, W>(Y.g, Y.h, Y.L64, Y.r, pbuf64(Y, c.pold), pbuf64(Y, c.pnew), Y.t,
                                          c.beta, restart, T.begin, T.end, pf);
        if constexpr (L16)
            return gloop_pM<D, float, W>(Y.g, (float)Y.h, link_src(Y), Y.r32, pbuf32(Y, c.pold),
                                         pbuf32(Y, c.pnew), Y.t32, (float)c.beta, restart, T.begin, T.end, pf);
        else
            return gloop_pM<D, float, W>(Y.g, (float)Y.h, Y.L32, Y.r32, pbuf32(Y, c.pold), pbuf32(Y, c.pnew),
                                         Y.t32, (float)c.beta, restart, T.begin, T.end, pf);
    }
    if (c.mode == MODE_RU) {
        if (c.prec == PREC_MIXED)
            gloop_accM<D, W>(Y.g, Y.h, Y.L64, Y.x, Y.x32, Y.t, T.begin, T.end);
        else
            gloop_M<D, double, W>(Y.g, Y.h, Y.L64, Y.x, Y.t, T.begin, T.end);
        return 0.0;
    }
    if (c.mode == MODE_PRE) {
        if (c.pre_j == 0)
            gloop_pM<D, double, W>(Y.g, Y.h, Y.L64, Y.r, Y.r, Y.z, Y.t, 0.0, true, T.begin, T.end, pf);
        else
            gloop_M<D, double, W>(Y.g, Y.h, Y.L64, (c.pre_j & 1) ? Y.u : Y.z, Y.t, T.begin, T.end, pf);
        return 0.0;
    }
    if (c.mode == MODE_INIT) slot1<D, W, PF>(Y, c, T);
    return 0.0;
}

// Dispatch on the lattice dimension (fixed when FD != 0) and the group width.
template <int SLOT, int FD>
__device__ double run_slot(const EngSystem &Y, const TileCtl &c, const EngTile &T)
{
#ifdef HH_BOUNDS_CHECK
    {
        // A tile outside its system is recorded and skipped.
        int b = T.begin, e = T.end;
        HH_CHECK(b, 0, Y.g.N + 1, BC_TILE);
        HH_CHECK(e, b, Y.g.N + 1, BC_TILE);
        if (b != T.begin || e != T.end) return 0.0;
    }
#endif
    if (FD == 4) {
        // Exact-block form: scalar loops, three-slot form (ENGINE_EXBLOCK).
        if (SLOT == 1) {
            slot1<1, 1>(Y, c, T);
            return 0.0;
        }
        if (SLOT == 2) return slot2_ex(Y, c, T);
        if (SLOT == 3) return slot3_ex(Y, c, T);
        return 0.0;
    }
    // The generic kernel (FD = 0) carries both dimensions' loops, with the L2
    // prefetch in the d = 3 ones only (the d = 1 systems run without it in
    // every kernel); measured on the 64-chain d = 3 batch forced onto this
    // kernel, the prefetch takes it from 29.0 to 32.9 mixed solves/s (the
    // d = 3 kernel: 34.8).  FD = 5 and 7 are the d = 1 and d = 3 kernels
    // whose FP32 steps read 16-bit links.
    constexpr bool L16 = FD == 5 || FD == 7;
#define HH_SLOT_CALL(D, W)                                   \
    if (SLOT == 1) {                                         \
        slot1<D, W, FD != 0 || D == 3>(Y, c, T);             \
        return 0.0;                                          \
    } else if (SLOT == 2) {                                  \
        return slot2<D, W, FD != 0 || D == 3, L16>(Y, c, T); \
    } else if (SLOT == 4) {                                  \
        return slotA<D, W, FD != 0 || D == 3, L16>(Y, c, T); \
    } else {                                                 \
        return slot3<D, W, FD != 0 || D == 3, L16>(Y, c, T); \
    }
    const int w = Y.w;
    if (FD == 3 || FD == 7 || (FD == 0 && Y.g.d == 3)) {
        if (w == 4) { HH_SLOT_CALL(3, 4) }
        if (w == 2) { HH_SLOT_CALL(3, 2) }
        HH_SLOT_CALL(3, 1)
    } else {
        if (w == 4) { HH_SLOT_CALL(1, 4) }
        if (w == 2) { HH_SLOT_CALL(1, 2) }
        HH_SLOT_CALL(1, 1)
    }
#undef HH_SLOT_CALL
}

// Per-block cache of the systems a block touches.  Every block that owns a
// tile of a system computes that system's state with the same pure decide(),
// so after the first iteration of a launch the block keeps the states in
// shared memory and reads only the per-tile partial sums from global memory;
// the owner block still writes each state to global memory for the host and
// for the next launch.  A block touching more systems or tiles than the cache
// holds falls back to reading the states from global memory.
constexpr int kCacheSys = 32;
constexpr int kCacheTiles = 128;

// A task the control warp posts to the compute warps: one slot of one tile.
struct TaskMsg {
    TileCtl c;
    int sl;             // slot kind: 1, 2, 3, or 4 (two-slot first slot)
    int j;              // index of the tile in this block's list
    int slot;           // cache index of its system
    int tile;           // index of the tile in the launch's tile list
    int exit;           // 1: no more tasks
    int pad;
};

// Where the publishing control warp stores a task's partial.
struct PubMsg {
    unsigned long long *now, *next;
    int part;
    int pad;
};

// Named barriers of the control / compute hand-off (0 is __syncthreads):
// kBarReady + b: a task is posted in s_task[b]; kBarDone + b: the compute
// warps have ended it and written their partials to s_part[b].
constexpr int kBarReady = 1;
constexpr int kBarDone = 3;

__device__ __forceinline__ void named_sync(int id, unsigned n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ void named_arrive(int id, unsigned n)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// The engine kernel.  One block per SM owns fixed tiles; every engine
// iteration runs the slots of each of its tiles' systems, each slot of a system
// starting once every tile of that system has published the previous one
// (signal slots, see EngCtl).  Two forms:
//  * flat (L.ctl_warp = 0): all 16 warps compute; the block waits, decides and
//    publishes between tiles;
//  * control warp (L.ctl_warp = 1; 2: warp 0 prepares and posts, warp 1 ends
//    tasks and publishes): warp 0 waits, decides, sums and publishes
//    while warps 1-15 run the tasks it posts (one slot of one tile), so that a
//    task's waits and the previous task's publication overlap the compute of
//    the current one.  A publication is held back past the next task's
//    preparation only when that cannot close a cycle of waits: the next task
//    is of another system at the same phase (level), or the launch is
//    homogeneous (every block holds one tile of each system, in the same
//    order), where a preparation needs only publications of tasks two or more
//    places back.  A block leaves once all its systems are done.
template <int FD, int MINB>
__global__ void __launch_bounds__(ENGINE_BLOCK, MINB) engine_kernel(EngLaunch L)
{
    __shared__ TaskMsg s_task[2];
    __shared__ double s_part[2][ENGINE_BLOCK / 32];
    // Two control warps: the preparing warp posts tasks (s_posted counts them,
    // s_pub says where each publishes); the publishing warp ends them
    // (s_published counts them).
    __shared__ PubMsg s_pub[2];
    __shared__ int s_posted, s_published, s_end, s_failed;
    __shared__ double s_red[ENGINE_BLOCK / 32];
    __shared__ int s_flag;
    __shared__ EngState s_cache[kCacheSys];
    __shared__ TileCtl s_tctl[kCacheSys];
    __shared__ int s_sys[kCacheSys];
    __shared__ unsigned char s_slot[kCacheTiles];
    __shared__ int s_ok;
    // Uncached blocks: the mode each system was given by this block's own
    // slot-1 decision of the current iteration (its full state is read back
    // from global memory only after the next wait, once the owner block's copy
    // is certainly written).
    __shared__ unsigned char s_umode[ENGINE_MAX_SYSTEMS];
    // Read-only descriptors of this block's tiles and systems, copied once:
    // re-reading them from global memory after each wait would cost two
    // dependent L2 round trips per slot.
    __shared__ EngTile s_tiles[kCacheTiles];
    __shared__ EngSystem s_sysd[kCacheSys];

    EngCtl *ctl = L.ctl;
    const unsigned G = gridDim.x;
    long long k = *(volatile long long *)&ctl->k;
    const int drop = *(volatile int *)&ctl->drop_sig;   // tile partial (+ 1) never published: tests only

    if (threadIdx.x == 0) {
        int n = 0, ok = 1, j = 0;
        for (int tile = blockIdx.x; tile < L.ntiles; tile += G, ++j) {
            if (j >= kCacheTiles) {
                ok = 0;
                break;
            }
            const int sys = L.tiles[tile].sys;
            int slot = -1;
            for (int q = 0; q < n; ++q)
                if (s_sys[q] == sys) slot = q;
            if (slot < 0) {
                if (n == kCacheSys) {
                    ok = 0;
                    break;
                }
                slot = n;
                s_sys[n++] = sys;
            }
            s_slot[j] = (unsigned char)slot;
        }
        s_ok = ok;
    }
    __syncthreads();
    const bool cached = s_ok != 0;
    if (cached) {
        int j = 0;
        for (int tile = blockIdx.x; tile < L.ntiles; tile += G, ++j)
            if ((int)threadIdx.x == (j % (int)blockDim.x)) s_tiles[j] = L.tiles[tile];
        __syncthreads();
        j = 0;
        for (int tile = blockIdx.x; tile < L.ntiles; tile += G, ++j) {
            const int slot = s_slot[j];
            if (threadIdx.x == 0 && s_sys[slot] == s_tiles[j].sys) s_sysd[slot] = L.sys[s_tiles[j].sys];
        }
        __syncthreads();
    }

    if (!L.ctl_warp) {
        // ---- flat form: every warp computes; the block waits and decides
        //      together ----
        if (threadIdx.x == 0) s_ctl_threads = 0;
        __syncthreads();
        const int two = L.two_slot;
        const int nph = two ? 2 : 3;
        const size_t stride = (size_t)L.sig_stride;
        for (long long it = 0; it < L.max_iters; ++it, ++k) {
            EngState *cur = (k & 1) ? L.state[1] : L.state[0];
            EngState *nxt = (k & 1) ? L.state[0] : L.state[1];
            const int q = (int)(k & 1);
            int live = 0;   // thread 0: a system of this block still runs after this iteration's decisions
            for (int ph = 0; ph < nph; ++ph) {
                // Slot of this phase: 1 (decide + direction), 2 (t = M p), 3 (update);
                // two-slot form: 4 (decide + direction fused with t = M p), 3.
                const int sl = ph == 0 ? (two ? 4 : 1) : (two ? 3 : ph + 1);
                // Signal index of this phase and of the one it waits for.
                const int id = ph == 0 ? 0 : (ph == nph - 1 ? 2 : 1);
                const int id_prev = ph == 0 ? 2 : (ph == 1 ? 0 : 1);
                unsigned long long *sig_now = L.sig + (size_t)(2 * id + q) * stride;
                unsigned long long *sig_next = L.sig + (size_t)(2 * id + (q ^ 1)) * stride;
                const unsigned long long *sig_wait = L.sig + (size_t)(2 * id_prev + (ph == 0 ? (q ^ 1) : q)) * stride;
                int last = -1, j = 0;
                for (int tile = blockIdx.x; tile < L.ntiles; tile += G, ++j) {
                    const int slot = cached ? s_slot[j] : 0;
                    const EngTile T = cached ? s_tiles[j] : L.tiles[tile];
                    const EngSystem &Y = cached ? s_sysd[slot] : L.sys[T.sys];
                    if (T.sys != last) {
                        __syncthreads();
                        if (sl == 1 || sl == 4) {
                            if (!cached || it == 0) {
                                if (threadIdx.x == 0) s_cache[slot] = cur[T.sys];
                                __syncthreads();
                            }
                            if (threadIdx.x < 32) {
                                // Wait for the previous iteration's slot 3 of this system
                                // (nothing to wait for at its first iteration or when done).
                                const EngState &P = s_cache[slot];
                                double rr = 0.0;
                                bool ok = true;
                                if (P.mode != MODE_NEW && P.mode != MODE_DONE)
                                    ok = poll_sum(sig_wait + Y.part0, Y.ntiles, ctl, rr);
                                if (threadIdx.x == 0) {
                                    s_flag = ok ? 1 : 0;
                                    if (ok) {
                                        EngState S = decide(Y, P, rr);
                                        if (two && S.mode == MODE_CG) S.pbuf = P.pbuf ^ 1;
                                        if ((int)blockIdx.x == Y.owner) {
                                            nxt[T.sys] = S;
                                            // A finished system's blocks leave at different
                                            // iterations: keep its final state in both buffers.
                                            if (S.mode == MODE_DONE && P.mode != MODE_DONE) cur[T.sys] = S;
                                        }
                                        if (S.mode != MODE_DONE) live = 1;
                                        s_cache[slot] = S;
                                        s_tctl[slot] = make_ctl(S, two, Y.x0_given);
                                        if (!cached) s_umode[T.sys] = (unsigned char)S.mode;
                                    }
                                }
                            }
                        } else {
                            // An uncached block re-reads the system's state from the
                            // owner block's copy, after the wait that orders it.
                            if (threadIdx.x < 32) {
                                bool ok = true;
                                double tt = 0.0;
                                const int m = cached ? s_tctl[slot].mode : (int)s_umode[T.sys];
                                if (m != MODE_DONE) ok = poll_sum(sig_wait + Y.part0, Y.ntiles, ctl, tt);
                                if (threadIdx.x == 0) {
                                    s_flag = ok ? 1 : 0;
                                    if (ok && !cached) {
                                        const EngState S = nxt[T.sys];
                                        s_cache[0] = S;
                                        s_tctl[0] = make_ctl(S, two, Y.x0_given);
                                    }
                                    if (ok && sl == 3 && s_tctl[slot].mode == MODE_CG)
                                        s_tctl[slot].alpha = s_cache[slot].rr_alpha / tt;
                                }
                            }
                        }
                        __syncthreads();
                        if (!s_flag) return;
                        last = T.sys;
                    }
                    const TileCtl c = s_tctl[slot];
                    if (c.mode == MODE_DONE) continue;
                    double v;
                    if (sl == 1) {
                        run_slot<1, FD>(Y, c, T);
                        v = 0.0;
                    } else if (sl == 2) {
                        v = run_slot<2, FD>(Y, c, T);
                    } else if (sl == 4) {
                        v = run_slot<4, FD>(Y, c, T);
                    } else {
                        v = run_slot<3, FD>(Y, c, T);
                    }
                    // |t|^2 (CG, slot 2 or 4), |r|^2 (CG, RU, INIT, slot 3), <r, z>
                    // after the last preconditioner sub-step, else 0; the block sum
                    // ends with a __syncthreads() after all of the tile's writes.
                    const double tot = block_sum(v, s_red);
                    if (threadIdx.x == 0 && T.part + 1 != drop) sig_publish(sig_now + T.part, sig_next + T.part, tot);
                }
                if (ph == 0) {
                    // Leave once every system of this block is done: no other block
                    // waits for its tiles any more.
                    __syncthreads();
                    if (threadIdx.x == 0) s_flag = live;
                    __syncthreads();
                    if (!s_flag) {
                        if (threadIdx.x == 0) atomicMax((long long *)&ctl->k_end, k + 1);
                        return;
                    }
                }
            }
        }
        if (threadIdx.x == 0) atomicMax((long long *)&ctl->k_end, k);
        return;
    }

    // Control warps: 1, or 2 (warp 0 prepares and posts, warp 1 publishes).
    const int nctl = L.ctl_warp >= 2 ? 2 : 1;
    // Threads of each hand-off barrier: the compute warps and one control warp.
    const unsigned nbar = blockDim.x - 32u * (unsigned)(nctl - 1);
    if (threadIdx.x == 0) {
        s_ctl_threads = kCtlThreads * nctl;
        s_posted = s_published = s_end = s_failed = 0;
    }
    __syncthreads();
    if (threadIdx.x >= kCtlThreads * nctl) {
        // ---- compute warps: run the tasks the control warp posts ----
        const int warp = ((int)threadIdx.x >> 5) - nctl;
        for (int buf = 0;; buf ^= 1) {
            named_sync(kBarReady + buf, nbar);
            const TaskMsg m = s_task[buf];
            if (m.exit) return;
            const EngTile T = cached ? s_tiles[m.j] : L.tiles[m.tile];
            const EngSystem &Y = cached ? s_sysd[m.slot] : L.sys[T.sys];
            double v = 0.0;
            if (m.sl == 1)
                run_slot<1, FD>(Y, m.c, T);
            else if (m.sl == 2)
                v = run_slot<2, FD>(Y, m.c, T);
            else if (m.sl == 4)
                v = run_slot<4, FD>(Y, m.c, T);
            else
                v = run_slot<3, FD>(Y, m.c, T);
            // |t|^2 (CG, slot 2 or 4), |r|^2 (CG, RU, INIT, slot 3), <r, z>
            // after the last preconditioner sub-step, else 0.
            v = warp_sum(v);
            if ((threadIdx.x & 31u) == 0) s_part[buf][warp] = v;
            named_arrive(kBarDone + buf, nbar);
        }
    }

    const int ncw = (int)(blockDim.x >> 5) - nctl;   // compute warps
    // Bounded spin on a shared counter written by the other control warp.
    auto wait_count = [&](volatile int *cnt, int target) -> bool {
        uint64_t t0 = 0;
        unsigned spins = 0;
        while (*cnt < target) {
            if ((++spins & 255u) == 0) {
                if (t0 == 0) t0 = global_ns();
                if ((long long)(global_ns() - t0) > 3 * ctl->timeout_ns) {
                    atomicCAS(&ctl->error, 0, -6);
                    return false;
                }
            }
        }
        return true;
    };
    if (nctl == 2 && threadIdx.x >= kCtlThreads) {
        // ---- publishing warp: ends posted tasks in order, publishes their
        //      partials (sum of the per-warp partials in warp order) ----
        const int lane = (int)threadIdx.x & 31;
        for (int t = 0;; ++t) {
            // the next posted task, or the end
            uint64_t t0 = 0;
            unsigned spins = 0;
            bool ok = true;
            while (*(volatile int *)&s_posted <= t && !*(volatile int *)&s_end) {
                if ((++spins & 255u) == 0) {
                    if (t0 == 0) t0 = global_ns();
                    if ((long long)(global_ns() - t0) > 3 * ctl->timeout_ns) {
                        ok = false;
                        break;
                    }
                }
            }
            if (!ok || *(volatile int *)&s_posted <= t) break;
            __threadfence_block();
            const int b = t & 1;
            named_sync(kBarDone + b, nbar);
            if (lane == 0) {
                double tot = 0.0;
                for (int w = 0; w < ncw; ++w) tot += s_part[b][w];
                const PubMsg pm = s_pub[b];
                if (!*(volatile int *)&s_failed && pm.part + 1 != drop)
                    sig_publish(pm.now + pm.part, pm.next + pm.part, tot);
                __threadfence_block();
                *(volatile int *)&s_published = t + 1;
            }
            __syncwarp();
        }
        return;
    }

    // ---- control warp (with two: the preparing warp): waits, decisions,
    //      partial sums and signals ----
    const int lane = (int)threadIdx.x;
    const int two = L.two_slot;
    const int nph = two ? 2 : 3;
    const size_t stride = (size_t)L.sig_stride;
    int buf = 0;
    // The posted task whose end has not been published yet.
    bool pend = false, failed = false, stop = false;
    int pend_buf = 0, pend_part = 0, pend_sys = -1;
    long long pend_level = 0;
    unsigned long long *pend_now = nullptr, *pend_next = nullptr;
    int posted = 0;
    // Waits for the compute warps to end the pending task, then publishes its
    // partial (the sum of the per-warp partials in warp order); with two
    // control warps, waits until the publishing warp has done so.
    auto finish = [&]() {
        if (nctl == 1) {
            named_sync(kBarDone + pend_buf, nbar);
            if (lane == 0) {
                double tot = 0.0;
                for (int w = 0; w < ncw; ++w) tot += s_part[pend_buf][w];
                if (!failed && pend_part + 1 != drop) sig_publish(pend_now + pend_part, pend_next + pend_part, tot);
            }
            __syncwarp();
        } else if (!wait_count(&s_published, posted)) {
            failed = true;
        }
        __syncwarp();
        pend = false;
    };
    for (long long it = 0; it < L.max_iters && !failed && !stop; ++it, ++k) {
        EngState *cur = (k & 1) ? L.state[1] : L.state[0];
        EngState *nxt = (k & 1) ? L.state[0] : L.state[1];
        const int q = (int)(k & 1);
        int live = 0;   // lane 0: a system of this block still runs after this iteration's decisions
        for (int ph = 0; ph < nph && !failed && !stop; ++ph) {
            // Slot of this phase: 1 (decide + direction), 2 (t = M p), 3 (update);
            // two-slot form: 4 (decide + direction fused with t = M p), 3.
            const int sl = ph == 0 ? (two ? 4 : 1) : (two ? 3 : ph + 1);
            // Signal index of this phase and of the one it waits for.
            const int id = ph == 0 ? 0 : (ph == nph - 1 ? 2 : 1);
            const int id_prev = ph == 0 ? 2 : (ph == 1 ? 0 : 1);
            unsigned long long *sig_now = L.sig + (size_t)(2 * id + q) * stride;
            unsigned long long *sig_next = L.sig + (size_t)(2 * id + (q ^ 1)) * stride;
            const unsigned long long *sig_wait = L.sig + (size_t)(2 * id_prev + (ph == 0 ? (q ^ 1) : q)) * stride;
            const long long level = it * nph + ph;
            int last = -1, j = 0;
            for (int tile = blockIdx.x; tile < L.ntiles; tile += G, ++j) {
                const int slot = cached ? s_slot[j] : 0;
                const EngTile T = cached ? s_tiles[j] : L.tiles[tile];
                const EngSystem &Y = cached ? s_sysd[slot] : L.sys[T.sys];
                if (T.sys != last) {
                    // The wait below may need the pending task's signal: its own
                    // system's, or, through another block, any of an earlier
                    // phase.  Publish it first, unless it is of another system
                    // and the phase is the same or every block runs the same
                    // sequence of systems (then the wait needs signals of tasks
                    // two or more places back, all published).
                    if (pend && (pend_sys == T.sys || (!L.homogeneous && pend_level != level))) finish();
                    bool ok = true;
                    if (sl == 1 || sl == 4) {
                        if (!cached || it == 0) {
                            if (lane == 0) s_cache[slot] = cur[T.sys];
                            __syncwarp();
                        }
                        const int pm = s_cache[slot].mode;
                        double rr = 0.0;
                        // Nothing to wait for at a system's first iteration or once done.
                        if (pm != MODE_NEW && pm != MODE_DONE) ok = poll_sum(sig_wait + Y.part0, Y.ntiles, ctl, rr);
                        if (ok && lane == 0) {
                            const EngState P = s_cache[slot];
                            EngState S = decide(Y, P, rr);
                            if (two && S.mode == MODE_CG) S.pbuf = P.pbuf ^ 1;
                            if ((int)blockIdx.x == Y.owner) {
                                nxt[T.sys] = S;
                                // A finished system's blocks leave at different
                                // iterations: keep its final state in both buffers.
                                if (S.mode == MODE_DONE && P.mode != MODE_DONE) cur[T.sys] = S;
                            }
                            if (S.mode != MODE_DONE) live = 1;
                            s_cache[slot] = S;
                            s_tctl[slot] = make_ctl(S, two, Y.x0_given);
                            if (!cached) s_umode[T.sys] = (unsigned char)S.mode;
                        }
                    } else {
                        // An uncached block re-reads the system's state from the
                        // owner block's copy, after the wait that orders it.
                        __syncwarp();
                        const int m = cached ? s_tctl[slot].mode : (int)s_umode[T.sys];
                        double tt = 0.0;
                        if (m != MODE_DONE) ok = poll_sum(sig_wait + Y.part0, Y.ntiles, ctl, tt);
                        if (ok && !cached) {
                            if (lane == 0) {
                                const EngState S = nxt[T.sys];
                                s_cache[0] = S;
                                s_tctl[0] = make_ctl(S, two, Y.x0_given);
                            }
                            __syncwarp();
                        }
                        if (ok && lane == 0 && sl == 3 && m == MODE_CG)
                            s_tctl[slot].alpha = s_cache[slot].rr_alpha / tt;
                    }
                    __syncwarp();
                    if (!ok) {
                        failed = true;
                        break;
                    }
                    last = T.sys;
                }
                const TileCtl c = s_tctl[slot];
                if (c.mode == MODE_DONE) continue;
                // The compute warps have read this buffer's previous task (two
                // back) once it is published.
                if (nctl == 2 && !wait_count(&s_published, posted - 1)) {
                    failed = true;
                    break;
                }
                if (lane == 0) {
                    TaskMsg &m = s_task[buf];
                    m.c = c;
                    m.sl = sl;
                    m.j = j;
                    m.slot = slot;
                    m.tile = tile;
                    m.exit = 0;
                    if (nctl == 2) {
                        PubMsg &pm = s_pub[buf];
                        pm.now = sig_now;
                        pm.next = sig_next;
                        pm.part = T.part;
                    }
                }
                __syncwarp();
                named_arrive(kBarReady + buf, nbar);
                ++posted;
                if (nctl == 2 && lane == 0) {
                    __threadfence_block();
                    *(volatile int *)&s_posted = posted;
                }
                if (nctl == 1 && pend) finish();
                pend = true;
                pend_buf = buf;
                pend_part = T.part;
                pend_level = level;
                pend_sys = T.sys;
                pend_now = sig_now;
                pend_next = sig_next;
                buf ^= 1;
            }
            if (ph == 0 && !failed) {
                // Leave once every system of this block is done: no other block
                // waits for its tiles any more.
                live = __shfl_sync(0xffffffffu, live, 0);
                if (!live) {
                    if (lane == 0) atomicMax((long long *)&ctl->k_end, k + 1);
                    stop = true;
                }
            }
        }
    }
    if (nctl == 2 && failed && lane == 0) *(volatile int *)&s_failed = 1;
    if (pend) finish();
    if (lane == 0) {
        s_task[buf].exit = 1;
        if (!stop && !failed) atomicMax((long long *)&ctl->k_end, k);
        if (nctl == 2) {
            __threadfence_block();
            *(volatile int *)&s_end = 1;
        }
    }
    __syncwarp();
    named_arrive(kBarReady + buf, nbar);
}

}  // namespace

// The kernels: generic (any mix of dimensions), the dimension-specialised
// ones and the exact-block one, each launched with one 512-thread block per SM
// (measured on GB300: two blocks per SM, at 64 registers, was slower than one
// block with fewer arrivals per synchronisation).
const void *kernel_of(int kind)
{
    switch (kind) {
    case ENGINE_D1: return (const void *)engine_kernel<1, 1>;
    case ENGINE_D3: return (const void *)engine_kernel<3, 1>;
    case ENGINE_EXBLOCK: return (const void *)engine_kernel<4, 1>;
    case ENGINE_D1_L16: return (const void *)engine_kernel<5, 1>;
    case ENGINE_D3_L16: return (const void *)engine_kernel<7, 1>;
    default: return (const void *)engine_kernel<0, 1>;
    }
}

cudaError_t engine_launch(const EngLaunch &L, int grid, int block, cudaStream_t stream, int kind)
{
    if (L.nsys > ENGINE_MAX_SYSTEMS) return cudaErrorInvalidValue;
    EngLaunch arg = L;
    void *args[] = {(void *)&arg};
    return cudaLaunchCooperativeKernel(kernel_of(kind), dim3(grid), dim3(block), args, 0, stream);
}

const void *engine_kernel_fn(int kind)
{
    return kernel_of(kind);
}

int engine_max_grid(int block, int kind)
{
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel_of(kind), block, 0) != cudaSuccess)
        return 0;
    return per * nsm;
}

int engine_default_grid(int kind)
{
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    int mx = engine_max_grid(ENGINE_BLOCK, kind);
    const char *env = getenv("HH_ENGINE_BLOCKS_PER_SM");
    int per = env ? atoi(env) : 1;
    if (per < 1) per = 1;
    int g = per * nsm;
    return g < mx ? g : mx;
}

}  // namespace hh
