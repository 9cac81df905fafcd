// C ABI of the library: contexts, applies, solves, observables and the HMC
// trajectory driver.  Every step of the path runs in the kernels of
// hh_kernels.cu, hh_apply.cu and hh_engine.cu; this file only allocates,
// validates, plans and enqueues.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/hubhmc.h"
#include "hh_apply.cuh"
#include "hh_engine.cuh"
#include "hh_kernels.cuh"
#include "hh_trace.cuh"

using namespace hh;

namespace {

struct EngStats {
    long long cg_iters;     // summed CG steps
    int max_iters;          // largest CG steps of one system
    int n_solves;
    int n_ru;
    int worst_status;       // most severe status among systems
    int error;              // device-side wait / launch error
    int pad;
    double max_relres;
};

// New solves: states MODE_NEW, empty signal slots for 'parts' tile partials,
// iteration counter 0.
__global__ void k_engine_reset(EngState *s0, EngState *s1, int nsys, unsigned long long *sig, int parts,
                               EngCtl *ctl, long long timeout_ns, int drop_sig)
{
    for (int s = threadIdx.x; s < nsys; s += blockDim.x) {
        EngState z;
        memset(&z, 0, sizeof(z));
        z.mode = MODE_NEW;
        s0[s] = z;
        s1[s] = z;
    }
    const int n = (int)engine_sig_count(parts);
    for (int i = threadIdx.x; i < n; i += blockDim.x) sig[i] = kSigEmpty;
    if (threadIdx.x == 0) {
        ctl->error = 0;
        ctl->k = 0;
        ctl->k_end = 0;
        ctl->timeout_ns = timeout_ns;
        ctl->drop_sig = drop_sig;
    }
}

// Fault injection for the failure-detection tests: HH_ENGINE_DROP_SIGNAL=j + 1
// makes the next engine launches never publish tile partial j (a signal that
// nothing sets), so their waits run out after the wait budget.  Read at every
// launch; unset or 0: none.
int engine_drop_signal()
{
    const char *e = getenv("HH_ENGINE_DROP_SIGNAL");
    return e ? atoi(e) : 0;
}

__device__ int severity(int st)
{
    // ETIMEOUT and ENUMERIC outrank ENOCONV.
    if (st == HH_ETIMEOUT) return 3;
    if (st == HH_ENUMERIC) return 2;
    if (st == HH_ENOCONV) return 1;
    return 0;
}

// Running totals across solves (not cleared by k_zero_stats).
struct EngTotals {
    long long cg_steps, ru_steps, solves, fp64_steps;
};

__global__ void k_engine_fold(EngState *s0, EngState *s1, int nsys, const EngCtl *ctl,
                              EngStats *stats, EngTotals *tot)
{
    if (threadIdx.x != 0) return;
    const EngState *st = (ctl->k_end & 1) ? s1 : s0;
    if (ctl->error != 0 && severity(ctl->error) > severity(stats->worst_status))
        stats->worst_status = ctl->error;
    if (ctl->error != 0) stats->error = ctl->error;
    for (int s = 0; s < nsys; ++s) {
        EngState S = st[s];
        int status = S.status;
        if (S.mode != MODE_DONE && status == 0) status = HH_ETIMEOUT;
        stats->cg_iters += S.cg_steps;
        tot->cg_steps += S.cg_steps;
        tot->ru_steps += S.n_ru;
        tot->solves += 1;
        tot->fp64_steps += S.fp64_steps;
        if (S.cg_steps > stats->max_iters) stats->max_iters = S.cg_steps;
        stats->n_solves += 1;
        stats->n_ru += S.n_ru;
        if (S.true_relres > stats->max_relres || S.true_relres != S.true_relres)
            stats->max_relres = S.true_relres;
        if (severity(status) > severity(stats->worst_status)) stats->worst_status = status;
    }
}

__global__ void k_zero_stats(EngStats *stats)
{
    if (threadIdx.x == 0) memset(stats, 0, sizeof(EngStats));
}

// Plan of one engine launch: the system table and tiles in device memory.
struct Plan {
    int nsys = 0, ntiles = 0, grid = 0, homogeneous = 0;
    int precision = -1;
    int x0 = 0;                  // systems start from the x passed in
    const double *b = nullptr;
    double *x = nullptr;
    EngSystem sys[64];           // host copy of the device system table (n_pf <= 64)
};

}  // namespace

struct hh_ctx {
    hh_lattice lat;
    hh_params prm;
    cudaStream_t stream;
    Geo geo;
    int N;
    int cap_rhs;
    int max_grid;
    int kind;               // engine kernel for this lattice's dimension
    long long timeout_ns;
    // fields
    double *sigma, *sigma0, *L64, *pi, *chi, *xsol, *tmp, *F;
    float *L32, *tmp32a, *tmp32b;
    // CG workspace (cap_rhs vectors each)
    double *r, *p, *t, *p2;
    double *xprev;          // chronological guesses by extrapolation (chrono 2)
    float *r32, *p32, *t32, *x32, *p32b;
    int two_slot;           // engine launches run the two-slot form
    // engine
    EngSystem *d_sys;
    EngState *d_state[2];
    EngTile *d_tiles;
    unsigned long long *d_sig;      // engine signal slots, engine_sig_count(max_tiles)
    EngCtl *d_ctl;
    EngStats *d_stats;
    int max_tiles;
    Plan plan;
    EngTotals *d_totals;
    // counters and optional CUDA-event profile of the engine launches
    long long n_launch, n_engine;
    int profile;
    int ev_cap, ev_used;
    cudaEvent_t *ev;
    // HMC scalars
    HmcScalars *d_sc;
    double *d_energy_part;
    double *d_energy_out;   // [0] S or H scratch
    void *h_pinned;         // host readback buffer
    int *d_apply_err;       // set by a fused apply whose bounded wait ran out
    int nsm;
    int mtm_path;           // Q apply path (HH_APPLY_MTM): 0 by size (see hh_apply), 1 two
                            // sweeps, 2 two sweeps with programmatic dependent launch, 3 the
                            // fused FP32 d = 3 kernel where it applies, 4 the multi-vector
                            // FP32 d = 3 kernel (also for one vector); hh_apply_multi uses
                            // the multi-vector kernel for two or more vectors unless 1-3
    double *z, *u;          // Chebyshev preconditioner vectors (cap_rhs each), or null
    double *d_cheb;         // its coefficient table
    // Observables: noise, M^T noise and solutions (obs_cap vectors each), the
    // reduction partials and the five results.
    double *obs_eta, *obs_rhs, *obs_y, *obs_part, *obs_out;
    int obs_cap;
    // 16-bit links of the FP32 steps (HH_MIXED_BF16LINK / HH_MIXED_FIX16LINK).
    unsigned short *L16;
    int l16_mode;           // 0 none, 1 bfloat16, 2 fixed point
    double l16_scale;       // fixed point: L = code * l16_scale
};

namespace {

#define HH_TRY(expr)                      \
    do {                                  \
        cudaError_t e__ = (expr);         \
        if (e__ != cudaSuccess) return HH_ECUDA; \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t n)
{
    *p = nullptr;
    if (n == 0) n = 1;
    return cudaMalloc((void **)p, n * sizeof(T));
}

void free_ctx(hh_ctx *c)
{
    void *ptrs[] = {c->sigma, c->sigma0, c->L64, c->pi, c->chi, c->xsol, c->tmp, c->F, c->L32,
                    c->tmp32a, c->tmp32b, c->r, c->p, c->p2, c->xprev, c->t, c->r32, c->p32, c->p32b, c->t32, c->x32,
                    c->d_sys, c->d_state[0], c->d_state[1], c->d_tiles, c->d_sig, c->d_ctl, c->d_stats, c->d_sc, c->d_energy_part,
                    c->d_energy_out};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    if (c->d_totals) cudaFree(c->d_totals);
    if (c->d_apply_err) cudaFree(c->d_apply_err);
    if (c->z) cudaFree(c->z);
    if (c->u) cudaFree(c->u);
    if (c->d_cheb) cudaFree(c->d_cheb);
    for (double *p : {c->obs_eta, c->obs_rhs, c->obs_y, c->obs_part, c->obs_out})
        if (p) cudaFree(p);
    if (c->L16) cudaFree(c->L16);
    if (c->ev) {
        for (int i = 0; i < c->ev_cap; ++i)
            if (c->ev[i]) cudaEventDestroy(c->ev[i]);
        free(c->ev);
    }
}

// Build (or reuse) the engine plan for n_rhs systems b_a -> x_a.
int make_plan(hh_ctx *c, const double *b, double *x, int n_rhs)
{
    Plan &P = c->plan;
    if (P.nsys == n_rhs && P.b == b && P.x == x && P.precision == c->prm.precision) return HH_OK;
    // Overlapped layout: every system is tiled over the whole grid, so each
    // block holds one tile of each system, in system order, and the engine's
    // control warp prepares and publishes one system's slots while the compute
    // warps run another's (EngLaunch::homogeneous).  It pays when a tile's slot
    // takes longer than the control warp's wait, decision and publication
    // (about 3.5 us on GB300): FP64 systems from 2^18 sites, mixed ones from
    // 2^21.  Otherwise the systems share the grid, one tile per block.
    const bool mixed = c->prm.precision != HH_FP64;
    const bool overlap = engine_overlap(n_rhs, c->N, mixed);
    Tiling tl = engine_tiling(c->N, overlap ? 1 : n_rhs, c->max_grid);
    int ntiles = tl.tiles * n_rhs;
    if (ntiles > c->max_tiles) return HH_EINVAL;
    const int grid = overlap ? tl.tiles : (ntiles < c->max_grid ? ntiles : c->max_grid);
    // Bytes the CG iteration streams per site: x, r, p, t, b, the links and
    // the second p buffer in FP64 (and z, u with the preconditioner); r, p,
    // t, x, links, p' in FP32 (mixed).
    const long long site_bytes = mixed ? 24 : (c->prm.cheb_degree > 0 ? 72 : 56);
    const int pf = engine_prefetch(site_bytes * (long long)c->N * n_rhs, c->lat.d);
    std::vector<EngSystem> sys(n_rhs);
    std::vector<EngTile> tiles;
    tiles.reserve(ntiles);
    const int chunk = tl.chunk;
    for (int a = 0; a < n_rhs; ++a) {
        EngSystem &Y = sys[a];
        memset(&Y, 0, sizeof(Y));
        Y.g = c->geo;
        Y.h = c->prm.t * c->prm.dtau;
        Y.L64 = c->L64;
        Y.L32 = c->L32;
        Y.b = b + (size_t)a * c->N;
        Y.x = x + (size_t)a * c->N;
        size_t off = (size_t)a * c->N;
        Y.r = c->r + off;
        Y.p = c->p + off;
        Y.p2 = c->p2 + off;
        Y.t = c->t + off;
        Y.r32 = c->r32 + off;
        Y.p32 = c->p32 + off;
        Y.p32b = c->p32b + off;
        Y.t32 = c->t32 + off;
        Y.x32 = c->x32 + off;
        Y.tile0 = (int)tiles.size();
        for (int s0 = 0; s0 < c->N; s0 += chunk) {
            EngTile T;
            T.sys = a;
            T.begin = s0;
            T.end = s0 + chunk < c->N ? s0 + chunk : c->N;
            T.part = (int)tiles.size();
            tiles.push_back(T);
        }
        Y.ntiles = (int)tiles.size() - Y.tile0;
        Y.part0 = Y.tile0;
        Y.owner = overlap ? a % grid : Y.tile0 % grid;
        Y.precision = mixed ? PREC_MIXED : PREC_FP64;
        Y.L16 = c->L16;
        Y.link16 = c->l16_mode;
        Y.l16_scale = (float)c->l16_scale;
        Y.tol2 = c->prm.cg_tol * c->prm.cg_tol;
        Y.delta2 = c->prm.reliable_delta * c->prm.reliable_delta;
        Y.maxit = c->prm.cg_maxit;
        Y.w = engine_group_width(c->lat.nx);
        Y.pf = pf;
        Y.stall_window = ENGINE_STALL_WINDOW;
        Y.cheb_n = c->prm.cheb_degree;
        Y.cheb = c->d_cheb;
        Y.link_order = c->prm.link_order;
        Y.z = c->z ? c->z + off : nullptr;
        Y.u = c->u ? c->u + off : nullptr;
    }
    ntiles = (int)tiles.size();
    // Pageable sources: the copies have consumed the host buffers on return.
    HH_TRY(cudaMemcpyAsync(c->d_sys, sys.data(), sizeof(EngSystem) * n_rhs, cudaMemcpyHostToDevice,
                           c->stream));
    for (int a = 0; a < n_rhs; ++a) P.sys[a] = sys[a];
    P.x0 = 0;
    HH_TRY(cudaMemcpyAsync(c->d_tiles, tiles.data(), sizeof(EngTile) * ntiles,
                           cudaMemcpyHostToDevice, c->stream));
    P.nsys = n_rhs;
    P.ntiles = ntiles;
    P.grid = grid;
    P.homogeneous = overlap ? 1 : 0;
    P.b = b;
    P.x = x;
    P.precision = c->prm.precision;
    return HH_OK;
}

// Whether the plan's systems start from the x passed in (an initial guess) or
// from x = 0; re-uploads the system table when that changes.
int set_guess(hh_ctx *c, int x0)
{
    Plan &P = c->plan;
    if (P.x0 == x0) return HH_OK;
    for (int a = 0; a < P.nsys; ++a) P.sys[a].x0_given = x0;
    // Pageable source: the copy has consumed it on return.
    HH_TRY(cudaMemcpyAsync(c->d_sys, P.sys, sizeof(EngSystem) * P.nsys, cudaMemcpyHostToDevice, c->stream));
    P.x0 = x0;
    return HH_OK;
}

// The force from the solutions in xsol (n_rhs right-hand sides): pi -= eps F
// (pi may be NULL) and F_out (may be NULL); returns the launches added.
int ctx_force(hh_ctx *c, int n_rhs, double *pi, double eps, double *F_out, int *launches)
{
    const double h = c->prm.t * c->prm.dtau, A = c->prm.A;
    if (c->prm.link_order == 0) {
        HH_TRY(launch_force(c->geo, h, A, c->sigma, c->L64, c->xsol, n_rhs, pi, eps, F_out, c->stream));
        *launches = 1;
    } else {
        HH_TRY(launch_force_ex(c->geo, h, A, c->prm.link_order, c->sigma, c->L64, c->xsol, n_rhs, c->tmp, c->F,
                               pi, eps, F_out, c->stream));
        *launches = 2 * n_rhs;
    }
    return HH_OK;
}

// Enqueue one complete solve of the current plan and fold its statistics.
int run_engine(hh_ctx *c)
{
    TraceRange tr("hh engine solve");
    const Plan &P = c->plan;
    k_engine_reset<<<1, 256, 0, c->stream>>>(c->d_state[0], c->d_state[1], P.nsys, c->d_sig,
                                             c->max_tiles, c->d_ctl, c->timeout_ns, engine_drop_signal());
    HH_TRY(cudaGetLastError());
    EngLaunch L;
    L.sys = c->d_sys;
    L.state[0] = c->d_state[0];
    L.state[1] = c->d_state[1];
    L.tiles = c->d_tiles;
    L.sig = c->d_sig;
    L.sig_stride = c->max_tiles;
    L.ctl_warp = engine_ctl_warps(P.homogeneous ? 1 : 0);
    L.ctl = c->d_ctl;
    L.nsys = P.nsys;
    L.ntiles = P.ntiles;
    // Each CG step is one engine iteration, each true-residual check one more,
    // and with the Chebyshev preconditioner each of them is followed by 2n
    // sub-steps; the cap is a safety bound well above maxit.
    L.max_iters = (2LL * c->prm.cheb_degree + 1) * (3LL * (long long)c->prm.cg_maxit + 64);
    L.two_slot = c->two_slot;
    L.homogeneous = P.homogeneous;
    bool rec = c->profile && c->ev_used + 2 <= c->ev_cap;
    if (rec) HH_TRY(cudaEventRecord(c->ev[c->ev_used], c->stream));
    HH_TRY(engine_launch(L, P.grid, ENGINE_BLOCK, c->stream, c->kind));
    if (rec) {
        HH_TRY(cudaEventRecord(c->ev[c->ev_used + 1], c->stream));
        c->ev_used += 2;
    }
    k_engine_fold<<<1, 32, 0, c->stream>>>(c->d_state[0], c->d_state[1], P.nsys, c->d_ctl,
                                           c->d_stats, c->d_totals);
    HH_TRY(cudaGetLastError());
    c->n_launch += 3;
    c->n_engine += 1;
    return HH_OK;
}

int read_stats(hh_ctx *c, EngStats *out)
{
    HH_TRY(cudaMemcpyAsync(c->h_pinned, c->d_stats, sizeof(EngStats), cudaMemcpyDeviceToHost,
                           c->stream));
    HH_TRY(cudaStreamSynchronize(c->stream));
    memcpy(out, c->h_pinned, sizeof(EngStats));
    return HH_OK;
}

int stats_status(const EngStats &s)
{
    if (s.error != 0) return s.error;
    return s.worst_status;
}

void fill_solve_info(const EngStats &s, hh_solve_info *info)
{
    if (!info) return;
    info->iterations = s.max_iters;
    info->reliable_updates = s.n_ru;
    info->true_relres = s.max_relres;
    info->converged = (s.worst_status == 0 && s.error == 0) ? 1 : 0;
}

int ensure_rhs(hh_ctx *c, int n_rhs)
{
    return n_rhs >= 1 && n_rhs <= c->cap_rhs ? HH_OK : HH_EINVAL;
}

// Vector arguments are read and written with 16-byte accesses.
bool aligned16(const void *p)
{
    return ((uintptr_t)p & 15u) == 0;
}

// After every change of the links: the 16-bit copy read by the FP32 steps.
cudaError_t links16_after(hh_ctx *c)
{
    if (!c->l16_mode) return cudaSuccess;
    return launch_links16(c->N, c->L64, c->L16, c->l16_mode, c->l16_scale, c->stream);
}

}  // namespace

extern "C" {

void hh_default_params(hh_params *p)
{
    if (!p) return;
    p->t = 1.0;
    p->dtau = 0.05;
    p->A = 0.5;
    p->precision = HH_FP64;
    p->cg_tol = 1e-10;
    p->cg_maxit = 1000000;
    p->reliable_delta = 0.1;
    p->seed = 0;
    p->n_pf = 2;
    p->chain_id = 0;
    p->cheb_degree = 0;
    p->cheb_eps = 1e-3;
    p->integrator = HH_LEAPFROG;
    p->chrono = 0;
    p->link_order = 0;
}

#ifdef HH_BOUNDS_CHECK
}  // extern "C"
namespace hh {
namespace bounds {
static std::vector<Reader> &readers()
{
    static std::vector<Reader> r;
    return r;
}
// Called by each translation unit's registrar while the library loads.
void register_reader(Reader r)
{
    readers().push_back(r);
}
}  // namespace bounds
}  // namespace hh
namespace {
__global__ void k_bounds_selftest(int n)
{
    int idx = n;   // one past [0, n): the check records it and substitutes 0
    HH_CHECK(idx, 0, n, hh::BC_SELFTEST);
}
}  // namespace
extern "C" {
#endif

int hh_bounds_check(int op, int *enabled, long long *record)
{
    if (op != HH_BOUNDS_READ && op != HH_BOUNDS_SELFTEST) return HH_EINVAL;
#ifdef HH_BOUNDS_CHECK
    if (enabled) *enabled = 1;
    if (op == HH_BOUNDS_SELFTEST) {
        k_bounds_selftest<<<1, 1>>>(1000);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return HH_ECUDA;
    } else if (cudaDeviceSynchronize() != cudaSuccess) {
        return HH_ECUDA;
    }
    unsigned long long first = 0;
    for (hh::bounds::Reader r : hh::bounds::readers()) {
        const unsigned long long v = r();
        if (v && !first) first = v;
    }
    if (record) *record = (long long)(first & ~(1ull << 63));
    return first ? HH_EBOUNDS : HH_OK;
#else
    if (enabled) *enabled = 0;
    if (record) *record = 0;
    return HH_OK;
#endif
}

const char *hh_strerror(int code)
{
    switch (code) {
    case HH_OK: return "ok";
    case HH_EINVAL: return "invalid argument";
    case HH_ENOMEM: return "out of memory";
    case HH_ECUDA: return "CUDA runtime error";
    case HH_ENOCONV: return "CG did not converge within cg_maxit";
    case HH_ENUMERIC: return "NaN or Inf in a reduction";
    case HH_ETIMEOUT: return "device-side wait timed out";
    case HH_EBUSY: return "no free slot or memory budget";
    case HH_ESIZE: return "problem larger than the static scratch";
    case HH_EBOUNDS: return "an index check of the debug build failed";
    default: return "unknown error";
    }
}

int hh_create(hh_ctx **out, const hh_lattice *lat, const hh_params *p, void *cuda_stream)
{
    if (!out || !lat || !p) return HH_EINVAL;
    *out = nullptr;
    if (lat->d != 1 && lat->d != 3) return HH_EINVAL;
    if (lat->nx < 2 || lat->ntau < 2) return HH_EINVAL;
    if (p->n_pf < 1 || p->n_pf > 64) return HH_EINVAL;
    if (p->precision < HH_FP64 || p->precision > HH_MIXED_FIX16LINK) return HH_EINVAL;
    // 16-bit links: the fixed-point scale needs (1 + |A|) < 2^15, and the
    // exact-block loops read FP32 links only.
    if (p->precision >= HH_MIXED_BF16LINK && (p->link_order != 0 || !(fabs(p->A) < 32766.0)))
        return HH_EINVAL;
    if (!(p->cg_tol > 0.0) || p->cg_maxit < 1) return HH_EINVAL;
    if (p->cheb_degree < 0 || p->cheb_degree > CHEB_MAX_DEGREE) return HH_EINVAL;
    if (p->cheb_degree > 0 && (p->precision != HH_FP64 || !(p->cheb_eps > 0.0 && p->cheb_eps < 1.0)))
        return HH_EINVAL;
    if (p->integrator != HH_LEAPFROG && p->integrator != HH_OMELYAN) return HH_EINVAL;
    if (p->chrono < 0 || p->chrono > 2) return HH_EINVAL;
    if (p->link_order < 0 || p->link_order > 2) return HH_EINVAL;
    // The Chebyshev normalisation bound is that of the R1 form.
    if (p->link_order != 0 && p->cheb_degree != 0) return HH_EINVAL;
    long long V = lat->d == 1 ? lat->nx : (long long)lat->nx * lat->nx * lat->nx;
    long long N = V * lat->ntau;
    if (N >= (1LL << 31) - 1024) return HH_EINVAL;

    hh_ctx *c = new (std::nothrow) hh_ctx;
    if (!c) return HH_ENOMEM;
    memset(c, 0, sizeof(*c));
    c->lat = *lat;
    c->prm = *p;
    c->stream = (cudaStream_t)cuda_stream;
    c->geo = make_geo(lat->d, lat->nx, lat->ntau);
    c->N = (int)N;
    c->cap_rhs = p->n_pf > 4 ? p->n_pf : 4;
    c->timeout_ns = 5LL * 1000 * 1000 * 1000;
    // The exact-block form of M runs in its own kernel.
    c->kind = p->link_order != 0 ? ENGINE_EXBLOCK
              : p->precision >= HH_MIXED_BF16LINK ? (lat->d == 1 ? ENGINE_D1_L16 : ENGINE_D3_L16)
                                                  : (lat->d == 1 ? ENGINE_D1 : ENGINE_D3);
    c->two_slot = p->link_order == 0 ? engine_two_slot(c->kind) : 0;
    int max_grid = engine_default_grid(c->kind);
    if (max_grid <= 0) {
        delete c;
        return HH_ECUDA;
    }
    c->max_grid = max_grid;
    c->max_tiles = c->cap_rhs * (max_grid + 1) + 64;

    size_t n = (size_t)N, nr = (size_t)c->cap_rhs * n;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dalloc(&c->sigma, n);
    if (e == cudaSuccess) e = dalloc(&c->sigma0, n);
    if (e == cudaSuccess) e = dalloc(&c->L64, n);
    if (e == cudaSuccess) e = dalloc(&c->pi, n);
    if (e == cudaSuccess) e = dalloc(&c->tmp, n);
    if (e == cudaSuccess) e = dalloc(&c->F, n);
    if (e == cudaSuccess) e = dalloc(&c->L32, n);
    if (e == cudaSuccess) e = dalloc(&c->tmp32a, n);
    if (e == cudaSuccess) e = dalloc(&c->tmp32b, n);
    if (e == cudaSuccess) e = dalloc(&c->chi, nr);
    if (e == cudaSuccess) e = dalloc(&c->xsol, nr);
    if (e == cudaSuccess) e = dalloc(&c->r, nr);
    if (e == cudaSuccess) e = dalloc(&c->p, nr);
    if (e == cudaSuccess) e = dalloc(&c->p2, nr);
    if (e == cudaSuccess && p->chrono == 2) e = dalloc(&c->xprev, nr);
    if (e == cudaSuccess) e = dalloc(&c->p32b, nr);
    if (e == cudaSuccess) e = dalloc(&c->t, nr);
    if (e == cudaSuccess) e = dalloc(&c->r32, nr);
    if (e == cudaSuccess) e = dalloc(&c->p32, nr);
    if (e == cudaSuccess) e = dalloc(&c->t32, nr);
    if (e == cudaSuccess) e = dalloc(&c->x32, nr);
    if (e == cudaSuccess) e = dalloc(&c->d_sys, (size_t)c->cap_rhs);
    if (e == cudaSuccess) e = dalloc(&c->d_state[0], (size_t)c->cap_rhs);
    if (e == cudaSuccess) e = dalloc(&c->d_state[1], (size_t)c->cap_rhs);
    if (e == cudaSuccess) e = dalloc(&c->d_tiles, (size_t)c->max_tiles);
    if (e == cudaSuccess) e = dalloc(&c->d_sig, engine_sig_count(c->max_tiles));
    if (e == cudaSuccess) e = dalloc(&c->d_ctl, 1);
    if (e == cudaSuccess) e = dalloc(&c->d_stats, 1);
    if (e == cudaSuccess) e = dalloc(&c->d_sc, 1);
    if (e == cudaSuccess) e = dalloc(&c->d_totals, 1);
    if (e == cudaSuccess) e = dalloc(&c->d_apply_err, 1);
    if (e == cudaSuccess) e = dalloc(&c->d_energy_part, (size_t)energy_blocks(c->N));
    if (e == cudaSuccess) e = dalloc(&c->d_energy_out, 4);
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_pinned, 4096);
    if (e == cudaSuccess && p->cheb_degree > 0) {
        e = dalloc(&c->z, nr);
        if (e == cudaSuccess) e = dalloc(&c->u, nr);
        if (e == cudaSuccess) e = dalloc(&c->d_cheb, (size_t)(2 + 3 * CHEB_MAX_DEGREE));
        if (e == cudaSuccess) {
            std::vector<double> tab(2 + 3 * CHEB_MAX_DEGREE);
            engine_cheb_table(lat->d, p->t * p->dtau, p->A, p->cheb_degree, p->cheb_eps, tab.data());
            e = cudaMemcpy(c->d_cheb, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice);
        }
    }
    if (e != cudaSuccess) {
        free_ctx(c);
        delete c;
        return e == cudaErrorMemoryAllocation ? HH_ENOMEM : HH_ECUDA;
    }
    e = cudaMemsetAsync(c->sigma, 0, n * sizeof(double), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_ctl, 0, sizeof(EngCtl), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_sc, 0, sizeof(HmcScalars), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_totals, 0, sizeof(EngTotals), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_apply_err, 0, sizeof(int), c->stream);
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev);
        if (const char *env = getenv("HH_APPLY_MTM")) c->mtm_path = atoi(env);
    }
    if (e == cudaSuccess && p->precision >= HH_MIXED_BF16LINK) {
        c->l16_mode = p->precision == HH_MIXED_BF16LINK ? 1 : 2;
        int ex = 14;
        while (ex > 0 && (1.0 + fabs(p->A)) * ldexp(1.0, ex) > 32767.0) --ex;
        c->l16_scale = ldexp(1.0, -ex);
        e = dalloc(&c->L16, n);
    }
    if (e == cudaSuccess) e = launch_links(c->geo, p->A, c->sigma, c->L64, c->L32, c->stream);
    if (e == cudaSuccess) e = links16_after(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        free_ctx(c);
        delete c;
        return HH_ECUDA;
    }
    *out = c;
    return HH_OK;
}

int hh_destroy(hh_ctx *c)
{
    if (!c) return HH_OK;
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
    delete c;
    return HH_OK;
}

long long hh_nsites(const hh_ctx *c)
{
    return c ? (long long)c->N : 0;
}

int hh_set_field(hh_ctx *c, const double *sigma, int on_device)
{
    if (!c || !sigma) return HH_EINVAL;
    size_t bytes = (size_t)c->N * sizeof(double);
    if (on_device) {
        HH_TRY(cudaMemcpyAsync(c->sigma, sigma, bytes, cudaMemcpyDeviceToDevice, c->stream));
    } else {
        HH_TRY(cudaMemcpyAsync(c->sigma, sigma, bytes, cudaMemcpyHostToDevice, c->stream));
    }
    HH_TRY(launch_links(c->geo, c->prm.A, c->sigma, c->L64, c->L32, c->stream));
    HH_TRY(links16_after(c));
    c->n_launch += c->l16_mode ? 2 : 1;
    if (!on_device) HH_TRY(cudaStreamSynchronize(c->stream));
    return HH_OK;
}

int hh_get_field(hh_ctx *c, double *sigma, int on_device)
{
    if (!c || !sigma) return HH_EINVAL;
    size_t bytes = (size_t)c->N * sizeof(double);
    if (on_device) {
        HH_TRY(cudaMemcpyAsync(sigma, c->sigma, bytes, cudaMemcpyDeviceToDevice, c->stream));
    } else {
        HH_TRY(cudaMemcpyAsync(sigma, c->sigma, bytes, cudaMemcpyDeviceToHost, c->stream));
        HH_TRY(cudaStreamSynchronize(c->stream));
    }
    return HH_OK;
}

int hh_init_field_random(hh_ctx *c, uint64_t seed)
{
    if (!c) return HH_EINVAL;
    HH_TRY(launch_init_field(c->sigma, c->N, seed, c->prm.chain_id, c->stream));
    HH_TRY(launch_links(c->geo, c->prm.A, c->sigma, c->L64, c->L32, c->stream));
    HH_TRY(links16_after(c));
    c->n_launch += c->l16_mode ? 3 : 2;
    return HH_OK;
}

int hh_apply(hh_ctx *c, int op, const void *x, void *y, int dtype)
{
    TraceRange tr("hh_apply");
    if (!c || !x || !y || x == y) return HH_EINVAL;
    if (op != HH_OP_M && op != HH_OP_MT && op != HH_OP_MTM) return HH_EINVAL;
    const double h = c->prm.t * c->prm.dtau;
    const int order = c->prm.link_order;
    int launches = 0;
    if (order != 0) {
        // Exact-block form: the scalar kernels.
        if (dtype == HH_DTYPE_F64) {
            const double *xd = (const double *)x;
            double *yd = (double *)y;
            if (op == HH_OP_MTM) {
                HH_TRY(launch_apply_f64(c->geo, 0, h, c->L64, xd, c->tmp, c->stream, order));
                HH_TRY(launch_apply_f64(c->geo, 1, h, c->L64, c->tmp, yd, c->stream, order));
            } else {
                HH_TRY(launch_apply_f64(c->geo, op, h, c->L64, xd, yd, c->stream, order));
            }
        } else if (dtype == HH_DTYPE_F32) {
            const float *xf = (const float *)x;
            float *yf = (float *)y;
            if (op == HH_OP_MTM) {
                HH_TRY(launch_apply_f32(c->geo, 0, (float)h, c->L32, xf, c->tmp32a, c->stream, order));
                HH_TRY(launch_apply_f32(c->geo, 1, (float)h, c->L32, c->tmp32a, yf, c->stream, order));
            } else {
                HH_TRY(launch_apply_f32(c->geo, op, (float)h, c->L32, xf, yf, c->stream, order));
            }
        } else {
            return HH_EINVAL;
        }
        c->n_launch += op == HH_OP_MTM ? 2 : 1;
        return HH_OK;
    }
    // Vector sweeps need 16-byte aligned x and y; the scalar kernels take any.
    const bool vec = aligned16(x) && aligned16(y);
    if (dtype == HH_DTYPE_F64) {
        const double *xd = (const double *)x;
        double *yd = (double *)y;
        if (op == HH_OP_MTM) {
            if (vec) {
                HH_TRY(launch_sweep_f64(c->geo, false, h, c->L64, xd, c->tmp, c->stream));
                HH_TRY(launch_sweep_f64(c->geo, true, h, c->L64, c->tmp, yd, c->stream, c->mtm_path != 1));
            } else {
                HH_TRY(launch_apply_f64(c->geo, 0, h, c->L64, xd, c->tmp, c->stream));
                HH_TRY(launch_apply_f64(c->geo, 1, h, c->L64, c->tmp, yd, c->stream));
            }
            launches = 2;
        } else {
            if (vec)
                HH_TRY(launch_sweep_f64(c->geo, op == HH_OP_MT, h, c->L64, xd, yd, c->stream));
            else
                HH_TRY(launch_apply_f64(c->geo, op, h, c->L64, xd, yd, c->stream));
            launches = 1;
        }
    } else if (dtype == HH_DTYPE_F32) {
        const float *xf = (const float *)x;
        float *yf = (float *)y;
        if (op == HH_OP_MTM) {
            // Two sweeps with t = M x kept in L2 while x, t, y and the links fit
            // in it (measured on GB300 at 4.2M sites: 26 us cold against 31 us
            // for the fused kernel); the fused kernel, which keeps t in shared
            // memory, beyond that.
            const bool big = (long long)c->N * 16 > (96LL << 20);
            const bool fused = c->mtm_path == 3 || (c->mtm_path == 0 && big);
            if (vec && c->mtm_path == 4 && multi_mtm_ok(c->geo, c->L32, xf, yf)) {
                // the multi-vector kernel with one vector (HH_APPLY_MTM=4)
                HH_TRY(launch_mtm_multi_f32(c->geo, (float)h, c->L32, xf, yf, 1, c->d_apply_err, c->nsm,
                                            c->timeout_ns, c->stream));
                launches = 1;
            } else if (vec && fused && fused_mtm_ok(c->geo, c->L32, xf, yf)) {
                HH_TRY(launch_mtm_fused_f32(c->geo, (float)h, c->L32, xf, yf, c->d_apply_err, c->nsm, c->stream));
                launches = 1;
            } else if (vec) {
                HH_TRY(launch_sweep_f32(c->geo, false, (float)h, c->L32, xf, c->tmp32a, c->stream));
                HH_TRY(launch_sweep_f32(c->geo, true, (float)h, c->L32, c->tmp32a, yf, c->stream,
                                        c->mtm_path != 1));
                launches = 2;
            } else {
                HH_TRY(launch_apply_f32(c->geo, 0, (float)h, c->L32, xf, c->tmp32a, c->stream));
                HH_TRY(launch_apply_f32(c->geo, 1, (float)h, c->L32, c->tmp32a, yf, c->stream));
                launches = 2;
            }
        } else {
            if (vec)
                HH_TRY(launch_sweep_f32(c->geo, op == HH_OP_MT, (float)h, c->L32, xf, yf, c->stream));
            else
                HH_TRY(launch_apply_f32(c->geo, op, (float)h, c->L32, xf, yf, c->stream));
            launches = 1;
        }
    } else {
        return HH_EINVAL;
    }
    c->n_launch += launches;
    return HH_OK;
}

int hh_set_timeout(hh_ctx *c, double seconds)
{
    if (!c || !(seconds >= 0.0) || seconds > 3600.0) return HH_EINVAL;
    c->timeout_ns = (long long)(seconds * 1e9);
    return HH_OK;
}

int hh_apply_multi(hh_ctx *c, int op, const void *x, void *y, int n_vec, int dtype)
{
    TraceRange tr("hh_apply_multi");
    if (!c || !x || !y || n_vec < 1) return HH_EINVAL;
    if (op != HH_OP_M && op != HH_OP_MT && op != HH_OP_MTM) return HH_EINVAL;
    if (dtype != HH_DTYPE_F64 && dtype != HH_DTYPE_F32) return HH_EINVAL;
    const size_t esz = dtype == HH_DTYPE_F64 ? sizeof(double) : sizeof(float);
    const size_t span = (size_t)n_vec * (size_t)c->N * esz;
    const uintptr_t xa = (uintptr_t)x, ya = (uintptr_t)y;
    if (xa < ya + span && ya < xa + span) return HH_EINVAL;   // x and y overlap
    if (op == HH_OP_MTM && dtype == HH_DTYPE_F32 && c->prm.link_order == 0 && n_vec >= 2 &&
        (c->mtm_path == 0 || c->mtm_path == 4) && multi_mtm_ok(c->geo, c->L32, x, y)) {
        HH_TRY(launch_mtm_multi_f32(c->geo, (float)(c->prm.t * c->prm.dtau), c->L32, (const float *)x,
                                    (float *)y, n_vec, c->d_apply_err, c->nsm, c->timeout_ns, c->stream));
        c->n_launch += 1;
        return HH_OK;
    }
    for (int v = 0; v < n_vec; ++v) {
        const size_t off = (size_t)v * (size_t)c->N * esz;
        const int rc = hh_apply(c, op, (const char *)x + off, (char *)y + off, dtype);
        if (rc) return rc;
    }
    return HH_OK;
}

// One solve of the current plan from x = 0 (x0 = 0) or from the x passed in.
static int solve_from(hh_ctx *c, const double *b, double *x, int n_rhs, int x0, hh_solve_info *info)
{
    TraceRange tr("hh_solve");
    if (!c || !b || !x || !aligned16(b) || !aligned16(x)) return HH_EINVAL;
    int rc = ensure_rhs(c, n_rhs);
    if (rc) return rc;
    rc = make_plan(c, b, x, n_rhs);
    if (rc) return rc;
    rc = set_guess(c, x0);
    if (rc) return rc;
    k_zero_stats<<<1, 32, 0, c->stream>>>(c->d_stats);
    HH_TRY(cudaGetLastError());
    c->n_launch += 1;
    rc = run_engine(c);
    if (rc) return rc;
    if (!info) return HH_OK;
    EngStats s;
    rc = read_stats(c, &s);
    if (rc) return rc;
    fill_solve_info(s, info);
    return stats_status(s);
}

int hh_solve(hh_ctx *c, const double *b, double *x, int n_rhs, hh_solve_info *info)
{
    return solve_from(c, b, x, n_rhs, 0, info);
}

int hh_solve_guess(hh_ctx *c, const double *b, double *x, int n_rhs, hh_solve_info *info)
{
    return solve_from(c, b, x, n_rhs, 1, info);
}

int hh_force(hh_ctx *c, const double *chi, int n_rhs, double *F, hh_solve_info *info)
{
    if (!c || !chi || !F || !aligned16(chi)) return HH_EINVAL;
    int rc = ensure_rhs(c, n_rhs);
    if (rc) return rc;
    rc = make_plan(c, chi, c->xsol, n_rhs);
    if (rc) return rc;
    rc = set_guess(c, 0);
    if (rc) return rc;
    k_zero_stats<<<1, 32, 0, c->stream>>>(c->d_stats);
    HH_TRY(cudaGetLastError());
    c->n_launch += 1;
    rc = run_engine(c);
    if (rc) return rc;
    int nl = 0;
    rc = ctx_force(c, n_rhs, nullptr, 0.0, F, &nl);
    if (rc) return rc;
    c->n_launch += nl;
    if (!info) return HH_OK;
    EngStats s;
    rc = read_stats(c, &s);
    if (rc) return rc;
    fill_solve_info(s, info);
    return stats_status(s);
}

int hh_action(hh_ctx *c, const double *chi, int n_rhs, double *S, hh_solve_info *info)
{
    if (!c || !chi || !S || !aligned16(chi)) return HH_EINVAL;
    int rc = ensure_rhs(c, n_rhs);
    if (rc) return rc;
    rc = make_plan(c, chi, c->xsol, n_rhs);
    if (rc) return rc;
    rc = set_guess(c, 0);
    if (rc) return rc;
    k_zero_stats<<<1, 32, 0, c->stream>>>(c->d_stats);
    HH_TRY(cudaGetLastError());
    c->n_launch += 1;
    rc = run_engine(c);
    if (rc) return rc;
    HH_TRY(launch_energy(c->N, nullptr, chi, c->xsol, n_rhs, c->d_energy_part, c->d_energy_out,
                         c->stream));
    c->n_launch += 2;
    EngStats s;
    rc = read_stats(c, &s);
    if (rc) return rc;
    HH_TRY(cudaMemcpy(S, c->d_energy_out, sizeof(double), cudaMemcpyDeviceToHost));
    fill_solve_info(s, info);
    return stats_status(s);
}

int hh_observables(hh_ctx *c, int n_noise, uint64_t traj, hh_obs_info *out)
{
    if (!c || !out || n_noise < 2 || n_noise > kObsMaxNoise || (n_noise & 1)) return HH_EINVAL;
    const size_t N = (size_t)c->N;
    if (c->obs_cap < n_noise) {
        for (double **p : {&c->obs_eta, &c->obs_rhs, &c->obs_y, &c->obs_part, &c->obs_out}) {
            if (*p) cudaFree(*p);
            *p = nullptr;
        }
        c->obs_cap = 0;
        cudaError_t e = dalloc(&c->obs_eta, N * n_noise);
        if (e == cudaSuccess) e = dalloc(&c->obs_rhs, N * n_noise);
        if (e == cudaSuccess) e = dalloc(&c->obs_y, N * n_noise);
        if (e == cudaSuccess) e = dalloc(&c->obs_part, (size_t)(n_noise + 3) * energy_blocks(c->N));
        if (e == cudaSuccess) e = dalloc(&c->obs_out, 8);
        if (e != cudaSuccess) return HH_ENOMEM;
        c->obs_cap = n_noise;
    }
    const double h = c->prm.t * c->prm.dtau;
    HH_TRY(launch_z2_noise(c->obs_eta, c->N, n_noise, c->prm.seed, traj, c->prm.chain_id, c->stream));
    for (int k = 0; k < n_noise; ++k)
        HH_TRY(launch_apply_f64(c->geo, 1, h, c->L64, c->obs_eta + k * N, c->obs_rhs + k * N, c->stream,
                                c->prm.link_order));
    c->n_launch += 1 + n_noise;
    // y_k = Q^{-1} M^T eta_k, in groups of at most cap_rhs right-hand sides.
    int iters = 0;
    double relres = 0.0;
    for (int k0 = 0; k0 < n_noise; k0 += c->cap_rhs) {
        const int m = n_noise - k0 < c->cap_rhs ? n_noise - k0 : c->cap_rhs;
        hh_solve_info si;
        int rc = solve_from(c, c->obs_rhs + k0 * N, c->obs_y + k0 * N, m, 0, &si);
        if (rc) return rc;
        if (si.iterations > iters) iters = si.iterations;
        if (si.true_relres > relres) relres = si.true_relres;
    }
    HH_TRY(launch_observables(c->N, n_noise, c->obs_eta, c->obs_y, c->sigma, c->obs_part, c->obs_out,
                              c->stream));
    c->n_launch += 2;
    double r[5];
    HH_TRY(cudaMemcpyAsync(c->h_pinned, c->obs_out, sizeof(r), cudaMemcpyDeviceToHost, c->stream));
    HH_TRY(cudaStreamSynchronize(c->stream));
    memcpy(r, c->h_pinned, sizeof(r));
    out->trace_Minv = r[0];
    out->trace_err = r[1];
    out->one_minus_g_sq = r[2];
    out->mean_sin = r[3];
    out->mean_sin2 = r[4];
    out->n_noise = n_noise;
    out->cg_iterations = iters;
    out->max_true_relres = relres;
    return HH_OK;
}

}  // extern "C"

namespace {

// Leapfrog on (ctx sigma, pi) at fixed chi (Sec. 4.1).  If h0/h1 are non-null
// the Hamiltonian before/after is written to those device doubles, reusing the
// first and last solves.  Enqueues only.
int leapfrog_enqueue(hh_ctx *c, double *pi, const double *chi, int n_rhs, int n_md, double dt,
                     double *h0, double *h1)
{
    const double h = c->prm.t * c->prm.dtau, A = c->prm.A;
    int rc = make_plan(c, chi, c->xsol, n_rhs);
    if (rc) return rc;
    double kick = 0.0, drift = 0.0;
    const int forces = md_schedule(c->prm.integrator, n_md, dt, 0, &kick, &drift);
    const int chrono = c->prm.chrono;
    const long long nx = (long long)n_rhs * c->N;
    for (int j = 0; j < forces; ++j) {
        TraceRange tr("hh md force");
        md_schedule(c->prm.integrator, n_md, dt, j, &kick, &drift);
        // Chronological initial guess (chrono 1: the previous force's
        // solution, already in xsol; 2: the linear extrapolation of the last
        // two); the trajectory's first solve starts from zero.
        if (chrono == 2 && j >= 2) {
            HH_TRY(launch_extrapolate(c->xsol, c->xprev, nx, c->stream));
            c->n_launch += 1;
        } else if (chrono == 2 && j == 1) {
            HH_TRY(cudaMemcpyAsync(c->xprev, c->xsol, sizeof(double) * (size_t)nx, cudaMemcpyDeviceToDevice,
                                   c->stream));
        }
        rc = set_guess(c, (chrono != 0 && j >= 1) ? 1 : 0);
        if (rc) return rc;
        rc = run_engine(c);
        if (rc) return rc;
        if (j == 0 && h0)
            HH_TRY(launch_energy(c->N, pi, chi, c->xsol, n_rhs, c->d_energy_part, h0, c->stream));
        int nl = 0;
        rc = ctx_force(c, n_rhs, pi, kick, nullptr, &nl);
        if (rc) return rc;
        c->n_launch += nl - 1;
        if (j + 1 < forces) {
            HH_TRY(launch_sigma_step(c->geo, A, drift, c->sigma, pi, c->L64, c->L32, c->stream));
            HH_TRY(links16_after(c));
        }
    }
    if (h1) HH_TRY(launch_energy(c->N, pi, chi, c->xsol, n_rhs, c->d_energy_part, h1, c->stream));
    c->n_launch += (h0 ? 2 : 0) + (h1 ? 2 : 0) + forces + (forces - 1) * (c->l16_mode ? 2 : 1);
    return HH_OK;
}

}  // namespace

extern "C" {

int hh_leapfrog(hh_ctx *c, double *pi, const double *chi, int n_rhs, int n_md, double dt,
                hh_solve_info *info)
{
    if (!c || !pi || !chi || n_md < 1 || !aligned16(chi)) return HH_EINVAL;
    int rc = ensure_rhs(c, n_rhs);
    if (rc) return rc;
    k_zero_stats<<<1, 32, 0, c->stream>>>(c->d_stats);
    HH_TRY(cudaGetLastError());
    c->n_launch += 1;
    rc = leapfrog_enqueue(c, pi, chi, n_rhs, n_md, dt, nullptr, nullptr);
    if (rc) return rc;
    if (!info) return HH_OK;
    EngStats s;
    rc = read_stats(c, &s);
    if (rc) return rc;
    fill_solve_info(s, info);
    return stats_status(s);
}

int hh_trajectory(hh_ctx *c, int n_md, double dt, uint64_t traj, hh_traj_info *info)
{
    if (!c || n_md < 1) return HH_EINVAL;
    const int npf = c->prm.n_pf;
    const double h = c->prm.t * c->prm.dtau;
    const uint64_t seed = c->prm.seed, chain = c->prm.chain_id;
    k_zero_stats<<<1, 32, 0, c->stream>>>(c->d_stats);
    HH_TRY(cudaGetLastError());
    c->n_launch += 1;
    TraceRange tr("hh_trajectory");
    // Momenta and pseudofermion heatbath chi_a = M^T xi_a (Eqs. (11)-(12)).
    {
        TraceRange th("hh heatbath");
        HH_TRY(launch_gaussian(c->pi, c->N, seed, 1, 0, traj, chain, c->stream));
        for (int a = 0; a < npf; ++a) {
            HH_TRY(launch_gaussian(c->tmp, c->N, seed, 2, a, traj, chain, c->stream));
            HH_TRY(launch_apply_f64(c->geo, 1, h, c->L64, c->tmp, c->chi + (size_t)a * c->N, c->stream,
                                    c->prm.link_order));
        }
    }
    HH_TRY(cudaMemcpyAsync(c->sigma0, c->sigma, (size_t)c->N * sizeof(double),
                           cudaMemcpyDeviceToDevice, c->stream));
    int rc = leapfrog_enqueue(c, c->pi, c->chi, npf, n_md, dt, &c->d_sc->H0, &c->d_sc->H1);
    if (rc) return rc;
    TraceRange tm("hh metropolis");
    HH_TRY(launch_metropolis(c->d_sc, seed, traj, chain, c->stream));
    HH_TRY(launch_restore(c->geo, c->prm.A, c->d_sc, c->sigma, c->sigma0, c->L64, c->L32, c->stream));
    HH_TRY(links16_after(c));
    c->n_launch += (1 + npf) + npf + 2 + (c->l16_mode ? 1 : 0);
    if (!info) return HH_OK;
    char *hp = (char *)c->h_pinned;
    HH_TRY(cudaMemcpyAsync(hp, c->d_stats, sizeof(EngStats), cudaMemcpyDeviceToHost, c->stream));
    HH_TRY(cudaMemcpyAsync(hp + 256, c->d_sc, sizeof(HmcScalars), cudaMemcpyDeviceToHost, c->stream));
    HH_TRY(cudaStreamSynchronize(c->stream));
    EngStats s;
    HmcScalars sc;
    memcpy(&s, hp, sizeof(s));
    memcpy(&sc, hp + 256, sizeof(sc));
    info->H0 = sc.H0;
    info->H1 = sc.H1;
    info->dH = sc.dH;
    info->u = sc.u;
    info->accepted = sc.accepted;
    info->cg_iterations = (int)s.cg_iters;
    info->n_solves = s.n_solves;
    info->max_true_relres = s.max_relres;
    return stats_status(s);
}

int hh_counters_reset(hh_ctx *c, int profile_engine)
{
    if (!c) return HH_EINVAL;
    HH_TRY(cudaStreamSynchronize(c->stream));
    c->n_launch = 0;
    c->n_engine = 0;
    c->ev_used = 0;
    c->profile = profile_engine ? 1 : 0;
    if (c->profile && !c->ev) {
        const int cap = 16384;
        c->ev = (cudaEvent_t *)calloc(cap, sizeof(cudaEvent_t));
        if (!c->ev) return HH_ENOMEM;
        c->ev_cap = cap;
        for (int i = 0; i < cap; ++i) HH_TRY(cudaEventCreate(&c->ev[i]));
    }
    HH_TRY(cudaMemsetAsync(c->d_totals, 0, sizeof(EngTotals), c->stream));
    HH_TRY(cudaMemsetAsync(c->d_apply_err, 0, sizeof(int), c->stream));
    HH_TRY(cudaStreamSynchronize(c->stream));
    return HH_OK;
}

int hh_counters_get(hh_ctx *c, hh_counters *out)
{
    if (!c || !out) return HH_EINVAL;
    EngTotals t;
    HH_TRY(cudaMemcpyAsync(c->h_pinned, c->d_totals, sizeof(EngTotals), cudaMemcpyDeviceToHost,
                           c->stream));
    HH_TRY(cudaStreamSynchronize(c->stream));
    memcpy(&t, c->h_pinned, sizeof(t));
    double ms = 0.0;
    for (int i = 0; i + 1 < c->ev_used; i += 2) {
        float m = 0.0f;
        HH_TRY(cudaEventElapsedTime(&m, c->ev[i], c->ev[i + 1]));
        ms += m;
    }
    int aerr = 0;
    HH_TRY(cudaMemcpy(&aerr, c->d_apply_err, sizeof(int), cudaMemcpyDeviceToHost));
    out->kernel_launches = c->n_launch;
    out->engine_launches = c->n_engine;
    out->engine_ms = ms;
    out->cg_steps = t.cg_steps;
    out->ru_steps = t.ru_steps;
    out->solves = t.solves;
    out->fp64_steps = t.fp64_steps;
    out->sites = c->N;
    return aerr ? aerr : HH_OK;
}

}  // extern "C"
