// Batched multi-chain engine and serving loop.
//
// Requests (CG solves and HMC trajectories of independent chains, any lattice)
// are admitted into slots carved from one device arena sized by the HBM budget.
// All active right-hand sides are systems of one persistent CG launch
// (hh_engine.cu), run for a chunk of iterations per launch; the launch is a
// CUDA-graph replay whose kernel node is updated when the membership changes.
// Between chunks the scheduling thread retires finished solves, advances each
// trajectory through the leapfrog of Sec. 4.1 (force and momentum update,
// sigma step, next solve, Metropolis) and admits queued requests.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/hubhmc.h"
#include "hh_engine.cuh"
#include "hh_kernels.cuh"
#include "hh_trace.cuh"

using namespace hh;

namespace {

constexpr int kMaxRhs = 4;
constexpr int kMaxSlots = 256;
constexpr int kMaxTiles = 1 << 16;
using Clock = std::chrono::steady_clock;

size_t align256(size_t v)
{
    return (v + 255) / 256 * 256;
}

// First-fit allocator over one device block, with coalescing of freed ranges.
struct Arena {
    char *base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> length

    cudaError_t init(size_t bytes)
    {
        size = align256(bytes);
        cudaError_t e = cudaMalloc((void **)&base, size);
        if (e == cudaSuccess) free_[0] = size;
        return e;
    }
    size_t alloc(size_t bytes)
    {
        bytes = align256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                size_t off = it->first, rem = it->second - bytes;
                free_.erase(it);
                if (rem) free_[off + bytes] = rem;
                return off;
            }
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = align256(bytes);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

// First-fit allocator of partial-sum index ranges (one range per slot, held
// for the slot's lifetime so that tile lists can be rebuilt freely).
struct IndexPool {
    std::map<int, int> free_;  // first -> count
    void init(int n)
    {
        free_.clear();
        free_[0] = n;
    }
    int alloc(int n)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= n) {
                int first = it->first, rem = it->second - n;
                free_.erase(it);
                if (rem) free_[first + n] = rem;
                return first;
            }
        return -1;
    }
    void release(int first, int n)
    {
        auto it = free_.emplace(first, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Pending {
    uint64_t ticket;
    hh_request req;
    std::vector<double> sigma, b;
    Clock::time_point t_submit;
};

// Device arrays of one slot, carved from the arena.
struct SlotMem {
    double *sigma, *sigma0, *L64, *pi, *tmp, *chi, *x, *r, *p, *p2, *t, *epart;
    float *L32, *r32, *p32, *p32b, *t32, *x32;
    double *z, *u, *cheb;   // Chebyshev preconditioner (requests with cheb_degree > 0)
    double *xprev;          // chronological guesses by extrapolation (chrono 2)
    HmcScalars *sc;
};

size_t slot_bytes(long long N, int nrhs, bool cheb, bool extrap, SlotMem *m, char *base)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return base ? base + o : nullptr;
    };
    size_t d = sizeof(double), f = sizeof(float);
    char *p;
    p = take(N * d); if (m) m->sigma = (double *)p;
    p = take(N * d); if (m) m->sigma0 = (double *)p;
    p = take(N * d); if (m) m->L64 = (double *)p;
    p = take(N * d); if (m) m->pi = (double *)p;
    p = take(N * d); if (m) m->tmp = (double *)p;
    p = take(nrhs * N * d); if (m) m->chi = (double *)p;
    p = take(nrhs * N * d); if (m) m->x = (double *)p;
    p = take(nrhs * N * d); if (m) m->r = (double *)p;
    p = take(nrhs * N * d); if (m) m->p = (double *)p;
    p = take(nrhs * N * d); if (m) m->p2 = (double *)p;
    p = take(nrhs * N * d); if (m) m->t = (double *)p;
    p = take(N * f); if (m) m->L32 = (float *)p;
    p = take(nrhs * N * f); if (m) m->r32 = (float *)p;
    p = take(nrhs * N * f); if (m) m->p32 = (float *)p;
    p = take(nrhs * N * f); if (m) m->p32b = (float *)p;
    p = take(nrhs * N * f); if (m) m->t32 = (float *)p;
    p = take(nrhs * N * f); if (m) m->x32 = (float *)p;
    p = take(sizeof(HmcScalars)); if (m) m->sc = (HmcScalars *)p;
    p = take(energy_blocks((int)N) * d); if (m) m->epart = (double *)p;
    if (m) m->z = m->u = m->cheb = m->xprev = nullptr;
    if (extrap) {
        p = take(nrhs * N * d); if (m) m->xprev = (double *)p;
    }
    if (cheb) {
        p = take(nrhs * N * d); if (m) m->z = (double *)p;
        p = take(nrhs * N * d); if (m) m->u = (double *)p;
        p = take((2 + 3 * CHEB_MAX_DEGREE) * d); if (m) m->cheb = (double *)p;
    }
    return off;
}

struct Slot {
    bool used = false;
    uint64_t ticket = 0;
    hh_request req;
    Geo geo;
    int N = 0, nrhs = 0;
    size_t off = 0, bytes = 0;
    SlotMem m;
    int md_step = 0;
    Clock::time_point t_submit, t_admit;
    long long cg_iters = 0;
    long long last_steps[kMaxRhs];
    bool rhs_done[kMaxRhs];
    int n_ru = 0, n_solves = 0, status = 0;
    double max_relres = 0.0;
    bool in_engine = false;
    int part_off = 0, tiles_per_rhs = 0;   // partial-sum range [part_off, + nrhs*tiles_per_rhs)
};

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct hh_batch {
    hh_batch_config cfg;
    cudaStream_t stream = nullptr;
    Arena arena;
    IndexPool parts;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Pending> queue;
    std::deque<hh_result> results;
    uint64_t next_ticket = 1;
    std::vector<Slot> slots;
    std::atomic<int> n_active{0};
    long long active_sites = 0;
    // engine
    EngSystem *d_sys = nullptr;
    EngState *d_state[2] = {nullptr, nullptr};
    EngTile *d_tiles = nullptr;
    unsigned long long *d_sig = nullptr;   // engine signal slots, engine_sig_count(kMaxTiles)
    EngCtl *d_ctl = nullptr;
    int max_sys = 0, ntiles = 0;
    int grid_of[4] = {0, 0, 0, 0};  // engine grid per kernel kind
    int kind = ENGINE_GENERIC;      // kernel of the current plan
    int two_slot_of[4] = {0, 0, 0, 0};  // engine form per kernel kind
    int ctl_warp = 1;               // engine launches use a control warp
    int graph_kind = -1;
    long long k = 0;
    bool plan_dirty = true;
    std::vector<EngSystem> h_sys;
    std::vector<EngTile> h_tiles;
    EngState *h_states = nullptr;   // pinned mirror of one state buffer
    EngCtl *h_ctl = nullptr;    // pinned
    // graph of one chunk launch
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraphNode_t gnode = nullptr;
    bool use_graph = true;
    EngLaunch launch_arg;   // kernel parameters of the current chunk
    // statistics
    double site_iters = 0.0;
    // worker
    std::thread worker;
    std::atomic<bool> running{false};
    bool failed = false;
    std::atomic<long long> timeout_ns{5LL * 1000 * 1000 * 1000};   // bound of every device-side wait
};

namespace {

#define HB_TRY(expr)                             \
    do {                                         \
        cudaError_t e__ = (expr);                \
        if (e__ != cudaSuccess) return HH_ECUDA; \
    } while (0)

long long lattice_sites(const hh_lattice &lat)
{
    long long V = lat.d == 1 ? lat.nx : (long long)lat.nx * lat.nx * lat.nx;
    return V * lat.ntau;
}

int validate(const hh_request &r)
{
    if (r.kind != HH_REQ_SOLVE && r.kind != HH_REQ_TRAJECTORY) return HH_EINVAL;
    if (r.lat.d != 1 && r.lat.d != 3) return HH_EINVAL;
    if (r.lat.nx < 2 || r.lat.ntau < 2) return HH_EINVAL;
    if (lattice_sites(r.lat) >= (1LL << 31) - 1024) return HH_EINVAL;
    if (r.prm.n_pf < 1 || r.prm.n_pf > kMaxRhs) return HH_EINVAL;
    if (r.prm.precision != HH_FP64 && r.prm.precision != HH_MIXED) return HH_EINVAL;
    if (!(r.prm.cg_tol > 0.0) || r.prm.cg_maxit < 1) return HH_EINVAL;
    if (r.kind == HH_REQ_TRAJECTORY && r.n_md < 1) return HH_EINVAL;
    if (r.prm.integrator != HH_LEAPFROG && r.prm.integrator != HH_OMELYAN) return HH_EINVAL;
    if (r.prm.chrono < 0 || r.prm.chrono > 2) return HH_EINVAL;
    if (r.prm.link_order != 0) return HH_EINVAL;   // the exact-block form runs in contexts only
    // Chebyshev-preconditioned CG (Sec. 4.2) is FP64 only, as in the context solver.
    if (r.prm.cheb_degree < 0 || r.prm.cheb_degree > CHEB_MAX_DEGREE) return HH_EINVAL;
    if (r.prm.cheb_degree > 0 && (r.prm.precision != HH_FP64 || !(r.prm.cheb_eps > 0.0 && r.prm.cheb_eps < 1.0)))
        return HH_EINVAL;
    return HH_OK;
}

void push_result(hh_batch *b, const hh_result &res)
{
    std::lock_guard<std::mutex> lk(b->mu);
    b->results.push_back(res);
}

// Put the systems of slot s into the engine as new solves (x0 = 0).
int start_solve(hh_batch *b, int s)
{
    Slot &S = b->slots[s];
    EngState z;
    memset(&z, 0, sizeof(z));
    z.mode = MODE_NEW;
    EngState *cur = b->d_state[b->k & 1];
    for (int a = 0; a < S.nrhs; ++a) {
        HB_TRY(cudaMemcpyAsync(cur + s * kMaxRhs + a, &z, sizeof(z), cudaMemcpyHostToDevice, b->stream));
        S.last_steps[a] = 0;
        S.rhs_done[a] = false;
    }
    // Empty signal slots for the slot's tile partials (all 2 x 3 phases).
    for (int ph = 0; ph < 6; ++ph)
        HB_TRY(cudaMemsetAsync(b->d_sig + (size_t)ph * kMaxTiles + S.part_off, 0xFF,
                               sizeof(unsigned long long) * (size_t)S.nrhs * S.tiles_per_rhs, b->stream));
    S.in_engine = true;
    b->plan_dirty = true;
    return HH_OK;
}

void release_slot(hh_batch *b, int s)
{
    Slot &S = b->slots[s];
    b->arena.release(S.off, S.bytes);
    b->parts.release(S.part_off, S.nrhs * S.tiles_per_rhs);
    b->active_sites -= S.N;
    b->n_active -= 1;
    S.used = false;
    S.in_engine = false;
    b->plan_dirty = true;
}

int admit(hh_batch *b, Pending &P, int s)
{
    Slot &S = b->slots[s];
    const hh_request &r = P.req;
    S.used = true;
    S.ticket = P.ticket;
    S.req = r;
    S.geo = make_geo(r.lat.d, r.lat.nx, r.lat.ntau);
    S.N = S.geo.N;
    S.nrhs = r.prm.n_pf;
    S.md_step = 0;
    S.t_submit = P.t_submit;
    S.t_admit = Clock::now();
    S.cg_iters = 0;
    S.n_ru = S.n_solves = S.status = 0;
    S.max_relres = 0.0;
    slot_bytes(S.N, S.nrhs, r.prm.cheb_degree > 0, r.prm.chrono == 2, &S.m, b->arena.base + S.off);
    b->active_sites += S.N;
    b->n_active += 1;
    const uint64_t seed = r.prm.seed, chain = r.prm.chain_id;
    const double h = r.prm.t * r.prm.dtau;
    cudaStream_t st = b->stream;
    if (!P.sigma.empty())
        HB_TRY(cudaMemcpyAsync(S.m.sigma, P.sigma.data(), sizeof(double) * S.N, cudaMemcpyHostToDevice, st));
    else
        HB_TRY(launch_init_field(S.m.sigma, S.N, seed, chain, st));
    HB_TRY(launch_links(S.geo, r.prm.A, S.m.sigma, S.m.L64, S.m.L32, st));
    HB_TRY(cudaMemsetAsync(S.m.sc, 0, sizeof(HmcScalars), st));
    if (S.m.cheb) {
        // Pageable source: the copy has consumed the host table on return.
        std::vector<double> tab(2 + 3 * CHEB_MAX_DEGREE);
        engine_cheb_table(r.lat.d, h, r.prm.A, r.prm.cheb_degree, r.prm.cheb_eps, tab.data());
        HB_TRY(cudaMemcpyAsync(S.m.cheb, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, st));
    }
    if (r.kind == HH_REQ_SOLVE) {
        if (!P.b.empty()) {
            HB_TRY(cudaMemcpyAsync(S.m.chi, P.b.data(), sizeof(double) * S.N * S.nrhs,
                                   cudaMemcpyHostToDevice, st));
        } else {
            for (int a = 0; a < S.nrhs; ++a)
                HB_TRY(launch_gaussian(S.m.chi + (size_t)a * S.N, S.N, seed, 2, a, r.traj_index, chain, st));
        }
    } else {
        // Momenta and pseudofermion heatbath chi_a = M^T xi_a (Eqs. (11)-(12)).
        HB_TRY(launch_gaussian(S.m.pi, S.N, seed, 1, 0, r.traj_index, chain, st));
        for (int a = 0; a < S.nrhs; ++a) {
            HB_TRY(launch_gaussian(S.m.tmp, S.N, seed, 2, a, r.traj_index, chain, st));
            HB_TRY(launch_apply_f64(S.geo, 1, h, S.m.L64, S.m.tmp, S.m.chi + (size_t)a * S.N, st));
        }
        HB_TRY(cudaMemcpyAsync(S.m.sigma0, S.m.sigma, sizeof(double) * S.N, cudaMemcpyDeviceToDevice, st));
    }
    return start_solve(b, s);
}

// Admit queued requests while slots, budget and the active-site window allow.
int admit_queued(hh_batch *b)
{
    for (;;) {
        Pending P;
        int s = -1;
        {
            std::lock_guard<std::mutex> lk(b->mu);
            if (b->queue.empty()) return HH_OK;
            const Pending &front = b->queue.front();
            long long N = lattice_sites(front.req.lat);
            if (b->cfg.max_active_sites > 0 && b->n_active > 0 &&
                b->active_sites + N > b->cfg.max_active_sites)
                return HH_OK;
            for (int j = 0; j < (int)b->slots.size(); ++j)
                if (!b->slots[j].used) {
                    s = j;
                    break;
                }
            if (s < 0) return HH_OK;
            size_t bytes = slot_bytes(N, front.req.prm.n_pf, front.req.prm.cheb_degree > 0,
                                      front.req.prm.chrono == 2, nullptr, nullptr);
            int tpr = (int)((N + b->cfg.tile_sites - 1) / b->cfg.tile_sites);
            int part = b->parts.alloc(tpr * front.req.prm.n_pf);
            if (part < 0) return HH_OK;
            size_t off = b->arena.alloc(bytes);
            if (off == SIZE_MAX) {
                b->parts.release(part, tpr * front.req.prm.n_pf);
                return HH_OK;
            }
            b->slots[s].off = off;
            b->slots[s].bytes = bytes;
            b->slots[s].part_off = part;
            b->slots[s].tiles_per_rhs = tpr;
            P = std::move(b->queue.front());
            b->queue.pop_front();
        }
        int rc = admit(b, P, s);
        if (rc) return rc;
    }
}

// Rebuild the system table and the tiles of the active systems.
int build_plan(hh_batch *b)
{
    b->h_tiles.clear();
    const int tile = b->cfg.tile_sites;
    // Prefetch distance from the bytes the active systems' CG steps stream
    // per iteration (per site: 56 B FP64, 72 B with the preconditioner, 24 B
    // mixed).
    long long bytes = 0;
    for (const Slot &S : b->slots)
        if (S.used && S.in_engine)
            bytes += (long long)S.N * S.nrhs *
                     (S.req.prm.precision == HH_MIXED ? 24 : (S.req.prm.cheb_degree > 0 ? 72 : 56));
    for (int s = 0; s < (int)b->slots.size(); ++s) {
        Slot &S = b->slots[s];
        if (!S.used || !S.in_engine) continue;
        for (int a = 0; a < S.nrhs; ++a) {
            int sid = s * kMaxRhs + a;
            EngSystem &Y = b->h_sys[sid];
            memset(&Y, 0, sizeof(Y));
            Y.g = S.geo;
            Y.h = S.req.prm.t * S.req.prm.dtau;
            Y.L64 = S.m.L64;
            Y.L32 = S.m.L32;
            size_t o = (size_t)a * S.N;
            Y.b = S.m.chi + o;
            Y.x = S.m.x + o;
            Y.r = S.m.r + o;
            Y.p = S.m.p + o;
            Y.p2 = S.m.p2 + o;
            Y.t = S.m.t + o;
            Y.r32 = S.m.r32 + o;
            Y.p32 = S.m.p32 + o;
            Y.p32b = S.m.p32b + o;
            Y.t32 = S.m.t32 + o;
            Y.x32 = S.m.x32 + o;
            Y.precision = S.req.prm.precision == HH_MIXED ? PREC_MIXED : PREC_FP64;
            Y.tol2 = S.req.prm.cg_tol * S.req.prm.cg_tol;
            Y.delta2 = S.req.prm.reliable_delta * S.req.prm.reliable_delta;
            Y.maxit = S.req.prm.cg_maxit;
            Y.w = engine_group_width(S.geo.nx);
            Y.pf = engine_prefetch(bytes, S.geo.d);
            Y.stall_window = ENGINE_STALL_WINDOW;
            Y.cheb_n = S.req.prm.cheb_degree;
            // Chronological initial guess of a trajectory's later solves.
            Y.x0_given = (S.req.kind == HH_REQ_TRAJECTORY && S.req.prm.chrono != 0 && S.md_step >= 1) ? 1 : 0;
            Y.cheb = S.m.cheb;
            Y.z = S.m.z ? S.m.z + o : nullptr;
            Y.u = S.m.u ? S.m.u + o : nullptr;
            Y.tile0 = (int)b->h_tiles.size();
            Y.part0 = S.part_off + a * S.tiles_per_rhs;
            for (int s0 = 0, j = 0; s0 < S.N; s0 += tile, ++j) {
                EngTile T;
                T.sys = sid;
                T.begin = s0;
                T.end = s0 + tile < S.N ? s0 + tile : S.N;
                T.part = Y.part0 + j;
                b->h_tiles.push_back(T);
            }
            Y.ntiles = (int)b->h_tiles.size() - Y.tile0;
        }
    }
    b->ntiles = (int)b->h_tiles.size();
    if (b->ntiles > kMaxTiles) return HH_EINVAL;
    // One dimension in the whole plan: the specialised kernel.
    int dims = 0;
    for (int s = 0; s < (int)b->slots.size(); ++s)
        if (b->slots[s].used && b->slots[s].in_engine) dims |= (b->slots[s].geo.d == 1) ? 1 : 2;
    b->kind = dims == 1 ? ENGINE_D1 : dims == 2 ? ENGINE_D3 : ENGINE_GENERIC;
    const int kgrid = b->grid_of[b->kind];
    int grid = b->ntiles < kgrid ? b->ntiles : kgrid;
    for (int s = 0; s < (int)b->slots.size(); ++s) {
        Slot &S = b->slots[s];
        if (!S.used || !S.in_engine) continue;
        for (int a = 0; a < S.nrhs; ++a) {
            EngSystem &Y = b->h_sys[s * kMaxRhs + a];
            Y.owner = Y.tile0 % grid;
        }
    }
    HB_TRY(cudaMemcpyAsync(b->d_sys, b->h_sys.data(), sizeof(EngSystem) * b->max_sys,
                           cudaMemcpyHostToDevice, b->stream));
    if (b->ntiles)
        HB_TRY(cudaMemcpyAsync(b->d_tiles, b->h_tiles.data(), sizeof(EngTile) * b->ntiles,
                               cudaMemcpyHostToDevice, b->stream));
    b->plan_dirty = false;
    return HH_OK;
}

EngLaunch make_launch(hh_batch *b)
{
    EngLaunch L;
    L.sys = b->d_sys;
    L.state[0] = b->d_state[0];
    L.state[1] = b->d_state[1];
    L.tiles = b->d_tiles;
    L.sig = b->d_sig;
    L.sig_stride = kMaxTiles;
    L.ctl_warp = b->ctl_warp;
    L.ctl = b->d_ctl;
    L.nsys = b->max_sys;
    L.ntiles = b->ntiles;
    L.max_iters = b->cfg.chunk_iters;
    L.two_slot = b->two_slot_of[b->kind];
    L.homogeneous = 0;
    return L;
}

// One chunk: a cooperative launch, replayed from a CUDA graph whose kernel
// node is updated with the current plan (falls back to a direct launch).
int launch_chunk(hh_batch *b, int grid)
{
    EngLaunch &arg = b->launch_arg;  // copied at node update / launch
    arg = make_launch(b);
    if (b->use_graph) {
        void *args[] = {(void *)&arg};
        cudaKernelNodeParams kp;
        memset(&kp, 0, sizeof(kp));
        kp.func = (void *)engine_kernel_fn(b->kind);
        kp.gridDim = dim3(grid);
        kp.blockDim = dim3(ENGINE_BLOCK);
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        bool ok = true;
        if (b->gexec && b->graph_kind != b->kind) {
            cudaGraphExecDestroy(b->gexec);
            cudaGraphDestroy(b->graph);
            b->gexec = nullptr;
            b->graph = nullptr;
        }
        if (!b->gexec) {
            b->graph_kind = b->kind;
            ok = cudaGraphCreate(&b->graph, 0) == cudaSuccess &&
                 cudaGraphAddKernelNode(&b->gnode, b->graph, nullptr, 0, &kp) == cudaSuccess;
            if (ok) {
                cudaLaunchAttributeValue v;
                memset(&v, 0, sizeof(v));
                v.cooperative = 1;
                ok = cudaGraphKernelNodeSetAttribute(b->gnode, cudaLaunchAttributeCooperative, &v) ==
                     cudaSuccess;
            }
            if (ok) ok = cudaGraphInstantiate(&b->gexec, b->graph, 0) == cudaSuccess;
        } else {
            ok = cudaGraphExecKernelNodeSetParams(b->gexec, b->gnode, &kp) == cudaSuccess;
        }
        if (ok) ok = cudaGraphLaunch(b->gexec, b->stream) == cudaSuccess;
        if (ok) return HH_OK;
        cudaGetLastError();
        b->use_graph = false;
    }
    HB_TRY(engine_launch(arg, grid, ENGINE_BLOCK, b->stream, b->kind));
    return HH_OK;
}

void fill_common(const Slot &S, hh_result &res)
{
    res.ticket = S.ticket;
    res.kind = S.req.kind;
    res.status = S.status;
    res.cg_iterations = (int)S.cg_iters;
    res.reliable_updates = S.n_ru;
    res.n_solves = S.n_solves;
    res.max_true_relres = S.max_relres;
}

// A slot's solve finished: retire it or advance its trajectory.
int advance(hh_batch *b, int s)
{
    Slot &S = b->slots[s];
    const hh_request &r = S.req;
    cudaStream_t st = b->stream;
    S.in_engine = false;
    b->plan_dirty = true;
    if (r.kind == HH_REQ_SOLVE || S.status == HH_ETIMEOUT || S.status == HH_ENUMERIC) {
        hh_result res;
        memset(&res, 0, sizeof(res));
        if (r.kind == HH_REQ_SOLVE && r.out)
            HB_TRY(cudaMemcpyAsync(r.out, S.m.x, sizeof(double) * S.N * S.nrhs, cudaMemcpyDeviceToHost, st));
        HB_TRY(cudaStreamSynchronize(st));
        fill_common(S, res);
        res.latency_ms = ms_between(S.t_submit, Clock::now());
        res.queue_ms = ms_between(S.t_submit, S.t_admit);
        release_slot(b, s);
        push_result(b, res);
        return HH_OK;
    }
    // Trajectory: the molecular dynamics (leapfrog of Sec. 4.1 or Omelyan) around
    // force number md_step, computed from the solve just finished.
    const double h = r.prm.t * r.prm.dtau, A = r.prm.A, dt = r.dt;
    const int k = S.md_step;
    double kick = 0.0, drift = 0.0;
    const int forces = md_schedule(r.prm.integrator, r.n_md, dt, k, &kick, &drift);
    if (k == 0)
        HB_TRY(launch_energy(S.N, S.m.pi, S.m.chi, S.m.x, S.nrhs, S.m.epart, &S.m.sc->H0, st));
    HB_TRY(launch_force(S.geo, h, A, S.m.sigma, S.m.L64, S.m.x, S.nrhs, S.m.pi, kick, nullptr, st));
    if (k + 1 < forces) {
        HB_TRY(launch_sigma_step(S.geo, A, drift, S.m.sigma, S.m.pi, S.m.L64, S.m.L32, st));
        S.md_step = k + 1;
        if (r.prm.chrono == 2 && k + 1 >= 2)
            HB_TRY(launch_extrapolate(S.m.x, S.m.xprev, (long long)S.nrhs * S.N, st));
        else if (r.prm.chrono == 2)
            HB_TRY(cudaMemcpyAsync(S.m.xprev, S.m.x, sizeof(double) * (size_t)S.nrhs * S.N,
                                   cudaMemcpyDeviceToDevice, st));
        return start_solve(b, s);
    }
    HB_TRY(launch_energy(S.N, S.m.pi, S.m.chi, S.m.x, S.nrhs, S.m.epart, &S.m.sc->H1, st));
    HB_TRY(launch_metropolis(S.m.sc, r.prm.seed, r.traj_index, r.prm.chain_id, st));
    HB_TRY(launch_restore(S.geo, A, S.m.sc, S.m.sigma, S.m.sigma0, S.m.L64, S.m.L32, st));
    HmcScalars sc;
    HB_TRY(cudaMemcpyAsync(&sc, S.m.sc, sizeof(sc), cudaMemcpyDeviceToHost, st));
    if (r.out) HB_TRY(cudaMemcpyAsync(r.out, S.m.sigma, sizeof(double) * S.N, cudaMemcpyDeviceToHost, st));
    HB_TRY(cudaStreamSynchronize(st));
    hh_result res;
    memset(&res, 0, sizeof(res));
    fill_common(S, res);
    res.H0 = sc.H0;
    res.H1 = sc.H1;
    res.dH = sc.dH;
    res.u = sc.u;
    res.accepted = sc.accepted;
    res.latency_ms = ms_between(S.t_submit, Clock::now());
    res.queue_ms = ms_between(S.t_submit, S.t_admit);
    release_slot(b, s);
    push_result(b, res);
    return HH_OK;
}

int fail_all_active(hh_batch *b, int code)
{
    for (int s = 0; s < (int)b->slots.size(); ++s) {
        Slot &S = b->slots[s];
        if (!S.used) continue;
        S.status = code;
        hh_result res;
        memset(&res, 0, sizeof(res));
        fill_common(S, res);
        res.latency_ms = ms_between(S.t_submit, Clock::now());
        res.queue_ms = ms_between(S.t_submit, S.t_admit);
        release_slot(b, s);
        push_result(b, res);
    }
    return HH_OK;
}

int step(hh_batch *b)
{
    int rc = admit_queued(b);
    if (rc) return rc;
    int n_sys = 0;
    for (auto &S : b->slots)
        if (S.used && S.in_engine) n_sys += S.nrhs;
    if (n_sys == 0) return HH_OK;
    if (b->plan_dirty) {
        rc = build_plan(b);
        if (rc) return rc;
    }
    const int kgrid = b->grid_of[b->kind];
    int grid = b->ntiles < kgrid ? b->ntiles : kgrid;
    EngCtl c;
    memset(&c, 0, sizeof(c));
    c.k = b->k;
    c.k_end = b->k;
    c.timeout_ns = b->timeout_ns.load();
    {
        // fault injection for tests (HH_ENGINE_DROP_SIGNAL, as for contexts)
        const char *e = getenv("HH_ENGINE_DROP_SIGNAL");
        c.drop_sig = e ? atoi(e) : 0;
    }
    TraceRange tr("hh batch chunk");
    HB_TRY(cudaMemcpyAsync(b->d_ctl, &c, sizeof(c), cudaMemcpyHostToDevice, b->stream));
    rc = launch_chunk(b, grid);
    if (rc) return rc;
    HB_TRY(cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(EngCtl), cudaMemcpyDeviceToHost, b->stream));
    HB_TRY(cudaStreamSynchronize(b->stream));
    if (b->h_ctl->error != 0) {
        fail_all_active(b, b->h_ctl->error);
        b->k = 0;
        return b->h_ctl->error;
    }
    b->k = b->h_ctl->k_end;
    HB_TRY(cudaMemcpyAsync(b->h_states, b->d_state[b->k & 1], sizeof(EngState) * b->max_sys,
                           cudaMemcpyDeviceToHost, b->stream));
    HB_TRY(cudaStreamSynchronize(b->stream));
    for (int s = 0; s < (int)b->slots.size(); ++s) {
        Slot &S = b->slots[s];
        if (!S.used || !S.in_engine) continue;
        bool done = true;
        for (int a = 0; a < S.nrhs; ++a) {
            const EngState &E = b->h_states[s * kMaxRhs + a];
            long long steps = (long long)E.cg_steps + E.n_ru;
            b->site_iters += (double)(steps - S.last_steps[a]) * S.N;
            S.last_steps[a] = steps;
            S.rhs_done[a] = (E.mode == MODE_DONE);
            if (E.mode != MODE_DONE) done = false;
        }
        if (!done) continue;
        for (int a = 0; a < S.nrhs; ++a) {
            const EngState &E = b->h_states[s * kMaxRhs + a];
            S.cg_iters += E.cg_steps;
            S.n_ru += E.n_ru;
            S.n_solves += 1;
            if (E.true_relres > S.max_relres) S.max_relres = E.true_relres;
            if (E.status != 0 && S.status == 0) S.status = E.status;
        }
        rc = advance(b, s);
        if (rc) return rc;
    }
    return HH_OK;
}

bool has_work(hh_batch *b)
{
    std::lock_guard<std::mutex> lk(b->mu);
    return !b->queue.empty() || b->n_active > 0;
}

void worker_loop(hh_batch *b)
{
    while (b->running.load()) {
        if (!has_work(b)) {
            std::unique_lock<std::mutex> lk(b->mu);
            b->cv.wait_for(lk, std::chrono::microseconds(200));
            continue;
        }
        if (step(b) != HH_OK && b->n_active == 0) {
            std::lock_guard<std::mutex> lk(b->mu);
            if (!b->queue.empty()) b->failed = true;
        }
    }
}

void free_batch(hh_batch *b)
{
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    void *ptrs[] = {b->d_sys, b->d_state[0], b->d_state[1], b->d_tiles, b->d_sig, b->d_ctl,
                    b->arena.base};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (b->h_states) cudaFreeHost(b->h_states);
    if (b->h_ctl) cudaFreeHost(b->h_ctl);
}

}  // namespace

extern "C" {

void hh_batch_default_config(hh_batch_config *cfg)
{
    if (!cfg) return;
    cfg->max_slots = 64;
    cfg->hbm_budget_bytes = (size_t)4 << 30;
    cfg->chunk_iters = 32;
    cfg->tile_sites = 4096;
    cfg->max_active_sites = 0;
}

int hh_batch_create(hh_batch **out, const hh_batch_config *cfg, void *cuda_stream)
{
    if (!out || !cfg) return HH_EINVAL;
    *out = nullptr;
    if (cfg->max_slots < 1 || cfg->max_slots > kMaxSlots) return HH_EINVAL;
    if (cfg->chunk_iters < 1 || cfg->tile_sites < 32 || cfg->tile_sites % 32) return HH_EINVAL;
    if (cfg->hbm_budget_bytes < (1u << 20)) return HH_EINVAL;
    hh_batch *b = new (std::nothrow) hh_batch;
    if (!b) return HH_ENOMEM;
    b->cfg = *cfg;
    b->stream = (cudaStream_t)cuda_stream;
    b->slots.resize(cfg->max_slots);
    b->max_sys = cfg->max_slots * kMaxRhs;
    b->h_sys.resize(b->max_sys);
    memset(b->h_sys.data(), 0, sizeof(EngSystem) * b->max_sys);
    b->grid_of[ENGINE_GENERIC] = engine_default_grid(ENGINE_GENERIC);
    b->grid_of[ENGINE_D1] = engine_default_grid(ENGINE_D1);
    b->grid_of[ENGINE_D3] = engine_default_grid(ENGINE_D3);
    for (int k : {ENGINE_GENERIC, ENGINE_D1, ENGINE_D3}) b->two_slot_of[k] = engine_two_slot(k);
    b->ctl_warp = engine_ctl_warps(1);
    cudaError_t e = (b->grid_of[0] > 0 && b->grid_of[1] > 0 && b->grid_of[3] > 0) ? cudaSuccess
                                                                                 : cudaErrorUnknown;
    if (e == cudaSuccess) e = b->arena.init(cfg->hbm_budget_bytes);
    b->parts.init(kMaxTiles);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_sys, sizeof(EngSystem) * b->max_sys);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_state[0], sizeof(EngState) * b->max_sys);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_state[1], sizeof(EngState) * b->max_sys);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tiles, sizeof(EngTile) * kMaxTiles);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_sig, sizeof(unsigned long long) * engine_sig_count(kMaxTiles));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ctl, sizeof(EngCtl));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_states, sizeof(EngState) * b->max_sys);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_ctl, sizeof(EngCtl));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_state[0], 0, sizeof(EngState) * b->max_sys, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_state[1], 0, sizeof(EngState) * b->max_sys, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_sys, 0, sizeof(EngSystem) * b->max_sys, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        free_batch(b);
        delete b;
        return e == cudaErrorMemoryAllocation ? HH_ENOMEM : HH_ECUDA;
    }
    // Unused system entries are DONE so a stale table entry never runs.
    std::vector<EngState> done(b->max_sys);
    memset(done.data(), 0, sizeof(EngState) * b->max_sys);
    for (auto &z : done) z.mode = MODE_DONE;
    cudaMemcpy(b->d_state[0], done.data(), sizeof(EngState) * b->max_sys, cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_state[1], done.data(), sizeof(EngState) * b->max_sys, cudaMemcpyHostToDevice);
    *out = b;
    return HH_OK;
}

int hh_batch_set_timeout(hh_batch *b, double seconds)
{
    if (!b || !(seconds >= 0.0) || seconds > 3600.0) return HH_EINVAL;
    b->timeout_ns.store((long long)(seconds * 1e9));
    return HH_OK;
}

int hh_batch_destroy(hh_batch *b)
{
    if (!b) return HH_OK;
    hh_batch_stop(b);
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    delete b;
    return HH_OK;
}

int hh_batch_submit(hh_batch *b, const hh_request *req, uint64_t *ticket)
{
    if (!b || !req) return HH_EINVAL;
    int rc = validate(*req);
    if (rc) return rc;
    long long N = lattice_sites(req->lat);
    if (slot_bytes(N, req->prm.n_pf, req->prm.cheb_degree > 0, req->prm.chrono == 2, nullptr, nullptr) >
        b->arena.size)
        return HH_EBUSY;
    Pending P;
    P.req = *req;
    if (req->sigma) P.sigma.assign(req->sigma, req->sigma + N);
    if (req->kind == HH_REQ_SOLVE && req->b) P.b.assign(req->b, req->b + N * req->prm.n_pf);
    P.req.sigma = nullptr;
    P.req.b = nullptr;
    P.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(b->mu);
        P.ticket = b->next_ticket++;
        if (ticket) *ticket = P.ticket;
        b->queue.push_back(std::move(P));
    }
    b->cv.notify_one();
    return HH_OK;
}

int hh_batch_step(hh_batch *b, int *n_busy)
{
    if (!b) return HH_EINVAL;
    if (b->running.load()) return HH_EBUSY;
    int rc = step(b);
    if (n_busy) {
        std::lock_guard<std::mutex> lk(b->mu);
        *n_busy = (int)b->queue.size() + b->n_active.load();
    }
    return rc;
}

int hh_batch_start(hh_batch *b)
{
    if (!b) return HH_EINVAL;
    if (b->running.exchange(true)) return HH_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    b->worker = std::thread([b, dev]() {
        cudaSetDevice(dev);
        worker_loop(b);
    });
    return HH_OK;
}

int hh_batch_stop(hh_batch *b)
{
    if (!b) return HH_EINVAL;
    if (!b->running.exchange(false)) return HH_OK;
    b->cv.notify_all();
    if (b->worker.joinable()) b->worker.join();
    return HH_OK;
}

int hh_batch_poll(hh_batch *b, hh_result *out, int max, int *n_done)
{
    if (!b || (!out && max > 0)) return HH_EINVAL;
    std::lock_guard<std::mutex> lk(b->mu);
    int n = 0;
    while (n < max && !b->results.empty()) {
        out[n++] = b->results.front();
        b->results.pop_front();
    }
    if (n_done) *n_done = n;
    return HH_OK;
}

int hh_batch_pending(hh_batch *b, int *queued, int *active)
{
    if (!b) return HH_EINVAL;
    std::lock_guard<std::mutex> lk(b->mu);
    if (queued) *queued = (int)b->queue.size();
    if (active) *active = b->n_active.load();
    return HH_OK;
}

int hh_batch_autotune(const hh_request *sample, int n, size_t budget, int rounds, const char *cache_path,
                      void *cuda_stream, hh_batch_config *best)
{
    if (!sample || n < 1 || !best || rounds < 1) return HH_EINVAL;
    long long total_sites = 0;
    for (int i = 0; i < n; ++i) {
        if (validate(sample[i]) || sample[i].kind != HH_REQ_SOLVE) return HH_EINVAL;
        total_sites += lattice_sites(sample[i].lat);
    }
    const int tiles[] = {2048, 8192};
    const int chunks[] = {16, 64};
    // Active-site windows: none, and about what keeps the FP32 CG vectors of
    // the active systems (roughly 40 B per site and right-hand side) inside
    // half of the 129 MB L2.
    const long long windows[] = {0, 1600000};
    double best_rate = -1.0;
    hh_batch_config cfg_best;
    hh_batch_default_config(&cfg_best);
    for (int ti : tiles)
        for (int ci : chunks)
            for (long long wi : windows) {
                hh_batch_config cfg;
                hh_batch_default_config(&cfg);
                cfg.max_slots = n < kMaxSlots ? n : kMaxSlots;
                cfg.hbm_budget_bytes = budget;
                cfg.tile_sites = ti;
                cfg.chunk_iters = ci;
                cfg.max_active_sites = wi;
                hh_batch *b = nullptr;
                int rc = hh_batch_create(&b, &cfg, cuda_stream);
                if (rc) return rc;
                for (int i = 0; i < n; ++i) hh_batch_submit(b, &sample[i], nullptr);
                step(b);  // warm-up round: admission, plan, first chunk
                double s0 = b->site_iters;
                auto t0 = Clock::now();
                for (int r = 0; r < rounds; ++r)
                    if (step(b) != HH_OK) break;
                double sec = std::chrono::duration<double>(Clock::now() - t0).count();
                double rate = (b->site_iters - s0) / (sec > 0 ? sec : 1e-9);
                hh_batch_destroy(b);
                if (rate > best_rate) {
                    best_rate = rate;
                    cfg_best = cfg;
                }
            }
    *best = cfg_best;
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (f) {
            fprintf(f,
                    "{\"key\": \"d%d_prec%d_n%d_sites%lld\", \"tile_sites\": %d, \"chunk_iters\": %d, "
                    "\"max_active_sites\": %lld, \"site_iters_per_s\": %.6g}\n",
                    sample[0].lat.d, sample[0].prm.precision, n, total_sites, cfg_best.tile_sites,
                    cfg_best.chunk_iters, cfg_best.max_active_sites, best_rate);
            fclose(f);
        }
    }
    return HH_OK;
}

}  // extern "C"
