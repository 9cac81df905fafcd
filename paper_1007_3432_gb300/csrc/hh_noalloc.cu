// A solve entry point that allocates nothing.
//
// Some callers cannot allocate memory at the point where they need a solve:
// plug-ins hosted by an application that owns the device allocator and
// forbids other allocations, or real-time loops that must not take the
// allocator's locks.  hh_solve_noalloc serves them: the
// caller passes the field sigma, the right-hand side b and the output x, and
// every other buffer the FP64 CG needs (links, CG vectors, the system table,
// tiles, signal slots, the control block) lives in one file-scope
// __device__ array of fixed size, reserved on every device that loads the
// library for as long as the process lives.
//
// The array is shared by all calls: each call overwrites it, and the parts
// that must start from a known value (the engine's signal slots, both engine
// state buffers, and the control block's error word and iteration counters)
// are reset by the call itself.  Calls whose GPU work overlaps (two host
// threads, or two streams running at once) race on the array and give wrong
// results; callers must serialise them.
//
// The array's device address is looked up on every call
// (cudaGetSymbolAddress, which allocates nothing): a caller that resets the
// device, or otherwise re-creates its primary context, gets the library's
// module loaded again and the array may then live at another address.  Only
// the engine's co-resident grid size, a property of the device, is kept
// between calls.
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/hubhmc.h"
#include "hh_engine.cuh"
#include "hh_kernels.cuh"

using namespace hh;

namespace {

constexpr int kMaxSites = HH_NOALLOC_MAX_SITES;
constexpr int kMaxTiles = 2048;

constexpr size_t align256(size_t v)
{
    return (v + 255) / 256 * 256;
}

// Byte layout of the scratch array.
constexpr size_t kOffL64 = 0;
constexpr size_t kOffL32 = kOffL64 + align256(sizeof(double) * kMaxSites);
constexpr size_t kOffR = kOffL32 + align256(sizeof(float) * kMaxSites);
constexpr size_t kOffP = kOffR + align256(sizeof(double) * kMaxSites);
constexpr size_t kOffT = kOffP + align256(sizeof(double) * kMaxSites);
constexpr size_t kOffSys = kOffT + align256(sizeof(double) * kMaxSites);
constexpr size_t kOffState = kOffSys + align256(sizeof(EngSystem));
constexpr size_t kOffTiles = kOffState + align256(2 * sizeof(EngState));
constexpr size_t kOffSig = kOffTiles + align256(sizeof(EngTile) * kMaxTiles);
constexpr size_t kOffCtl = kOffSig + align256(sizeof(unsigned long long) * engine_sig_count(kMaxTiles));
constexpr size_t kScratchBytes = kOffCtl + align256(sizeof(EngCtl));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
int g_max_grid[kMaxDevices][2];   // engine grid for d = 1 and d = 3 (0: not yet queried)

// With the device 'dev' current: the device address of the scratch array
// (the host-side symbol is only a stand-in for it), looked up on every call,
// and the engine's co-resident grid size, queried on the first call on that
// device and kept.
int setup_device(int dev, int d, unsigned char **base, int *max_grid)
{
    if (dev < 0 || dev >= kMaxDevices) return HH_EINVAL;
    void *addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || !addr) return HH_ECUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_max_grid[dev][0] <= 0) {
        int g1 = engine_default_grid(ENGINE_D1), g3 = engine_default_grid(ENGINE_D3);
        if (g1 <= 0 || g3 <= 0) return HH_ECUDA;
        g_max_grid[dev][0] = g1;
        g_max_grid[dev][1] = g3;
    }
    *base = (unsigned char *)addr;
    *max_grid = g_max_grid[dev][d == 1 ? 0 : 1];
    return HH_OK;
}

// Writes the system table and the tiles into the scratch array, and resets
// the engine state, the signal slots of the tiles and the control block.
__global__ void k_noalloc_plan(unsigned char *base, Geo g, double h, const double *b, double *x,
                               double tol, int maxit, int chunk, int ntiles, int grid,
                               long long timeout_ns)
{
    EngTile *tiles = (EngTile *)(base + kOffTiles);
    for (int j = threadIdx.x; j < ntiles; j += blockDim.x) {
        EngTile T;
        T.sys = 0;
        T.begin = j * chunk;
        T.end = (j + 1) * chunk < g.N ? (j + 1) * chunk : g.N;
        T.part = j;
        tiles[j] = T;
    }
    unsigned long long *sig = (unsigned long long *)(base + kOffSig);
    for (int ph = 0; ph < 6; ++ph)
        for (int j = threadIdx.x; j < ntiles; j += blockDim.x) sig[(size_t)ph * kMaxTiles + j] = kSigEmpty;
    if (threadIdx.x == 0) {
        EngSystem Y;
        memset(&Y, 0, sizeof(Y));
        Y.g = g;
        Y.h = h;
        Y.L64 = (const double *)(base + kOffL64);
        Y.L32 = (const float *)(base + kOffL32);
        Y.b = b;
        Y.x = x;
        Y.r = (double *)(base + kOffR);
        Y.p = (double *)(base + kOffP);
        Y.t = (double *)(base + kOffT);
        Y.tile0 = 0;
        Y.ntiles = ntiles;
        Y.part0 = 0;
        Y.owner = 0;
        Y.precision = PREC_FP64;
        Y.tol2 = tol * tol;
        Y.delta2 = 0.0;
        Y.maxit = maxit;
        Y.w = engine_group_width(g.nx);
        Y.stall_window = ENGINE_STALL_WINDOW;
        *(EngSystem *)(base + kOffSys) = Y;
        EngState z;
        memset(&z, 0, sizeof(z));
        z.mode = MODE_NEW;
        EngState *st = (EngState *)(base + kOffState);
        st[0] = z;
        st[1] = z;
        EngCtl *ctl = (EngCtl *)(base + kOffCtl);
        ctl->error = 0;
        ctl->k = 0;
        ctl->k_end = 0;
        ctl->timeout_ns = timeout_ns;
        ctl->drop_sig = 0;
    }
}

}  // namespace

extern "C" int hh_solve_noalloc(const hh_lattice *lat, const hh_params *p, const double *sigma,
                                const double *b, double *x, void *cuda_stream, hh_solve_info *info)
{
    if (!lat || !p || !sigma || !b || !x) return HH_EINVAL;
    if (((uintptr_t)b & 15u) || ((uintptr_t)x & 15u)) return HH_EINVAL;
    if (lat->d != 1 && lat->d != 3) return HH_EINVAL;
    if (lat->nx < 2 || lat->ntau < 2) return HH_EINVAL;
    if (p->precision != HH_FP64 || !(p->cg_tol > 0.0) || p->cg_maxit < 1) return HH_EINVAL;
    if (p->link_order != 0 || p->cheb_degree != 0) return HH_EINVAL;
    long long V = lat->d == 1 ? lat->nx : (long long)lat->nx * lat->nx * lat->nx;
    long long N = V * lat->ntau;
    if (N > kMaxSites) return HH_ESIZE;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (info) {
        // Filling info copies the outcome to the host and synchronises the
        // stream, which a stream in capture mode does not allow.
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return HH_ECUDA;
        if (cap != cudaStreamCaptureStatusNone) return HH_EINVAL;
    }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HH_ECUDA;
    unsigned char *base = nullptr;
    int max_grid = 0;
    int rc = setup_device(dev, lat->d, &base, &max_grid);
    if (rc) return rc;

    Geo g = make_geo(lat->d, lat->nx, lat->ntau);
    // The same grid and tiling rule as the context solver.
    Tiling tl = engine_tiling(g.N, 1, max_grid);
    int chunk = tl.chunk, ntiles = tl.tiles;
    if (ntiles > kMaxTiles) return HH_ESIZE;
    int grid = ntiles < max_grid ? ntiles : max_grid;

    double *L64 = (double *)(base + kOffL64);
    float *L32 = (float *)(base + kOffL32);
    if (launch_links(g, p->A, sigma, L64, L32, st) != cudaSuccess) return HH_ECUDA;
    k_noalloc_plan<<<1, 256, 0, st>>>(base, g, p->t * p->dtau, b, x, p->cg_tol, p->cg_maxit, chunk,
                                      ntiles, grid, 5LL * 1000 * 1000 * 1000);
    if (cudaGetLastError() != cudaSuccess) return HH_ECUDA;

    EngLaunch L;
    L.sys = (const EngSystem *)(base + kOffSys);
    L.state[0] = (EngState *)(base + kOffState);
    L.state[1] = L.state[0] + 1;
    L.tiles = (const EngTile *)(base + kOffTiles);
    L.sig = (unsigned long long *)(base + kOffSig);
    L.sig_stride = kMaxTiles;
    L.ctl_warp = 0;
    L.ctl = (EngCtl *)(base + kOffCtl);
    L.nsys = 1;
    L.ntiles = ntiles;
    L.max_iters = 3LL * (long long)p->cg_maxit + 64;
    L.two_slot = 0;     // one p buffer in the static scratch
    L.homogeneous = 0;
    if (engine_launch(L, grid, ENGINE_BLOCK, st, lat->d == 1 ? ENGINE_D1 : ENGINE_D3) != cudaSuccess)
        return HH_ECUDA;
    if (!info) return HH_OK;

    // Results into caller stack memory (pageable copies, no allocation).
    EngCtl ctl;
    EngState S;
    if (cudaMemcpyAsync(&ctl, L.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return HH_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HH_ECUDA;
    if (cudaMemcpyAsync(&S, L.state[ctl.k_end & 1], sizeof(S), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return HH_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HH_ECUDA;
    info->iterations = S.cg_steps;
    info->reliable_updates = S.n_ru;
    info->true_relres = S.true_relres;
    info->converged = (S.mode == MODE_DONE && S.status == 0 && ctl.error == 0) ? 1 : 0;
    if (ctl.error != 0) return ctl.error;
    if (S.mode != MODE_DONE) return HH_ETIMEOUT;
    return S.status;
}
