// Persistent conjugate-gradient engine: host/device shared declarations.
//
// One cooperative launch runs CG (Sec. 4.1) on a table of independent linear
// systems Q_s x_s = b_s (right-hand sides of one lattice, or chains of
// different lattices).  Each system is cut into tiles of contiguous sites; the
// blocks of the grid own fixed tiles.  An engine iteration has three slots,
// and each system executes one mode per iteration:
//
//   mode   slot 1                 slot 2                slot 3
//   INIT   x = 0                  -                     r = b, partial |r|^2
//   CG     p = r + beta p         t = M p, partial |t|^2  alpha = rr/|t|^2 (|t|^2 = p.Qp),
//                                                       x += alpha p, r -= alpha M^T t,
//                                                       partial |r|^2
//   RU     x64 += x32, x32 = 0    t64 = M x64 (FP64)    r = b - M^T t64 (FP64),
//          (mixed only)                                 partial |r|^2
//
// Slots are ordered per system, not across the grid: at the end of each slot
// every tile publishes its partial sum into a signal slot (see EngCtl), and a
// block starts the next slot of a system once every tile of that system has
// published; the poll that waits also delivers the partials.  A block whose
// systems are all done leaves the kernel.  At slot 1 every block that owns a
// tile of system s sums that system's per-tile partials in a fixed order and
// takes the same decision (next mode, beta, convergence), so no atomics are
// needed; one designated block writes the system's state.  RU recomputes the
// true residual in FP64: it is the stopping test in FP64 mode (with residual
// replacement when the recursive residual has drifted) and the reliable
// update of the mixed mode (FP32 inner iteration, FP64 solution).
//
// Two-slot form (EngLaunch::two_slot): slot 1 is folded into slot 2.  The new
// direction p = r + beta p_old is written to the other of two p buffers while
// t = M p is computed from p recomputed at the neighbour sites (r and p_old
// are final there), and the reliable update's x64 + x32 likewise; slot 3 is
// unchanged.  One synchronisation and one read-write of p fewer per
// iteration, for one extra read of r and p_old at each neighbour row.
// Measured on GB300, it is faster for d = 1 (two x-halo sites and one earlier
// row) and slower for d = 3 (six neighbour rows), so the d = 1 kernel runs it
// and the others do not.  The result is bitwise the same in both forms.
#pragma once

#include "hh_device.cuh"

namespace hh {

enum EngMode : int { MODE_NEW = 0, MODE_INIT = 1, MODE_CG = 2, MODE_RU = 3, MODE_DONE = 4, MODE_PRE = 5 };

// Chebyshev preconditioner (Sec. 4.2): z = P(Q/lam) r is applied as n real
// quadratic factors ((Q/lam - a_k)^2 + b_k^2) / q_k, each two applications of
// Q, i.e. 2n engine iterations in MODE_PRE (sub-step j: t = M v in slot 2, the
// factor update in slot 3).  Coefficient table: [0] = 1/lam, [1] = 1/m with
// m = (1 + eps)/2, then (a_k, b_k^2, 1/q_k) for k = 1..n.
constexpr int CHEB_MAX_DEGREE = 64;

enum EngPrecision : int { PREC_FP64 = 0, PREC_MIXED = 1 };

struct EngSystem {
    Geo g;
    double h;
    const double *L64;
    const float *L32;
    const double *b;
    double *x;                        // FP64 solution
    double *r, *p, *t;                // FP64 CG vectors (t also FP64 scratch for RU)
    float *r32, *p32, *t32, *x32;     // FP32 inner vectors (mixed)
    int tile0, ntiles;                // tiles [tile0, tile0 + ntiles) of the global tile list
    int part0;                        // partial sums of its tiles: [part0, part0 + ntiles),
                                      // stable for the system's lifetime even when the
                                      // tile list is rebuilt between launches
    int owner;                        // block that writes this system's state
    int precision;                    // PREC_FP64 or PREC_MIXED
    double tol2;                      // cg_tol^2
    double delta2;                    // reliable_delta^2 (mixed)
    int maxit;
    int w;                            // x sites per thread group: 4, 2 or 1 (divides Nx)
    int pf;                           // CG site loops prefetch into L2 this many rounds of the
                                      // loop ahead (0: none; see engine_prefetch)
    int stall_window;                 // mixed: forced RU after this many FP32 steps without one
    int cheb_n;                       // Chebyshev preconditioner degree n (0: plain CG; FP64 only)
    int x0_given;                     // 1: x holds an initial guess when the system starts (MODE_NEW)
    int link_order;                   // form of M: 0 reading R1; 1, 2 exact-block (three-slot form,
                                      // no preconditioner, scalar site loops)
    const double *cheb;               // coefficient table (see CHEB_MAX_DEGREE)
    double *z, *u;                    // FP64 preconditioner vectors (when cheb_n > 0)
    double *p2;                       // second FP64 p buffer (two-slot launches)
    float *p32b;                      // second FP32 p buffer (two-slot launches)
    const unsigned short *L16;        // 16-bit links of the FP32 steps (link16 != 0)
    int link16;                       // links of the FP32 steps: 0 L32; 1 L16 as bfloat16;
                                      // 2 L16 as fixed point times l16_scale (see LinkSrc)
    float l16_scale;
};

// FP32 steps after which a mixed system takes a reliable update even if its
// FP32 residual has not dropped by reliable_delta (a plateau of the FP32
// iteration when eps_32 * cond(Q) >~ 1).
constexpr int ENGINE_STALL_WINDOW = 2000;

// Group width for a lattice: the largest of 4, 2, 1 that divides Nx.
__host__ __device__ inline int engine_group_width(int nx)
{
    return (nx % 4 == 0) ? 4 : (nx % 2 == 0) ? 2 : 1;
}

struct EngState {
    double bb;          // |b|^2
    double rr_alpha;    // |r|^2 of the residual the current CG step starts from
    double rr_last;     // last reduced |r|^2
    double maxr2;       // max |r|^2 since the last reliable update (mixed)
    double beta;
    double true_relres; // last true relative residual (RU)
    double rr_ru;       // true |r|^2 at the last RU (stall detection)
    int mode;           // mode executed in the iteration that wrote this state
    int cg_steps;
    int n_ru;
    int status;         // 0, or HH_ENOCONV / HH_ENUMERIC
    int final_ru;       // RU forced by the iteration cap
    int prec;           // precision of the CG steps now running (a mixed system
                        // switches to PREC_FP64 when FP32 steps stop reducing
                        // the true residual)
    int stall;          // consecutive reliable updates without progress
    int fp64_steps;     // CG steps run in FP64
    int since_ru;       // CG steps since the last RU
    int pre_j;          // MODE_PRE sub-step, 0 .. 2 cheb_n - 1
    int pbuf;           // two-slot launches: p buffer (0: p/p32, 1: p2/p32b) holding p
    int no_guess;       // the initial guess was dropped (b = 0): INIT zeroes x
};

struct EngTile {
    int sys;
    int begin, end;     // sites [begin, end) of the system
    int part;           // index of this tile's partial sums (part0 of its system + j)
};

struct EngLaunch {
    const EngSystem *sys;
    EngState *state[2];     // double buffer by engine-iteration parity
    const EngTile *tiles;
    // Signal slots (see EngCtl): slot of tile part p for the phase with index
    // ph (0: first slot, 1: slot 2 of the three-slot form, 2: slot 3) at
    // iteration parity q is sig[(2 * ph + q) * sig_stride + p].  A system's
    // slots must be empty (kSigEmpty) when it enters as MODE_NEW.
    unsigned long long *sig;
    int sig_stride;
    int ctl_warp;           // control warps (see the kernel): 0 flat, 1 warp 0, 2 warps 0 and 1
    EngCtl *ctl;
    int nsys, ntiles;
    long long max_iters;    // engine iterations this launch may run
    int two_slot;           // 1: two phases per iteration (see above)
    int homogeneous;        // 1: every block holds one tile of each of the (two or
                            // more) systems, in the same order (requires ctl_warp)
};

// Signal slots needed for 'parts' tile partial indices.
__host__ __device__ constexpr size_t engine_sig_count(int parts)
{
    return (size_t)6 * (size_t)parts;
}

// Engine kernels: ENGINE_GENERIC handles systems of both dimensions in one
// launch; ENGINE_D1 / ENGINE_D3 require every system of the launch to have
// that dimension and are compiled for it.
// ENGINE_EXBLOCK runs systems with the exact-block form of M (link_order 1,
// 2) only, with scalar site loops, kept apart so that the other kernels do
// not carry its code.  ENGINE_D1_L16 / ENGINE_D3_L16 are the d = 1 / d = 3
// kernels whose FP32 steps read 16-bit links (EngSystem::link16 != 0 for
// every mixed system of the launch), likewise kept apart.
enum EngKind : int {
    ENGINE_GENERIC = 0,
    ENGINE_D1 = 1,
    ENGINE_D3 = 3,
    ENGINE_EXBLOCK = 4,
    ENGINE_D1_L16 = 5,
    ENGINE_D3_L16 = 7
};

// Host launcher: runs the engine with a cooperative launch of 'grid' blocks.
// When the launch starts, the signal slots of every system entering as
// MODE_NEW must be empty (kSigEmpty), ctl->error must be zero, and ctl->k must
// hold the iteration counter the state buffers were written at (0 for a fresh
// plan).  Launches with more than ENGINE_MAX_SYSTEMS systems are refused
// (cudaErrorInvalidValue).  Returns a cudaError_t from the launch.
cudaError_t engine_launch(const EngLaunch &L, int grid, int block, cudaStream_t stream, int kind);

// The engine kernel of a kind, for CUDA-graph kernel nodes.
const void *engine_kernel_fn(int kind);

// Largest co-resident grid for the engine kernel of a kind at 'block' threads.
int engine_max_grid(int block, int kind);

constexpr int ENGINE_BLOCK = 512;
// Systems of one launch, at most (the per-block record of decided modes).
constexpr int ENGINE_MAX_SYSTEMS = 1024;
constexpr int ENGINE_MIN_TILE = 512;   // sites per tile, at least one per thread

// Default grid: one block per SM (fewer blocks per wait), capped
// by co-residency.
// HH_ENGINE_BLOCKS_PER_SM overrides the blocks per SM.
int engine_default_grid(int kind);

// 1 if launches of a kernel kind run the two-slot form: by default for
// ENGINE_D1 only; HH_ENGINE_SLOTS=2 or 3 forces one form.  The forms give
// bitwise identical results.
int engine_two_slot(int kind);

// Coefficient table of the Chebyshev preconditioner of degree n (see
// CHEB_MAX_DEGREE) for the lattice dimension d, hop h = t dtau and coupling A:
// writes 2 + 3 CHEB_MAX_DEGREE doubles.
void engine_cheb_table(int d, double h, double A, int n, double eps, double *tab);

// Control warps of an engine launch: 'dflt', unless HH_ENGINE_CTL_WARPS (0, 1
// or 2) overrides it.
int engine_ctl_warps(int dflt);

// Whether a launch of nsys systems of 'sites' sites each uses the overlapped
// layout (see EngLaunch::homogeneous); HH_ENGINE_OVERLAP=0 or 1 forces it.
bool engine_overlap(int nsys, long long sites, bool mixed);

// L2 prefetch distance (EngSystem::pf) of a system of dimension d in a
// launch whose CG vectors take 'bytes' in all: one round of the site loop
// ahead for d = 3 when they overflow about half of the L2 (the loops then wait
// on DRAM, one round trip per round; measured on GB300: 13% less time per
// mixed iteration on 32^3 x 128), else none (d = 1 loops run 2-9% slower with
// it).  HH_ENGINE_PREFETCH sets the distance.
int engine_prefetch(long long bytes, int d);

// Tiles of one system: 'tiles' contiguous ranges of 'chunk' sites (the last
// one shorter), enough to give every block of the grid a tile when 'nsys'
// systems share the launch.
struct Tiling {
    int tiles, chunk;
};

inline Tiling engine_tiling(int N, int nsys, int max_grid)
{
    int by_size = (N + ENGINE_MIN_TILE - 1) / ENGINE_MIN_TILE;
    int want = (max_grid + nsys - 1) / (nsys > 0 ? nsys : 1);
    if (want < 1) want = 1;
    int tps = by_size < want ? by_size : want;
    if (tps < 1) tps = 1;
    int chunk = (N + tps - 1) / tps;
    chunk = (chunk + 31) / 32 * 32;
    Tiling t;
    t.chunk = chunk;
    t.tiles = (N + chunk - 1) / chunk;
    return t;
}

}  // namespace hh
