// Persistent conjugate-gradient engine: host/device shared declarations.
//
// One cooperative launch runs CG (Sec. 4.1) on a table of independent linear
// systems Q_s x_s = b_s (right-hand sides of one lattice, or chains of
// different lattices).  Each system is cut into tiles of contiguous sites; the
// blocks of the grid own fixed tiles.  An engine iteration has three slots
// separated by grid barriers, and each system executes one mode per iteration:
//
//   mode   slot 1                 slot 2                slot 3
//   INIT   x = 0                  -                     r = b, partial |r|^2
//   CG     p = r + beta p         t = M p, partial |t|^2  alpha = rr/|t|^2 (|t|^2 = p.Qp),
//                                                       x += alpha p, r -= alpha M^T t,
//                                                       partial |r|^2
//   RU     x64 += x32, x32 = 0    t64 = M x64 (FP64)    r = b - M^T t64 (FP64),
//          (mixed only)                                 partial |r|^2
//
// At slot 1 every block that owns a tile of system s sums that system's
// per-tile partials in a fixed order and takes the same decision (next mode,
// beta, convergence), so no atomics or extra barriers are needed; one
// designated block writes the system's state.  RU recomputes the true
// residual in FP64: it is the stopping test in FP64 mode (with residual
// replacement when the recursive residual has drifted) and the reliable update
// of the mixed mode (FP32 inner iteration, FP64 solution).
#pragma once

#include "hh_device.cuh"

namespace hh {

enum EngMode : int { MODE_NEW = 0, MODE_INIT = 1, MODE_CG = 2, MODE_RU = 3, MODE_DONE = 4 };

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
    int owner;                        // block that writes this system's state
    int precision;                    // PREC_FP64 or PREC_MIXED
    double tol2;                      // cg_tol^2
    double delta2;                    // reliable_delta^2 (mixed)
    int maxit;
    int pad;
};

struct EngState {
    double bb;          // |b|^2
    double rr_alpha;    // |r|^2 of the residual the current CG step starts from
    double rr_last;     // last reduced |r|^2
    double maxr2;       // max |r|^2 since the last reliable update (mixed)
    double beta;
    double true_relres; // last true relative residual (RU)
    int mode;           // mode executed in the iteration that wrote this state
    int cg_steps;
    int n_ru;
    int status;         // 0, or HH_ENOCONV / HH_ENUMERIC
    int final_ru;       // RU forced by the iteration cap
    int pad;
};

struct EngTile {
    int sys;
    int begin, end;     // sites [begin, end) of the system
};

struct EngLaunch {
    const EngSystem *sys;
    EngState *state[2];     // double buffer by engine-iteration parity
    const EngTile *tiles;
    double *part_tt;        // per-tile partials of |t|^2
    double *part_rr;        // per-tile partials of |r|^2
    BarrierCtl *ctl;
    int nsys, ntiles;
    long long max_iters;    // engine iterations this launch may run
};

// Host launcher: runs the engine with a cooperative launch of 'grid' blocks.
// Returns a cudaError_t from the launch.
cudaError_t engine_launch(const EngLaunch &L, int grid, int block, cudaStream_t stream);

// Largest co-resident grid for the engine kernel at 'block' threads.
int engine_max_grid(int block);

constexpr int ENGINE_BLOCK = 256;

}  // namespace hh
