/*
 * hubhmc: Hybrid Monte Carlo for the Hubbard model on one GB300 GPU.
 *
 * C ABI of the library.  The method is that of K. A. Wendt, J. E. Drut and
 * T. A. Laehde, "Toward large-scale Hybrid Monte Carlo simulations of the
 * Hubbard model on graphics processing units" (arXiv:1007.3432):
 *   - the fermion matrix M on a (d+1)-dimensional space-time lattice
 *     (Sec. 2, Eqs. (7)-(10)): unit diagonal, -h = -t*dtau on the 2d spatial
 *     nearest neighbours (periodic), and one time link per site carrying
 *     L(n,tau) = -(1 + A sin sigma(n,tau)) into slice tau+1, with the sign
 *     flipped on the wrap link N_tau-1 -> 0 (antiperiodic in time);
 *   - the normal matrix Q = M^T M and the linear problem Q x = b solved by
 *     conjugate gradient (Sec. 4.1);
 *   - the pseudofermion action S_pf = 1/2 sum_a chi_a^T Q^{-1} chi_a
 *     (Eqs. (11)-(12)), its force dS_pf/dsigma, leapfrog molecular dynamics and
 *     the Metropolis accept/reject step of the phi-algorithm (Sec. 4.1);
 *   - the Chebyshev-polynomial preconditioner of Sec. 4.2 and the exact-block
 *     form of Eq. (7) as options.
 * Beyond the paper: FP32 inner CG with FP64 reliable updates (optionally with
 * 16-bit links), the Omelyan integrator and chronological initial guesses,
 * noise estimators of diag M^{-1} (observables), a batched multi-chain engine
 * with a serving loop, and an allocation-free solve.
 *
 * Conventions for every call:
 *   - Arrays are indexed by site i = x + Nx*(y + Nx*(z + Nx*tau)) for d = 3 and
 *     i = x + Nx*tau for d = 1 (x fastest).  A "vector" holds N = Nx^d * Ntau
 *     elements; n_rhs vectors are stored back to back (vector a at a*N).
 *   - Pointers documented as device pointers must point to CUDA device memory
 *     of the current device; the caller owns them and keeps them alive until
 *     the call's work on the context stream has finished.  Vector arguments
 *     (b, x, chi) must be 16-byte aligned (they are accessed with 16-byte
 *     loads and stores); a misaligned one is refused with HH_EINVAL.
 *   - All GPU work of a context is ordered on the stream given at creation.
 *     Calls that return results in host structures (an info argument, host
 *     output pointers) synchronise that stream before they return; the other
 *     calls only enqueue work.
 *   - Every call returns HH_OK (0) or a negative error code; no C++ exception
 *     crosses the ABI.  After an error the context stays valid unless the
 *     error is HH_ECUDA from a sticky CUDA fault.
 *   - A context is not thread safe: one host thread at a time may use it.
 */
#ifndef HUBHMC_H
#define HUBHMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define HH_OK 0
#define HH_EINVAL (-1)   /* invalid argument (shape, pointer, enum) */
#define HH_ENOMEM (-2)   /* device or host allocation failed */
#define HH_ECUDA (-3)    /* a CUDA runtime call failed */
#define HH_ENOCONV (-4)  /* CG reached its iteration cap above tolerance */
#define HH_ENUMERIC (-5) /* NaN or Inf met in a reduction */
#define HH_ETIMEOUT (-6) /* a bounded device-side wait ran out */
#define HH_EBUSY (-7)    /* no free slot or memory budget for the request */

/* Precision of the CG solve.
 *   HH_FP64:  every stencil apply, vector update and reduction in FP64.
 *   HH_MIXED: FP32 inner CG (FP32 links, vectors and stencil, products summed
 *             per thread in FP32 and across threads in FP64) with reliable
 *             updates that accumulate the solution and recompute the true
 *             residual b - Q x in FP64; the stopping test is on that FP64 true
 *             residual, so both modes meet the same tolerance.
 *   HH_MIXED_BF16LINK, HH_MIXED_FIX16LINK: HH_MIXED with the links of the
 *             FP32 steps stored in 16 bits (2 bytes per site fewer per
 *             stencil sweep): the bfloat16 rounding of the FP32 link (8
 *             significant bits), or a fixed-point code c with L = c * 2^-e,
 *             e = 14 while (1 + |A|) 2^14 fits in 15 bits (absolute error
 *             <= 2^-(e+1)).  The reliable updates use the FP64 links, so the
 *             result meets the same tolerance; the inner iteration solves a
 *             perturbed system, which costs extra reliable updates once
 *             cond(Q) times the link error approaches reliable_delta
 *             (bfloat16 on hot lattices of cond(Q) ~ 1e4 and above).
 *             Contexts with link_order 0 only. */
#define HH_FP64 0
#define HH_MIXED 1
#define HH_MIXED_BF16LINK 2
#define HH_MIXED_FIX16LINK 3

/* Operators for hh_apply. */
#define HH_OP_M 0   /* y = M x */
#define HH_OP_MT 1  /* y = M^T x */
#define HH_OP_MTM 2 /* y = M^T M x = Q x */

/* Element types for hh_apply. */
#define HH_DTYPE_F64 0
#define HH_DTYPE_F32 1

typedef struct hh_ctx hh_ctx;

typedef struct {
    int d;    /* spatial dimension: 1 or 3 */
    int nx;   /* spatial extent N_x >= 2 (periodic) */
    int ntau; /* time slices N_tau >= 2 (antiperiodic) */
} hh_lattice;

typedef struct {
    double t;              /* hopping amplitude; h = t * dtau */
    double dtau;           /* Trotter time step */
    double A;              /* auxiliary-field coupling in 1 + A sin(sigma) */
    int precision;         /* HH_FP64, HH_MIXED, HH_MIXED_BF16LINK or HH_MIXED_FIX16LINK */
    double cg_tol;         /* stop when ||b - Q x||_2 <= cg_tol * ||b||_2 */
    int cg_maxit;          /* cap on CG iterations per solve */
    double reliable_delta; /* HH_MIXED: reliable update when ||r|| < delta * max ||r|| */
    uint64_t seed;         /* Philox key for all random draws of the context */
    int n_pf;              /* real pseudofermion components (2: weight (det M)^2) */
    uint64_t chain_id;     /* Philox counter word identifying the Markov chain */
    int cheb_degree;       /* n of the Chebyshev preconditioner P(Q) of Sec. 4.2
                              (degree 2n, Eqs. (13)-(15)); 0: plain CG.  HH_FP64
                              contexts only. */
    double cheb_eps;       /* its interval (eps, 1] for Q scaled by the Gershgorin
                              bound (2 + 2 d h + A)^2 of its spectrum */
    int integrator;        /* molecular dynamics: HH_LEAPFROG (Sec. 4.1; n_md + 1
                              forces) or HH_OMELYAN (second-order minimum-norm
                              scheme of Omelyan, Mryglod and Folk, Comput. Phys.
                              Commun. 151 (2003) 272; 2 n_md + 1 forces, energy
                              violation about 20x smaller at equal dt) */
    int chrono;            /* initial guess of a trajectory's solves after the
                              first: 0 zero (MD exactly reversible); 1 the
                              previous force's solution; 2 the linear
                              extrapolation of the last two.  1 and 2 make the
                              MD reversible only to the CG tolerance. */
    int link_order;        /* form of M.  0: reading R1, diagonal blocks 1 - h H
                              (H: sum over the 2d spatial neighbours) and links
                              L = -(1 + A sin sigma).  1, 2: the exact-block form
                              of Eq. (7), B = e^{-dtau K} e^{-dtau V} with
                              e^{-dtau K} = e^{h H} expanded to that order:
                              (M x)(n,tau) = x(n,tau) + [E (L x)](n,tau-1),
                              E = 1 + h H (+ h^2 H^2 / 2).  Contexts only (not
                              batch requests or hh_solve_noalloc); no Chebyshev
                              preconditioner; scalar kernels. */
} hh_params;

#define HH_LEAPFROG 0
#define HH_OMELYAN 1

typedef struct {
    int iterations;       /* CG iterations of the solve (largest over right-hand sides) */
    int reliable_updates; /* true-residual recomputations (summed over right-hand sides) */
    double true_relres;   /* largest ||b - Q x|| / ||b|| over right-hand sides */
    int converged;        /* 1 if every right-hand side met cg_tol */
} hh_solve_info;

typedef struct {
    double H0, H1, dH;     /* Hamiltonian 1/2 |pi|^2 + S_pf before / after the MD */
    double u;              /* Metropolis uniform (Philox tag 3) */
    int accepted;          /* 1 iff u < exp(-dH); on 0 sigma is restored */
    int cg_iterations;     /* CG iterations summed over all solves */
    int n_solves;          /* right-hand sides solved: n_pf * forces (H0 and H1
                              reuse the first and last solve) */
    double max_true_relres;/* largest true relative residual over the solves */
} hh_traj_info;

/* Fill p with the defaults t = 1, dtau = 0.05, A = 0.5, FP64, cg_tol = 1e-10,
 * cg_maxit = 1000000, reliable_delta = 0.1, seed = 0, n_pf = 2, chain_id = 0,
 * cheb_degree = 0 (plain CG), cheb_eps = 1e-3, integrator = HH_LEAPFROG, chrono = 0,
 * link_order = 0. */
void hh_default_params(hh_params *p);

/* Create a context for one lattice and one Markov chain.  Allocates sigma,
 * the links (FP64 and FP32), the HMC fields and the CG workspace on the
 * current device.  stream: a cudaStream_t (NULL = legacy default stream).
 * sigma starts at zero.  Errors: HH_EINVAL (d not 1 or 3, nx < 2, ntau < 2,
 * N >= 2^31, n_pf < 1, unknown precision), HH_ENOMEM, HH_ECUDA. */
int hh_create(hh_ctx **out, const hh_lattice *lat, const hh_params *p, void *cuda_stream);

/* Free every device and host resource of the context (after synchronising
 * its stream).  NULL is accepted. */
int hh_destroy(hh_ctx *ctx);

/* Number of sites N of the context's lattice (0 for NULL). */
long long hh_nsites(const hh_ctx *ctx);

/* Copy N doubles into the context's auxiliary field sigma (Eq. (8): the
 * field of time slice tau lives on the link out of that slice) and recompute
 * the links.  on_device = 1: sigma is a device pointer (copy on the stream);
 * 0: a host pointer (synchronous copy).  Errors: HH_EINVAL for NULL. */
int hh_set_field(hh_ctx *ctx, const double *sigma, int on_device);

/* Copy the context's sigma out (N doubles), to device (on_device = 1, on the
 * stream) or host memory (0, synchronous). */
int hh_get_field(hh_ctx *ctx, double *sigma, int on_device);

/* sigma(i) = -pi + 2 pi u_i with u_i the Philox uniform of tag 0, block i/4,
 * word i%4, trajectory word 0 and the context's chain_id, key (seed, 0);
 * recompute the links. */
int hh_init_field_random(hh_ctx *ctx, uint64_t seed);

/* y = op(x) for op in {HH_OP_M, HH_OP_MT, HH_OP_MTM} (Eq. (10); Q = M^T M
 * as in Sec. 4.3).  x and y are device pointers of N elements of dtype
 * HH_DTYPE_F64 (links in FP64) or HH_DTYPE_F32 (links rounded to FP32); they
 * must not overlap.  Errors: HH_EINVAL. */
int hh_apply(hh_ctx *ctx, int op, const void *x, void *y, int dtype);

/* y_v = op(x_v) for n_vec vectors that share the context's field (Eq. (10);
 * Q = M^T M applied as M then M^T, Sec. 4.3): x_v = x + v N and y_v = y + v N
 * elements of dtype, v = 0 .. n_vec-1, stored back to back.  Equivalent to
 * n_vec calls of hh_apply.  For op = HH_OP_MTM in FP32 on d = 3 lattices with
 * 4 | Nx <= 32 (and 16-byte aligned x, y) the n_vec >= 2 vectors go through
 * one persistent launch that reads the links once: HBM traffic (8 n_vec + 4)
 * bytes per site, against 12 n_vec for separate applies.  Typical vectors:
 * the pseudofermion components of a trajectory, the noise vectors of
 * hh_observables, a block of right-hand sides.  x and y are device pointers
 * owned by the caller; the two ranges must not overlap.  Only enqueues work.
 * Errors: HH_EINVAL (NULL, n_vec < 1, bad op or dtype, overlap).  A bounded
 * device-side wait that ran out is reported by the next hh_counters_get
 * (HH_ETIMEOUT). */
int hh_apply_multi(hh_ctx *ctx, int op, const void *x, void *y, int n_vec, int dtype);

/* Solve Q x_a = b_a for a = 0..n_rhs-1 by CG with x0 = 0 (Sec. 4.1) in the
 * context's precision, all right-hand sides in one persistent launch.  With
 * cheb_degree = n > 0 the CG is preconditioned by the Chebyshev polynomial
 * P(Q) of Sec. 4.2, applied as n real quadratic factors (2n applications of
 * Q per step); info->iterations then counts preconditioned steps.
 * b, x: device pointers to n_rhs * N doubles.  info may be NULL (then the call
 * does not synchronise).  Returns HH_ENOCONV if a right-hand side missed
 * cg_tol within cg_maxit (x then holds the last iterate), HH_ETIMEOUT if a
 * bounded device-side wait ran out, HH_ENUMERIC on NaN/Inf. */
int hh_solve(hh_ctx *ctx, const double *b, double *x, int n_rhs, hh_solve_info *info);

/* As hh_solve, from the initial guess x0 held in x on entry: the engine first
 * computes the true residual b - Q x0 in FP64 (counted as a reliable update;
 * info->iterations is 0 if it already meets cg_tol), then runs CG from it.
 * b = 0 gives x = 0.  Used for chronological guesses in the molecular
 * dynamics (hh_params.chrono); not part of the paper's method, which starts
 * every solve from zero. */
int hh_solve_guess(hh_ctx *ctx, const double *b, double *x, int n_rhs, hh_solve_info *info);

/* F = dS_pf/dsigma for S_pf = 1/2 sum_a chi_a^T Q^{-1} chi_a: solves for
 * x_a = Q^{-1} chi_a, then F(n,tau) = -sum_a (M x_a)(n,tau+1) s(tau)
 * A cos sigma(n,tau) x_a(n,tau), s = -1 except +1 on the wrap link.
 * chi: device, n_rhs * N doubles; F: device, N doubles.  info may be NULL. */
int hh_force(hh_ctx *ctx, const double *chi, int n_rhs, double *F, hh_solve_info *info);

/* S_pf = 1/2 sum_a chi_a^T Q^{-1} chi_a (Eq. (12)) for the current sigma.
 * chi: device, n_rhs * N doubles; S: host double.  Synchronises. */
int hh_action(hh_ctx *ctx, const double *chi, int n_rhs, double *S, hh_solve_info *info);

/* One HMC trajectory of the phi-algorithm (Sec. 4.1) for trajectory number
 * traj_index: momenta pi ~ N(0,1) (Philox tag 1), pseudofermion sources
 * xi_a ~ N(0,1) (tag 2, component a in counter bits 8+), chi_a = M^T xi_a;
 * H0; leapfrog with n_md steps of size dt (n_md + 1 force evaluations);
 * H1; accept iff u < exp(-(H1 - H0)) with u the tag-3 uniform; on
 * rejection sigma is restored.  info may be NULL (then nothing synchronises).
 * Errors: HH_EINVAL (n_md < 1), solver errors as in hh_solve. */
int hh_trajectory(hh_ctx *ctx, int n_md, double dt, uint64_t traj_index, hh_traj_info *info);

/* Observables: noise estimators of the diagonal of M^{-1}.  For the block
 * form of Eq. (7) (link_order 1, 2) the diagonal blocks of M^{-1} are the
 * equal-time Green's functions (1 + B_tau ... B_{tau+1})^{-1}, so 1 -
 * M^{-1}_ii is the occupation of one spin state at site i and slice tau; for
 * reading R1 (link_order 0, M = e^{dtau K} times that form to first order)
 * the diagonal carries an O(dtau) admixture of the nearest-neighbour Green's
 * function.  The paper names no observables; these are the standard
 * stochastic estimators.
 *
 * n_noise (even, 2..64) Z2 vectors eta_k: element i is +1 when the top bit of
 * word i & 3 of Philox block i >> 2 (tag 6, a = k, trajectory traj, the
 * context's chain) is set, else -1.  y_k = M^{-1} eta_k = Q^{-1} M^T eta_k by
 * the context's solver (precision, preconditioner as set), in groups of at
 * most max(n_pf, 4) right-hand sides.  The field is the context's current
 * sigma.  Synchronises.  Errors: HH_EINVAL (out NULL, n_noise odd or out of
 * range), HH_ENOMEM, solver errors as in hh_solve. */
typedef struct {
    double trace_Minv;      /* mean over k of (1/N) eta_k . y_k: unbiased for (1/N) tr M^{-1} */
    double trace_err;       /* its standard error (sample deviation / sqrt(n_noise)) */
    double one_minus_g_sq;  /* (1/N) sum_i (1 - gA_i)(1 - gB_i), gA and gB the means of
                               eta_k(i) y_k(i) over the first and second half of the
                               vectors: unbiased for (1/N) sum_i (1 - M^{-1}_ii)^2, the
                               double occupancy when 1 - M^{-1}_ii is the occupation */
    double mean_sin;        /* (1/N) sum_i sin sigma_i */
    double mean_sin2;       /* (1/N) sum_i sin^2 sigma_i */
    int n_noise;
    int cg_iterations;      /* largest CG iteration count over the solve groups */
    double max_true_relres; /* largest true relative residual of the solves */
} hh_obs_info;

int hh_observables(hh_ctx *ctx, int n_noise, uint64_t traj, hh_obs_info *out);

/* Leapfrog only, on caller-owned fields: integrates (sigma_ctx, pi) for n_md
 * steps of size dt at fixed chi (device, n_rhs * N), updating the context's
 * sigma and the device array pi (N doubles) in place.  No Metropolis step. */
int hh_leapfrog(hh_ctx *ctx, double *pi, const double *chi, int n_rhs, int n_md, double dt,
                hh_solve_info *info);

/* Bound, in seconds, of every device-side wait of the context's kernels (the
 * persistent CG engine's waits for other blocks' partial sums, the
 * multi-vector apply's waits for its bulk copies); default 5.  A wait that
 * runs out makes the kernel record HH_ETIMEOUT and leave: hh_solve and the
 * calls built on it return HH_ETIMEOUT, an apply reports it at the next
 * hh_counters_get.  The context stays usable: every solve starts from a reset
 * engine state.  Errors: HH_EINVAL (seconds < 0 or > 3600). */
int hh_set_timeout(hh_ctx *ctx, double seconds);

/* Work counters of a context, for throughput and roofline accounting. */
typedef struct {
    long long kernel_launches; /* kernels this context launched since the last reset */
    long long engine_launches; /* persistent CG launches among them */
    double engine_ms;          /* summed CUDA-event time of those launches on the
                                  context stream (0 unless profiling was enabled) */
    long long cg_steps;        /* CG steps, summed over right-hand sides */
    long long ru_steps;        /* FP64 true-residual recomputations (checks and
                                  reliable updates), summed over right-hand sides */
    long long solves;          /* right-hand sides solved */
    long long fp64_steps;      /* CG steps run in FP64 (all of them in HH_FP64;
                                  in HH_MIXED, the steps after a stalled system
                                  switched to FP64) */
    long long sites;           /* N of the context's lattice */
} hh_counters;

/* Zero the counters and clear a device-side error recorded by an apply.
 * profile_engine = 1 records a CUDA event pair around every persistent CG
 * launch (on the context stream) until the next reset. */
int hh_counters_reset(hh_ctx *ctx, int profile_engine);

/* Read the counters; synchronises the context stream.  Returns HH_ETIMEOUT
 * if an apply since the last reset recorded a bounded wait that ran out (the
 * counters are filled all the same). */
int hh_counters_get(hh_ctx *ctx, hh_counters *out);

/* ---- Batched multi-chain engine and serving loop ---------------------------
 * Many independent Markov chains and solves, of different lattices, share one
 * persistent CG launch (an extension: the paper's Sec. 5 runs one lattice at
 * a time).  Requests are admitted into slots
 * while the HBM budget and the active-site window allow, each slot's state
 * stays resident on the device, and the engine advances every active system
 * by 'chunk_iters' CG iterations per launch (a CUDA-graph replay).  Between
 * launches the host retires finished solves, advances trajectories through
 * their leapfrog stages (force, sigma step, next solve, Metropolis) and admits
 * queued requests, so work that arrives while others run joins at the next
 * chunk (continuous batching).  Every system is tiled by its own size only and
 * reduced in a fixed order, so its bits do not depend on the other requests
 * in the mix. */
#define HH_REQ_SOLVE 0
#define HH_REQ_TRAJECTORY 1

typedef struct hh_batch hh_batch;

typedef struct {
    int kind;            /* HH_REQ_SOLVE or HH_REQ_TRAJECTORY */
    hh_lattice lat;
    hh_params prm;       /* as for hh_create; for a solve, n_pf is the number of
                            right-hand sides (1..4); cheb_degree > 0 (FP64 only)
                            preconditions the request's solves as in hh_solve;
                            precision HH_FP64 or HH_MIXED (the 16-bit link
                            precisions and link_order != 0 are for contexts
                            only: HH_EINVAL) */
    const double *sigma; /* host, N doubles, copied at submit; NULL: sigma from
                            Philox tag 0 with prm.seed (as hh_init_field_random) */
    const double *b;     /* solve: host, n_pf*N doubles copied at submit; NULL:
                            N(0,1) sources (Philox tag 2, trajectory word traj_index) */
    double *out;         /* host, written on completion (x for a solve, n_pf*N
                            doubles; sigma after Metropolis for a trajectory, N
                            doubles); NULL: not written.  Owned by the caller and
                            kept alive until the result has been polled. */
    int n_md;            /* trajectory: leapfrog steps */
    double dt;           /* trajectory: step size */
    uint64_t traj_index; /* trajectory number (Philox counter word) */
} hh_request;

typedef struct {
    uint64_t ticket;
    int kind;
    int status;             /* HH_OK or an error code of the request */
    int cg_iterations;      /* summed over the request's solves and right-hand sides */
    int reliable_updates;
    int n_solves;
    double max_true_relres;
    double H0, H1, dH, u;   /* trajectory only */
    int accepted;
    double queue_ms;        /* submit -> admitted into a slot */
    double latency_ms;      /* submit -> result ready */
} hh_result;

typedef struct {
    int max_slots;           /* concurrent requests on the device (<= 256) */
    size_t hbm_budget_bytes; /* device memory for slots (arena allocated at create) */
    int chunk_iters;         /* CG iterations per engine launch */
    int tile_sites;          /* sites per tile (multiple of 32) */
    long long max_active_sites; /* admission window on summed active sites (0: none) */
} hh_batch_config;

/* Defaults: 64 slots, 4 GiB, 32 iterations per chunk, 4096-site tiles, no window. */
void hh_batch_default_config(hh_batch_config *cfg);

/* Create a batch engine on the current device and stream.  Allocates the
 * slot arena (hbm_budget_bytes) and the engine tables.  Errors: HH_EINVAL,
 * HH_ENOMEM, HH_ECUDA. */
int hh_batch_create(hh_batch **out, const hh_batch_config *cfg, void *cuda_stream);

/* Stop the worker (if running), free everything.  NULL is accepted. */
int hh_batch_destroy(hh_batch *b);

/* Queue a request (thread safe, non-blocking); host arrays are copied now.
 * Returns HH_EBUSY if the request alone needs more than the whole budget,
 * HH_EINVAL for bad shapes. */
int hh_batch_submit(hh_batch *b, const hh_request *req, uint64_t *ticket);

/* One scheduling round on the calling thread: admit, run one engine chunk,
 * advance or retire requests.  *n_busy (may be NULL) receives queued + active
 * requests.  Must not be called while the worker thread runs. */
int hh_batch_step(hh_batch *b, int *n_busy);

/* Bound, in seconds, of every device-side wait of the batch engine's
 * launches (default 5; thread safe, read at each launch).  A launch whose wait
 * runs out fails the requests on the device with HH_ETIMEOUT; requests
 * admitted afterwards start from empty signal slots.  Errors: HH_EINVAL. */
int hh_batch_set_timeout(hh_batch *b, double seconds);

/* Run scheduling rounds on a background thread until hh_batch_stop. */
int hh_batch_start(hh_batch *b);
int hh_batch_stop(hh_batch *b);

/* Move up to max finished results into out (thread safe). */
int hh_batch_poll(hh_batch *b, hh_result *out, int max, int *n_done);

/* Requests waiting for a slot and requests on the device. */
int hh_batch_pending(hh_batch *b, int *queued, int *active);

/* Autotuner: time each candidate configuration (tile size, chunk length,
 * active-site window) on copies of the given solve requests for 'rounds'
 * scheduling rounds, return the fastest in *best (CG site-iterations per
 * second), and, if cache_path is not NULL, record it as a JSON line keyed by
 * the request mix.  Uses a scratch batch of the given budget. */
int hh_batch_autotune(const hh_request *sample, int n, size_t hbm_budget_bytes, int rounds,
                      const char *cache_path, void *cuda_stream, hh_batch_config *best);

/* ---- Time-slab decomposition over several ranks ---------------------------
 * One lattice split by time slices over R ranks (processes, typically one GPU
 * each): rank r owns slices [tau0, tau1) of every vector.  M couples slice tau
 * to tau - 1 and M^T couples it to tau + 1 (Eq. (10)), so an apply of M needs
 * the previous rank's last slice of x, an apply of M^T the next rank's first
 * slice of t = M x, and CG (Sec. 4.1) two global sums per iteration.  The
 * sign of the antiperiodic wrap link N_tau - 1 -> 0 follows the global slice
 * index, so it stays with the rank owning slice N_tau - 1.  Ranks form a ring:
 * the rank owning slice 0 has the rank owning N_tau - 1 as its previous one.
 *
 * The library is communication-agnostic: the caller supplies the callbacks
 * of hh_comm, which move halo slices and sums between kernel launches (no
 * kernel ever waits for another rank).  Each returns 0 on success (any other
 * value: HH_ECUDA).  Two forms; a slab uses the device form when both of its
 * callbacks are set, else the host form:
 *   host form, called after the slab's stream has been synchronised, on host
 *   buffers, complete on return:
 *   exchange(user, dir, send, recv, bytes): dir = +1: send the host buffer
 *     send (bytes) to the next rank and receive the previous rank's into recv;
 *     dir = -1: send to the previous rank and receive from the next.  With
 *     one rank, copy send into recv.
 *   allreduce_sum(user, vals, n): replace the n host doubles by their sums
 *     over all ranks.
 *   device form, on device buffers (the slab's own slices and scalars): the
 *   callback enqueues the transfer on cuda_stream (the slab's stream) and may
 *   return before it completes, e.g. NCCL send/recv and all-reduce on that
 *   stream or peer copies staged into the receiving slab's buffer; the slab
 *   then runs its CG iterations without synchronising, with the CG scalars on
 *   the device, and reads them every few iterations to test convergence.
 *   exchange_device(user, dir, send, recv, bytes, cuda_stream): as exchange.
 *   allreduce_sum_device(user, vals, n, cuda_stream): as allreduce_sum.
 *   The slab records its first full batch of iterations into a CUDA graph
 *   (stream capture of cuda_stream, unless it is the legacy default stream)
 *   and replays it; a device callback that cannot be captured must return
 *   non-zero before enqueuing anything when the stream is capturing, and the
 *   slab then launches its iterations directly. */
typedef struct hh_slab hh_slab;

typedef struct {
    int (*exchange)(void *user, int dir, const void *send, void *recv, size_t bytes);
    int (*allreduce_sum)(void *user, double *vals, int n);
    void *user;
    int (*exchange_device)(void *user, int dir, const void *send, void *recv, size_t bytes, void *cuda_stream);
    int (*allreduce_sum_device)(void *user, double *vals, int n, void *cuda_stream);
} hh_comm;

/* Slab of slices [tau0, tau1) of the lattice lat (FP64 only, link_order 0,
 * no preconditioner).  Allocates the slab's field, links and work vectors on
 * the current device; stream: cudaStream_t (NULL: legacy default stream).
 * Errors: HH_EINVAL (shapes, empty slab, neither callback form complete,
 * other precision), HH_ENOMEM, HH_ECUDA. */
int hh_slab_create(hh_slab **out, const hh_lattice *lat, const hh_params *p, int tau0, int tau1,
                   const hh_comm *comm, void *cuda_stream);
int hh_slab_destroy(hh_slab *s);

/* The slab's part of sigma: (tau1 - tau0) * V doubles (slice tau0 first),
 * device (on_device = 1) or host memory; exchanges the slice before tau0 with
 * the previous rank (collective: every rank calls it) and computes the links.
 * Synchronises. */
int hh_slab_set_field(hh_slab *s, const double *sigma, int on_device);

/* y = op(x) on the slab's slices, op in {HH_OP_M, HH_OP_MT, HH_OP_MTM}; x and
 * y: device pointers to (tau1 - tau0) * V doubles.  Collective.  Synchronises. */
int hh_slab_apply(hh_slab *s, int op, const double *x, double *y);

/* Q x = b by FP64 CG over all ranks, x0 = 0, stopping on the global true
 * residual ||b - Q x|| <= cg_tol ||b|| as hh_solve; b, x: device pointers to
 * the slab's part.  Collective.  info (may be NULL): iterations, true-residual
 * checks (reliable_updates), final true relative residual, converged flag.
 * Returns HH_ENOCONV at the iteration cap, HH_ENUMERIC on a non-finite or
 * non-positive <p, Q p>. */
int hh_slab_solve(hh_slab *s, const double *b, double *x, hh_solve_info *info);

/* ---- Debug build: index checks ---------------------------------------------
 * Not part of the method.  A library compiled with -DHH_BOUNDS_CHECK
 * (libhubhmc_check.so, built by build(bounds_check=True); the Python binding
 * loads it when HH_BOUNDS_CHECK=1) checks the neighbour indices of every
 * stencil (scalar and W-site groups, the shifts by one time slice), the tile
 * ranges of the CG engine and the source ranges of the multi-vector apply's
 * bulk copies.  An index outside its range is recorded in a device error word
 * (the first per translation unit) and replaced by an in-range one, so no
 * access leaves its buffer and nothing traps; results are then wrong and the
 * record says where.
 *   op: HH_BOUNDS_READ reads and clears the records; HH_BOUNDS_SELFTEST first
 *       runs a one-thread kernel whose check of an index past its range must
 *       fail (nothing is accessed), then reads and clears (synchronises the
 *       device).
 *   enabled (may be NULL): 1 in the checked build, 0 otherwise.
 *   record (may be NULL): the first record, (check code << 32) | index, or 0.
 * Returns HH_EBOUNDS if a check failed since the last read, HH_OK otherwise
 * (always HH_OK in the default build), HH_ECUDA if the device cannot be read. */
#define HH_EBOUNDS (-9)     /* an index check of the debug build failed */
#define HH_BOUNDS_READ 0
#define HH_BOUNDS_SELFTEST 1
int hh_bounds_check(int op, int *enabled, long long *record);

/* ---- Allocation-free solve ------------------------------------------------
 * The paper has no counterpart of this entry point; it exists for callers
 * that cannot allocate memory when they need a solve: plug-ins inside
 * applications that own the device allocator, and loops that must not take
 * allocator locks.  Everything the FP64 CG needs beyond the
 * caller's sigma, b and x lives in one file-scope device array of
 * HH_NOALLOC_SCRATCH_MB (about 9 MiB), which every device that loads the
 * library keeps until the process exits.
 *
 * hh_solve_noalloc solves Q x = b, Q = M^T M with M built from sigma and the
 * parameters t, dtau, A of p exactly as for a context (link_order 0), by FP64
 * CG with x0 = 0 and one right-hand side: the same algorithm and stopping
 * test (true relative residual <= cg_tol) as hh_solve.
 *   lat, p:  lattice and parameters; p->precision must be HH_FP64, and
 *            N = Nx^d * Ntau must not exceed HH_NOALLOC_MAX_SITES, else the
 *            call returns HH_ESIZE without touching the device.
 *   sigma, b, x: device pointers to N doubles owned by the caller.
 *   cuda_stream: the cudaStream_t to run on (NULL: legacy default stream).
 *   info: if non-NULL the call synchronises the stream and fills it, and
 *            returns the solve's status (HH_ENOCONV, HH_ETIMEOUT, HH_ENUMERIC).
 *            A non-NULL info on a stream in capture mode is refused with
 *            HH_EINVAL (the synchronisation is not allowed there).  With info
 *            NULL the call only enqueues the work and returns HH_OK: the
 *            solve's outcome is not reported, and the next call overwrites
 *            it in the shared array.
 * Every call looks up the array's device address, which stays valid if the
 * caller resets the device; the first call on a device also queries the
 * kernel's occupancy (which allocates nothing).
 * The call allocates no device or host memory.  All calls share the array and
 * overwrite it (the call clears what must start at zero); calls whose GPU work
 * overlaps in time race on it and must be serialised by the caller. */
#define HH_ESIZE (-8) /* problem larger than the static scratch of hh_solve_noalloc */
#define HH_NOALLOC_MAX_SITES 262144
#define HH_NOALLOC_SCRATCH_MB 9
int hh_solve_noalloc(const hh_lattice *lat, const hh_params *p, const double *sigma,
                     const double *b, double *x, void *cuda_stream, hh_solve_info *info);

/* Text for an error code. */
const char *hh_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* HUBHMC_H */
