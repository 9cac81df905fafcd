// Time-slab decomposition of one lattice over several ranks (processes, one
// GPU each): rank r owns the time slices [tau0, tau1) of every vector, the
// links out of them and one halo slice on each side.  M couples slice tau to
// tau - 1 and M^T to tau + 1 (Eq. (10)), so an apply of M needs the previous
// rank's last slice of x and an apply of M^T the next rank's first slice of
// t = M x; CG adds two global sums per iteration (Sec. 4.1).  The antiperiodic
// sign of the wrap link N_tau - 1 -> 0 is taken from the global slice index, so
// it stays with the rank that owns slice N_tau - 1.
//
// The library is communication-agnostic: the caller supplies callbacks
// (hh_comm) that exchange a time slice with the neighbouring ranks and sum a
// few doubles over all ranks, between kernel launches; no kernel ever waits
// for another rank.  Host form: the library synchronises its stream, stages
// the slice through pinned host memory and calls the exchange; the CG
// scalars live on the host.  Device form: the callbacks enqueue the transfers
// on the slab's stream (NCCL or peer copies) straight into the halo slots;
// the CG scalars (dot products, alpha, beta, convergence) stay on the device,
// each iteration is a sequence of launches with no synchronisation, and the
// host reads the scalars every kCheckEvery iterations.


//
// Layout of a slab vector: nl = tau1 - tau0 own slices; the library's device
// vectors carry nl + 2 slices (halo before, own, halo after), so the standard
// stencil sweeps run unchanged on an extended lattice of nl + 2 slices and
// their results are kept on the own slices only.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/hubhmc.h"
#include "hh_apply.cuh"
#include "hh_kernels.cuh"
#include "hh_trace.cuh"

using namespace hh;

namespace {

constexpr int kRedBlock = 256;

// L_ext(e) for extended slice e (global slice (tau0 - 1 + e) mod N_tau):
// the link out of that slice, -(1 + A sin sigma) except +(1 + A sin sigma) on
// the wrap link out of slice N_tau - 1.
__global__ void k_slab_links(int V, int ne, int tau_first, int ntau, double A, const double *sigma_ext,
                             double *L_ext)
{
    const long long n = (long long)V * ne;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(i / V);
        int g = (tau_first + e) % ntau;
        if (g < 0) g += ntau;
        const double s = (g == ntau - 1) ? 1.0 : -1.0;
        L_ext[i] = s * (1.0 + A * sin(sigma_ext[i]));
    }
}

// Block partials of sum_i a_i b_i over [0, n) in a fixed order.
__global__ void k_slab_dot(const double *a, const double *b, long long n, double *part)
{
    __shared__ double red[kRedBlock];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc = fma(a[i], b[i], acc);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kRedBlock / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_slab_sum(const double *part, int nb, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int j = 0; j < nb; ++j) s += part[j];
        *out = s;
    }
}

// x += alpha p, r -= alpha q over [0, n).
__global__ void k_slab_update(double *x, const double *p, double *r, const double *q, double alpha, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        r[i] = fma(-alpha, q[i], r[i]);
    }
}

// p = r + beta p over [0, n).
__global__ void k_slab_direction(double *p, const double *r, double beta, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], r[i]);
}

// out = a - b over [0, n).
__global__ void k_slab_sub(double *out, const double *a, const double *b, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = a[i] - b[i];
}

// CG scalars of the device form.
struct SlabScalars {
    double bb, rr, pq, rr_new, tol2;
    int done;   // the recursive residual met the tolerance: the vector kernels leave the vectors alone
    int bad;    // a non-finite or non-positive <p, Q p> or |r|^2 was met
    int it;     // CG iterations run
};

constexpr int kCheckEvery = 8;   // device form: iterations between host reads of the scalars

// Block sums of a block's values, written to part[blockIdx.x]; the last block
// to finish adds the partials in block order (so the result does not depend
// on timing), stores the total in *out and resets the counter.
__device__ void block_total(double acc, double *part, unsigned *count, double *out)
{
    __shared__ double red[kRedBlock];
    __shared__ bool last;
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = kRedBlock / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = red[0];
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double t = 0.0;
        for (unsigned j = 0; j < gridDim.x; ++j) t += ((volatile double *)part)[j];
        *out = t;
        *count = 0;
    }
}

// *out = sum_i a_i b_i over [0, n) (skipped once the solve is done, if sc).
__global__ void k_dev_dot(const double *a, const double *b, long long n, double *part, unsigned *count, double *out,
                          const SlabScalars *sc)
{
    if (sc && (sc->done || sc->bad)) return;
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc = fma(a[i], b[i], acc);
    block_total(acc, part, count, out);
}

// alpha = rr / <p, Q p>; x += alpha p, r -= alpha q; rr_new = |r|^2 (local).
__global__ void k_dev_update(double *x, const double *p, double *r, const double *q, long long n, SlabScalars *sc,
                             double *part, unsigned *count)
{
    if (sc->done || sc->bad) return;
    const double pq = sc->pq;
    if (!(pq > 0.0) || !isfinite(pq)) {   // every block takes this branch alike
        if (blockIdx.x == 0 && threadIdx.x == 0) sc->bad = 1;
        return;
    }
    const double alpha = sc->rr / pq;
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
    }
    block_total(acc, part, count, &sc->rr_new);
}

// End of an iteration: p = r + (rr_new / rr) p unless the new residual meets
// the tolerance; then the last block to finish (every block has read the
// scalars by then) counts the iteration, sets rr = rr_new and tests the
// recursive residual.
__global__ void k_dev_direction(double *p, const double *r, long long n, SlabScalars *sc, unsigned *count)
{
    const bool live = !(sc->done || sc->bad);
    const double rn = sc->rr_new, tol2 = sc->tol2;
    if (live && rn > tol2 && isfinite(rn)) {
        const double beta = rn / sc->rr;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x)
            p[i] = fma(beta, p[i], r[i]);
    }
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        if (live) {
            sc->it += 1;
            if (!isfinite(rn)) {
                sc->bad = 1;
            } else {
                sc->rr = rn;
                if (rn <= tol2) sc->done = 1;
            }
        }
        *count = 0;
    }
}

// Start (or restart from the true residual rr_true = *rr_src): rr, tol2, flags.
__global__ void k_dev_start(SlabScalars *sc, double tol, int first)
{
    if (first) {
        sc->tol2 = tol * tol * sc->bb;
        sc->rr = sc->bb;
        sc->it = 0;
        sc->done = sc->bb == 0.0 ? 1 : 0;
    } else {
        sc->rr = sc->rr_new;
        sc->done = 0;
    }
    sc->bad = 0;
}

}  // namespace

struct hh_slab {
    hh_lattice lat;
    hh_params prm;
    hh_comm comm;
    cudaStream_t stream;
    int tau0, tau1, nl, V;
    long long own;           // V * nl
    Geo gext;                // the lattice of nl + 2 slices the sweeps run on
    double *sigma_ext, *L_ext;
    double *xe, *te, *pe;    // extended work vectors (nl + 2 slices)
    double *r, *q, *xs;      // own-slice CG vectors (q: the own slices of pe, the M^T sweep's output)
    double *part, *dsum;
    double *h_stage;         // pinned: 2 slices (send, receive) + scalars
    int nb;
    int dev_mode;            // the device form of the callbacks
    SlabScalars *sc;         // device form: the CG scalars
    unsigned *count;         // device form: block counter of the last-block sums
    // device form: kCheckEvery iterations as one CUDA graph (captured at the
    // first full batch; 0 not tried, 1 captured, -1 capture failed: launch
    // the iterations one by one)
    int graph_state;
    cudaGraphExec_t graph;
};

namespace {

#define HS_TRY(expr)                             \
    do {                                         \
        cudaError_t e__ = (expr);                \
        if (e__ != cudaSuccess) return HH_ECUDA; \
    } while (0)

int grid_for(long long n)
{
    long long b = (n + 255) / 256;
    if (b > 1216) b = 1216;
    return b < 1 ? 1 : (int)b;
}

// Exchange of one slice: dir = +1 sends send_dev (V doubles) to the next rank
// and receives the previous rank's slice into recv_dev; dir = -1 the other way.
int exchange_slice(hh_slab *s, int dir, const double *send_dev, double *recv_dev)
{
    TraceRange tr(dir > 0 ? "hh slab halo +1" : "hh slab halo -1");
    const size_t bytes = sizeof(double) * (size_t)s->V;
    if (s->dev_mode)   // enqueued on the stream, straight into the halo slot
        return s->comm.exchange_device(s->comm.user, dir, send_dev, recv_dev, bytes, (void *)s->stream) ? HH_ECUDA
                                                                                                       : HH_OK;
    double *hs = s->h_stage, *hr = s->h_stage + s->V;
    HS_TRY(cudaMemcpyAsync(hs, send_dev, bytes, cudaMemcpyDeviceToHost, s->stream));
    HS_TRY(cudaStreamSynchronize(s->stream));
    if (s->comm.exchange(s->comm.user, dir, hs, hr, bytes) != 0) return HH_ECUDA;
    HS_TRY(cudaMemcpyAsync(recv_dev, hr, bytes, cudaMemcpyHostToDevice, s->stream));
    return HH_OK;
}

// Global sum of the dot products of n own-slice pairs: local partials on the
// device, then the caller's all-reduce on the host.
int global_dots(hh_slab *s, const double *const *a, const double *const *b, int n, double *out)
{
    for (int k = 0; k < n; ++k) {
        k_slab_dot<<<s->nb, kRedBlock, 0, s->stream>>>(a[k], b[k], s->own, s->part);
        k_slab_sum<<<1, 32, 0, s->stream>>>(s->part, s->nb, s->dsum + k);
    }
    HS_TRY(cudaGetLastError());
    double *hv = s->h_stage + 2 * (size_t)s->V;
    HS_TRY(cudaMemcpyAsync(hv, s->dsum, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
    HS_TRY(cudaStreamSynchronize(s->stream));
    if (s->comm.allreduce_sum(s->comm.user, hv, n) != 0) return HH_ECUDA;
    for (int k = 0; k < n; ++k) out[k] = hv[k];
    return HH_OK;
}

// q (own slices) = op(x) for x given on the own slices of the extended
// vector xe (its halo slices are filled here).  op: HH_OP_M, HH_OP_MT, HH_OP_MTM.
int slab_apply_ext(hh_slab *s, int op, double *q_own)
{
    const double h = s->prm.t * s->prm.dtau;
    const size_t V = (size_t)s->V;
    double *xe_own = s->xe + V;
    if (op == HH_OP_M || op == HH_OP_MTM) {
        // previous rank's last slice of x into the halo before
        int rc = exchange_slice(s, +1, s->xe + V * s->nl, s->xe);
        if (rc) return rc;
        HS_TRY(launch_sweep_f64(s->gext, false, h, s->L_ext, s->xe, s->te, s->stream));
        if (op == HH_OP_M) {
            HS_TRY(cudaMemcpyAsync(q_own, s->te + V, sizeof(double) * s->own, cudaMemcpyDeviceToDevice, s->stream));
            return HH_OK;
        }
    } else {
        HS_TRY(cudaMemcpyAsync(s->te + V, xe_own, sizeof(double) * s->own, cudaMemcpyDeviceToDevice, s->stream));
    }
    // next rank's first slice of t into the halo after
    int rc = exchange_slice(s, -1, s->te + V, s->te + V * (s->nl + 1));
    if (rc) return rc;
    HS_TRY(launch_sweep_f64(s->gext, true, h, s->L_ext, s->te, s->pe, s->stream));
    if (q_own != s->pe + V)
        HS_TRY(cudaMemcpyAsync(q_own, s->pe + V, sizeof(double) * s->own, cudaMemcpyDeviceToDevice, s->stream));
    return HH_OK;
}

void free_slab(hh_slab *s)
{
    for (double *p : {s->sigma_ext, s->L_ext, s->xe, s->te, s->pe, s->r, s->xs, s->part, s->dsum})
        if (p) cudaFree(p);
    if (s->sc) cudaFree(s->sc);
    if (s->count) cudaFree(s->count);
    if (s->graph) cudaGraphExecDestroy(s->graph);
    if (s->h_stage) cudaFreeHost(s->h_stage);
}

// k iterations of the device-form CG, enqueued on the slab's stream.
int enqueue_iterations(hh_slab *s, int k)
{
    const size_t V = (size_t)s->V;
    const long long n = s->own;
    const int g = s->nb;
    double *p = s->xe + V;
    SlabScalars *sc = s->sc;
    for (int j = 0; j < k; ++j) {
        int rc = slab_apply_ext(s, HH_OP_MTM, s->q);
        if (rc) return rc;
        k_dev_dot<<<g, kRedBlock, 0, s->stream>>>(p, s->q, n, s->part, s->count, &sc->pq, sc);
        if (s->comm.allreduce_sum_device(s->comm.user, &sc->pq, 1, (void *)s->stream) != 0) return HH_ECUDA;
        k_dev_update<<<g, kRedBlock, 0, s->stream>>>(s->xs, p, s->r, s->q, n, sc, s->part, s->count);
        if (s->comm.allreduce_sum_device(s->comm.user, &sc->rr_new, 1, (void *)s->stream) != 0) return HH_ECUDA;
        k_dev_direction<<<g, kRedBlock, 0, s->stream>>>(p, s->r, n, sc, s->count);
    }
    HS_TRY(cudaGetLastError());
    return HH_OK;
}

// A batch of kCheckEvery iterations: replayed from a CUDA graph once one has
// been captured (the iterations' pointers are fixed per slab and their
// scalars live on the device, so the graph serves every later batch and
// solve).  The capture is tried once, on a stream of the caller's (not the
// legacy default stream); if it fails the iterations are launched directly.
int run_batch(hh_slab *s)
{
    if (s->graph_state == 0 && s->stream != nullptr) {
        s->graph_state = -1;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
            const int rc = enqueue_iterations(s, kCheckEvery);
            const cudaError_t e = cudaStreamEndCapture(s->stream, &g);
            if (rc == HH_OK && e == cudaSuccess && g &&
                cudaGraphInstantiate(&s->graph, g, 0) == cudaSuccess)
                s->graph_state = 1;
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();
    }
    if (s->graph_state == 1) {
        HS_TRY(cudaGraphLaunch(s->graph, s->stream));
        return HH_OK;
    }
    return enqueue_iterations(s, kCheckEvery);
}

// Device form of the CG of hh_slab_solve: no synchronisation inside an
// iteration; the host reads the scalars every kCheckEvery iterations.
int slab_solve_device(hh_slab *s, const double *b, double *x, hh_solve_info *info)
{
    const size_t V = (size_t)s->V;
    const long long n = s->own;
    const int g = s->nb;
    double *p = s->xe + V;
    SlabScalars *sc = s->sc;
    HS_TRY(cudaMemsetAsync(s->xs, 0, sizeof(double) * n, s->stream));
    HS_TRY(cudaMemcpyAsync(s->r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream));
    HS_TRY(cudaMemcpyAsync(p, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream));
    k_dev_dot<<<g, kRedBlock, 0, s->stream>>>(b, b, n, s->part, s->count, &sc->bb, nullptr);
    HS_TRY(cudaGetLastError());
    if (s->comm.allreduce_sum_device(s->comm.user, &sc->bb, 1, (void *)s->stream) != 0) return HH_ECUDA;
    k_dev_start<<<1, 1, 0, s->stream>>>(sc, s->prm.cg_tol, 1);
    HS_TRY(cudaGetLastError());
    SlabScalars *hs = reinterpret_cast<SlabScalars *>(s->h_stage + 2 * V);
    auto read = [&]() -> int {
        HS_TRY(cudaMemcpyAsync(hs, sc, sizeof(SlabScalars), cudaMemcpyDeviceToHost, s->stream));
        HS_TRY(cudaStreamSynchronize(s->stream));
        return HH_OK;
    };
    int rc = read();
    if (rc) return rc;
    const double bb = hs->bb;
    int status = HH_OK, n_true = 0;
    double true_rel = bb > 0.0 ? 1.0 : 0.0;
    bool done = bb == 0.0;
    while (!done) {
        if (hs->bad) {
            status = HH_ENUMERIC;
            break;
        }
        if (!hs->done) {
            if (hs->it >= s->prm.cg_maxit) {
                status = HH_ENOCONV;
                break;
            }
            const int k = s->prm.cg_maxit - hs->it < kCheckEvery ? s->prm.cg_maxit - hs->it : kCheckEvery;
            rc = k == kCheckEvery ? run_batch(s) : enqueue_iterations(s, k);
            if (rc) return rc;
            rc = read();
            if (rc) return rc;
            continue;
        }
        // The recursive residual met the tolerance: confirm with the true
        // residual b - Q x, and continue from it if it is not met.
        HS_TRY(cudaMemcpyAsync(s->xe + V, s->xs, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream));
        rc = slab_apply_ext(s, HH_OP_MTM, s->q);
        if (rc) return rc;
        k_slab_sub<<<g, 256, 0, s->stream>>>(s->r, b, s->q, n);
        k_dev_dot<<<g, kRedBlock, 0, s->stream>>>(s->r, s->r, n, s->part, s->count, &sc->rr_new, nullptr);
        HS_TRY(cudaGetLastError());
        if (s->comm.allreduce_sum_device(s->comm.user, &sc->rr_new, 1, (void *)s->stream) != 0) return HH_ECUDA;
        rc = read();
        if (rc) return rc;
        ++n_true;
        true_rel = std::sqrt(hs->rr_new / bb);
        if (hs->rr_new <= hs->tol2) {
            done = true;
            break;
        }
        HS_TRY(cudaMemcpyAsync(p, s->r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream));
        k_dev_start<<<1, 1, 0, s->stream>>>(sc, s->prm.cg_tol, 0);
        HS_TRY(cudaGetLastError());
        rc = read();
        if (rc) return rc;
    }
    HS_TRY(cudaMemcpyAsync(x, s->xs, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream));
    HS_TRY(cudaStreamSynchronize(s->stream));
    if (info) {
        info->iterations = hs->it;
        info->reliable_updates = n_true;
        info->true_relres = true_rel;
        info->converged = (done && status == HH_OK) ? 1 : 0;
    }
    return status;
}

}  // namespace

extern "C" {

int hh_slab_create(hh_slab **out, const hh_lattice *lat, const hh_params *p, int tau0, int tau1,
                   const hh_comm *comm, void *cuda_stream)
{
    if (!out || !lat || !p || !comm) return HH_EINVAL;
    const bool dev_form = comm->exchange_device && comm->allreduce_sum_device;
    if (!dev_form && !(comm->exchange && comm->allreduce_sum)) return HH_EINVAL;
    *out = nullptr;
    if (lat->d != 1 && lat->d != 3) return HH_EINVAL;
    if (lat->nx < 2 || lat->ntau < 2 || tau0 < 0 || tau1 > lat->ntau || tau1 - tau0 < 1) return HH_EINVAL;
    if (p->precision != HH_FP64 || p->link_order != 0 || p->cheb_degree != 0) return HH_EINVAL;
    if (!(p->cg_tol > 0.0) || p->cg_maxit < 1) return HH_EINVAL;
    const long long V = lat->d == 1 ? lat->nx : (long long)lat->nx * lat->nx * lat->nx;
    const long long ne = tau1 - tau0 + 2;
    if (V * ne >= (1LL << 31) - 1024) return HH_EINVAL;
    hh_slab *s = new (std::nothrow) hh_slab;
    if (!s) return HH_ENOMEM;
    memset(s, 0, sizeof(*s));
    s->lat = *lat;
    s->prm = *p;
    s->comm = *comm;
    s->stream = (cudaStream_t)cuda_stream;
    s->tau0 = tau0;
    s->tau1 = tau1;
    s->nl = tau1 - tau0;
    s->V = (int)V;
    s->own = V * s->nl;
    s->gext = make_geo(lat->d, lat->nx, (int)ne);
    s->nb = grid_for(s->own) < 512 ? grid_for(s->own) : 512;
    s->dev_mode = dev_form ? 1 : 0;
    const size_t ext = (size_t)(V * ne);
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&s->sigma_ext, sizeof(double) * ext);
    if (e == cudaSuccess) e = cudaMalloc(&s->L_ext, sizeof(double) * ext);
    if (e == cudaSuccess) e = cudaMalloc(&s->xe, sizeof(double) * ext);
    if (e == cudaSuccess) e = cudaMalloc(&s->te, sizeof(double) * ext);
    if (e == cudaSuccess) e = cudaMalloc(&s->pe, sizeof(double) * ext);
    if (e == cudaSuccess) e = cudaMalloc(&s->r, sizeof(double) * s->own);

    if (e == cudaSuccess) e = cudaMalloc(&s->xs, sizeof(double) * s->own);
    if (e == cudaSuccess) e = cudaMalloc(&s->part, sizeof(double) * 512);
    if (e == cudaSuccess) e = cudaMalloc(&s->dsum, sizeof(double) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&s->sc, sizeof(SlabScalars));
    if (e == cudaSuccess) e = cudaMalloc(&s->count, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemsetAsync(s->count, 0, sizeof(unsigned), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->sc, 0, sizeof(SlabScalars), s->stream);
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_stage, sizeof(double) * (2 * (size_t)V + 16));
    if (e == cudaSuccess) s->q = s->pe + V;
    if (e == cudaSuccess) e = cudaMemsetAsync(s->sigma_ext, 0, sizeof(double) * ext, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->xe, 0, sizeof(double) * ext, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->te, 0, sizeof(double) * ext, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        free_slab(s);
        delete s;
        return e == cudaErrorMemoryAllocation ? HH_ENOMEM : HH_ECUDA;
    }
    *out = s;
    return HH_OK;
}

int hh_slab_destroy(hh_slab *s)
{
    if (!s) return HH_OK;
    cudaStreamSynchronize(s->stream);
    free_slab(s);
    delete s;
    return HH_OK;
}

int hh_slab_set_field(hh_slab *s, const double *sigma, int on_device)
{
    if (!s || !sigma) return HH_EINVAL;
    const size_t V = (size_t)s->V;
    HS_TRY(cudaMemcpyAsync(s->sigma_ext + V, sigma, sizeof(double) * s->own,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream));
    // the previous rank's last slice of sigma carries the link into tau0
    int rc = exchange_slice(s, +1, s->sigma_ext + V * s->nl, s->sigma_ext);
    if (rc) return rc;
    const int ne = s->nl + 2;
    k_slab_links<<<grid_for(V * ne), 256, 0, s->stream>>>(s->V, ne, s->tau0 - 1, s->lat.ntau, s->prm.A,
                                                         s->sigma_ext, s->L_ext);
    HS_TRY(cudaGetLastError());
    HS_TRY(cudaStreamSynchronize(s->stream));
    return HH_OK;
}

int hh_slab_apply(hh_slab *s, int op, const double *x, double *y)
{
    if (!s || !x || !y) return HH_EINVAL;
    if (op != HH_OP_M && op != HH_OP_MT && op != HH_OP_MTM) return HH_EINVAL;
    HS_TRY(cudaMemcpyAsync(s->xe + s->V, x, sizeof(double) * s->own, cudaMemcpyDeviceToDevice, s->stream));
    int rc = slab_apply_ext(s, op, y);
    if (rc) return rc;
    HS_TRY(cudaStreamSynchronize(s->stream));
    return HH_OK;
}

int hh_slab_solve(hh_slab *s, const double *b, double *x, hh_solve_info *info)
{
    TraceRange tr("hh_slab_solve");
    if (!s || !b || !x) return HH_EINVAL;
    if (s->dev_mode) return slab_solve_device(s, b, x, info);
    const size_t V = (size_t)s->V;
    const long long n = s->own;
    const int g = grid_for(n);
    double *p = s->xe + V;   // the direction lives in the extended vector (its halos are exchanged)
    // x = 0, r = b, p = r
    HS_TRY(cudaMemsetAsync(s->xs, 0, sizeof(double) * n, s->stream));
    HS_TRY(cudaMemcpyAsync(s->r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream));
    HS_TRY(cudaMemcpyAsync(p, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream));
    double bb, rr;
    {
        const double *a[1] = {b}, *c[1] = {b};
        int rc = global_dots(s, a, c, 1, &bb);
        if (rc) return rc;
    }
    const double tol2 = s->prm.cg_tol * s->prm.cg_tol * bb;
    rr = bb;
    int it = 0, status = HH_OK, n_true = 0;
    double true_rel = bb > 0.0 ? 1.0 : 0.0;
    bool done = bb == 0.0;
    while (!done) {
        if (it >= s->prm.cg_maxit) {
            status = HH_ENOCONV;
            break;
        }
        // q = Q p, <p, q>
        int rc = slab_apply_ext(s, HH_OP_MTM, s->q);
        if (rc) return rc;
        double pq;
        {
            const double *a[1] = {p}, *c[1] = {s->q};
            rc = global_dots(s, a, c, 1, &pq);
            if (rc) return rc;
        }
        if (!std::isfinite(pq) || pq <= 0.0) {
            status = HH_ENUMERIC;
            break;
        }
        const double alpha = rr / pq;
        k_slab_update<<<g, 256, 0, s->stream>>>(s->xs, p, s->r, s->q, alpha, n);
        HS_TRY(cudaGetLastError());
        double rr_new;
        {
            const double *a[1] = {s->r}, *c[1] = {s->r};
            rc = global_dots(s, a, c, 1, &rr_new);
            if (rc) return rc;
        }
        ++it;
        if (!std::isfinite(rr_new)) {
            status = HH_ENUMERIC;
            break;
        }
        if (rr_new <= tol2) {
            // confirm with the true residual b - Q x (FP64); continue from it if not met
            HS_TRY(cudaMemcpyAsync(s->xe + V, s->xs, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream));
            rc = slab_apply_ext(s, HH_OP_MTM, s->q);
            if (rc) return rc;
            k_slab_sub<<<g, 256, 0, s->stream>>>(s->r, b, s->q, n);
            HS_TRY(cudaGetLastError());
            const double *a[1] = {s->r}, *c[1] = {s->r};
            rc = global_dots(s, a, c, 1, &rr_new);
            if (rc) return rc;
            ++n_true;
            true_rel = std::sqrt(rr_new / bb);
            if (rr_new <= tol2) {
                done = true;
                break;
            }
            // restart the direction from the true residual
            HS_TRY(cudaMemcpyAsync(p, s->r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream));
            rr = rr_new;
            continue;
        }
        k_slab_direction<<<g, 256, 0, s->stream>>>(p, s->r, rr_new / rr, n);
        HS_TRY(cudaGetLastError());
        rr = rr_new;
    }
    HS_TRY(cudaMemcpyAsync(x, s->xs, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream));
    HS_TRY(cudaStreamSynchronize(s->stream));
    if (info) {
        info->iterations = it;
        info->reliable_updates = n_true;
        info->true_relres = true_rel;
        info->converged = (done && status == HH_OK) ? 1 : 0;
    }
    return status;
}

}  // extern "C"
