// Persistent conjugate-gradient engine (Sec. 4.1: CG on Q = M^T M).
// The slot/mode structure is described in hh_engine.cuh.
#include "hh_engine.cuh"

namespace hh {

namespace {

constexpr int kNumericErr = -5;
constexpr int kNoConv = -4;

// Fixed-order sum of per-tile partials [t0, t0 + n): lane-strided sequential
// sums in warp 0 followed by a fixed shuffle tree; the value is broadcast to
// the whole block.  Every block that calls it on the same data gets the same
// bits.
__device__ double sum_partials(const double *part, int t0, int n, double *s_val)
{
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int j = threadIdx.x; j < n; j += 32) v += part[t0 + j];
        v = warp_sum(v);
        if (threadIdx.x == 0) *s_val = v;
    }
    __syncthreads();
    double r = *s_val;
    __syncthreads();
    return r;
}

__device__ __forceinline__ bool finite(double v)
{
    return isfinite(v);
}

// Next mode of a system from its previous state and the |r|^2 reduced from the
// previous iteration's slot 3.  Pure function of its inputs: all blocks agree.
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
        return S;
    case MODE_INIT:
        S.bb = rr;
        S.rr_last = rr;
        if (!finite(rr)) {
            S.mode = MODE_DONE;
            S.status = kNumericErr;
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
        return S;
    case MODE_CG: {
        S.cg_steps = P.cg_steps + 1;
        S.rr_last = rr;
        if (!finite(rr)) {
            S.mode = MODE_DONE;
            S.status = kNumericErr;
            return S;
        }
        bool need = rr <= Y.tol2 * P.bb;
        if (Y.precision == PREC_MIXED && rr < Y.delta2 * P.maxr2) need = true;
        if (S.cg_steps >= Y.maxit) {
            need = true;
            S.final_ru = 1;
        }
        if (need) {
            S.mode = MODE_RU;
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
        if (!finite(rr)) {
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
        return S;
    }
    }
}

// ---- slot 1 -----------------------------------------------------------------
__device__ void slot1_work(const EngSystem &Y, const EngState &S, const EngTile &T)
{
    if (S.mode == MODE_CG) {
        if (Y.precision == PREC_FP64) {
            const double beta = S.beta;
            if (beta == 0.0) {
                for (int i = T.begin + threadIdx.x; i < T.end; i += blockDim.x) Y.p[i] = Y.r[i];
            } else {
                for (int i = T.begin + threadIdx.x; i < T.end; i += blockDim.x)
                    Y.p[i] = fma(beta, Y.p[i], Y.r[i]);
            }
        } else {
            const float beta = (float)S.beta;
            if (S.beta == 0.0) {
                for (int i = T.begin + threadIdx.x; i < T.end; i += blockDim.x) Y.p32[i] = Y.r32[i];
            } else {
                for (int i = T.begin + threadIdx.x; i < T.end; i += blockDim.x)
                    Y.p32[i] = fmaf(beta, Y.p32[i], Y.r32[i]);
            }
        }
    } else if (S.mode == MODE_RU) {
        if (Y.precision == PREC_MIXED) {
            for (int i = T.begin + threadIdx.x; i < T.end; i += blockDim.x) {
                Y.x[i] += (double)Y.x32[i];
                Y.x32[i] = 0.0f;
            }
        }
    } else if (S.mode == MODE_INIT) {
        for (int i = T.begin + threadIdx.x; i < T.end; i += blockDim.x) Y.x[i] = 0.0;
        if (Y.precision == PREC_MIXED)
            for (int i = T.begin + threadIdx.x; i < T.end; i += blockDim.x) Y.x32[i] = 0.0f;
    }
}

// ---- slot 2: t = M p (CG) or t64 = M x64 (RU); returns this thread's |t|^2 --
__device__ double slot2_work(const EngSystem &Y, const EngState &S, const EngTile &T)
{
    const Geo &g = Y.g;
    Nbr nb;
    if (S.mode == MODE_CG) {
        if (Y.precision == PREC_FP64) {
            double acc = 0.0;
            for (int i = T.begin + threadIdx.x; i < T.end; i += blockDim.x) {
                neighbours(g, i, nb);
                double v = stencil_M<double>(g, Y.h, Y.L64, Y.p, i, nb);
                Y.t[i] = v;
                acc = fma(v, v, acc);
            }
            return acc;
        } else {
            float acc = 0.0f;
            const float h = (float)Y.h;
            for (int i = T.begin + threadIdx.x; i < T.end; i += blockDim.x) {
                neighbours(g, i, nb);
                float v = stencil_M<float>(g, h, Y.L32, Y.p32, i, nb);
                Y.t32[i] = v;
                acc = fmaf(v, v, acc);
            }
            return (double)acc;
        }
    } else if (S.mode == MODE_RU) {
        for (int i = T.begin + threadIdx.x; i < T.end; i += blockDim.x) {
            neighbours(g, i, nb);
            Y.t[i] = stencil_M<double>(g, Y.h, Y.L64, Y.x, i, nb);
        }
    }
    return 0.0;
}

// ---- slot 3: returns this thread's |r|^2 -------------------------------------
__device__ double slot3_work(const EngSystem &Y, const EngState &S, const EngTile &T, double alpha)
{
    const Geo &g = Y.g;
    Nbr nb;
    if (S.mode == MODE_CG) {
        if (Y.precision == PREC_FP64) {
            double acc = 0.0;
            for (int i = T.begin + threadIdx.x; i < T.end; i += blockDim.x) {
                neighbours(g, i, nb);
                double q = stencil_MT<double>(g, Y.h, Y.L64, Y.t, i, nb);
                Y.x[i] = fma(alpha, Y.p[i], Y.x[i]);
                double r = fma(-alpha, q, Y.r[i]);
                Y.r[i] = r;
                acc = fma(r, r, acc);
            }
            return acc;
        } else {
            float acc = 0.0f;
            const float a = (float)alpha, h = (float)Y.h;
            for (int i = T.begin + threadIdx.x; i < T.end; i += blockDim.x) {
                neighbours(g, i, nb);
                float q = stencil_MT<float>(g, h, Y.L32, Y.t32, i, nb);
                Y.x32[i] = fmaf(a, Y.p32[i], Y.x32[i]);
                float r = fmaf(-a, q, Y.r32[i]);
                Y.r32[i] = r;
                acc = fmaf(r, r, acc);
            }
            return (double)acc;
        }
    } else if (S.mode == MODE_RU) {
        double acc = 0.0;
        for (int i = T.begin + threadIdx.x; i < T.end; i += blockDim.x) {
            neighbours(g, i, nb);
            double res = Y.b[i] - stencil_MT<double>(g, Y.h, Y.L64, Y.t, i, nb);
            if (Y.precision == PREC_FP64)
                Y.r[i] = res;
            else
                Y.r32[i] = (float)res;
            acc = fma(res, res, acc);
        }
        return acc;
    } else if (S.mode == MODE_INIT) {
        double acc = 0.0;
        for (int i = T.begin + threadIdx.x; i < T.end; i += blockDim.x) {
            double bi = Y.b[i];
            if (Y.precision == PREC_FP64)
                Y.r[i] = bi;
            else
                Y.r32[i] = (float)bi;
            acc = fma(bi, bi, acc);
        }
        return acc;
    }
    return 0.0;
}

__global__ void __launch_bounds__(ENGINE_BLOCK) engine_kernel(EngLaunch L)
{
    __shared__ double s_red[ENGINE_BLOCK / 32];
    __shared__ double s_val;
    __shared__ int s_flag;
    __shared__ unsigned s_gen;

    BarrierCtl *ctl = L.ctl;
    const unsigned G = gridDim.x;
    if (threadIdx.x == 0) s_gen = *(volatile unsigned *)&ctl->gen;
    __syncthreads();
    unsigned gen = s_gen;
    long long k = *(volatile long long *)&ctl->k;

    for (long long it = 0; it < L.max_iters; ++it, ++k) {
        EngState *cur = L.state[k & 1];
        EngState *nxt = L.state[(k + 1) & 1];

        // ---- slot 1: decide, then p update / reliable-update accumulate ----
        {
            int last = -1;
            EngState S;
            for (int tile = blockIdx.x; tile < L.ntiles; tile += G) {
                const EngTile T = L.tiles[tile];
                const EngSystem &Y = L.sys[T.sys];
                if (T.sys != last) {
                    const EngState P = cur[T.sys];
                    double rr = 0.0;
                    if (P.mode == MODE_INIT || P.mode == MODE_CG || P.mode == MODE_RU)
                        rr = sum_partials(L.part_rr, Y.tile0, Y.ntiles, &s_val);
                    S = decide(Y, P, rr);
                    last = T.sys;
                    if ((int)blockIdx.x == Y.owner && threadIdx.x == 0) {
                        nxt[T.sys] = S;
                        if (S.mode == MODE_DONE && P.mode != MODE_DONE) atomicSub(&ctl->active, 1);
                    }
                }
                slot1_work(Y, S, T);
            }
        }
        if (!grid_barrier(ctl, G, gen, &s_flag)) return;
        if (ld_volatile_i32(&ctl->active) <= 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) ctl->k = k + 1;
            return;
        }

        // ---- slot 2 ----
        for (int tile = blockIdx.x; tile < L.ntiles; tile += G) {
            const EngTile T = L.tiles[tile];
            const EngSystem &Y = L.sys[T.sys];
            const EngState S = nxt[T.sys];
            double v = slot2_work(Y, S, T);
            if (S.mode == MODE_CG) {
                double tot = block_sum(v, s_red);
                if (threadIdx.x == 0) L.part_tt[tile] = tot;
            }
        }
        if (!grid_barrier(ctl, G, gen, &s_flag)) return;

        // ---- slot 3 ----
        {
            int last = -1;
            double alpha = 0.0;
            for (int tile = blockIdx.x; tile < L.ntiles; tile += G) {
                const EngTile T = L.tiles[tile];
                const EngSystem &Y = L.sys[T.sys];
                const EngState S = nxt[T.sys];
                if (S.mode == MODE_CG && T.sys != last) {
                    double tt = sum_partials(L.part_tt, Y.tile0, Y.ntiles, &s_val);
                    alpha = S.rr_alpha / tt;
                    last = T.sys;
                }
                double v = slot3_work(Y, S, T, alpha);
                if (S.mode == MODE_CG || S.mode == MODE_RU || S.mode == MODE_INIT) {
                    double tot = block_sum(v, s_red);
                    if (threadIdx.x == 0) L.part_rr[tile] = tot;
                }
            }
        }
        if (!grid_barrier(ctl, G, gen, &s_flag)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->k = k;
}

}  // namespace

cudaError_t engine_launch(const EngLaunch &L, int grid, int block, cudaStream_t stream)
{
    EngLaunch arg = L;
    void *args[] = {(void *)&arg};
    return cudaLaunchCooperativeKernel((const void *)engine_kernel, dim3(grid), dim3(block), args, 0,
                                       stream);
}

int engine_max_grid(int block)
{
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, engine_kernel, block, 0) != cudaSuccess)
        return 0;
    return per * nsm;
}

}  // namespace hh
