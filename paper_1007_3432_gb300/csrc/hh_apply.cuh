// Launchers of the standalone applies of M, M^T and Q = M^T M.
#pragma once

#include "hh_device.cuh"
#include "hh_engine.cuh"

namespace hh {

// y = M x (trans = false) or y = M^T x (trans = true): one sweep in x groups
// of W sites with 16-byte accesses (x, y, L 16-byte aligned).  pdl: launch
// with programmatic stream serialization, so that the sweep's blocks start
// while the previous sweep on the stream finishes (they wait for its
// completion before reading).
cudaError_t launch_sweep_f64(const Geo &g, bool trans, double h, const double *L, const double *x, double *y,
                             cudaStream_t st, bool pdl = false);
cudaError_t launch_sweep_f32(const Geo &g, bool trans, float h, const float *L, const float *x, float *y,
                             cudaStream_t st, bool pdl = false);

// Whether the fused FP32 d=3 Q kernel applies to this lattice and these
// pointers (x-y plane fits in shared memory, 16-byte alignment).
bool fused_mtm_ok(const Geo &g, const void *L, const void *x, const void *y);
size_t fused_mtm_smem(int nx, int tz);

// y = M^T M x in one pass (FP32, d = 3).  *err is set to HH_ETIMEOUT if a
// bounded wait for a bulk copy ran out.  nsm: SM count (grid sizing).
cudaError_t launch_mtm_fused_f32(const Geo &g, float h, const float *L, const float *x, float *y, int *err,
                                 int nsm, cudaStream_t st);

// Whether the multi-vector FP32 d = 3 Q kernel applies to this lattice and
// these pointers (4 | Nx, Nx <= 32, 16-byte alignment).
bool multi_mtm_ok(const Geo &g, const void *L, const void *x, const void *y);

// y_v = M^T M x_v for the k FP32 vectors x_v = x + v N (y likewise) in one
// persistent launch that reads the links once (hh_apply_multi.cu).  *err is
// set to HH_ETIMEOUT if a bounded wait ran out (timeout_ns each).
cudaError_t launch_mtm_multi_f32(const Geo &g, float h, const float *L, const float *x, float *y, int k, int *err,
                                 int nsm, long long timeout_ns, cudaStream_t st);

}  // namespace hh
