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

}  // namespace hh
