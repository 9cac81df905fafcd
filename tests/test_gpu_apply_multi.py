"""GPU parity of hh_apply_multi: y_v = op(x_v) for several vectors sharing one
field, against the FP64 oracle on the same seeded inputs, per element.

The FP32 Q = M^T M of d = 3 lattices with 4 | Nx <= 32 runs in the persistent
multi-vector kernel (pipeline forms selected by HH_APPLY_MULTI_FORM: 4- or
8-plane slabs, one or two parts, one float4 group per thread or, for
Nx = 32, a pair of rows per thread; the x halo by warp shuffles when a row of
float4 groups divides a warp, else from shared memory); the shapes below
cover every form, both halo forms, slabs that wrap onto themselves (Nx = 4,
8), short and odd N_tau (uneven ranges per CTA, ranges that cross from one
vector to the next), and the full 32^3 x 128 lattice.  Other operators, dtypes and lattices go
through one hh_apply per vector.  Tolerance as for the single applies:
|y - y_ref|_i <= 2e-6 (|M| |x|)_i in FP32, 1e-12 in FP64.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads  # noqa: E402

H = workloads.T_HOP * workloads.DTAU
A = workloads.A_HS


@pytest.fixture(scope="module")
def hh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1007_3432_gb300 as pkg
    from paper_1007_3432_gb300 import build
    build.build()
    pkg.load()
    return pkg


def _ref_and_bound(lat, op, L, x64, tol):
    f = {"M": oracle.apply_M, "MT": oracle.apply_MT, "MTM": oracle.apply_MTM}[op]
    La, xa = np.abs(L), np.abs(x64)
    mag = {"M": lambda: oracle.apply_M(lat, -H, La, xa),
           "MT": lambda: oracle.apply_MT(lat, -H, La, xa),
           "MTM": lambda: oracle.apply_MT(lat, -H, La, oracle.apply_M(lat, -H, La, xa))}[op]()
    return f(lat, H, L, x64), tol * mag


def _run(hh, d, nx, ntau, k, op="MTM", dtype=np.float32, seed=0):
    lat = oracle.lattice(d, nx, ntau)
    n = oracle.nsites(lat)
    sigma = workloads.sigma_field(n, seed=500 + nx + ntau + seed)
    xs = np.stack([workloads.source(n, seed=600 + nx + seed, rhs=a) for a in range(k)]).astype(dtype)
    L = oracle.links(lat, A, sigma)
    code = {"M": hh.HH_OP_M, "MT": hh.HH_OP_MT, "MTM": hh.HH_OP_MTM}[op]
    with hh.Context(d, nx, ntau) as ctx:
        ctx.set_field(torch.from_numpy(sigma).cuda())
        x_d = torch.from_numpy(xs.reshape(-1)).cuda()
        y_d = torch.full_like(x_d, float("nan"))
        ctx.apply_multi(code, x_d, y_d, k)
        cnt = ctx.counters()            # raises on a recorded device-side timeout
        got = y_d.cpu().numpy().reshape(k, n).astype(np.float64)
    tol = 2e-6 if dtype == np.float32 else 1e-12
    for v in range(k):
        ref, bound = _ref_and_bound(lat, op, L, xs[v].astype(np.float64), tol)
        err = np.abs(got[v] - ref)
        assert np.all(err <= bound), (v, float(np.max(err / bound)))
    return cnt


# (nx, ntau, k): 8-plane slabs with shuffles (8, 16, 32), without (24);
# 4-plane slabs without shuffles (4, 12, 20, 28); ragged per-CTA ranges.
MULTI_SHAPES = [(8, 12, 3), (16, 10, 2), (32, 10, 4), (24, 5, 2), (4, 3, 5), (12, 9, 2), (20, 7, 3),
                (28, 2, 2), (32, 3, 8), (16, 33, 7)]


@pytest.mark.parametrize("nx,ntau,k", MULTI_SHAPES)
def test_multi_mtm_fp32_per_element(hh, nx, ntau, k):
    _run(hh, 3, nx, ntau, k)


@pytest.mark.parametrize("form", [1, 2, 3, 4])
@pytest.mark.parametrize("nx,ntau,k", [(32, 6, 3), (32, 3, 8), (32, 17, 5), (16, 10, 2), (8, 5, 4)])
def test_multi_mtm_fp32_pipeline_forms(hh, monkeypatch, form, nx, ntau, k):
    """Every pipeline form besides the defaults (form 5 for Nx = 32, form 2
    otherwise), which run in the tests above; form 4 takes Nx = 32 only, other
    lattices fall back to form 2."""
    monkeypatch.setenv("HH_APPLY_MULTI_FORM", str(form))
    _run(hh, 3, nx, ntau, k)


@pytest.mark.parametrize("form", [2, 4])
def test_multi_mtm_other_forms_full_size(hh, monkeypatch, form):
    """The one-row form 2 and the row-pair form 4 on the 32^3 x 128 lattice,
    three vectors (the default form 5 runs in test_multi_mtm_full_size_lattice)."""
    monkeypatch.setenv("HH_APPLY_MULTI_FORM", str(form))
    wl = workloads.C2
    _run(hh, wl.d, wl.nx, wl.ntau, 3, seed=wl.seed + 1)


def test_multi_kernel_single_vector_path(hh, monkeypatch):
    """hh_apply through the multi-vector kernel with one vector (HH_APPLY_MTM=4)."""
    monkeypatch.setenv("HH_APPLY_MTM", "4")
    _run(hh, 3, 16, 11, 1)


def test_multi_mtm_full_size_lattice(hh):
    """The 32^3 x 128 lattice (4.2M sites), two vectors in one launch, every
    element against the oracle."""
    wl = workloads.C2
    _run(hh, wl.d, wl.nx, wl.ntau, 2, seed=wl.seed)


@pytest.mark.parametrize("d,nx,ntau,op,dtype", [(1, 32, 16, "MTM", np.float64), (3, 8, 6, "M", np.float32),
                                                 (3, 6, 5, "MTM", np.float32), (3, 5, 4, "MT", np.float64),
                                                 (1, 36, 9, "MTM", np.float32)])
def test_multi_fallback_paths(hh, d, nx, ntau, op, dtype):
    """Operators, dtypes and lattices outside the multi-vector kernel: one
    apply per vector."""
    _run(hh, d, nx, ntau, 3, op=op, dtype=dtype)


def test_multi_rejects_bad_arguments(hh):
    from paper_1007_3432_gb300.binding import HH_EINVAL, HHError
    n = 8 ** 3 * 4
    with hh.Context(3, 8, 4) as ctx:
        buf = torch.zeros(3 * n, dtype=torch.float32, device="cuda")
        with pytest.raises(HHError) as e:
            ctx.apply_multi(hh.HH_OP_MTM, buf, buf[n:], 2)        # overlapping x and y
        assert e.value.code == HH_EINVAL
        with pytest.raises(HHError) as e:
            ctx.apply_multi(hh.HH_OP_MTM, buf, buf, 0)
        assert e.value.code == HH_EINVAL
