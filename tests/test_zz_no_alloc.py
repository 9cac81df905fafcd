"""The allocation-free solve entry point against the context solver.

hh_solve_noalloc is for callers that cannot allocate when they need a solve
(inside applications that own the allocator, loops that must not take its
locks); its scratch is a fixed device array shared by all calls.  This file is collected
last on purpose.  It checks, through the C ABI, that two calls in a row (the
second on a different lattice, over whatever the first left in the shared
array) give the same solution as hh_solve within the solver tolerance the
other tests use, and that a lattice above the array's capacity is refused.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads  # noqa: E402


@pytest.fixture(scope="module")
def hh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1007_3432_gb300 as pkg
    from paper_1007_3432_gb300 import build
    build.build()
    pkg.load()
    return pkg


def _case(d, nx, ntau, seed):
    n = nx ** d * ntau
    sigma = workloads.sigma_field(n, seed=seed)
    b = workloads.source(n, seed=seed + 1)
    return n, sigma, b


def test_noalloc_matches_context_solver_twice(hh):
    from paper_1007_3432_gb300.binding import solve_noalloc
    h = workloads.T_HOP * workloads.DTAU
    for d, nx, ntau, seed in [(1, 64, 96, 21), (3, 8, 20, 22)]:
        n, sigma, b = _case(d, nx, ntau, seed)
        sig_d = torch.from_numpy(sigma).cuda()
        b_d = torch.from_numpy(b).cuda()
        x_na = torch.full((n,), 3.0, dtype=torch.float64, device="cuda")
        rc, info = solve_noalloc(d, nx, ntau, sig_d, b_d, x_na)
        assert rc == 0 and info["converged"] == 1 and info["true_relres"] <= 1e-10, info

        with hh.Context(d, nx, ntau) as ctx:
            ctx.set_field(sig_d)
            x_ctx = torch.zeros(n, dtype=torch.float64, device="cuda")
            rc2, info2 = ctx.solve(b_d, x_ctx, 1)
        assert rc2 == 0
        xa, xc = x_na.cpu().numpy(), x_ctx.cpu().numpy()
        # Same tolerance as the solver parity tests: both meet 1e-10 in the
        # true residual, so the solutions agree to kappa * 2e-10.
        assert np.linalg.norm(xa - xc) <= 1e-4 * np.linalg.norm(xc)
        lat = oracle.lattice(d, nx, ntau)
        L = oracle.links(lat, workloads.A_HS, sigma)
        res = b - oracle.apply_MTM(lat, h, L, xa)
        assert np.linalg.norm(res) <= 1.0001e-10 * np.linalg.norm(b)


def test_noalloc_rejects_oversize(hh):
    from paper_1007_3432_gb300.binding import HH_ESIZE, HH_NOALLOC_MAX_SITES, solve_noalloc
    d, nx, ntau = 1, 1024, HH_NOALLOC_MAX_SITES // 1024 + 1
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc, _ = solve_noalloc(d, nx, ntau, x, x, x)
    assert rc == HH_ESIZE
