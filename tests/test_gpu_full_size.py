"""Parity at the benchmark's full sizes, in the launch configurations that
bench.py times (the context solver with two right-hand sides):

* d = 1, 1024 x 512 (524,288 sites): FP64 CG in the overlapped layout (every
  block holds a tile of both systems, control warp), mixed CG in the flat one;
* d = 3, 32^3 x 128 (4.2M sites): mixed CG, overlapped layout; and every
  element of its FP64 M, M^T and Q applies.

The oracle cannot run CG at these sizes in a test's time, so it checks what
holds at any size: the true residual b - Q x of the returned solutions with its
own Q (must be <= 1e-10 |b|), and the force at sampled sites from its formula
(dS/dsigma = -sum_a y_a(n, tau+1) s(tau) A cos sigma x_a, y_a = M x_a with the
oracle's M) applied to the GPU solutions.
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _solve_full(hh, wl, precision):
    n = wl.nsites
    sigma = workloads.sigma_field(n, seed=wl.seed)
    b = np.stack([workloads.source(n, seed=wl.seed, rhs=a) for a in range(2)])
    with hh.Context(wl.d, wl.nx, wl.ntau, precision=precision) as ctx:
        ctx.set_field(dev(sigma))
        x = torch.zeros(2, n, dtype=torch.float64, device="cuda")
        rc, info = ctx.solve(dev(b), x, 2)
        F = torch.empty(n, dtype=torch.float64, device="cuda")
        ctx.force(dev(b), 2, F)
        return sigma, b, x.cpu().numpy(), info, rc, F.cpu().numpy()


@pytest.mark.parametrize("wl,precision", [(workloads.C1, "fp64"), (workloads.C1, "mixed"),
                                          (workloads.C2, "mixed")])
def test_full_size_solve_residual_and_force(hh, wl, precision):
    sigma, b, x, info, rc, F = _solve_full(hh, wl, precision)
    assert rc == 0 and info["converged"] == 1 and info["true_relres"] <= 1e-10
    lat = oracle.lattice(wl.d, wl.nx, wl.ntau)
    L = oracle.links(lat, A, sigma)
    for a in range(2):
        res = b[a] - oracle.apply_MTM(lat, H, L, x[a])
        assert np.linalg.norm(res) <= 1.0001e-10 * np.linalg.norm(b[a]), np.linalg.norm(res) / np.linalg.norm(b[a])
    # The force of the same solves (hh_force solves again from zero; the
    # solutions agree to the tolerance) at sampled sites, from the oracle's M.
    n = wl.nsites
    V = wl.nx ** wl.d
    y = [oracle.apply_M(lat, H, L, x[a]) for a in range(2)]
    rng = np.random.default_rng(7)
    sites = rng.choice(n, size=512, replace=False)
    scale = np.max(np.abs(F))
    for i in sites:
        tau = i // V
        inext = (i + V) % n
        s = 1.0 if tau == wl.ntau - 1 else -1.0
        ref = -sum(y[a][inext] * s * A * np.cos(sigma[i]) * x[a][i] for a in range(2))
        assert abs(F[i] - ref) <= 1e-6 * scale, (i, F[i], ref)


@pytest.mark.parametrize("op", ["M", "MT", "MTM"])
def test_full_size_fp64_apply_per_element(hh, op):
    """Every element of the FP64 M, M^T and Q = M^T M applies on the d = 3,
    32^3 x 128 lattice (4.2M sites) against the oracle, to 1e-12 of the sum
    of the magnitudes of each row's terms (the tolerance of the small-lattice
    FP64 parity tests)."""
    wl = workloads.C2
    lat = oracle.lattice(wl.d, wl.nx, wl.ntau)
    n = wl.nsites
    sigma = workloads.sigma_field(n, seed=wl.seed)
    x = workloads.source(n, seed=wl.seed + 5)
    L = oracle.links(lat, A, sigma)
    f = {"M": oracle.apply_M, "MT": oracle.apply_MT, "MTM": oracle.apply_MTM}[op]
    ref = f(lat, H, L, x)
    La, xa = np.abs(L), np.abs(x)
    if op == "M":
        mag = oracle.apply_M(lat, -H, La, xa)
    elif op == "MT":
        mag = oracle.apply_MT(lat, -H, La, xa)
    else:
        mag = oracle.apply_MT(lat, -H, La, oracle.apply_M(lat, -H, La, xa))
    code = {"M": hh.HH_OP_M, "MT": hh.HH_OP_MT, "MTM": hh.HH_OP_MTM}[op]
    with hh.Context(wl.d, wl.nx, wl.ntau) as ctx:
        ctx.set_field(dev(sigma))
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        ctx.apply(code, dev(x), y)
        got = y.cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-12 * mag), np.max(np.abs(got - ref) / mag)
