"""GPU parity of the exact-block form of M (hh_params.link_order 1, 2) against
the oracle: the blocks of Eq. (7) with B = e^{-dtau K} e^{-dtau V}, the hopping
factor e^{-dtau K} = e^{h H} expanded to first or second order in dtau K.

* applies M, M^T, M^T M per element (FP64 to 1e-12 of the magnitude of the
  terms, FP32 to 1e-5);
* solves (FP64 and mixed) to the true residual 1e-10 of the oracle's operator;
* the force and whole trajectories (energies, accept decisions);
* unsupported combinations are refused.
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


SHAPES = [(1, 16, 12), (1, 2, 6), (1, 37, 9), (3, 4, 6), (3, 5, 3), (3, 2, 4)]


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("d,nx,ntau", SHAPES)
@pytest.mark.parametrize("op", ["M", "MT", "MTM"])
def test_exact_block_apply_per_element(hh, order, d, nx, ntau, op):
    lat = oracle.lattice(d, nx, ntau)
    n = oracle.nsites(lat)
    sigma = workloads.sigma_field(n, seed=300 + nx + ntau)
    x = workloads.source(n, seed=301 + nx)
    L = oracle.links(lat, A, sigma)
    fn = {"M": oracle.apply_M_ex, "MT": oracle.apply_MT_ex, "MTM": oracle.apply_MTM_ex}[op]
    ref = fn(lat, H, L, order, x)
    # magnitude of the terms: the same operator on |x| with |L|
    mag = fn(lat, H, np.abs(L), order, np.abs(x)) if op != "MTM" else \
        oracle.apply_MT_ex(lat, H, np.abs(L), order, oracle.apply_M_ex(lat, H, np.abs(L), order, np.abs(x)))
    code = {"M": hh.HH_OP_M, "MT": hh.HH_OP_MT, "MTM": hh.HH_OP_MTM}[op]
    with hh.Context(d, nx, ntau, link_order=order) as ctx:
        ctx.set_field(dev(sigma))
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        ctx.apply(code, dev(x), y)
        got = y.cpu().numpy()
        yf = torch.empty(n, dtype=torch.float32, device="cuda")
        ctx.apply(code, dev(x.astype(np.float32)), yf, dtype=hh.HH_DTYPE_F32)
        gotf = yf.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 1e-12 * mag + 1e-300)
    assert np.all(np.abs(gotf - ref) <= 1e-5 * mag)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("d,nx,ntau", [(1, 32, 24), (3, 6, 8)])
def test_exact_block_solve(hh, order, precision, d, nx, ntau):
    lat = oracle.lattice(d, nx, ntau)
    n = oracle.nsites(lat)
    sigma = workloads.sigma_field(n, seed=310 + nx)
    L = oracle.links(lat, A, sigma)
    b = np.stack([workloads.source(n, seed=311, rhs=a) for a in range(2)])
    with hh.Context(d, nx, ntau, precision=precision, link_order=order) as ctx:
        ctx.set_field(dev(sigma))
        x = torch.zeros(2, n, dtype=torch.float64, device="cuda")
        rc, info = ctx.solve(dev(b), x, 2)
        xg = x.cpu().numpy()
    assert rc == 0 and info["true_relres"] <= 1e-10
    for a in range(2):
        res = b[a] - oracle.apply_MTM_ex(lat, H, L, order, xg[a])
        assert np.linalg.norm(res) <= 1.0001e-10 * np.linalg.norm(b[a])
        xo, st, it, rr = oracle.cg_ex(lat, H, L, order, b[a])
        assert st == 0 and np.linalg.norm(xg[a] - xo) <= 1e-4 * np.linalg.norm(xo)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("d,nx,ntau", [(1, 16, 24), (3, 4, 6)])
def test_exact_block_force(hh, order, d, nx, ntau):
    lat = oracle.lattice(d, nx, ntau)
    n = oracle.nsites(lat)
    sigma = workloads.sigma_field(n, seed=320 + nx)
    chi = np.stack([workloads.source(n, seed=321, rhs=a) for a in range(2)])
    prm = oracle.params(link_order=order)
    F_ref, *_ = oracle.force(lat, prm, sigma, chi)
    with hh.Context(d, nx, ntau, link_order=order) as ctx:
        ctx.set_field(dev(sigma))
        F = torch.empty(n, dtype=torch.float64, device="cuda")
        ctx.force(dev(chi), 2, F)
        got = F.cpu().numpy()
    assert np.max(np.abs(got - F_ref)) <= 1e-7 * np.max(np.abs(F_ref))


@pytest.mark.parametrize("order", [1, 2])
def test_exact_block_trajectories_match_oracle(hh, order):
    d, nx, ntau = 1, 16, 32
    lat = oracle.lattice(d, nx, ntau)
    n = nx * ntau
    seed = 330 + order
    sigma = workloads.sigma_field(n, seed=seed)
    prm = oracle.params(seed=seed, n_pf=2, link_order=order)
    s_ref = sigma.copy()
    with hh.Context(d, nx, ntau, seed=seed, n_pf=2, link_order=order) as ctx:
        ctx.set_field(dev(sigma))
        for traj in range(2):
            info = ctx.trajectory(4, 0.05, traj)
            s_ref, oinfo = oracle.trajectory(lat, prm, s_ref, 4, 0.05, traj)
            assert info["max_true_relres"] <= 1e-10 and info["u"] == oinfo["u"]
            assert abs(info["H0"] - oinfo["H0"]) <= 1e-8 * abs(oinfo["H0"])
            assert abs(info["dH"] - oinfo["dH"]) <= 1e-6, (info, oinfo)
            if abs(oinfo["dH"] + np.log(oinfo["u"])) > 1e-5:
                assert info["accepted"] == oinfo["accepted"]
            if info["accepted"] != oinfo["accepted"]:
                break
            got = torch.empty(n, dtype=torch.float64, device="cuda")
            ctx.get_field(got)
            assert np.max(np.abs(got.cpu().numpy() - s_ref)) <= 1e-6


def test_exact_block_refusals(hh):
    from paper_1007_3432_gb300 import binding as B
    with pytest.raises(hh.HHError):
        hh.Context(1, 8, 8, link_order=3)
    with pytest.raises(hh.HHError):
        hh.Context(1, 8, 8, link_order=1, cheb_degree=2)
    batch = B.Batch(max_slots=2, hbm_budget_bytes=1 << 26)
    req = B.make_request(B.HH_REQ_SOLVE, 1, 8, 8, sigma=np.zeros(64), n_pf=1, link_order=1)
    rc, _ = batch.submit(req, allow=(B.HH_EINVAL,))
    batch.close()
    assert rc == B.HH_EINVAL
