"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs.

Tolerances:
  * FP64 stencil applies: |y_gpu - y_ref|_i <= 1e-12 * (|M| |x|)_i, where
    (|M| |x|)_i is the sum of the magnitudes of the terms of row i (obtained
    from the oracle with h -> -h, L -> |L|, x -> |x|).  Rounding differences
    of FP64 sums of a handful of terms are ~1e-16 of that bound's scale.
  * FP32 applies: the same form with 2e-6 (a few FP32 ulps of each term).
  * CG: true relative residual ||b - Q x|| / ||b|| <= 1e-10, recomputed by the
    oracle in FP64 from the GPU's x.
  * Trajectories: identical accept/reject decisions (except a decision within
    the estimated dH error of the threshold), dH within 1e-6 absolute.
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


def magnitude(lat, which, L, x):
    """Row-wise sum of |terms| of op(x)."""
    La, xa = np.abs(L), np.abs(x)
    if which == "M":
        return oracle.apply_M(lat, -H, La, xa)
    if which == "MT":
        return oracle.apply_MT(lat, -H, La, xa)
    return oracle.apply_MT(lat, -H, La, oracle.apply_M(lat, -H, La, xa))


SHAPES = [(1, 32, 64), (1, 37, 13), (1, 2, 6), (1, 1024, 8), (3, 5, 7), (3, 8, 12), (3, 2, 4),
          (3, 3, 2), (3, 10, 9)]


@pytest.mark.parametrize("d,nx,ntau", SHAPES)
@pytest.mark.parametrize("op", ["M", "MT", "MTM"])
def test_apply_fp64_per_element(hh, d, nx, ntau, op):
    lat = oracle.lattice(d, nx, ntau)
    n = oracle.nsites(lat)
    sigma = workloads.sigma_field(n, seed=100 + nx + ntau)
    x = workloads.source(n, seed=200 + nx)
    L = oracle.links(lat, A, sigma)
    ref = {"M": oracle.apply_M, "MT": oracle.apply_MT, "MTM": oracle.apply_MTM}[op](lat, H, L, x)
    bound = 1e-12 * magnitude(lat, op, L, x)
    code = {"M": hh.HH_OP_M, "MT": hh.HH_OP_MT, "MTM": hh.HH_OP_MTM}[op]
    with hh.Context(d, nx, ntau) as ctx:
        ctx.set_field(dev(sigma))
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        ctx.apply(code, dev(x), y)
        got = y.cpu().numpy()
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / bound)


FP32_SHAPES = [(1, 32, 64), (3, 8, 12), (3, 5, 7), (3, 4, 3), (3, 6, 5), (3, 12, 9), (3, 32, 10),
               (3, 10, 40)]


# Q apply paths (HH_APPLY_MTM): by size (two sweeps with programmatic
# dependent launch here), plain two sweeps, the fused FP32 d = 3 kernel.
MTM_PATHS = ["0", "1", "3"]


@pytest.mark.parametrize("d,nx,ntau", FP32_SHAPES)
@pytest.mark.parametrize("op,path", [("M", "0"), ("MT", "0")] + [("MTM", p) for p in MTM_PATHS])
def test_apply_fp32_per_element(hh, monkeypatch, d, nx, ntau, op, path):
    monkeypatch.setenv("HH_APPLY_MTM", path)
    lat = oracle.lattice(d, nx, ntau)
    n = oracle.nsites(lat)
    sigma = workloads.sigma_field(n, seed=300 + nx)
    x = workloads.source(n, seed=400 + nx).astype(np.float32)
    L = oracle.links(lat, A, sigma)
    x64 = x.astype(np.float64)
    ref = {"M": oracle.apply_M, "MT": oracle.apply_MT, "MTM": oracle.apply_MTM}[op](lat, H, L, x64)
    bound = 2e-6 * magnitude(lat, op, L, x64)
    code = {"M": hh.HH_OP_M, "MT": hh.HH_OP_MT, "MTM": hh.HH_OP_MTM}[op]
    with hh.Context(d, nx, ntau) as ctx:
        ctx.set_field(dev(sigma))
        y = torch.empty(n, dtype=torch.float32, device="cuda")
        ctx.apply(code, dev(x), y)
        got = y.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / bound)


@pytest.mark.parametrize("path", MTM_PATHS)
def test_mtm_fp32_full_size_lattice(hh, monkeypatch, path):
    """Q x on the d=3, 32^3 x 128 lattice (4.2M sites) on every Q apply path,
    the default one being the launch configuration the benchmark times; every
    element against the oracle."""
    monkeypatch.setenv("HH_APPLY_MTM", path)
    wl = workloads.C2
    lat = oracle.lattice(wl.d, wl.nx, wl.ntau)
    n = wl.nsites
    sigma = workloads.sigma_field(n, seed=wl.seed)
    x = workloads.source(n, seed=wl.seed).astype(np.float32)
    L = oracle.links(lat, A, sigma)
    x64 = x.astype(np.float64)
    ref = oracle.apply_MTM(lat, H, L, x64)
    bound = 2e-6 * magnitude(lat, "MTM", L, x64)
    with hh.Context(wl.d, wl.nx, wl.ntau) as ctx:
        ctx.set_field(dev(sigma))
        y = torch.empty(n, dtype=torch.float32, device="cuda")
        ctx.apply(hh.HH_OP_MTM, dev(x), y)
        got = y.cpu().numpy().astype(np.float64)
        assert ctx.counters()["sites"] == n      # also checks the fused kernel's wait flag
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / bound)


def test_field_roundtrip_and_random_init(hh):
    d, nx, ntau = 3, 6, 5
    n = nx ** 3 * ntau
    with hh.Context(d, nx, ntau, chain_id=3) as ctx:
        s = workloads.sigma_field(n, seed=5)
        ctx.set_field(s)                      # host pointer path
        back = np.empty(n)
        ctx.get_field(back)
        assert np.array_equal(back, s)
        ctx.init_field_random(77)
        got = torch.empty(n, dtype=torch.float64, device="cuda")
        ctx.get_field(got)
        assert np.array_equal(got.cpu().numpy(), oracle.init_field(77, 3, n))


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed-bf16link", "mixed-fix16link"])
@pytest.mark.parametrize("d,nx,ntau,n_rhs", [(1, 32, 64, 2), (1, 19, 11, 1), (3, 6, 8, 2), (3, 4, 16, 3)])
def test_solve_true_residual_and_solution(hh, precision, d, nx, ntau, n_rhs):
    lat = oracle.lattice(d, nx, ntau)
    n = oracle.nsites(lat)
    sigma = workloads.sigma_field(n, seed=500 + nx)
    L = oracle.links(lat, A, sigma)
    b = np.stack([workloads.source(n, seed=600, rhs=a) for a in range(n_rhs)])
    with hh.Context(d, nx, ntau, precision=precision) as ctx:
        ctx.set_field(dev(sigma))
        x = torch.zeros(n_rhs, n, dtype=torch.float64, device="cuda")
        rc, info = ctx.solve(dev(b), x, n_rhs)
        xg = x.cpu().numpy()
    assert rc == 0 and info["converged"] == 1
    assert info["true_relres"] <= 1e-10
    for a in range(n_rhs):
        res = b[a] - oracle.apply_MTM(lat, H, L, xg[a])
        assert np.linalg.norm(res) <= 1.0001e-10 * np.linalg.norm(b[a])
        x_ref, st, it, rr = oracle.cg(lat, H, L, b[a])
        assert st == 0
        # Both solutions meet 1e-10; they differ by at most kappa * 2e-10.
        assert np.linalg.norm(xg[a] - x_ref) <= 1e-4 * np.linalg.norm(x_ref)


def test_solve_zero_rhs_and_iteration_cap(hh):
    d, nx, ntau = 1, 16, 32
    n = nx * ntau
    with hh.Context(d, nx, ntau, cg_maxit=5) as ctx:
        ctx.set_field(dev(workloads.sigma_field(n, seed=9)))
        x = torch.full((1, n), 7.0, dtype=torch.float64, device="cuda")
        rc, info = ctx.solve(torch.zeros(1, n, dtype=torch.float64, device="cuda"), x, 1)
        assert rc == 0 and info["converged"] == 1 and not torch.any(x)
        b = dev(workloads.source(n, seed=1))
        rc, info = ctx.solve(b, x, 1, allow=(hh.binding.HH_ENOCONV,))
        assert rc == hh.binding.HH_ENOCONV and info["converged"] == 0
        assert info["iterations"] == 5 and info["true_relres"] > 1e-10


@pytest.mark.parametrize("d,nx,ntau", [(1, 16, 24), (3, 4, 6)])
def test_force_matches_oracle(hh, d, nx, ntau):
    lat = oracle.lattice(d, nx, ntau)
    n = oracle.nsites(lat)
    sigma = workloads.sigma_field(n, seed=700)
    chi = np.stack([workloads.source(n, seed=800, rhs=a) for a in range(2)])
    prm = oracle.params(cg_tol=1e-12)
    F_ref, *_ = oracle.force(lat, prm, sigma, chi)
    with hh.Context(d, nx, ntau, cg_tol=1e-12) as ctx:
        ctx.set_field(dev(sigma))
        F = torch.empty(n, dtype=torch.float64, device="cuda")
        ctx.force(dev(chi), 2, F)
        got = F.cpu().numpy()
    assert np.max(np.abs(got - F_ref)) <= 1e-7 * np.max(np.abs(F_ref))


def test_action_heatbath_identity(hh):
    d, nx, ntau = 1, 16, 24
    n = nx * ntau
    lat = oracle.lattice(d, nx, ntau)
    sigma = workloads.sigma_field(n, seed=900)
    prm = oracle.params(seed=31, chain=0)
    chi = oracle.heatbath(lat, prm, sigma, traj=2)
    S_ref, *_ = oracle.action(lat, prm, sigma, chi)
    with hh.Context(d, nx, ntau) as ctx:
        ctx.set_field(dev(sigma))
        S, info = ctx.action(dev(chi), 2)
    assert abs(S - S_ref) <= 1e-9 * S_ref


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed-fix16link"])
def test_trajectories_match_oracle(hh, precision):
    """Several trajectories of the d=1, 32 x 64 lattice from the same seed:
    identical accept/reject sequences and matching energies."""
    wl = workloads.C0
    lat = oracle.lattice(wl.d, wl.nx, wl.ntau)
    n = wl.nsites
    sigma = workloads.sigma_field(n, seed=wl.seed)
    prm = oracle.params(seed=wl.seed, n_pf=2)
    n_md, dt = 5, 0.04
    s_ref = sigma.copy()
    with hh.Context(wl.d, wl.nx, wl.ntau, seed=wl.seed, n_pf=2, precision=precision) as ctx:
        ctx.set_field(dev(sigma))
        for traj in range(3):
            info = ctx.trajectory(n_md, dt, traj)
            s_ref, oinfo = oracle.trajectory(lat, prm, s_ref, n_md, dt, traj)
            assert info["n_solves"] == 2 * (n_md + 1)
            assert info["max_true_relres"] <= 1e-10
            assert info["u"] == oinfo["u"]
            assert abs(info["H0"] - oinfo["H0"]) <= 1e-8 * abs(oinfo["H0"])
            assert abs(info["dH"] - oinfo["dH"]) <= 1e-6, (info, oinfo)
            margin = abs(oinfo["dH"] + np.log(oinfo["u"]))
            if margin > 1e-5:
                assert info["accepted"] == oinfo["accepted"]
            if info["accepted"] != oinfo["accepted"]:
                break
            got = torch.empty(n, dtype=torch.float64, device="cuda")
            ctx.get_field(got)
            assert np.max(np.abs(got.cpu().numpy() - s_ref)) <= 1e-6


OVL = dict(d=1, nx=128, ntau=96, seed=1013, n_md=4, dt=0.005, trajs=2)


@pytest.fixture(scope="module")
def overlapped_reference():
    """The oracle's trajectories of the lattice below (about 20 s each)."""
    lat = oracle.lattice(OVL["d"], OVL["nx"], OVL["ntau"])
    s = workloads.sigma_field(oracle.nsites(lat), seed=OVL["seed"])
    prm = oracle.params(seed=OVL["seed"], n_pf=2)
    out = []
    for traj in range(OVL["trajs"]):
        s, oinfo = oracle.trajectory(lat, prm, s, OVL["n_md"], OVL["dt"], traj)
        out.append((s.copy(), oinfo))
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_overlapped_layout_trajectories_match_oracle(hh, monkeypatch, overlapped_reference, precision):
    """The engine form of the C1 trajectories (every right-hand side tiled
    over the whole grid, control warp, two-slot iterations), forced onto a
    d = 1, 128 x 96 lattice that the oracle runs in seconds: identical
    accept/reject decisions, matching energies and fields over two
    trajectories."""
    monkeypatch.setenv("HH_ENGINE_OVERLAP", "1")
    d, nx, ntau, seed = OVL["d"], OVL["nx"], OVL["ntau"], OVL["seed"]
    n = nx * ntau
    sigma = workloads.sigma_field(n, seed=seed)
    n_md, dt = OVL["n_md"], OVL["dt"]
    with hh.Context(d, nx, ntau, seed=seed, n_pf=2, precision=precision) as ctx:
        ctx.set_field(dev(sigma))
        for traj in range(OVL["trajs"]):
            info = ctx.trajectory(n_md, dt, traj)
            s_ref, oinfo = overlapped_reference[traj]
            assert info["n_solves"] == 2 * (n_md + 1) and info["max_true_relres"] <= 1e-10
            assert info["u"] == oinfo["u"]
            assert abs(info["H0"] - oinfo["H0"]) <= 1e-8 * abs(oinfo["H0"])
            assert abs(info["dH"] - oinfo["dH"]) <= 1e-6 + 1e-9 * abs(oinfo["H0"]), (info, oinfo)
            if abs(oinfo["dH"] + np.log(oinfo["u"])) > 1e-5:
                assert info["accepted"] == oinfo["accepted"]
            if info["accepted"] != oinfo["accepted"]:
                break
            got = torch.empty(n, dtype=torch.float64, device="cuda")
            ctx.get_field(got)
            assert np.max(np.abs(got.cpu().numpy() - s_ref)) <= 1e-6


def test_leapfrog_reversible_on_gpu(hh):
    d, nx, ntau = 1, 16, 16
    n = nx * ntau
    lat = oracle.lattice(d, nx, ntau)
    sigma = workloads.sigma_field(n, seed=41)
    pi0 = workloads.unit_normal(n, seed=41, stream=1)
    chi = np.stack([workloads.source(n, seed=42, rhs=a) for a in range(2)])
    with hh.Context(d, nx, ntau, cg_tol=1e-12) as ctx:
        ctx.set_field(dev(sigma))
        pi = dev(pi0)
        ctx.leapfrog(pi, dev(chi), 2, 8, 0.05)
        pi.neg_()
        ctx.leapfrog(pi, dev(chi), 2, 8, 0.05)
        back = torch.empty(n, dtype=torch.float64, device="cuda")
        ctx.get_field(back)
    assert np.max(np.abs(back.cpu().numpy() - sigma)) < 1e-8
    assert np.max(np.abs(pi.cpu().numpy() + pi0)) < 1e-8


def test_invalid_arguments(hh):
    with hh.Context(1, 8, 8) as ctx:
        x = torch.zeros(64, dtype=torch.float64, device="cuda")
        with pytest.raises(hh.HHError):
            ctx.apply(7, x, torch.empty_like(x))
        with pytest.raises(hh.HHError):
            ctx.apply(hh.HH_OP_M, x, x)
        with pytest.raises(hh.HHError):
            ctx.solve(x, torch.empty_like(x), 0)
        with pytest.raises(hh.HHError):
            ctx.trajectory(0, 0.1, 0)


def test_checkpoint_resume_is_bit_identical(hh):
    """The chain state is (sigma, trajectory index): the random streams are
    counter-based, so saving sigma after trajectory 1 and resuming in a fresh
    context reproduces the uninterrupted run bit for bit."""
    d, nx, ntau = 1, 16, 24
    n = nx * ntau
    sigma = workloads.sigma_field(n, seed=51)
    kw = dict(seed=51, n_pf=2, chain_id=4)
    with hh.Context(d, nx, ntau, **kw) as ctx:
        ctx.set_field(dev(sigma))
        infos = [ctx.trajectory(3, 0.1, t) for t in range(3)]
        full = np.empty(n)
        ctx.get_field(full)
    with hh.Context(d, nx, ntau, **kw) as ctx:
        ctx.set_field(dev(sigma))
        first = ctx.trajectory(3, 0.1, 0)
        saved = np.empty(n)
        ctx.get_field(saved)
    with hh.Context(d, nx, ntau, **kw) as ctx:
        ctx.set_field(saved)
        rest = [ctx.trajectory(3, 0.1, t) for t in (1, 2)]
        resumed = np.empty(n)
        ctx.get_field(resumed)
    assert np.array_equal(full, resumed)
    assert [i["dH"] for i in infos] == [first["dH"]] + [i["dH"] for i in rest]


@pytest.mark.parametrize("d,nx,ntau,n,eps", [(1, 32, 64, 4, 1e-3), (3, 6, 8, 3, 1e-2), (1, 20, 40, 8, 1e-4)])
def test_chebyshev_pcg_matches_oracle(hh, d, nx, ntau, n, eps):
    """Preconditioned CG with the Chebyshev polynomial of Sec. 4.2: true
    residual 1e-10, the oracle's solution, and the oracle's step count (the
    two run the same algorithm; rounding may move the stop by a step or two)."""
    lat = oracle.lattice(d, nx, ntau)
    nsite = oracle.nsites(lat)
    sigma = workloads.sigma_field(nsite, seed=900 + nx)
    L = oracle.links(lat, A, sigma)
    b = np.stack([workloads.source(nsite, seed=901, rhs=a) for a in range(2)])
    lam = oracle.gershgorin_lambda_max(d, H, A)
    with hh.Context(d, nx, ntau, cheb_degree=n, cheb_eps=eps) as ctx:
        ctx.set_field(dev(sigma))
        x = torch.zeros(2, nsite, dtype=torch.float64, device="cuda")
        rc, info = ctx.solve(dev(b), x, 2)
        xg = x.cpu().numpy()
    assert rc == 0 and info["converged"] == 1 and info["true_relres"] <= 1e-10
    its = []
    for a in range(2):
        res = b[a] - oracle.apply_MTM(lat, H, L, xg[a])
        assert np.linalg.norm(res) <= 1.0001e-10 * np.linalg.norm(b[a])
        x_ref, st, it, rr = oracle.pcg(lat, H, L, b[a], n, eps, lam)
        assert st == 0
        assert np.linalg.norm(xg[a] - x_ref) <= 1e-4 * np.linalg.norm(x_ref)
        its.append(it)
    assert abs(info["iterations"] - max(its)) <= 2 + 0.03 * max(its), (info, its)


def test_chebyshev_pcg_trajectory_matches_plain_cg(hh):
    d, nx, ntau = 1, 16, 32
    n = nx * ntau
    sigma = workloads.sigma_field(n, seed=61)
    out = []
    for deg in (0, 4):
        with hh.Context(d, nx, ntau, seed=61, n_pf=2, cheb_degree=deg, cheb_eps=1e-3) as ctx:
            ctx.set_field(dev(sigma))
            out.append(ctx.trajectory(4, 0.1, 0))
    assert abs(out[0]["dH"] - out[1]["dH"]) <= 1e-6
    assert out[0]["accepted"] == out[1]["accepted"]


def test_chebyshev_rejected_for_mixed_precision(hh):
    with pytest.raises(hh.HHError):
        hh.Context(1, 8, 8, precision="mixed", cheb_degree=2)


# Both forms of the engine iteration (three slots, or the direction update
# fused into t = M p) do the same arithmetic on the same operands in the same
# order: solutions, iteration counts and residuals agree bit for bit.  The
# overlapped layout (each block holds a tile of every system) tiles the
# systems differently, so its partial sums, and the last bits, differ; both
# layouts meet the tolerance.
SLOT_CASES = [(1, 32, 64, "fp64", 0), (1, 48, 24, "mixed", 0), (3, 6, 8, "fp64", 0), (3, 8, 10, "mixed", 0),
              (1, 32, 64, "fp64", 4), (3, 6, 8, "fp64", 3), (1, 19, 11, "mixed", 0)]


@pytest.mark.parametrize("d,nx,ntau,precision,cheb", SLOT_CASES)
def test_two_and_three_slot_forms_agree_bitwise(hh, monkeypatch, d, nx, ntau, precision, cheb):
    n = nx ** d * ntau
    sigma = workloads.sigma_field(n, seed=700 + nx)
    b = np.stack([workloads.source(n, seed=701, rhs=a) for a in range(2)])
    lat = oracle.lattice(d, nx, ntau)
    L = oracle.links(lat, A, sigma)
    by_layout = {}
    for overlap in ("0", "1"):
        got = []
        for slots in ("3", "2"):
            monkeypatch.setenv("HH_ENGINE_SLOTS", slots)
            monkeypatch.setenv("HH_ENGINE_OVERLAP", overlap)
            with hh.Context(d, nx, ntau, precision=precision, cheb_degree=cheb, cheb_eps=1e-3) as ctx:
                ctx.set_field(dev(sigma))
                x = torch.zeros(2, n, dtype=torch.float64, device="cuda")
                rc, info = ctx.solve(dev(b), x, 2)
                got.append((rc, info, x.cpu().numpy()))
        (rc3, i3, x3), (rc2, i2, x2) = got
        assert rc3 == 0 and rc2 == 0
        assert np.array_equal(x3, x2)
        assert i3["iterations"] == i2["iterations"] and i3["true_relres"] == i2["true_relres"]
        for a in range(2):
            res = b[a] - oracle.apply_MTM(lat, H, L, x3[a])
            assert np.linalg.norm(res) <= 1.0001e-10 * np.linalg.norm(b[a])
        by_layout[overlap] = x3
    assert np.linalg.norm(by_layout["0"] - by_layout["1"]) <= 1e-4 * np.linalg.norm(by_layout["0"])


def test_two_and_three_slot_forms_agree_through_fp64_fallback(hh, monkeypatch):
    """A mixed solve on the d = 1, 1024 x 512 lattice stalls in FP32 and
    continues in FP64 steps (Sec. 4.1 solver with FP32 inner iterations); both
    forms take the same path through the switch."""
    wl = workloads.C1
    n = wl.nsites
    sigma = workloads.sigma_field(n, seed=wl.seed)
    b = workloads.source(n, seed=1)[None, :]
    got = []
    for slots in ("3", "2"):
        monkeypatch.setenv("HH_ENGINE_SLOTS", slots)
        with hh.Context(wl.d, wl.nx, wl.ntau, precision="mixed") as ctx:
            ctx.set_field(dev(sigma))
            x = torch.zeros(1, n, dtype=torch.float64, device="cuda")
            ctx.counters_reset(True)
            rc, info = ctx.solve(dev(b), x, 1)
            got.append((rc, info, ctx.counters(), x.cpu().numpy()))
    (rc3, i3, c3, x3), (rc2, i2, c2, x2) = got
    assert rc3 == 0 and rc2 == 0 and i3["true_relres"] <= 1e-10
    assert c3["fp64_steps"] > 0
    assert np.array_equal(x3, x2)
    assert i3["iterations"] == i2["iterations"]
    assert c3["ru_steps"] == c2["ru_steps"] and c3["fp64_steps"] == c2["fp64_steps"]


def test_chebyshev_pcg_iteration_cap_reports_no_convergence(hh):
    """The cap counts PCG steps; each is followed by 2n preconditioner
    sub-steps (Sec. 4.2), which must not exhaust the engine before it."""
    d, nx, ntau = 1, 32, 64
    n = nx * ntau
    with hh.Context(d, nx, ntau, cg_maxit=7, cheb_degree=8, cheb_eps=1e-3) as ctx:
        ctx.set_field(dev(workloads.sigma_field(n, seed=31)))
        x = torch.zeros(1, n, dtype=torch.float64, device="cuda")
        rc, info = ctx.solve(dev(workloads.source(n, seed=32))[None, :], x, 1,
                             allow=(hh.binding.HH_ENOCONV,))
    assert rc == hh.binding.HH_ENOCONV and info["converged"] == 0 and info["iterations"] == 7


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_omelyan_trajectories_match_oracle(hh, precision):
    """The second-order minimum-norm integrator (2 n_md + 1 forces): energies,
    accept decisions and fields of the oracle's trajectories."""
    wl = workloads.C0
    lat = oracle.lattice(wl.d, wl.nx, wl.ntau)
    n = wl.nsites
    sigma = workloads.sigma_field(n, seed=wl.seed)
    prm = oracle.params(seed=wl.seed, n_pf=2, integrator=1)
    n_md, dt = 3, 0.1
    s_ref = sigma.copy()
    with hh.Context(wl.d, wl.nx, wl.ntau, seed=wl.seed, n_pf=2, precision=precision,
                    integrator="omelyan") as ctx:
        ctx.set_field(dev(sigma))
        for traj in range(3):
            info = ctx.trajectory(n_md, dt, traj)
            s_ref, oinfo = oracle.trajectory(lat, prm, s_ref, n_md, dt, traj)
            assert info["n_solves"] == 2 * (2 * n_md + 1)
            assert info["max_true_relres"] <= 1e-10
            assert info["u"] == oinfo["u"]
            assert abs(info["H0"] - oinfo["H0"]) <= 1e-8 * abs(oinfo["H0"])
            assert abs(info["dH"] - oinfo["dH"]) <= 1e-6, (info, oinfo)
            if abs(oinfo["dH"] + np.log(oinfo["u"])) > 1e-5:
                assert info["accepted"] == oinfo["accepted"]
            if info["accepted"] != oinfo["accepted"]:
                break
            got = torch.empty(n, dtype=torch.float64, device="cuda")
            ctx.get_field(got)
            assert np.max(np.abs(got.cpu().numpy() - s_ref)) <= 1e-6


def test_omelyan_reversible_on_gpu(hh):
    d, nx, ntau = 1, 16, 24
    n = nx * ntau
    sigma = workloads.sigma_field(n, seed=91)
    pi = workloads.unit_normal(n, seed=92, stream=1)
    chi = np.stack([workloads.unit_normal(n, seed=93, stream=2 + a) for a in range(2)])
    with hh.Context(d, nx, ntau, integrator="omelyan", cg_tol=1e-12) as ctx:
        ctx.set_field(dev(sigma))
        p = dev(pi)
        ctx.leapfrog(p, dev(chi), 2, 6, 0.08)
        mid = torch.empty(n, dtype=torch.float64, device="cuda")
        ctx.get_field(mid)
        p.neg_()
        ctx.leapfrog(p, dev(chi), 2, 6, 0.08)
        back = torch.empty(n, dtype=torch.float64, device="cuda")
        ctx.get_field(back)
    assert np.max(np.abs(mid.cpu().numpy() - sigma)) > 1e-3
    assert np.max(np.abs(back.cpu().numpy() - sigma)) <= 1e-8
    assert np.max(np.abs(p.cpu().numpy() + pi)) <= 1e-8


def test_batched_omelyan_trajectory_matches_context(hh):
    from paper_1007_3432_gb300 import binding as B
    d, nx, nt, seed = 1, 16, 16, 95
    n = nx * nt
    sigma = workloads.sigma_field(n, seed=seed)
    out = np.zeros(n)
    batch = B.Batch(max_slots=2, hbm_budget_bytes=1 << 28, chunk_iters=32, tile_sites=1024)
    req = B.make_request(B.HH_REQ_TRAJECTORY, d, nx, nt, sigma=sigma, out=out, n_md=3, dt=0.1, traj_index=4,
                         precision="fp64", seed=seed, n_pf=2, integrator="omelyan")
    batch.submit(req, keep=(sigma, out))
    r = batch.run_until_idle()[0]
    batch.close()
    assert r["status"] == 0 and r["n_solves"] == 2 * 7
    with hh.Context(d, nx, nt, seed=seed, n_pf=2, integrator="omelyan") as ctx:
        ctx.set_field(dev(sigma))
        info = ctx.trajectory(3, 0.1, 4)
    assert abs(info["dH"] - r["dH"]) <= 1e-6 and info["u"] == r["u"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_from_initial_guess(hh, precision):
    """hh_solve_guess: from a guess near the dense-LU solution the solve takes
    few steps and meets the true residual; the oracle's CG from the same guess
    agrees; b = 0 gives x = 0 whatever the guess."""
    d, nx, ntau = 1, 16, 12
    n = nx * ntau
    lat = oracle.lattice(d, nx, ntau)
    sigma = workloads.sigma_field(n, seed=120)
    L = oracle.links(lat, A, sigma)
    b = np.stack([workloads.source(n, seed=121, rhs=a) for a in range(2)])
    Q = oracle.dense(lat, H, L, "MTM")
    x_lu = np.linalg.solve(Q, b.T).T
    rng = np.random.default_rng(122)
    x0 = x_lu + 1e-6 * rng.standard_normal(x_lu.shape) * np.abs(x_lu).max()
    with hh.Context(d, nx, ntau, precision=precision) as ctx:
        ctx.set_field(dev(sigma))
        x = dev(x0.copy())
        rc, info = ctx.solve(dev(b), x, 2, guess=True)
        xg = x.cpu().numpy()
        x_zero = torch.zeros(2, n, dtype=torch.float64, device="cuda")
        rc0, info0 = ctx.solve(dev(b), x_zero, 2)
        xb = dev(rng.standard_normal((2, n)))
        rcz, infoz = ctx.solve(torch.zeros(2, n, dtype=torch.float64, device="cuda"), xb, 2, guess=True)
        assert rcz == 0 and not torch.any(xb)
    assert rc == 0 and info["converged"] == 1 and info["true_relres"] <= 1e-10
    assert info["iterations"] < 0.7 * info0["iterations"], (info, info0)
    for a in range(2):
        res = b[a] - oracle.apply_MTM(lat, H, L, xg[a])
        assert np.linalg.norm(res) <= 1.0001e-10 * np.linalg.norm(b[a])
        xo, st, it, rr = oracle.cg_guess(lat, H, L, b[a], x0[a])
        assert st == 0 and np.linalg.norm(xg[a] - xo) <= 1e-4 * np.linalg.norm(xo)
        if precision == "fp64":
            assert abs(info["iterations"] - it) <= 2 + 0.05 * it or a == 0


@pytest.mark.parametrize("chrono", [1, 2])
def test_chronological_guess_trajectory_matches_oracle(hh, chrono):
    wl = workloads.C0
    lat = oracle.lattice(wl.d, wl.nx, wl.ntau)
    n = wl.nsites
    sigma = workloads.sigma_field(n, seed=wl.seed)
    prm = oracle.params(seed=wl.seed, n_pf=2, chrono=chrono)
    n_md, dt = 5, 0.04
    with hh.Context(wl.d, wl.nx, wl.ntau, seed=wl.seed, n_pf=2, chrono=chrono) as ctx:
        ctx.set_field(dev(sigma))
        info = ctx.trajectory(n_md, dt, 0)
    with hh.Context(wl.d, wl.nx, wl.ntau, seed=wl.seed, n_pf=2) as ctx:
        ctx.set_field(dev(sigma))
        info0 = ctx.trajectory(n_md, dt, 0)
    _, oinfo = oracle.trajectory(lat, prm, sigma, n_md, dt, 0)
    assert info["max_true_relres"] <= 1e-10 and info["u"] == oinfo["u"]
    assert abs(info["dH"] - oinfo["dH"]) <= 1e-6 and abs(info["dH"] - info0["dH"]) <= 1e-6
    if abs(oinfo["dH"] + np.log(oinfo["u"])) > 1e-5:
        assert info["accepted"] == oinfo["accepted"] == info0["accepted"]
    assert info["cg_iterations"] < info0["cg_iterations"], (info, info0)


def test_batched_chronological_trajectory_matches_context(hh):
    from paper_1007_3432_gb300 import binding as B
    d, nx, nt, seed = 1, 16, 16, 97
    n = nx * nt
    sigma = workloads.sigma_field(n, seed=seed)
    out = np.zeros(n)
    batch = B.Batch(max_slots=2, hbm_budget_bytes=1 << 28, chunk_iters=32, tile_sites=1024)
    req = B.make_request(B.HH_REQ_TRAJECTORY, d, nx, nt, sigma=sigma, out=out, n_md=4, dt=0.1, traj_index=2,
                         precision="fp64", seed=seed, n_pf=2, chrono=2)
    batch.submit(req, keep=(sigma, out))
    r = batch.run_until_idle()[0]
    batch.close()
    assert r["status"] == 0
    with hh.Context(d, nx, nt, seed=seed, n_pf=2, chrono=2) as ctx:
        ctx.set_field(dev(sigma))
        info = ctx.trajectory(4, 0.1, 2)
    assert abs(info["dH"] - r["dH"]) <= 1e-6 and info["u"] == r["u"]


@pytest.mark.parametrize("d,nx,ntau,precision,order", [(1, 16, 16, "fp64", 0), (1, 16, 16, "mixed", 0),
                                                       (3, 4, 8, "fp64", 0), (1, 12, 10, "fp64", 1),
                                                       (3, 4, 6, "mixed", 2)])
def test_observables_match_oracle(hh, d, nx, ntau, precision, order):
    """hh_observables against the oracle's estimators on the same Z2 noise
    (Philox tag 6): the noise is bit-identical, the solves agree to the CG
    tolerance, so the estimates agree to the solution error."""
    lat = oracle.lattice(d, nx, ntau)
    n = oracle.nsites(lat)
    sigma = workloads.sigma_field(n, seed=900 + nx)
    ref = oracle.observables(lat, oracle.params(seed=77, link_order=order), sigma, 6, 2)
    assert ref["status"] == 0
    with hh.Context(d, nx, ntau, seed=77, precision=precision, link_order=order) as ctx:
        ctx.set_field(dev(sigma))
        got = ctx.observables(6, 2)
    assert got["n_noise"] == 6 and got["max_true_relres"] <= 1e-10
    for key in ("trace_Minv", "one_minus_g_sq"):
        assert abs(got[key] - ref[key]) <= 1e-6 * abs(ref[key]) + 1e-9, key
    assert abs(got["trace_err"] - ref["trace_err"]) <= 1e-5 * ref["trace_err"] + 1e-9
    for key in ("mean_sin", "mean_sin2"):
        assert abs(got[key] - ref[key]) <= 1e-13, key


def test_observables_reject_bad_noise_counts(hh):
    with hh.Context(1, 8, 8) as ctx:
        for nn in (0, 1, 3, 66):
            with pytest.raises(hh.HHError):
                ctx.observables(nn, 0)


@pytest.mark.parametrize("precision", ["mixed-bf16link", "mixed-fix16link"])
def test_16bit_links_rejected_where_unsupported(hh, precision):
    with pytest.raises(hh.HHError):
        hh.Context(1, 8, 8, precision=precision, link_order=1)
    with pytest.raises(hh.HHError):
        hh.Context(1, 8, 8, precision=precision, cheb_degree=8)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_prefetch_leaves_results_bitwise_unchanged(hh, monkeypatch, precision):
    """The L2 prefetch of the CG site loops is a hint: solutions are bitwise
    the same at every distance.  16^3 x 80 gives tiles of two or more loop
    rounds, so the prefetches are issued."""
    from paper_1007_3432_gb300.binding import HH_ENOCONV
    d, nx, ntau = 3, 16, 80
    n = nx ** 3 * ntau
    sigma = workloads.sigma_field(n, seed=41)
    b = np.stack([workloads.source(n, seed=42, rhs=a) for a in range(2)])
    outs = []
    for pf in ("0", "1", "3"):
        monkeypatch.setenv("HH_ENGINE_PREFETCH", pf)
        with hh.Context(d, nx, ntau, precision=precision, cg_maxit=300) as ctx:
            ctx.set_field(dev(sigma))
            x = torch.zeros(2, n, dtype=torch.float64, device="cuda")
            ctx.solve(dev(b), x, 2, allow=(HH_ENOCONV,))
            outs.append(x.cpu())
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_dependent_launch_leaves_apply_bitwise_unchanged(hh, monkeypatch, dtype):
    """The two Q sweeps with and without the programmatic dependent launch."""
    d, nx, ntau = 3, 8, 12
    n = nx ** 3 * ntau
    sigma = workloads.sigma_field(n, seed=43)
    x = dev(workloads.source(n, seed=44)).to(dtype)
    outs = []
    for path in ("1", "2"):
        monkeypatch.setenv("HH_APPLY_MTM", path)
        with hh.Context(d, nx, ntau) as ctx:
            ctx.set_field(dev(sigma))
            y = torch.empty_like(x)
            ctx.apply(hh.HH_OP_MTM, x, y)
            outs.append(y.cpu())
    assert torch.equal(outs[0], outs[1])
