"""GPU tests of the batched multi-chain engine and the serving loop.

* every batched solve meets the FP64 true residual 1e-10 (recomputed by the
  oracle) and agrees with the single-context solver within the solver
  tolerance;
* a request's result is bit-for-bit the same alone and in a mix of other
  lattices, precisions and kinds (fixed per-system tiling, fixed-order
  reductions);
* batched trajectories reproduce the single-context trajectories (energies,
  accept decisions, final field);
* admission under a small HBM budget queues requests and still completes
  them; a request larger than the budget is refused;
* the background worker admits requests that arrive while others run.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads  # noqa: E402

H = workloads.T_HOP * workloads.DTAU


@pytest.fixture(scope="module")
def hh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1007_3432_gb300 as pkg
    from paper_1007_3432_gb300 import build
    build.build()
    pkg.load()
    return pkg


def _solve_req(B, d, nx, ntau, seed, precision="fp64", n_rhs=2):
    from paper_1007_3432_gb300.binding import HH_REQ_SOLVE
    n = nx ** d * ntau
    sigma = workloads.sigma_field(n, seed=seed)
    b = np.stack([workloads.source(n, seed=seed, rhs=a) for a in range(n_rhs)])
    out = np.zeros((n_rhs, n))
    req = B.make_request(HH_REQ_SOLVE, d, nx, ntau, sigma=sigma, b=b, out=out, precision=precision,
                         n_pf=n_rhs)
    return req, (sigma, b, out)


def _traj_req(B, d, nx, ntau, seed, n_md, dt, traj, precision="fp64"):
    from paper_1007_3432_gb300.binding import HH_REQ_TRAJECTORY
    n = nx ** d * ntau
    sigma = workloads.sigma_field(n, seed=seed)
    out = np.zeros(n)
    req = B.make_request(HH_REQ_TRAJECTORY, d, nx, ntau, sigma=sigma, out=out, n_md=n_md, dt=dt,
                         traj_index=traj, precision=precision, seed=seed, n_pf=2)
    return req, (sigma, out)


MIX = [(1, 32, 64, 11, "fp64"), (3, 6, 8, 12, "mixed"), (1, 48, 24, 13, "mixed"), (3, 8, 10, 14, "fp64"),
       (1, 19, 16, 15, "fp64")]


def test_batched_solves_match_context_solver(hh):
    from paper_1007_3432_gb300 import binding as B
    batch = B.Batch(max_slots=8, hbm_budget_bytes=1 << 30, chunk_iters=16, tile_sites=1024)
    keep = []
    for d, nx, nt, seed, prec in MIX:
        req, k = _solve_req(B, d, nx, nt, seed, prec)
        keep.append((d, nx, nt, seed, prec, k))
        batch.submit(req, keep=k)
    res = {r["ticket"]: r for r in batch.run_until_idle()}
    batch.close()
    assert len(res) == len(MIX)
    for ticket, (d, nx, nt, seed, prec, (sigma, b, out)) in enumerate(keep, start=1):
        r = res[ticket]
        assert r["status"] == 0 and r["n_solves"] == 2 and r["max_true_relres"] <= 1e-10, r
        lat = oracle.lattice(d, nx, nt)
        L = oracle.links(lat, workloads.A_HS, sigma)
        for a in range(2):
            res_a = b[a] - oracle.apply_MTM(lat, H, L, out[a])
            assert np.linalg.norm(res_a) <= 1.0001e-10 * np.linalg.norm(b[a])
        with hh.Context(d, nx, nt, precision=prec) as ctx:
            ctx.set_field(torch.from_numpy(sigma).cuda())
            x = torch.zeros(2, nx ** d * nt, dtype=torch.float64, device="cuda")
            ctx.solve(torch.from_numpy(b).cuda(), x, 2)
            assert np.linalg.norm(x.cpu().numpy() - out) <= 1e-4 * np.linalg.norm(out)


def test_result_is_identical_alone_and_in_the_mix(hh):
    from paper_1007_3432_gb300 import binding as B
    outs = []
    for with_mix in (False, True):
        batch = B.Batch(max_slots=8, hbm_budget_bytes=1 << 30, chunk_iters=16, tile_sites=1024)
        if with_mix:
            for d, nx, nt, seed, prec in MIX[1:]:
                req, k = _solve_req(B, d, nx, nt, seed, prec)
                batch.submit(req, keep=k)
            treq, tk = _traj_req(B, 1, 16, 12, 71, 3, 0.1, 5)
            batch.submit(treq, keep=tk)
        d, nx, nt, seed, prec = MIX[0]
        req, k = _solve_req(B, d, nx, nt, seed, "mixed")
        batch.submit(req, keep=k)
        treq2, tk2 = _traj_req(B, 1, 16, 16, 72, 4, 0.1, 2)
        batch.submit(treq2, keep=tk2)
        res = batch.run_until_idle()
        batch.close()
        assert all(r["status"] == 0 for r in res)
        traj = [r for r in res if r["kind"] == 1 and r["n_solves"] == 2 * 5][0]
        outs.append((k[2].copy(), tk2[1].copy(), traj["dH"], traj["accepted"]))
    (xa, sa, dha, acca), (xb, sb, dhb, accb) = outs
    assert np.array_equal(xa, xb)
    assert np.array_equal(sa, sb)
    assert dha == dhb and acca == accb


def test_many_systems_per_block_uncached_path(hh):
    """80 two-source requests of 40 tiles each: 6400 tiles over one block per
    SM, so every block holds tiles of more distinct systems than its
    shared-memory cache (32) and runs the uncached path, which re-reads each
    system's state from global memory after the wait that orders it.  Every
    request converges to the FP64 true residual, and two of them agree bit
    for bit with the same request run alone (where the block caches)."""
    from paper_1007_3432_gb300 import binding as B
    d, nx, nt = 3, 8, 40                       # 20480 sites = 40 tiles of 512
    specs = [(1000 + j, "mixed" if j % 2 else "fp64") for j in range(80)]
    alone = {}
    for j in (0, 1):
        with B.Batch(max_slots=2, hbm_budget_bytes=1 << 30, chunk_iters=32, tile_sites=512) as batch:
            req, k = _solve_req(B, d, nx, nt, *specs[j])
            batch.submit(req, keep=k)
            res = batch.run_until_idle()
            assert res[0]["status"] == 0, res
            alone[j] = k[2].copy()
    keeps = []
    with B.Batch(max_slots=80, hbm_budget_bytes=4 << 30, chunk_iters=32, tile_sites=512) as batch:
        for seed, prec in specs:
            req, k = _solve_req(B, d, nx, nt, seed, prec)
            batch.submit(req, keep=k)
            keeps.append(k)
        res = {r["ticket"]: r for r in batch.run_until_idle()}
    assert len(res) == len(specs)
    for t in range(1, len(specs) + 1):
        assert res[t]["status"] == 0 and res[t]["max_true_relres"] <= 1e-10, res[t]
    for j in (0, 1):
        assert np.array_equal(keeps[j][2], alone[j])
    sigma, b, out = keeps[5]
    lat = oracle.lattice(d, nx, nt)
    L = oracle.links(lat, workloads.A_HS, sigma)
    for a in range(2):
        assert np.linalg.norm(b[a] - oracle.apply_MTM(lat, H, L, out[a])) <= 1.0001e-10 * np.linalg.norm(b[a])


def test_batched_trajectories_match_context(hh):
    from paper_1007_3432_gb300 import binding as B
    cases = [(1, 16, 16, 81, 4, 0.1, 0), (3, 4, 6, 82, 3, 0.1, 1), (1, 32, 64, 83, 5, 0.04, 2)]
    batch = B.Batch(max_slots=4, hbm_budget_bytes=1 << 30, chunk_iters=32, tile_sites=2048)
    keep = []
    for d, nx, nt, seed, n_md, dt, traj in cases:
        req, k = _traj_req(B, d, nx, nt, seed, n_md, dt, traj)
        keep.append(k)
        batch.submit(req, keep=k)
    res = {r["ticket"]: r for r in batch.run_until_idle()}
    batch.close()
    for ticket, ((d, nx, nt, seed, n_md, dt, traj), (sigma, out)) in enumerate(zip(cases, keep), start=1):
        r = res[ticket]
        assert r["status"] == 0 and r["n_solves"] == 2 * (n_md + 1)
        with hh.Context(d, nx, nt, seed=seed, n_pf=2) as ctx:
            ctx.set_field(torch.from_numpy(sigma).cuda())
            info = ctx.trajectory(n_md, dt, traj)
            s_ctx = torch.empty(nx ** d * nt, dtype=torch.float64, device="cuda")
            ctx.get_field(s_ctx)
        assert abs(info["dH"] - r["dH"]) <= 1e-6 and info["u"] == r["u"]
        assert abs(info["H0"] - r["H0"]) <= 1e-9 * abs(info["H0"])
        if abs(info["dH"] + np.log(info["u"])) > 1e-5:
            assert info["accepted"] == r["accepted"]
            assert np.max(np.abs(s_ctx.cpu().numpy() - out)) <= 1e-7


def test_budget_admission_and_refusal(hh):
    from paper_1007_3432_gb300 import binding as B
    # Each d=1, 64 x 64 request needs about 0.6 MB; a 2 MB budget admits a few at a time.
    batch = B.Batch(max_slots=8, hbm_budget_bytes=2 << 20, chunk_iters=64, tile_sites=1024)
    for j in range(6):
        req, k = _solve_req(B, 1, 64, 64, 200 + j, "fp64", n_rhs=1)
        batch.submit(req, keep=k)
    big, kb = _solve_req(B, 1, 256, 512, 300, "fp64", n_rhs=1)
    rc, _ = batch.submit(big, keep=kb, allow=(B.HH_EBUSY,))
    assert rc == B.HH_EBUSY
    q, a = batch.pending()
    assert q == 6 and a == 0
    batch.step()
    q, a = batch.pending()
    assert a >= 1 and q >= 1 and q + a <= 6
    res = batch.run_until_idle()
    batch.close()
    assert len(res) == 6 and all(r["status"] == 0 for r in res)
    assert max(r["queue_ms"] for r in res) > 0.0


def test_worker_admits_requests_arriving_during_work(hh):
    from paper_1007_3432_gb300 import binding as B
    batch = B.Batch(max_slots=16, hbm_budget_bytes=1 << 30, chunk_iters=16, tile_sites=1024)
    batch.start()
    keep = []
    arrivals = workloads.poisson_requests(200.0, 10, seed=5, d1_nx=(16, 48), d1_ntau=(16, 64),
                                          d3_nx=(4, 6), d3_ntau=(8, 16))
    t0 = time.perf_counter()
    for r in arrivals:
        while time.perf_counter() - t0 < r.arrival_s:
            time.sleep(0.0005)
        if r.kind == "solve":
            req, k = _solve_req(B, r.d, r.nx, r.ntau, r.seed % 100000, "mixed", n_rhs=1)
        else:
            req, k = _traj_req(B, r.d, r.nx, r.ntau, r.seed % 100000, 2, 0.1, r.rid)
        keep.append((r, k))
        batch.submit(req, keep=k)
    got = []
    deadline = time.perf_counter() + 120
    while len(got) < len(arrivals) and time.perf_counter() < deadline:
        got += batch.poll()
        time.sleep(0.002)
    batch.stop()
    batch.close()
    assert len(got) == len(arrivals)
    assert all(g["status"] == 0 and g["latency_ms"] > 0 for g in got)
    assert all(g["max_true_relres"] <= 1e-10 for g in got)
    # Each served solve matches a standalone batched solve of the same request.
    for r, k in keep[:4]:
        if r.kind != "solve":
            continue
        solo = B.Batch(max_slots=1, hbm_budget_bytes=1 << 28, chunk_iters=16, tile_sites=1024)
        req, k2 = _solve_req(B, r.d, r.nx, r.ntau, r.seed % 100000, "mixed", n_rhs=1)
        solo.submit(req, keep=k2)
        solo.run_until_idle()
        solo.close()
        assert np.array_equal(k2[2], k[2])


def test_autotuner_returns_a_candidate(hh, tmp_path):
    from paper_1007_3432_gb300 import binding as B
    reqs, keep = [], []
    for j in range(3):
        req, k = _solve_req(B, 3, 8, 16, 400 + j, "mixed")
        reqs.append(req)
        keep.append(k)
    cache = str(tmp_path / "tune.jsonl")
    best = B.autotune(reqs, hbm_budget_bytes=1 << 29, rounds=3, cache_path=cache)
    assert best["tile_sites"] in (2048, 8192) and best["chunk_iters"] in (16, 64)
    assert '"tile_sites"' in open(cache).read()


def test_batched_chebyshev_pcg_matches_context(hh):
    """FP64 requests with the Chebyshev preconditioner (Sec. 4.2) in the batch:
    true residual 1e-10 by the oracle, the context solver's PCG solution within
    the solver tolerance, and the same bits alone and next to plain-CG and
    mixed requests."""
    from paper_1007_3432_gb300 import binding as B
    cases = [(1, 32, 64, 21, 4, 1e-3), (3, 6, 8, 22, 3, 1e-2)]

    def pcg_req(d, nx, nt, seed, deg, eps):
        n = nx ** d * nt
        sigma = workloads.sigma_field(n, seed=seed)
        b = np.stack([workloads.source(n, seed=seed, rhs=a) for a in range(2)])
        out = np.zeros((2, n))
        req = B.make_request(B.HH_REQ_SOLVE, d, nx, nt, sigma=sigma, b=b, out=out, precision="fp64", n_pf=2,
                             cheb_degree=deg, cheb_eps=eps)
        return req, (sigma, b, out)

    outs = []
    for with_mix in (False, True):
        batch = B.Batch(max_slots=8, hbm_budget_bytes=1 << 30, chunk_iters=16, tile_sites=1024)
        keep = []
        if with_mix:
            for d, nx, nt, seed, prec in MIX[:3]:
                req, k = _solve_req(B, d, nx, nt, seed, prec)
                batch.submit(req, keep=k)
        for c in cases:
            req, k = pcg_req(*c)
            keep.append(k)
            batch.submit(req, keep=k)
        res = batch.run_until_idle()
        batch.close()
        assert all(r["status"] == 0 for r in res), res
        outs.append([k[2].copy() for k in keep])
        if with_mix:
            continue
        for (d, nx, nt, seed, deg, eps), (sigma, b, out) in zip(cases, keep):
            lat = oracle.lattice(d, nx, nt)
            L = oracle.links(lat, workloads.A_HS, sigma)
            for a in range(2):
                res_a = b[a] - oracle.apply_MTM(lat, H, L, out[a])
                assert np.linalg.norm(res_a) <= 1.0001e-10 * np.linalg.norm(b[a])
            with hh.Context(d, nx, nt, cheb_degree=deg, cheb_eps=eps) as ctx:
                ctx.set_field(torch.from_numpy(sigma).cuda())
                x = torch.zeros(2, nx ** d * nt, dtype=torch.float64, device="cuda")
                ctx.solve(torch.from_numpy(b).cuda(), x, 2)
                assert np.linalg.norm(x.cpu().numpy() - out) <= 1e-4 * np.linalg.norm(out)
    for xa, xb in zip(*outs):
        assert np.array_equal(xa, xb)


def test_batched_chebyshev_rejected_for_mixed_precision(hh):
    from paper_1007_3432_gb300 import binding as B
    batch = B.Batch(max_slots=2, hbm_budget_bytes=1 << 26)
    n = 8 * 8
    req = B.make_request(B.HH_REQ_SOLVE, 1, 8, 8, sigma=np.zeros(n), precision="mixed", n_pf=1, cheb_degree=2)
    rc, _ = batch.submit(req, allow=(B.HH_EINVAL,))
    batch.close()
    assert rc == B.HH_EINVAL
