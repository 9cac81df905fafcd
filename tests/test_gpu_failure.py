"""Failure detection on the GPU, injected without faulting or hanging it.

* A device-side wait that runs out: the test makes the engine drop one tile's
  partial-sum signal (HH_ENGINE_DROP_SIGNAL, a signal that nothing sets) or
  makes the multi-vector apply expect 16 bytes more than its first stage
  copies (HH_APPLY_MULTI_DROP_TX), with a short wait budget (hh_set_timeout,
  hh_batch_set_timeout).  Every wait on it runs out, the kernel records
  HH_ETIMEOUT and leaves; the call returns that status, and the same context
  (batch) then solves correctly with the injection removed.
* A NaN in the auxiliary field: the links, hence |M p|^2, become NaN, and the
  engine's decision turns it into HH_ENUMERIC for hh_solve and for a batched
  request, without affecting the other requests of the batch.
* A forced iteration cap is covered by test_gpu_parity (HH_ENOCONV).
"""
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


def _check_solution(d, nx, ntau, sigma, b, x):
    lat = oracle.lattice(d, nx, ntau)
    L = oracle.links(lat, workloads.A_HS, sigma)
    for a in range(b.shape[0]):
        res = b[a] - oracle.apply_MTM(lat, H, L, x[a])
        assert np.linalg.norm(res) <= 1.0001e-10 * np.linalg.norm(b[a])


# (precision, Nx, Ntau): 98k-site systems share the grid in the flat engine
# form; 332k-site FP64 systems are each tiled over the whole grid, with the
# control warp (overlapped layout).
@pytest.mark.parametrize("precision,nx,ntau", [("fp64", 16, 24), ("mixed", 16, 24), ("fp64", 24, 24)])
def test_engine_wait_runs_out_then_context_recovers(hh, monkeypatch, precision, nx, ntau):
    from paper_1007_3432_gb300.binding import HH_ETIMEOUT
    d = 3
    n = nx ** d * ntau
    sigma = workloads.sigma_field(n, seed=901)
    b = np.stack([workloads.source(n, seed=902, rhs=a) for a in range(2)])
    with hh.Context(d, nx, ntau, precision=precision) as ctx:
        ctx.set_field(torch.from_numpy(sigma).cuda())
        b_d = torch.from_numpy(b).cuda()
        x = torch.zeros_like(b_d)
        ctx.set_timeout(0.05)
        monkeypatch.setenv("HH_ENGINE_DROP_SIGNAL", "1")      # tile partial 0 is never published
        rc, info = ctx.solve(b_d, x, 2, allow=(HH_ETIMEOUT,))
        assert rc == HH_ETIMEOUT and info["converged"] == 0, (rc, info)
        monkeypatch.delenv("HH_ENGINE_DROP_SIGNAL")
        ctx.set_timeout(5.0)
        rc, info = ctx.solve(b_d, x, 2)
        assert rc == 0 and info["converged"] == 1 and info["true_relres"] <= 1e-10, info
        _check_solution(d, nx, ntau, sigma, b, x.cpu().numpy())


@pytest.mark.parametrize("form", ["5", "2"])
def test_multi_apply_wait_runs_out_then_recovers(hh, monkeypatch, form):
    """The multi-vector apply's bounded waits for its bulk copies: when the
    first stage's barrier cannot complete, the kernel records HH_ETIMEOUT
    (reported by hh_counters_get), waits (bounded) for the copies it issued
    and leaves; without the injection the same context's apply matches the
    oracle.  In the row-pair form (5) and the one-row form (2)."""
    from paper_1007_3432_gb300.binding import HH_ETIMEOUT, HHError
    monkeypatch.setenv("HH_APPLY_MULTI_FORM", form)
    d, nx, ntau, k = 3, 32, 10, 3
    n = nx ** d * ntau
    sigma = workloads.sigma_field(n, seed=903)
    xs = np.stack([workloads.source(n, seed=904, rhs=a) for a in range(k)]).astype(np.float32)
    with hh.Context(d, nx, ntau) as ctx:
        ctx.set_field(torch.from_numpy(sigma).cuda())
        x_d = torch.from_numpy(xs.reshape(-1)).cuda()
        y_d = torch.zeros_like(x_d)
        ctx.set_timeout(0.05)
        monkeypatch.setenv("HH_APPLY_MULTI_DROP_TX", "1")
        ctx.apply_multi(hh.HH_OP_MTM, x_d, y_d, k)
        with pytest.raises(HHError) as e:
            ctx.counters()
        assert e.value.code == HH_ETIMEOUT
        monkeypatch.delenv("HH_APPLY_MULTI_DROP_TX")
        ctx.counters_reset()             # clears the recorded error
        ctx.set_timeout(5.0)
        ctx.apply_multi(hh.HH_OP_MTM, x_d, y_d, k)
        ctx.counters()
        got = y_d.cpu().numpy().reshape(k, n).astype(np.float64)
    lat = oracle.lattice(d, nx, ntau)
    L = oracle.links(lat, workloads.A_HS, sigma)
    La = np.abs(L)
    for v in range(k):
        x64 = xs[v].astype(np.float64)
        ref = oracle.apply_MTM(lat, H, L, x64)
        bound = 2e-6 * oracle.apply_MT(lat, -H, La, oracle.apply_M(lat, -H, La, np.abs(x64)))
        assert np.all(np.abs(got[v] - ref) <= bound)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nan_field_gives_enumeric_then_context_recovers(hh, precision):
    from paper_1007_3432_gb300.binding import HH_ENUMERIC
    d, nx, ntau = 1, 64, 32
    n = nx * ntau
    sigma = workloads.sigma_field(n, seed=905)
    bad = sigma.copy()
    bad[n // 3] = np.nan
    b = np.stack([workloads.source(n, seed=906, rhs=a) for a in range(2)])
    with hh.Context(d, nx, ntau, precision=precision) as ctx:
        b_d = torch.from_numpy(b).cuda()
        x = torch.zeros_like(b_d)
        ctx.set_field(bad)                       # host copy, NaN at one site
        rc, info = ctx.solve(b_d, x, 2, allow=(HH_ENUMERIC,))
        assert rc == HH_ENUMERIC and info["converged"] == 0, (rc, info)
        ctx.set_field(sigma)
        rc, info = ctx.solve(b_d, x, 2)
        assert rc == 0 and info["true_relres"] <= 1e-10, info
        _check_solution(d, nx, ntau, sigma, b, x.cpu().numpy())


def test_batch_nan_request_fails_alone(hh):
    """A request whose field holds a NaN ends with HH_ENUMERIC; the other
    requests of the same batch are unaffected (bitwise the same as alone)."""
    from paper_1007_3432_gb300 import binding as B
    from paper_1007_3432_gb300.binding import HH_ENUMERIC, HH_REQ_SOLVE

    def req(d, nx, ntau, seed, poison):
        n = nx ** d * ntau
        sigma = workloads.sigma_field(n, seed=seed)
        if poison:
            sigma[n // 2] = np.nan
        b = np.stack([workloads.source(n, seed=seed, rhs=a) for a in range(2)])
        out = np.zeros((2, n))
        return B.make_request(HH_REQ_SOLVE, d, nx, ntau, sigma=sigma, b=b, out=out, precision="mixed",
                              n_pf=2), (sigma, b, out)

    good = [(1, 40, 32, 911), (3, 8, 12, 912)]
    alone = []
    for d, nx, nt, seed in good:
        with B.Batch(max_slots=4, hbm_budget_bytes=1 << 30, chunk_iters=16, tile_sites=1024) as batch:
            r, keep = req(d, nx, nt, seed, False)
            batch.submit(r, keep=keep)
            res = batch.run_until_idle()
            assert res[0]["status"] == 0
            alone.append(keep[2].copy())
    with B.Batch(max_slots=4, hbm_budget_bytes=1 << 30, chunk_iters=16, tile_sites=1024) as batch:
        keeps = []
        for j, (d, nx, nt, seed) in enumerate(good):
            r, keep = req(d, nx, nt, seed, False)
            batch.submit(r, keep=keep)
            keeps.append(keep)
            if j == 0:
                rb, kb = req(3, 6, 8, 913, True)
                batch.submit(rb, keep=kb)
        res = {r["ticket"]: r for r in batch.run_until_idle()}
    assert res[2]["status"] == HH_ENUMERIC, res[2]
    for t, keep, ref in zip((1, 3), keeps, alone):
        assert res[t]["status"] == 0 and res[t]["max_true_relres"] <= 1e-10, res[t]
        assert np.array_equal(keep[2], ref)


def test_batch_wait_runs_out_then_batch_recovers(hh, monkeypatch):
    from paper_1007_3432_gb300 import binding as B
    from paper_1007_3432_gb300.binding import HH_ETIMEOUT, HH_REQ_SOLVE
    d, nx, ntau = 3, 12, 16
    n = nx ** d * ntau
    sigma = workloads.sigma_field(n, seed=921)
    b = np.stack([workloads.source(n, seed=922, rhs=a) for a in range(2)])
    with B.Batch(max_slots=4, hbm_budget_bytes=1 << 30, chunk_iters=16, tile_sites=512) as batch:
        batch.set_timeout(0.05)
        monkeypatch.setenv("HH_ENGINE_DROP_SIGNAL", "1")
        out1 = np.zeros((2, n))
        batch.submit(B.make_request(HH_REQ_SOLVE, d, nx, ntau, sigma=sigma, b=b, out=out1, precision="fp64",
                                    n_pf=2), keep=(sigma, b, out1))
        res = batch.run_until_idle(allow=(HH_ETIMEOUT,))
        assert len(res) == 1 and res[0]["status"] == HH_ETIMEOUT, res
        monkeypatch.delenv("HH_ENGINE_DROP_SIGNAL")
        batch.set_timeout(5.0)
        out2 = np.zeros((2, n))
        batch.submit(B.make_request(HH_REQ_SOLVE, d, nx, ntau, sigma=sigma, b=b, out=out2, precision="fp64",
                                    n_pf=2), keep=(sigma, b, out2))
        res = batch.run_until_idle()
        assert len(res) == 1 and res[0]["status"] == 0 and res[0]["max_true_relres"] <= 1e-10, res
    _check_solution(d, nx, ntau, sigma, b, out2)


def test_timeout_argument_checks(hh):
    from paper_1007_3432_gb300.binding import HH_EINVAL, HHError
    with hh.Context(1, 8, 4) as ctx:
        for bad in (-1.0, 1e9, float("nan")):
            with pytest.raises(HHError) as e:
                ctx.set_timeout(bad)
            assert e.value.code == HH_EINVAL
