"""The metrics log on the GPU paths: a context writes one record per solve
and per trajectory with the solver's figures, and a batch one record per
polled result with the queue depth at that poll."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def test_context_and_batch_records(hh, tmp_path):
    from paper_1007_3432_gb300 import binding as B
    path = tmp_path / "metrics.jsonl"
    d, nx, nt = 1, 32, 16
    n = nx * nt
    sigma = workloads.sigma_field(n, seed=31)
    b = np.stack([workloads.source(n, seed=32, rhs=a) for a in range(2)])
    with hh.Context(d, nx, nt, seed=33, n_pf=2, log=str(path)) as ctx:
        ctx.set_field(torch.from_numpy(sigma).cuda())
        bd = torch.from_numpy(b).cuda()
        x = torch.zeros_like(bd)
        rc, info = ctx.solve(bd, x, 2)
        tinfo = ctx.trajectory(3, 0.05, 0)
        ctx.log.close()
    log = B.MetricsLog(str(path))
    with B.Batch(max_slots=2, hbm_budget_bytes=1 << 28, chunk_iters=16, tile_sites=512, log=log) as batch:
        out = np.zeros((2, n))
        batch.submit(B.make_request(B.HH_REQ_SOLVE, d, nx, nt, sigma=sigma, b=b, out=out, n_pf=2),
                     keep=(sigma, b, out))
        res = batch.run_until_idle()
    log.close()
    recs = [json.loads(l) for l in path.read_text().splitlines()]
    kinds = [r["record"] for r in recs]
    assert kinds == ["solve", "trajectory", "result"], kinds
    s, t, r = recs
    assert s["iterations"] == info["iterations"] and s["true_relres"] == info["true_relres"] and s["status"] == 0
    assert (s["d"], s["nx"], s["ntau"], s["n_rhs"]) == (d, nx, nt, 2)
    assert t["dH"] == tinfo["dH"] and t["accepted"] == tinfo["accepted"] and t["n_md"] == 3
    assert r["status"] == 0 and r["ticket"] == res[0]["ticket"] and r["cg_iterations"] == res[0]["cg_iterations"]
    assert r["queued"] >= 0 and r["active"] >= 0
