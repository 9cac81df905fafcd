"""Runs GPU parity cases through the index-checking debug build of the
library (HH_BOUNDS_CHECK=1 is set by the caller, so the binding loads
libhubhmc_check.so) and reports, as one JSON line, whether any index check
failed.  Started as a subprocess by tests/test_gpu_bounds_check.py."""
import json
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import oracle  # noqa: E402
import workloads  # noqa: E402
import paper_1007_3432_gb300 as hh  # noqa: E402
from paper_1007_3432_gb300 import binding as B  # noqa: E402

H = workloads.T_HOP * workloads.DTAU
OPS = {"M": (hh.HH_OP_M, oracle.apply_M), "MT": (hh.HH_OP_MT, oracle.apply_MT),
       "MTM": (hh.HH_OP_MTM, oracle.apply_MTM)}


def rel_err(got, ref):
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def main():
    out = {"checks": []}
    B.load()
    rc, enabled, rec = B.bounds_check(selftest=True)
    out["selftest"] = [rc, enabled, rec]
    rc, _, rec = B.bounds_check()
    out["after_selftest"] = [rc, rec]
    worst = {}
    # tiny lattices (N_x = 2, 3: wrap-around duplicates) and ordinary ones
    for d, nx, nt in [(1, 2, 4), (1, 3, 5), (1, 16, 8), (3, 2, 3), (3, 3, 4), (3, 4, 6), (3, 8, 5)]:
        lat = oracle.lattice(d, nx, nt)
        n = oracle.nsites(lat)
        sigma = workloads.sigma_field(n, seed=700 + 10 * d + nx)
        L = oracle.links(lat, workloads.A_HS, sigma)
        x = workloads.source(n, seed=800 + nx, rhs=0)
        with hh.Context(d, nx, nt) as ctx:
            ctx.set_field(torch.from_numpy(sigma).cuda())
            for name, (op, fn) in OPS.items():
                for dt in (np.float64, np.float32):
                    xd = torch.from_numpy(x.astype(dt)).cuda()
                    yd = torch.empty_like(xd)
                    ctx.apply(op, xd, yd)
                    e = rel_err(yd.cpu().numpy().astype(np.float64), fn(lat, H, L, x.astype(dt).astype(np.float64)))
                    key = "apply_%s_%s" % (name, "f64" if dt == np.float64 else "f32")
                    worst[key] = max(worst.get(key, 0.0), e)
        for prec in ("fp64", "mixed"):
            b = np.stack([workloads.source(n, seed=900 + nx, rhs=a) for a in range(2)])
            with hh.Context(d, nx, nt, precision=prec) as ctx:
                ctx.set_field(torch.from_numpy(sigma).cuda())
                bd = torch.from_numpy(b).cuda()
                xs = torch.zeros_like(bd)
                rc, info = ctx.solve(bd, xs, 2)
                xs = xs.cpu().numpy()
            res = max(np.linalg.norm(b[a] - oracle.apply_MTM(lat, H, L, xs[a])) / np.linalg.norm(b[a])
                      for a in range(2))
            worst["solve_" + prec] = max(worst.get("solve_" + prec, 0.0), float(res))
    # multi-vector apply: the row-pair form (N_x = 32) and the one-row form
    for nx, nt, k in [(32, 5, 3), (8, 6, 2)]:
        lat = oracle.lattice(3, nx, nt)
        n = oracle.nsites(lat)
        sigma = workloads.sigma_field(n, seed=950 + nx)
        L = oracle.links(lat, workloads.A_HS, sigma)
        xs = np.stack([workloads.source(n, seed=960 + nx, rhs=a) for a in range(k)]).astype(np.float32)
        with hh.Context(3, nx, nt) as ctx:
            ctx.set_field(torch.from_numpy(sigma).cuda())
            xd = torch.from_numpy(xs.reshape(-1)).cuda()
            yd = torch.empty_like(xd)
            ctx.apply_multi(hh.HH_OP_MTM, xd, yd, k)
            ctx.counters()
            got = yd.cpu().numpy().reshape(k, n).astype(np.float64)
        e = max(rel_err(got[v], oracle.apply_MTM(lat, H, L, xs[v].astype(np.float64))) for v in range(k))
        worst["apply_multi"] = max(worst.get("apply_multi", 0.0), e)
    # trajectories (heatbath, force, leapfrog, Metropolis)
    for d, nx, nt in [(1, 16, 12), (3, 4, 6)]:
        with hh.Context(d, nx, nt, seed=1234, n_pf=2) as ctx:
            ctx.init_field_random(1234)
            info = ctx.trajectory(3, 0.05, 0)
        worst["traj_dH_%d" % d] = abs(float(info["dH"]))
    # batch: solves of two dimensions in one launch (generic kernel)
    with B.Batch(max_slots=4, hbm_budget_bytes=1 << 30, chunk_iters=16, tile_sites=512) as batch:
        keeps = []
        for d, nx, nt, seed in [(1, 24, 16, 41), (3, 6, 8, 42)]:
            n = nx ** d * nt
            sigma = workloads.sigma_field(n, seed=seed)
            b = np.stack([workloads.source(n, seed=seed, rhs=a) for a in range(2)])
            o = np.zeros((2, n))
            batch.submit(B.make_request(B.HH_REQ_SOLVE, d, nx, nt, sigma=sigma, b=b, out=o, precision="mixed",
                                        n_pf=2), keep=(sigma, b, o))
            keeps.append((d, nx, nt, sigma, b, o))
        res = batch.run_until_idle()
    out["batch_status"] = sorted(r["status"] for r in res)
    for d, nx, nt, sigma, b, o in keeps:
        lat = oracle.lattice(d, nx, nt)
        L = oracle.links(lat, workloads.A_HS, sigma)
        r = max(np.linalg.norm(b[a] - oracle.apply_MTM(lat, H, L, o[a])) / np.linalg.norm(b[a]) for a in range(2))
        worst["batch_solve"] = max(worst.get("batch_solve", 0.0), float(r))
    torch.cuda.synchronize()
    rc, enabled, rec = B.bounds_check()
    out["final"] = [rc, enabled, rec]
    out["worst"] = worst
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
