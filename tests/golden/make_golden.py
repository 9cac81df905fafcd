"""Writes oracle_regression.json: values of the FP64 oracle on small seeded
inputs, so that any later change of the oracle's arithmetic shows up in
tests/test_golden.py.  Calls only the oracle (and the seeded input
generators); run from the repository root:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads  # noqa: E402

H = workloads.T_HOP * workloads.DTAU
SAMPLE = [0, 1, 17, 255, 1000, 2047]


def record():
    out = {}
    wl = workloads.C0
    lat = oracle.lattice(wl.d, wl.nx, wl.ntau)
    n = wl.nsites
    sigma = workloads.sigma_field(n, seed=wl.seed)
    L = oracle.links(lat, workloads.A_HS, sigma)
    x = workloads.source(n, seed=wl.seed)
    out["links_sample"] = [float(L[i]) for i in SAMPLE]
    for name, fn in (("M", oracle.apply_M), ("MT", oracle.apply_MT), ("MTM", oracle.apply_MTM)):
        y = fn(lat, H, L, x)
        out[name + "_sample"] = [float(y[i]) for i in SAMPLE]
    for order in (1, 2):
        y = oracle.apply_M_ex(lat, H, L, order, x)
        out["M_ex%d_sample" % order] = [float(y[i]) for i in SAMPLE]
    xs, st, it, rr = oracle.cg(lat, H, L, x)
    out["cg"] = {"status": int(st), "iterations": int(it), "sample": [float(xs[i]) for i in SAMPLE]}
    prm = oracle.params(seed=wl.seed, n_pf=2)
    s = sigma.copy()
    trajs = []
    for traj in range(2):
        s, info = oracle.trajectory(lat, prm, s, 5, 0.04, traj)
        trajs.append({k: (float(v) if isinstance(v, float) else int(v)) for k, v in info.items()})
    out["trajectories_n_md5_dt0.04"] = trajs
    ob = oracle.observables(lat, prm, sigma, 4, 1)
    out["observables_n4_traj1"] = {k: (float(v) if not isinstance(v, int) else v) for k, v in ob.items()}
    out["gaussian_tag2_sample"] = [float(v) for v in oracle.gaussian(wl.seed, 2, 1, 3, 0, 8)]
    out["z2_tag6_sample"] = [float(v) for v in oracle.z2_noise(wl.seed, 2, 3, 0, 8)]
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(record(), f, indent=1, sort_keys=True)
    print("wrote", os.path.join(HERE, "oracle_regression.json"))
