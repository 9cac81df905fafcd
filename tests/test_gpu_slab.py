"""The time-slab decomposition (hh_slab_*) on the GPU against the oracle.

One, two and three ranks (gloo processes sharing the one GPU; halos are
staged through host memory between kernel launches, so no kernel waits for
another rank) each own a contiguous part of the time slices, uneven where
N_tau does not divide.  The parts of M x, M^T x and Q x are assembled and
compared per element with the oracle's applies on the whole lattice (1e-12 of
the magnitude of the terms), and the assembled CG solution's true residual,
recomputed by the oracle, must be <= 1e-10.  The wrap link's sign and the
ring's end (the rank owning slice 0 receives from the rank owning N_tau - 1)
are covered by every case.  The device form of the callbacks (transfers and
sums enqueued on the slab's stream, CG scalars on the device) runs with one
rank: several ranks in that form need one GPU each (NCCL).
"""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
H = workloads.T_HOP * workloads.DTAU


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("world,d,nx,ntau,form", [(1, 1, 32, 16, "host"), (2, 1, 48, 13, "host"),
                                                  (2, 3, 8, 12, "host"), (3, 3, 6, 11, "host"),
                                                  (1, 1, 40, 18, "device"), (1, 3, 8, 10, "device")])
def test_slab_apply_and_solve_match_oracle(tmp_path, world, d, nx, ntau, form):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1007_3432_gb300 import build
    build.build()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", str(world),
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "tests", "_slab_worker.py"), "gpu", str(tmp_path), str(d), str(nx), str(ntau), form]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    parts = [np.load(os.path.join(tmp_path, "rank%d.npz" % k)) for k in range(world)]
    V = nx ** d
    n = V * ntau
    assert [tuple(p["range"]) for p in parts] == [(k * ntau // world, (k + 1) * ntau // world)
                                                  for k in range(world)]
    lat = oracle.lattice(d, nx, ntau)
    sigma = workloads.sigma_field(n, seed=700 + nx + ntau)
    x = workloads.source(n, seed=701)
    b = workloads.source(n, seed=702)
    L = oracle.links(lat, workloads.A_HS, sigma)
    La, xa = np.abs(L), np.abs(x)
    refs = {"M": (oracle.apply_M(lat, H, L, x), oracle.apply_M(lat, -H, La, xa)),
            "MT": (oracle.apply_MT(lat, H, L, x), oracle.apply_MT(lat, -H, La, xa)),
            "MTM": (oracle.apply_MTM(lat, H, L, x), oracle.apply_MT(lat, -H, La, oracle.apply_M(lat, -H, La, xa)))}
    for name, (ref, mag) in refs.items():
        got = np.concatenate([p[name] for p in parts])
        assert got.shape == (n,)
        assert np.all(np.abs(got - ref) <= 1e-12 * mag), (name, np.max(np.abs(got - ref) / mag))
    for p in parts:
        rc, it, rel, conv = p["info"]
        assert rc == 0 and conv == 1 and rel <= 1e-10, p["info"]
    xs = np.concatenate([p["x"] for p in parts])
    res = b - oracle.apply_MTM(lat, H, L, xs)
    assert np.linalg.norm(res) <= 1.0001e-10 * np.linalg.norm(b)
