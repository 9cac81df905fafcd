"""The plain C program tests/native/c_consumer.c, run on the GPU, against the
oracle: the boundary exercised from C rather than through ctypes.

Checks on what the program writes: its field from hh_init_field_random is the
oracle's Philox field bit for bit; its two solutions meet the 1e-10 true
residual recomputed by the oracle; its Q b from hh_apply_multi matches the
oracle per element to 1e-12 of the magnitude of the terms; its trajectory has
the oracle's Metropolis uniform u exactly, H0 and dH within the tolerances of
the trajectory parity tests, the same accept decision (outside a margin of
the dH error) and the same final field to 1e-6.
"""
import os
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads  # noqa: E402

H = workloads.T_HOP * workloads.DTAU


def test_c_consumer_matches_oracle(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from test_abi import build_c_consumer
    exe, libdirs = build_c_consumer(tmp_path)
    out = str(tmp_path / "c_consumer.bin")
    env = dict(os.environ)
    env["LD_LIBRARY_PATH"] = ":".join(libdirs + [env.get("LD_LIBRARY_PATH", "")])
    run = subprocess.run([exe, out], env=env, capture_output=True, text=True, timeout=600)
    assert run.returncode == 0, run.stdout + run.stderr
    raw = open(out, "rb").read()
    n = int(np.frombuffer(raw[:8], dtype=np.int64)[0])
    v = np.frombuffer(raw[8:], dtype=np.float64)
    assert v.size == n + 2 * n + 2 * n + 2 * n + 5 + n
    s0, v = v[:n], v[n:]
    b, v = v[:2 * n].reshape(2, n), v[2 * n:]
    x, v = v[:2 * n].reshape(2, n), v[2 * n:]
    qb, v = v[:2 * n].reshape(2, n), v[2 * n:]
    tr, s1 = v[:5], v[5:]
    d, nx, ntau, seed = 1, 32, 64, 1007
    lat = oracle.lattice(d, nx, ntau)
    assert n == nx * ntau
    assert np.array_equal(s0, oracle.init_field(seed, 0, n))
    L = oracle.links(lat, workloads.A_HS, s0)
    La = np.abs(L)
    for a in range(2):
        res = b[a] - oracle.apply_MTM(lat, H, L, x[a])
        assert np.linalg.norm(res) <= 1.0001e-10 * np.linalg.norm(b[a])
        ref = oracle.apply_MTM(lat, H, L, b[a])
        bound = 1e-12 * oracle.apply_MT(lat, -H, La, oracle.apply_M(lat, -H, La, np.abs(b[a])))
        assert np.all(np.abs(qb[a] - ref) <= bound)
    prm = oracle.params(seed=seed, n_pf=2)
    s_ref, oinfo = oracle.trajectory(lat, prm, s0, 5, 0.04, 0)
    H0, H1, dH, u, acc = tr
    assert u == oinfo["u"]
    assert abs(H0 - oinfo["H0"]) <= 1e-8 * abs(oinfo["H0"])
    assert abs(dH - oinfo["dH"]) <= 1e-6, (dH, oinfo)
    if abs(oinfo["dH"] + np.log(oinfo["u"])) > 1e-5:
        assert int(acc) == oinfo["accepted"]
        assert np.max(np.abs(s1 - s_ref)) <= 1e-6
