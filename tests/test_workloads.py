"""The seeded input recipe: distributions, ranges and determinism of the
synthetic lattices, right-hand sides, batch shapes and request streams."""
import numpy as np

import workloads as W


def test_fields_and_sources():
    s = W.sigma_field(200000, seed=1)
    assert s.min() >= -np.pi and s.max() < np.pi
    assert abs(s.mean()) < 0.02 and abs(s.var() - np.pi ** 2 / 3) < 0.03
    assert np.array_equal(s, W.sigma_field(200000, seed=1))
    assert not np.array_equal(s[:100], W.sigma_field(100, seed=1, chain=1))
    b = W.source(200000, seed=2)
    assert abs(b.mean()) < 0.01 and abs(b.var() - 1) < 0.02
    assert not np.array_equal(b[:100], W.source(100, seed=2, rhs=1))


def test_configs():
    assert (W.C0.d, W.C0.nx, W.C0.ntau, W.C0.nsites, W.C0.seed) == (1, 32, 64, 2048, 1007)
    assert (W.C1.d, W.C1.nx, W.C1.ntau, W.C1.nsites, W.C1.seed, W.C1.n_md) == (1, 1024, 512, 524288, 1008, 20)
    assert (W.C2.d, W.C2.nx, W.C2.ntau, W.C2.nsites, W.C2.seed) == (3, 32, 128, 4194304, 1009)
    assert (W.T_HOP, W.DTAU, W.A_HS) == (1.0, 0.05, 0.5)


def test_batch_chains():
    ch = W.batch_chains(64)
    assert len(ch) == 64 and [c.chain for c in ch] == list(range(64))
    assert all(c.d == 3 and c.nx in W.BATCH_NX and c.ntau in W.BATCH_NTAU for c in ch)
    assert [c.nsites for c in ch] == [c.nsites for c in W.batch_chains(64)]
    many = W.batch_chains(4000)
    for v in W.BATCH_NX:
        assert abs(sum(c.nx == v for c in many) / 4000 - 1 / len(W.BATCH_NX)) < 0.03
    for v in W.BATCH_NTAU:
        assert abs(sum(c.ntau == v for c in many) / 4000 - 1 / len(W.BATCH_NTAU)) < 0.03


def test_poisson_requests():
    rate, n = 100.0, 4000
    rq = W.poisson_requests(rate, n)
    t = np.array([r.arrival_s for r in rq])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and abs(gaps.mean() * rate - 1) < 0.05
    assert abs(np.std(gaps) * rate - 1) < 0.06          # exponential: sd = mean
    d1 = [r for r in rq if r.d == 1]
    d3 = [r for r in rq if r.d == 3]
    assert abs(len(d1) / n - 0.5) < 0.03
    assert all(64 <= r.nx <= 2048 and 64 <= r.ntau <= 512 and r.ntau % 8 == 0 for r in d1)
    assert all(8 <= r.nx <= 24 and 40 <= r.ntau <= 256 and r.ntau % 8 == 0 for r in d3)
    assert abs(sum(r.kind == "solve" for r in rq) / n - 0.5) < 0.03
    assert len({r.seed for r in rq}) == n
    assert [r.nsites for r in rq[:50]] == [r.nsites for r in W.poisson_requests(rate, 50)]
