"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these checks re-types an oracle formula: each compares the oracle with
an independent route to the same number (a closed form, a library routine, a
finite difference, an exact invariant of the algorithm), chosen so that a
dropped term, a wrong sign, a wrong slice index or a transposed operand fails
at least one of them.
"""
import itertools

import numpy as np
import pytest

H = 0.05  # h = t * dtau with t = 1, dtau = 0.05


def _free_eigs(d, nx, ntau, h, c):
    """Closed-form spectrum of M for a uniform link factor c = 1 + A sin sigma0.

    Plane waves exp(i k.n + i w tau) with lattice momenta k_j = 2 pi m_j / N_x
    (periodic, Sec. 2) and antiperiodic Matsubara frequencies
    w = pi (2m + 1) / N_tau diagonalise M with eigenvalue
    lambda = 1 - 2h sum_j cos k_j - c exp(-i w)."""
    eps = []
    for ms in itertools.product(range(nx), repeat=d):
        eps.append(1.0 - 2.0 * h * sum(np.cos(2 * np.pi * m / nx) for m in ms))
    out = []
    for e in eps:
        for m in range(ntau):
            w = np.pi * (2 * m + 1) / ntau
            out.append(e - c * np.exp(-1j * w))
    return np.array(out)


def _match_spectra(a, b):
    """Greedy nearest matching of two multisets of complex numbers."""
    b = list(b)
    worst = 0.0
    for z in a:
        j = int(np.argmin([abs(z - w) for w in b]))
        worst = max(worst, abs(z - b[j]))
        b.pop(j)
    return worst


@pytest.mark.parametrize("d,nx,ntau", [(1, 6, 8), (1, 4, 5), (3, 3, 4), (3, 2, 3)])
@pytest.mark.parametrize("sigma0", [0.0, 0.7])
def test_uniform_field_spectrum_closed_form(orc, d, nx, ntau, sigma0):
    A = 0.5
    lat = orc.lattice(d, nx, ntau)
    n = orc.nsites(lat)
    L = orc.links(lat, A, np.full(n, sigma0))
    M = orc.dense(lat, H, L, "M")
    got = np.linalg.eigvals(M)
    want = _free_eigs(d, nx, ntau, H, 1.0 + A * np.sin(sigma0))
    assert _match_spectra(got, want) < 1e-10


@pytest.mark.parametrize("d,nx,ntau", [(1, 8, 6), (3, 4, 4)])
def test_plane_waves_are_eigenvectors_per_element(orc, d, nx, ntau):
    """M v = lambda v and M^T v = conj(lambda) v, element by element, for a
    plane wave with a lattice momentum and an antiperiodic frequency."""
    A, sigma0 = 0.5, -1.1
    c = 1.0 + A * np.sin(sigma0)
    lat = orc.lattice(d, nx, ntau)
    n = orc.nsites(lat)
    L = orc.links(lat, A, np.full(n, sigma0))
    V = nx ** d
    idx = np.arange(n)
    tau = idx // V
    s = idx % V
    coords = [(s // nx ** j) % nx for j in range(d)]
    rng = np.random.default_rng(3)
    for _ in range(4):
        ms = rng.integers(0, nx, size=d)
        m = rng.integers(0, ntau)
        k = 2 * np.pi * ms / nx
        w = np.pi * (2 * m + 1) / ntau
        phase = sum(k[j] * coords[j] for j in range(d)) + w * tau
        v = np.exp(1j * phase)
        lam = 1.0 - 2.0 * H * np.sum(np.cos(k)) - c * np.exp(-1j * w)
        Mv = orc.apply_M(lat, H, L, v.real) + 1j * orc.apply_M(lat, H, L, v.imag)
        MTv = orc.apply_MT(lat, H, L, v.real) + 1j * orc.apply_MT(lat, H, L, v.imag)
        assert np.max(np.abs(Mv - lam * v)) < 1e-13
        assert np.max(np.abs(MTv - np.conj(lam) * v)) < 1e-13


@pytest.mark.parametrize("d,nx,ntau", [(1, 6, 8), (3, 3, 4)])
def test_free_determinant_closed_form(orc, d, nx, ntau):
    """det M = prod_k (eps_k^N_tau + c^N_tau) for a uniform link factor c."""
    A, sigma0 = 0.5, 0.3
    c = 1.0 + A * np.sin(sigma0)
    lat = orc.lattice(d, nx, ntau)
    n = orc.nsites(lat)
    L = orc.links(lat, A, np.full(n, sigma0))
    sign, logdet = np.linalg.slogdet(orc.dense(lat, H, L, "M"))
    want = 1.0
    for ms in itertools.product(range(nx), repeat=d):
        e = 1.0 - 2.0 * H * sum(np.cos(2 * np.pi * m / nx) for m in ms)
        want *= e ** ntau + c ** ntau
    assert sign == np.sign(want)
    assert abs(logdet - np.log(abs(want))) < 1e-11


@pytest.mark.parametrize("d,nx,ntau", [(1, 5, 6), (1, 2, 4), (3, 3, 3), (3, 2, 4)])
def test_random_field_determinant_block_reduction(orc, d, nx, ntau):
    """det M = det(D)^N_tau det(1 + T_{N-1} ... T_0), T_tau = D^{-1} diag(c_tau),
    with D = 1 - h K_hop the time-diagonal block and c = 1 + A sin sigma: the
    block-cyclic structure of Eq. (7) with the link signs -1 and the +1 corner.
    Built here from sigma directly, as V x V products, not from the oracle."""
    A = 0.5
    lat = orc.lattice(d, nx, ntau)
    n = orc.nsites(lat)
    V = nx ** d
    rng = np.random.default_rng(5)
    sigma = rng.uniform(-np.pi, np.pi, n)
    L = orc.links(lat, A, sigma)
    sign_o, logdet_o = np.linalg.slogdet(orc.dense(lat, H, L, "M"))

    hop = np.zeros((V, V))
    for s in range(V):
        c = [(s // nx ** j) % nx for j in range(d)]
        for j in range(d):
            for step in (1, -1):
                cc = list(c)
                cc[j] = (cc[j] + step) % nx
                t = sum(cc[q] * nx ** q for q in range(d))
                hop[s, t] += 1.0
    D = np.eye(V) - H * hop
    Dinv = np.linalg.inv(D)
    prod = np.eye(V)
    for tau in range(ntau):
        c_tau = 1.0 + A * np.sin(sigma[tau * V:(tau + 1) * V])
        prod = Dinv @ np.diag(c_tau) @ prod
    sD, lD = np.linalg.slogdet(D)
    sP, lP = np.linalg.slogdet(np.eye(V) + prod)
    assert sign_o == sD ** ntau * sP
    assert abs(logdet_o - (ntau * lD + lP)) < 1e-10


@pytest.mark.parametrize("d,nx,ntau", [(1, 7, 5), (1, 2, 3), (3, 3, 4), (3, 2, 2)])
def test_transpose_and_normal_matrix_are_exact(orc, d, nx, ntau):
    lat = orc.lattice(d, nx, ntau)
    n = orc.nsites(lat)
    rng = np.random.default_rng(9)
    L = orc.links(lat, 0.5, rng.uniform(-np.pi, np.pi, n))
    M = orc.dense(lat, H, L, "M")
    MT = orc.dense(lat, H, L, "MT")
    Q = orc.dense(lat, H, L, "MTM")
    assert np.array_equal(MT, M.T)
    assert np.allclose(Q, M.T @ M, rtol=0, atol=1e-14)
    assert np.min(np.linalg.eigvalsh(Q)) > 0


@pytest.mark.parametrize("d,nx,ntau", [(1, 6, 4), (1, 2, 4), (3, 3, 3), (3, 2, 3)])
def test_sparsity_pattern_of_eq10(orc, d, nx, ntau):
    """Each row has the site, 2d spatial neighbours and one temporal link
    (2d + 2 reads per site, Sec. 4.3); neighbours coincide when N_x = 2."""
    lat = orc.lattice(d, nx, ntau)
    n = orc.nsites(lat)
    rng = np.random.default_rng(2)
    L = orc.links(lat, 0.5, rng.uniform(-np.pi, np.pi, n))
    M = orc.dense(lat, H, L, "M")
    nnz = np.count_nonzero(M, axis=1)
    expect = 2 * d + 2 if nx > 2 else d + 2
    assert np.all(nnz == expect)
    assert np.all(np.diag(M) == 1.0)
    offdiag_spatial = M[np.abs(M + H * (1 if nx > 2 else 2)) < 1e-15]
    assert offdiag_spatial.size == n * 2 * d // (1 if nx > 2 else 2)


def test_adjointness_large(orc):
    lat = orc.lattice(3, 5, 7)
    n = orc.nsites(lat)
    rng = np.random.default_rng(4)
    L = orc.links(lat, 0.5, rng.uniform(-np.pi, np.pi, n))
    x, y = rng.standard_normal(n), rng.standard_normal(n)
    lhs = orc.apply_M(lat, H, L, x) @ y
    rhs = x @ orc.apply_MT(lat, H, L, y)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs) + 1e-12


@pytest.mark.parametrize("d,nx,ntau", [(1, 4, 8), (1, 16, 12), (3, 3, 4)])
def test_cg_matches_dense_lu(orc, d, nx, ntau):
    lat = orc.lattice(d, nx, ntau)
    n = orc.nsites(lat)
    rng = np.random.default_rng(12)
    L = orc.links(lat, 0.5, rng.uniform(-np.pi, np.pi, n))
    b = rng.standard_normal(n)
    x, st, it, relres = orc.cg(lat, H, L, b, tol=1e-10)
    assert st == 0 and relres <= 1e-10
    M = orc.dense(lat, H, L, "M")
    Q = M.T @ M
    x_lu = np.linalg.solve(Q, b)
    kappa = np.linalg.cond(Q)
    assert np.linalg.norm(x - x_lu) <= 2 * kappa * 1e-10 * np.linalg.norm(x_lu)
    assert np.linalg.norm(b - Q @ x) <= 1.01e-10 * np.linalg.norm(b)


def test_cg_zero_rhs_and_maxit(orc):
    lat = orc.lattice(1, 8, 8)
    n = orc.nsites(lat)
    rng = np.random.default_rng(1)
    L = orc.links(lat, 0.5, rng.uniform(-np.pi, np.pi, n))
    x, st, it, rr = orc.cg(lat, H, L, np.zeros(n))
    assert st == 0 and it == 0 and not np.any(x)
    x, st, it, rr = orc.cg(lat, H, L, rng.standard_normal(n), tol=1e-10, maxit=3)
    assert st == -4 and it == 3 and rr > 1e-10


def _dense_action(orc, lat, prm, sigma, chi):
    """S_pf = 1/2 sum_a chi_a^T (M^T M)^{-1} chi_a with a dense LU solve."""
    L = orc.links(lat, prm.A, sigma)
    M = orc.dense(lat, prm.t * prm.dtau, L, "M")
    Q = M.T @ M
    return 0.5 * sum(c @ np.linalg.solve(Q, c) for c in chi)


@pytest.mark.parametrize("d,nx,ntau", [(1, 4, 6), (3, 2, 3)])
def test_force_matches_finite_differences(orc, d, nx, ntau):
    lat = orc.lattice(d, nx, ntau)
    n = orc.nsites(lat)
    prm = orc.params(cg_tol=1e-13, seed=77)
    rng = np.random.default_rng(8)
    sigma = rng.uniform(-np.pi, np.pi, n)
    chi = rng.standard_normal((prm.n_pf, n))
    F, it, rr, st = orc.force(lat, prm, sigma, chi)
    assert st == 0
    eps = 1e-5
    for i in rng.choice(n, size=min(n, 8), replace=False):
        sp, sm = sigma.copy(), sigma.copy()
        sp[i] += eps
        sm[i] -= eps
        fd = (_dense_action(orc, lat, prm, sp, chi) - _dense_action(orc, lat, prm, sm, chi)) / (2 * eps)
        assert abs(F[i] - fd) <= 1e-6 * max(1.0, abs(fd))


def test_action_matches_dense_and_heatbath_identity(orc):
    """S_pf(chi = M^T xi) = 1/2 |xi|^2 (Eqs. (11)-(12)); xi from NumPy's Philox."""
    lat = orc.lattice(1, 8, 16)
    n = orc.nsites(lat)
    prm = orc.params(seed=2024, chain=3)
    rng = np.random.default_rng(21)
    sigma = rng.uniform(-np.pi, np.pi, n)
    chi = orc.heatbath(lat, prm, sigma, traj=5)
    S, it, rr, st = orc.action(lat, prm, sigma, chi)
    xi = np.stack([_numpy_gaussian(prm.seed, 2, a, 5, 3, n) for a in range(prm.n_pf)])
    assert st == 0
    assert abs(S - 0.5 * np.sum(xi * xi)) < 1e-8 * S
    assert abs(S - _dense_action(orc, lat, prm, sigma, chi)) < 1e-8 * S


# --- Philox and the random streams ------------------------------------------


def _numpy_philox_block(ctr, key):
    """Philox4x64-10 from NumPy; its generator increments the counter before it
    encrypts, so the stored counter is ctr - 1 (as a 256-bit integer)."""
    c = sum(int(v) << (64 * j) for j, v in enumerate(ctr))
    c = (c - 1) % (1 << 256)
    words = np.array([(c >> (64 * j)) & ((1 << 64) - 1) for j in range(4)], dtype=np.uint64)
    bg = np.random.Philox(counter=words, key=np.array(key, dtype=np.uint64))
    return [int(v) for v in bg.random_raw(4)]


def _numpy_gaussian(seed, tag, a, traj, chain, n):
    out = np.empty(n)
    for i in range(n):
        w = _numpy_philox_block([i >> 2, tag | (a << 8), traj, chain], [seed, 0])
        j = (i >> 1) & 1
        u1 = (w[2 * j] >> 11) * 2.0 ** -53
        u2 = (w[2 * j + 1] >> 11) * 2.0 ** -53
        r = np.sqrt(-2.0 * np.log(1.0 - u1))
        out[i] = r * (np.sin(2 * np.pi * u2) if i & 1 else np.cos(2 * np.pi * u2))
    return out


@pytest.mark.parametrize("ctr,key", [
    ([0, 0, 0, 0], [0, 0]),
    ([1, 0, 0, 0], [5, 0]),
    ([2 ** 64 - 1, 7, 9, 11], [123456789, 987654321]),
    ([0, 2 ** 64 - 1, 2 ** 63, 3], [2 ** 64 - 1, 2 ** 64 - 1]),
    ([31337, 2 | (1 << 8), 17, 4], [1008, 0]),
])
def test_philox_matches_numpy(orc, ctr, key):
    assert orc.philox4x64(ctr, key) == _numpy_philox_block(ctr, key)


def test_gaussian_and_uniform_streams(orc):
    g = orc.gaussian(99, 1, 0, 4, 2, 37)
    assert np.allclose(g, _numpy_gaussian(99, 1, 0, 4, 2, 37), rtol=0, atol=1e-15)
    big = orc.gaussian(7, 2, 1, 0, 0, 200000)
    assert abs(big.mean()) < 0.01 and abs(big.var() - 1) < 0.01
    for i in (0, 1, 2, 3, 4, 1001):
        w = _numpy_philox_block([i >> 2, 3, 8, 1], [42, 0])
        assert orc.uniform(42, 3, 8, 1, i) == (w[i & 3] >> 11) * 2.0 ** -53
    s = orc.init_field(5, 2, 1000)
    assert s.min() >= -np.pi and s.max() < np.pi
    w = _numpy_philox_block([0, 0, 0, 2], [5, 0])
    assert s[1] == -np.pi + 2 * np.pi * ((w[1] >> 11) * 2.0 ** -53)


# --- molecular dynamics and the Markov chain -------------------------------


def _md_setup(orc, d=1, nx=6, ntau=8, seed=31):
    lat = orc.lattice(d, nx, ntau)
    n = orc.nsites(lat)
    prm = orc.params(cg_tol=1e-12, seed=seed)
    rng = np.random.default_rng(seed)
    sigma = rng.uniform(-np.pi, np.pi, n)
    pi = rng.standard_normal(n)
    chi = orc.heatbath(lat, prm, sigma, traj=0)
    return lat, prm, sigma, pi, chi


def test_leapfrog_reversible(orc):
    lat, prm, sigma, pi, chi = _md_setup(orc)
    s1, p1, *_ = orc.leapfrog(lat, prm, sigma, pi, chi, 10, 0.05)
    s2, p2, *_ = orc.leapfrog(lat, prm, s1, -p1, chi, 10, 0.05)
    assert np.max(np.abs(s2 - sigma)) < 1e-9
    assert np.max(np.abs(p2 + pi)) < 1e-9
    assert np.max(np.abs(s1 - sigma)) > 1e-2


def _hamiltonian(orc, lat, prm, sigma, pi, chi):
    return 0.5 * pi @ pi + orc.action(lat, prm, sigma, chi)[0]


def test_energy_violation_scales_as_dt_squared(orc):
    lat, prm, sigma, pi, chi = _md_setup(orc, nx=4, ntau=6, seed=3)
    pi = 0.5 * pi
    H0 = _hamiltonian(orc, lat, prm, sigma, pi, chi)
    steps = np.array([16, 32, 64])
    dH = []
    for n_md in steps:
        s1, p1, *_ = orc.leapfrog(lat, prm, sigma, pi, chi, int(n_md), 0.25 / n_md)
        dH.append(abs(_hamiltonian(orc, lat, prm, s1, p1, chi) - H0))
    slope = np.polyfit(np.log(0.25 / steps), np.log(dH), 1)[0]
    assert 1.8 < slope < 2.2, (dH, slope)


@pytest.mark.slow
# --- Omelyan's second-order minimum-norm integrator ---------------------------


def _omelyan_prm(orc, prm):
    return orc.params(t=prm.t, dtau=prm.dtau, A=prm.A, cg_tol=prm.cg_tol, cg_maxit=prm.cg_maxit,
                      n_pf=prm.n_pf, seed=prm.seed, chain=prm.chain, integrator=1)


def test_omelyan_reversible_and_symplectic_order(orc):
    """Reversible (momentum flip), and the energy violation falls as dt^2 with
    a coefficient several times below leapfrog's at equal step size (the
    scheme's minimum-norm property)."""
    lat, prm, sigma, pi, chi = _md_setup(orc)
    om = _omelyan_prm(orc, prm)
    s1, p1, *_ = orc.leapfrog(lat, om, sigma, pi, chi, 10, 0.05)
    s2, p2, *_ = orc.leapfrog(lat, om, s1, -p1, chi, 10, 0.05)
    assert np.max(np.abs(s2 - sigma)) < 1e-9 and np.max(np.abs(p2 + pi)) < 1e-9
    assert np.max(np.abs(s1 - sigma)) > 1e-2

    lat, prm, sigma, pi, chi = _md_setup(orc, nx=4, ntau=6, seed=3)
    om = _omelyan_prm(orc, prm)
    pi = 0.5 * pi
    H0 = _hamiltonian(orc, lat, prm, sigma, pi, chi)
    steps = np.array([8, 16, 32])
    dH_om, dH_lf = [], []
    for n_md in steps:
        s1, p1, *_ = orc.leapfrog(lat, om, sigma, pi, chi, int(n_md), 0.25 / n_md)
        dH_om.append(abs(_hamiltonian(orc, lat, prm, s1, p1, chi) - H0))
        s1, p1, *_ = orc.leapfrog(lat, prm, sigma, pi, chi, int(n_md), 0.25 / n_md)
        dH_lf.append(abs(_hamiltonian(orc, lat, prm, s1, p1, chi) - H0))
    slope = np.polyfit(np.log(0.25 / steps), np.log(dH_om), 1)[0]
    assert 1.8 < slope < 2.2, (dH_om, slope)
    assert all(o < 0.1 * l for o, l in zip(dH_om, dH_lf)), (dH_om, dH_lf)   # 0.046 measured


def test_omelyan_step_sequence(orc):
    """One Omelyan step on a quadratic action S = 0 (A = 0: the force
    vanishes) is a free drift sigma += dt pi, and its 2 n_md + 1 forces are
    counted in the trajectory's solves."""
    lat = orc.lattice(1, 4, 4)
    n = orc.nsites(lat)
    prm = orc.params(A=0.0, integrator=1)
    rng = np.random.default_rng(5)
    sigma, pi = rng.uniform(-1, 1, n), rng.standard_normal(n)
    chi = rng.standard_normal((2, n))
    s1, p1, *_ = orc.leapfrog(lat, prm, sigma, pi, chi, 3, 0.1)
    assert np.allclose(s1, sigma + 0.3 * pi, atol=1e-14) and np.allclose(p1, pi, atol=0)
    _, info = orc.trajectory(lat, prm, sigma, 3, 0.1, 0)
    assert info["n_solves"] == 2 * (2 * 3 + 1 + 2)


# --- Chronological initial guesses -------------------------------------------


def test_cg_from_initial_guess(orc):
    """From the dense-LU solution CG stops at once; from a perturbed one it
    meets the tolerance in fewer steps than from zero; b = 0 gives x = 0."""
    lat = orc.lattice(1, 8, 12)
    n = orc.nsites(lat)
    rng = np.random.default_rng(31)
    L = orc.links(lat, 0.5, rng.uniform(-np.pi, np.pi, n))
    b = rng.standard_normal(n)
    x_lu = np.linalg.solve(orc.dense(lat, H, L, "MTM"), b)
    x, st, it, rr = orc.cg_guess(lat, H, L, b, x_lu)
    assert st == 0 and it == 0 and rr <= 1e-10
    _, _, it0, _ = orc.cg(lat, H, L, b)
    x, st, it, rr = orc.cg_guess(lat, H, L, b, x_lu + 1e-6 * rng.standard_normal(n))
    assert st == 0 and rr <= 1e-10 and 0 < it < it0
    assert np.linalg.norm(x - x_lu) <= 1e-6 * np.linalg.norm(x_lu)
    x, st, it, rr = orc.cg_guess(lat, H, L, np.zeros(n), rng.standard_normal(n))
    assert st == 0 and it == 0 and not np.any(x)


@pytest.mark.parametrize("chrono", [1, 2])
def test_chronological_guess_md(orc, chrono):
    """The MD with guesses from earlier solves (reversible only to the CG
    tolerance: the solves start from the history) stays within the
    tolerance's effect of the zero-guess MD and never spends more CG steps;
    at a small step, extrapolation saves at least 5% even on this 48-site
    lattice, whose CG converges in about its dimension from any start."""
    lat, prm, sigma, pi, chi = _md_setup(orc)

    def with_chrono(c):
        return orc.params(t=prm.t, dtau=prm.dtau, A=prm.A, cg_tol=prm.cg_tol, cg_maxit=prm.cg_maxit,
                          n_pf=prm.n_pf, seed=prm.seed, chain=prm.chain, chrono=c)

    base = orc.leapfrog(lat, prm, sigma, pi, chi, 10, 0.05)
    got = orc.leapfrog(lat, with_chrono(chrono), sigma, pi, chi, 10, 0.05)
    assert got[4] == 0 and got[3] <= 1e-10
    assert np.max(np.abs(got[0] - base[0])) < 1e-7 and np.max(np.abs(got[1] - base[1])) < 1e-7
    assert got[2] <= base[2], (got[2], base[2])
    if chrono == 2:
        small = orc.leapfrog(lat, prm, sigma, pi, chi, 20, 0.002)[2]
        assert orc.leapfrog(lat, with_chrono(2), sigma, pi, chi, 20, 0.002)[2] < 0.95 * small


def test_creutz_equality_mean_exp_minus_dH_is_one(orc):
    """<exp(-dH)> = 1 for an area-preserving, reversible integrator (Sec. 4.1:
    the Metropolis step makes HMC exact)."""
    lat = orc.lattice(1, 4, 6)
    n = orc.nsites(lat)
    prm = orc.params(seed=4242)
    sigma = np.random.default_rng(0).uniform(-np.pi, np.pi, n)
    vals = []
    for traj in range(400):
        sigma, info = orc.trajectory(lat, prm, sigma, 8, 1.0 / 8, traj)
        assert info["status"] == 0
        assert info["accepted"] == (info["u"] < np.exp(-info["dH"]))
        if traj >= 20:
            vals.append(np.exp(-info["dH"]))
    vals = np.array(vals)
    blocks = vals[: len(vals) // 20 * 20].reshape(20, -1).mean(axis=1)
    err = blocks.std(ddof=1) / np.sqrt(len(blocks))
    assert abs(vals.mean() - 1.0) < 3 * err + 1e-3, (vals.mean(), err)


def test_trajectory_draws_and_metropolis(orc):
    lat = orc.lattice(1, 8, 8)
    n = orc.nsites(lat)
    prm = orc.params(seed=606, chain=2)
    sigma = np.random.default_rng(1).uniform(-np.pi, np.pi, n)
    pi = _numpy_gaussian(606, 1, 0, 9, 2, n)
    xi = np.stack([_numpy_gaussian(606, 2, a, 9, 2, n) for a in range(2)])
    s1, info = orc.trajectory(lat, prm, sigma, 6, 1.0 / 6, 9)
    assert abs(info["H0"] - 0.5 * (pi @ pi + np.sum(xi * xi))) < 1e-8 * info["H0"]
    assert info["u"] == orc.uniform(606, 3, 9, 2, 0)
    assert info["accepted"] == (info["u"] < np.exp(-info["dH"]))
    assert info["n_solves"] == 2 * (6 + 3)
    if not info["accepted"]:
        assert np.array_equal(s1, sigma)
    # Several trajectories, one with a step so large that dH >> 1: the decision
    # must follow u < exp(-dH) in every case, and a rejection restores sigma.
    seen_reject = False
    for traj, (n_md, dt) in enumerate([(2, 2.0), (4, 0.25), (4, 0.5), (3, 1.0)], start=10):
        s2, info2 = orc.trajectory(lat, prm, sigma, n_md, dt, traj)
        assert info2["accepted"] == (info2["u"] < np.exp(-info2["dH"]))
        if not info2["accepted"]:
            seen_reject = True
            assert np.array_equal(s2, sigma)
    assert seen_reject


@pytest.mark.slow
def test_hmc_reproduces_exact_expectation_on_2x2(orc):
    """On N_x = N_tau = 2 (4 sites), <sin^2 sigma> under the weight det(M)^2
    (Eq. (6) with S_g = 0) by quadrature must match the HMC average."""
    A = 0.5
    lat = orc.lattice(1, 2, 2)
    g = 28
    th = -np.pi + 2 * np.pi * (np.arange(g) + 0.5) / g
    S = np.stack(np.meshgrid(th, th, th, th, indexing="ij"), -1).reshape(-1, 4)
    # Dense M for every grid point via the oracle's own links is too slow;
    # the 4x4 matrix is assembled from its definition in Eq. (10) instead:
    # sites i = x + 2 tau; neighbours of x are both 1 - x (coefficient -2h).
    c = 1.0 + A * np.sin(S)
    Mg = np.zeros((S.shape[0], 4, 4))
    for tau in range(2):
        for x in range(2):
            i = x + 2 * tau
            Mg[:, i, i] = 1.0
            Mg[:, i, (1 - x) + 2 * tau] = -2 * H
            j = x + 2 * (1 - tau)
            sign = 1.0 if (1 - tau) == 1 else -1.0
            Mg[:, i, j] = sign * c[:, j]
    # cross-check the hand assembly against the oracle on one point
    Lone = orc.links(lat, A, S[123])
    assert np.allclose(orc.dense(lat, H, Lone, "M"), Mg[123], atol=1e-15)
    w = np.linalg.det(Mg) ** 2
    exact = np.sum(w * np.mean(np.sin(S) ** 2, axis=1)) / np.sum(w)

    prm = orc.params(seed=99)
    sigma = np.zeros(4)
    obs = []
    for traj in range(3000):
        sigma, info = orc.trajectory(lat, prm, sigma, 5, 0.3, traj)
        if traj >= 100:
            obs.append(np.mean(np.sin(sigma) ** 2))
    obs = np.array(obs)
    blocks = obs[: len(obs) // 50 * 50].reshape(50, -1).mean(axis=1)
    err = blocks.std(ddof=1) / np.sqrt(len(blocks))
    assert abs(obs.mean() - exact) < 4 * err, (obs.mean(), exact, err)


# --- Chebyshev polynomial preconditioner (Sec. 4.2) ---------------------------


@pytest.mark.parametrize("n,eps", [(2, 0.1), (4, 0.01), (8, 1e-3), (16, 1e-4), (12, 0.05)])
def test_chebyshev_error_bound(orc, n, eps):
    """|z P(z) - 1| <= 2 ((1 - sqrt(eps)) / (1 + sqrt(eps)))^(2n+1) on [eps, 1]
    (Eqs. (16)-(17)); P(z) > 0 on [0, 1]."""
    bound = 2 * ((1 - np.sqrt(eps)) / (1 + np.sqrt(eps))) ** (2 * n + 1)
    zs = np.concatenate([np.linspace(eps, 1.0, 4001), np.geomspace(eps, 1.0, 2001)])
    worst = max(abs(z * orc.cheb_poly(n, eps, z) - 1.0) for z in zs)
    assert worst <= bound * (1 + 1e-9), (worst, bound)
    # the bound is nearly attained: the polynomial is the minimax one
    assert worst >= 0.5 * bound
    assert all(orc.cheb_poly(n, eps, z) > 0 for z in np.linspace(0.0, 1.0, 501))


def test_chebyshev_limit_cases(orc):
    """n = 0 gives P = 1/m (m = (1+eps)/2), and P(z) -> 1/z on [eps, 1] as n
    grows, at the exponential rate of the bound (Eq. (16))."""
    assert abs(orc.cheb_poly(0, 0.3, 0.7) - 1 / 0.65) < 1e-15
    eps = 0.01
    for n in (20, 40, 60):
        bound = 2 * ((1 - np.sqrt(eps)) / (1 + np.sqrt(eps))) ** (2 * n + 1)
        for z in (0.05, 0.3, 0.9):
            assert abs(orc.cheb_poly(n, eps, z) * z - 1) <= bound


@pytest.mark.parametrize("d,nx,ntau", [(1, 8, 6), (3, 4, 4)])
def test_chebyshev_apply_plane_waves(orc, d, nx, ntau):
    """Uniform field: plane waves are eigenvectors of Q with eigenvalue
    |lambda|^2, so P(Q/lam) v = P(|lambda|^2/lam) v element by element."""
    A, sigma0, n, eps = 0.5, 0.4, 6, 0.02
    c = 1.0 + A * np.sin(sigma0)
    lat = orc.lattice(d, nx, ntau)
    nsite = orc.nsites(lat)
    L = orc.links(lat, A, np.full(nsite, sigma0))
    lam = orc.gershgorin_lambda_max(d, H, A)
    V = nx ** d
    idx = np.arange(nsite)
    tau = idx // V
    s = idx % V
    coords = [(s // nx ** j) % nx for j in range(d)]
    ms = np.array([1] * d)
    k = 2 * np.pi * ms / nx
    w = np.pi * 3 / ntau
    v = np.cos(sum(k[j] * coords[j] for j in range(d)) + w * tau)
    # a real plane wave mixes w and -w; both have the same |lambda|
    lam_m = 1.0 - 2.0 * H * np.sum(np.cos(k)) - c * np.exp(-1j * w)
    ev = abs(lam_m) ** 2
    got = orc.cheb_apply(lat, H, L, n, eps, lam, v)
    assert np.max(np.abs(got - orc.cheb_poly(n, eps, ev / lam) * v)) < 1e-12


def test_chebyshev_operator_is_spd_and_commutes(orc):
    lat = orc.lattice(1, 5, 4)
    nsite = orc.nsites(lat)
    rng = np.random.default_rng(3)
    L = orc.links(lat, 0.5, rng.uniform(-np.pi, np.pi, nsite))
    lam = orc.gershgorin_lambda_max(1, H, 0.5)
    P = np.stack([orc.cheb_apply(lat, H, L, 5, 0.01, lam, e) for e in np.eye(nsite)], axis=1)
    Q = orc.dense(lat, H, L, "MTM")
    assert np.max(np.linalg.eigvalsh(Q)) <= lam
    assert np.allclose(P, P.T, atol=1e-12)
    assert np.min(np.linalg.eigvalsh(0.5 * (P + P.T))) > 0
    assert np.allclose(P @ Q, Q @ P, atol=1e-10)


@pytest.mark.parametrize("n,eps", [(8, 1e-4), (32, 1e-5), (64, 1e-6)])
def test_chebyshev_apply_matches_spectral_evaluation(orc, n, eps):
    """Random field: P(Q/lam) b from the factors equals V P(Lambda/lam) V^T b from
    the eigendecomposition of the dense Q, with P evaluated as the scalar product
    over all 2n roots (Eq. (15)).  Multiplying scalars keeps the relative
    precision in any order; applied to a vector the order of the factors
    matters, and the order k = 1..n misses this by many orders of magnitude at
    n = 32 and 64."""
    lat = orc.lattice(1, 8, 12)
    nsite = orc.nsites(lat)
    rng = np.random.default_rng(21)
    L = orc.links(lat, 0.5, rng.uniform(-np.pi, np.pi, nsite))
    lam = orc.gershgorin_lambda_max(1, H, 0.5)
    b = rng.standard_normal(nsite)
    w, V = np.linalg.eigh(orc.dense(lat, H, L, "MTM"))
    ref = V @ (np.array([orc.cheb_poly(n, eps, z / lam) for z in w]) * (V.T @ b))
    got = orc.cheb_apply(lat, H, L, n, eps, lam, b)
    assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("d,nx,ntau", [(1, 8, 12), (3, 3, 4)])
def test_pcg_matches_dense_lu(orc, d, nx, ntau):
    lat = orc.lattice(d, nx, ntau)
    nsite = orc.nsites(lat)
    rng = np.random.default_rng(12)
    L = orc.links(lat, 0.5, rng.uniform(-np.pi, np.pi, nsite))
    b = rng.standard_normal(nsite)
    lam = orc.gershgorin_lambda_max(d, H, 0.5)
    x, st, it, relres = orc.pcg(lat, H, L, b, 4, 1e-3, lam)
    assert st == 0 and relres <= 1e-10
    Q = orc.dense(lat, H, L, "MTM")
    x_lu = np.linalg.solve(Q, b)
    assert np.linalg.norm(x - x_lu) <= 2 * np.linalg.cond(Q) * 1e-10 * np.linalg.norm(x_lu)
    x0, st0, it0, _ = orc.cg(lat, H, L, b)
    assert it < it0   # each PCG step applies Q 2n+1 times: far fewer steps


# --- Exact-block form of M (Eq. (7) with B = e^{-dtau K} e^{-dtau V}) ---------


def _free_block_eigenvalues(d, nx, ntau, h, order):
    """A = 0: plane waves with lattice momenta k_j = 2 pi m_j / N_x and
    antiperiodic frequencies w = pi (2m + 1) / N_tau are eigenvectors, with
    lambda = 1 - B_k e^{-i w}, B_k = 1 + h e_k (+ (h e_k)^2 / 2), e_k = sum_j
    2 cos k_j the eigenvalue of the neighbour sum."""
    ks = np.array(np.meshgrid(*[2 * np.pi * np.arange(nx) / nx] * d, indexing="ij")).reshape(d, -1)
    ek = 2 * np.cos(ks).sum(axis=0)
    B = 1 + h * ek + (0.5 * (h * ek) ** 2 if order == 2 else 0.0)
    w = np.pi * (2 * np.arange(ntau) + 1) / ntau
    return (1 - B[:, None] * np.exp(-1j * w[None, :])).ravel(), B


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("d,nx,ntau", [(1, 6, 8), (3, 3, 4)])
def test_exact_block_free_field_spectrum_and_determinant(orc, order, d, nx, ntau):
    """Free field: the singular values of M are |lambda| (M is normal), and
    det M = prod_k (1 + B_k^{N_tau}) (the block-cyclic determinant of Eq. (7)
    with the antiperiodic corner)."""
    lat = orc.lattice(d, nx, ntau)
    n = orc.nsites(lat)
    h = 0.3
    L = orc.links(lat, 0.0, np.zeros(n))
    M = orc.dense(lat, h, L, "M", order=order)
    lam, B = _free_block_eigenvalues(d, nx, ntau, h, order)
    sv = np.sort(np.linalg.svd(M, compute_uv=False))
    assert np.allclose(sv, np.sort(np.abs(lam)), rtol=1e-12, atol=1e-12)
    sign, logdet = np.linalg.slogdet(M)
    ref = 1 + B ** ntau
    assert np.isclose(logdet, np.sum(np.log(np.abs(ref))), rtol=1e-12)
    assert sign == np.prod(np.sign(ref))


@pytest.mark.parametrize("order", [1, 2])
def test_exact_block_structure(orc, order):
    """M^T is the transpose of M; A = 0 and h -> 0 recover the R1 form with
    h = 0; a row of M couples its site, the same site one slice earlier and,
    at order 1, its 2d spatial neighbours there (order 2: distance 2 too)."""
    lat = orc.lattice(1, 7, 5)
    n = orc.nsites(lat)
    rng = np.random.default_rng(4)
    L = orc.links(lat, 0.5, rng.uniform(-np.pi, np.pi, n))
    M = orc.dense(lat, 0.2, L, "M", order=order)
    MT = orc.dense(lat, 0.2, L, "MT", order=order)
    # entries agree to rounding (order 2 sums the same products in another order)
    assert np.allclose(MT, M.T, rtol=1e-15, atol=1e-17)
    assert np.allclose(orc.dense(lat, 0.0, L, "M", order=order), orc.dense(lat, 0.0, L, "M"), atol=0)
    row = 7 * 2 + 3                 # x = 3, tau = 2
    cols = set(np.nonzero(M[row])[0])
    expect = {row, 7 * 1 + 3, 7 * 1 + 2, 7 * 1 + 4}
    if order == 2:
        expect |= {7 * 1 + 1, 7 * 1 + 5}
    assert cols == expect


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("d,nx,ntau", [(1, 4, 6), (3, 2, 3)])
def test_exact_block_force_and_cg(orc, order, d, nx, ntau):
    """Force against central differences of the dense-LU action of the same M,
    CG against dense LU, and the heatbath identity S = |xi|^2 / 2."""
    lat = orc.lattice(d, nx, ntau)
    n = orc.nsites(lat)
    prm = orc.params(cg_tol=1e-13, seed=78, link_order=order)
    rng = np.random.default_rng(9)
    sigma = rng.uniform(-np.pi, np.pi, n)
    chi = rng.standard_normal((prm.n_pf, n))
    h = prm.t * prm.dtau

    def dense_action(s):
        M = orc.dense(lat, h, orc.links(lat, prm.A, s), "M", order=order)
        Q = M.T @ M
        return 0.5 * sum(c @ np.linalg.solve(Q, c) for c in chi)

    F, it, rr, st = orc.force(lat, prm, sigma, chi)
    assert st == 0
    eps = 1e-5
    for i in rng.choice(n, size=min(n, 8), replace=False):
        sp, sm = sigma.copy(), sigma.copy()
        sp[i] += eps
        sm[i] -= eps
        fd = (dense_action(sp) - dense_action(sm)) / (2 * eps)
        assert abs(F[i] - fd) <= 1e-6 * max(1.0, abs(fd))
    L = orc.links(lat, prm.A, sigma)
    Q = orc.dense(lat, h, L, "MTM", order=order)
    x, st, it, rr = orc.cg_ex(lat, h, L, order, chi[0])
    assert st == 0 and np.linalg.norm(x - np.linalg.solve(Q, chi[0])) <= 1e-6 * np.linalg.norm(x)
    xi_chi = orc.heatbath(lat, prm, sigma, traj=3)
    S, *_ = orc.action(lat, prm, sigma, xi_chi)
    Minv_chi = [np.linalg.solve(orc.dense(lat, h, L, "MT", order=order), c) for c in xi_chi]
    assert abs(S - 0.5 * sum(v @ v for v in Minv_chi)) <= 1e-9 * S


# --- observables: noise estimators of diag M^{-1} (reading R13) -------------


def _free_block_energies(d, nx, h, order):
    """E_k = 1 + x (+ x^2 / 2), x = 2h sum_j cos k_j: the hopping factor of the
    exact-block form on a plane wave of lattice momentum k."""
    out = []
    for ms in itertools.product(range(nx), repeat=d):
        x = 2.0 * h * sum(np.cos(2 * np.pi * m / nx) for m in ms)
        out.append(1.0 + x + (0.5 * x * x if order == 2 else 0.0))
    return np.array(out)


@pytest.mark.parametrize("d,nx,ntau,order", [(1, 8, 8, 1), (1, 6, 10, 2), (3, 3, 4, 1), (3, 4, 6, 2)])
def test_free_field_trace_is_fermi_dirac(orc, d, nx, ntau, order):
    """At A = 0 the diagonal of M^{-1} of the block form of Eq. (7) is the free
    equal-time Green's function: (1/N) tr M^{-1} = (1/V) sum_k 1 / (1 + E_k^N_tau),
    i.e. one minus the Fermi-Dirac occupation with E_k^N_tau in place of
    exp(-beta eps_k) (the antiperiodic Matsubara sum of 1 / (1 - E_k e^{-i w})).
    For reading R1 the trace is sum 1/lambda over the closed-form spectrum."""
    lat = orc.lattice(d, nx, ntau)
    n = orc.nsites(lat)
    L = orc.links(lat, 0.0, np.zeros(n))
    tr_ex = np.trace(np.linalg.inv(orc.dense(lat, H, L, "M", order=order))) / n
    E = _free_block_energies(d, nx, H, order)
    assert abs(tr_ex - np.mean(1.0 / (1.0 + E ** ntau))) < 1e-12
    tr_r1 = np.trace(np.linalg.inv(orc.dense(lat, H, L, "M"))) / n
    assert abs(tr_r1 - np.mean(1.0 / _free_eigs(d, nx, ntau, H, 1.0)).real) < 1e-12


def test_z2_noise_matches_numpy_philox(orc):
    for k, traj, chain in [(0, 0, 0), (3, 7, 2)]:
        eta = orc.z2_noise(11, k, traj, chain, 37)
        for i in range(37):
            w = _numpy_philox_block([i >> 2, 6 | (k << 8), traj, chain], [11, 0])
            assert eta[i] == (1.0 if w[i & 3] >> 63 else -1.0)
    big = orc.z2_noise(5, 1, 0, 0, 100000)
    assert set(np.unique(big)) == {-1.0, 1.0} and abs(big.mean()) < 0.02


@pytest.mark.parametrize("d,nx,ntau,order", [(1, 8, 8, 0), (1, 6, 6, 1), (3, 3, 4, 0), (3, 3, 4, 2)])
def test_observable_estimators_match_dense_inverse(orc, d, nx, ntau, order):
    """Every term of the estimators against the dense inverse, with the same
    noise vectors: t_k = (1/N) eta_k . M^{-1} eta_k, the half-set diagonal
    estimates and the field moments."""
    lat = orc.lattice(d, nx, ntau)
    n = orc.nsites(lat)
    prm = orc.params(cg_tol=1e-13, seed=21, link_order=order)
    sigma = orc.init_field(21, 0, n)
    Minv = np.linalg.inv(orc.dense(lat, H, orc.links(lat, 0.5, sigma), "M", order=order))
    nn = 6
    etas = [orc.z2_noise(21, k, 3, 0, n) for k in range(nn)]
    t = np.array([e @ Minv @ e / n for e in etas])
    g = [e * (Minv @ e) for e in etas]
    gA, gB = np.mean(g[: nn // 2], axis=0), np.mean(g[nn // 2:], axis=0)
    got = orc.observables(lat, prm, sigma, nn, 3)
    assert got["status"] == 0
    assert abs(got["trace_Minv"] - t.mean()) < 1e-9
    assert abs(got["trace_err"] - t.std(ddof=1) / np.sqrt(nn)) < 1e-9
    assert abs(got["one_minus_g_sq"] - np.mean((1 - gA) * (1 - gB))) < 1e-9
    assert abs(got["mean_sin"] - np.mean(np.sin(sigma))) < 1e-14
    assert abs(got["mean_sin2"] - np.mean(np.sin(sigma) ** 2)) < 1e-14


def test_observable_estimators_are_unbiased(orc):
    """Over many noise vectors the estimates approach the exact trace and
    (1/N) sum_i (1 - M^{-1}_ii)^2 of the dense inverse (within 5 standard
    errors; the product's error from the spread over independent runs)."""
    lat = orc.lattice(1, 6, 8)
    n = orc.nsites(lat)
    prm = orc.params(cg_tol=1e-12, seed=4)
    sigma = orc.init_field(4, 0, n)
    Minv = np.linalg.inv(orc.dense(lat, H, orc.links(lat, 0.5, sigma), "M"))
    exact_tr = np.trace(Minv) / n
    exact_p = np.mean((1 - np.diag(Minv)) ** 2)
    runs = [orc.observables(lat, prm, sigma, 32, traj) for traj in range(8)]
    tr = np.array([r["trace_Minv"] for r in runs])
    err = np.sqrt(np.sum([r["trace_err"] ** 2 for r in runs])) / len(runs)
    assert abs(tr.mean() - exact_tr) < 5 * err
    p = np.array([r["one_minus_g_sq"] for r in runs])
    assert abs(p.mean() - exact_p) < 5 * p.std(ddof=1) / np.sqrt(len(p))


@pytest.mark.parametrize("order", [1, 2])
def test_free_field_double_occupancy_estimate(orc, order):
    """At A = 0 every M^{-1}_ii of the block form is the same (translations in
    space and time), so (1/N) sum_i (1 - M^{-1}_ii)^2 = (1 - n_F)^2 with
    1 - n_F the Fermi-Dirac trace of the free-field pin: the product estimate
    over independent noise runs agrees within five standard errors."""
    d, nx, ntau = 1, 8, 8
    lat = orc.lattice(d, nx, ntau)
    n = orc.nsites(lat)
    prm = orc.params(cg_tol=1e-12, seed=9, A=0.0, link_order=order)
    E = _free_block_energies(d, nx, H, order)
    g = np.mean(1.0 / (1.0 + E ** ntau))
    runs = [orc.observables(lat, prm, np.zeros(n), 16, traj) for traj in range(8)]
    p = np.array([r["one_minus_g_sq"] for r in runs])
    assert abs(p.mean() - (1.0 - g) ** 2) < 5 * p.std(ddof=1) / np.sqrt(len(p)) + 1e-12
    assert all(abs(r["mean_sin"]) == 0.0 and r["mean_sin2"] == 0.0 for r in runs)


def _hop_matrix(d, nx):
    """Adjacency H of the periodic d-dimensional spatial lattice (x fastest)."""
    V = nx ** d
    Hm = np.zeros((V, V))
    for s in range(V):
        c = [(s // nx ** k) % nx for k in range(d)]
        for k in range(d):
            for step in (1, -1):
                cc = list(c)
                cc[k] = (cc[k] + step) % nx
                Hm[s, sum(cc[j] * nx ** j for j in range(d))] += 1.0
    return Hm


@pytest.mark.parametrize("d,nx,ntau,order", [(1, 4, 5, 1), (1, 5, 4, 2), (3, 2, 3, 1), (3, 3, 3, 2)])
def test_diagonal_blocks_are_equal_time_greens_functions(orc, d, nx, ntau, order):
    """The reading behind the observables (R13): for the block form of Eq. (7)
    with B_tau = E diag(1 + A sin sigma(., tau-1)) and the +B corner of the
    antiperiodic boundary, the tau-th diagonal block of M^{-1} is
    (1 + B_tau B_{tau-1} ... B_{tau+1})^{-1}, built here from sigma directly."""
    lat = orc.lattice(d, nx, ntau)
    n = orc.nsites(lat)
    V = nx ** d
    sigma = orc.init_field(3 + order, 0, n)
    Minv = np.linalg.inv(orc.dense(lat, H, orc.links(lat, 0.5, sigma), "M", order=order))
    Hm = _hop_matrix(d, nx)
    E = np.eye(V) + H * Hm + (0.5 * H * H * Hm @ Hm if order == 2 else 0.0)
    c = 1.0 + 0.5 * np.sin(sigma.reshape(ntau, V))
    B = [E @ np.diag(c[(tau - 1) % ntau]) for tau in range(ntau)]
    for tau in range(ntau):
        P = np.eye(V)
        for k in range(ntau):
            P = P @ B[(tau - k) % ntau]
        G = np.linalg.inv(np.eye(V) + P)
        assert np.max(np.abs(G - Minv[tau * V:(tau + 1) * V, tau * V:(tau + 1) * V])) < 1e-12


@pytest.mark.parametrize("d,nx,ntau", [(1, 6, 4), (3, 3, 3)])
def test_reading_r1_is_exp_k_times_block_form_to_first_order(orc, d, nx, ntau):
    """Reading R1 against the exact-block form at order 1: with D the diagonal
    blocks 1 - hH of M_R1 and S = M_R1 - D its link part, D M_ex1 = D + (1 - h^2
    H^2) S, so M_R1 = (1 - hH) M_ex1 + h^2 H^2 S: the two forms differ by the
    factor e^{dtau K} ~ 1 - hH on the left, to first order in h."""
    lat = orc.lattice(d, nx, ntau)
    n = orc.nsites(lat)
    V = nx ** d
    L = orc.links(lat, 0.5, orc.init_field(17, 0, n))
    M_r1 = orc.dense(lat, H, L, "M")
    M_ex1 = orc.dense(lat, H, L, "M", order=1)
    Hm = _hop_matrix(d, nx)
    D = np.kron(np.eye(ntau), np.eye(V) - H * Hm)
    S = M_r1 - D
    H2 = np.kron(np.eye(ntau), Hm @ Hm)
    assert np.max(np.abs(M_r1 - D @ M_ex1 - H * H * H2 @ S)) < 1e-13
