"""Pins of the oracle's polar coupling (Eq. e_ph_long), band velocities
(Eqs. velocity, wannier_4), iterative BTE (Eqs. BTE_lin, BTE_iter, BTE_W) and
mobility (Eq. cond)."""
import numpy as np
import scipy.special

import synthetic as S
from oracle import eph as O


C3 = None


def c3():
    global C3
    if C3 is None:
        C3 = S.model_c3()
    return C3


def test_frohlich_periodic_and_conjugate():
    m = c3()
    q = np.random.default_rng(1).uniform(-0.5, 0.5, (7, 3))
    L = O.frohlich_wannier(m, q)
    assert np.abs(L).max() > 0.1
    # the G sum runs over every q+G, so a reciprocal-lattice shift changes nothing
    assert np.abs(O.frohlich_wannier(m, q + np.array([2.0, -1.0, 1.0])) - L).max() <= 1e-12 * np.abs(L).max()
    # (q+G).Z* and the phase are odd, the rest even: L(-q) = conj(L(q))
    assert np.abs(O.frohlich_wannier(m, -q) - np.conj(L)).max() <= 1e-12 * np.abs(L).max()


def test_frohlich_small_q_limit():
    # q -> 0 along u: only G = 0 diverges, t L(t u) -> i (e^2/eps0 Omega) (u.Z*)_a / (u.eps.u)
    m = c3()
    B = O.reciprocal_vectors(m.A)
    omega = abs(np.linalg.det(m.A))
    pref = 4 * np.pi * O.HARTREE_EV / omega
    for u in (np.array([0.3, -0.1, 0.2]), np.array([0.0, 0.0, 1.0])):
        t = 1e-6
        L = O.frohlich_wannier(m, (t * u)[None])[0].reshape(m.nat, 3)
        uc = u @ B
        den = uc @ m.eps_inf @ uc
        ref = np.stack([1j * pref * (uc @ m.zstar[k]) / den for k in range(m.nat)])
        assert np.abs(t * L - ref).max() <= 1e-5 * np.abs(ref).max()


def test_frohlich_matches_plain_g_loop():
    # independent enumeration: a much larger integer box, one G at a time
    m = c3()
    B = O.reciprocal_vectors(m.A)
    omega = abs(np.linalg.det(m.A))
    lam = m.ewald_lambda
    q = np.array([0.17, -0.05, 0.31])
    ref = np.zeros((m.nat, 3), complex)
    for n1 in range(-9, 10):
        for n2 in range(-9, 10):
            for n3 in range(-9, 10):
                v = (q + np.array([n1, n2, n3])) @ B
                x = v @ m.eps_inf @ v
                if x / (4 * lam) > O.EWALD_CUT:
                    continue
                for k in range(m.nat):
                    ref[k] += (1j * 4 * np.pi * O.HARTREE_EV / omega * (v @ m.zstar[k])
                               * np.exp(-1j * v @ m.tau[k]) * np.exp(-x / (4 * lam)) / x)
    L = O.frohlich_wannier(m, q[None])[0].reshape(m.nat, 3)
    assert np.abs(L - ref).max() <= 1e-12 * np.abs(ref).max()


def test_long_range_term_is_the_smooth_phase_braket():
    # Eq. smooth_phase: the Bloch-gauge long-range term is L [U^dagger(k+q) U(k)]_mn
    m = c3()
    rng = np.random.default_rng(2)
    k, q = rng.uniform(size=(1, 3)), rng.uniform(size=(1, 3))
    _, Uk = O.bands(m, k)
    _, Ukq = O.bands(m, k + q)
    full = O.g_bloch(O.g_wannier_full(m, k, q)[0, 0], Uk[0], Ukq[0])
    short = O.g_bloch(O.g_wannier(m, k, q)[0, 0], Uk[0], Ukq[0])
    L = O.frohlich_wannier(m, q)[0]
    ref = short + L[:, None, None] * (np.conj(Ukq[0]).T @ Uk[0])[None]
    assert np.abs(full - ref).max() <= 1e-12 * np.abs(ref).max()


def test_velocities_are_band_derivatives():
    m = c3()
    k = np.random.default_rng(3).uniform(size=(4, 3))
    v = O.velocities(m, k)
    h = 1e-6
    for a in range(3):
        dk = np.zeros(3)
        dk[a] = h
        dkc = dk @ m.A.T / (2 * np.pi)              # Cartesian step in crystal coordinates
        ep, _ = O.bands(m, k + dkc)
        em, _ = O.bands(m, k - dkc)
        fd = (ep - em) / (2 * h) * O.BOHR_M / O.HBAR_EVS
        assert np.abs(fd - v[:, :, a]).max() <= 1e-6 * np.abs(v).max()


def _split_pair_model(t=-0.2, delta=0.05, a=6.0):
    # H(k) = V [2t cos(2 pi k_x) I + delta sin(2 pi k_x) sigma_z] V^dagger: the two bands
    # touch at k_x = 0 with slopes 2 pi delta a-units apart
    R = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0]], dtype=np.int32)
    sz = np.diag([1.0, -1.0])
    th = 0.7
    V = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]]) * np.exp(0.3j)
    Hp = t * np.eye(2) + delta / 2j * sz
    H = np.stack([np.zeros((2, 2)), V @ Hp @ V.conj().T, V @ Hp.conj().T @ V.conj().T]).astype(complex)
    z = np.zeros((3, 3, 3))
    return S.Model("split", a * np.eye(3), np.zeros((1, 3)), np.array([1.0]), R, H, R, z, R, R,
                   np.zeros((1, 1, 3, 2, 2)))


def test_degenerate_velocities_are_the_one_sided_slopes():
    m = _split_pair_model()
    k = np.array([[0.0, 0.2, 0.4]])                 # degenerate point (k_x = 0)
    v = O.velocities(m, k)[0]                        # [2, 3]
    h = 1e-7
    dkc = np.array([h, 0, 0]) @ m.A.T / (2 * np.pi)
    e0, _ = O.bands(m, k)
    ep, _ = O.bands(m, k + dkc)
    slopes = np.sort((ep - e0)[0] / h) * O.BOHR_M / O.HBAR_EVS
    assert np.abs(np.sort(v[:, 0]) - slopes).max() <= 1e-5 * np.abs(slopes).max()
    assert abs(slopes[1] - slopes[0]) > 0.1 * np.abs(slopes).max()   # the two really differ


def test_bte_weights_sum_to_the_rates():
    # Gamma_nk = (1/N_q) sum_{m nu q} W (Eq. scatter_rate) on a full unscreened list
    m = S.model_c1()
    grid = (2, 2, 2)
    L = O.collision_list_grid(m, grid, 0, m.nw)
    T, mu, sig = 300.0, 0.4, 0.05
    w = O.bte_weights(L["eps"], L["row"], L["col"], L["hw"], L["g2"], T, mu, sig, L["nq"])
    gam = np.zeros(L["nstates"])
    np.add.at(gam, L["row"], w)
    ref = O.scattering_rates_grid(m, grid, grid, np.arange(8), T, mu, sig).reshape(-1)
    assert np.abs(gam - ref).max() <= 1e-9 * ref.max()


def test_bte_iteration_reaches_the_direct_solution():
    rng = np.random.default_rng(5)
    ns, nnz = 12, 60
    row = np.sort(rng.integers(0, ns, nnz))
    col = rng.integers(0, ns, nnz)
    w = rng.uniform(0, 1e13, nnz)
    gam = np.zeros(ns)
    np.add.at(gam, row, w)
    tau = 1.0 / (gam + 2e13)                          # keeps tau W a contraction
    v = rng.normal(size=(ns, 3)) * 1e5
    F, it = O.bte_iterate(tau, v, row, col, w, max_iter=500, tol=1e-14)
    Wd = np.zeros((ns, ns))
    np.add.at(Wd, (row, col), w)
    ref = np.linalg.solve(np.eye(ns) - tau[:, None] * Wd, tau[:, None] * v)
    assert it < 500
    assert np.abs(F - ref).max() <= 1e-12 * np.abs(ref).max()
    F1, it1 = O.bte_iterate(tau, v, row, col, np.zeros(nnz))
    assert it1 == 1 and np.array_equal(F1, tau[:, None] * v)


def test_mobility_constant_tau_tight_binding_closed_form():
    # one cosine band, constant tau, Boltzmann statistics (mu far below the band):
    # mu_xx = (tau / kT) <v_x^2>, and on an N-point axis with x = -2t/kT
    # <sin^2> = (1 - r)/2, r = sum_p I_{2+pN}(x) / sum_p I_{pN}(x) (exact, aliased Bessel sums)
    t, a, T, N, tau = -0.1, 5.0, 300.0, 16, 1e-14
    m = S.model_sc_tight_binding(eps0=0.0, t=t, a=a)
    pts = S.mp_grid(N, N, N)
    eps, _ = O.bands(m, pts)
    v = O.velocities(m, pts)[:, 0, :]
    mu_chem = eps.min() - 1.0
    mob = O.mobility(v, tau * v, eps[:, 0], T, mu_chem)
    kT = O.KB_EVK * T
    x = -2 * t / kT
    ps = np.arange(-4, 5)
    r = scipy.special.iv(2 + ps * N, x).sum() / scipy.special.iv(ps * N, x).sum()
    v0 = 2 * abs(t) * a * O.BOHR_M / O.HBAR_EVS       # 2|t| a / hbar in m/s
    ref = 1e4 * tau / kT * v0 ** 2 * (1 - r) / 2
    assert abs(mob[0, 0] - ref) <= 1e-9 * ref
    assert np.allclose(np.diag(mob), ref, rtol=1e-9)
    assert np.abs(mob - np.diag(np.diag(mob))).max() <= 1e-9 * ref
