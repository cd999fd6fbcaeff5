"""Pins of the oracle's RTA rates and collision integral (Eqs. scatter_rate, BTE_W, e_ph_scattering)."""
import numpy as np
import pytest

import synthetic as S
from oracle import eph as O

HBAR, EV, AMU, BOHR, KB = 6.582119569e-16, 1.602176634e-19, 1.66053906660e-27, 0.529177210903e-10, 8.617333262e-5


def einstein_holstein(eps0=0.0, t=-0.1, kE=2.0, mass=28.0, g0=(0.02, 0.02, 0.02)):
    m = S.model_sc_tight_binding(eps0=eps0, t=t, mass=mass, g0=np.array(g0, dtype=complex))
    r0 = int(np.nonzero((m.R_D == 0).all(1))[0][0])
    D = np.zeros_like(m.D)
    D[r0] = kE * np.eye(3)        # dispersionless (Einstein) phonon, no other R
    m.D = D
    return m


def test_rates_one_band_einstein_closed_form():
    """1 band eps(k) = eps0 + 2t sum cos, Einstein phonon hw0, local coupling g0.

    Gamma_k = (2pi/hbar)(1/Nq) sum_q G2 [delta(e_k - hw0 - e_k+q)(1 + N - f_k+q)
                                         + delta(e_k + hw0 - e_k+q)(N + f_k+q)],
    G2 = hbar/(2 M w0) sum_a |g0_a|^2, evaluated by hand loops over the grid.
    """
    kE, M, t, T, mu, sig = 2.0, 28.0, -0.02, 300.0, 0.01, 0.004
    g0 = np.array([0.02, 0.01 + 0.02j, 0.015])
    m = einstein_holstein(t=t, kE=kE, mass=M, g0=g0)
    grid = (4, 4, 4)
    kidx = [0, 5, 21, 63]
    gam = O.scattering_rates_grid(m, grid, grid, kidx, T, mu, sig)
    w0 = np.sqrt(kE / M * EV / (AMU * BOHR ** 2))            # rad/s
    hw0 = HBAR * w0
    G2 = HBAR * EV / (2 * M * AMU * w0) / BOHR ** 2 * np.sum(np.abs(g0) ** 2)
    N = 1 / (np.exp(hw0 / (KB * T)) - 1)
    pts = S.mp_grid(*grid)

    def eps(k):
        return 2 * t * sum(np.cos(2 * np.pi * k[i]) for i in range(3))

    def dl(x):
        return np.exp(-(x / sig) ** 2) / (sig * np.sqrt(np.pi))

    for a, ik in enumerate(kidx):
        tot = 0.0
        for q in pts:
            ekq = eps(pts[ik] + q)
            fkq = 1 / (np.exp((ekq - mu) / (KB * T)) + 1)
            ek = eps(pts[ik])
            tot += G2 * (dl(ek - hw0 - ekq) * (1 + N - fkq) + dl(ek + hw0 - ekq) * (N + fkq))
        ref = 2 * np.pi / HBAR * tot / len(pts)
        assert np.isclose(gam[a, 0], ref, rtol=1e-11), (gam[a, 0], ref)


@pytest.fixture(scope="module")
def c1_list():
    m = S.model_c1()
    return m, O.collision_list_grid(m, (3, 3, 3), 0, 2)


def test_rates_positive_and_mode_sum(c1_list):
    m, _ = c1_list
    kidx = list(range(27))
    g = O.scattering_rates_grid(m, (3, 3, 3), (3, 3, 3), kidx, 300.0, 0.5, 0.05)
    gm = O.scattering_rates_grid(m, (3, 3, 3), (3, 3, 3), kidx, 300.0, 0.5, 0.05, mode_resolved=True)
    assert np.all(g >= 0) and np.mean(g > 0) > 0.9   # the band bottom can have no final state
    assert np.allclose(gm.sum(axis=1), g, rtol=1e-13)


def test_rates_equal_minus_diagonal_of_collision(c1_list):
    """Gamma_s = -dI_s/df_s at equilibrium occupations.

    I_s is affine in f_s when the other occupations are fixed, and its slope is
    minus the bracket of Eq. BTE_W, so two independently written functions
    (grid rates vs entry-list collision) must agree.  The q = 0, m = n self
    terms differ (the collision slope cancels there); they carry
    delta(hw_optical) ~ exp(-(50 meV/sigma)^2) and are negligible.
    """
    m, L = c1_list
    T, mu, sig = 300.0, 0.5, 0.02
    g = O.scattering_rates_grid(m, (3, 3, 3), (3, 3, 3), list(range(27)), T, mu, sig)
    f0 = O.fermi_dirac(L["eps"], mu, T)
    base = O.collision(f0, L["eps"], L["row"], L["col"], L["hw"], L["g2"], T, sig, L["nq"])
    for s in (0, 7, 30, 53):
        h = 1e-3
        f1 = f0.copy()
        f1[s] += h
        I1 = O.collision(f1, L["eps"], L["row"], L["col"], L["hw"], L["g2"], T, sig, L["nq"])
        slope = (I1[s] - base[s]) / h
        assert np.isclose(-slope, g.reshape(-1)[s], rtol=1e-8), (s, -slope, g.reshape(-1)[s])


def test_collision_conserves_carriers(c1_list):
    _, L = c1_list
    rng = np.random.default_rng(3)
    f = rng.uniform(0, 1, L["nstates"])
    I = O.collision(f, L["eps"], L["row"], L["col"], L["hw"], L["g2"], 300.0, 0.02, L["nq"])
    scale = np.abs(I).max()
    assert abs(I.sum()) < 1e-12 * scale * len(I)


def test_detailed_balance_ladder():
    # Flat bands spaced by exactly hw0 and an Einstein phonon of energy hw0:
    # every process conserves energy, so Fermi-Dirac electrons with Bose-Einstein
    # phonons give I = 0 up to the Gaussian tails exp(-(hw0/sigma)^2) ~ 1e-44.
    s, M = 0.05, 28.0
    kE = s ** 2 * M / O.C_OMEGA
    m = S.model_ladder(nw=3, spacing=s, einstein_k=kE, mass=M)
    L = O.collision_list_grid(m, (2, 2, 2), 0, 3)
    T, mu, sig = 300.0, 0.04, 0.005
    f0 = O.fermi_dirac(L["eps"], mu, T)
    I = O.collision(f0, L["eps"], L["row"], L["col"], L["hw"], L["g2"], T, sig, L["nq"])
    # scale: the out-scattering rate alone
    g = O.scattering_rates_grid(m, (2, 2, 2), (2, 2, 2), list(range(8)), T, mu, sig).reshape(-1)
    assert np.abs(I).max() < 1e-12 * np.max(g * f0)
    # a non-equilibrium occupation does scatter
    I2 = O.collision(f0 * 1.1, L["eps"], L["row"], L["col"], L["hw"], L["g2"], T, sig, L["nq"])
    assert np.abs(I2).max() > 1e-3 * np.max(g * f0)


def test_collision_rows_match_list_and_window():
    # The per-row evaluation (interpolation at the initial k only) and the
    # symmetric list give the same I_s; a window removes out-of-window states
    # from both.
    m = S.model_c1()
    rng = np.random.default_rng(5)
    L = O.collision_list_grid(m, (3, 3, 3), 0, 2)
    f = rng.uniform(0, 1, L["nstates"])
    I = O.collision(f, L["eps"], L["row"], L["col"], L["hw"], L["g2"], 300.0, 0.02, L["nq"])
    rows = [1, 9, 30, 53]
    r = O.collision_rows(m, (3, 3, 3), 0, 2, rows, f, 300.0, 0.02)
    assert np.allclose(r, I[rows], rtol=1e-11, atol=1e-12 * np.abs(I).max())
    win = (np.median(L["eps"]) - 0.5, np.median(L["eps"]) + 1.0)
    Lw = O.collision_list_grid(m, (3, 3, 3), 0, 2, window=win)
    inw = (L["eps"] >= win[0]) & (L["eps"] <= win[1])
    assert inw.sum() < len(inw) and np.all(inw[Lw["row"]]) and np.all(inw[Lw["col"]])
    Iw = O.collision(f, Lw["eps"], Lw["row"], Lw["col"], Lw["hw"], Lw["g2"], 300.0, 0.02, Lw["nq"])
    sel = [s for s in range(54) if inw[s]][:4]
    rw = O.collision_rows(m, (3, 3, 3), 0, 2, sel, f, 300.0, 0.02, window=win)
    assert np.allclose(rw, Iw[sel], rtol=1e-11, atol=1e-12 * np.abs(Iw).max())
    assert abs(Iw.sum()) < 1e-12 * np.abs(Iw).max() * len(Iw)
