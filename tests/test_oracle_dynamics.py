"""Pins of the oracle's time stepping (Sec. 2.1.1: explicit RK4 and Euler)."""
import numpy as np
import scipy.linalg

import synthetic as S
from oracle import eph as O


def test_rk4_is_the_degree4_taylor_polynomial_on_linear_systems():
    # For df/dt = A f the classic RK4 step is exactly P(dt A) f with
    # P(z) = 1 + z + z^2/2 + z^3/6 + z^4/24; Euler is 1 + z.
    rng = np.random.default_rng(5)
    A = rng.normal(size=(4, 4))
    f = rng.normal(size=4)
    dt = 0.1
    Z = dt * A
    P4 = np.eye(4) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    assert np.allclose(O.rk4_step(f, dt, lambda x: A @ x), P4 @ f, rtol=1e-14, atol=1e-14)
    assert np.allclose(O.euler_step(f, dt, lambda x: A @ x), f + Z @ f, rtol=1e-15)


def test_convergence_orders_two_state():
    # Two states exchanging carriers at rates a (1->2) and b (2->1):
    # the exact solution is expm(t A) f0.  RK4 error ~ dt^4, Euler ~ dt.
    a, b = 2.0, 0.7
    A = np.array([[-a, b], [a, -b]])
    f0 = np.array([0.9, 0.1])
    t_end = 1.0
    exact = scipy.linalg.expm(t_end * A) @ f0

    def run(step, n):
        f = f0.copy()
        for _ in range(n):
            f = step(f, t_end / n, lambda x: A @ x)
        return np.abs(f - exact).max()

    e1, e2 = run(O.rk4_step, 20), run(O.rk4_step, 40)
    assert 14 < e1 / e2 < 18          # 2^4
    e1, e2 = run(O.euler_step, 200), run(O.euler_step, 400)
    assert 1.8 < e1 / e2 < 2.2        # 2^1


def test_carrier_number_conserved_and_equilibrates_ladder():
    # Flat ladder with exact energy conservation: the carrier number is conserved
    # to rounding and f relaxes to Fermi-Dirac at the lattice temperature with
    # the chemical potential fixed by the conserved number (the paper's long-time
    # limit, Sec. 5.4).
    s, M = 0.05, 28.0
    kE = s ** 2 * M / O.C_OMEGA
    m = S.model_ladder(nw=3, spacing=s, einstein_k=kE, mass=M, g0=0.05)
    L = O.collision_list_grid(m, (2, 2, 2), 0, 3)
    T, sig = 300.0, 0.005
    eps = L["eps"]
    f0 = S.pulse_occupations(eps, 0.0, centre=0.1, width=0.03, amplitude=0.3)

    def rhs(f):
        return O.collision(f, eps, L["row"], L["col"], L["hw"], L["g2"], T, sig, L["nq"])

    rate = np.abs(rhs(f0)).max() / f0.max()
    dt_fs = 0.2 / rate / O.FS
    f = O.evolve(f0, dt_fs, 400, rhs)
    assert abs(f.sum() - f0.sum()) < 1e-12 * f0.sum()
    # fit mu from the conserved number and compare with Fermi-Dirac
    lo, hi = -1.0, 1.0
    for _ in range(200):
        mu = 0.5 * (lo + hi)
        if O.fermi_dirac(eps, mu, T).sum() > f.sum():
            hi = mu
        else:
            lo = mu
    assert np.abs(f - O.fermi_dirac(eps, mu, T)).max() < 1e-6


def test_rk4_conserves_on_c1_list():
    m = S.model_c1()
    L = O.collision_list_grid(m, (3, 3, 3), 0, 2)
    T, sig = 300.0, 0.02
    eps = L["eps"]
    f0 = S.pulse_occupations(eps, eps.min(), centre=3.0, width=1.0, amplitude=0.2)

    def rhs(f):
        return O.collision(f, eps, L["row"], L["col"], L["hw"], L["g2"], T, sig, L["nq"])

    f = O.evolve(f0, 1.0, 30, rhs)
    assert abs(f.sum() - f0.sum()) < 1e-13 * f0.sum()
    assert not np.allclose(f, f0)
