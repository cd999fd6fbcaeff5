"""Pins of the oracle's reverse-mode derivatives of I[f] (Eq. e_ph_scattering)
and of the RK4 time stepping (Sec. 2.1.1)."""
import numpy as np

import synthetic as S
from oracle import eph as O


def _random_list(rng, ns=9, nnz=70):
    """An unsymmetric list with self-terms and a few dead (hw < omega_min) entries."""
    row = np.sort(rng.integers(0, ns, nnz))
    col = rng.integers(0, ns, nnz)
    col[:5] = row[:5]                                  # self-terms s -> s
    hw = rng.uniform(0.01, 0.06, nnz)
    hw[5:8] = 0.5 * O.OMEGA_MIN_EV
    g2 = rng.uniform(1e-4, 3e-3, nnz)
    eps = rng.uniform(0.0, 0.2, ns)
    return row, col, hw, g2, eps


def test_collision_vjp_matches_central_differences_unsymmetric_list():
    # I is quadratic in f and linear in |g|^2: central differences are exact up
    # to rounding, for any step.  An unsymmetric list makes J and J^T differ.
    rng = np.random.default_rng(11)
    row, col, hw, g2, eps = _random_list(rng)
    ns = len(eps)
    T, sig, nq = 300.0, 0.03, 8
    f = rng.uniform(0.05, 0.95, ns)
    lam = rng.normal(size=ns)

    def I(ff, gg):
        return O.collision(ff, eps, row, col, hw, gg, T, sig, nq)

    h = 1e-3
    J = np.empty((ns, ns))
    for c in range(ns):
        e = np.zeros(ns)
        e[c] = h
        J[:, c] = (I(f + e, g2) - I(f - e, g2)) / (2 * h)
    assert np.abs(J - J.T).max() > 1e-3 * np.abs(J).max()
    jt, dg2 = O.collision_vjp(f, lam, eps, row, col, hw, g2, T, sig, nq)
    ref = J.T @ lam
    assert np.abs(jt - ref).max() <= 1e-9 * np.abs(ref).max()

    hg = 1e-4
    fd = np.empty(len(g2))
    for e in range(len(g2)):
        d = np.zeros(len(g2))
        d[e] = hg
        fd[e] = lam @ (I(f, g2 + d) - I(f, g2 - d)) / (2 * hg)
    assert np.abs(dg2 - fd).max() <= 1e-9 * np.abs(fd).max()
    assert np.all(dg2[5:8] == 0.0)                     # dead entries carry nothing


def test_collision_vjp_symmetric_list_invariants():
    # On a symmetric list sum_s I_s = 0 for every f, so J^T 1 = 0; for a
    # partner pair (s -> s', s' -> s) with one shared |g|^2, the two |g|^2
    # derivatives of sum_s I_s cancel.
    m = S.model_c1()
    L = O.collision_list_grid(m, (2, 2, 2), 0, 2)
    T, sig = 300.0, 0.05
    rng = np.random.default_rng(3)
    f = rng.uniform(0.1, 0.9, L["nstates"])
    one = np.ones(L["nstates"])
    jt, dg2 = O.collision_vjp(f, one, L["eps"], L["row"], L["col"], L["hw"], L["g2"], T, sig, L["nq"])
    lam = rng.normal(size=L["nstates"])
    jt_l, _ = O.collision_vjp(f, lam, L["eps"], L["row"], L["col"], L["hw"], L["g2"], T, sig, L["nq"])
    assert np.abs(jt).max() <= 1e-12 * np.abs(jt_l).max()
    key = {(r, c, mo): i for i, (r, c, mo) in enumerate(zip(L["row"], L["col"], L["mode"]))}
    partner = np.array([key[(c, r, mo)] for r, c, mo in zip(L["row"], L["col"], L["mode"])])
    assert np.abs(dg2 + dg2[partner]).max() <= 1e-10 * np.abs(dg2).max()


def test_rk4_adjoint_is_the_transposed_taylor_polynomial_on_linear_systems():
    # rhs = A f: one RK4 step is P(dt A) f with P(z) = 1 + z + z^2/2 + z^3/6 + z^4/24,
    # so the adjoint of n steps is (P(dt A)^T)^n lam.
    rng = np.random.default_rng(8)
    A = rng.normal(size=(5, 5)) * 1e14                 # 1/s
    lam = rng.normal(size=5)
    f0 = rng.normal(size=5)
    dt_fs, n = 0.7, 6
    Z = dt_fs * O.FS * A
    P = np.eye(5) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    ref = np.linalg.matrix_power(P.T, n) @ lam
    got, th = O.rk4_adjoint(f0, dt_fs, n, lambda x: A @ x, lambda x, k: (A.T @ k, 0.0), lam)
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    assert th == 0.0


def _c1_dynamics():
    m = S.model_c1()
    L = O.collision_list_grid(m, (2, 2, 2), 0, 2)
    T, sig = 300.0, 0.05
    eps = L["eps"]
    f0 = S.pulse_occupations(eps, eps.min(), centre=2.0, width=1.0, amplitude=0.3)

    def rhs_g(f, g2):
        return O.collision(f, eps, L["row"], L["col"], L["hw"], g2, T, sig, L["nq"])

    def vjp(x, k):
        return O.collision_vjp(x, k, eps, L["row"], L["col"], L["hw"], L["g2"], T, sig, L["nq"])

    # step from the largest absolute row sum of the Jacobian (the stiffest rate)
    J = np.array([vjp(f0, e)[0] for e in np.eye(len(f0))])
    dt_fs = 0.2 / np.abs(J).sum(axis=1).max() / O.FS
    return L, f0, rhs_g, vjp, dt_fs


def test_rk4_adjoint_matches_finite_differences_of_evolve():
    L, f0, rhs_g, vjp, dt_fs = _c1_dynamics()
    n = 12
    rng = np.random.default_rng(21)
    w = rng.normal(size=len(f0))
    lam0, dg2 = O.rk4_adjoint(f0, dt_fs, n, lambda f: rhs_g(f, L["g2"]), vjp, w)

    def loss(f_init, g2):
        return w @ O.evolve(f_init, dt_fs, n, lambda f: rhs_g(f, g2))

    h = 1e-6
    for _ in range(3):
        d = rng.normal(size=len(f0))
        fd = (loss(f0 + h * d, L["g2"]) - loss(f0 - h * d, L["g2"])) / (2 * h)
        assert abs(lam0 @ d - fd) <= 1e-7 * max(abs(fd), np.abs(lam0).max())
    for _ in range(3):
        d = rng.normal(size=len(L["g2"])) * L["g2"]
        fd = (loss(f0, L["g2"] + h * d) - loss(f0, L["g2"] - h * d)) / (2 * h)
        assert abs(dg2 @ d - fd) <= 1e-7 * max(abs(fd), np.abs(dg2 * L["g2"]).max())


def test_rk4_adjoint_carries_the_number_covector_unchanged():
    # The carrier number sum_s f_s is conserved on a symmetric list, so
    # d(sum f(t_end))/df0 = 1 and its |g|^2 derivative vanishes.
    L, f0, rhs_g, vjp, dt_fs = _c1_dynamics()
    lam0, dg2 = O.rk4_adjoint(f0, dt_fs, 10, lambda f: rhs_g(f, L["g2"]), vjp, np.ones(len(f0)))
    assert np.abs(lam0 - 1.0).max() < 1e-12
    _, dg2w = O.rk4_adjoint(f0, dt_fs, 10, lambda f: rhs_g(f, L["g2"]), vjp, np.linspace(-1, 1, len(f0)))
    assert np.abs(np.sum(dg2 * L["g2"])) <= 1e-10 * np.abs(dg2w * L["g2"]).max()
