"""Pins of the oracle's Monte-Carlo q sampling (Sec. 4.3) and of the linear
tetrahedron population (Eq. pop)."""
import numpy as np

import synthetic as S
from oracle import eph as O


def test_cauchy_density_normalised_and_inverse_cdf():
    c = 0.15
    x = np.linspace(-0.5, 0.5, 200001)
    # density of the tangent map integrates to 1 over the zone (trapezoid on a fine grid)
    p = c / (c * c * np.cos(np.pi * x) ** 2 + np.sin(np.pi * x) ** 2)
    assert abs(np.trapezoid(p, x) - 1.0) < 1e-8
    # CDF of that density, F(x) = 1/2 + atan(tan(pi x)/c)/pi, inverts the map
    rng = np.random.default_rng(4)
    uu = rng.uniform(size=(1000, 3))
    q, pinv = O.mc_qpoints(uu, O.Q_CAUCHY, c)
    F = 0.5 + np.arctan(np.tan(np.pi * q) / c) / np.pi
    assert np.abs(F - uu).max() < 1e-12
    assert np.all(np.abs(q) <= 0.5)
    pd = c / (c * c * np.cos(np.pi * q) ** 2 + np.sin(np.pi * q) ** 2)
    assert np.allclose(1.0 / pinv, pd.prod(1), rtol=1e-13)
    # width 1 is the uniform map
    q1, w1 = O.mc_qpoints(uu, O.Q_CAUCHY, 1.0)
    q0, w0 = O.mc_qpoints(uu, O.Q_UNIFORM)
    assert np.allclose(q1, q0, atol=1e-14) and np.allclose(w1, 1.0) and np.all(w0 == 1.0)


def test_importance_weights_integrate_exactly_known_function():
    # int over the zone of g(q) = prod_i (1 + cos(2 pi q_i)) = 1; the Cauchy estimator
    # with weights 1/p is unbiased: the mean over many samples is 1 within 5 standard errors
    rng = np.random.default_rng(5)
    u = rng.uniform(size=(400000, 3))
    q, pinv = O.mc_qpoints(u, O.Q_CAUCHY, 0.3)
    y = np.prod(1 + np.cos(2 * np.pi * q), axis=1) * pinv
    se = y.std(ddof=1) / np.sqrt(len(y))
    assert abs(y.mean() - 1.0) < 5 * se


def test_uniform_mc_on_grid_points_is_the_grid_sum():
    # q = u - 1/2 on grid points (shifted by a whole grid step where needed) reproduces
    # the full-grid Gamma of scattering_rates_grid exactly
    m = S.model_c1()
    grid = (4, 4, 4)
    T, mu, sig = 300.0, 0.5, 0.05
    qg = S.mp_grid(*grid)
    u = (qg + 0.5) % 1.0
    kidx = np.array([0, 5, 37])
    kpts = S.mp_grid(*grid)[kidx]
    gam, err = O.scattering_rates_mc(m, kpts, u, O.Q_UNIFORM, 1.0, T, mu, sig)
    ref = O.scattering_rates_grid(m, grid, grid, kidx, T, mu, sig)
    assert np.abs(gam - ref).max() <= 1e-10 * ref.max()
    assert np.all(err >= 0)


def _tet_geometry_integral(V, e, f, E, npts=5):
    """int_T f theta(E - eps) dV / V_T for linear eps, f: slices eps = e' are triangles or
    quadrilaterals; int f delta(eps - e') dV = (int over the slice of f dA) / |grad eps|,
    a quadratic in e' on each interval between corner energies, integrated by Gauss-Legendre."""
    V = np.asarray(V, float)
    M = np.stack([V[1] - V[0], V[2] - V[0], V[3] - V[0]])
    vol = abs(np.linalg.det(M)) / 6.0
    grad = np.linalg.solve(M, np.array([e[1] - e[0], e[2] - e[0], e[3] - e[0]]))

    def slice_integral(ep):
        pts, vals = [], []
        for i in range(4):
            for j in range(i + 1, 4):
                if (ep - e[i]) * (ep - e[j]) < 0:
                    t = (ep - e[i]) / (e[j] - e[i])
                    pts.append(V[i] + t * (V[j] - V[i]))
                    vals.append(f[i] + t * (f[j] - f[i]))
        if len(pts) < 3:
            return 0.0
        pts, vals = np.array(pts), np.array(vals)
        cen = pts.mean(0)
        nrm = grad / np.linalg.norm(grad)
        ax = pts[0] - cen
        ax -= nrm * (ax @ nrm)
        ax /= np.linalg.norm(ax)
        ay = np.cross(nrm, ax)
        ang = np.arctan2((pts - cen) @ ay, (pts - cen) @ ax)
        o = np.argsort(ang)
        pts, vals = pts[o], vals[o]
        tot = 0.0
        for a in range(1, len(pts) - 1):     # fan triangulation of the convex polygon
            area = 0.5 * np.linalg.norm(np.cross(pts[a] - pts[0], pts[a + 1] - pts[0]))
            tot += area * (vals[0] + vals[a] + vals[a + 1]) / 3.0
        return tot / np.linalg.norm(grad)

    xs, ws = np.polynomial.legendre.leggauss(npts)
    es = np.sort(e)
    total = 0.0
    for lo, hi in zip(es[:-1], es[1:]):
        hi = min(hi, E)
        if hi <= lo:
            continue
        mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
        total += half * sum(w * slice_integral(mid + half * x) for x, w in zip(xs, ws))
    return total / vol


def test_tetra_weights_exact_for_linear_functions():
    rng = np.random.default_rng(6)
    for _ in range(6):
        V = rng.normal(size=(4, 3))
        e = rng.normal(size=4)
        f = rng.normal(size=4)
        for E in np.concatenate([np.sort(e) + 1e-3, np.linspace(e.min() - 0.2, e.max() + 0.2, 7)]):
            got = O.tetra_theta_weights(e[None], E)[0] @ f
            ref = _tet_geometry_integral(V, e, f, E)
            assert abs(got - ref) <= 1e-10 * (1 + abs(ref)), (E, got, ref)


def test_tetra_weights_continuous_and_full():
    rng = np.random.default_rng(7)
    e = rng.normal(size=(50, 4))
    for row in e:           # continuity across each corner energy
        for E0 in row:
            a = O.tetra_theta_weights(row[None], E0 - 1e-9)[0]
            b = O.tetra_theta_weights(row[None], E0 + 1e-9)[0]
            assert np.abs(a - b).max() < 1e-6
    assert np.allclose(O.tetra_theta_weights(e, 10.0), 0.25)
    assert np.all(O.tetra_theta_weights(e, -10.0) == 0.0)


def test_population_counts_and_monotone():
    # f = 1 on every state: N(E) above all bands = nb and 0 below; N is monotone for
    # f >= 0 and ends at the zone average of f summed over bands
    m = S.model_c1()
    grid = (6, 6, 6)
    eps, _ = O.bands(m, S.mp_grid(*grid))
    one = np.ones_like(eps)
    N = O.population_cumulative(eps, one, grid, [eps.min() - 1, eps.max() + 1])
    assert abs(N[0]) < 1e-14 and abs(N[1] - eps.shape[1]) < 1e-12
    # monotone in E for f >= 0
    E = np.linspace(eps.min(), eps.max(), 25)
    f = np.random.default_rng(8).uniform(size=eps.shape)
    Nf = O.population_cumulative(eps, f, grid, E)
    assert np.all(np.diff(Nf) >= -1e-15)
    assert abs(Nf[-1] - f.mean(0).sum()) < 1e-12
