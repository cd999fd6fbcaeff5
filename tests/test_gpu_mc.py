"""Monte-Carlo q rates and tetrahedron populations on the GPU (through the C ABI)
against the FP64 oracle, on the same caller-supplied uniforms."""
import numpy as np
import pytest

import synthetic as S
from oracle import eph as O

from helpers import assert_rates_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_02045_gb300 import build
    build.build()
    from paper_2002_02045_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def test_mc_uniform_on_grid_points_equals_grid_rates(ctx):
    from paper_2002_02045_gb300 import PGB_FP64, PGB_Q_UNIFORM
    m = S.model_c1()
    grid = (6, 6, 6)
    T, mu, sig = 300.0, 0.5, 0.02
    ctx.pgb_set_model(m)
    ctx.pgb_set_grids(grid, grid)
    kidx = np.array([0, 7, 100, 215], np.int32)
    ref = np.zeros((4, 2))
    ctx.pgb_scattering_rates(kidx, T, mu, sig, PGB_FP64, ref)
    u = (S.mp_grid(*grid) + 0.5) % 1.0
    got = np.zeros((4, 2))
    err = np.zeros((4, 2))
    ctx.pgb_scattering_rates_mc(S.mp_grid(*grid)[kidx], u, PGB_Q_UNIFORM, 1.0, T, mu, sig, PGB_FP64, got, err)
    assert_rates_close(got, ref, 1e-10, label="mc on grid")
    assert np.all(err >= 0) and np.all(err[ref > 0] > 0)


@pytest.mark.parametrize("sampling,width", [(0, 1.0), (1, 0.2)])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5), ("tf32x3", 1e-5), ("bf16x3", 1e-3)])
def test_mc_random_matches_oracle(ctx, sampling, width, prec, tol):
    from paper_2002_02045_gb300 import PRECISIONS
    m = S.model_c1()
    T, mu, sig = 300.0, 0.5, 0.02
    ctx.pgb_set_model(m)
    rng = np.random.default_rng(50 + sampling)
    k = rng.uniform(-0.5, 0.5, (3, 3))
    u = rng.uniform(size=(9001, 3))        # several q chunks and a ragged tail
    got = np.zeros((3, 2))
    err = np.zeros((3, 2))
    ctx.pgb_scattering_rates_mc(k, u, sampling, width, T, mu, sig, PRECISIONS[prec], got, err)
    ref, ref_err = O.scattering_rates_mc(m, k, u, sampling, width, T, mu, sig)
    assert_rates_close(got, ref, tol, label=f"mc {sampling} {prec}")
    assert np.abs(err - ref_err).max() <= 1e3 * tol * ref_err.max() + 1e-300


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("tf32x3", 1e-5), ("bf16x3", 1e-3)])
def test_mc_polar_c3(ctx, prec, tol):
    from paper_2002_02045_gb300 import PRECISIONS, PGB_Q_CAUCHY
    m = S.model_c3(rcut=13.0)
    ctx.pgb_set_model(m)
    ctx.pgb_set_lattice(m.A, m.tau)
    ctx.pgb_set_polar(m.zstar, m.eps_inf, m.ewald_lambda)
    T, sig = 300.0, 0.02
    rng = np.random.default_rng(52)
    k = rng.uniform(-0.2, 0.2, (2, 3))
    eps_k, _ = O.bands(m, k)
    mu = eps_k.min() - 0.3
    u = rng.uniform(size=(700, 3))
    got = np.zeros((2, 8))
    ctx.pgb_scattering_rates_mc(k, u, PGB_Q_CAUCHY, 0.1, T, mu, sig, PRECISIONS[prec], got)
    ref, _ = O.scattering_rates_mc(m, k, u, O.Q_CAUCHY, 0.1, T, mu, sig)
    assert_rates_close(got, ref, tol, label=f"mc polar {prec}")


def test_mc_argument_errors(ctx):
    from paper_2002_02045_gb300 import PgbError, PGB_FP64
    ctx.pgb_set_model(S.model_c1())
    k = np.zeros((1, 3))
    out = np.zeros((1, 2))
    for u, samp, w, prec in ((np.full((4, 3), 1.0), 0, 1.0, PGB_FP64), (np.full((4, 3), 0.2), 1, 0.0, PGB_FP64),
                             (np.full((4, 3), 0.2), 0, 1.0, 99), (np.full((4, 3), 0.2), 7, 1.0, PGB_FP64)):
        with pytest.raises(PgbError):
            ctx.pgb_scattering_rates_mc(k, u, samp, w, 300.0, 0.5, 0.02, prec, out)


@pytest.mark.parametrize("grid", [(6, 6, 6), (5, 4, 7)])
def test_population_matches_oracle(ctx, grid):
    m = S.model_c1()
    ctx.pgb_set_model(m)
    ctx.pgb_set_grids(grid, grid)
    e = np.zeros(0, np.int32)
    ctx.pgb_build_collision(0, 2, 300.0, 0.02, e, e, e, np.zeros(0, np.float32))
    nk = int(np.prod(grid))
    es = np.zeros(2 * nk)
    ctx.pgb_collision_energies(es)
    f = np.random.default_rng(53).uniform(size=2 * nk)
    E = np.linspace(es.min() - 0.1, es.max() + 0.1, 41)
    N = np.zeros(len(E))
    ctx.pgb_population(f, E, N)
    eps, _ = O.bands(m, S.mp_grid(*grid))
    ref = O.population_cumulative(eps, f.reshape(nk, 2), grid, E)
    assert np.abs(N - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    assert abs(N[-1] - f.reshape(nk, 2).mean(0).sum()) < 1e-12
