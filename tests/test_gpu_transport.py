"""Polar coupling, band velocities and the iterative BTE on the GPU (through the
C ABI) against the FP64 oracle."""
import numpy as np
import pytest

import synthetic as S
from oracle import eph as O

from helpers import assert_close_blocks, assert_rates_close, degenerate_sum

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


@pytest.fixture(scope="module")
def c3():
    return S.model_c3()


@pytest.fixture(scope="module")
def c3s():
    # the polar model with its 19 shortest lattice vectors (fast oracle)
    return S.model_c3(rcut=13.0)


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def empty(shape, dtype=torch.float64):
    return torch.empty(shape, dtype=dtype, device="cuda")


def set_polar_model(ctx, m):
    ctx.pgb_set_model(m)
    ctx.pgb_set_lattice(m.A, m.tau)
    ctx.pgb_set_polar(m.zstar, m.eps_inf, m.ewald_lambda)


def test_long_range_g_matches_oracle(ctx, c3s):
    m = c3s
    rng = np.random.default_rng(30)
    q = np.concatenate([rng.uniform(-1, 1, (9, 3)), [[0.0, 0.0, 0.0], [1e-3, 0.0, 0.0], [0.0, -2e-4, 5e-4]]])
    set_polar_model(ctx, m)
    out = np.zeros((len(q), m.nmode, 2))
    ctx.pgb_long_range_g(q, out)
    got = out[..., 0] + 1j * out[..., 1]
    ref = O.frohlich_wannier(m, q)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
    ctx.pgb_set_polar(None)
    ctx.pgb_long_range_g(q, out)
    assert np.all(out == 0.0)


def oracle_g2_full(m, k, q):
    ek, Uk = O.bands(m, k)
    hw, e = O.phonons(m, q)
    out = np.zeros((len(k), len(q), m.nmode, m.nw, m.nw))
    for a in range(len(k)):
        _, Ukq = O.bands(m, k[a:a + 1] + q)
        gw = O.g_wannier_full(m, k[a:a + 1], q)[0]
        out[a] = np.abs(O.g_modes(O.g_bloch(gw, Uk[a][None], Ukq), hw, e, m.mass)) ** 2
    return out, hw


@pytest.mark.parametrize("prec,tol,floor", [("fp64", 1e-10, 1e-3), ("fp32", 1e-5, 1e-2), ("tf32x3", 1e-5, 1e-2),
                                            ("bf16x3", 1e-3, 1e-2)])
def test_polar_interpolate_g(ctx, c3, prec, tol, floor):
    from paper_2002_02045_gb300 import PGB_G2_FULL, PRECISIONS
    m = c3
    rng = np.random.default_rng(31)
    k = rng.uniform(-0.5, 0.5, (2, 3))
    q = np.concatenate([rng.uniform(-0.5, 0.5, (4, 3)), [[0.02, -0.01, 0.0]]])
    set_polar_model(ctx, m)
    out = empty((2, 5, 6, 8, 8))
    ctx.pgb_interpolate_g(dev(k), dev(q), PRECISIONS[prec], PGB_G2_FULL, out)
    ref, hw = oracle_g2_full(m, k, q)
    got = out.cpu().numpy()
    hwb = np.broadcast_to(hw[None], (2, 5, 6))
    assert_close_blocks(degenerate_sum(got, hwb, 2), degenerate_sum(ref, hwb, 2), tol, block_axes=(2, 3, 4),
                        floor=floor, label=f"polar g2 {prec}")
    # the long-range term is not negligible here (small q)
    ctx.pgb_set_polar(None)
    ctx.pgb_interpolate_g(dev(k), dev(q), PRECISIONS[prec], PGB_G2_FULL, out)
    assert np.abs(out.cpu().numpy() - got).max() > 0.05 * np.abs(got).max()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5), ("tf32x3", 1e-5), ("bf16x3", 1e-3)])
def test_polar_rates(ctx, c3, prec, tol):
    from paper_2002_02045_gb300 import PRECISIONS
    m = c3
    T, sig = 300.0, 0.010
    kg, qg = (12, 12, 12), (6, 6, 6)
    set_polar_model(ctx, m)
    ctx.pgb_set_grids(kg, qg)
    e_ref, _ = O.bands(m, S.mp_grid(*kg))
    emin = e_ref.min()
    mu = emin - 0.3
    win = np.nonzero(((e_ref >= emin + 1e-9) & (e_ref <= emin + 0.5)).any(1))[0].astype(np.int32)
    sample = win[:: max(1, len(win) // 5)][:5]
    gam = empty((len(sample), 8))
    ctx.pgb_scattering_rates(dev(sample), T, mu, sig, PRECISIONS[prec], gam)
    ref = O.scattering_rates_grid(m, kg, qg, sample, T, mu, sig)
    assert_rates_close(gam.cpu().numpy(), ref, tol, label=f"polar gamma {prec}")


def test_band_velocities_match_oracle(ctx, c3):
    m = c3
    ctx.pgb_set_model(m)
    ctx.pgb_set_lattice(m.A, m.tau)
    grid = (10, 10, 10)
    ctx.pgb_set_grids(grid, grid)
    kidx = np.arange(0, 1000, 37, dtype=np.int32)
    v = np.zeros((len(kidx), 8, 3))
    ctx.pgb_band_velocities(kidx, v)
    ref = O.velocities(m, S.mp_grid(*grid)[kidx])
    assert np.abs(v - ref).max() <= 1e-10 * np.abs(ref).max()


def test_band_velocities_degenerate_point(ctx):
    # two bands touching along k_x = 0 in an arbitrary gauge (see the oracle pin)
    R = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0]], dtype=np.int32)
    sz = np.diag([1.0, -1.0])
    V = np.array([[np.cos(0.7), -np.sin(0.7)], [np.sin(0.7), np.cos(0.7)]]) * np.exp(0.3j)
    Hp = -0.2 * np.eye(2) + 0.05 / 2j * sz
    H = np.stack([np.zeros((2, 2)), V @ Hp @ V.conj().T, V @ Hp.conj().T @ V.conj().T]).astype(complex)
    D = np.stack([np.eye(3), -0.5 * np.eye(3), -0.5 * np.eye(3)])
    m = S.Model("split", 6.0 * np.eye(3), np.zeros((1, 3)), np.array([1.0]), R, H, R, D, R, R,
                np.zeros((3, 3, 3, 2, 2), complex))
    ctx.pgb_set_model(m)
    ctx.pgb_set_lattice(m.A, m.tau)
    grid = (4, 5, 5)
    ctx.pgb_set_grids(grid, grid)
    kidx = np.arange(100, dtype=np.int32)
    v = np.zeros((100, 2, 3))
    ctx.pgb_band_velocities(kidx, v)
    ref = O.velocities(m, S.mp_grid(*grid)[kidx])
    assert np.abs(v - ref).max() <= 1e-9 * np.abs(ref).max()
    assert np.abs(ref[0, 1, 0] - ref[0, 0, 0]) > 0.1 * np.abs(ref[0, :, 0]).max()   # k = 0: split slopes


def _oracle_transport(m, grid, T, mu, sig, L, win, n_iter):
    pts = S.mp_grid(*grid)
    es = L["eps"]
    ns = len(es)
    kw = np.unique(np.nonzero(win)[0] // 2)
    gam = O.scattering_rates_grid(m, grid, grid, kw, T, mu, sig)
    vel = O.velocities(m, pts[kw])
    pos = {k: i for i, k in enumerate(kw)}
    tau = np.zeros(ns)
    v = np.zeros((ns, 3))
    for s in np.nonzero(win)[0]:
        tau[s] = 1.0 / gam[pos[s // 2], s % 2]
        v[s] = vel[pos[s // 2], s % 2]
    w = O.bte_weights(es, L["row"], L["col"], L["hw"], L["g2"], T, mu, sig, L["nq"])
    F, it = O.bte_iterate(tau, v, L["row"], L["col"], w, n_iter, 0.0)
    mob_rta = O.mobility(v[win], (tau[:, None] * v)[win], es[win], T, mu)
    mob = O.mobility(v[win], F[win], es[win], T, mu)
    _oracle_transport.last = {"v": v, "w": w}
    return tau, F, it, mob_rta, mob


def test_transport_shared_list_matches_oracle(ctx, c3s):
    # the oracle's own list (every state, FP32 |g|^2 shared by both sides):
    # tau, 300 iterations of F and both mobilities
    from paper_2002_02045_gb300 import PGB_FP64
    m = c3s
    grid, T, sig = (4, 4, 4), 300.0, 0.03
    set_polar_model(ctx, m)
    ctx.pgb_set_grids(grid, grid)
    L = O.collision_list_grid(m, grid, 0, 2)
    L["g2"] = L["g2"].astype(np.float32).astype(np.float64)
    ctx.pgb_build_collision(0, 2, T, sig, L["row"].astype(np.int32), L["col"].astype(np.int32),
                            L["mode"].astype(np.int32), L["g2"].astype(np.float32))
    mu = L["eps"].min() - 0.2
    ns = L["nstates"]
    F = np.zeros((ns, 3))
    tau = np.zeros(ns)
    mob_rta, mob, it = ctx.pgb_transport(mu, PGB_FP64, 300, 0.0, F, tau)
    tau_r, F_r, it_r, mr_r, m_r = _oracle_transport(m, grid, T, mu, sig, L, np.ones(ns, bool), 300)
    assert it == it_r == 300
    assert np.abs(tau - tau_r).max() <= 1e-9 * tau_r.max()
    assert np.abs(F - F_r).max() <= 1e-7 * np.abs(F_r).max()
    assert np.abs(mob_rta - mr_r).max() <= 1e-8 * np.abs(mr_r).max()
    assert np.abs(mob - m_r).max() <= 1e-7 * np.abs(m_r).max()
    assert np.abs(mob - mob_rta).max() > 1e-3 * np.abs(mob_rta).max()   # the iteration matters


def test_transport_grid_list_window(ctx, c3s):
    # the device-built list with an energy window: tau and the RTA mobility are
    # tight; F after 200 iterations carries the list's FP32 |g|^2 rounding,
    # amplified by the near-unit spectral radius of tau W
    from paper_2002_02045_gb300 import PGB_FP64
    m = c3s
    grid, T, sig = (6, 6, 6), 300.0, 0.02
    set_polar_model(ctx, m)
    ctx.pgb_set_grids(grid, grid)
    pts = S.mp_grid(*grid)
    eps_all, _ = O.bands(m, pts)
    emin = eps_all[:, :2].min()
    # window edges away from any state energy (membership must not hang on rounding)
    lo, hi = emin - 1e-6, emin + 0.4
    assert np.abs(eps_all[:, :2] - hi).min() > 1e-6
    mu = emin - 0.2
    nnz = ctx.pgb_build_collision_grid(0, 2, lo, hi, T, sig)
    ns = 2 * len(pts)
    F = np.zeros((ns, 3))
    tau = np.zeros(ns)
    mob_rta, mob, it = ctx.pgb_transport(mu, PGB_FP64, 200, 0.0, F, tau)
    L = O.collision_list_grid(m, grid, 0, 2, window=(lo, hi))
    win = (L["eps"] >= lo) & (L["eps"] <= hi)
    n_it = 200
    tau_r, F_r, it_r, mr_r, m_r = _oracle_transport(m, grid, T, mu, sig, L, win, n_it)
    assert it == it_r == n_it
    assert np.abs(tau - tau_r).max() <= 1e-9 * tau_r.max()
    assert np.all(tau[~win] == 0.0) and np.all(F[~win] == 0.0)
    assert np.abs(mob_rta - mr_r).max() <= 1e-8 * np.abs(mr_r).max()
    assert np.abs(F - F_r).max() <= 1e-3 * np.abs(F_r).max()
    assert np.abs(mob - m_r).max() <= 1e-3 * np.abs(m_r).max()
    # A bound from the conditioning of the iteration F <- tau (v + W F) (Eq. BTE_iter): the
    # device list's |g|^2 (FP32 interpolation, 7 sigma screen) give W + dW, and after n
    # iterations
    #   |dF|_inf <= sum_{j<n} r^j |tau dW|_inf max_i |F_i|_inf  (first order),
    # r = |tau W|_inf <= 1 since the row sums of W over a full list are the rates 1/tau.
    # The iteration sees W only through its mode sums per (row, col) pair, which are gauge
    # free at degenerate q; W, tau and F are the oracle's, dW = the device list's pair sums
    # (its entries take hbar*omega from the oracle's entry of the same key) minus the oracle's.
    row = np.zeros(nnz, np.int32)
    col = np.zeros(nnz, np.int32)
    mode = np.zeros(nnz, np.int32)
    g2 = np.zeros(nnz, np.float32)
    ctx.pgb_collision_list(row, col, mode, g2)
    nm = m.D.shape[1]
    key_d = (row.astype(np.int64) * ns + col) * nm + mode
    key_o = (L["row"].astype(np.int64) * ns + L["col"]) * nm + L["mode"]
    oo = np.argsort(key_o)
    pos = np.searchsorted(key_o[oo], key_d)
    assert np.all(pos < len(oo)) and np.array_equal(key_o[oo][pos], key_d)   # device keys within the oracle's
    match = oo[pos]
    w_o = _oracle_transport.last["w"]
    w_d = O.bte_weights(L["eps"], row, col, L["hw"][match], g2.astype(np.float64), T, mu, sig, L["nq"])
    pair_o = L["row"].astype(np.int64) * ns + L["col"]
    pair_d = row.astype(np.int64) * ns + col
    pairs, inv = np.unique(np.concatenate([pair_o, pair_d]), return_inverse=True)
    dWp = np.bincount(inv[len(pair_o):], weights=w_d, minlength=len(pairs)) - \
        np.bincount(inv[:len(pair_o)], weights=w_o, minlength=len(pairs))
    prow = pairs // ns
    rs = L["row"]
    r_inf = np.bincount(rs, weights=tau_r[rs] * w_o, minlength=ns).max()
    dW_inf = np.bincount(prow, weights=tau_r[prow] * np.abs(dWp), minlength=ns).max()
    amp = float(n_it) if r_inf >= 1.0 else (1.0 - r_inf ** n_it) / (1.0 - r_inf)
    # plus the tau deviation (<= 1e-9 relative, checked above), which enters F^0 and tau W
    bound_F = 2.0 * amp * (dW_inf + 2e-9) * np.abs(F_r).max() + 1e-10 * np.abs(F_r).max()
    err_F = np.abs(F - F_r).max()
    assert err_F <= bound_F, f"F: {err_F:.3g} > conditioning bound {bound_F:.3g} (r = {r_inf:.6f})"
    v_r = _oracle_transport.last["v"]
    bound_mob = O.mobility(np.abs(v_r[win]), np.full((int(win.sum()), 3), bound_F), L["eps"][win], T, mu)
    assert np.all(np.abs(mob - m_r) <= bound_mob + 1e-10 * np.abs(m_r).max())


@pytest.mark.slow
def test_transport_full_size_polar(ctx, c3):
    # the polar model at full size: 60^3 k = q grid, states within 0.2 eV of the band minimum,
    # tau from the BF16-split rates over all 216,000 q.  The oracle cannot run at
    # this size; check properties that hold at any size.
    from paper_2002_02045_gb300 import PGB_TC_BF16X3
    m = c3
    grid = (60, 60, 60)
    set_polar_model(ctx, m)
    ctx.pgb_set_grids(grid, grid)
    nk = 216000
    eps = empty((nk, 8))
    ctx.pgb_get_grid_energies(eps, None)
    emin = float(eps[:, :2].min())
    nnz = ctx.pgb_build_collision_grid(0, 2, emin - 1e-6, emin + 0.2, 300.0, 0.010)
    assert nnz > 0
    ns = 2 * nk
    F = empty((ns, 3))
    tau = empty((ns,))
    mob_rta, mob, it = ctx.pgb_transport(emin - 0.3, PGB_TC_BF16X3, 3000, 1e-6, F, tau)
    assert it < 3000
    assert np.all(np.isfinite(mob)) and np.all(np.diag(mob) > 0) and np.all(np.diag(mob_rta) > 0)
    # RTA mobility from the returned tau and the velocities equals the library's
    es = empty((ns,))
    ctx.pgb_collision_energies(es)
    es = es.cpu().numpy()
    t = tau.cpu().numpy()
    win = (es >= emin - 1e-6) & (es <= emin + 0.2)
    assert np.all(t[win] > 0) and np.all(t[~win] == 0)
    ks = np.unique(np.nonzero(win)[0] // 2).astype(np.int32)
    v = np.zeros((len(ks), 8, 3))
    ctx.pgb_band_velocities(ks, v)
    pos = {k: i for i, k in enumerate(ks)}
    s_w = np.nonzero(win)[0]
    vs = np.stack([v[pos[s // 2], s % 2] for s in s_w])
    ref_rta = O.mobility(vs, t[s_w, None] * vs, es[s_w], 300.0, emin - 0.3)
    assert np.abs(mob_rta - ref_rta).max() <= 1e-10 * np.abs(ref_rta).max()
