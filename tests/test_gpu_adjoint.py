"""Reverse-mode derivatives on the GPU (through the C ABI) against the FP64 oracle.

The library's entry coefficients are FP32 and its entry products FP32 with
compensated sums, like the forward collision kernel, so the derivatives are
held to 1e-5 (one application) and 1e-4 (40 RK4 steps, |g|^2 derivative)
of the largest reference component.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import eph as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

T, SIG, GRID = 300.0, 0.02, (3, 3, 3)


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
def c1():
    return S.model_c1()


@pytest.fixture(scope="module")
def full_list(c1):
    return O.collision_list_grid(c1, GRID, 0, 2)


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def sub_list(L, keep):
    return {**L, **{k: L[k][keep] for k in ("row", "col", "mode", "g2", "hw")}}


def build(ctx, c1, L):
    ctx.pgb_set_model(c1)
    ctx.pgb_set_grids(GRID, GRID)
    ctx.pgb_build_collision(0, 2, T, SIG, dev(L["row"].astype(np.int32)), dev(L["col"].astype(np.int32)),
                            dev(L["mode"].astype(np.int32)), dev(L["g2"].astype(np.float32)))


def oracle_fns(L):
    g2 = L["g2"].astype(np.float32).astype(np.float64)   # the list is handed over in FP32

    def rhs(f):
        return O.collision(f, L["eps"], L["row"], L["col"], L["hw"], g2, T, SIG, L["nq"])

    def vjp(x, k):
        return O.collision_vjp(x, k, L["eps"], L["row"], L["col"], L["hw"], g2, T, SIG, L["nq"])
    return rhs, vjp


def close(got, ref, tol):
    return np.abs(got - ref).max() <= tol * np.abs(ref).max()


def test_collision_vjp_unsymmetric_list(ctx, c1, full_list):
    # dropping a random 30% of the entries leaves a list whose J is not the
    # transpose of itself: the column sums must run over the true transpose
    rng = np.random.default_rng(40)
    L = sub_list(full_list, rng.uniform(size=len(full_list["row"])) < 0.7)
    build(ctx, c1, L)
    ns = L["nstates"]
    f = rng.uniform(0.05, 0.95, ns)
    lam = rng.normal(size=ns)
    vf = torch.empty(ns, dtype=torch.float64, device="cuda")
    vg = torch.empty(len(L["row"]), dtype=torch.float64, device="cuda")
    ctx.pgb_collision_vjp(dev(f), dev(lam), vf, vg)
    _, vjp = oracle_fns(L)
    rf, rg = vjp(f, lam)
    assert close(vf.cpu().numpy(), rf, 1e-5)
    assert close(vg.cpu().numpy(), rg, 1e-5)
    # host buffers give the same numbers
    hf, hg = np.zeros(ns), np.zeros(len(L["row"]))
    ctx.pgb_collision_vjp(f, lam, hf, hg)
    assert np.array_equal(hf, vf.cpu().numpy()) and np.array_equal(hg, vg.cpu().numpy())


def test_collision_vjp_symmetric_list_number_covector(ctx, c1, full_list):
    L = full_list
    build(ctx, c1, L)
    ns = L["nstates"]
    rng = np.random.default_rng(41)
    f = rng.uniform(0.05, 0.95, ns)
    vf = np.zeros(ns)
    ctx.pgb_collision_vjp(f, np.ones(ns), vf, None)
    ref, _ = oracle_fns(L)[1](f, rng.normal(size=ns))
    assert np.abs(vf).max() <= 1e-5 * np.abs(ref).max()


def test_rk4_adjoint_matches_oracle(ctx, c1, full_list):
    L = full_list
    build(ctx, c1, L)
    ns, nnz = L["nstates"], len(L["row"])
    f0 = S.pulse_occupations(L["eps"], L["eps"].min(), centre=3.0, width=1.0, amplitude=0.2)
    rng = np.random.default_rng(42)
    lam_end = rng.normal(size=ns)
    n, dt = 40, 1.0
    rhs, vjp = oracle_fns(L)
    r0, rg = O.rk4_adjoint(f0, dt, n, rhs, vjp, lam_end)
    outs = {}
    for ck in (1, 7, 40, 1000):
        lam0 = torch.empty(ns, dtype=torch.float64, device="cuda")
        dg2 = torch.empty(nnz, dtype=torch.float64, device="cuda")
        fe = torch.empty(ns, dtype=torch.float64, device="cuda")
        ctx.pgb_rk4_adjoint(dev(f0), dt, n, ck, dev(lam_end), lam0, dg2, fe)
        outs[ck] = (lam0.cpu().numpy(), dg2.cpu().numpy(), fe.cpu().numpy())
    lam0, dg2, fe = outs[7]
    assert close(lam0, r0, 1e-5)
    assert close(dg2, rg, 1e-4)
    assert np.abs(lam0 - lam_end).max() > 1e-3 * np.abs(lam_end).max()   # the dynamics did act
    # checkpoint spacing changes nothing: recomputed states are bit-identical
    for ck in (1, 40, 1000):
        assert all(np.array_equal(a, b) for a, b in zip(outs[ck], outs[7]))
    # f(t_end) is pgb_step_rk4's, bit for bit
    f = dev(f0)
    ctx.pgb_step_rk4(f, dt, n)
    assert np.array_equal(fe, f.cpu().numpy())


def test_rk4_adjoint_with_empty_rows(ctx, c1):
    # an energy window leaves states without entries: their f stays f0 and
    # their derivative is lam_end, in every buffer of the checkpointed sweep
    eps = O.collision_list_grid(c1, GRID, 0, 2)["eps"]
    lo = float(np.quantile(eps, 0.2))
    L = O.collision_list_grid(c1, GRID, 0, 2, window=(lo, float(eps.max())))
    build(ctx, c1, L)
    ns, nnz = L["nstates"], len(L["row"])
    empty = np.setdiff1d(np.arange(ns), np.union1d(L["row"], L["col"]))
    assert len(empty) > 0
    f0 = S.pulse_occupations(L["eps"], L["eps"].min(), centre=3.0, width=1.0, amplitude=0.2)
    lam_end = np.random.default_rng(45).normal(size=ns)
    n, dt = 23, 1.0
    lam0, dg2, fe = np.zeros(ns), np.zeros(nnz), np.zeros(ns)
    ctx.pgb_rk4_adjoint(f0, dt, n, 5, lam_end, lam0, dg2, fe)
    f = f0.copy()
    ctx.pgb_step_rk4(f, dt, n)
    assert np.array_equal(fe, f)
    assert np.array_equal(fe[empty], f0[empty]) and np.array_equal(lam0[empty], lam_end[empty])
    r0, rg = O.rk4_adjoint(f0, dt, n, *oracle_fns(L), lam_end)
    assert close(lam0, r0, 1e-5)
    assert close(dg2, rg, 1e-4)


def test_rk4_adjoint_number_covector_and_zero_steps(ctx, c1, full_list):
    L = full_list
    build(ctx, c1, L)
    ns, nnz = L["nstates"], len(L["row"])
    f0 = S.pulse_occupations(L["eps"], L["eps"].min(), centre=3.0, width=1.0, amplitude=0.2)
    lam0 = np.zeros(ns)
    ctx.pgb_rk4_adjoint(f0, 1.0, 30, 8, np.ones(ns), lam0)
    assert np.abs(lam0 - 1.0).max() < 1e-6
    lam_end = np.linspace(-1, 1, ns)
    dg2 = np.full(nnz, 7.0)
    fe = np.zeros(ns)
    ctx.pgb_rk4_adjoint(f0, 1.0, 0, 8, lam_end, lam0, dg2, fe)
    assert np.array_equal(lam0, lam_end) and np.all(dg2 == 0.0) and np.array_equal(fe, f0)


def test_adjoint_empty_list(ctx, c1):
    ctx.pgb_set_model(c1)
    ctx.pgb_set_grids((2, 2, 2), (2, 2, 2))
    e = np.zeros(0, np.int32)
    ctx.pgb_build_collision(0, 2, T, SIG, e, e, e, np.zeros(0, np.float32))
    ns = 16
    lam_end = np.arange(ns, dtype=np.float64)
    lam0 = np.zeros(ns)
    ctx.pgb_rk4_adjoint(np.full(ns, 0.5), 1.0, 5, 2, lam_end, lam0)
    assert np.array_equal(lam0, lam_end)
    vf = np.ones(ns)
    ctx.pgb_collision_vjp(np.full(ns, 0.5), lam_end, vf, None)
    assert np.all(vf == 0.0)


def test_set_g2_scales_exactly(ctx, c1, full_list):
    # a, b are linear in |g|^2 and doubling is exact in floating point
    L = full_list
    build(ctx, c1, L)
    ns = L["nstates"]
    rng = np.random.default_rng(43)
    f, lam = rng.uniform(0.05, 0.95, ns), rng.normal(size=ns)
    I1, v1 = np.zeros(ns), np.zeros(ns)
    ctx.pgb_collision(f, I1)
    ctx.pgb_collision_vjp(f, lam, v1, None)
    ctx.pgb_collision_set_g2(dev(2 * L["g2"].astype(np.float32)))
    I2, v2 = np.zeros(ns), np.zeros(ns)
    ctx.pgb_collision(f, I2)
    ctx.pgb_collision_vjp(f, lam, v2, None)
    assert np.array_equal(I2, 2 * I1) and np.array_equal(v2, 2 * v1)
    g2 = np.zeros(len(L["row"]), np.float32)
    ctx.pgb_collision_list(g2=g2)
    assert np.array_equal(g2, 2 * L["g2"].astype(np.float32))


def test_autograd_functions(ctx, c1, full_list):
    from paper_2002_02045_gb300 import autograd as AG
    L = full_list
    build(ctx, c1, L)
    ns, nnz = L["nstates"], len(L["row"])
    g2 = dev(L["g2"].astype(np.float32)).requires_grad_(True)
    lst = AG.CollisionList(ctx, g2)
    f0 = S.pulse_occupations(L["eps"], L["eps"].min(), centre=3.0, width=1.0, amplitude=0.2)
    f0t = dev(f0).requires_grad_(True)
    w = dev(np.random.default_rng(44).normal(size=ns))
    loss = (AG.rk4(f0t, g2, lst, 1.0, 25, checkpoint=10) * w).sum()
    loss.backward()
    lam0, dg2 = np.zeros(ns), np.zeros(nnz)
    ctx.pgb_rk4_adjoint(f0, 1.0, 25, 10, w.cpu().numpy(), lam0, dg2)
    assert np.array_equal(f0t.grad.cpu().numpy(), lam0)
    assert np.array_equal(g2.grad.cpu().numpy(), dg2.astype(np.float32))
    # the single-application function as well
    f0t.grad = None
    g2.grad = None
    I = AG.collision(f0t, g2, lst)
    (I * w).sum().backward()
    vf, vg = np.zeros(ns), np.zeros(nnz)
    ctx.pgb_collision_vjp(f0, w.cpu().numpy(), vf, vg)
    assert np.array_equal(f0t.grad.cpu().numpy(), vf)
    assert np.array_equal(g2.grad.cpu().numpy(), vg.astype(np.float32))
    # a new |g|^2 tensor updates the list before the next evaluation
    I_ref = I.detach().cpu().numpy()
    I2 = AG.collision(f0t.detach(), (2 * g2).detach(), lst)
    assert np.array_equal(I2.cpu().numpy(), 2 * I_ref)


@pytest.mark.slow
def test_rk4_adjoint_full_size_finite_differences(ctx):
    # The real-time workload: fcc model, 30^3 grid, two lowest bands, states
    # within 0.6 eV of the band minimum, ~1.2e8 entries; 1000 steps of 1 fs from
    # the hot-carrier pulse; L = mean carrier energy at t_end.  At this size the
    # oracle cannot run, so the gradients are checked against central
    # differences of the library's own forward along random directions (the
    # step h = 1e-3 relative keeps the FP32 rounding of the gathered f far
    # below the perturbation), and the carrier-number covector must come back
    # as 1.
    m = S.model_c2()
    ctx.pgb_set_model(m)
    grid = (30, 30, 30)
    ctx.pgb_set_grids(grid, grid)
    nk = 27000
    eps = torch.empty((nk, m.nw), dtype=torch.float64, device="cuda")
    ctx.pgb_get_grid_energies(eps, None)
    emin = float(eps[:, :2].min())
    nnz = ctx.pgb_build_collision_grid(0, 2, emin, emin + 0.6, 300.0, 0.010)
    assert nnz > 5e7
    ns = 2 * nk
    es = torch.empty(ns, dtype=torch.float64, device="cuda")
    ctx.pgb_collision_energies(es)
    f0 = torch.as_tensor(S.pulse_occupations(es.cpu().numpy(), emin)).cuda()
    g2 = torch.empty(nnz, dtype=torch.float32, device="cuda")
    ctx.pgb_collision_list(g2=g2)
    n_steps, dt = 1000, 1.0

    def loss(f_init):
        f = f_init.clone()
        ctx.pgb_step_rk4(f, dt, n_steps)
        return float((es * f).sum() / f.sum()), f

    L0, fe = loss(f0)
    lam_end = (es - L0) / fe.sum()
    lam0 = torch.empty_like(f0)
    dg2 = torch.empty(nnz, dtype=torch.float64, device="cuda")
    fe2 = torch.empty_like(f0)
    ctx.pgb_rk4_adjoint(f0, dt, n_steps, 50, lam_end, lam0, dg2, fe2)
    assert torch.equal(fe, fe2)
    gen = torch.Generator(device="cuda").manual_seed(7)
    h = 1e-3
    for _ in range(2):
        d = torch.randn(ns, generator=gen, device="cuda", dtype=torch.float64) * f0
        fd = (loss(f0 + h * d)[0] - loss(f0 - h * d)[0]) / (2 * h)
        ad = float((lam0 * d).sum())
        assert abs(ad - fd) <= 2e-3 * abs(fd)
    d = torch.randn(nnz, generator=gen, device="cuda", dtype=torch.float32) * g2
    ctx.pgb_collision_set_g2((g2 + h * d).contiguous())
    lp = loss(f0)[0]
    ctx.pgb_collision_set_g2((g2 - h * d).contiguous())
    lm = loss(f0)[0]
    ctx.pgb_collision_set_g2(g2)
    fd = (lp - lm) / (2 * h)
    ad = float((dg2 * d.double()).sum())
    assert abs(ad - fd) <= 2e-3 * abs(fd)
    ones = torch.ones(ns, dtype=torch.float64, device="cuda")
    ctx.pgb_rk4_adjoint(f0, dt, 200, 50, ones, lam0)
    assert float((lam0 - 1.0).abs().max()) < 1e-5
