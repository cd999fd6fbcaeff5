"""Batched rates of uneven instances (one persistent launch under a captured
graph) against the per-instance FP64 oracle."""
import numpy as np
import pytest

import synthetic as S
from oracle import eph as O

from helpers import assert_rates_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GRID = (8, 8, 8)
T, SIG = 300.0, 0.05


@pytest.fixture(scope="module")
def members():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_02045_gb300 import build
    build.build()
    from paper_2002_02045_gb300 import Context
    models = [S.model_batch_instance(i) for i in (1, 2, 3, 7, 8, 9)] + [S.model_c3(rcut=13.0)]
    ctxs, ks, mus = [], [], []
    rng = np.random.default_rng(60)
    for m in models:
        c = Context(0)
        c.pgb_set_model(m)
        if m.zstar is not None:
            c.pgb_set_lattice(m.A, m.tau)
            c.pgb_set_polar(m.zstar, m.eps_inf, m.ewald_lambda)
        c.pgb_set_grids(GRID, GRID)
        eps = np.zeros((512, m.nw))
        c.pgb_get_grid_energies(eps, None)
        ctxs.append(c)
        ks.append(np.sort(rng.choice(512, 3, replace=False)).astype(np.int32))
        mus.append(float(0.5 * (eps.min() + eps.max())))
    yield models, ctxs, ks, mus
    for c in ctxs:
        c.close()


def test_batch_matches_oracle_and_single_calls(members):
    from paper_2002_02045_gb300 import Batch, PGB_FP32
    models, ctxs, ks, mus = members
    b = Batch(ctxs)
    outs = [np.zeros((len(k), m.nw)) for k, m in zip(ks, models)]
    b.pgb_batch_rates(ks, T, mus, SIG, outs)
    tun = b.pgb_batch_tuning()
    assert tun["tile_q"] in (8, 16, 32, 64) and tun["threads"] in (128, 256, 512)
    assert min(x for x in tun["candidate_ms"] if x >= 0) > 0
    for i, (m, c, k, mu) in enumerate(zip(models, ctxs, ks, mus)):
        single = np.zeros((len(k), m.nw))
        c.pgb_scattering_rates(k, T, mu, SIG, PGB_FP32, single)
        assert_rates_close(outs[i], single, 1e-5, label=f"batch vs single {i}")
        ref = O.scattering_rates_grid(m, GRID, GRID, k, T, mu, SIG)
        assert_rates_close(outs[i], ref, 1e-5, label=f"batch vs oracle {i}")
        assert np.abs(outs[i]).max() > 0
    # the same arguments replay the captured graph, bit for bit
    outs2 = [np.zeros_like(o) for o in outs]
    b.pgb_batch_rates(ks, T, mus, SIG, outs2)
    assert b.pgb_batch_tuning()["graph_launches"] == 2
    assert all(np.array_equal(x, y) for x, y in zip(outs, outs2))
    # new arguments re-capture (device buffers in and out)
    k_dev = [torch.as_tensor(k[:2]).cuda() for k in ks]
    out_dev = [torch.empty((2, m.nw), dtype=torch.float64, device="cuda") for m in models]
    b.pgb_batch_rates(k_dev, T, mus, SIG, out_dev)
    for o, o1 in zip(out_dev, outs):
        assert np.array_equal(o.cpu().numpy(), o1[:2])
    b.close()


def test_batch_argument_errors(members):
    from paper_2002_02045_gb300 import Batch, PgbError
    models, ctxs, ks, mus = members
    b = Batch(ctxs[:2])
    outs = [np.zeros((3, m.nw)) for m in models[:2]]
    bad = [ks[0], np.array([0, 10 ** 6], np.int32)]
    with pytest.raises(PgbError):
        b.pgb_batch_rates(bad, T, mus[:2], SIG, outs)
    with pytest.raises(PgbError):
        b.pgb_batch_rates(ks[:2], -1.0, mus[:2], SIG, outs)
    b.close()


@pytest.mark.parametrize("prec,tol", [("bf16x3", 1e-3), ("tf32x3", 1e-5)])
def test_batch_tensor_core_route(members, prec, tol):
    """With a split precision every instance takes the R_p sum on the tensor cores
    (columns padded to a multiple of 96 where needed: two of the six random ones
    here; the polar instance with its long-range rows) inside the same graph."""
    from paper_2002_02045_gb300 import Batch, PGB_FP32, PRECISIONS, PgbError
    models, ctxs, ks, mus = members
    eligible = [m.zstar is None for m in models]
    assert 0 < sum(eligible) < len(models)
    b = Batch(ctxs)
    with pytest.raises(PgbError):
        b.pgb_batch_set_precision(99)
    b.pgb_batch_set_precision(PRECISIONS[prec])
    outs = [np.zeros((len(k), m.nw)) for k, m in zip(ks, models)]
    b.pgb_batch_rates(ks, T, mus, SIG, outs)
    for i, (m, k, mu) in enumerate(zip(models, ks, mus)):
        ref = O.scattering_rates_grid(m, GRID, GRID, k, T, mu, SIG)
        assert_rates_close(outs[i], ref, tol, label=f"batch {prec} vs oracle {i}")
        assert np.abs(outs[i]).max() > 0
    # replay is bit for bit; back to FP32 re-plans and re-tunes
    outs2 = [np.zeros_like(o) for o in outs]
    b.pgb_batch_rates(ks, T, mus, SIG, outs2)
    assert all(np.array_equal(x, y) for x, y in zip(outs, outs2))
    b.pgb_batch_set_precision(PGB_FP32)
    outs3 = [np.zeros_like(o) for o in outs]
    b.pgb_batch_rates(ks, T, mus, SIG, outs3)
    for i in range(len(models)):
        assert_rates_close(outs3[i], outs[i], max(tol, 1e-5), label=f"fp32 vs {prec} {i}")
    b.close()


@pytest.mark.slow
def test_batch_own_settings_against_oracle():
    """The batched instances at their own settings: sigma = 5 meV and T = 300 K on the instances'
    own grids (8^3 to 32^3), with nw = 16, nat = 5 and the 123-vector R shell among
    them, in FP32, TF32x3 and BF16x3 through one batch, against the per-instance FP64
    oracle on sampled k-points (the full q grid of each)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_02045_gb300 import Batch, Context, PRECISIONS, build
    build.build()
    # (instance, sampled k): 44 = nw 16, nat 5, 123 R, 32^3; 34 = nw 8, nat 5, 123 R, 32^3;
    # 13 = nw 4, nat 5, 32^3; 10 = nw 2, nat 1, 32^3; 17 = nw 16, nat 5, 33 R, 12^3;
    # 41 = nw 12, nat 5, 24^3; 5 = nw 8, nat 3, 123 R, 8^3
    pick = {44: 1, 34: 1, 13: 1, 10: 2, 17: 2, 41: 1, 5: 2}
    sig = 0.005
    models = [S.model_batch_instance(i) for i in pick]
    rng = np.random.default_rng(61)
    ctxs, ks, mus, refs = [], [], [], []
    for m, nk in zip(models, pick.values()):
        g = m.meta["grid"]
        assert m.meta["sigma"] == sig
        c = Context(0)
        c.pgb_set_model(m)
        c.pgb_set_grids(g, g)
        ngrid = int(np.prod(g))
        eps = np.zeros((ngrid, m.nw))
        c.pgb_get_grid_energies(eps, None)
        ctxs.append(c)
        ks.append(np.sort(rng.choice(ngrid, nk, replace=False)).astype(np.int32))
        mus.append(float(0.5 * (eps.min() + eps.max())))
        refs.append(O.scattering_rates_grid(m, g, g, ks[-1], T, mus[-1], sig, q_chunk=4096))
    assert any(m.nw == 16 and m.nat == 5 and m.meta["grid"][0] == 32 for m in models)
    b = Batch(ctxs)
    for prec, tol in (("fp32", 1e-5), ("tf32x3", 1e-5), ("bf16x3", 1e-3)):
        b.pgb_batch_set_precision(PRECISIONS[prec])
        outs = [np.zeros((len(k), m.nw)) for k, m in zip(ks, models)]
        b.pgb_batch_rates(ks, T, mus, sig, outs)
        for i, (o, r) in enumerate(zip(outs, refs)):
            assert np.abs(r).max() > 0
            assert_rates_close(o, r, tol, label=f"batched {prec} instance {list(pick)[i]}")
    b.close()
    for c in ctxs:
        c.close()
