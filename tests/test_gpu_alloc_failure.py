"""Device-allocation failures, injected on the host.

Every device allocation of libpertgb goes through one counted call, and
pgb_diag_fail_alloc(n) makes the n-th next one return cudaErrorMemoryAllocation
without touching the GPU (an out-of-memory device, simulated on the host: no
kernel faults and nothing is left running).  For each call sequence below, a
clean run counts its allocations; then each allocation in turn (or a spread of
them) is made to fail: the sequence must stop with PGB_ENOMEM, and the same
context must then run it again cleanly with the clean run's results.
"""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MAX_CASES = 28


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_02045_gb300 import build, load
    build.build()
    lb = load()
    yield lb
    lb.pgb_diag_fail_alloc(-1)


def _sweep(lib, fn, label):
    from paper_2002_02045_gb300 import PGB_ENOMEM, PgbError
    fn()                                   # warm-up: grow-only scratch reaches its size
    n0 = lib.pgb_diag_alloc_count()
    ref = fn()
    n = lib.pgb_diag_alloc_count() - n0
    assert n > 0, f"{label}: no device allocation counted"
    cases = range(n) if n <= MAX_CASES else sorted(set(np.linspace(0, n - 1, MAX_CASES).astype(int).tolist()))
    for i in cases:
        lib.pgb_diag_fail_alloc(i)
        try:
            with pytest.raises(PgbError) as e:
                fn()
            assert e.value.status == PGB_ENOMEM, f"{label}: allocation {i} of {n}: status {e.value.status}"
        finally:
            lib.pgb_diag_fail_alloc(-1)
        got = fn()
        for a, b in zip(got, ref):
            np.testing.assert_allclose(a, b, rtol=1e-12, atol=0, err_msg=f"{label}: rerun after failure {i}")
    return n


def test_enomem_model_grids_rates(lib):
    from paper_2002_02045_gb300 import PGB_FP32, PGB_TC_BF16X3, Context
    m = S.model_c2(rcut=12.0)
    ctx = Context(0)
    kidx = np.array([0, 33, 400], np.int32)

    def run():
        ctx.pgb_set_model(m)
        ctx.pgb_set_grids((8, 8, 8), (8, 8, 8))
        out = []
        for prec in (PGB_FP32, PGB_TC_BF16X3):
            g = np.zeros((3, 8))
            ctx.pgb_scattering_rates(kidx, 300.0, 0.0, 0.02, prec, g)
            out.append(g)
        return out

    assert _sweep(lib, run, "set_model/set_grids/rates") > 10
    ctx.close()


def test_enomem_interpolate_g_split(lib):
    from paper_2002_02045_gb300 import PGB_G2_FULL, PGB_TC_BF16X3, Context
    m = S.model_c2(rcut=12.0)
    ctx = Context(0)
    ctx.pgb_set_model(m)
    rng = np.random.default_rng(5)
    k, q = rng.uniform(-0.5, 0.5, (2, 3)), rng.uniform(-0.5, 0.5, (20, 3))

    def run():
        out = np.zeros((2, 20, 6, 8, 8))
        ctx.pgb_interpolate_g(k, q, PGB_TC_BF16X3, PGB_G2_FULL, out)
        return [out]

    _sweep(lib, run, "interpolate_g bf16x3")
    ctx.close()


def test_enomem_collision_list_rk4_adjoint(lib):
    from paper_2002_02045_gb300 import Context
    m = S.model_c1()
    ctx = Context(0)

    def run():
        ctx.pgb_set_model(m)
        ctx.pgb_set_grids((4, 4, 4), (4, 4, 4))
        nnz = ctx.pgb_build_collision_grid(0, 2, -10.0, 10.0, 300.0, 0.02)
        ns = 128
        eps = np.zeros(ns)
        ctx.pgb_collision_energies(eps)
        f0 = 0.1 * np.exp(-((eps - eps.min() - 0.5) / 0.3) ** 2)
        lam_end = eps / ns
        lam0, dg2, fe = np.zeros(ns), np.zeros(nnz), np.zeros(ns)
        ctx.pgb_rk4_adjoint(f0, 1.0, 12, 5, lam_end, lam0, dg2, fe)
        return [np.array([nnz], float), fe, lam0, dg2]

    _sweep(lib, run, "build_collision_grid/rk4_adjoint")
    ctx.close()


def test_enomem_batch(lib):
    from paper_2002_02045_gb300 import Batch, Context
    models = [S.model_batch_instance(i) for i in (1, 2)]
    ctxs = []
    for m in models:
        c = Context(0)
        c.pgb_set_model(m)
        c.pgb_set_grids((8, 8, 8), (8, 8, 8))
        ctxs.append(c)
    ks = [np.array([0, 5], np.int32), np.array([7, 100, 511], np.int32)]

    def run():
        b = Batch(ctxs)
        try:
            outs = [np.zeros((len(k), m.nw)) for k, m in zip(ks, models)]
            b.pgb_batch_rates(ks, 300.0, [0.0, 0.0], 0.05, outs)
        finally:
            b.close()
        return outs

    # batch creation and planning allocate; a failed pgb_batch_create raises too
    from paper_2002_02045_gb300 import PGB_ENOMEM, PgbError
    run()
    n0 = lib.pgb_diag_alloc_count()
    ref = run()
    n = lib.pgb_diag_alloc_count() - n0
    assert n > 0
    for i in sorted(set(np.linspace(0, n - 1, min(n, MAX_CASES)).astype(int).tolist())):
        lib.pgb_diag_fail_alloc(i)
        try:
            with pytest.raises(PgbError) as e:
                run()
            assert e.value.status == PGB_ENOMEM, (i, n, e.value.status)
        finally:
            lib.pgb_diag_fail_alloc(-1)
        got = run()
        for a, b in zip(got, ref):
            np.testing.assert_allclose(a, b, rtol=1e-12, atol=0)
    for c in ctxs:
        c.close()
