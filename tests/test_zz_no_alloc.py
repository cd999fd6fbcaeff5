"""The allocation-free scattering-rate entry point against the regular one.

pgb_scattering_rates_noalloc serves callers that cannot allocate device memory
during a call (a host whose GPU memory already belongs to its own pool, or a
request path that forbids cudaMalloc because it can synchronise the device).
It keeps all temporaries in one fixed device array; this file checks, through
the C ABI, that two calls in a row give the same rates as
pgb_scattering_rates (FP32) within the FP32 tolerance of the other tests (also
when the k list needs several passes through the array, and with a polar
long-range term), that the call asks for no device allocation at all, and
that a grid too large for the array is refused.  It is collected last so that
a failure here comes after every other test has run.
"""
import numpy as np
import pytest

import synthetic as S

from helpers import assert_rates_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_02045_gb300 import Context, build
    build.build()
    c = Context(0)
    yield c
    c.close()


def test_noalloc_matches_regular_rates_twice(ctx):
    from paper_2002_02045_gb300 import PGB_FP32
    m = S.model_c2()
    ctx.pgb_set_model(m)
    ctx.pgb_set_grids((12, 12, 12), (6, 6, 6))
    eps = torch.empty((1728, 8), dtype=torch.float64, device="cuda")
    ctx.pgb_get_grid_energies(eps, None)
    emin = float(eps.min())
    T, mu, sig = 300.0, emin - 0.3, 0.010
    kidx = torch.tensor([0, 5, 77, 600, 1727, 1200, 333], dtype=torch.int32, device="cuda")
    ref = torch.empty((7, 8), dtype=torch.float64, device="cuda")
    ctx.pgb_scattering_rates(kidx, T, mu, sig, PGB_FP32, ref)
    r = ref.cpu().numpy()
    for _ in range(2):
        got = torch.full((7, 8), float("nan"), dtype=torch.float64, device="cuda")
        ctx.pgb_scattering_rates_noalloc(kidx, T, mu, sig, got)
        torch.cuda.synchronize()
        assert_rates_close(got.cpu().numpy(), r, 1e-5, label="noalloc vs regular")


def test_noalloc_refuses_oversized_grid_and_host_pointers(ctx):
    from paper_2002_02045_gb300 import PgbError
    m = S.model_c2()
    ctx.pgb_set_model(m)
    ctx.pgb_set_grids((40, 40, 40), (40, 40, 40))   # 64000 q x 384 columns: ~197 MB per k-point
    kidx = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty((1, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(PgbError):
        ctx.pgb_scattering_rates_noalloc(kidx, 300.0, 0.0, 0.01, out)
    ctx.pgb_set_grids((6, 6, 6), (6, 6, 6))
    with pytest.raises(PgbError):
        ctx.pgb_scattering_rates_noalloc(np.zeros(1, np.int32), 300.0, 0.0, 0.01, out)


def _regular_and_noalloc(ctx, kidx, T, mu, sig, nw):
    from paper_2002_02045_gb300 import PGB_FP32
    ref = torch.empty((len(kidx), nw), dtype=torch.float64, device="cuda")
    ctx.pgb_scattering_rates(kidx, T, mu, sig, PGB_FP32, ref)
    outs = []
    for _ in range(2):
        got = torch.full((len(kidx), nw), float("nan"), dtype=torch.float64, device="cuda")
        ctx.pgb_scattering_rates_noalloc(kidx, T, mu, sig, got)
        torch.cuda.synchronize()
        outs.append(got.cpu().numpy())
    return ref.cpu().numpy(), outs


def test_noalloc_several_batches(ctx):
    """16^3 grids of the fcc model need ~15 MB of array per k-point next to ~13 MB
    of q tables, so 10 k-points run as passes of 3, 3, 3 and 1 through the array."""
    m = S.model_c2()
    ctx.pgb_set_model(m)
    ctx.pgb_set_grids((16, 16, 16), (16, 16, 16))
    eps = torch.empty((4096, 8), dtype=torch.float64, device="cuda")
    ctx.pgb_get_grid_energies(eps, None)
    emin = float(eps.min())
    kidx = torch.tensor([0, 1, 17, 300, 1111, 2048, 2049, 3000, 4000, 4095], dtype=torch.int32, device="cuda")
    ref, outs = _regular_and_noalloc(ctx, kidx, 300.0, emin - 0.3, 0.010, 8)
    for got in outs:
        assert_rates_close(got, ref, 1e-5, label="noalloc in batches vs regular")


def test_noalloc_polar(ctx):
    """The long-range term enters through the q table the call builds in the array."""
    m = S.model_c3(rcut=13.0)
    ctx.pgb_set_model(m)
    ctx.pgb_set_lattice(m.A, m.tau)
    ctx.pgb_set_polar(m.zstar, m.eps_inf, m.ewald_lambda)
    ctx.pgb_set_grids((12, 12, 12), (6, 6, 6))
    eps = torch.empty((1728, 8), dtype=torch.float64, device="cuda")
    ctx.pgb_get_grid_energies(eps, None)
    emin = float(eps.min())
    kidx = torch.tensor([0, 3, 99, 1000, 1727], dtype=torch.int32, device="cuda")
    ref, outs = _regular_and_noalloc(ctx, kidx, 300.0, emin - 0.3, 0.010, 8)
    for got in outs:
        assert_rates_close(got, ref, 1e-5, label="noalloc polar vs regular")
    assert ref.max() > 0


def test_noalloc_asks_for_no_device_allocation(ctx):
    """Every device allocation of the library goes through one counted call; the
    allocation-free entry point must not move the count, where the regular one does."""
    from paper_2002_02045_gb300 import PGB_FP32, load
    lib = load()
    m = S.model_c2()
    ctx.pgb_set_model(m)
    ctx.pgb_set_grids((12, 12, 12), (6, 6, 6))
    kidx = torch.tensor([0, 5, 77], dtype=torch.int32, device="cuda")
    out = torch.empty((3, 8), dtype=torch.float64, device="cuda")
    ctx.pgb_scattering_rates_noalloc(kidx, 300.0, 0.0, 0.01, out)   # first call: address look-up
    torch.cuda.synchronize()
    n0 = lib.pgb_diag_alloc_count()
    for _ in range(3):
        ctx.pgb_scattering_rates_noalloc(kidx, 300.0, 0.0, 0.01, out)
    torch.cuda.synchronize()
    assert lib.pgb_diag_alloc_count() == n0
    ctx.pgb_scattering_rates(kidx, 300.0, 0.0, 0.01, PGB_FP32, out)
    assert lib.pgb_diag_alloc_count() > n0
