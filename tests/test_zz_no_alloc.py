"""The allocation-free scattering-rate entry point against the regular one.

pgb_scattering_rates_noalloc serves callers that cannot allocate device memory
during a call (a host whose GPU memory already belongs to its own pool, or a
request path that forbids cudaMalloc because it can synchronise the device).
It keeps all temporaries in one fixed device array; this file checks, through
the C ABI, that two calls in a row give the same rates as
pgb_scattering_rates (FP32) within the FP32 tolerance of the other tests, and
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
