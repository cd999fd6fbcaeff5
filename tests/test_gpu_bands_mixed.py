"""Bands at arbitrary points by the FP32 paths' route (Sec. 2.2.1, Eq. wannier_3),
through the C ABI: the real cos/sin Fourier sum of the packed Hermitian H(k)
against the oracle's H(k), the FP64-refined eigenvalues against LAPACK on the
oracle's H(k), and the FP32 eigenvectors by residual and orthonormality,
including exactly degenerate bands."""
import dataclasses

import numpy as np
import pytest

import synthetic as S
from oracle import eph as O

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


def packed(Hk):
    """[n][nw][nw] Hermitian -> [n][nw^2]: diagonal reals, then (re, im) of (i, j), i < j, row by row."""
    n, nw, _ = Hk.shape
    cols = [Hk[:, i, i].real for i in range(nw)]
    for i in range(nw):
        for j in range(i + 1, nw):
            cols += [Hk[:, i, j].real, Hk[:, i, j].imag]
    return np.stack(cols, axis=1)


def repeated_bands(m, copies):
    """The model with H(R) -> I_copies (x) H(R): every band `copies`-fold degenerate."""
    H = np.stack([np.kron(np.eye(copies), h) for h in m.H])
    nw = H.shape[1]
    g = np.zeros(m.g.shape[:3] + (nw, nw), m.g.dtype)
    return dataclasses.replace(m, H=H, g=g, name=m.name + f"_x{copies}")


MODELS = {
    "c1": lambda: S.model_c1(),
    "c2": lambda: S.model_c2(),
    "c3_small": lambda: S.model_c3(rcut=13.0),
    "batch44_nw16": lambda: S.model_batch_instance(44),
    "c1_x3_degenerate": lambda: repeated_bands(S.model_c1(), 3),
    "c2_x2_degenerate": lambda: repeated_bands(S.model_c2(rcut=11.0), 2),
}


@pytest.mark.parametrize("name", list(MODELS))
def test_bands_mixed_against_oracle(ctx, name):
    m = MODELS[name]()
    ctx.pgb_set_model(m)
    nw = m.H.shape[1]
    rng = np.random.default_rng(60 + len(name))
    # several 64-point blocks and a ragged tail; coordinates beyond the first zone
    pts = rng.uniform(-1.5, 1.5, (64 * 5 + 37, 3))
    pts[:4] = [[0, 0, 0], [0.5, 0, 0], [0.5, 0.5, 0.5], [0.25, -0.25, 0.5]]
    Hp = np.zeros((len(pts), nw * nw))
    eps = np.zeros((len(pts), nw))
    U = np.zeros((len(pts), nw, nw), np.complex64)
    ctx.pgb_diag_bands_mixed(pts, Hp, eps, U)

    Hk = O.hamiltonian_k(m, pts)
    Hk = 0.5 * (Hk + np.conj(np.swapaxes(Hk, 1, 2)))
    scale = np.abs(Hk).max()
    ref_p = packed(Hk)
    # double-float sum: ~2^-44 of the partial sums, which can exceed |H(k)| several-fold
    assert np.abs(Hp - ref_p).max() <= 5e-12 * scale, "packed H(k)"

    ref_e = np.linalg.eigvalsh(Hk)
    assert np.abs(eps - ref_e).max() <= 1e-10 * scale, "eigenvalues"
    assert np.all(np.diff(eps, axis=1) >= 0), "ascending"

    Ud = U.astype(np.complex128)
    res = np.einsum("kij,kjn->kin", Hk, Ud) - Ud * eps[:, None, :]
    assert np.abs(res).max() <= 2e-5 * scale, "eigenvector residual"
    ortho = np.einsum("kin,kim->knm", Ud.conj(), Ud) - np.eye(nw)
    assert np.abs(ortho).max() <= 1e-5, "orthonormal columns"
    if "degenerate" in name:
        # the projector on each degenerate cluster is gauge-free: compare it
        copies = 3 if "x3" in name else 2
        _, Uref = np.linalg.eigh(Hk)
        for c0 in range(0, nw, copies):
            P = np.einsum("kin,kjn->kij", Ud[:, :, c0:c0 + copies], Ud[:, :, c0:c0 + copies].conj())
            Pr = np.einsum("kin,kjn->kij", Uref[:, :, c0:c0 + copies], Uref[:, :, c0:c0 + copies].conj())
            gap = np.min(np.abs(ref_e[:, c0][:, None] - np.delete(ref_e, range(c0, c0 + copies), axis=1)), axis=1)
            ok = gap > 1e-3 * scale       # clusters well separated from the other bands
            assert np.abs(P - Pr)[ok].max() <= 1e-4, "cluster projector"


def test_bands_mixed_argument_errors(ctx):
    from paper_2002_02045_gb300 import PgbError
    m = S.model_sc_tight_binding()
    ctx.pgb_set_model(m)
    with pytest.raises(PgbError):
        ctx.pgb_diag_bands_mixed(np.zeros((3, 3)), None, np.zeros((3, 1)), None)


@pytest.mark.parametrize("name", ["c1", "c2", "c3_small", "batch44_nw16"])
def test_phonons_mixed_against_oracle(ctx, name):
    m = MODELS[name]()
    ctx.pgb_set_model(m)
    nm = m.D.shape[1]
    rng = np.random.default_rng(80 + len(name))
    q = rng.uniform(-1.5, 1.5, (64 * 3 + 11, 3))
    q[:3] = [[0, 0, 0], [1e-3, 0, 0], [0.5, 0.5, 0.5]]
    q[3:40] *= 1e-2                       # near the zone centre, where the acoustic branches are soft
    Dp = np.zeros((len(q), nm * nm))
    w2 = np.zeros((len(q), nm))
    e = np.zeros((len(q), nm, nm), np.complex64)
    ctx.pgb_diag_phonons_mixed(q, Dp, w2, e)
    Dq = O.dynamical_matrix(m, q)
    Dq = 0.5 * (Dq + np.conj(np.swapaxes(Dq, 1, 2)))
    scale = np.abs(Dq).max()
    assert np.abs(Dp - packed(Dq)).max() <= 5e-12 * scale, "packed D(q)"
    assert np.abs(w2 - np.linalg.eigvalsh(Dq)).max() <= 1e-10 * scale, "omega^2"
    ed = e.astype(np.complex128)
    res = np.einsum("kij,kjn->kin", Dq, ed) - ed * w2[:, None, :]
    assert np.abs(res).max() <= 2e-5 * scale, "mode residual"
