"""Pins of the oracle's e-ph matrix elements (Eqs. eph_mat_wann2, eph_mat, g_abs)."""
import numpy as np
import pytest
import scipy.linalg

import synthetic as S
from oracle import eph as O

RNG = np.random.default_rng(11)


def _deg_blocks(vals, tol=1e-8):
    """Groups of consecutive (sorted) indices whose values agree within tol."""
    blocks, start = [], 0
    for i in range(1, len(vals) + 1):
        if i == len(vals) or abs(vals[i] - vals[i - 1]) > tol:
            blocks.append(list(range(start, i)))
            start = i
    return blocks


def test_factorised_matches_brute_double_sum(c1):
    k = RNG.uniform(-1, 1, (3, 3))
    q = RNG.uniform(-1, 1, (4, 3))
    a = O.g_wannier(c1, k, q)
    b = O.g_wannier_brute(c1, k, q)
    assert np.abs(a - b).max() < 1e-13 * np.abs(b).max() * 50


def test_single_r_pair_hand_value(c1):
    # g~ nonzero on one (Re, Rp) pair only: the sum reduces to one phase factor.
    m = S.model_c1()
    g = np.zeros_like(m.g)
    ie, ip = 5, 19
    g[ie, ip] = m.g[ie, ip]
    m.g = g
    k = np.array([[0.13, -0.4, 0.27]])
    q = np.array([[0.31, 0.05, -0.22]])
    out = O.g_wannier(m, k, q)[0, 0]
    ph = np.exp(2j * np.pi * (k[0] @ m.R_ge[ie] + q[0] @ m.R_gp[ip]))
    assert np.allclose(out, ph * m.g[ie, ip], atol=1e-15)


def test_hamiltonian_coupling_rotation_identity(c1):
    """Rotation into the band basis (outer sum of Eq. eph_mat_wann2).

    With g~(Re,Rp) = H(Re) delta_{Rp,Re} the Wannier-gauge sum is H^(W)(k+q), so
    g_mn = eps_m(k+q) [U^dag(k+q) U(k)]_mn; with g~ = H(Re) delta_{Rp,0} it is
    H^(W)(k), so g_mn = [U^dag(k+q) U(k)]_mn eps_n(k).  A swapped or
    un-conjugated rotation breaks one of the two.
    """
    nR = len(c1.R_H)
    r0 = int(np.nonzero((c1.R_H == 0).all(1))[0][0])
    m1 = S.model_c1()
    m2 = S.model_c1()
    g1 = np.zeros((nR, nR, 3, 2, 2), complex)
    g2 = np.zeros_like(g1)
    for r in range(nR):
        g1[r, r, 0] = c1.H[r]
        g2[r, r0, 0] = c1.H[r]
    m1.g, m2.g = g1, g2
    k = RNG.uniform(-1, 1, (4, 3))
    q = RNG.uniform(-1, 1, (4, 3))
    for a in range(4):
        kk, kq = k[a:a + 1], k[a:a + 1] + q[a:a + 1]
        ek, Uk = O.bands(c1, kk)
        ekq, Ukq = O.bands(c1, kq)
        ov = np.conj(Ukq[0]).T @ Uk[0]
        b1 = O.g_bloch(O.g_wannier(m1, kk, q[a:a + 1])[0, 0], Uk[0], Ukq[0])[0]
        b2 = O.g_bloch(O.g_wannier(m2, kk, q[a:a + 1])[0, 0], Uk[0], Ukq[0])[0]
        assert np.allclose(b1, ekq[0][:, None] * ov, atol=1e-12)
        assert np.allclose(b2, ov * ek[0][None, :], atol=1e-12)


def test_holstein_closed_form():
    # 1 band, local constant coupling g0 on every axis, isotropic springs:
    # sum_nu |g_nu|^2 = hbar/(2 M w(q)) * sum_alpha |g0_alpha|^2 with the three
    # degenerate modes of frequency w(q), independent of k.
    g0 = np.array([0.02, 0.03 + 0.01j, -0.015j])
    m = S.model_sc_tight_binding(g0=g0, kspring=1.0, mass=28.0)
    k = RNG.uniform(-1, 1, (3, 3))
    q = RNG.uniform(0.1, 0.9, (5, 3))
    hw, e = O.phonons(m, q)
    for a in range(3):
        ek, Uk = O.bands(m, k[a:a + 1])
        ekq, Ukq = O.bands(m, k[a:a + 1] + q)
        gw = O.g_wannier(m, k[a:a + 1], q)[0]
        gb = O.g_bloch(gw, Uk[0][None], Ukq)
        gm = O.g_modes(gb, hw, e, m.mass)
        tot = (np.abs(gm) ** 2).sum(axis=(1, 2, 3))
        hbar, ev, amu, bohr = 6.582119569e-16, 1.602176634e-19, 1.66053906660e-27, 0.529177210903e-10
        w = hw[:, 0] / hbar                                   # rad/s
        length2 = hbar * ev / (2 * 28.0 * amu * w) / bohr ** 2  # bohr^2
        ref = length2 * np.sum(np.abs(g0) ** 2)
        assert np.allclose(tot, ref, rtol=1e-12)


def test_mode_projection_matrix_function():
    """sum_nu |g_nu|^2 = (C/2) y^T (C D~(q))^{-1/2} conj(y), y_ka = g^{ka}/sqrt(M_k).

    The right side uses only a matrix square root and inverse of the mass-scaled
    dynamical matrix (library routines), not its eigenvectors, so it pins the
    placement and conjugation of e_nu q in Eq. eph_mat and the 1/sqrt(M) factor
    (masses differ between the two atoms).
    """
    m = S.model_c2(g_dtype=np.complex128)
    m.mass = np.array([28.0, 69.7])
    q = np.array([[0.17, 0.31, -0.23], [0.4, -0.1, 0.05]])
    hw, e = O.phonons(m, q)
    Dq = O.dynamical_matrix(m, q)
    x = RNG.normal(size=(2, 6, 3, 3)) + 1j * RNG.normal(size=(2, 6, 3, 3))   # g^{ka}_mn
    gm = O.g_modes(x, hw, e, m.mass)
    lhs = (np.abs(gm) ** 2).sum(axis=1)
    minv = 1 / np.sqrt(np.repeat(m.mass, 3))
    for a in range(2):
        Minv = np.linalg.inv(scipy.linalg.sqrtm(O.C_OMEGA * Dq[a]))
        y = x[a] * minv[:, None, None]
        rhs = 0.5 * O.C_OMEGA * np.einsum("amn,ab,bmn->mn", y, Minv, np.conj(y)).real
        assert np.allclose(lhs[a], rhs, rtol=1e-9)


def test_gauge_invariance_degenerate_sums(c1):
    # Random U(1) phases on band eigenvectors and random U(3) rotations inside the
    # (everywhere threefold degenerate) phonon subspace leave the mode- and
    # degenerate-band-summed |g|^2 unchanged.
    k = RNG.uniform(-1, 1, (2, 3))
    q = RNG.uniform(0.1, 0.9, (3, 3))
    hw, e = O.phonons(c1, q)
    for a in range(2):
        ek, Uk = O.bands(c1, k[a:a + 1])
        ekq, Ukq = O.bands(c1, k[a:a + 1] + q)
        gw = O.g_wannier(c1, k[a:a + 1], q)[0]
        base = np.abs(O.g_modes(O.g_bloch(gw, Uk[0][None], Ukq), hw, e, c1.mass)) ** 2
        Uk2 = Uk * np.exp(1j * RNG.uniform(0, 2 * np.pi, (1, 1, 2)))
        Ukq2 = Ukq * np.exp(1j * RNG.uniform(0, 2 * np.pi, (3, 1, 2)))
        V = np.linalg.qr(RNG.normal(size=(3, 3, 3)) + 1j * RNG.normal(size=(3, 3, 3)))[0]
        e2 = e @ V
        rot = np.abs(O.g_modes(O.g_bloch(gw, Uk2[0][None], Ukq2), hw, e2, c1.mass)) ** 2
        assert np.allclose(base.sum(axis=1), rot.sum(axis=1), rtol=1e-12, atol=1e-20)
        # without the mode sum the two generally differ (the modes are degenerate)
        assert not np.allclose(base, rot, rtol=1e-6)


def test_time_reversal_partner(c1):
    # g~_ij(Re,Rp) = conj(g~_ji(-Re, Rp-Re)) implies
    # sum_nu |g_mn nu(k,q)|^2 = sum_nu |g_nm nu(k+q,-q)|^2.
    k = RNG.uniform(-1, 1, (3, 3))
    q = RNG.uniform(0.1, 0.9, (3, 3))
    for a in range(3):
        kk, kq, qq = k[a:a + 1], k[a:a + 1] + q[a:a + 1], q[a:a + 1]
        ek, Uk = O.bands(c1, kk)
        ekq, Ukq = O.bands(c1, kq)
        hw, e = O.phonons(c1, qq)
        hwm, em = O.phonons(c1, -qq)
        f = O.g_modes(O.g_bloch(O.g_wannier(c1, kk, qq)[0, 0], Uk[0], Ukq[0]), hw[0], e[0], c1.mass)
        b = O.g_modes(O.g_bloch(O.g_wannier(c1, kq, -qq)[0, 0], Ukq[0], Uk[0]), hwm[0], em[0], c1.mass)
        fs = (np.abs(f) ** 2).sum(0)
        bs = (np.abs(b) ** 2).sum(0)
        assert np.allclose(fs, bs.T, rtol=1e-11)


def test_time_reversal_partner_nondegenerate_modes():
    # Same identity per mode on the fcc model, whose modes are non-degenerate at
    # generic q.
    m = S.model_c2(g_dtype=np.complex128)
    k = np.array([[0.11, -0.23, 0.37]])
    q = np.array([[0.29, 0.13, -0.41]])
    ek, Uk = O.bands(m, k)
    ekq, Ukq = O.bands(m, k + q)
    hw, e = O.phonons(m, q)
    hwm, em = O.phonons(m, -q)
    assert np.min(np.diff(hw[0])) > 1e-4
    f = O.g_modes(O.g_bloch(O.g_wannier(m, k, q)[0, 0], Uk[0], Ukq[0]), hw[0], e[0], m.mass)
    b = O.g_modes(O.g_bloch(O.g_wannier(m, k + q, -q)[0, 0], Ukq[0], Uk[0]), hwm[0], em[0], m.mass)
    assert np.allclose(np.abs(f) ** 2, np.swapaxes(np.abs(b) ** 2, -1, -2), rtol=1e-9, atol=1e-16)


def test_g_abs_definition():
    gm = RNG.normal(size=(4, 6, 3, 3)) + 1j * RNG.normal(size=(4, 6, 3, 3))
    ga = O.g_abs(gm)
    for a in range(4):
        for nu in range(6):
            assert np.isclose(ga[a, nu] ** 2 * 3, sum(abs(gm[a, nu, i, j]) ** 2 for i in range(3) for j in range(3)))


@pytest.mark.parametrize("nb", [2])
def test_symmetry_equivalent_pairs_equal_abs_g(nb):
    # The paper's own check (Sec. 4.1): symmetry-equivalent (k, q) pairs give equal
    # gauge-invariant |g|.  On a noise-free cubic model (isotropic springs,
    # a coupling that is a function of |Re|, |Rp| only), cubic rotations of
    # (k, q) leave sum_nu |g_nu|^2 unchanged.
    m = S.model_sc_tight_binding(t=-0.2)
    R = m.R_ge.astype(float)
    n = np.linalg.norm(R, axis=1)
    g = np.zeros_like(m.g)
    for a in range(len(R)):
        for b in range(len(R)):
            for al in range(3):
                # a scalar coupling that depends on the alpha-component of Rp only
                g[a, b, al, 0, 0] = 0.05 * np.exp(-(n[a] + n[b])) * (1.0 + R[b, al])
    m.g = g
    k = np.array([[0.1, 0.2, 0.3]])
    q = np.array([[0.05, -0.15, 0.25]])
    vals = []
    for P in ([0, 1, 2], [1, 2, 0], [2, 0, 1], [1, 0, 2]):
        kk, qq = k[:, P], q[:, P]
        ek, Uk = O.bands(m, kk)
        ekq, Ukq = O.bands(m, kk + qq)
        hw, e = O.phonons(m, qq)
        gm = O.g_modes(O.g_bloch(O.g_wannier(m, kk, qq)[0, 0], Uk[0], Ukq[0]), hw[0], e[0], m.mass)
        vals.append(np.sum(np.abs(gm) ** 2))
    assert np.allclose(vals, vals[0], rtol=1e-12)
