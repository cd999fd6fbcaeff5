"""Pins of the oracle's electron and phonon interpolation (Eqs. wannier_3, IFC2).

Each pin is fixed by something other than the oracle's own code: a textbook
closed form, an invariant of the construction, or an identity of the
eigen-decomposition.
"""
import numpy as np

import synthetic as S
from oracle import eph as O

RNG = np.random.default_rng(7)


def test_sc_tight_binding_closed_form():
    # One s band, nearest-neighbour hopping t on a simple-cubic lattice:
    # eps(k) = eps0 + 2 t sum_i cos(2 pi k_i)  (textbook tight binding).
    m = S.model_sc_tight_binding(eps0=0.3, t=-0.25)
    k = RNG.uniform(-1, 1, (50, 3))
    eps, U = O.bands(m, k)
    ref = 0.3 + 2 * (-0.25) * np.cos(2 * np.pi * k).sum(axis=1)
    assert np.allclose(eps[:, 0], ref, atol=1e-13)


def test_hamiltonian_hermitian_and_decomposition(c1):
    k = RNG.uniform(-1, 1, (20, 3))
    Hk = O.hamiltonian_k(c1, k)
    assert np.abs(Hk - np.conj(np.swapaxes(Hk, -1, -2))).max() < 1e-14
    eps, U = O.bands(c1, k)
    assert np.all(np.diff(eps, axis=1) >= 0)
    rec = np.einsum("kin,kn,kjn->kij", U, eps, np.conj(U))
    assert np.abs(rec - Hk).max() < 1e-12


def test_isotropic_springs_closed_form():
    # Nearest-neighbour isotropic springs on a simple-cubic lattice:
    # M w^2(q) = 2 k sum_i (1 - cos 2 pi q_i) for all three modes.
    m = S.model_sc_tight_binding(kspring=1.3, mass=17.0)
    q = RNG.uniform(-1, 1, (40, 3))
    hw, e = O.phonons(m, q)
    lam = 2 * 1.3 / 17.0 * (1 - np.cos(2 * np.pi * q)).sum(axis=1)
    # hbar w in eV from lambda in eV/(bohr^2 amu): CODATA constants
    hbar, ev, amu, bohr = 6.582119569e-16, 1.602176634e-19, 1.66053906660e-27, 0.529177210903e-10
    ref = hbar * np.sqrt(lam * ev / (amu * bohr ** 2))
    assert np.allclose(hw, ref[:, None], rtol=1e-12, atol=1e-15)


def test_acoustic_sum_rule_and_inversion(c1):
    q0 = np.zeros((1, 3))
    for m in (c1, S.model_sc_tight_binding()):
        hw, _ = O.phonons(m, q0)
        assert np.abs(hw[0, :3]).max() < 1e-10
    q = RNG.uniform(-1, 1, (30, 3))
    hw_p, e_p = O.phonons(c1, q)
    hw_m, _ = O.phonons(c1, -q)
    assert np.allclose(hw_p, hw_m, atol=1e-14)
    assert np.all(hw_p[np.linalg.norm(q, axis=1) > 1e-3] > 0)


def test_mass_scaling_two_atoms():
    # For a 2-atom cell the mass-scaled matrix must be D/sqrt(M_k M_k'); check
    # the identity sum_nu (hbar w)^2 = C * trace(D(q) M^-1) for unequal masses.
    m = S.model_ladder(nw=1)
    m.mass = np.array([10.0, 40.0])
    m.tau = np.zeros((2, 3))
    m.D = np.array([[[2.0, 0.1, 0, -1.0, 0, 0],
                     [0.1, 2.0, 0, 0, -1.0, 0],
                     [0, 0, 2.0, 0, 0, -1.0],
                     [-1.0, 0, 0, 2.0, 0, 0],
                     [0, -1.0, 0, 0, 2.0, 0],
                     [0, 0, -1.0, 0, 0, 2.0]]])
    hw, _ = O.phonons(m, np.zeros((1, 3)))
    minv = np.repeat(1 / m.mass, 3)
    hbar, ev, amu, bohr = 6.582119569e-16, 1.602176634e-19, 1.66053906660e-27, 0.529177210903e-10
    C = hbar ** 2 * ev / (amu * bohr ** 2)
    assert np.isclose((hw[0] ** 2).sum(), C * np.sum(np.diag(m.D[0]) * minv), rtol=1e-12)


def test_c2_model_shapes_and_asr():
    m = S.model_c2(g_dtype=np.complex64)
    assert m.H.shape == (381, 8, 8) and m.D.shape == (381, 6, 6)
    assert m.g.shape == (381, 381, 6, 8, 8) and m.g.dtype == np.complex64
    hw, _ = O.phonons(m, np.zeros((1, 3)))
    assert np.abs(hw[0, :3]).max() < 1e-7 and hw[0, 3:].min() > 0.02
    q = RNG.uniform(-1, 1, (10, 3))
    hw, _ = O.phonons(m, q)
    assert hw.min() > 0 and hw.max() < 0.12
    Hk = O.hamiltonian_k(m, q)
    assert np.abs(Hk - np.conj(np.swapaxes(Hk, -1, -2))).max() < 1e-13
