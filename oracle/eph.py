"""FP64 oracle: Wannier interpolation, e-ph matrix elements, RTA rates, collision integral, RK4.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every function is the
plain definition from the paper, in FP64, using NumPy's matmul/einsum and
LAPACK's Hermitian eigensolver (``numpy.linalg.eigh``) as library steps.

Notation (paper Sec. 2): k, q crystal coordinates; R integer lattice vectors
in crystal coordinates, so k.R = 2 pi k.n; bands n (initial, at k) and m
(final, at k+q); phonon modes nu; atom kappa with Cartesian direction alpha
(index ka = 3 kappa + alpha).

Units and readings (the paper does not fix them):
  * energies, |g| and hbar*omega in eV; D(R) in eV/bohr^2; masses in amu;
    g~(Re,Rp) numerically in eV/bohr, so that the zero-point length
    sqrt(hbar / (2 M omega)) in bohr times g~ is in eV;
  * Gamma and I[f] in 1/s, time step in fs;
  * Gaussian delta: delta_s(x) = exp(-x^2/s^2) / (s sqrt(pi));
  * modes with hbar*omega < OMEGA_MIN_EV contribute nothing (the acoustic modes at
    q = Gamma), and negative eigenvalues of D(q) are clamped to 0;
  * 1/N_q is the full q-grid count.

Pins (tests/test_oracle_*.py):
  * ``hamiltonian_k``/``bands``: closed form of the 1-band simple-cubic tight
    binding; Hermiticity; H = U diag(eps) U^dagger.
  * ``dynamical_matrix``/``phonons``: closed form of isotropic nearest-neighbour
    springs; three zero modes at Gamma (acoustic sum rule); omega(-q) = omega(q).
  * ``g_wannier``: the brute-force double sum ``g_wannier_brute`` on tiny
    inputs (a different summation structure), and a hand-evaluated single
    R-pair case.
  * ``g_bloch``/``g_modes``: the Holstein-like closed form; gauge invariance of
    degenerate-summed |g|^2 under random U(1)/U(d) eigenvector rotations; the
    time-reversal partner identity |g_mn nu(k,q)|^2 = |g_nm nu(k+q,-q)|^2.
  * ``scattering_rates``: brute-force pure-Python loops on a tiny grid; the
    1-band Einstein closed form; Gamma >= 0; mode-resolved rates sum to total.
  * ``collision``: sum over states vanishes for a symmetric list; it equals
    -Gamma * delta f to first order around equilibrium (the RTA link of
    Eq. scatter_rate); detailed balance on the ladder model.
  * ``rk4_step``/``euler_step``: fourth / first order convergence on the
    two-state closed form; carrier number conserved.
  * ``collision_vjp``: central finite differences on an unsymmetric random
    list with self-terms (I is quadratic in f and linear in |g|^2, so the
    differences are exact up to rounding); J^T 1 = 0 and opposite |g|^2
    derivatives of partner entries on a symmetric list.
  * ``rk4_adjoint``: (P(dt A)^T)^n lam on linear systems, P the degree-4
    Taylor polynomial; finite differences of ``evolve`` on a grid list; the
    carrier-number covector 1 is carried back unchanged.
  * ``frohlich_wannier``: invariance under reciprocal-lattice shifts of q;
    L(-q) = conj L(q); the q -> 0 closed form of the G = 0 term; a plain
    one-G-at-a-time loop over a larger box; ``g_wannier_full`` rotated equals
    the short-range part plus L [U^dagger(k+q) U(k)] (Eq. smooth_phase).
  * ``velocities``: central differences of ``bands``; at a degeneracy, the
    one-sided slopes of the split bands.
  * ``bte_weights``: its row sums on a full list equal ``scattering_rates``;
    ``bte_iterate``: the dense solution of (1 - tau W) F = tau v; RTA when W = 0.
  * ``mobility``: constant-tau cosine band under Boltzmann statistics against
    the exact aliased Bessel-function average.
  * ``mc_qpoints``: the Cauchy density integrates to one and its CDF inverts
    the map; width 1 is the uniform map; the weighted estimator integrates a
    known function without bias.  ``scattering_rates_mc`` with the grid points
    as samples equals ``scattering_rates_grid``.
  * ``tetra_theta_weights``: against an independent geometric integral (iso-
    energy slices of the tetrahedron integrated by Gauss-Legendre), continuity
    at the corner energies; ``population_cumulative``: carrier counts.
Parity unpinned: absolute Gamma of real materials (no DFT data here).
"""
from __future__ import annotations

import numpy as np

# CODATA 2018
HBAR_EVS = 6.582119569e-16        # eV s
KB_EVK = 8.617333262e-5           # eV / K
AMU_KG = 1.66053906660e-27        # kg
BOHR_M = 0.529177210903e-10       # m
EV_J = 1.602176634e-19            # J

# (hbar omega)^2 [eV^2] = C_OMEGA * lambda, lambda an eigenvalue of the mass-scaled
# dynamical matrix in eV/(bohr^2 amu).  The same number gives the squared
# zero-point length: hbar/(2 M omega) [bohr^2] = C_OMEGA / (2 M[amu] hbar*omega[eV]).
C_OMEGA = HBAR_EVS ** 2 * EV_J / (AMU_KG * BOHR_M ** 2)
OMEGA_MIN_EV = 1e-4
TWO_PI_OVER_HBAR = 2.0 * np.pi / HBAR_EVS   # 1/(eV s)
HARTREE_EV = 27.211386245988      # eV; e^2/(4 pi eps_0) = 1 hartree * bohr
EWALD_CUT = 40.0                  # G terms with (q+G).eps.(q+G)/(4 Lambda) above this are dropped


# ----------------------------------------------------------------------------
# Fourier phases
# ----------------------------------------------------------------------------

def phases(pts: np.ndarray, R: np.ndarray) -> np.ndarray:
    """e^{i k.R} for every point and lattice vector: shape (npts, nR)."""
    return np.exp(2j * np.pi * (np.asarray(pts, np.float64) @ np.asarray(R, np.float64).T))


# ----------------------------------------------------------------------------
# electrons: Sec. 2.2.1, Eq. wannier_3
# ----------------------------------------------------------------------------

def hamiltonian_k(model, kpts: np.ndarray) -> np.ndarray:
    """H^(W)(k) = sum_R e^{ik.R} H(R)  (Eq. wannier_3, first equality)."""
    return np.einsum("kr,rij->kij", phases(kpts, model.R_H), model.H.astype(np.complex128))


def bands(model, kpts: np.ndarray):
    """eps_nk ascending and U(k) with H^(W)(k) = U diag(eps) U^dagger (Eq. wannier_3).

    ``U[k, :, n]`` is the eigenvector of band n.
    """
    eps, U = np.linalg.eigh(hamiltonian_k(model, kpts))
    return eps, U


# ----------------------------------------------------------------------------
# phonons: Sec. 2.2.2, Eq. IFC2
# ----------------------------------------------------------------------------

def dynamical_matrix(model, qpts: np.ndarray) -> np.ndarray:
    """Mass-scaled D(q)_{ka,k'b} = sum_R e^{iq.R} D_{ka,k'b}(R) / sqrt(M_k M_k')  (Eq. IFC2).

    D(R) is stored without the mass factor, as the paper states for Eq. IFC1.
    """
    Dq = np.einsum("qr,rab->qab", phases(qpts, model.R_D), model.D.astype(np.complex128))
    m = np.repeat(np.asarray(model.mass, np.float64), 3)
    return Dq / np.sqrt(m[:, None] * m[None, :])


def phonons(model, qpts: np.ndarray):
    """hbar*omega_nu q (eV, ascending) and eigenvectors e_nu q (columns) of D(q)."""
    lam, e = np.linalg.eigh(dynamical_matrix(model, qpts))
    hw = np.sqrt(C_OMEGA * np.clip(lam, 0.0, None))
    return hw, e


# ----------------------------------------------------------------------------
# e-ph matrix elements: Sec. 2.2.3, Eqs. eph_mat_wann2, eph_mat, g_abs
# ----------------------------------------------------------------------------

def g_wannier_brute(model, kpts: np.ndarray, qpts: np.ndarray) -> np.ndarray:
    """sum_{Re,Rp} e^{i(k.Re + q.Rp)} g~(Re,Rp) as a direct double sum (Eq. eph_mat_wann2).

    One combined phase per (k, q, Re, Rp); pure loops over the point pairs.
    Output [nk, nq, nmode, nw, nw].  Tiny inputs only.
    """
    g = model.g.astype(np.complex128)
    Re = model.R_ge.astype(np.float64)
    Rp = model.R_gp.astype(np.float64)
    nk, nq = len(kpts), len(qpts)
    out = np.zeros((nk, nq) + g.shape[2:], dtype=np.complex128)
    for a in range(nk):
        for b in range(nq):
            arg = (Re @ kpts[a])[:, None] + (Rp @ qpts[b])[None, :]
            ph = np.exp(2j * np.pi * arg)
            out[a, b] = np.einsum("ep,epxij->xij", ph, g)
    return out


def g_wannier(model, kpts: np.ndarray, qpts: np.ndarray) -> np.ndarray:
    """Same sum as ``g_wannier_brute`` with e^{i(k.Re+q.Rp)} = e^{ik.Re} e^{iq.Rp}:

    first over Re for each k, then over Rp for each q.  Output
    [nk, nq, nmode, nw, nw] (Wannier gauge, indices i j).
    """
    g = model.g
    nge, ngp = g.shape[:2]
    tail = g.shape[2:]
    gk = phases(kpts, model.R_ge) @ g.reshape(nge, -1).astype(np.complex128)      # [nk, ngp*ncol]
    gk = gk.reshape(len(kpts), ngp, -1)
    pq = phases(qpts, model.R_gp)                                                   # [nq, ngp]
    out = pq[None] @ gk                                                             # [nk, nq, ncol]
    return out.reshape((len(kpts), len(qpts)) + tail)


def reciprocal_vectors(A: np.ndarray) -> np.ndarray:
    """Rows b_i (1/bohr) with a_i . b_j = 2 pi delta_ij; a crystal point k is the Cartesian k @ B."""
    return 2.0 * np.pi * np.linalg.inv(np.asarray(A, np.float64)).T


def frohlich_wannier(model, qpts: np.ndarray) -> np.ndarray:
    """Long-range coupling of Eq. e_ph_long in the Wannier gauge, [nq, nmode] complex, eV/bohr.

    L^{ka}(q) = i (e^2 / (eps_0 Omega)) sum_{G, q+G != 0} [(q+G).Z*_k]_a e^{-i tau_k.(q+G)}
                e^{-(q+G).eps.(q+G) / (4 Lambda)} / ((q+G).eps.(q+G)),
    with every G whose exponent (q+G).eps.(q+G)/(4 Lambda) is at most EWALD_CUT.
    With the smooth-phase bra-ket of Eq. smooth_phase the Bloch-gauge term is
    L^{ka}(q) [U^dagger(k+q) U(k)]_mn, i.e. L^{ka}(q) delta_ij added to the
    Wannier-gauge g before the rotation.  Zero for models without Born charges.
    """
    qpts = np.asarray(qpts, np.float64)
    nm = model.nmode
    if model.zstar is None:
        return np.zeros((len(qpts), nm), dtype=np.complex128)
    A = np.asarray(model.A, np.float64)
    B = reciprocal_vectors(A)
    omega = abs(np.linalg.det(A))
    eps = np.asarray(model.eps_inf, np.float64)
    lam = float(model.ewald_lambda)
    vmax = np.sqrt(4.0 * lam * EWALD_CUT / np.linalg.eigvalsh(eps).min())
    nmax = int(np.ceil(vmax * np.linalg.norm(A, axis=1).max() / (2 * np.pi))) + 2
    r = np.arange(-nmax, nmax + 1)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    pref = 4.0 * np.pi * HARTREE_EV / omega                  # e^2/(eps_0 Omega), eV/bohr^2
    out = np.zeros((len(qpts), model.nat, 3), dtype=np.complex128)
    for q0 in range(0, len(qpts), 1024):
        q = qpts[q0:q0 + 1024]
        v = (q[:, None, :] + n[None, :, :]) @ B                # q + G, Cartesian [nq, nG, 3]
        x = np.einsum("qga,ab,qgb->qg", v, eps, v)
        keep = (x > 0.0) & (x / (4.0 * lam) <= EWALD_CUT)
        w = np.where(keep, np.exp(-x / (4.0 * lam)) / np.where(keep, x, 1.0), 0.0)
        for k in range(model.nat):
            vz = v @ np.asarray(model.zstar[k], np.float64)    # [(q+G).Z*]_a
            ph = np.exp(-1j * (v @ np.asarray(model.tau[k], np.float64)))
            out[q0:q0 + 1024, k] = 1j * pref * np.einsum("qg,qga->qa", w * ph, vz)
    return out.reshape(len(qpts), nm)


def g_wannier_full(model, kpts: np.ndarray, qpts: np.ndarray) -> np.ndarray:
    """Wannier-gauge g of ``g_wannier`` plus the long-range term L^{ka}(q) delta_ij
    (Sec. 2.2.4: short-range part interpolated, long-range part added)."""
    out = g_wannier(model, kpts, qpts)
    if model.zstar is None:
        return out
    L = frohlich_wannier(model, qpts)                           # [nq, nmode]
    return out + L[None, :, :, None, None] * np.eye(model.nw)[None, None, None]


def g_bloch(gw: np.ndarray, Uk: np.ndarray, Ukq: np.ndarray) -> np.ndarray:
    """g_mn = sum_ij U^dagger_mi(k+q) g_ij U_jn(k)  (Eq. eph_mat_wann2, outer sum).

    gw [..., nmode, nw, nw], Uk [..., nw, nw] (broadcast over the mode axis),
    Ukq [..., nw, nw].  Returns [..., nmode, nw(m), nw(n)].  Evaluated as the two
    matrix products U^dagger(k+q) g, then (U^dagger(k+q) g) U(k).
    """
    udag = np.swapaxes(np.conj(Ukq), -1, -2)[..., None, :, :]     # U^dagger(k+q), per mode
    return (udag @ gw) @ np.asarray(Uk)[..., None, :, :]


def g_modes(gb: np.ndarray, hw: np.ndarray, e: np.ndarray, mass: np.ndarray) -> np.ndarray:
    """g_mn nu = sqrt(hbar/(2 omega_nu)) sum_ka e^{ka}_nu / sqrt(M_k) g^{ka}_mn  (Eq. eph_mat).

    gb [..., nmode(ka), nw, nw]; hw [..., nmode(nu)] in eV; e [..., nmode(ka), nmode(nu)].
    Modes with hbar*omega below OMEGA_MIN_EV are set to zero.  Output [..., nu, m, n] in eV.
    """
    m = np.repeat(np.asarray(mass, np.float64), 3)                 # per ka
    hw_safe = np.where(hw >= OMEGA_MIN_EV, hw, 1.0)
    length = np.sqrt(C_OMEGA / (2.0 * m[..., :, None] * hw_safe[..., None, :]))   # [..., ka, nu] bohr
    length = np.where(hw[..., None, :] >= OMEGA_MIN_EV, length, 0.0)
    coef = e * length                                               # [..., ka, nu]
    lead = gb.shape[:-3]
    nmode, nw1, nw2 = gb.shape[-3:]
    cT = np.broadcast_to(np.swapaxes(coef, -1, -2), lead + (coef.shape[-1], nmode))   # [..., nu, ka]
    return (cT @ gb.reshape(lead + (nmode, nw1 * nw2))).reshape(lead + (coef.shape[-1], nw1, nw2))


def g_abs(gm: np.ndarray) -> np.ndarray:
    """|g_nu(k,q)| = sqrt(sum_mn |g_mn nu|^2 / N_b)  (Eq. g_abs).  gm [..., nu, m, n]."""
    nb = gm.shape[-1]
    return np.sqrt(np.sum(np.abs(gm) ** 2, axis=(-1, -2)) / nb)


# ----------------------------------------------------------------------------
# occupations and the broadened delta
# ----------------------------------------------------------------------------

def fermi_dirac(eps, mu: float, T: float):
    return 1.0 / (np.exp((np.asarray(eps) - mu) / (KB_EVK * T)) + 1.0)


def bose_einstein(hw, T: float):
    """N = 1/(e^{hw/kT} - 1); zero for modes below OMEGA_MIN_EV (they carry no weight)."""
    hw = np.asarray(hw, np.float64)
    safe = np.where(hw >= OMEGA_MIN_EV, hw, 1.0)
    return np.where(hw >= OMEGA_MIN_EV, 1.0 / np.expm1(safe / (KB_EVK * T)), 0.0)


def delta_gauss(x, sigma: float):
    return np.exp(-(np.asarray(x) / sigma) ** 2) / (sigma * np.sqrt(np.pi))


# ----------------------------------------------------------------------------
# RTA scattering rates: Sec. 2.1.2, Eqs. scatter_rate and BTE_W
# ----------------------------------------------------------------------------

def scattering_rates(eps_k, eps_kq, hw, g2, T, mu, sigma, nq_total, mode_resolved=False):
    """Gamma_nk = (1/N_q) sum_{m nu q} W (Eq. scatter_rate) with W of Eq. BTE_W.

    eps_k [nk, nw(n)], eps_kq [nk, nq, nw(m)], hw [nq, nmode], g2 = |g_mn nu|^2
    [nk, nq, nmode, nw(m), nw(n)].  Every term is kept (no delta truncation).
    Returns Gamma [nk, nw] in 1/s, or [nk, nmode, nw] when ``mode_resolved``.
    """
    fm = fermi_dirac(eps_kq, mu, T)[:, :, None, :, None]           # final state occupation
    N = bose_einstein(hw, T)[None, :, :, None, None]
    en = eps_k[:, None, None, None, :]
    em = eps_kq[:, :, None, :, None]
    w = hw[None, :, :, None, None]
    emit = delta_gauss(en - w - em, sigma) * (1.0 + N - fm)
    absb = delta_gauss(en + w - em, sigma) * (N + fm)
    live = (hw >= OMEGA_MIN_EV)[None, :, :, None, None]
    W = TWO_PI_OVER_HBAR * g2 * np.where(live, emit + absb, 0.0)
    if mode_resolved:
        return W.sum(axis=(1, 3)) / nq_total                        # [nk, nmode, nw(n)]
    return W.sum(axis=(1, 2, 3)) / nq_total


def scattering_rates_grid(model, kgrid, qgrid, k_indices, T, mu, sigma, mode_resolved=False,
                          q_chunk=None):
    """Gamma_nk for the listed k-grid points with q summed over the full q grid.

    k and k+q are both on the k grid (the q grid is commensurate), as the paper
    requires for dynamics and the iterative BTE (Sec. 4.3).  Works one k (and
    optionally one chunk of q) at a time to bound memory.
    """
    from synthetic import mp_grid  # point lists only
    kg = np.asarray(kgrid)
    qg = np.asarray(qgrid)
    kpts_all = mp_grid(*kg)
    qpts = mp_grid(*qg)
    nq = len(qpts)
    eps_all, U_all = bands(model, kpts_all)
    hw, e = phonons(model, qpts)
    nw, nm = model.nw, model.nmode
    out = np.zeros((len(k_indices), nm, nw)) if mode_resolved else np.zeros((len(k_indices), nw))
    q_chunk = q_chunk or nq
    for a, ik in enumerate(k_indices):
        k = kpts_all[ik:ik + 1]
        kq_row = _kplusq_row(kg, qg, ik)
        for q0 in range(0, nq, q_chunk):
            qs = slice(q0, min(nq, q0 + q_chunk))
            ikq = kq_row[qs]
            gw = g_wannier_full(model, k, qpts[qs])[0]                  # [nq, nm, nw, nw]
            gb = g_bloch(gw, U_all[ik][None], U_all[ikq])
            gm = g_modes(gb, hw[qs], e[qs], model.mass)
            g2 = np.abs(gm) ** 2
            r = scattering_rates(eps_all[ik][None], eps_all[ikq][None], hw[qs], g2[None],
                                 T, mu, sigma, nq, mode_resolved)
            out[a] += r[0]
    return out


def _kplusq_row(kgrid, qgrid, ik):
    """Index of k+q on the k grid for one k-grid point and every q-grid point."""
    kg = np.asarray(kgrid)
    qg = np.asarray(qgrid)
    assert np.all(kg % qg == 0), "q grid must divide the k grid"
    k = np.array([ik // (kg[1] * kg[2]), (ik // kg[2]) % kg[1], ik % kg[2]])
    qi = np.stack(np.meshgrid(*[np.arange(n) for n in qg], indexing="ij"), -1).reshape(-1, 3)
    s = (k[None, :] + qi * (kg // qg)) % kg
    return (s[:, 0] * kg[1] + s[:, 1]) * kg[2] + s[:, 2]


def _kplusq_index(kgrid, qgrid):
    """Index of k+q on the k grid for every k-grid point k and q-grid point q."""
    kg = np.asarray(kgrid)
    qg = np.asarray(qgrid)
    assert np.all(kg % qg == 0), "q grid must divide the k grid"
    step = kg // qg
    ki = np.stack(np.meshgrid(*[np.arange(n) for n in kg], indexing="ij"), -1).reshape(-1, 3)
    qi = np.stack(np.meshgrid(*[np.arange(n) for n in qg], indexing="ij"), -1).reshape(-1, 3)
    s = (ki[:, None, :] + qi[None, :, :] * step) % kg
    return (s[..., 0] * kg[1] + s[..., 1]) * kg[2] + s[..., 2]


# ----------------------------------------------------------------------------
# collision integral: Sec. 2.1, Eq. e_ph_scattering with F_abs, F_em
# ----------------------------------------------------------------------------

def collision(f, eps, row, col, hw, g2, T, sigma, nq_total):
    """I[f]_s for every state s (Eq. e_ph_scattering).

    Each entry e is one (n k -> m k+q, nu) term: initial state row[e], final
    state col[e], phonon energy hw[e] (eV), |g|^2 = g2[e] (eV^2).  Phonon
    occupations are the equilibrium N(hw, T) (kept fixed, Sec. 2.1.1).
    I_s = -(2 pi/hbar)(1/N_q) sum_{e: row=s} |g|^2 [delta(e_n - hw - e_m) F_em
                                                  + delta(e_n + hw - e_m) F_abs].
    """
    f = np.asarray(f, np.float64)
    fn, fm = f[row], f[col]
    en, em = eps[row], eps[col]
    N = bose_einstein(hw, T)
    live = np.asarray(hw) >= OMEGA_MIN_EV
    F_abs = fn * (1 - fm) * N - fm * (1 - fn) * (N + 1)
    F_em = fn * (1 - fm) * (N + 1) - fm * (1 - fn) * N
    term = np.asarray(g2, np.float64) * (delta_gauss(en - hw - em, sigma) * F_em
                                         + delta_gauss(en + hw - em, sigma) * F_abs)
    term = np.where(live, term, 0.0)
    out = np.zeros_like(f)
    np.add.at(out, row, term)
    return -TWO_PI_OVER_HBAR / nq_total * out


# ----------------------------------------------------------------------------
# time stepping: Sec. 2.1.1 (explicit RK4, Euler)
# ----------------------------------------------------------------------------

def rk4_step(f, dt, rhs):
    """Classic 4-stage Runge-Kutta step of df/dt = rhs(f)."""
    k1 = rhs(f)
    k2 = rhs(f + 0.5 * dt * k1)
    k3 = rhs(f + 0.5 * dt * k2)
    k4 = rhs(f + dt * k3)
    return f + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)


def euler_step(f, dt, rhs):
    return f + dt * rhs(f)


FS = 1e-15  # seconds per femtosecond


def evolve(f0, dt_fs, nsteps, rhs, method="rk4"):
    """Integrate df/dt = I[f] (1/s) for ``nsteps`` steps of ``dt_fs`` femtoseconds."""
    step = rk4_step if method == "rk4" else euler_step
    f = np.array(f0, np.float64)
    for _ in range(nsteps):
        f = step(f, dt_fs * FS, rhs)
    return f


# ----------------------------------------------------------------------------
# reverse-mode derivatives of I[f] (Eq. e_ph_scattering) and of RK4 (Sec. 2.1.1)
# ----------------------------------------------------------------------------

def collision_vjp(f, lam, eps, row, col, hw, g2, T, sigma, nq_total):
    """Products with the transposed derivatives of I[f] (Eq. e_ph_scattering).

    Returns (J^T lam, d) with J_sc = dI_s/df_c and d[e] = sum_s lam_s dI_s/d|g|^2_e,
    by the chain rule applied to each term of ``collision``: term e depends on
    f_n = f[row[e]] and f_m = f[col[e]] through F_em and F_abs, is linear in
    |g|^2_e, and enters I_row[e] with the factor -(2 pi/hbar)/N_q.
    """
    f = np.asarray(f, np.float64)
    lam = np.asarray(lam, np.float64)
    fn, fm = f[row], f[col]
    en, em = eps[row], eps[col]
    N = bose_einstein(hw, T)
    live = np.asarray(hw) >= OMEGA_MIN_EV
    d_em = delta_gauss(en - hw - em, sigma)
    d_abs = delta_gauss(en + hw - em, sigma)
    F_abs = fn * (1 - fm) * N - fm * (1 - fn) * (N + 1)
    F_em = fn * (1 - fm) * (N + 1) - fm * (1 - fn) * N
    dFabs_dfn = (1 - fm) * N + fm * (N + 1)
    dFabs_dfm = -fn * N - (1 - fn) * (N + 1)
    dFem_dfn = (1 - fm) * (N + 1) + fm * N
    dFem_dfm = -fn * (N + 1) - (1 - fn) * N
    w = np.where(live, -TWO_PI_OVER_HBAR / nq_total * lam[row], 0.0)
    g2 = np.asarray(g2, np.float64)
    out = np.zeros_like(f)
    np.add.at(out, row, w * g2 * (d_em * dFem_dfn + d_abs * dFabs_dfn))
    np.add.at(out, col, w * g2 * (d_em * dFem_dfm + d_abs * dFabs_dfm))
    return out, w * (d_em * F_em + d_abs * F_abs)


def rk4_adjoint(f0, dt_fs, nsteps, rhs, vjp, lam_end):
    """Derivatives of a loss L(f(t_end)) through ``evolve(f0, dt_fs, nsteps, rhs)``.

    ``vjp(x, kappa)`` returns (J(x)^T kappa, dtheta) for J = d rhs/dx at x and
    dtheta = kappa . d rhs/dtheta of the rhs parameters theta.  Given
    lam_end = dL/df(t_end), returns (dL/df0, dL/dtheta): reverse-mode
    differentiation of each step f' = f + dt/6 (k1 + 2 k2 + 2 k3 + k4),
    k1 = rhs(f), k2 = rhs(f + dt/2 k1), k3 = rhs(f + dt/2 k2), k4 = rhs(f + dt k3),
    taken from the last step back to the first.  All forward states are kept.
    """
    dt = dt_fs * FS
    states = [np.array(f0, np.float64)]
    for _ in range(nsteps):
        states.append(rk4_step(states[-1], dt, rhs))
    lam = np.array(lam_end, np.float64)
    dtheta = 0.0
    for x1 in reversed(states[:-1]):
        k1 = rhs(x1)
        x2 = x1 + 0.5 * dt * k1
        k2 = rhs(x2)
        x3 = x1 + 0.5 * dt * k2
        k3 = rhs(x3)
        x4 = x1 + dt * k3
        # adjoints of k4, k3, k2, k1 in turn; v_i is the adjoint reaching x_i
        v4, t4 = vjp(x4, dt / 6.0 * lam)
        v3, t3 = vjp(x3, dt / 3.0 * lam + dt * v4)
        v2, t2 = vjp(x2, dt / 3.0 * lam + 0.5 * dt * v3)
        v1, t1 = vjp(x1, dt / 6.0 * lam + 0.5 * dt * v2)
        lam = lam + v1 + v2 + v3 + v4
        dtheta = dtheta + t1 + t2 + t3 + t4
    return lam, dtheta


# ----------------------------------------------------------------------------
# (k, q)-pair scattering list on commensurate grids: Sec. 4.3
# ----------------------------------------------------------------------------

def collision_list_grid(model, grid, band_lo, band_hi, sigma=None, screen=0.0, window=None):
    """All scattering terms between states (n, k) with k on ``grid`` and n in [band_lo, band_hi).

    States are numbered s = ik * nb + (n - band_lo).  The q grid equals the k
    grid, so k+q is always a state.  For each term (s -> s', nu, q) the list
    holds |g_mn nu(k,q)|^2 and hbar*omega_nu q.  The unordered process
    {s, s'} gets ONE |g|^2 value for both directions: the value computed in
    the direction with s < s' (the reverse direction s' -> s at -q has the same
    |g|^2 by the hermiticity of the perturbation), so that the sum of I[f]
    over states vanishes to rounding.  With ``screen > 0`` a term is dropped
    when both Gaussian factors exp(-x^2/sigma^2) are below ``screen``; the
    rule is symmetric between the two directions.  With ``window = (lo, hi)``
    only states with lo <= eps <= hi take part (Sec. 4.3 energy window).

    Returns dict with row, col, mode (int arrays, ordered by row), g2, hw
    (float64), eps (state energies) and nq.
    """
    from synthetic import mp_grid
    g = np.asarray(grid)
    pts = mp_grid(*g)
    nk = len(pts)
    nb = band_hi - band_lo
    eps_all, U_all = bands(model, pts)
    hw_all, e_all = phonons(model, pts)
    kq = _kplusq_index(g, g)
    neg_q = _kplusq_index(g, g)[0]            # index of -q: solve 0 + q' = -q on the grid
    negidx = np.empty(nk, dtype=np.int64)
    ki = np.stack(np.meshgrid(*[np.arange(n) for n in g], indexing="ij"), -1).reshape(-1, 3)
    nki = (-ki) % g
    negidx[:] = (nki[:, 0] * g[1] + nki[:, 1]) * g[2] + nki[:, 2]
    del neg_q
    nm = model.nmode
    g2_all = np.empty((nk, nk, nm, nb, nb))       # [k, q, nu, m, n]
    sel = slice(band_lo, band_hi)
    for ik in range(nk):
        gw = g_wannier_full(model, pts[ik:ik + 1], pts)[0]
        gb = g_bloch(gw, U_all[ik][None], U_all[kq[ik]])
        gm = g_modes(gb, hw_all, e_all, model.mass)[:, :, sel, sel]
        g2_all[ik] = np.abs(gm) ** 2
    rows, cols, modes, vals, hws = [], [], [], [], []
    eps_state = eps_all[:, sel].reshape(-1)
    inwin = np.ones(len(eps_state), bool)
    if window is not None:
        inwin = (eps_state >= window[0]) & (eps_state <= window[1])
    for ik in range(nk):
        for iq in range(nk):
            ikq = kq[ik, iq]
            for nu in range(nm):
                for n in range(nb):
                    s = ik * nb + n
                    if not inwin[s]:
                        continue
                    for m in range(nb):
                        sp = ikq * nb + m
                        if not inwin[sp]:
                            continue
                        if s <= sp:
                            val = g2_all[ik, iq, nu, m, n]
                        else:
                            # reverse process: sp -> s at -q, initial band m, final band n
                            val = g2_all[ikq, negidx[iq], nu, n, m]
                        hw = hw_all[iq, nu]
                        if hw < OMEGA_MIN_EV:
                            continue      # carries no weight (acoustic modes at q = Gamma)
                        if screen > 0.0:
                            x1 = eps_state[s] - hw - eps_state[sp]
                            x2 = eps_state[s] + hw - eps_state[sp]
                            if max(np.exp(-(x1 / sigma) ** 2), np.exp(-(x2 / sigma) ** 2)) < screen:
                                continue
                        rows.append(s)
                        cols.append(sp)
                        modes.append(nu)
                        vals.append(val)
                        hws.append(hw)
    order = np.argsort(np.array(rows, np.int64), kind="stable")   # entries grouped by initial state
    return {"row": np.array(rows, np.int64)[order], "col": np.array(cols, np.int64)[order],
            "mode": np.array(modes, np.int64)[order], "g2": np.array(vals)[order],
            "hw": np.array(hws)[order], "eps": eps_state, "nq": nk, "nstates": nk * nb}


def collision_rows(model, grid, band_lo, band_hi, states, f, T, sigma, window=None):
    """I[f]_s (Eq. e_ph_scattering) for selected states s = ik*nb + (n - band_lo).

    Sums over every q of the grid (= k grid), every final band m in
    [band_lo, band_hi) whose state lies in the window, and every mode, with
    |g_mn nu(k,q)|^2 interpolated at the initial k (no screening).  Needs only
    the interpolation at the listed k-points, so it serves as a per-row check of
    lists too large for ``collision_list_grid``.
    """
    from synthetic import mp_grid
    g = np.asarray(grid)
    pts = mp_grid(*g)
    nk = len(pts)
    nb = band_hi - band_lo
    sel = slice(band_lo, band_hi)
    eps_all, U_all = bands(model, pts)
    hw_all, e_all = phonons(model, pts)
    eps_state = eps_all[:, sel].reshape(-1)
    inwin = np.ones(len(eps_state), bool)
    if window is not None:
        inwin = (eps_state >= window[0]) & (eps_state <= window[1])
    f = np.asarray(f, np.float64)
    N = bose_einstein(hw_all, T)                                   # [q, nu]
    live = hw_all >= OMEGA_MIN_EV
    out = []
    for s in states:
        ik, n = divmod(int(s), nb)
        kq = _kplusq_row(g, g, ik)
        gw = g_wannier_full(model, pts[ik:ik + 1], pts)[0]
        gb = g_bloch(gw, U_all[ik][None], U_all[kq])
        g2 = np.abs(g_modes(gb, hw_all, e_all, model.mass)[:, :, sel, sel][:, :, :, n]) ** 2       # [q, nu, m]
        sp = kq[:, None] * nb + np.arange(nb)[None, :]              # [q, m]
        fn, fm = f[s], f[sp][:, None, :]
        en, em = eps_state[s], eps_state[sp][:, None, :]
        w = hw_all[:, :, None]
        Nq = N[:, :, None]
        F_abs = fn * (1 - fm) * Nq - fm * (1 - fn) * (Nq + 1)
        F_em = fn * (1 - fm) * (Nq + 1) - fm * (1 - fn) * Nq
        term = g2 * (delta_gauss(en - w - em, sigma) * F_em + delta_gauss(en + w - em, sigma) * F_abs)
        mask = live[:, :, None] & inwin[sp][:, None, :]
        out.append(-TWO_PI_OVER_HBAR / nk * np.sum(np.where(mask, term, 0.0)))
    return np.array(out)


# ----------------------------------------------------------------------------
# band velocities (Eqs. velocity, wannier_4), iterative BTE (Eqs. BTE_lin,
# BTE_iter, BTE_W) and the mobility (Eq. cond), Sec. 2.1.2 and 2.2.1
# ----------------------------------------------------------------------------

def velocities(model, kpts: np.ndarray, deg_tol: float = 1e-6) -> np.ndarray:
    """v_nk (m/s), [nk, nw, 3]: hbar v^a = [U^dagger(k) H_a(k) U(k)]_nn with
    H_a(k) = sum_R e^{ik.R} H(R) (i R^a), R^a Cartesian (Eq. wannier_4).

    For bands degenerate within ``deg_tol`` eV the velocities along each
    Cartesian direction are the eigenvalues (ascending) of that direction's
    matrix restricted to the degenerate subspace (the degenerate extension).
    """
    kpts = np.asarray(kpts, np.float64)
    Rc = np.asarray(model.R_H, np.float64) @ np.asarray(model.A, np.float64)      # [nR, 3] bohr
    ph = phases(kpts, model.R_H)
    Ha = np.einsum("kr,ra,rij->kaij", ph, 1j * Rc, model.H.astype(np.complex128))   # eV bohr
    eps, U = bands(model, kpts)
    M = np.einsum("kin,kaij,kjm->kanm", np.conj(U), Ha, U)
    v = np.real(np.einsum("kann->kan", M)).copy()
    for k in range(len(kpts)):
        n = 0
        while n < model.nw:
            e = n + 1
            while e < model.nw and eps[k, e] - eps[k, e - 1] <= deg_tol:
                e += 1
            if e - n > 1:
                for a in range(3):
                    v[k, a, n:e] = np.linalg.eigvalsh(M[k, a, n:e, n:e])
            n = e
    return np.transpose(v, (0, 2, 1)) * (BOHR_M / HBAR_EVS)


def bte_weights(eps, row, col, hw, g2, T, mu, sigma, nq_total):
    """W_{nk,mk+q}^{nu q} / N_q per list entry (Eq. BTE_W), 1/s."""
    f_m = fermi_dirac(eps[col], mu, T)
    N = bose_einstein(hw, T)
    live = np.asarray(hw) >= OMEGA_MIN_EV
    d = eps[row] - eps[col]
    W = TWO_PI_OVER_HBAR * np.asarray(g2, np.float64) * (
        delta_gauss(d - hw, sigma) * (1.0 + N - f_m) + delta_gauss(d + hw, sigma) * (N + f_m))
    return np.where(live, W, 0.0) / nq_total


def bte_iterate(tau, v, row, col, w, max_iter=200, tol=1e-10):
    """F^{i+1} = tau v + tau sum_e w_e F^i_col (Eq. BTE_iter from F^0 = tau v).

    tau [ns] s, v [ns, 3] m/s, w per list entry (``bte_weights``).  Stops when
    max |F^{i+1} - F^i| <= tol max |F^0|.  Returns (F [ns, 3] in m, iterations).
    """
    tau = np.asarray(tau, np.float64)
    F0 = tau[:, None] * np.asarray(v, np.float64)
    F = F0.copy()
    scale = np.abs(F0).max()
    for it in range(1, max_iter + 1):
        S = np.zeros_like(F)
        np.add.at(S, row, np.asarray(w, np.float64)[:, None] * F[col])
        Fn = F0 + tau[:, None] * S
        diff = np.abs(Fn - F).max()
        F = Fn
        if diff <= tol * scale:
            return F, it
    return F, max_iter


def mobility(v, F, eps, T, mu):
    """mu_ab = sigma_ab / (e n_c) (Eq. cond) in cm^2/(V s).

    With n_c = (S / (N_k Omega)) sum f0 over the same states, the prefactors
    cancel: mu_ab = sum v^a F^b (-df0/de) / sum f0, with -df0/de = f0 (1 - f0) / kT
    in 1/eV, v in m/s and F in m.
    """
    f = fermi_dirac(eps, mu, T)
    w = f * (1.0 - f) / (KB_EVK * T)
    return 1e4 * np.einsum("s,sa,sb->ab", w, np.asarray(v), np.asarray(F)) / f.sum()


# ----------------------------------------------------------------------------
# Monte-Carlo q sampling of Gamma_nk (Sec. 4.3: random q, uniform or Cauchy)
# ----------------------------------------------------------------------------

Q_UNIFORM, Q_CAUCHY = 0, 1


def mc_qpoints(u, sampling, width=1.0):
    """q points (crystal coordinates) and 1/p(q) from uniforms u [nq, 3] in [0, 1).

    Uniform: q_i = u_i - 1/2, p = 1.  Cauchy (reading of the paper's Cauchy
    sampling on the periodic zone): each coordinate by the tangent map
    q_i = atan(c tan(pi (u_i - 1/2))) / pi, whose density on [-1/2, 1/2) is
    p(q_i) = c / (c^2 cos^2(pi q_i) + sin^2(pi q_i)) (Lorentzian of width ~c/pi
    near q_i = 0, normalised over the zone); p(q) is the product over i.
    """
    u = np.asarray(u, np.float64)
    if sampling == Q_UNIFORM:
        return u - 0.5, np.ones(len(u))
    c = float(width)
    q = np.arctan(c * np.tan(np.pi * (u - 0.5))) / np.pi
    p = c / (c * c * np.cos(np.pi * q) ** 2 + np.sin(np.pi * q) ** 2)
    return q, 1.0 / np.prod(p, axis=1)


def scattering_rates_mc(model, kpts, u, sampling, width, T, mu, sigma):
    """Gamma_nk at arbitrary k (Eqs. scatter_rate, BTE_W) by Monte-Carlo q sampling.

    With samples q_j of density p: Gamma = (1/N) sum_j y_j, y_j = sum_{m nu} W(q_j) / p(q_j),
    bands at k + q_j and phonons at q_j interpolated per sample, g from the
    short- plus long-range Wannier sum.  Returns (Gamma [nk, nw], standard error
    [nk, nw] = sqrt(sum_j (y_j - Gamma)^2 / (N (N - 1)))).
    """
    q, pinv = mc_qpoints(u, sampling, width)
    kpts = np.asarray(kpts, np.float64)
    nq = len(q)
    eps_k, U_k = bands(model, kpts)
    hw, e = phonons(model, q)
    gam = np.zeros((len(kpts), model.nw))
    err = np.zeros((len(kpts), model.nw))
    for a in range(len(kpts)):
        eps_kq, U_kq = bands(model, kpts[a] + q)
        gw = g_wannier_full(model, kpts[a:a + 1], q)[0]
        g2 = np.abs(g_modes(g_bloch(gw, U_k[a][None], U_kq), hw, e, model.mass)) ** 2   # [q, nu, m, n]
        f_m = fermi_dirac(eps_kq, mu, T)[:, None, :, None]
        N = bose_einstein(hw, T)[:, :, None, None]
        d = eps_k[a][None, None, None, :] - eps_kq[:, None, :, None]
        w = hw[:, :, None, None]
        live = (hw >= OMEGA_MIN_EV)[:, :, None, None]
        W = TWO_PI_OVER_HBAR * g2 * np.where(live, delta_gauss(d - w, sigma) * (1 + N - f_m)
                                             + delta_gauss(d + w, sigma) * (N + f_m), 0.0)
        y = W.sum(axis=(1, 2)) * pinv[:, None]                       # [q, n]
        gam[a] = y.mean(axis=0)
        err[a] = np.sqrt(((y - gam[a]) ** 2).sum(axis=0) / (nq * (nq - 1))) if nq > 1 else 0.0
    return gam, err


# ----------------------------------------------------------------------------
# carrier population p(E, t) by the linear tetrahedron method (Eq. pop)
# ----------------------------------------------------------------------------

def grid_tetrahedra(grid):
    """Six tetrahedra per cell of a periodic grid, split along the cell's (0,0,0)-(1,1,1)
    diagonal: [6 N, 4] indices of grid points (the corners of each tetrahedron)."""
    n1, n2, n3 = grid
    corners = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0), (0, 0, 1), (1, 0, 1), (0, 1, 1), (1, 1, 1)]
    # the six paths 0 -> 7 through the cube, one tetrahedron each
    paths = [(0, 1, 3, 7), (0, 1, 5, 7), (0, 2, 3, 7), (0, 2, 6, 7), (0, 4, 5, 7), (0, 4, 6, 7)]
    i1, i2, i3 = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
    base = np.stack([i1.ravel(), i2.ravel(), i3.ravel()], -1)
    out = []
    for path in paths:
        idx = []
        for cidx in path:
            d = np.array(corners[cidx])
            p = (base + d) % np.array(grid)
            idx.append((p[:, 0] * n2 + p[:, 1]) * n3 + p[:, 2])
        out.append(np.stack(idx, -1))
    return np.concatenate(out, 0)


def tetra_theta_weights(e, E):
    """Corner weights w [.., 4] with int_T f theta(E - eps) dk = V_T sum_i w_i f_i for eps and f
    linear in the tetrahedron T (corner energies e [.., 4], any order); the weights
    are per unit volume of T, so sum_i w_i is the fraction of T below E (Bloechl's
    linear tetrahedron integration weights)."""
    e = np.asarray(e, np.float64)
    order = np.argsort(e, axis=-1, kind="stable")
    es = np.take_along_axis(e, order, -1)
    e1, e2, e3, e4 = (es[..., i] for i in range(4))
    ws = np.zeros(es.shape)
    x = E
    with np.errstate(divide="ignore", invalid="ignore"):
        # e1 <= E < e2
        m = (x >= e1) & (x < e2)
        if np.any(m):
            d1, d21, d31, d41 = x - e1[m], e2[m] - e1[m], e3[m] - e1[m], e4[m] - e1[m]
            C = 0.25 * d1 ** 3 / (d21 * d31 * d41)
            ws[m, 0] = C * (4 - d1 * (1 / d21 + 1 / d31 + 1 / d41))
            ws[m, 1] = C * d1 / d21
            ws[m, 2] = C * d1 / d31
            ws[m, 3] = C * d1 / d41
        # e2 <= E < e3
        m = (x >= e2) & (x < e3)
        if np.any(m):
            a1, a2, b3, b4 = x - e1[m], x - e2[m], e3[m] - x, e4[m] - x
            d31, d41, d32, d42 = e3[m] - e1[m], e4[m] - e1[m], e3[m] - e2[m], e4[m] - e2[m]
            C1 = 0.25 * a1 ** 2 / (d41 * d31)
            C2 = 0.25 * a1 * a2 * b3 / (d41 * d32 * d31)
            C3 = 0.25 * a2 ** 2 * b4 / (d42 * d32 * d41)
            ws[m, 0] = C1 + (C1 + C2) * b3 / d31 + (C1 + C2 + C3) * b4 / d41
            ws[m, 1] = C1 + C2 + C3 + (C2 + C3) * b3 / d32 + C3 * b4 / d42
            ws[m, 2] = (C1 + C2) * a1 / d31 + (C2 + C3) * a2 / d32
            ws[m, 3] = (C1 + C2 + C3) * a1 / d41 + C3 * a2 / d42
        # e3 <= E < e4
        m = (x >= e3) & (x < e4)
        if np.any(m):
            b4, d41, d42, d43 = e4[m] - x, e4[m] - e1[m], e4[m] - e2[m], e4[m] - e3[m]
            C = 0.25 * b4 ** 3 / (d41 * d42 * d43)
            ws[m, 0] = 0.25 - C * b4 / d41
            ws[m, 1] = 0.25 - C * b4 / d42
            ws[m, 2] = 0.25 - C * b4 / d43
            ws[m, 3] = 0.25 - C * (4 - b4 * (1 / d41 + 1 / d42 + 1 / d43))
        m = x >= e4
        ws[m] = 0.25
    w = np.zeros(es.shape)
    np.put_along_axis(w, order, ws, -1)
    return w


def population_cumulative(eps, f, grid, E_edges):
    """N(E) = sum_n (1/V_BZ) int f_n(k) theta(E - eps_n(k)) dk (carriers per cell below E) for
    each E in E_edges, by the linear tetrahedron method on the k grid; eps, f [Nk, nb].
    The carrier population of Eq. pop integrated over a bin is N(E_b) - N(E_a)."""
    tet = grid_tetrahedra(grid)
    ntet = len(tet)
    eps = np.asarray(eps, np.float64)
    f = np.asarray(f, np.float64)
    out = np.zeros(len(E_edges))
    for n in range(eps.shape[1]):
        et, ft = eps[tet, n], f[tet, n]
        for j, E in enumerate(E_edges):
            out[j] += np.sum(tetra_theta_weights(et, E) * ft) / ntet
    return out
