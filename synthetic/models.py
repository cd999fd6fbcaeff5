"""Seeded synthetic real-space models shaped like the paper's workloads.

The paper's inputs are H(R_e) (Sec. 2.2.1, Eq. wannier_2), the interatomic
force constants D(R_p) without mass factor (Sec. 2.2.2, Eq. IFC1) and the
Wannier-basis e-ph matrix elements g~(R_e, R_p) (Sec. 2.2.3, Eq. eph_mat_wann),
all produced by DFT/DFPT + Wannier90 on real materials.  None of that data is
available, so every model here is drawn from a fixed seed with the sizes,
decay lengths and symmetry constraints of the paper's workloads.

Conventions shared by every consumer (oracle and CUDA path):

* ``A[i]`` is lattice vector a_i in bohr; R vectors are integer crystal
  coordinates n (R = n @ A); k and q points are crystal coordinates in units
  of the reciprocal vectors, so that k.R = 2*pi * sum_i k_i n_i.
* ``H[r, n, n']`` = <n 0|H|n' R_r> in eV, with H(-R) = H(R)^dagger.
* ``D[r, ka, k'b]`` = force constant in eV/bohr^2 (no mass factor), real,
  D(-R) = D(R)^T.  Mode index ka = 3*kappa + alpha.
* ``g[re, rp, ka, i, j]`` = g~_ij^{ka}(R_e, R_p) numerically in eV/bohr on the
  dense product of the two R lists.  It obeys the hermiticity of the
  perturbation potential, g~_ij(R_e,R_p) = conj(g~_ji(-R_e, R_p - R_e)).
* Masses in amu.
* Polar models carry Born charges, the dielectric tensor and the Ewald
  parameter of the long-range coupling (Eq. e_ph_long); the short-range g~
  is then the part left to the Wannier sum.

Nothing here evaluates the method (no Fourier sum, eigensolve or rate).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 200202045  # "2002.02045" as an integer; workload c uses SEED_BASE + c


@dataclass
class Model:
    name: str
    A: np.ndarray          # (3,3) bohr, rows are lattice vectors
    tau: np.ndarray        # (nat,3) bohr, Cartesian atom positions
    mass: np.ndarray       # (nat,) amu
    R_H: np.ndarray        # (nRH,3) int32
    H: np.ndarray          # (nRH,nw,nw) complex128, eV
    R_D: np.ndarray        # (nRD,3) int32
    D: np.ndarray          # (nRD,nmode,nmode) float64, eV/bohr^2
    R_ge: np.ndarray       # (nge,3) int32
    R_gp: np.ndarray       # (ngp,3) int32
    g: np.ndarray          # (nge,ngp,nmode,nw,nw) complex64 or complex128, eV/bohr
    meta: dict = field(default_factory=dict)
    # polar materials (Sec. 2.2.4): Born effective charges Z*[kappa][beta][alpha]
    # (the alpha component of (q+G).Z* is sum_beta (q+G)_beta Z*[kappa][beta][alpha]),
    # high-frequency dielectric tensor, Ewald parameter Lambda in 1/bohr^2
    zstar: np.ndarray = None
    eps_inf: np.ndarray = None
    ewald_lambda: float = 0.0

    @property
    def nw(self) -> int:
        return int(self.H.shape[1])

    @property
    def nat(self) -> int:
        return int(self.mass.shape[0])

    @property
    def nmode(self) -> int:
        return 3 * self.nat


# ----------------------------------------------------------------------------
# point lists
# ----------------------------------------------------------------------------

def mp_grid(n1: int, n2: int, n3: int) -> np.ndarray:
    """Gamma-centred Monkhorst-Pack grid (Sec. 4.3) in crystal coordinates.

    Point index p = (i1*n2 + i2)*n3 + i3 holds (i1/n1, i2/n2, i3/n3); no
    folding into the first zone is applied (phases are periodic).
    """
    i1, i2, i3 = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
    pts = np.stack([i1 / n1, i2 / n2, i3 / n3], axis=-1).reshape(-1, 3)
    return pts.astype(np.float64)


# ----------------------------------------------------------------------------
# helpers that build lattice-vector sets and enforce the stated symmetries
# ----------------------------------------------------------------------------

def _cube_vectors(rmax: int) -> np.ndarray:
    n = np.arange(-rmax, rmax + 1)
    N = np.stack(np.meshgrid(n, n, n, indexing="ij"), axis=-1).reshape(-1, 3)
    return N.astype(np.int32)


def _ball_vectors(A: np.ndarray, rcut: float, nmax: int = 10) -> np.ndarray:
    N = _cube_vectors(nmax)
    d = np.linalg.norm(N @ A, axis=1)
    keep = d <= rcut + 1e-9
    N, d = N[keep], d[keep]
    order = np.lexsort((N[:, 2], N[:, 1], N[:, 0], np.round(d, 9)))
    return N[order]


def _index_map(R: np.ndarray):
    table = {tuple(r): i for i, r in enumerate(R.tolist())}

    def find(v):
        return table.get(tuple(int(x) for x in v), -1)

    return find


def _hermitian_symmetrise_hr(R: np.ndarray, H: np.ndarray) -> np.ndarray:
    """H(R) <- (H(R) + H(-R)^dagger)/2 so that H(k) is Hermitian."""
    find = _index_map(R)
    neg = np.array([find(-r) for r in R])
    assert (neg >= 0).all(), "R set must be closed under inversion"
    return 0.5 * (H + np.conj(np.swapaxes(H[neg], -1, -2)))


def _partner_symmetrise_g(R_e: np.ndarray, R_p: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Impose g~_ij(Re,Rp) = conj(g~_ji(-Re, Rp-Re)) on a finite R-pair set.

    Pairs whose partner (-Re, Rp-Re) is outside the set are zeroed first, then
    g <- (g + partner)/2.  The partner map is an involution, so the result
    satisfies the constraint exactly.
    """
    fe, fp = _index_map(R_e), _index_map(R_p)
    neg_e = np.array([fe(-r) for r in R_e])
    assert (neg_e >= 0).all()
    nge, ngp = len(R_e), len(R_p)
    part_p = np.full((nge, ngp), -1, dtype=np.int64)
    for a in range(nge):
        for b in range(ngp):
            part_p[a, b] = fp(R_p[b] - R_e[a])
    valid = part_p >= 0
    out = np.zeros_like(g)
    for a in range(nge):
        bs = np.nonzero(valid[a])[0]
        if bs.size == 0:
            continue
        pa = neg_e[a]
        pb = part_p[a, bs]
        partner = np.conj(np.swapaxes(g[pa, pb], -1, -2))
        out[a, bs] = 0.5 * (g[a, bs] + partner)
    return out


def _spring_network(A, tau, R, k0, d0, ell, ktrans):
    """Bond springs between every atom pair whose separation lies in the R set.

    Bond (kappa,0)-(kappa',R) of length d gets the symmetric 3x3 stiffness
    K = k(d) [e e^T + ktrans (1 - e e^T)], k(d) = k0 exp(-(d-d0)/ell).  Each
    ordered triple adds -K to D_{kk'}(R) and +K to D_{kk}(0); summed over the
    two orientations of a bond this gives D(-R) = D(R)^T and the acoustic sum
    rule sum_{k',R} D_{kk'}(R) = 0 exactly.
    """
    nat = len(tau)
    find = _index_map(R)
    r0 = find(np.zeros(3, dtype=np.int32))
    D = np.zeros((len(R), 3 * nat, 3 * nat))
    Rc = R @ A
    for k in range(nat):
        for kp in range(nat):
            for r in range(len(R)):
                d = Rc[r] + tau[kp] - tau[k]
                dn = np.linalg.norm(d)
                if dn < 1e-8:
                    continue
                e = d / dn
                kk = k0 * np.exp(-(dn - d0) / ell)
                K = kk * (np.outer(e, e) + ktrans * (np.eye(3) - np.outer(e, e)))
                D[r, 3 * k:3 * k + 3, 3 * kp:3 * kp + 3] -= K
                D[r0, 3 * k:3 * k + 3, 3 * k:3 * k + 3] += K
    return D


# ----------------------------------------------------------------------------
# workload models
# ----------------------------------------------------------------------------

def model_c1(seed: int = SEED_BASE + 1) -> Model:
    """Tiny simple-cubic model: a = 5 bohr, 2 Wannier bands, 1 atom (3 modes).

    * H on the 27 R with |n_i| <= 1: H(0) = diag(0, 1) eV plus N(0, 0.05)
      complex noise off the diagonal; for R != 0 every entry is
      -0.5 exp(-|n|) + N(0, 0.05) (|R| in lattice-constant units), then
      H(R) <- (H(R) + H(-R)^dagger)/2.
    * Isotropic nearest-neighbour springs k = 1 eV/bohr^2: D(+-a_i) = -k I,
      D(0) = 6k I (acoustic sum rule), mass 28 amu.
    * g~ complex128 on the 27 x 27 R pairs, |g~| = 0.05 exp(-(|n_e| + |n_p|)),
      uniform phase, then the partner symmetrisation.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    a = 5.0
    A = a * np.eye(3)
    tau = np.zeros((1, 3))
    mass = np.array([28.0])
    R = _cube_vectors(1)
    nR = len(R)
    Rn = np.linalg.norm(R.astype(float), axis=1)

    nw = 2
    H = np.zeros((nR, nw, nw), dtype=np.complex128)
    for r in range(nR):
        noise = rng.normal(0, 0.05, (nw, nw)) + 1j * rng.normal(0, 0.05, (nw, nw))
        if Rn[r] == 0:
            H[r] = np.diag([0.0, 1.0]) + noise * (1 - np.eye(nw))
        else:
            H[r] = -0.5 * np.exp(-Rn[r]) + noise
    H = _hermitian_symmetrise_hr(R, H)

    kspring = 1.0
    D = np.zeros((nR, 3, 3))
    for r in range(nR):
        if Rn[r] == 0:
            D[r] = 6 * kspring * np.eye(3)
        elif Rn[r] == 1:
            D[r] = -kspring * np.eye(3)

    nm = 3
    mag = 0.05 * np.exp(-(Rn[:, None] + Rn[None, :]))
    phase = rng.uniform(0, 2 * np.pi, (nR, nR, nm, nw, nw))
    g = mag[:, :, None, None, None] * np.exp(1j * phase)
    g = _partner_symmetrise_g(R, R, g)

    return Model("c1_sc_2band", A, tau, mass, R.copy(), H, R.copy(), D, R.copy(), R.copy(), g,
                 meta={"seed": seed, "T": 300.0, "sigma": 0.005, "mu": 0.5, "kgrid": (6, 6, 6),
                       "qgrid": (6, 6, 6)})


C2_LATTICE = 10.26
C2_RCUT = 29.02          # bohr: 381 fcc lattice vectors, the count nearest 400


def model_c2(seed: int = SEED_BASE + 2, rcut: float = C2_RCUT, g_dtype=np.complex64) -> Model:
    """Silicon-like fcc model: a = 10.26 bohr, 8 bands, 2 atoms (6 modes), 28 amu.

    * R sets: the 381 fcc lattice vectors with |R| <= 29.02 bohr (shared by H,
      D and both indices of g~).
    * H(0) = diag(onsite) + N(0, 0.05) complex coupling; H(R != 0) has
      complex N(0,1) entries scaled by 1.85 exp(-|R|/3 bohr) eV; Hermitised (this scale keeps about 5% of
      a 40^3 grid in a 0.3 eV window above the band minimum).
    * D(R): bond springs between all atom pairs inside the R set,
      k(d) = 1.2 exp(-(d - d_nn)/3 bohr) eV/bohr^2 (longitudinal) and 0.3 of
      that transverse, d_nn = sqrt(3) a / 4; acoustic sum rule exact.
    * g~ on the 381 x 381 R pairs, |g~| = 0.1 exp(-(|R_e|/4 + |R_p|/4)) with
      |R| in bohr, uniform phase, partner-symmetrised, stored complex64.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    a = C2_LATTICE
    A = 0.5 * a * np.array([[0, 1, 1], [1, 0, 1], [1, 1, 0]], dtype=np.float64)
    tau = np.array([[0.0, 0.0, 0.0], [0.25 * a, 0.25 * a, 0.25 * a]])
    mass = np.array([28.0, 28.0])
    R = _ball_vectors(A, rcut)
    nR = len(R)
    Rd = np.linalg.norm(R @ A, axis=1)

    nw = 8
    onsite = np.array([0.0, 0.55, 1.1, 1.6, 2.2, 2.8, 3.3, 3.9])
    H = np.zeros((nR, nw, nw), dtype=np.complex128)
    for r in range(nR):
        X = rng.normal(0, 1, (nw, nw)) + 1j * rng.normal(0, 1, (nw, nw))
        if Rd[r] == 0:
            H[r] = np.diag(onsite) + 0.05 * X * (1 - np.eye(nw))
        else:
            H[r] = 1.85 * np.exp(-Rd[r] / 3.0) * X / np.sqrt(2.0)
    H = _hermitian_symmetrise_hr(R, H)

    dnn = np.sqrt(3.0) * a / 4.0
    D = _spring_network(A, tau, R, k0=1.2, d0=dnn, ell=3.0, ktrans=0.3)

    nm = 6
    mag = (0.1 * np.exp(-(Rd[:, None] / 4.0 + Rd[None, :] / 4.0))).astype(np.float64)
    g = np.empty((nR, nR, nm, nw, nw), dtype=np.complex128)
    for re in range(nR):
        ph = rng.uniform(0, 2 * np.pi, (nR, nm, nw, nw))
        g[re] = mag[re][:, None, None, None] * np.exp(1j * ph)
    g = _partner_symmetrise_g(R, R, g).astype(g_dtype)

    return Model("c2_fcc_8band", A, tau, mass, R.copy(), H, R.copy(), D, R.copy(), R.copy(), g,
                 meta={"seed": seed, "T": 300.0, "sigma": 0.010, "kgrid": (40, 40, 40),
                       "qgrid": (40, 40, 40), "window_width": 0.3, "mu_below_min": 0.3})


C3_LATTICE = 10.68
C3_HOP = 2.0             # eV: about 2000 points of a 60^3 grid within 0.2 eV of the band minimum


def model_c3(seed: int = SEED_BASE + 3, rcut: float = C2_RCUT * C3_LATTICE / C2_LATTICE,
             g_dtype=np.complex64) -> Model:
    """Polar GaAs-like zincblende model: a = 10.68 bohr, 8 bands, 2 atoms of 69.7 and 74.9 amu.

    Built like ``model_c2`` (same R sets scaled with the lattice, spring
    network, short-range |g~| = 0.1 exp(-(|R_e|/4 + |R_p|/4))), with hoppings
    scaled by 2.0 exp(-|R|/3 bohr) eV so that about 2000 points of a 60^3 grid lie
    within 0.2 eV of the band minimum, and the long-range coupling of Eq. e_ph_long:
    Z* = +2 I (cation), -2 I (anion), eps_inf = 10.9 I, Lambda = (2 pi / a)^2.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    a = C3_LATTICE
    A = 0.5 * a * np.array([[0, 1, 1], [1, 0, 1], [1, 1, 0]], dtype=np.float64)
    tau = np.array([[0.0, 0.0, 0.0], [0.25 * a, 0.25 * a, 0.25 * a]])
    mass = np.array([69.7, 74.9])
    R = _ball_vectors(A, rcut)
    nR = len(R)
    Rd = np.linalg.norm(R @ A, axis=1)

    nw = 8
    onsite = np.array([0.0, 0.55, 1.1, 1.6, 2.2, 2.8, 3.3, 3.9])
    H = np.zeros((nR, nw, nw), dtype=np.complex128)
    for r in range(nR):
        X = rng.normal(0, 1, (nw, nw)) + 1j * rng.normal(0, 1, (nw, nw))
        if Rd[r] == 0:
            H[r] = np.diag(onsite) + 0.05 * X * (1 - np.eye(nw))
        else:
            H[r] = C3_HOP * np.exp(-Rd[r] / 3.0) * X / np.sqrt(2.0)
    H = _hermitian_symmetrise_hr(R, H)

    dnn = np.sqrt(3.0) * a / 4.0
    D = _spring_network(A, tau, R, k0=1.2, d0=dnn, ell=3.0, ktrans=0.3)

    nm = 6
    mag = (0.1 * np.exp(-(Rd[:, None] / 4.0 + Rd[None, :] / 4.0))).astype(np.float64)
    g = np.empty((nR, nR, nm, nw, nw), dtype=np.complex128)
    for re in range(nR):
        ph = rng.uniform(0, 2 * np.pi, (nR, nm, nw, nw))
        g[re] = mag[re][:, None, None, None] * np.exp(1j * ph)
    g = _partner_symmetrise_g(R, R, g).astype(g_dtype)
    zstar = np.stack([2.0 * np.eye(3), -2.0 * np.eye(3)])
    return Model("c3_zincblende_polar", A, tau, mass, R.copy(), H, R.copy(), D, R.copy(), R.copy(), g,
                 meta={"seed": seed, "T": 300.0, "sigma": 0.010, "kgrid": (60, 60, 60),
                       "qgrid": (60, 60, 60), "window_width": 0.2},
                 zstar=zstar, eps_inf=10.9 * np.eye(3), ewald_lambda=(2 * np.pi / a) ** 2)


BATCH_NW = (2, 4, 8, 12, 16)
BATCH_GRIDS = (8, 12, 16, 24, 32)


def model_batch_instance(i: int, seed: int = SEED_BASE + 5) -> Model:
    """Instance i of the batched workload: a random simple-cubic model.

    Drawn from its own seed: nw in {2, 4, 8, 12, 16}, nat in {1, ..., 5} atoms at
    random positions, one R set of the lattice vectors with |n| <= r, r in {1, 2, 3}
    (shared by H, D and both g~ indices), a grid size in {8, 12, 16, 24, 32} per
    axis (meta "grid").  H(0) = diag of bands 0.25 eV apart + N(0, 0.02) coupling,
    H(R != 0) complex N(0, 1) 0.3 exp(-|n|) eV; bond springs k(d) = 1.5 exp(-(d -
    d_min)/2 bohr) eV/bohr^2 (acoustic sum rule exact); |g~| = 0.05 exp(-(|n_e| +
    |n_p|)/2) eV/bohr with a uniform phase, partner-symmetrised, complex64.
    """
    rng = np.random.Generator(np.random.PCG64([seed, i]))
    nw = int(rng.choice(BATCH_NW))
    nat = int(rng.integers(1, 6))
    r = int(rng.integers(1, 4))
    ng = int(rng.choice(BATCH_GRIDS))
    a = float(rng.uniform(5.0, 7.0))
    A = a * np.eye(3)
    R = _ball_vectors(A, r * a, nmax=r)
    nR = len(R)
    Rn = np.linalg.norm(R.astype(np.float64), axis=1)
    while True:                               # atoms at least 1.5 bohr apart (with images)
        tau = rng.uniform(0, a, (nat, 3))
        dmin = np.inf
        for k in range(nat):
            for kp in range(nat):
                for sh in _cube_vectors(1):
                    if k == kp and not sh.any():
                        continue
                    dmin = min(dmin, np.linalg.norm(tau[kp] + sh * a - tau[k]))
        if dmin > 1.5:
            break
    mass = rng.uniform(10.0, 80.0, nat)
    H = np.zeros((nR, nw, nw), dtype=np.complex128)
    for j in range(nR):
        X = rng.normal(0, 1, (nw, nw)) + 1j * rng.normal(0, 1, (nw, nw))
        if Rn[j] == 0:
            H[j] = np.diag(0.25 * np.arange(nw)) + 0.02 * X * (1 - np.eye(nw))
        else:
            H[j] = 0.3 * np.exp(-Rn[j]) * X / np.sqrt(2.0)
    H = _hermitian_symmetrise_hr(R, H)
    D = _spring_network(A, tau, R, k0=1.5, d0=dmin, ell=2.0, ktrans=0.3)
    nm = 3 * nat
    mag = 0.05 * np.exp(-(Rn[:, None] + Rn[None, :]) / 2.0)
    g = mag[:, :, None, None, None] * np.exp(1j * rng.uniform(0, 2 * np.pi, (nR, nR, nm, nw, nw)))
    g = _partner_symmetrise_g(R, R, g).astype(np.complex64)
    return Model(f"batch_{i}", A, tau, mass, R.copy(), H, R.copy(), D, R.copy(), R.copy(), g,
                 meta={"seed": seed, "index": i, "grid": (ng, ng, ng), "T": 300.0, "sigma": 0.005})


# ----------------------------------------------------------------------------
# special models with closed forms (used as pins)
# ----------------------------------------------------------------------------

def model_sc_tight_binding(eps0: float = 0.3, t: float = -0.25, a: float = 5.0,
                           kspring: float = 1.0, mass: float = 28.0, g0=None) -> Model:
    """One s band on a simple-cubic lattice with nearest-neighbour hopping t.

    Its band is eps(k) = eps0 + 2 t sum_i cos(2 pi k_i).  Phonons are the
    isotropic springs of ``model_c1`` (three degenerate modes with
    (hbar w)^2 proportional to (2k/M) sum_i (1 - cos 2 pi q_i)).  The coupling
    is local and constant, g~^{alpha}(0,0) = g0[alpha], zero elsewhere
    (a Holstein-like model: g(k,q) does not depend on k or q).
    """
    R = _cube_vectors(1)
    nR = len(R)
    Rn = np.abs(R).sum(axis=1)
    H = np.zeros((nR, 1, 1), dtype=np.complex128)
    D = np.zeros((nR, 3, 3))
    for r in range(nR):
        if Rn[r] == 0:
            H[r] = eps0
            D[r] = 6 * kspring * np.eye(3)
        elif Rn[r] == 1 and np.count_nonzero(R[r]) == 1:
            H[r] = t
            D[r] = -kspring * np.eye(3)
    if g0 is None:
        g0 = np.array([0.02, 0.03 + 0.01j, -0.015j])
    g = np.zeros((nR, nR, 3, 1, 1), dtype=np.complex128)
    r0 = int(np.nonzero(Rn == 0)[0][0])
    g[r0, r0, :, 0, 0] = g0
    return Model("sc_tb_1band", a * np.eye(3), np.zeros((1, 3)), np.array([mass]),
                 R.copy(), H, R.copy(), D, R.copy(), R.copy(), g,
                 meta={"eps0": eps0, "t": t, "kspring": kspring, "g0": np.asarray(g0)})


def model_holstein(g0: complex = 0.03, eps0: float = 0.0, t: float = -0.25,
                   kspring: float = 1.0, mass: float = 28.0) -> Model:
    """``model_sc_tight_binding`` with the same local coupling g0 on all three axes."""
    return model_sc_tight_binding(eps0=eps0, t=t, kspring=kspring, mass=mass,
                                  g0=np.array([g0, g0, g0], dtype=np.complex128))


def model_ladder(nw: int = 3, spacing: float = 0.05, einstein_k: float = 0.0,
                 mass: float = 28.0, g0: float = 0.02, seed: int = SEED_BASE + 90) -> Model:
    """Flat bands eps_n = n * spacing and one dispersionless (Einstein) atom.

    ``einstein_k`` sets D(0) = k I with no other R, so every mode has the same
    frequency (the acoustic sum rule is deliberately absent).  When hbar*w
    equals ``spacing`` every emission/absorption term conserves energy
    exactly, which makes the equilibrium collision integral vanish up to the
    Gaussian tails exp(-(spacing/sigma)^2).  The coupling is a random local
    g~^{alpha}_ij(0, 0), partner-symmetrised.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    R = np.zeros((1, 3), dtype=np.int32)
    H = np.diag(np.arange(nw) * spacing).astype(np.complex128)[None]
    D = (einstein_k * np.eye(3))[None]
    g = g0 * (rng.normal(size=(1, 1, 3, nw, nw)) + 1j * rng.normal(size=(1, 1, 3, nw, nw)))
    g = _partner_symmetrise_g(R, R, g)
    return Model("ladder", 5.0 * np.eye(3), np.zeros((1, 3)), np.array([mass]),
                 R.copy(), H, R.copy(), D, R.copy(), R.copy(), g,
                 meta={"spacing": spacing, "einstein_k": einstein_k})


def pulse_occupations(eps: np.ndarray, eps_edge: float, centre: float = 0.5,
                      width: float = 0.1, amplitude: float = 0.1) -> np.ndarray:
    """Hot-carrier Gaussian pulse f0 = A exp(-(eps - eps_edge - centre)^2 / (2 width^2))."""
    return amplitude * np.exp(-((eps - eps_edge - centre) ** 2) / (2 * width ** 2))
