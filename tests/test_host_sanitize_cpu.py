"""Host code of the library under AddressSanitizer and UndefinedBehaviorSanitizer (no GPU).

tests/host_harness.cpp is built with g++ -fsanitize=address,undefined against the
library's host-only headers: the cos/sin table of the Hermitian Fourier sums
(herm_table.h, Sec. 2.2.1 Eq. wannier_3 and Sec. 2.2.2 Eq. IFC2) and the Jacobi
eigensolver template (heevj.cuh, which the device kernels instantiate too).  Each
run must exit cleanly with no sanitizer report, and its results must match the
oracle: the table applied at random points reproduces the oracle's H(k) and
mass-scaled D(q); the eigenpairs reproduce LAPACK's eigenvalues and A V = V diag(w)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import synthetic as S
from oracle import eph as O

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2002_02045_gb300", "csrc")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    out = str(tmp_path_factory.mktemp("san") / "host_harness")
    cmd = [gxx, "-std=c++17", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
           "-fno-omit-frame-pointer", "-I", CUDA_INC, "-I", CSRC, os.path.join(HERE, "host_harness.cpp"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("sanitizer runtime unavailable: " + r.stderr[-200:])
    assert r.returncode == 0, r.stderr
    return out


def run(harness, args):
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0:halt_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    r = subprocess.run([harness] + args, capture_output=True, text=True, env=env)
    assert "runtime error" not in r.stderr and "Sanitizer" not in r.stderr, r.stderr[-2000:]
    assert r.returncode == 0, (r.returncode, r.stderr[-2000:])


def packed(M):
    n = M.shape[1]
    cols = [M[:, i, i].real for i in range(n)]
    for i in range(n):
        for j in range(i + 1, n):
            cols += [M[:, i, j].real, M[:, i, j].imag]
    return np.stack(cols, axis=1)


def table(harness, tmp_path, R, X):
    R = np.ascontiguousarray(R, np.int32)
    X = np.ascontiguousarray(X, np.complex128)
    fin, fout = str(tmp_path / "t.in"), str(tmp_path / "t.out")
    with open(fin, "wb") as f:
        np.array([len(R), X.shape[1]], np.int32).tofile(f)
        R.tofile(f)
        X.view(np.float64).tofile(f)
    run(harness, ["herm_table", fin, fout])
    raw = open(fout, "rb").read()
    ok, nrep, M = np.frombuffer(raw[:12], np.int32)
    if not ok:
        return None
    reps = np.frombuffer(raw[12:12 + 12 * nrep], np.int32).reshape(nrep, 3)
    T = np.frombuffer(raw[12 + 12 * nrep:], np.float64).reshape(2 * nrep, -1)
    return reps, T, int(M)


def apply(reps, T, pts):
    ph = 2 * np.pi * pts @ reps.T.astype(np.float64)
    A = np.empty((len(pts), T.shape[0]))
    A[:, 0::2] = np.cos(ph)
    A[:, 1::2] = np.sin(ph)
    return A @ T


CASES = {
    "c1_H": lambda: (S.model_c1(), "H"),
    "c2_H": lambda: (S.model_c2(rcut=14.0), "H"),
    "c3_D": lambda: (S.model_c3(rcut=13.0), "D"),
    "batch44_H": lambda: (S.model_batch_instance(44), "H"),
    "batch44_D": lambda: (S.model_batch_instance(44), "D"),
}


@pytest.mark.parametrize("name", list(CASES))
def test_herm_table_reproduces_oracle(harness, tmp_path, name):
    m, which = CASES[name]()
    pts = np.random.default_rng(5).uniform(-1.5, 1.5, (40, 3))
    if which == "H":
        R, X = m.R_H, m.H
        ref = O.hamiltonian_k(m, pts)
    else:
        sc = 1.0 / np.sqrt(np.repeat(np.asarray(m.mass, np.float64), 3))
        R, X = m.R_D, m.D * sc[None, :, None] * sc[None, None, :]
        ref = O.dynamical_matrix(m, pts)
    ref = 0.5 * (ref + np.conj(np.swapaxes(ref, 1, 2)))
    out = table(harness, tmp_path, R, X)
    assert out is not None
    reps, T, M = out
    # one representative of each {R, -R}: zero or lexicographically positive
    assert len(reps) == (len(R) + 1) // 2
    lex_pos = (reps[:, 0] > 0) | ((reps[:, 0] == 0) & ((reps[:, 1] > 0) | ((reps[:, 1] == 0) & (reps[:, 2] >= 0))))
    assert np.all(lex_pos) and M == np.abs(reps).max()
    got = apply(reps, T, pts)
    assert np.abs(got - packed(ref)).max() <= 1e-12 * np.abs(ref).max()


def test_herm_table_rejects_an_open_set(harness, tmp_path):
    m = S.model_c1()
    R, X = np.asarray(m.R_H), np.asarray(m.H)
    keep = np.ones(len(R), bool)
    keep[np.nonzero(np.any(R != 0, axis=1))[0][0]] = False     # drop one nonzero R, keep its -R
    assert table(harness, tmp_path, R[keep], X[keep]) is None


@pytest.mark.parametrize("n", [2, 3, 6, 8, 16])
def test_host_jacobi_against_lapack(harness, tmp_path, n):
    rng = np.random.default_rng(40 + n)
    mats = []
    for t in range(24):
        Xr = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
        H = Xr + Xr.conj().T
        if t % 3 == 1:       # an exact degeneracy
            w, U = np.linalg.eigh(H)
            w[1] = w[0]
            H = (U * w) @ U.conj().T
            H = 0.5 * (H + H.conj().T)
        mats.append(H)
    mats = np.ascontiguousarray(np.stack(mats), np.complex128)
    fin, fout = str(tmp_path / "h.in"), str(tmp_path / "h.out")
    mats.view(np.float64).tofile(fin)
    run(harness, ["heevj", str(n), str(len(mats)), fin, fout])
    raw = np.fromfile(fout, np.float64)
    ev = raw[:len(mats) * n].reshape(len(mats), n)
    V = raw[len(mats) * n:].view(np.complex128).reshape(len(mats), n, n)
    scale = np.abs(mats).max()
    assert np.abs(ev - np.linalg.eigvalsh(mats)).max() <= 1e-12 * scale
    assert np.all(np.diff(ev, axis=1) >= 0)
    res = np.einsum("kij,kjn->kin", mats, V) - V * ev[:, None, :]
    assert np.abs(res).max() <= 1e-12 * scale
    assert np.abs(np.einsum("kin,kim->knm", V.conj(), V) - np.eye(n)).max() <= 1e-12
