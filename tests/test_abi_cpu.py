"""C-ABI checks that need no GPU: the library loads, exports what the header
declares, refuses to run without a device, and its eigensolver template is
pinned on the host against LAPACK."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2002_02045_gb300 import build, native
    build.build()
    return native.load()


def header_symbols(name="pertgb.h"):
    src = open(os.path.join(ROOT, "include", name)).read()
    return sorted(set(re.findall(r"\b(pgb_[a-z0-9_]+)\s*\(", src)))


def test_header_symbols_exported(lib):
    from paper_2002_02045_gb300 import native
    assert set(header_symbols()) == set(native.ABI_SYMBOLS)
    assert set(header_symbols("pertgb_diag.h")) == set(native.DIAG_SYMBOLS)
    declared = header_symbols() + header_symbols("pertgb_diag.h")
    out = subprocess.run(["nm", "-D", "--defined-only", native.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pgb_\w+)", out))
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    for s in declared:
        getattr(lib, s)


def test_create_without_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    st = lib.pgb_create(C.byref(h), 0, None)
    assert st == -4 and not h.value
    assert lib.pgb_status_string(-4) == b"CUDA error"
    from paper_2002_02045_gb300 import Context, PgbError
    with pytest.raises(PgbError):
        Context(0, stream=0)


def test_null_context_is_rejected(lib):
    assert lib.pgb_set_grids(None, None, None) == -1
    assert lib.pgb_collision(None, None, None) == -1
    assert lib.pgb_last_error(None) == b"null context"


@pytest.mark.parametrize("n", [1, 2, 3, 6, 8, 16])
def test_host_jacobi_matches_lapack(lib, n):
    """The device eigensolver template, run on the host, against numpy.linalg.eigh."""
    fn = lib.pgb_selftest_heevj
    fn.restype = C.c_int
    fn.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
    rng = np.random.default_rng(n)
    cnt = 20
    A = rng.normal(size=(cnt, n, n)) + 1j * rng.normal(size=(cnt, n, n))
    A = A + np.conj(np.swapaxes(A, -1, -2))
    if n >= 3:
        # exact degeneracy: a doubly degenerate eigenvalue in some matrices
        Q = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))[0]
        w = np.arange(n, dtype=float)
        w[1] = w[0]
        A[0] = Q @ np.diag(w) @ np.conj(Q.T)
    A = np.ascontiguousarray(A)
    ev = np.zeros((cnt, n))
    V = np.zeros((cnt, n, n), complex)
    assert fn(n, cnt, A.ctypes.data, ev.ctypes.data, V.ctypes.data) == 0
    ref = np.linalg.eigh(A)[0]
    assert np.allclose(ev, ref, atol=1e-12 * np.abs(ref).max())
    rec = np.einsum("kin,kn,kjn->kij", V, ev, np.conj(V))
    assert np.abs(rec - A).max() < 1e-12 * np.abs(A).max()
    eye = np.einsum("kin,kim->knm", np.conj(V), V)
    assert np.abs(eye - np.eye(n)).max() < 1e-13


def test_every_device_allocation_goes_through_the_counted_call():
    """The allocation-failure hook and the allocation-free entry point's check rely
    on every device allocation of the library passing through one call."""
    csrc = os.path.join(ROOT, "paper_2002_02045_gb300", "csrc")
    offenders = []
    for name in sorted(os.listdir(csrc)):
        for no, line in enumerate(open(os.path.join(csrc, name)), 1):
            code = line.split("//")[0]
            if re.search(r"\bcudaMalloc(Async|Managed|Host|Pitch|3D|Array)?\s*\(", code) or "cudaHostAlloc" in code:
                offenders.append(f"{name}:{no}: {line.strip()}")
    # the one sanctioned call site, inside the wrapper itself
    allowed = [o for o in offenders if o.startswith("api.cu:") and "async ? cudaMallocAsync" in o]
    assert len(allowed) == 1 and len(offenders) == 1, offenders


def test_allocation_hook_without_gpu(lib):
    fn_count, fn_fail = lib.pgb_diag_alloc_count, lib.pgb_diag_fail_alloc
    n0 = fn_count()
    fn_fail(0)
    fn_fail(-1)
    assert fn_count() == n0
