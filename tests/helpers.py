"""Comparison helpers for GPU-vs-oracle parity (tolerance norms of the design notes)."""
import numpy as np


def degenerate_sum(x, vals, axis, tol=1e-8):
    """Replace each entry of x along ``axis`` by the sum over its degenerate group.

    ``vals`` holds the (ascending) energies that label ``axis`` and has shape
    x.shape[:axis + 1]; indices whose energies agree within ``tol`` form a
    group.  Gauge-invariant comparisons of |g|^2 use these group sums.
    """
    x = np.asarray(x)
    vals = np.asarray(vals)
    assert vals.shape == x.shape[:axis + 1], (vals.shape, x.shape, axis)
    out = x.copy()
    n = x.shape[axis]
    for lead in np.ndindex(*x.shape[:axis]):
        v = vals[lead]
        start = 0
        for i in range(1, n + 1):
            if i == n or abs(v[i] - v[i - 1]) > tol:
                sl = lead + (slice(start, i),)
                out[sl] = x[sl].sum(axis=0, keepdims=True)
                start = i
    return out


def assert_close_blocks(got, ref, tol, block_axes, floor=1e-3, label=""):
    """|got - ref| <= tol (|ref| + floor * max over the block of |ref|), plus normwise."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    bmax = np.abs(ref).max(axis=block_axes, keepdims=True)
    bound = tol * (np.abs(ref) + floor * bmax) + 1e-300
    err = np.abs(got - ref)
    worst = np.max(err / bound)
    assert worst <= 1.0, f"{label}: worst error / bound = {worst:.3g}"
    nrm = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
    assert nrm <= tol, f"{label}: normwise {nrm:.3g}"


def assert_rates_close(got, ref, tol, floor=1e-6, label=""):
    """Relative per state with a floor of floor * max(ref)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    bound = tol * (np.abs(ref) + floor * np.abs(ref).max())
    worst = np.max(np.abs(got - ref) / bound)
    assert worst <= 1.0, f"{label}: worst error / bound = {worst:.3g}"
