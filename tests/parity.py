"""Comparison helpers shared by the GPU parity tests (no method arithmetic).

Spectra span many decades across k, so they are compared bin by bin: the
relative difference of every bin against the reference bin, not against the
largest bin."""
import numpy as np


def nrel(a, b):
    """Normwise relative difference: max |a - b| / max |b|."""
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def bin_rel(got, ref):
    """Largest per-bin relative difference |g - r| / |r|.  Bins where the
    reference is 0 must be exactly 0, and NaN bins (an undefined quantity, such
    as an occupation number with w^2 <= 0) must be NaN on both sides."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    nan_g, nan_r = np.isnan(got), np.isnan(ref)
    assert np.array_equal(nan_g, nan_r), "NaN bins differ"
    ok = ~nan_r
    g, r = got[ok], ref[ok]
    zero = r == 0.0
    assert np.all(g[zero] == 0.0), "bins that are 0 in the reference are not 0"
    if not np.any(~zero):
        return 0.0
    return float(np.max(np.abs(g[~zero] - r[~zero]) / np.abs(r[~zero])))


def assert_bins(got, ref, tol, what=""):
    e = bin_rel(got, ref)
    assert e <= tol, "%s: per-bin relative difference %.3g > %.3g" % (what, e, tol)
    return e
