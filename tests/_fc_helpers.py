"""Shared helpers of the GPU parity tests (oracle vs the CUDA path through the C ABI)."""

import numpy as np

import oracle as O

TOL = 1e-5  # FP32 path: |gpu - ref| <= TOL * max(1, |ref|)


def close(gpu, ref, tol=TOL):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    both_nan = np.isnan(gpu) & np.isnan(ref)
    err = np.abs(gpu - ref)
    ok = (err <= tol * np.maximum(1.0, np.abs(ref))) | both_nan
    return ok


def assert_close(gpu, ref, tol=TOL, what=""):
    ok = close(gpu, ref, tol)
    if not ok.all():
        g = np.asarray(gpu, np.float64)[~ok]
        r = np.asarray(ref, np.float64)[~ok]
        i = int(np.argmax(np.abs(g - r)))
        raise AssertionError(f"{what}: {int((~ok).sum())}/{ok.size} outside tol {tol}; worst gpu={g[i]!r} ref={r[i]!r}")


U32 = 2.0 ** -24
NONLIN_CHUNK = 36  # most trials per FP32 partial sum of the mixed-precision non-linear sums


def dswpli_mixed_tolerance(X, I, J):
    """Per-pair bound on |DSWPLI_gpu - DSWPLI_oracle| of the mixed-precision full window (band
    average), from its arithmetic. Its non-linear sums add Im, |Im| and Im^2 in FP32 over
    chunks of m = min(K, 36) trials before double-word window sums, so (sum Im)^2,
    (sum |Im|)^2 and sum Im^2 each carry at most ~m u (sum |Im|)^2 (u = 2^-24); each debiased
    difference is off by at most 3 m u (sum |Im|)^2 and the ratio (|DSWPLI| <= 1) by at most
    6 m u (sum |Im|)^2 / ((sum |Im|)^2 - sum Im^2) per bin: the conditioning, large where one
    term dominates a short window. X: the window's spectra [K][n][B]. Plus the 1e-5 of the
    other exact-term metrics."""
    sums = O.pair_sums_pairs(X, I, J)
    m = min(np.asarray(X).shape[0], NONLIN_CHUNK)
    den = sums["abs"] ** 2 - sums["sq"]
    with np.errstate(divide="ignore", invalid="ignore"):
        cond = np.where(den > 0, sums["abs"] ** 2 / np.where(den > 0, den, 1.0), 0.0)
    return 1e-5 + np.mean(6.0 * m * U32 * cond, axis=1)


def assert_close_bound(gpu, ref, bound, what=""):
    """|gpu - ref| <= max(1e-5 max(1, |ref|), bound) element by element (NaN matches NaN)."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(gpu - ref)
    ok = (err <= np.maximum(TOL * np.maximum(1.0, np.abs(ref)), bound)) | (np.isnan(gpu) & np.isnan(ref))
    if not ok.all():
        i = int(np.argmax(np.where(ok, 0.0, err)))
        raise AssertionError(f"{what}: {int((~ok).sum())}/{ok.size} outside the bound; "
                             f"worst gpu={gpu[i]!r} ref={ref[i]!r} bound={np.broadcast_to(bound, err.shape)[i]!r}")


def window_spectra(sess, K):
    """GPU spectra of the K trials in the window, oldest first: complex64 [K][n][B]."""
    out = [sess.spectra(age) for age in range(K)][::-1]  # each [B][n]
    return np.stack([o.T for o in out])


def packed_to_dense(v, n, antisym=False):
    d = np.zeros((n, n), np.float64)
    iu = np.triu_indices(n, 1)
    d[iu] = v
    d.T[iu] = -v if antisym else v
    return d


def upper(mat):
    n = mat.shape[0]
    return mat[np.triu_indices(n, 1)]


def packed_index(i, j, n):
    i = np.asarray(i, np.int64)
    j = np.asarray(j, np.int64)
    return i * n - i * (i + 1) // 2 + (j - i - 1)


def oracle_spectral(X, I=None, J=None):
    """Oracle networks from spectra X [K][n][B]: packed upper arrays (or the listed pairs)."""
    n = X.shape[1]
    if I is None:
        I, J = np.triu_indices(n, 1)
    return O.spectral_networks_pairs(X, I, J)
