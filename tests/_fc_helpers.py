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
