"""Plain, slow, FP64 CPU oracle of the connectivity hot path.

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline / reference leg of ``bench.py`` use this module; the product path never
does. It shares no code with the CUDA library.

What it computes, in the paper's order (Esch et al., "Online functional
connectivity analysis of large all-to-all networks"):

1. per trial and node, the spectrum of the tapered trial (§2.4: "for each trial,
   the frequency spectrum, CSD and PSD are calculated"), here a direct DFT over
   the selected band bins;
2. per trial, PSD_x = A_x^2 and CSD_xy = x y* (Supplementary §1, Frequency Domain);
3. running sums of those over the trials of the window (§2.4, running average);
4. each metric from the sums (Supplementary §1: COHY, COH, IMAGCOHY, PLV, PLI,
   USPLI, WPLI, DSWPLI);
5. the band average over the selected bins (§3.2.3: bins averaged to form
   the edge weights);
6. the time-domain metrics COR and XCOR (Supplementary §1, Time Domain; §2.4
   describes XCOR via FFT convolution and returning the highest value and its
   index).

Readings where the paper is silent or garbled:
* COHY's printed second form repeats PSD_y; the first form (PSD_x, PSD_y) is used.
* DSWPLI is printed as WPLI^2; the debiased estimator of the cited Vinck et al.
  (2011) is used: ((sum Im)^2 - sum Im^2) / ((sum |Im|)^2 - sum Im^2).
* Taper: periodic Hann by default; spectra unnormalised (every metric is a
  scale-free ratio).
* Band: bins k with f_lo <= k fs / nfft < f_hi.
* sign(0) = 0; u = X/|X| is 0 where X = 0; a zero denominator gives 0;
  USPLI is NaN for K < 2; the diagonal is 0.
* XCOR: full-length energies in the denominator (the value stays in [-1, 1]),
  lags |tau| <= N-1, signed maximum, ties to the smallest |tau| then negative tau.
* COR / XCOR networks are the mean over trials of the per-trial values.
"""

from __future__ import annotations

import math

import numpy as np

SPECTRAL_METRICS = ("COH", "IMAGCOHY", "PLV", "PLI", "USPLI", "WPLI", "DSWPLI")
TIME_METRICS = ("COR", "XCOR")
ALL_METRICS = TIME_METRICS + SPECTRAL_METRICS
ANTISYMMETRIC = ("IMAGCOHY",)

__all__ = [
    "SPECTRAL_METRICS", "TIME_METRICS", "ALL_METRICS", "ANTISYMMETRIC",
    "band_bins", "taper", "spectra", "phasor", "sign_im",
    "pair_sums_dense", "pair_sums_pairs", "metrics_from_sums", "band_average",
    "spectral_networks_dense", "spectral_networks_pairs",
    "cor_trial", "cor_network", "xcor_trial_pair", "xcor_trial_dense", "xcor_network",
    "window_trials", "networks_dense", "network_top", "project", "fir_design", "fir_filter_stream",
]


# ---------------------------------------------------------------------------
# 1. Band and taper


def band_bins(fs: float, nfft: int, f_lo: float, f_hi: float) -> np.ndarray:
    """Bins k (0 <= k <= nfft/2) whose centre frequency k*fs/nfft lies in [f_lo, f_hi).

    The paper selects bins by frequency (§3.1: 8-12 Hz with 1 Hz bins; §3.2.3:
    bins 18 to 30). The half-open rule is the reading that reproduces the
    workloads' bin counts.
    """
    ks = [k for k in range(nfft // 2 + 1) if k * fs >= f_lo * nfft and k * fs < f_hi * nfft]
    return np.asarray(ks, dtype=np.int64)


def taper(n_samples: int, kind: str = "hann") -> np.ndarray:
    """Window applied before the DFT: 'hann' (periodic), 'hann_sym' or 'none'."""
    t = np.arange(n_samples, dtype=np.float64)
    if kind == "hann":
        return 0.5 - 0.5 * np.cos(2.0 * math.pi * t / n_samples)
    if kind == "hann_sym":
        if n_samples == 1:
            return np.ones(1)
        return 0.5 - 0.5 * np.cos(2.0 * math.pi * t / (n_samples - 1))
    if kind == "none":
        return np.ones(n_samples)
    raise ValueError(kind)


# ---------------------------------------------------------------------------
# 2. Spectra (§2.4: frequency spectrum per trial)


def spectra(x: np.ndarray, bins: np.ndarray, nfft: int, taper_kind: str = "hann") -> np.ndarray:
    """Band spectrum X(f) = sum_{t<N} x(t) w(t) exp(-2 pi i f t / nfft), f in ``bins``.

    x: [..., N] real. Returns complex128 [..., B]. The trial is zero-padded to
    nfft (N <= nfft), so only t < N contributes. The angle is reduced exactly
    with the integer (f * t) mod nfft before the cosine/sine.
    """
    x = np.asarray(x, dtype=np.float64)
    n_samples = x.shape[-1]
    if n_samples > nfft:
        raise ValueError("n_samples must not exceed nfft")
    t = np.arange(n_samples, dtype=np.int64)
    m = np.outer(t, np.asarray(bins, dtype=np.int64)) % nfft
    ang = 2.0 * math.pi * m.astype(np.float64) / nfft
    E = np.cos(ang) - 1j * np.sin(ang)  # [N][B]
    xw = x * taper(n_samples, taper_kind)
    return xw @ E


def phasor(X: np.ndarray) -> np.ndarray:
    """u = X / |X| (the unit phase factor e^{i Phi} used by PLV), 0 where X = 0."""
    X = np.asarray(X, dtype=np.complex128)
    mag = np.abs(X)
    out = np.zeros_like(X)
    nz = mag > 0
    out[nz] = X[nz] / mag[nz]
    return out


def _re_im(X):
    X = np.asarray(X)
    if X.dtype == np.complex64:
        X = X.astype(np.complex128)  # exact widening
    return X.real.astype(np.float64), X.imag.astype(np.float64)


def sign_im(ai, bi, aj, bj):
    """sign(Im(X_i X_j*)) with Im = b_i a_j - a_i b_j evaluated in FP64.

    For FP32 inputs both products are exact in FP64 and the difference is a
    single correctly rounded operation, so the sign is exact.
    """
    return np.sign(bi * aj - ai * bj).astype(np.int64)


# ---------------------------------------------------------------------------
# 3. Running sums over trials (§2.4), per ordered pair and bin


def pair_sums_dense(X: np.ndarray) -> dict:
    """Sums over the K trials of X [K][n][B] for every ordered node pair.

    Returns arrays [B][n][n] (csd complex, u complex, sign int64, im, abs, sq)
    and psd [B][n]:
      csd  = sum_k X_i X_j*            (CSD_xy = x y*; Re = a_i a_j + b_i b_j, Im = Im_k)
      psd  = sum_k |X_i|^2             (PSD_x = A_x^2 = a^2 + b^2)
      u    = sum_k u_i u_j*            (u = X/|X|, PLV)
      sign = sum_k sign(Im_k),  im = sum_k Im_k,  abs = sum_k |Im_k|,  sq = sum_k Im_k^2
    with Im_k = Im(X_i X_j*) = b_i a_j - a_i b_j.
    """
    X = np.asarray(X)
    K, n, B = X.shape
    A, Bm = _re_im(X)
    Xc = A + 1j * Bm
    U = phasor(Xc)
    out = {
        "csd": np.empty((B, n, n), np.complex128),
        "u": np.empty((B, n, n), np.complex128),
        "sign": np.zeros((B, n, n), np.int64),
        "im": np.zeros((B, n, n)),
        "abs": np.zeros((B, n, n)),
        "sq": np.zeros((B, n, n)),
        "psd": np.empty((B, n)),
        "K": K,
    }
    for b in range(B):
        Ub = U[:, :, b]
        Ab, Bb = A[:, :, b], Bm[:, :, b]
        out["u"][b] = Ub.T @ np.conj(Ub)
        out["psd"][b] = np.sum(Ab * Ab + Bb * Bb, axis=0)
        for k in range(K):
            a, bb = A[k, :, b], Bm[k, :, b]
            im = np.outer(bb, a) - np.outer(a, bb)  # [i][j] = b_i a_j - a_i b_j
            out["sign"][b] += np.sign(im).astype(np.int64)
            out["im"][b] += im
            out["abs"][b] += np.abs(im)
            out["sq"][b] += im * im
        # Re CSD = sum (a_i a_j + b_i b_j); Im CSD is the same Im_k sum as above
        out["csd"][b] = (Ab.T @ Ab + Bb.T @ Bb) + 1j * out["im"][b]
    return out


def pair_sums_pairs(X: np.ndarray, I, J) -> dict:
    """Same sums as :func:`pair_sums_dense`, only for the listed pairs (I[p], J[p]).

    Returns arrays [P][B] plus psd_i, psd_j [P][B].
    """
    X = np.asarray(X)
    I = np.asarray(I, dtype=np.int64)
    J = np.asarray(J, dtype=np.int64)
    A, Bm = _re_im(X)
    ai, bi = A[:, I, :], Bm[:, I, :]
    aj, bj = A[:, J, :], Bm[:, J, :]
    Ui, Uj = phasor(ai + 1j * bi), phasor(aj + 1j * bj)
    im = bi * aj - ai * bj
    im_sum = np.sum(im, axis=0)
    return {
        "csd": np.sum(ai * aj + bi * bj, axis=0) + 1j * im_sum,
        "u": np.sum(Ui * np.conj(Uj), axis=0),
        "sign": np.sum(np.sign(im).astype(np.int64), axis=0),
        "im": im_sum,
        "abs": np.sum(np.abs(im), axis=0),
        "sq": np.sum(im * im, axis=0),
        "psd_i": np.sum(ai * ai + bi * bi, axis=0),
        "psd_j": np.sum(aj * aj + bj * bj, axis=0),
        "K": X.shape[0],
    }


# ---------------------------------------------------------------------------
# 4. Metrics from the sums (Supplementary §1, Frequency Domain)


def metrics_from_sums(csd, psd_i, psd_j, u, sign, im, abs_, sq, K: int) -> dict:
    """Per-bin metrics from trial sums (all arrays broadcast together).

    COHY     = (1/K sum CSD) / sqrt((1/K sum PSD_x)(1/K sum PSD_y))  (the 1/K cancel)
    COH      = |COHY|
    IMAGCOHY = Im(COHY)
    PLV      = |1/K sum u_x u_y*|
    PLI      = |1/K sum sign(Im CSD)|
    USPLI    = (K PLI^2 - 1)/(K - 1) = (S_sign^2 - K) / (K (K - 1))
    WPLI     = |1/K sum Im CSD| / (1/K sum |Im CSD|)
    DSWPLI   = ((sum Im)^2 - sum Im^2) / ((sum |Im|)^2 - sum Im^2)
    """
    den = np.sqrt(np.asarray(psd_i, np.float64) * np.asarray(psd_j, np.float64))
    with np.errstate(divide="ignore", invalid="ignore"):
        cohy = np.where(den > 0, csd / np.where(den > 0, den, 1.0), 0.0)
        s = np.asarray(sign, np.float64)
        if K >= 2:
            uspli = (s * s - K) / (K * (K - 1.0))
        else:
            uspli = np.full(np.shape(s), np.nan)
        wpli = np.where(abs_ > 0, np.abs(im) / np.where(abs_ > 0, abs_, 1.0), 0.0)
        dnum = im * im - sq
        dden = abs_ * abs_ - sq
        dswpli = np.where(dden != 0, dnum / np.where(dden != 0, dden, 1.0), 0.0)
    return {
        "COHY": cohy,
        "COH": np.abs(cohy),
        "IMAGCOHY": np.imag(cohy),
        "PLV": np.abs(u) / K,
        "PLI": np.abs(s) / K,
        "USPLI": uspli,
        "WPLI": wpli,
        "DSWPLI": dswpli,
    }


def band_average(per_bin: np.ndarray, axis: int) -> np.ndarray:
    """Mean of a per-bin metric over the selected bins (§3.2.3, §3.2.1)."""
    return np.mean(per_bin, axis=axis)


def spectral_networks_dense(X: np.ndarray, per_bin: bool = False) -> dict:
    """All spectral metrics for every ordered pair of X [K][n][B].

    Returns metric -> [n][n] band-averaged network (diagonal 0), or with
    ``per_bin`` metric -> [B][n][n].
    """
    s = pair_sums_dense(X)
    K = s["K"]
    psd = s["psd"]
    m = metrics_from_sums(s["csd"], psd[:, :, None], psd[:, None, :], s["u"], s["sign"],
                          s["im"], s["abs"], s["sq"], K)
    n = X.shape[1]
    out = {}
    for name in SPECTRAL_METRICS:
        v = m[name]
        if not per_bin:
            v = band_average(v, axis=0)
            v = v.copy()
            v[np.arange(n), np.arange(n)] = 0.0
        out[name] = v
    if per_bin:
        out["COHY"] = m["COHY"]
    return out


def spectral_networks_pairs(X: np.ndarray, I, J, per_bin: bool = False) -> dict:
    """Spectral metrics for the listed pairs only: metric -> [P] (or [P][B])."""
    s = pair_sums_pairs(X, I, J)
    m = metrics_from_sums(s["csd"], s["psd_i"], s["psd_j"], s["u"], s["sign"],
                          s["im"], s["abs"], s["sq"], s["K"])
    return {k: (m[k] if per_bin else band_average(m[k], axis=-1)) for k in SPECTRAL_METRICS}


# ---------------------------------------------------------------------------
# 6. Time-domain metrics (Supplementary §1, Time Domain; §2.4)


def cor_trial(x: np.ndarray) -> np.ndarray:
    """Pearson correlation COR_xy for all node pairs of one trial x [n][N] (diag 0).

    COR_xy = sum (x - xbar)(y - ybar) / sqrt(sum (x - xbar)^2 sum (y - ybar)^2);
    a zero-variance node gives 0.
    """
    x = np.asarray(x, np.float64)
    d = x - x.mean(axis=1, keepdims=True)
    nrm = np.sqrt(np.sum(d * d, axis=1))
    z = np.zeros_like(d)
    nz = nrm > 0
    z[nz] = d[nz] / nrm[nz, None]
    c = z @ z.T
    np.fill_diagonal(c, 0.0)
    return c


def cor_network(x: np.ndarray) -> np.ndarray:
    """COR network: mean over trials of the per-trial correlation, x [K][n][N]."""
    return np.mean([cor_trial(xk) for xk in np.asarray(x)], axis=0)


def _lag_order(n_samples: int) -> np.ndarray:
    """Lags 0, -1, +1, -2, +2, ... so that a first-max search applies the tie rule."""
    out = [0]
    for m in range(1, n_samples):
        out += [-m, m]
    return np.asarray(out, dtype=np.int64)


def xcor_trial_pair(xi: np.ndarray, xj: np.ndarray):
    """Normalised cross-correlation of one node pair in one trial, by direct sums.

    R(tau) = sum_t (x_i(t+tau) - xbar_i)(x_j(t) - xbar_j) over the overlapping t,
    |tau| <= N-1; value = max_tau R(tau) / sqrt(E_i E_j) with the full-length
    energies E = sum (x - xbar)^2. Returns (value, tau); (0, 0) if E_i E_j = 0.
    """
    xi = np.asarray(xi, np.float64) - np.mean(xi, dtype=np.float64)
    xj = np.asarray(xj, np.float64) - np.mean(xj, dtype=np.float64)
    N = xi.shape[0]
    e = math.sqrt(float(np.dot(xi, xi)) * float(np.dot(xj, xj)))
    if e == 0.0:
        return 0.0, 0
    best, best_tau = -math.inf, 0
    for tau in _lag_order(N):
        if tau >= 0:
            r = float(np.dot(xi[tau:], xj[: N - tau]))
        else:
            r = float(np.dot(xi[: N + tau], xj[-tau:]))
        if r / e > best:
            best, best_tau = r / e, int(tau)
    return best, best_tau


def xcor_trial_dense(x: np.ndarray):
    """XCOR of every ordered pair of one trial x [n][N] via FFT convolution (§2.4).

    Spectra of the mean-removed, zero-padded signals (length L = next power of
    two >= 2N-1) are multiplied as Z_i Z_j*, transformed back to the lag domain,
    and the largest normalised value and its lag are taken.
    Returns (value [n][n] with diag 0, lag [n][n]).
    """
    x = np.asarray(x, np.float64)
    n, N = x.shape
    d = x - x.mean(axis=1, keepdims=True)
    E = np.sum(d * d, axis=1)
    L = 1
    while L < 2 * N - 1:
        L *= 2
    Z = np.fft.rfft(d, n=L, axis=1)
    order = _lag_order(N)
    idx = order % L
    val = np.zeros((n, n))
    lag = np.zeros((n, n), np.int64)
    for i in range(n):
        R = np.fft.irfft(Z[i][None, :] * np.conj(Z), n=L, axis=1)  # [j][m]
        Ro = R[:, idx]
        a = np.argmax(Ro, axis=1)
        den = np.sqrt(E[i] * E)
        v = Ro[np.arange(n), a]
        ok = den > 0
        val[i, ok] = v[ok] / den[ok]
        lag[i, ok] = order[a[ok]]
    np.fill_diagonal(val, 0.0)
    np.fill_diagonal(lag, 0)
    return val, lag


def xcor_network(x: np.ndarray):
    """XCOR network: mean over trials of the per-trial maxima; also per-trial lags."""
    vals, lags = zip(*(xcor_trial_dense(xk) for xk in np.asarray(x)))
    return np.mean(vals, axis=0), np.stack(lags)


# ---------------------------------------------------------------------------
# Windows (§2.5: each new trial is added; the user sets the number of trials)


def window_trials(n_pushed: int, window: int) -> range:
    """0-based indices of the trials in the window after ``n_pushed`` pushes.

    window = 0 keeps every trial (cumulative); window = W > 0 keeps the last W.
    """
    if window <= 0:
        return range(0, n_pushed)
    return range(max(0, n_pushed - window), n_pushed)


def networks_dense(x: np.ndarray, fs: float, nfft: int, f_lo: float, f_hi: float,
                   taper_kind: str = "hann", metrics=ALL_METRICS) -> dict:
    """Full pipeline for raw trials x [K][n][N]: every requested metric's network."""
    bins = band_bins(fs, nfft, f_lo, f_hi)
    out = {}
    if any(m in SPECTRAL_METRICS for m in metrics):
        X = spectra(x, bins, nfft, taper_kind)
        out.update({k: v for k, v in spectral_networks_dense(X).items() if k in metrics})
    if "COR" in metrics:
        out["COR"] = cor_network(x)
    if "XCOR" in metrics:
        out["XCOR"], out["XCOR_LAG"] = xcor_network(x)
    return out


# ---------------------------------------------------------------------------
# Network post-processing (the paper's display pipeline)


def network_top(w_packed, n: int, percent: float):
    """Normalize a network by its maximum edge weight, keep its strongest ``percent`` % of
    edges and give the kept network's node degree and node strength.

    §3.1.2 and §3.2.2: every network is normalized by its maximum edge weight; §3.2.2,
    §3.2.3 and the figure captions: only the strongest 5 %, 10 % or 25 % of the edges are
    shown; §1: node degree and node strength are the graph measures drawn.

    Readings: maximum and strength are taken by magnitude |w| (IMAGCOHY is signed); the
    number of edges kept is ceil(percent * P / 100); among equal magnitudes the lower packed
    index is kept first; a NaN edge (USPLI with fewer than two trials) counts as 0; node
    strength is the sum of the kept normalized magnitudes. The edge ranking uses the
    magnitudes of the given (FP32) weights exactly.

    Returns (weights [P]: normalized kept weights, 0 elsewhere; degree [n] int64;
    strength [n]; max_abs; kept).
    """
    w = np.asarray(w_packed, np.float64).copy()
    P = n * (n - 1) // 2
    assert w.shape == (P,)
    w[np.isnan(w)] = 0.0
    mag = np.abs(w)
    max_abs = float(mag.max()) if P else 0.0
    kept = min(P, max(0, int(math.ceil(percent * P / 100.0))))
    order = np.lexsort((np.arange(P), -mag))  # by magnitude descending, then index
    keep = np.zeros(P, bool)
    keep[order[:kept]] = True
    out = np.zeros(P)
    if max_abs > 0:
        out[keep] = w[keep] / max_abs
    I, J = np.triu_indices(n, 1)
    degree = np.zeros(n, np.int64)
    strength = np.zeros(n)
    for e in np.nonzero(keep)[0]:
        for node in (I[e], J[e]):
            degree[node] += 1
            strength[node] += abs(out[e])
    return out, degree, strength, max_abs, kept


# ---------------------------------------------------------------------------
# Source projection ahead of the spectrum


def project(op, x):
    """Source trials from sensor trials: y_k = M x_k for every trial k.

    §2.5 / Figure 1: in the source-level pipeline each trial is mapped to the source
    space (RTC-MNE) before the connectivity step; the inverse operator M is a
    [n_sources][n_channels] matrix applied to the [n_channels][n_samples] trial. A matmul
    is the library step here.
    """
    M = np.asarray(op, np.float64)
    X = np.asarray(x, np.float64)
    if X.ndim == 2:
        return M @ X
    return np.stack([M @ xk for xk in X])


# ---------------------------------------------------------------------------
# FIR filtering of the incoming stream (upstream of the connectivity path)


def fir_design(fs: float, kind: str, f_lo: float, f_hi: float, transition_hz: float, n_taps: int = 0):
    """Linear-phase FIR taps by the window method with a Hamming window.

    §2.4 (Noise Reduction plug-in): FIR low-, high- and band-pass filters are designed
    on the fly from the cut-off frequencies, the transition bandwidth and the number of
    taps; every filter has a linear phase. Here: odd length T (from the transition width,
    T ~ 3.3 fs / transition for a Hamming window, when n_taps is 0), centre m = (T - 1) / 2,
    ideal responses as differences of sinc low-passes, times the Hamming window
    w[k] = 0.54 - 0.46 cos(2 pi k / (T - 1)), unscaled.
    """
    if n_taps <= 0:
        n_taps = int(math.ceil(3.3 * fs / transition_hz))
    if n_taps % 2 == 0:
        n_taps += 1
    m = (n_taps - 1) / 2.0
    k = np.arange(n_taps, dtype=np.float64)

    def lowpass(fc):  # ideal low-pass with cut-off fc (Hz), sampled at k - m
        return 2.0 * fc / fs * np.sinc(2.0 * fc / fs * (k - m))

    if kind == "lowpass":
        h = lowpass(f_hi)
    elif kind == "highpass":
        h = -lowpass(f_lo)
        h[int(m)] += 1.0
    elif kind == "bandpass":
        h = lowpass(f_hi) - lowpass(f_lo)
    else:
        raise ValueError(kind)
    w = 0.54 - 0.46 * np.cos(2.0 * np.pi * k / (n_taps - 1)) if n_taps > 1 else np.ones(1)
    return h * w


def fir_filter_stream(h, blocks):
    """Causal FIR filtering of a multichannel stream delivered in blocks.

    §2.4: the filter runs as an FFT convolution on blocks, and overlap-add carries the
    convolution tail across block boundaries, so the output is the filtered continuous
    stream: y[c, t] = sum_k h[k] x[c, t - k] with x = 0 before the first sample. Written
    here as the convolution of the concatenated stream (a library step), then cut back into
    the blocks.
    """
    h = np.asarray(h, np.float64)
    x = np.concatenate([np.asarray(b, np.float64) for b in blocks], axis=1)
    y = np.stack([np.convolve(xc, h)[: x.shape[1]] for xc in x])
    out, o = [], 0
    for b in blocks:
        L = np.asarray(b).shape[1]
        out.append(y[:, o:o + L])
        o += L
    return out
