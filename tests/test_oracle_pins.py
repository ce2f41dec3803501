"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a library
routine (numpy FFT, corrcoef, correlate), a closed form, an identity, a
hand-derived example (tests/golden/), exact rational arithmetic, brute-force
loops, or a known sampling distribution.
"""

import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from synth import eeg_sinusoid_trials

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- band, taper


def test_band_bins_workloads():
    # bin counts of the paper-shaped workloads (half-open Hz rule)
    assert list(O.band_bins(1000.0, 512, 1.0, 50.0)) == list(range(1, 26))
    assert list(O.band_bins(1000.0, 1024, 1.0, 100.0)) == list(range(2, 103))
    assert list(O.band_bins(1000.0, 1000, 4.0, 44.0)) == list(range(4, 44))
    # §3.1 timing setup: fs = nfft = 600, 8-12 Hz -> 4 bins
    assert list(O.band_bins(600.0, 600, 8.0, 12.0)) == [8, 9, 10, 11]


def test_taper_closed_forms():
    w = O.taper(64, "hann")
    assert w[0] == 0.0 and abs(w.sum() - 32.0) < 1e-12  # periodic Hann sums to N/2
    ws = O.taper(65, "hann_sym")
    assert ws[0] == 0.0 and abs(ws[-1]) < 1e-15 and abs(ws[32] - 1.0) < 1e-15
    assert np.all(O.taper(7, "none") == 1.0)


# ---------------------------------------------------------------- spectra


@pytest.mark.parametrize("taper_kind", ["none", "hann", "hann_sym"])
def test_spectra_match_numpy_rfft(taper_kind):
    rng = np.random.default_rng(1)
    N, nfft = 37, 64
    x = rng.standard_normal((3, 5, N))
    bins = np.arange(nfft // 2 + 1)
    X = O.spectra(x, bins, nfft, taper_kind)
    ref = np.fft.rfft(x * O.taper(N, taper_kind), n=nfft, axis=-1)
    assert np.max(np.abs(X - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_parseval():
    rng = np.random.default_rng(2)
    N = 48
    x = rng.standard_normal(N)
    X = O.spectra(x, np.arange(N // 2 + 1), N, "none")
    p = np.abs(X) ** 2
    energy = (p[0] + 2 * p[1:N // 2].sum() + p[N // 2]) / N
    assert abs(energy - np.dot(x, x)) < 1e-10 * np.dot(x, x)


def test_hann_tone_closed_form():
    # cos(2 pi f0 t / N) under a periodic Hann: X(f0) = N/4, X(f0 +- 1) = -N/8, else 0
    N, f0 = 64, 9
    t = np.arange(N)
    x = np.cos(2 * math.pi * f0 * t / N)
    X = O.spectra(x, np.arange(N // 2 + 1), N, "hann")
    expect = np.zeros(N // 2 + 1)
    expect[f0] = N / 4
    expect[f0 - 1] = expect[f0 + 1] = -N / 8
    assert np.max(np.abs(X - expect)) < 1e-12


# ---------------------------------------------------------------- metrics


def test_golden_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "worked_example_2x2.json")))
    X = np.asarray(g["spectra_re"]) + 1j * np.asarray(g["spectra_im"])  # [K][n][B]
    s = O.pair_sums_pairs(X, [0], [1])
    e = g["expected_sums_ij"]
    assert s["csd"][0, 0] == complex(e["csd_re"], e["csd_im"])
    assert s["psd_i"][0, 0] == e["psd_i"] and s["psd_j"][0, 0] == e["psd_j"]
    for k in ("sign", "im", "abs", "sq"):
        assert s[k][0, 0] == e[k], k
    m = O.spectral_networks_pairs(X, [0, 1], [1, 0])
    for name, v in g["expected_ij"].items():
        assert abs(m[name][0] - v) < 1e-14, name
        expect_ji = -v if name == "IMAGCOHY" else v
        assert abs(m[name][1] - expect_ji) < 1e-14, name
    dense = O.spectral_networks_dense(X)
    for name, v in g["expected_ij"].items():
        assert abs(dense[name][0, 1] - v) < 1e-14, name


def _rand_spectra(seed, K, n, B):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((K, n, B)) + 1j * rng.standard_normal((K, n, B))


def test_identical_channels():
    X = _rand_spectra(3, 12, 6, 5)
    X[:, 4, :] = X[:, 1, :]
    m = O.spectral_networks_pairs(X, [1], [4])
    assert abs(m["COH"][0] - 1) < 1e-12 and abs(m["PLV"][0] - 1) < 1e-12
    assert m["PLI"][0] == 0.0 and m["IMAGCOHY"][0] == 0.0 and m["WPLI"][0] == 0.0
    assert m["DSWPLI"][0] == 0.0  # 0/0 -> 0 reading
    K = X.shape[0]
    assert abs(m["USPLI"][0] - (-1.0 / (K - 1))) < 1e-15


@pytest.mark.parametrize("phi", [0.3, math.pi / 2, 2.5])
def test_phase_lag_sinusoids(phi):
    # x = sin(w t + th_k), y = sin(w t + th_k - phi): COHY = e^{i phi} in f0-1..f0+1
    N, f0, K = 128, 12, 9
    rng = np.random.default_rng(4)
    t = np.arange(N)
    th = rng.uniform(0, 2 * math.pi, K)
    x = np.stack([np.stack([np.sin(2 * math.pi * f0 * t / N + a),
                            np.sin(2 * math.pi * f0 * t / N + a - phi)]) for a in th])
    X = O.spectra(x, np.array([f0 - 1, f0, f0 + 1]), N, "hann")
    m = O.spectral_networks_pairs(X, [0], [1])
    for name in ("COH", "PLV", "PLI", "WPLI", "USPLI", "DSWPLI"):
        assert abs(m[name][0] - 1.0) < 1e-9, name
    assert abs(m["IMAGCOHY"][0] - math.sin(phi)) < 1e-9


def test_dense_and_pairwise_agree_and_symmetry():
    X = _rand_spectra(5, 7, 9, 4)
    dense = O.spectral_networks_dense(X, per_bin=True)
    I, J = np.meshgrid(np.arange(9), np.arange(9), indexing="ij")
    I, J = I.ravel(), J.ravel()
    off = I != J
    pw = O.spectral_networks_pairs(X, I[off], J[off], per_bin=True)
    for name in O.SPECTRAL_METRICS:
        d = dense[name][:, I[off], J[off]].T  # [P][B]
        assert np.max(np.abs(d - pw[name])) < 1e-12, name
    cohy = dense["COHY"]
    assert np.max(np.abs(cohy - np.conj(np.transpose(cohy, (0, 2, 1))))) < 1e-12
    net = O.spectral_networks_dense(X)
    for name in O.SPECTRAL_METRICS:
        sgn = -1.0 if name in O.ANTISYMMETRIC else 1.0
        assert np.max(np.abs(net[name] - sgn * net[name].T)) < 1e-12, name
        assert np.all(np.diag(net[name]) == 0)


def test_debiased_estimators_by_pair_loops():
    # USPLI and DSWPLI equal the explicit sums over trial pairs j != k
    for seed, K in [(6, 2), (7, 3), (8, 5), (9, 6)]:
        X = _rand_spectra(seed, K, 2, 3)
        m = O.spectral_networks_pairs(X, [0], [1], per_bin=True)
        for b in range(3):
            im = [(X[k, 0, b] * np.conj(X[k, 1, b])).imag for k in range(K)]
            s = [float(np.sign(v)) for v in im]
            num_s = sum(s[a] * s[c] for a in range(K) for c in range(K) if a != c)
            assert abs(m["USPLI"][0, b] - num_s / (K * (K - 1))) < 1e-12
            num = sum(im[a] * im[c] for a in range(K) for c in range(K) if a != c)
            den = sum(abs(im[a]) * abs(im[c]) for a in range(K) for c in range(K) if a != c)
            assert abs(m["DSWPLI"][0, b] - num / den) < 1e-12
            # direct loops for PLI, WPLI, PLV, COH as printed
            assert abs(m["PLI"][0, b] - abs(sum(s)) / K) < 1e-15
            assert abs(m["WPLI"][0, b] - abs(sum(im) / K) / (sum(abs(v) for v in im) / K)) < 1e-12
            ph = sum(np.exp(1j * (np.angle(X[k, 0, b]) - np.angle(X[k, 1, b]))) for k in range(K))
            assert abs(m["PLV"][0, b] - abs(ph) / K) < 1e-12
            csd = sum(X[k, 0, b] * np.conj(X[k, 1, b]) for k in range(K)) / K
            pi = sum(abs(X[k, 0, b]) ** 2 for k in range(K)) / K
            pj = sum(abs(X[k, 1, b]) ** 2 for k in range(K)) / K
            assert abs(m["COH"][0, b] - abs(csd) / math.sqrt(pi * pj)) < 1e-12
            assert abs(m["IMAGCOHY"][0, b] - (csd / math.sqrt(pi * pj)).imag) < 1e-12


def test_null_hypothesis_bias():
    # independent complex Gaussian spectra: E[COH^2] = E[PLV^2] = E[PLI^2] = 1/K, E[USPLI] = 0
    K, n, B = 10, 400, 25
    X = _rand_spectra(10, K, n, B)
    I = np.arange(0, n, 2)
    J = I + 1  # disjoint pairs -> independent samples
    m = O.spectral_networks_pairs(X, I, J, per_bin=True)
    ns = m["COH"].size
    coh2 = (m["COH"] ** 2).ravel()
    var_beta = (K - 1) / (K * K * (K + 1.0))  # MSC ~ Beta(1, K-1)
    assert abs(coh2.mean() - 1.0 / K) < 4 * math.sqrt(var_beta / ns)
    for name in ("PLV", "PLI"):
        v = (m[name] ** 2).ravel()
        assert abs(v.mean() - 1.0 / K) < 4 * v.std() / math.sqrt(ns), name
    us = m["USPLI"].ravel()
    assert abs(us.mean()) < 4 * us.std() / math.sqrt(ns)


def test_zero_spectrum_conventions():
    X = _rand_spectra(11, 4, 3, 2)
    X[:, 2, :] = 0
    m = O.spectral_networks_pairs(X, [0], [2], per_bin=True)
    for name in ("COH", "IMAGCOHY", "PLV", "PLI", "WPLI", "DSWPLI"):
        assert np.all(m[name] == 0.0), name
    m1 = O.spectral_networks_pairs(X[:1], [0], [1], per_bin=True)
    assert np.all(np.isnan(m1["USPLI"]))  # K = 1


def test_sign_exact_against_rationals():
    rng = np.random.default_rng(12)
    a = rng.standard_normal((4, 4000)).astype(np.float32)
    # plant near-ties: b_i a_j == a_i b_j up to one ulp
    a[3, :2000] = (a[0, :2000].astype(np.float64) * a[2, :2000] / a[1, :2000]).astype(np.float32)
    a[3, 2000:2100] = np.nextafter(a[3, 2000:2100], np.float32(np.inf))
    ai, bi, aj, bj = (a[k].astype(np.float64) for k in range(4))
    # Im = b_i a_j - a_i b_j, with (ai, bi, aj, bj) = rows (0, 1, 2, 3)
    got = O.sign_im(ai, bi, aj, bj)
    for p in range(a.shape[1]):
        exact = Fraction(float(bi[p])) * Fraction(float(aj[p])) - Fraction(float(ai[p])) * Fraction(float(bj[p]))
        assert got[p] == (exact > 0) - (exact < 0)


# ---------------------------------------------------------------- time domain


def test_cor_matches_corrcoef():
    rng = np.random.default_rng(13)
    x = rng.standard_normal((6, 50))
    c = O.cor_trial(x)
    ref = np.corrcoef(x)
    np.fill_diagonal(ref, 0)
    assert np.max(np.abs(c - ref)) < 1e-13


def test_xcor_fft_matches_direct_sums_and_correlate():
    rng = np.random.default_rng(14)
    x = rng.standard_normal((4, 33))
    val, lag = O.xcor_trial_dense(x)
    for i in range(4):
        for j in range(4):
            if i == j:
                continue
            v, tau = O.xcor_trial_pair(x[i], x[j])
            assert abs(val[i, j] - v) < 1e-12 and lag[i, j] == tau
            di, dj = x[i] - x[i].mean(), x[j] - x[j].mean()
            c = np.correlate(di, dj, "full")  # index k <-> lag k - (N - 1)
            k = int(np.argmax(c))
            assert k - 32 == tau
            assert abs(c[k] / math.sqrt(np.dot(di, di) * np.dot(dj, dj)) - v) < 1e-12
    # symmetry: same value, negated lag
    assert np.max(np.abs(val - val.T)) < 1e-12
    assert np.all(lag == -lag.T)



@pytest.mark.parametrize("N", [2049, 4097, 8192])
def test_xcor_fft_matches_correlate_at_long_trials(N):
    """The FFT form at the longest trials XCOR sessions take (transforms of 4096 to 16384
    points): value and lag of every ordered pair against numpy's direct correlation."""
    rng = np.random.default_rng(N)
    x = rng.standard_normal((3, N))
    x[1] = np.roll(x[0], 11) + 0.3 * x[1]
    val, lag = O.xcor_trial_dense(x)
    for i in range(3):
        for j in range(3):
            if i == j:
                continue
            di, dj = x[i] - x[i].mean(), x[j] - x[j].mean()
            c = np.correlate(di, dj, "full")  # index k <-> lag k - (N - 1)
            k = int(np.argmax(c))
            assert lag[i, j] == k - (N - 1)
            assert abs(c[k] / math.sqrt(np.dot(di, di) * np.dot(dj, dj)) - val[i, j]) < 1e-10
    assert abs(lag[1, 0]) == 11 and val[1, 0] > 0.9

def test_xcor_recovers_shift():
    rng = np.random.default_rng(15)
    s = rng.standard_normal(300)
    d = 7
    xi, xj = s[d:d + 200], s[:200]  # x_i(t) = s(t + d), x_j(t) = s(t)
    v, tau = O.xcor_trial_pair(xi, xj)
    assert tau == -d and v > 0.9


def test_window_trials():
    assert list(O.window_trials(3, 0)) == [0, 1, 2]
    assert list(O.window_trials(3, 5)) == [0, 1, 2]
    assert list(O.window_trials(9, 4)) == [5, 6, 7, 8]


def test_eeg_workload_planted_couplings_visible():
    # at the 10 Hz bin the coupled pairs stand out in COH, and the pi/2 pairs in IMAGCOHY
    x, pairs = eeg_sinusoid_trials(21)
    nets = O.networks_dense(x, 1000.0, 512, 9.0, 11.0, metrics=("COH", "IMAGCOHY", "PLV"))
    coh = nets["COH"]
    off = coh[~np.eye(60, dtype=bool)]
    for a, b, lag in pairs:
        assert coh[a, b] > np.percentile(off, 99)
        if abs(lag - math.pi / 2) < 1e-9:
            assert abs(nets["IMAGCOHY"][a, b]) > np.percentile(np.abs(nets["IMAGCOHY"]), 99)


# ------------------------------------------------------------ network post-processing


def test_network_top_golden_example_with_a_tie():
    g = json.load(open(os.path.join(GOLDEN, "network_top_4nodes.json")))
    w = np.array([np.nan if v == "nan" else v for v in g["weights"]], np.float64)
    out, deg, stren, mx, kept = O.network_top(w, g["n_nodes"], g["percent"])
    assert kept == g["expected_kept"] and mx == pytest.approx(g["expected_max_abs"])
    np.testing.assert_allclose(out, g["expected_weights"], rtol=0, atol=1e-15)
    assert deg.tolist() == g["expected_degree"]
    np.testing.assert_allclose(stren, g["expected_strength"], rtol=0, atol=1e-15)


@pytest.mark.parametrize("n,percent", [(30, 5.0), (41, 10.0), (17, 25.0), (9, 0.0)])
def test_network_top_invariants(n, percent):
    rng = np.random.default_rng(n)
    w = rng.standard_normal(n * (n - 1) // 2).astype(np.float32)
    out, deg, stren, mx, kept = O.network_top(w, n, percent)
    P = w.size
    assert kept == math.ceil(percent * P / 100)
    keep = out != 0
    assert keep.sum() == kept and deg.sum() == 2 * kept
    if kept:
        assert np.abs(w[keep]).min() >= np.abs(w[~keep]).max()  # strongest edges kept
        assert np.abs(out).max() == 1.0
        np.testing.assert_allclose(out[keep], w[keep] / np.abs(w).max())
    np.testing.assert_allclose(stren.sum(), 2 * np.abs(out).sum())


def test_network_top_everything_kept_gives_dense_row_sums():
    n = 23
    rng = np.random.default_rng(5)
    w = rng.uniform(-1, 1, n * (n - 1) // 2)
    out, deg, stren, mx, kept = O.network_top(w, n, 100.0)
    dense = np.zeros((n, n))
    dense[np.triu_indices(n, 1)] = np.abs(w)
    dense = dense + dense.T
    assert (deg == n - 1).all()
    np.testing.assert_allclose(stren, dense.sum(axis=1) / np.abs(w).max(), rtol=1e-13)


def test_network_top_equal_weights_keep_lowest_indices():
    n = 10
    w = np.full(n * (n - 1) // 2, 0.25)
    out, deg, stren, mx, kept = O.network_top(w, n, 20.0)
    assert kept == 9 and (out[:9] == 1.0).all() and (out[9:] == 0).all()
    assert deg[0] == 9 and (deg[1:] == 1).all()  # pairs (0, 1) .. (0, 9)


# ------------------------------------------------------------------------- projection


def test_project_hand_example_and_identity():
    M = np.array([[1.0, 0.0, 2.0], [0.0, -1.0, 0.5]])  # 2 sources x 3 sensors
    x = np.array([[1.0, 2.0], [3.0, 4.0], [5.0, 6.0]])  # 3 sensors x 2 samples
    # y_0 = x_0 + 2 x_2 = (11, 14); y_1 = -x_1 + 0.5 x_2 = (-0.5, -1)
    np.testing.assert_array_equal(O.project(M, x), [[11.0, 14.0], [-0.5, -1.0]])
    t = np.random.default_rng(0).standard_normal((4, 7, 9))
    np.testing.assert_array_equal(O.project(np.eye(7), t), t)


def test_projected_networks_of_a_permutation_are_permuted():
    """A permutation operator relabels the nodes: the networks are the permuted ones."""
    x, _ = eeg_sinusoid_trials(7, 8, 12, 256, n_pairs=5)
    perm = np.random.default_rng(1).permutation(12)
    M = np.eye(12)[perm]
    a = O.networks_dense(x, 1000.0, 256, 1.0, 50.0, metrics=("COH", "PLI", "COR"))
    b = O.networks_dense(O.project(M, x), 1000.0, 256, 1.0, 50.0, metrics=("COH", "PLI", "COR"))
    for m in ("COH", "PLI", "COR"):
        np.testing.assert_allclose(b[m], a[m][np.ix_(perm, perm)], atol=1e-12)


# ------------------------------------------------------------------------------ FIR


def test_fir_design_matches_scipy_firwin():
    signal = pytest.importorskip("scipy.signal")
    fs = 1000.0
    for kind, lo, hi, T in (("lowpass", 0.0, 40.0, 101), ("highpass", 2.0, 0.0, 301), ("bandpass", 8.0, 30.0, 201)):
        h = O.fir_design(fs, kind, lo, hi, 10.0, T)
        cut = {"lowpass": hi, "highpass": lo, "bandpass": [lo, hi]}[kind]
        ref = signal.firwin(T, cut, pass_zero={"lowpass": True, "highpass": False, "bandpass": False}[kind],
                            window="hamming", scale=False, fs=fs)
        np.testing.assert_allclose(h, ref, rtol=0, atol=1e-15)


def test_fir_design_properties():
    h = O.fir_design(600.0, "bandpass", 8.0, 12.0, 4.0)
    T = h.size
    assert T % 2 == 1 and T == 2 * (int(math.ceil(3.3 * 600 / 4.0)) // 2) + 1
    np.testing.assert_allclose(h, h[::-1], atol=1e-17)  # symmetric: linear phase
    lp = O.fir_design(1000.0, "lowpass", 0.0, 50.0, 10.0, 0)
    ripple = 10 ** (-53 / 20)  # Hamming window: about -53 dB stop band / pass-band ripple
    assert abs(lp.sum() - 1.0) < ripple  # unit DC gain up to the ripple
    hp = O.fir_design(1000.0, "highpass", 2.0, 0.0, 2.0, 0)
    assert abs(hp.sum()) < ripple  # DC in the stop band


def test_fir_stream_blocks_equal_whole_stream_and_impulse_response():
    rng = np.random.default_rng(4)
    h = O.fir_design(500.0, "bandpass", 4.0, 40.0, 4.0, 63)
    x = rng.standard_normal((3, 700))
    blocks = [x[:, :250], x[:, 250:251], x[:, 251:700]]
    y = np.concatenate(O.fir_filter_stream(h, blocks), axis=1)
    direct = np.array([[sum(h[k] * x[c, t - k] for k in range(h.size) if t - k >= 0) for t in range(700)]
                       for c in range(3)])
    np.testing.assert_allclose(y, direct, atol=1e-12)
    imp = np.zeros((1, 100))
    imp[0, 0] = 1.0
    np.testing.assert_allclose(O.fir_filter_stream(h, [imp])[0][0, :63], h, atol=1e-15)
