"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Two comparisons per workload:
* against the oracle run on the GPU's own FP32 spectra (read back through the test
  hook): isolates the pair kernels; sign counts (PLI, USPLI) are exact integers and
  every float metric is within 1e-5 relative;
* against the oracle's own FP64 spectra of the raw trials: the spectrum kernel's FP32
  rounding moves COH, IMAGCOHY, PLV, WPLI, COR, XCOR by less than 1e-5; the sign of
  Im(X_i X_j*) may flip where it is within FP32 rounding of zero, and the rate of such
  disagreements is reported and bounded.
"""

import math

import numpy as np
import pytest

import oracle as O
from synth import eeg_sinusoid_trials, meg_pink_trials, white_trials, ar2_source_model, ar2_source_trials
from _fc_helpers import (TOL, assert_close, close, window_spectra, packed_index, oracle_spectral, upper)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_03279_gb300 import fc  # noqa: E402

SPECTRAL = O.SPECTRAL_METRICS


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fc.load()


def _session(n, N, fs, band, window, mask=fc.FC_ALL_METRICS, mode=fc.FC_MODE_STREAM, taper="hann", **kw):
    return fc.Session(n, N, fs, band, taper, mask, window, mode=mode, **kw)


def _nets(sess, names, packed=True):
    return {m: sess.network(m, packed=packed)[0].astype(np.float64) for m in names}


def _sign_sum_from_network(pli_net, K, B):
    """sum_b |S_sign(b)| recovered exactly from the band-averaged PLI (= that sum / (K B))."""
    return np.rint(np.asarray(pli_net, np.float64) * K * B).astype(np.int64)


# ----------------------------------------------------------------------- spectra


SPECTRUM_CASES = [
    (70, 500, 512, (1.0, 50.0), "hann"),
    (33, 1000, 1024, (1.0, 100.0), "hann_sym"),
    (5, 37, 64, (0.0, 501.0), "none"),          # every bin 0 .. nfft/2, N < nfft
    (40, 2000, 4096, (0.0, 501.0), "hann"),     # wide band: 2049 bins
    (3, 10000, 16384, (10.0, 60.0), "hann"),    # largest transform (one warp per CTA)
    (50, 500, 1000, (4.0, 44.0), "hann"),       # nfft/2 = 500: radix 4, 5, 5, 5
    (20, 600, 600, (8.0, 12.0), "hann_sym"),    # nfft/2 = 300: radix 4, 3, 5, 5
    (7, 100, 240, (0.0, 501.0), "none"),        # nfft/2 = 120: radix 4, 2, 3, 5; every bin
    (9, 300, 448, (0.0, 501.0), "hann"),        # nfft/2 = 224: radix 4, 4, 2, 7; every bin
    (4, 4000, 4200, (8.0, 12.0), "hann"),       # nfft/2 = 2100: radix 4, 3, 5, 5, 7
]


@pytest.mark.parametrize("method", ["dft", "fft"])
@pytest.mark.parametrize("n,N,nfft,band,taper", SPECTRUM_CASES)
def test_spectrum_kernel_matches_fp64_dft(n, N, nfft, band, taper, method):
    """Band spectra of both methods (band DFT against a factor table; mixed-radix real FFT of
    the zero-padded trial with the even/odd split, including the bins 0 and nfft/2) against
    the FP64 DFT of the tapered trial, within 1e-5 of sum_t |x(t) w(t)|."""
    fs = 1000.0
    x = white_trials(1, 1, n, N)
    sp = fc.FC_SPECTRUM_FFT if method == "fft" else fc.FC_SPECTRUM_DFT
    with _session(n, N, fs, (band[0], band[1], nfft), 1, fc.FC_COH, taper=taper, spectrum=sp) as s:
        assert s.info().spectrum == sp
        s.push(x[0])
        scale = fc.fc_debug_get_scale(s.handle)
        Xg = s.spectra(0).T.astype(np.complex128) / scale  # [n][B]
    bins = O.band_bins(fs, nfft, *band)
    Xr = O.spectra(x[0], bins, nfft, taper)
    # FP32 dot product error bound scale: sum_t |x(t) w(t)|
    bound = np.sum(np.abs(x[0].astype(np.float64) * O.taper(N, taper)), axis=1)[:, None]
    assert np.all(np.abs(Xg - Xr) <= 1e-5 * bound), np.max(np.abs(Xg - Xr) / bound)


@pytest.mark.parametrize("mode", ["stream", "full"])
def test_fft_spectra_sessions_against_oracle(mode):
    """Sessions on the real-FFT method over a wide band (0 - 250 Hz at nfft 512: all 257
    bins, including DC and the Nyquist bin of fs = 500 Hz): every spectral metric against the
    oracle on the window's GPU spectra (1e-5, exact sign sums), the spectra themselves
    against the FP64 DFT, through a bulk fill and single pushes that slide the window."""
    n, N, W, T = 72, 400, 6, 10
    fs = 500.0
    x = white_trials(31, T, n, N)
    x[:, 3] = 0.8 * x[:, 40] + 0.2 * x[:, 3]
    md = fc.FC_MODE_STREAM if mode == "stream" else fc.FC_MODE_FULL
    with _session(n, N, fs, (0.0, 251.0, 512), W, fc.FC_SPECTRAL_METRICS, mode=md,
                  spectrum=fc.FC_SPECTRUM_FFT) as s:
        assert s.info().spectrum == fc.FC_SPECTRUM_FFT and s.B == 257
        s.push(x[:W])
        for t in range(W, T):
            s.push(x[t])
        _check_against_gpu_spectra(s, W)
        scale = fc.fc_debug_get_scale(s.handle)
        Xg = s.spectra(0).T.astype(np.complex128) / scale
    Xr = O.spectra(x[T - 1], O.band_bins(fs, 512, 0.0, 251.0), 512, "hann")
    bound = np.sum(np.abs(x[T - 1].astype(np.float64) * O.taper(N, "hann")), axis=1)[:, None]
    assert np.all(np.abs(Xg - Xr) <= 1e-5 * bound)


def test_prescale_is_a_power_of_two_and_invariant():
    n, N = 20, 200
    x = white_trials(2, 6, n, N)
    outs = []
    for amp in (1.0, 1e-12):
        with _session(n, N, 1000.0, (5.0, 60.0, 256), 6) as s:
            s.push(x * np.float32(amp))
            sc = fc.fc_debug_get_scale(s.handle)
            assert sc > 0 and math.frexp(sc)[0] == 0.5
            outs.append(_nets(s, SPECTRAL + ("COR", "XCOR")))
    for m in outs[0]:
        assert_close(outs[1][m], outs[0][m], what=m)


# ------------------------------------------------------------ full window, EEG size


def _check_against_gpu_spectra(sess, K, names=SPECTRAL, I=None, J=None):
    X = window_spectra(sess, K)
    ref = oracle_spectral(X, I, J)
    nets = _nets(sess, names)
    for m in names:
        g = nets[m] if I is None else nets[m][packed_index(I, J, sess.n)]
        assert_close(g, ref[m], what=m)
    # sign counts: exact
    g = nets["PLI"] if I is None else nets["PLI"][packed_index(I, J, sess.n)]
    got = _sign_sum_from_network(g, K, sess.B)
    exact = _sign_sum_from_network(ref["PLI"], K, sess.B)
    assert np.array_equal(got, exact)
    return X, nets



def _sign_disagreement(Xg, Xr, n):
    """Fraction of (trial, pair, bin) terms whose sign of Im(X_i X_j*) differs between the
    GPU's FP32 spectra and the FP64 oracle spectra of the same raw trials. Both signs are
    exact for their spectra (FP32 x FP32 products are exact in FP64, one rounding keeps the
    sign of the difference)."""
    I, J = np.triu_indices(n, 1)
    flips = 0
    for k in range(Xg.shape[0]):
        g = Xg[k].astype(np.complex128)
        sg = np.sign((g[I] * np.conj(g[J])).imag)
        sr = np.sign((Xr[k][I] * np.conj(Xr[k][J])).imag)
        flips += int(np.count_nonzero(sg != sr))
    return flips / (Xg.shape[0] * len(I) * Xg.shape[2])


@pytest.mark.parametrize("workload", ["eeg", "meg"])
def test_sign_disagreement_rate_against_fp64_spectra(workload, record_property):
    """PLI, USPLI, WPLI and DSWPLI count signs of Im(X_i X_j*). On the GPU's own FP32 spectra
    the counts are exact; against spectra computed in FP64 from the raw trials a sign can
    differ only where Im is within FP32 rounding of zero. The rate of such terms is measured
    and reported here (EEG: 60 channels with coupled sinusoids; MEG: 306 channels of pink
    noise, 1000 samples, 100 bins). Measured on GB300: 0 of 885,000 terms (EEG) and 6.4e-8
    (3 of 46.7 M terms, MEG)."""
    if workload == "eeg":
        x, _ = eeg_sinusoid_trials(7)
        fs, nfft, band = 1000.0, 512, (1.0, 50.0)
    else:
        x, _ = meg_pink_trials(8, n_trials=10)
        fs, nfft, band = 1000.0, 1000, (0.0, 100.0)
    K, n, N = x.shape
    with _session(n, N, fs, (band[0], band[1], nfft), K, mode=fc.FC_MODE_FULL) as s:
        s.push(x)
        Xg = window_spectra(s, K)
    bins = O.band_bins(fs, nfft, *band)
    Xr = np.stack([O.spectra(x[k], bins, nfft, "hann") for k in range(K)])  # [K][n][B]
    assert Xr.shape == Xg.shape
    rate = _sign_disagreement(Xg, Xr, n)
    record_property("sign_disagreement_rate", rate)
    print(f"\nsign disagreement vs FP64 spectra ({workload}, {K} trials x {n * (n - 1) // 2} pairs x "
          f"{Xg.shape[2]} bins): {rate:.3e}")
    assert rate < 1e-5, rate

def test_full_window_eeg_all_metrics():
    x, pairs = eeg_sinusoid_trials(7)  # 60 ch x 20 trials x 500 samples
    K, n, N = x.shape
    fs, nfft, band = 1000.0, 512, (1.0, 50.0)
    with _session(n, N, fs, (band[0], band[1], nfft), K, mode=fc.FC_MODE_FULL) as s:
        s.push(x)
        assert s.info().k_used == K
        X, nets = _check_against_gpu_spectra(s, K)
        # per-bin PLI/USPLI: integer-derived, exact per bin
        Xb = O.pair_sums_pairs(X, *np.triu_indices(n, 1))
        pli_b = s.network_bins("PLI")  # [B][P]
        assert np.array_equal(np.rint(pli_b * K).astype(np.int64), np.abs(Xb["sign"]).T)
        us_b = s.network_bins("USPLI").astype(np.float64)
        assert np.array_equal(np.rint(us_b * K * (K - 1) + K).astype(np.int64), (Xb["sign"] ** 2).T)
        # against the FP64 oracle of the raw trials
        ref = O.networks_dense(x, fs, nfft, *band)
        nets.update(_nets(s, ("COR", "XCOR")))
        for m in ("COH", "IMAGCOHY", "PLV", "WPLI", "COR", "XCOR"):
            assert_close(nets[m], upper(ref[m]), what=m + " vs FP64")
        for m in ("PLI", "USPLI", "DSWPLI"):
            frac = 1.0 - close(nets[m], upper(ref[m])).mean()
            assert frac < 0.02, (m, frac)
        # dense output: symmetric, IMAGCOHY antisymmetric, diagonal 0
        for m in ("COH", "IMAGCOHY", "XCOR"):
            d = s.network(m, packed=False)[0]
            sgn = -1 if m == "IMAGCOHY" else 1
            assert np.array_equal(d, sgn * d.T) and np.all(np.diag(d) == 0)
        # XCOR lag of the newest trial attains the maximum
        lags = s.xcor_lags()
        val_last, lag_last = O.xcor_trial_dense(x[-1])
        iu = np.triu_indices(n, 1)
        agree = lags == lag_last[iu]
        assert agree.mean() > 0.99
        for p in np.flatnonzero(~agree)[:20]:
            i, j = iu[0][p], iu[1][p]
            v, _ = O.xcor_trial_pair(x[-1][i], x[-1][j])
            xi = x[-1][i].astype(np.float64) - x[-1][i].mean()
            xj = x[-1][j].astype(np.float64) - x[-1][j].mean()
            tau = int(lags[p])
            r = np.dot(xi[tau:], xj[:N - tau]) if tau >= 0 else np.dot(xi[:N + tau], xj[-tau:])
            assert r / math.sqrt(np.dot(xi, xi) * np.dot(xj, xj)) >= v - 1e-5


# -------------------------------------------------------------- full window, MEG size


def test_full_window_meg_full_size_sampled():
    x, _ = meg_pink_trials(8)  # 306 ch x 100 trials x 1000 samples
    K, n, N = x.shape
    fs, nfft, band = 1000.0, 1024, (1.0, 100.0)
    rng = np.random.default_rng(0)
    with _session(n, N, fs, (band[0], band[1], nfft), K, mode=fc.FC_MODE_FULL) as s:
        s.push(x)
        assert s.B == 101
        iu = np.triu_indices(n, 1)
        pick = rng.choice(len(iu[0]), 1500, replace=False)
        I, J = iu[0][pick], iu[1][pick]
        X, nets = _check_against_gpu_spectra(s, K, I=I, J=J)
        # COR on all pairs against the oracle
        assert_close(nets["COR"] if "COR" in nets else s.network("COR", True)[0],
                     upper(O.cor_network(x)), what="COR")
        # XCOR on the pairs among 24 sampled nodes
        nodes = np.sort(rng.choice(n, 24, replace=False))
        xv = np.mean([O.xcor_trial_dense(x[k][nodes])[0] for k in range(K)], axis=0)
        a, b = np.triu_indices(len(nodes), 1)
        got = s.network("XCOR", True)[0][packed_index(nodes[a], nodes[b], n)]
        assert_close(got, xv[a, b], what="XCOR")


# ------------------------------------------------------------------------ streaming


@pytest.mark.parametrize("resum_period", [0, -1, 3])
def test_stream_matches_window_replay(resum_period):
    n, N, W = 70, 200, 8
    fs, nfft, band = 500.0, 256, (4.0, 60.0)
    x = white_trials(3, 21, n, N)
    x[:, 5] += x[:, 9] * 0.7  # one coupled pair
    with _session(n, N, fs, (band[0], band[1], nfft), W, resum_period=resum_period) as s:
        for t in range(x.shape[0]):
            s.push(x[t])
            if t + 1 in (1, 3, 8, 9, 15, 21):
                K = min(t + 1, W)
                X, nets = _check_against_gpu_spectra(s, K, names=SPECTRAL)
                sums = O.pair_sums_pairs(X, *np.triu_indices(n, 1))
                sg = s.accumulators("sign").reshape(s.B, -1)
                assert np.array_equal(sg.astype(np.int64), sums["sign"].T)
                mag = np.sqrt(sums["psd_i"] * sums["psd_j"]).T  # >= sum_k |X_i||X_j|
                for f, ref, bound in (("csd_re", np.real(sums["csd"]).T, mag),
                                      ("csd_im", np.imag(sums["csd"]).T, mag),
                                      ("abs", sums["abs"].T, sums["abs"].T),
                                      ("sq", sums["sq"].T, sums["sq"].T)):
                    acc = s.accumulators(f).reshape(s.B, -1)
                    assert np.all(np.abs(acc - ref) <= 1e-6 * bound + 1e-30), f
                psd = s.accumulators("psd").reshape(s.B, n)
                psd_ref = np.sum(np.abs(X.astype(np.complex128)) ** 2, axis=0).T
                assert np.all(np.abs(psd - psd_ref) <= 1e-12 * psd_ref)
                # COR and XCOR over the same window
                win = x[max(0, t + 1 - W): t + 1]
                assert_close(nets.get("COR", s.network("COR", True)[0]), upper(O.cor_network(win)), what="COR")
                assert_close(s.network("XCOR", True)[0], upper(O.xcor_network(win)[0]), what="XCOR")


def test_stream_cumulative_window():
    n, N = 40, 128
    x = white_trials(4, 6, n, N)
    with _session(n, N, 256.0, (8.0, 40.0, 128), 0, mask=fc.FC_SPECTRAL_METRICS | fc.FC_COR) as s:
        spectra = []
        for t in range(6):
            s.push(x[t])
            spectra.append(s.spectra(0).T)  # cumulative mode keeps only the newest spectra
        assert s.info().k_used == 6
        X = np.stack(spectra)
        ref = oracle_spectral(X)
        nets = _nets(s, SPECTRAL)
        for m in SPECTRAL:
            assert_close(nets[m], ref[m], what=m)
        assert np.array_equal(_sign_sum_from_network(nets["PLI"], 6, s.B),
                              _sign_sum_from_network(ref["PLI"], 6, s.B))
        assert_close(s.network("COR", True)[0], upper(O.cor_network(x)), what="COR")


def test_stream_bulk_then_single_pushes():
    n, N, W = 45, 160, 10
    x = white_trials(5, 17, n, N)
    with _session(n, N, 400.0, (3.0, 90.0, 200), W) as s:
        s.push(x[:12])  # bulk: re-sum path
        _check_against_gpu_spectra(s, W)
        for t in range(12, 17):
            s.push(x[t])
        _check_against_gpu_spectra(s, W)
        assert_close(s.network("XCOR", True)[0], upper(O.xcor_network(x[7:17])[0]), what="XCOR")


# ------------------------------------------------------------------------ edge cases


def test_two_nodes_single_trial():
    x = white_trials(6, 1, 2, 64)
    with _session(2, 64, 128.0, (2.0, 30.0, 64), 4) as s:
        s.push(x[0])
        nets = _nets(s, SPECTRAL)
        assert nets["PLV"].shape == (1,)
        assert abs(nets["COH"][0] - 1.0) < 1e-5 and abs(nets["PLV"][0] - 1.0) < 1e-5  # K = 1
        assert np.isnan(nets["USPLI"][0])
        _check_against_gpu_spectra(s, 1, names=("COH", "IMAGCOHY", "PLV", "PLI", "WPLI", "DSWPLI"))


def test_zero_and_identical_channels():
    n, N = 36, 100
    x = white_trials(7, 5, n, N)
    x[:, 3] = 0.0
    x[:, 7] = x[:, 11]
    x[:, 20] = 3.25  # constant, nonzero: centered to exactly 0, so COR and XCOR are 0
    with _session(n, N, 100.0, (1.0, 40.0, 128), 5) as s:
        s.push(x)
        nets = _nets(s, SPECTRAL + ("COR", "XCOR"))
        for m in ("COH", "IMAGCOHY", "PLV", "PLI", "WPLI", "DSWPLI", "COR", "XCOR"):
            assert np.all(nets[m][packed_index(3, np.arange(4, n), n)] == 0.0), m
        others = np.array([k for k in range(n) if k != 20])
        lo, hi = np.minimum(others, 20), np.maximum(others, 20)
        for m in ("COR", "XCOR"):
            assert np.all(nets[m][packed_index(lo, hi, n)] == 0.0), m
        p = packed_index(7, 11, n)
        assert abs(nets["COH"][p] - 1) < 1e-5 and abs(nets["PLV"][p] - 1) < 1e-5
        assert nets["PLI"][p] == 0 and nets["IMAGCOHY"][p] == 0 and nets["WPLI"][p] == 0
        assert abs(nets["COR"][p] - 1) < 1e-5 and abs(nets["XCOR"][p] - 1) < 1e-5
        _check_against_gpu_spectra(s, 5)


@pytest.mark.parametrize("mode,prec", [("stream", "fp32"), ("stream", "bf16"), ("full", "fp32"), ("full", "bf16")])
def test_sign_exact_where_im_is_within_rounding_of_zero(mode, prec):
    """Channels that are real multiples of others: Im(X_i X_j*) of their FP32 spectra is a
    few ulps from zero (or exactly zero) with either sign, the hardest input for the exact
    sign. Sign sums must equal the FP64 evaluation on the same spectra: per bin and signed
    (streaming accumulators), per bin in magnitude (FP32 per-bin PLI), over the band (PLI)."""
    n, N, K = 48, 200, 6
    x = white_trials(11, K, n, N)
    rng = np.random.default_rng(5)
    c = rng.uniform(0.3, 3.0, 24) * rng.choice([-1.0, 1.0], 24)
    x[:, 24:] = (x[:, :24].astype(np.float64) * c[None, :, None]).astype(np.float32)
    kw = dict(mode=fc.FC_MODE_STREAM if mode == "stream" else fc.FC_MODE_FULL,
              precision=fc.FC_PREC_FP32 if prec == "fp32" else fc.FC_PREC_BF16)
    with _session(n, N, 200.0, (1.0, 60.0, 256), K, **kw) as s:
        for k in range(K):
            s.push(x[k])
        X = window_spectra(s, K)
        iu = np.triu_indices(n, 1)
        sums = O.pair_sums_pairs(X, *iu)
        copies = packed_index(np.arange(24), np.arange(24) + 24, n)
        # the copies' products really are at the rounding level (and not all exactly zero)
        rel = np.abs(np.imag(sums["csd"][copies])) / np.abs(sums["csd"][copies])
        assert np.median(rel) < 1e-5 and np.any(sums["sign"][copies] != 0)
        if mode == "stream":
            sg = s.accumulators("sign").reshape(s.B, -1)
            assert np.array_equal(sg.astype(np.int64), sums["sign"].T)
        if prec == "fp32":  # per-bin values exist for FP32 sessions only
            pli_b = s.network_bins("PLI").astype(np.float64)
            assert np.array_equal(np.rint(pli_b * K).astype(np.int64), np.abs(sums["sign"]).T)
        names = ("PLI", "USPLI", "WPLI", "DSWPLI") if prec == "bf16" else SPECTRAL
        _check_against_gpu_spectra(s, K, names=names)


def test_nonfinite_trial_is_rejected_and_state_kept():
    n, N, W = 34, 64, 3
    x = white_trials(8, 5, n, N)
    with _session(n, N, 128.0, (4.0, 40.0, 64), W) as s:
        for t in range(3):
            s.push(x[t])
        before = _nets(s, SPECTRAL + ("COR", "XCOR"))
        acc_before = {f: s.accumulators(f) for f in ("csd_re", "csd_im", "u_re", "abs", "sq", "sign")}
        bad = x[3].copy()
        bad[5, 7] = np.nan
        s.push(bad)
        with pytest.raises(fc.FcError) as e:
            fc.fc_sync(s.handle)
        assert e.value.status == fc.FC_ERR_NONFINITE
        fc.fc_sync(s.handle)  # reported once
        after = _nets(s, SPECTRAL + ("COR", "XCOR"))
        for m in before:
            assert np.array_equal(before[m], after[m], equal_nan=True), m
        # the rejected push's drift re-sum slice (a third of the tile pairs at W = 3) left the
        # accumulators as they were
        for f, v in acc_before.items():
            assert np.array_equal(v, s.accumulators(f)), f
        info = s.info()
        assert info.pushes == 3 and info.rejected == 1
        s.push(x[3])
        _check_against_gpu_spectra(s, W)


def test_not_ready_and_argument_errors():
    with _session(8, 32, 64.0, (2.0, 20.0, 32), 2) as s:
        out = np.empty(s.P, np.float32)
        with pytest.raises(fc.FcError) as e:
            fc.fc_get_network(s.handle, fc.FC_COH, 1, out)
        assert e.value.status == fc.FC_ERR_NOT_READY
        s.push(white_trials(9, 1, 8, 32)[0])
        with pytest.raises(fc.FcError) as e:
            fc.fc_get_network(s.handle, fc.FC_COH | fc.FC_PLV, 1, out)
        assert e.value.status == fc.FC_ERR_INVALID_ARG
        with pytest.raises(fc.FcError) as e:
            fc.fc_get_network(s.handle, fc.FC_COH, 0, out)  # too small for dense
        assert e.value.status == fc.FC_ERR_INVALID_ARG


def test_metric_switching_reuses_the_sums():
    n, N, W = 50, 128, 6
    x = white_trials(10, 9, n, N)
    with _session(n, N, 256.0, (4.0, 60.0, 128), W, mask=fc.FC_COH | fc.FC_COR) as s:
        for t in range(9):
            s.push(x[t])
        fc.fc_set_metric_mask(s.handle, fc.FC_PLI | fc.FC_DSWPLI | fc.FC_COR)
        X = window_spectra(s, W)
        ref = oracle_spectral(X)
        for m in ("PLI", "DSWPLI"):
            assert_close(s.network(m, True)[0], ref[m], what=m)
        with pytest.raises(fc.FcError):
            s.network("COH", True)
        with pytest.raises(fc.FcError):
            fc.fc_set_metric_mask(s.handle, fc.FC_XCOR)


def test_device_tensors_in_and_out():
    n, N, W = 40, 96, 4
    x = white_trials(11, 4, n, N)
    with _session(n, N, 192.0, (4.0, 60.0, 128), W) as s:
        xd = torch.from_numpy(x).cuda()
        torch.cuda.synchronize()
        for t in range(4):
            fc.fc_push_trial(s.handle, xd[t].contiguous())
        out = torch.empty(s.P, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        fc.fc_get_network(s.handle, fc.FC_COH, 1, out)
        fc.fc_sync(s.handle)
        host = s.network("COH", True)[0]
        assert np.array_equal(out.cpu().numpy(), host)
        dense = torch.empty(n * n, dtype=torch.float32, device="cuda")
        fc.fc_get_network(s.handle, fc.FC_COH, 0, dense)
        fc.fc_sync(s.handle)
        assert np.array_equal(dense.cpu().numpy().reshape(n, n), s.network("COH")[0])


# --------------------------------------------- full size of the benchmarked workload


def test_large_source_space_full_size_sampled():
    """5124 nodes, W = 100, 500 samples, 40 bins (4-44 Hz): the benchmarked configuration.

    Bulk fill (re-sum path) then streaming pushes; sampled pairs against the oracle
    run on the GPU's spectra of the window, sign counts exact.
    """
    n, N, W, fs = 5124, 500, 100, 1000.0
    model = ar2_source_model(42, n)
    rng = np.random.default_rng(1)
    with _session(n, N, fs, (4.0, 44.0, 1000), W, mask=fc.FC_SPECTRAL_METRICS) as s:
        assert s.B == 40
        s.push(ar2_source_trials(model, 0, W, N))
        for t in range(W, W + 3):
            s.push(ar2_source_trials(model, t, 1, N)[0])
        I = rng.integers(0, n - 1, 1200)
        J = rng.integers(I + 1, n)
        # include pairs in the ragged last tile and on diagonal tiles
        I = np.concatenate([I, [n - 2, 0, 31, 5120]])
        J = np.concatenate([J, [n - 1, 1, 32, 5123]])
        _check_against_gpu_spectra(s, W, I=I, J=J)
