"""Band change without recomputation (fc_set_band).

The per-bin sums hold everything the band average needs: after fc_set_band the networks
equal the oracle's band average over the new sub-band of the same window (GPU spectra,
1e-5; 5e-3 absolute for the tensor-core metrics of a BF16 session), and later pushes keep
averaging over it.
"""

import numpy as np
import pytest

from synth import white_trials, eeg_sinusoid_trials
from _fc_helpers import assert_close, window_spectra, oracle_spectral

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_03279_gb300 import fc  # noqa: E402

SPECTRAL = ("COH", "IMAGCOHY", "PLV", "PLI", "USPLI", "WPLI", "DSWPLI")
LINEAR = ("COH", "IMAGCOHY", "PLV")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fc.load()


def _check_band(s, K, k_lo, k_hi, first_bin, tol_linear=None):
    X = window_spectra(s, K)[:, :, k_lo - first_bin:k_hi - first_bin]
    ref = oracle_spectral(X.astype(np.complex128))
    for m in SPECTRAL:
        got = s.network(m, packed=True)[0]
        if tol_linear and m in LINEAR:
            assert np.nanmax(np.abs(got - ref[m])) <= tol_linear, m
        else:
            assert_close(got, ref[m], what=f"{m} bins {k_lo}..{k_hi - 1}")


@pytest.mark.parametrize("n", [128, 300])
def test_stream_band_change_and_later_pushes(n):
    N, fs, W = 500, 1000.0, 10
    x = white_trials(21, W + 6, n, N)
    with fc.Session(n, N, fs, (4.0, 44.0, 1000), "hann", fc.FC_SPECTRAL_METRICS, W) as s:
        assert s.B == 40 and s.first_bin == 4
        for t in range(W + 4):
            s.push(x[t])
        fc.fc_set_band(s.handle, 8.0, 13.0)  # bins 8..12
        _check_band(s, W, 8, 13, 4)
        for t in range(W + 4, W + 6):
            s.push(x[t])
        _check_band(s, W, 8, 13, 4)
        fc.fc_set_band(s.handle, 43.0, 44.0)  # the last bin alone
        _check_band(s, W, 43, 44, 4)
        fc.fc_set_band(s.handle, 4.0, 44.0)  # back to the whole band
        _check_band(s, W, 4, 44, 4)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_full_mode_band_change(precision):
    prec = {"fp32": fc.FC_PREC_FP32, "bf16": fc.FC_PREC_BF16}[precision]
    x, _ = eeg_sinusoid_trials(5, 20, 60, 500)
    with fc.Session(60, 500, 1000.0, (1.0, 50.0, 512), "hann", fc.FC_SPECTRAL_METRICS, 20,
                    mode=fc.FC_MODE_FULL, precision=prec) as s:
        s.push(x)
        fc.fc_set_band(s.handle, 9.0, 12.0)  # bins 5..6 at nfft 512 (k * 1000 / 512 in [9, 12))
        k_lo = int(np.ceil(9.0 * 512 / 1000.0))
        k_hi = int(np.ceil(12.0 * 512 / 1000.0))
        _check_band(s, 20, k_lo, k_hi, s.first_bin, tol_linear=5e-3 if precision == "bf16" else None)


def test_band_change_errors():
    with fc.Session(20, 128, 128.0, (8.0, 30.0, 128), "hann", fc.FC_SPECTRAL_METRICS, 3) as s:
        s.push(white_trials(2, 3, 20, 128))
        for lo, hi in ((2.0, 10.0), (20.0, 40.0), (10.2, 10.5), (12.0, 11.0)):
            with pytest.raises(fc.FcError) as e:
                fc.fc_set_band(s.handle, lo, hi)
            assert e.value.status == fc.FC_ERR_INVALID_ARG
        fc.fc_set_band(s.handle, 8.0, 30.0)


def test_bf16_band_change_at_1024_nodes_matches_fp32():
    """1024 nodes: the tensor-core band sums run over groups of several bins (reductions after
    each unit's first bin) starting inside the computed bins. After a band change and back,
    the BF16 session's linear metrics stay within 5e-3 of an FP32 session's on the same
    trials (itself checked against the oracle elsewhere), the non-linear ones within 1e-5."""
    n, N, W = 1024, 500, 20
    x = white_trials(31, W, n, N)
    x[:, 7] += 0.8 * x[:, 300]
    nets = {}
    for prec in (fc.FC_PREC_FP32, fc.FC_PREC_BF16):
        with fc.Session(n, N, 1000.0, (4.0, 44.0, 1000), "hann", fc.FC_SPECTRAL_METRICS, W,
                        mode=fc.FC_MODE_FULL, precision=prec) as s:
            s.push(x)
            out = []
            for lo, hi in ((10.0, 35.0), (4.0, 44.0)):
                fc.fc_set_band(s.handle, lo, hi)
                out.append({m: s.network(m, packed=True)[0].astype(np.float64) for m in SPECTRAL})
            nets[prec] = out
    for k in range(2):
        a, b = nets[fc.FC_PREC_FP32][k], nets[fc.FC_PREC_BF16][k]
        for m in SPECTRAL:
            d = np.nanmax(np.abs(a[m] - b[m]))
            assert d <= (5e-3 if m in LINEAR else 1e-5 * max(1.0, np.nanmax(np.abs(a[m])))), (k, m, d)
        assert a["COH"][7 * n - 7 * 8 // 2 + (300 - 7 - 1)] > 0.5  # the coupled pair stands out
