"""Network post-processing on the GPU against the oracle (normalization by the maximum edge
weight, strongest p % of the edges, node degree and strength).

The oracle runs on the GPU's own FP32 network (read back through fc_get_network), so the
edge ranking is decided on identical values: the kept set and the degrees are exact; the
normalized weights are the correctly rounded FP32 quotient (<= 1 ulp of the FP64 value);
strengths within 1e-6 relative.
"""

import numpy as np
import pytest

import oracle as O
from synth import eeg_sinusoid_trials, white_trials

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_03279_gb300 import fc  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fc.load()


def _check(s, metric, percent, device=False):
    n, P = s.n, s.P
    w = s.network(metric, packed=True)[0]
    ref_w, ref_deg, ref_str, ref_max, ref_kept = O.network_top(w, n, percent)
    if device:
        gw = torch.empty(P, dtype=torch.float32, device="cuda")
        gd = torch.empty(n, dtype=torch.int32, device="cuda")
        gs = torch.empty(n, dtype=torch.float32, device="cuda")
        info = fc.fc_get_network_top(s.handle, fc.METRIC_BITS[metric], percent, gw, gd, gs)
        gw, gd, gs = gw.cpu().numpy(), gd.cpu().numpy(), gs.cpu().numpy()
    else:
        gw = np.empty(P, np.float32)
        gd = np.empty(n, np.int32)
        gs = np.empty(n, np.float32)
        info = fc.fc_get_network_top(s.handle, fc.METRIC_BITS[metric], percent, gw, gd, gs)
    assert info["kept"] == ref_kept
    assert info["max_abs"] == np.float32(ref_max)
    assert np.array_equal(gd, ref_deg), (metric, percent)
    np.testing.assert_allclose(gw, ref_w, rtol=1.2e-7, atol=0, err_msg=f"{metric} {percent}")
    np.testing.assert_allclose(gs, ref_str, rtol=1e-6, atol=1e-7, err_msg=f"{metric} {percent}")
    return info


@pytest.mark.parametrize("percent", [5.0, 10.0, 25.0, 100.0, 0.0])
def test_post_processing_eeg_all_metrics(percent):
    x, _ = eeg_sinusoid_trials(11, 20, 60, 500)
    with fc.Session(60, 500, 1000.0, (1.0, 50.0, 512), "hann", fc.FC_ALL_METRICS, 20) as s:
        s.push(x)
        for m in ("COR", "XCOR", "COH", "IMAGCOHY", "PLV", "PLI", "USPLI", "WPLI", "DSWPLI"):
            _check(s, m, percent)


def test_post_processing_ties_and_device_outputs():
    """Half of the channels are zero: every pair touching one has COH 0, so the threshold
    falls among equal magnitudes and the lowest packed indices are kept."""
    x = white_trials(3, 6, 64, 256)
    x[:, 32:, :] = 0.0
    with fc.Session(64, 256, 256.0, (4.0, 40.0, 256), "hann", fc.FC_SPECTRAL_METRICS, 6) as s:
        s.push(x)
        for pct in (30.0, 60.0, 99.0):
            _check(s, "COH", pct)
            _check(s, "IMAGCOHY", pct, device=True)


def test_post_processing_nan_network():
    """USPLI with one trial is NaN on every edge: counts as 0, so the first edges are kept."""
    with fc.Session(40, 128, 128.0, (4.0, 30.0, 128), "hann", fc.FC_SPECTRAL_METRICS, 0) as s:
        s.push(white_trials(4, 1, 40, 128)[0])
        info = _check(s, "USPLI", 10.0)
        assert info["max_abs"] == 0.0


def test_post_processing_source_space_2000_nodes():
    n = 2000
    with fc.Session(n, 500, 1000.0, (4.0, 44.0, 1000), "hann", fc.FC_SPECTRAL_METRICS, 4) as s:
        s.push(white_trials(8, 4, n, 500))
        for m, pct in (("COH", 5.0), ("PLI", 10.0), ("IMAGCOHY", 25.0)):
            _check(s, m, pct)


def test_post_processing_argument_errors():
    with fc.Session(10, 64, 64.0, (4.0, 20.0, 64), "hann", fc.FC_COH, 2) as s:
        with pytest.raises(fc.FcError) as e:
            fc.fc_get_network_top(s.handle, fc.FC_COH, 5.0)
        assert e.value.status == fc.FC_ERR_NOT_READY
        s.push(white_trials(1, 1, 10, 64)[0])
        for bad in (-1.0, 100.5, float("nan")):
            with pytest.raises(fc.FcError):
                fc.fc_get_network_top(s.handle, fc.FC_COH, bad)
        with pytest.raises(fc.FcError):
            fc.fc_get_network_top(s.handle, fc.FC_PLI, 5.0)  # not in the mask
        assert fc.fc_get_network_top(s.handle, fc.FC_COH, 5.0)["kept"] == 3  # ceil(0.05 * 45)
