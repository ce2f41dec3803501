"""fc_window_networks_noalloc against the session path, two calls in a row.

The allocation-free entry point serves callers that must not call cudaMalloc (a
real-time loop that cannot afford an allocation's device-wide synchronization, or a
host whose device memory belongs to another allocator). Its results must equal those of
a full-window session (fc_session_create / fc_push_trials / fc_get_network) on the same
spectra, within the tolerance of the other parity tests, on two consecutive calls with
different shapes (the second call must not see the first call's leftovers in the shared
scratch array). This file is collected last so that a failure here cannot hide others.
"""

import numpy as np
import pytest

from synth import eeg_sinusoid_trials, white_trials
from _fc_helpers import assert_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_03279_gb300 import fc  # noqa: E402

ORDER = ("COH", "IMAGCOHY", "PLV", "PLI", "USPLI", "WPLI", "DSWPLI")


def _session_reference(x, fs, band):
    K, n, N = x.shape
    s = fc.Session(n, N, fs, band, "hann", fc.FC_SPECTRAL_METRICS, K, mode=fc.FC_MODE_FULL)
    s.push(x)
    nets = {m: s.network(m, packed=True)[0] for m in ORDER}
    spectra = np.stack([s.spectra(age) for age in range(K)][::-1])  # [K][B][n] complex64
    B = s.B
    s.close()
    return nets, spectra, B


def test_noalloc_matches_session_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cases = [
        (eeg_sinusoid_trials(31)[0], 1000.0, (1.0, 50.0, 512)),    # 60 nodes, 20 trials, 25 bins
        (white_trials(32, 7, 45, 128), 256.0, (4.0, 60.0, 128)),  # 45 nodes, 7 trials, 28 bins
    ]
    stream = torch.cuda.Stream()
    for x, fs, band in cases:
        ref, spectra, B = _session_reference(x, fs, band)
        K, n, _ = x.shape
        P = n * (n - 1) // 2
        dev_in = torch.from_numpy(np.ascontiguousarray(spectra.view(np.float32).reshape(K, B, n, 2))).cuda()
        out = torch.full((7 * P,), float("nan"), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        fc.fc_window_networks_noalloc(dev_in, K, B, n, fc.FC_SPECTRAL_METRICS, out, stream=stream.cuda_stream)
        stream.synchronize()
        got = out.cpu().numpy().reshape(7, P)
        for i, m in enumerate(ORDER):
            assert_close(got[i], ref[m], what=f"no-alloc {m} (n={n})")


def test_noalloc_rejects_sizes_beyond_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n, B, K = 2000, 1000, 1  # PSD sums alone exceed the fixed scratch
    dev_in = torch.zeros(K * B * n * 2, dtype=torch.float32, device="cuda")
    out = torch.zeros(7 * n * (n - 1) // 2, dtype=torch.float32, device="cuda")
    with pytest.raises(fc.FcError) as e:
        fc.fc_window_networks_noalloc(dev_in, K, B, n, fc.FC_SPECTRAL_METRICS, out)
    assert e.value.status == fc.FC_ERR_INVALID_ARG
    assert "scratch" in fc.fc_last_error()
