"""fc_window_networks_noalloc against the session path and the oracle, calls in a row.

The allocation-free entry point serves callers that must not call cudaMalloc (a
real-time loop that cannot afford an allocation's device-wide synchronization, or a
host whose device memory belongs to another allocator). Its results must equal those of
a full-window session (fc_session_create / fc_push_trials / fc_get_network) on the same
spectra, and the FP64 oracle's on those spectra, within the tolerance of the other
parity tests, on consecutive calls with different shapes (a call must not see the
previous call's leftovers in the shared scratch array). The cases cover both ways the
band average is written (one bin group straight into the output; several groups through
partial sums, including a window whose group count is cut down to fit the scratch), a
partial metric mask (the other planes are left untouched) and spectra in physical units
(scaled by 2^-60: the call's power-of-two prescale makes the result identical). This file
is collected last so that a failure here cannot hide others.
"""

import numpy as np
import pytest

from synth import eeg_sinusoid_trials, white_trials
from _fc_helpers import assert_close, oracle_spectral

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_03279_gb300 import fc  # noqa: E402

ORDER = ("COH", "IMAGCOHY", "PLV", "PLI", "USPLI", "WPLI", "DSWPLI")
SCRATCH = 16 << 20  # FC_NOALLOC_SCRATCH_BYTES


def _session_reference(x, fs, band):
    K, n, N = x.shape
    s = fc.Session(n, N, fs, band, "hann", fc.FC_SPECTRAL_METRICS, K, mode=fc.FC_MODE_FULL)
    s.push(x)
    nets = {m: s.network(m, packed=True)[0] for m in ORDER}
    spectra = np.stack([s.spectra(age) for age in range(K)][::-1])  # [K][B][n] complex64
    B = s.B
    s.close()
    return nets, spectra, B


def _call(spectra, mask, stream, scale=1.0):
    K, B, n = spectra.shape
    P = n * (n - 1) // 2
    host = np.ascontiguousarray(spectra.view(np.float32).reshape(K, B, n, 2)) * np.float32(scale)
    dev_in = torch.from_numpy(host).cuda()
    out = torch.full((7 * P,), float("nan"), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    fc.fc_window_networks_noalloc(dev_in, K, B, n, mask, out, stream=stream.cuda_stream)
    stream.synchronize()
    return out.cpu().numpy().reshape(7, P)


def _groups(n, B):
    """Bin groups of the call: enough CTAs for the GPU, cut down to what fits the scratch."""
    nt = -(-n // 32)
    ntp = nt * (nt + 1) // 2
    P = n * (n - 1) // 2
    sms = torch.cuda.get_device_properties(0).multi_processor_count

    def a256(v):
        return (v + 255) & ~255

    off_part = a256(a256(a256(a256(a256(64) + 8 * B * n) + 4 * B * n) + 2 * ntp) + 2 * ntp)
    first = min(B, max(1, -(-(sms * 4) // ntp)))
    g = first
    while g > 1 and off_part + 28 * P * g > SCRATCH:
        g -= 1
    gb = -(-B // g)
    return first, -(-B // gb)


CASES = [  # x, fs, band, metric mask
    (eeg_sinusoid_trials(31)[0], 1000.0, (1.0, 50.0, 512), fc.FC_SPECTRAL_METRICS),  # 60 nodes, 20 trials, 25 bins
    (white_trials(32, 7, 45, 128), 256.0, (4.0, 60.0, 128), fc.FC_SPECTRAL_METRICS),  # 45 nodes, 7 trials, 28 bins
    (white_trials(34, 5, 70, 500), 1000.0, (10.0, 11.0, 1000), fc.FC_SPECTRAL_METRICS),  # one bin: direct write
    (white_trials(35, 2, 500, 500), 1000.0, (4.0, 44.0, 1000), fc.FC_COH | fc.FC_PLI | fc.FC_DSWPLI),  # groups cut
]


def test_noalloc_matches_session_and_oracle_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stream = torch.cuda.Stream()
    paths = set()
    for x, fs, band, mask in CASES:
        ref, spectra, B = _session_reference(x, fs, band)
        K, n, _ = x.shape
        first, groups = _groups(n, B)
        paths.add("direct" if groups == 1 else ("cut" if groups < first else "partials"))
        got = _call(spectra, mask, stream)
        orc = oracle_spectral(np.transpose(spectra, (0, 2, 1)).astype(np.complex128))
        for i, m in enumerate(ORDER):
            if mask & fc.METRIC_BITS[m]:
                assert_close(got[i], ref[m], what=f"no-alloc {m} vs session (n={n})")
                assert_close(got[i], orc[m], what=f"no-alloc {m} vs oracle (n={n})")
            else:
                assert np.isnan(got[i]).all(), f"plane {m} outside the mask was written (n={n})"
    assert paths == {"direct", "partials", "cut"}, paths


def test_noalloc_prescales_spectra_in_physical_units():
    """Spectra of order 1e-18 (MEG in tesla): Im^2 and |X|^2 would underflow in FP32; the
    call's power-of-two prescale gives exactly the result of the unscaled spectra."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stream = torch.cuda.Stream()
    x, fs, band, _ = CASES[0]
    ref, spectra, B = _session_reference(x, fs, band)
    base = _call(spectra, fc.FC_SPECTRAL_METRICS, stream)
    tiny = _call(spectra, fc.FC_SPECTRAL_METRICS, stream, scale=2.0 ** -60)
    assert np.array_equal(base, tiny, equal_nan=True)
    for i, m in enumerate(ORDER):
        assert_close(tiny[i], ref[m], what=f"no-alloc {m}, spectra x 2^-60")


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
