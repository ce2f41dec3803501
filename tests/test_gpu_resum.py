"""Sliced re-sum of the streaming accumulators (drift reset spread over the pushes).

Push r of every period of R pushes re-sums the tile pairs [ntp r / R, ntp (r+1) / R) of
the accumulators from the stored spectra of the window. The re-summed slice must hold
exactly (bit for bit) what a bulk push of the same window computes; the other tile pairs
hold the streamed sums, equal to it up to double-float rounding.
"""

import numpy as np
import pytest

from synth import white_trials

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_03279_gb300 import fc  # noqa: E402

T = 32  # node tile


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fc.load()


def _tile_pair_of_pairs(n):
    nt = (n + T - 1) // T
    i, j = np.triu_indices(n, 1)
    a, b = i // T, j // T
    return a * nt - a * (a - 1) // 2 + (b - a), nt * (nt + 1) // 2


def _acc(s, field):
    out = np.empty(s.B * s.P, np.float64)
    fc.fc_debug_get_accumulators(s.handle, field, out)
    return out.reshape(s.B, s.P)


@pytest.mark.parametrize("R,pushes", [(2, 12), (3, 13), (4, 14), (1, 9)])
def test_resum_slice_is_bit_identical_to_bulk_window(R, pushes):
    n, N, fs, band, W = 100, 128, 256.0, (8.0, 40.0, 128), 5
    x = white_trials(77, pushes, n, N)
    tp, ntp = _tile_pair_of_pairs(n)
    with fc.Session(n, N, fs, band, "hann", fc.FC_SPECTRAL_METRICS, W, resum_period=R) as a, \
         fc.Session(n, N, fs, band, "hann", fc.FC_SPECTRAL_METRICS, W) as b:
        for k in range(pushes):
            a.push(x[k])
        b.push(x[pushes - W:])  # bulk push: the window's sums computed at once
        r = (pushes - 1) % R  # slice re-summed by the last push
        lo, hi = ntp * r // R, ntp * (r + 1) // R
        in_slice = (tp >= lo) & (tp < hi)
        assert in_slice.any()
        # each session has its own power-of-two prescale: rescale a's sums exactly to b's
        ratio = fc.fc_debug_get_scale(b.handle) / fc.fc_debug_get_scale(a.handle)
        power = {"csd_re": 2, "csd_im": 2, "abs": 2, "sq": 4, "u_re": 0, "u_im": 0, "sign": 0}
        for field, pw in power.items():
            va, vb = _acc(a, field) * ratio ** pw, _acc(b, field)
            assert np.array_equal(va[:, in_slice], vb[:, in_slice]), (field, R)
            scale = np.maximum(1.0, np.abs(vb[:, ~in_slice]))
            assert (np.abs(va[:, ~in_slice] - vb[:, ~in_slice]) <= 1e-9 * scale).all(), (field, R)
        for m in ("COH", "PLI", "WPLI", "DSWPLI"):
            np.testing.assert_allclose(a.network(m, packed=True)[0], b.network(m, packed=True)[0],
                                       rtol=1e-5, atol=1e-6)
