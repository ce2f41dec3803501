"""Pipelined host I/O: single trials pushed from pinned host memory go through the input
stream and alternating device buffers, networks are read with fc_get_network_async and
fc_network_wait. Every result must equal, bit for bit, what the same session computes when
fed device tensors and read synchronously."""

import numpy as np
import pytest

from synth import white_trials

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_03279_gb300 import fc  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fc.load()


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()


@pytest.mark.parametrize("mode", [fc.FC_MODE_STREAM, fc.FC_MODE_FULL])
def test_async_reads_match_synchronous_path(mode):
    n, N, W, T = 70, 200, 8, 14
    x = white_trials(21, T, n, N)
    x[:, 4] += 0.6 * x[:, 9]
    band = (4.0, 60.0, 256)
    ref = []
    with fc.Session(n, N, 500.0, band, "hann", fc.FC_SPECTRAL_METRICS, W, mode=mode) as s:
        for t in range(T):
            s.push(torch.from_numpy(x[t]).cuda())
            ref.append(s.network("COH", packed=True)[0].copy())
    pin = [_pinned(x[t]) for t in range(T)]
    outs = [torch.empty(n * (n - 1) // 2, dtype=torch.float32).pin_memory() for _ in range(2)]
    got = []
    with fc.Session(n, N, 500.0, band, "hann", fc.FC_SPECTRAL_METRICS, W, mode=mode) as s:
        fc.fc_network_wait(s.handle)  # nothing in flight: returns at once
        for t in range(T):
            fc.fc_push_trial(s.handle, pin[t].numpy())
            fc.fc_get_network_async(s.handle, fc.FC_COH, outs[t % 2].numpy())
            if t >= 1:
                fc.fc_network_wait(s.handle)
                got.append(outs[(t - 1) % 2].numpy().copy())
        fc.fc_network_wait(s.handle)
        got.append(outs[(T - 1) % 2].numpy().copy())
        fc.fc_sync(s.handle)
        # the synchronous read agrees with the last async one
        assert np.array_equal(s.network("COH", packed=True)[0], got[-1])
    for t in range(T):
        assert np.array_equal(got[t], ref[t]), t


def test_third_read_waits_for_the_oldest():
    n, N, W = 40, 128, 5
    x = white_trials(22, 6, n, N)
    P = n * (n - 1) // 2
    with fc.Session(n, N, 256.0, (2.0, 40.0, 128), "hann", fc.FC_COH | fc.FC_PLV, W) as s:
        for t in range(6):
            s.push(x[t])
        want_coh = s.network("COH", packed=True)[0].copy()
        want_plv = s.network("PLV", packed=True)[0].copy()
        bufs = [torch.empty(P, dtype=torch.float32).pin_memory() for _ in range(3)]
        fc.fc_get_network_async(s.handle, fc.FC_COH, bufs[0].numpy())
        fc.fc_get_network_async(s.handle, fc.FC_PLV, bufs[1].numpy())
        fc.fc_get_network_async(s.handle, fc.FC_COH, bufs[2].numpy())  # waits for bufs[0] first
        assert np.array_equal(bufs[0].numpy(), want_coh)
        fc.fc_network_wait(s.handle)
        fc.fc_network_wait(s.handle)
        fc.fc_network_wait(s.handle)  # none left
        assert np.array_equal(bufs[1].numpy(), want_plv)
        assert np.array_equal(bufs[2].numpy(), want_coh)


def test_async_read_argument_errors():
    n, N = 20, 64
    with fc.Session(n, N, 128.0, (2.0, 30.0, 64), "hann", fc.FC_COH, 4) as s:
        out = np.empty(n * (n - 1) // 2, np.float32)
        with pytest.raises(fc.FcError):  # nothing pushed yet
            fc.fc_get_network_async(s.handle, fc.FC_COH, out)
        s.push(white_trials(23, 1, n, N)[0])
        with pytest.raises(fc.FcError):  # not in the mask
            fc.fc_get_network_async(s.handle, fc.FC_PLV, out)
        with pytest.raises(fc.FcError):  # too short
            fc.fc_get_network_async(s.handle, fc.FC_COH, out[:-1])
