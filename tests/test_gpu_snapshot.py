"""Session snapshot / restore: a session restored from a snapshot continues exactly (bit for
bit) as the snapshotted one, through later pushes, re-sum slices and window slides."""

import numpy as np
import pytest

from synth import eeg_sinusoid_trials

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_03279_gb300 import fc  # noqa: E402

ALL = ("COR", "XCOR", "COH", "IMAGCOHY", "PLV", "PLI", "USPLI", "WPLI", "DSWPLI")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fc.load()


def _nets(s):
    out = {m: s.network(m, packed=True)[0] for m in ALL}
    lags = np.empty(s.P, np.int32)
    fc.fc_get_xcor_lags(s.handle, lags)
    out["lags"] = lags
    return out


@pytest.mark.parametrize("mode", [fc.FC_MODE_STREAM, fc.FC_MODE_FULL])
def test_restored_session_continues_identically(mode):
    x, _ = eeg_sinusoid_trials(17, 20, 60, 500)
    kw = dict(mode=mode, resum_period=3) if mode == fc.FC_MODE_STREAM else dict(mode=mode)
    args = (60, 500, 1000.0, (1.0, 50.0, 512), "hann", fc.FC_ALL_METRICS, 8)
    with fc.Session(*args, **kw) as a, fc.Session(*args, **kw) as b:
        for t in range(12):
            a.push(x[t])
        snap = fc.fc_session_snapshot(a.handle)
        fc.fc_session_restore(b.handle, snap)
        ref, got = _nets(a), _nets(b)
        for k in ref:
            assert np.array_equal(ref[k], got[k], equal_nan=True), k
        for t in range(12, 20):
            a.push(x[t])
            b.push(x[t])
        ref, got = _nets(a), _nets(b)
        for k in ref:
            assert np.array_equal(ref[k], got[k], equal_nan=True), k


def test_restore_refuses_foreign_snapshots():
    x, _ = eeg_sinusoid_trials(3, 4, 30, 256)
    with fc.Session(30, 256, 1000.0, (1.0, 50.0, 256), "hann", fc.FC_SPECTRAL_METRICS, 4) as a, \
         fc.Session(30, 256, 1000.0, (1.0, 50.0, 256), "hann", fc.FC_SPECTRAL_METRICS, 5) as other:
        a.push(x)
        snap = fc.fc_session_snapshot(a.handle)
        for bad in (snap[:100], snap[:-1], np.zeros_like(snap)):
            with pytest.raises(fc.FcError) as e:
                fc.fc_session_restore(a.handle, bad)
            assert e.value.status == fc.FC_ERR_INVALID_ARG
        with pytest.raises(fc.FcError) as e:
            fc.fc_session_restore(other.handle, snap)  # other window length
        assert e.value.status == fc.FC_ERR_INVALID_ARG
        fc.fc_session_restore(a.handle, snap)  # its own snapshot is fine
