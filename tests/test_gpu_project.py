"""Source projection ahead of the spectrum (fc_set_projection) against the oracle.

The session's networks equal the oracle pipeline on the projected trials: COH, IMAGCOHY,
PLV, WPLI, COR and XCOR against the pure FP64 oracle (M x in FP64, then spectra) within
1e-5; PLI, USPLI and DSWPLI against the oracle on the GPU's own spectra (sign counts exact).
"""

import numpy as np
import pytest

import oracle as O
from synth import white_trials
from _fc_helpers import assert_close, window_spectra, oracle_spectral

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_03279_gb300 import fc  # noqa: E402

N_SRC, N_CH, N, FS, BAND, W = 100, 60, 500, 1000.0, (4.0, 44.0, 1000), 8


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fc.load()


def _operator(seed):
    return (np.random.default_rng(seed).standard_normal((N_SRC, N_CH)) / np.sqrt(N_CH)).astype(np.float32)


def _compare(s, x_window, M):
    y = O.project(M, x_window)
    ref = O.networks_dense(y, FS, BAND[2], BAND[0], BAND[1])
    iu = np.triu_indices(N_SRC, 1)
    for m in ("COH", "IMAGCOHY", "PLV", "WPLI", "COR", "XCOR"):
        assert_close(s.network(m, packed=True)[0], ref[m][iu], what=f"projected {m}")
    X = window_spectra(s, x_window.shape[0])
    ref_gpu = oracle_spectral(X.astype(np.complex128))
    for m in ("PLI", "USPLI", "DSWPLI"):
        assert_close(s.network(m, packed=True)[0], ref_gpu[m], what=f"projected {m} (GPU spectra)")


@pytest.mark.parametrize("mode", [fc.FC_MODE_STREAM, fc.FC_MODE_FULL])
def test_projected_session_matches_oracle(mode):
    M = _operator(1)
    x = white_trials(31, W + 5, N_CH, N)
    with fc.Session(N_SRC, N, FS, BAND, "hann", fc.FC_ALL_METRICS, W, mode=mode) as s:
        fc.fc_set_projection(s.handle, M)
        s.push(x[:W])                               # bulk push of sensor trials (host)
        for t in range(W, W + 3):
            s.push(x[t])                            # single pushes (host)
        xd = torch.from_numpy(x[W + 3:]).cuda()
        for t in range(2):
            fc.fc_push_trial(s.handle, xd[t])       # device input
        _compare(s, x[5:], M)


def test_projection_from_device_operator_and_removal():
    M = _operator(2)
    x = white_trials(32, 4, N_CH, N)
    with fc.Session(N_SRC, N, FS, BAND, "hann", fc.FC_SPECTRAL_METRICS, 4) as s:
        fc.fc_set_projection(s.handle, torch.from_numpy(M).cuda())
        s.push(x)
        ref = O.networks_dense(O.project(M, x), FS, BAND[2], BAND[0], BAND[1], metrics=("COH",))
        assert_close(s.network("COH", packed=True)[0], ref["COH"][np.triu_indices(N_SRC, 1)], what="COH")
        fc.fc_set_projection(s.handle, None)  # source trials again
        y = white_trials(33, 1, N_SRC, N)[0]
        s.push(y)
        X = window_spectra(s, 4)
        assert_close(s.network("COH", packed=True)[0], oracle_spectral(X.astype(np.complex128))["COH"],
                     what="after removal")
        with pytest.raises(fc.FcError):
            fc.fc_set_projection(s.handle, np.zeros((N_SRC, 0), np.float32))


@pytest.mark.parametrize("mode", [fc.FC_MODE_STREAM, fc.FC_MODE_FULL])
def test_spectral_projection_in_the_frequency_domain(mode):
    """A session whose metrics are all spectral projects the band spectra of the sensor
    trials (the operator acts on the node axis, the taper and the DFT on the sample axis, so
    they commute): its networks equal the FP64 oracle pipeline (projection in the time
    domain, then spectra) and those of a session that also holds COR (time-domain path)."""
    M = _operator(3)
    x = white_trials(34, W + 4, N_CH, N)
    spec = fc.FC_SPECTRAL_METRICS
    nets, X = {}, None
    for mask in (spec, spec | fc.FC_COR):
        with fc.Session(N_SRC, N, FS, BAND, "hann", mask, W, mode=mode) as s:
            fc.fc_set_projection(s.handle, M)
            s.push(x[:W])
            for t in range(W, W + 4):
                s.push(x[t])
            nets[mask] = {m: s.network(m, packed=True)[0] for m in
                          ("COH", "IMAGCOHY", "PLV", "PLI", "USPLI", "WPLI", "DSWPLI")}
            if mask == spec:
                X = window_spectra(s, W)
    iu = np.triu_indices(N_SRC, 1)
    ref = O.networks_dense(O.project(M, x[4:]), FS, BAND[2], BAND[0], BAND[1],
                           metrics=("COH", "IMAGCOHY", "PLV", "WPLI"))
    ref_gpu = oracle_spectral(X.astype(np.complex128))
    for m in ("COH", "IMAGCOHY", "PLV", "WPLI"):
        assert_close(nets[spec][m], ref[m][iu], what=f"frequency-domain projection {m}")
        assert_close(nets[spec][m], nets[spec | fc.FC_COR][m], what=f"frequency vs time domain {m}")
    for m in ("PLI", "USPLI", "DSWPLI"):
        assert_close(nets[spec][m], ref_gpu[m], what=f"frequency-domain projection {m} (GPU spectra)")
