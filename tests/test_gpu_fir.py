"""FIR filtering of the incoming stream (fc_fir_*) against the oracle.

* taps equal the oracle's FP64 window-method design;
* the filtered blocks equal the oracle's filtering of the continuous stream within
  1e-5 x sum|h| x max|x| (an FP32 chain of T FMAs);
* any division of the stream into blocks gives bit-identical output (the state carries
  over), and reset starts a fresh stream.
"""

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_03279_gb300 import fc  # noqa: E402

FILTERS = [  # kind, fs, f_lo, f_hi, transition, taps
    ("bandpass", 1000.0, 8.0, 30.0, 4.0, 0),
    ("highpass", 600.0, 2.0, 0.0, 2.0, 0),
    ("lowpass", 1792.0, 0.0, 40.0, 10.0, 255),
]


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fc.load()


def _run(f, x, splits, device=False):
    out, o = [], 0
    for L in splits:
        blk = np.ascontiguousarray(x[:, o:o + L])
        if device:
            xb = torch.from_numpy(blk).cuda()
            yb = torch.empty_like(xb)
            fc.fc_fir_process(f, xb, yb)
            torch.cuda.synchronize()
            out.append(yb.cpu().numpy())
        else:
            yb = np.empty_like(blk)
            fc.fc_fir_process(f, blk, yb)
            out.append(yb)
        o += L
    return np.concatenate(out, axis=1)


@pytest.mark.parametrize("kind,fs,lo,hi,tr,taps", FILTERS)
def test_fir_matches_oracle_and_is_block_invariant(kind, fs, lo, hi, tr, taps):
    C, total = 64, 3000
    x = np.random.default_rng(5).standard_normal((C, total)).astype(np.float32)
    f = fc.fc_fir_create(C, fs, kind, lo, hi, tr, taps)
    try:
        h = fc.fc_fir_get_taps(f)
        ref_h = O.fir_design(fs, kind, lo, hi, tr, taps)
        np.testing.assert_allclose(h, ref_h, rtol=0, atol=1e-12)
        splits_a = [500, 500, 1000, 1000]
        splits_b = [1, 7, 250, 742, 1000, 999, 1]
        ya = _run(f, x, splits_a)
        fc.fc_fir_reset(f)
        yb = _run(f, x, splits_b, device=True)
        assert np.array_equal(ya, yb)  # block division does not matter
        ref = np.concatenate(O.fir_filter_stream(ref_h, [x[:, :1500], x[:, 1500:]]), axis=1)
        tol = 1e-5 * np.abs(ref_h).sum() * np.abs(x).max()
        assert np.abs(ya - ref).max() <= tol
    finally:
        fc.fc_fir_destroy(f)


def test_fir_argument_errors():
    for args in ((0, 1000.0, "lowpass", 0.0, 40.0, 10.0, 0), (4, 1000.0, "lowpass", 0.0, 600.0, 10.0, 0),
                 (4, 1000.0, "bandpass", 30.0, 8.0, 4.0, 0), (4, 1000.0, "highpass", 1.0, 0.0, 0.0, 0),
                 (4, 1000.0, "lowpass", 0.0, 40.0, 0.1, 0)):
        with pytest.raises(fc.FcError) as e:
            fc.fc_fir_create(*args)
        assert e.value.status == fc.FC_ERR_INVALID_ARG
