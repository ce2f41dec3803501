"""Mixed-precision full-window path against the FP64 oracle.

COH, IMAGCOHY and PLV come from the tensor-core Hermitian products (tcgen05, BF16 / FP16
/ TF32 operands, FP32 accumulation): |gpu - oracle| <= 5e-3 absolute. PLI, USPLI, WPLI and
DSWPLI come from the CUDA-core non-linear sums on the exact FP32 terms: 1e-5 relative,
with the sign sums recovered exactly; DSWPLI within the bound its FP32 chunk sums give
(1e-5 plus 6 m u times the conditioning of its debiased differences, see _fc_helpers). The oracle runs on the GPU's own FP32 spectra, so
the differences isolate the operand rounding of the contraction.
"""

import numpy as np
import pytest

import oracle as O
from synth import eeg_sinusoid_trials, meg_pink_trials, white_trials
from _fc_helpers import assert_close, assert_close_bound, dswpli_mixed_tolerance, window_spectra, packed_index

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_03279_gb300 import fc  # noqa: E402

LINEAR = ("COH", "IMAGCOHY", "PLV")
NONLINEAR = ("PLI", "USPLI", "WPLI", "DSWPLI")
PRECISIONS = {"bf16": fc.FC_PREC_BF16, "fp16": fc.FC_PREC_FP16, "tf32": fc.FC_PREC_TF32,
              "tf32x3": fc.FC_PREC_TF32X3}
TOL_TC = {"bf16": 5e-3, "fp16": 5e-3, "tf32": 5e-3, "tf32x3": 1e-5}  # split TF32: FP32-class


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fc.load()


def _check(s, K, I=None, J=None, prec="bf16"):
    X = window_spectra(s, K)
    n = s.n
    if I is None:
        I, J = np.triu_indices(n, 1)
    ref = O.spectral_networks_pairs(X, I, J)
    p = packed_index(I, J, n)
    errs = {}
    for m in LINEAR:
        got = s.network(m, packed=True)[0].astype(np.float64)[p]
        err = np.abs(got - ref[m])
        errs[m] = float(err.max())
        assert err.max() <= TOL_TC[prec], (m, prec, err.max())
    dsw_tol = dswpli_mixed_tolerance(X, I, J)
    for m in NONLINEAR:
        got = s.network(m, packed=True)[0].astype(np.float64)[p]
        if m == "DSWPLI":  # FP32 chunk sums: the bound grows with the debiasing's conditioning
            assert_close_bound(got, ref[m], dsw_tol, what=f"{m} ({prec})")
        else:
            assert_close(got, ref[m], what=f"{m} ({prec})")
        errs[m] = float(np.abs(got - ref[m]).max())
    pli = s.network("PLI", packed=True)[0].astype(np.float64)[p]
    assert np.array_equal(np.rint(pli * K * s.B), np.rint(ref["PLI"] * K * s.B))
    print(f"[{prec}] max |gpu - oracle|:", {k: f"{v:.2e}" for k, v in errs.items()})
    return errs


@pytest.mark.parametrize("prec", sorted(PRECISIONS))
def test_mixed_full_window_eeg(prec):
    x, _ = eeg_sinusoid_trials(7)  # 60 ch, 20 trials, 500 samples
    K, n, N = x.shape
    with fc.Session(n, N, 1000.0, (1.0, 50.0, 512), "hann", fc.FC_SPECTRAL_METRICS, K,
                    mode=fc.FC_MODE_FULL, precision=PRECISIONS[prec]) as s:
        s.push(x)
        _check(s, K, prec=prec)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_mixed_full_window_meg_sampled(prec):
    x, _ = meg_pink_trials(8)  # 306 ch, 100 trials, 1000 samples, 101 bins
    K, n, N = x.shape
    rng = np.random.default_rng(3)
    with fc.Session(n, N, 1000.0, (1.0, 100.0, 1024), "hann", fc.FC_SPECTRAL_METRICS, K,
                    mode=fc.FC_MODE_FULL, precision=PRECISIONS[prec]) as s:
        s.push(x)
        iu = np.triu_indices(n, 1)
        pick = rng.choice(len(iu[0]), 2000, replace=False)
        # include pairs across the 128-node tile boundaries and in the ragged last tile
        I = np.concatenate([iu[0][pick], [0, 127, 127, 255, 300]])
        J = np.concatenate([iu[1][pick], [1, 128, 255, 256, 305]])
        _check(s, K, I, J, prec=prec)


def _herk_groups(nt128, nsel, sms, P, cap):
    """Bin groups the library picks for the tensor-core band sums of a window whose operands
    fit the resident form (its makespan model over work items of a row tile and at most three
    column tiles: ceil(items / SMs) rounds of a group's bins at ~1.2 us per column tile and
    ~1.5 us per resident fill, plus the band-sum planes' traffic), restated here only to
    assert that a case runs several groups."""
    segs = []
    for ta in range(nt128):
        length = nt128 - ta
        parts = (length + 2) // 3
        segs += [length * (q + 1) // parts - length * q // parts for q in range(parts)]
    nseg, seg_max = len(segs), max(segs)
    best, groups = None, 1
    for g in range(1, min(nsel, max(1, cap)) + 1):
        gb = -(-nsel // g)
        if -(-nsel // gb) != g:
            continue
        rounds = -(-(2 * nseg * g) // sms)
        t = rounds * gb * (seg_max * 1.2e-6 + 1.5e-6) + g * 3 * P * 8 / 6e12
        if best is None or t < best:
            best, groups = t, g
    return groups


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_mixed_band_groups_against_oracle(prec):
    """1100 nodes x 40 bins: the tensor-core band sums run over several bin groups (the first
    bin of a (tile pair, bin group) unit stores its values, the later bins add to them by
    reductions), over nine 128-node tiles of which the last is ragged (76 nodes), with the
    row tile's operands resident across segments of column tiles. Sampled
    pairs, including pairs across the 128-node tile edges, inside diagonal tiles and in the
    ragged tile, against the oracle on the GPU's spectra: COH, IMAGCOHY, PLV within 5e-3,
    PLI, USPLI, WPLI, DSWPLI within 1e-5 with exact sign sums."""
    n, N, W = 1100, 500, 20
    nt = -(-n // 128)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    groups = _herk_groups(nt, 40, sms, n * (n - 1) // 2, 40)
    assert 1 < groups < 40  # several groups of several bins
    x = white_trials(33, W, n, N)
    x[:, 7] += 0.8 * x[:, 1090]  # a coupled pair reaching into the ragged tile
    rng = np.random.default_rng(5)
    with fc.Session(n, N, 1000.0, (4.0, 44.0, 1000), "hann", fc.FC_SPECTRAL_METRICS, W,
                    mode=fc.FC_MODE_FULL, precision=PRECISIONS[prec]) as s:
        assert s.B == 40
        s.push(x)
        iu = np.triu_indices(n, 1)
        pick = rng.choice(len(iu[0]), 3000, replace=False)
        I = np.concatenate([iu[0][pick], [0, 127, 127, 128, 255, 1023, 1023, 1024, 7, 1098, 0]])
        J = np.concatenate([iu[1][pick], [1, 128, 1099, 255, 256, 1024, 1099, 1099, 1090, 1099, 1099]])
        errs = _check(s, W, I, J, prec=prec)
        coh = s.network("COH", packed=True)[0]
        assert coh[packed_index(7, 1090, n)] > 0.5  # the coupled pair stands out
    assert errs["COH"] > 0.0  # the contracted metrics carry the operand rounding


def test_mixed_window_fill_and_slide():
    # the window fills (K < W), then slides; the contraction length follows K
    n, N, W = 150, 128, 6
    x = white_trials(17, 9, n, N)
    with fc.Session(n, N, 256.0, (4.0, 60.0, 128), "hann", fc.FC_SPECTRAL_METRICS, W,
                    mode=fc.FC_MODE_FULL, precision=fc.FC_PREC_BF16) as s:
        for t in range(9):
            s.push(x[t])
            if t + 1 in (1, 4, 9):
                _check(s, min(t + 1, W))


@pytest.mark.parametrize("n", [97, 98])
def test_mixed_window_odd_and_even_node_counts(n):
    """The non-linear sums stage the spectra one node per copy for an odd node count and two
    nodes per copy for an even one; both, with a ragged last 32-node tile, a window of two
    chunks of trials (K = 40) and a ring that has wrapped, against the oracle."""
    N, W = 128, 40
    x = white_trials(29, W + 3, n, N)
    with fc.Session(n, N, 256.0, (4.0, 60.0, 128), "hann", fc.FC_SPECTRAL_METRICS, W,
                    mode=fc.FC_MODE_FULL, precision=fc.FC_PREC_BF16) as s:
        s.push(x[:W + 2])
        s.push(x[W + 2])
        _check(s, W)


def test_mixed_degenerate_channels_and_single_trial():
    """Degenerate inputs on the mixed path, against the oracle's conventions: a zero channel
    (every metric 0 with it), an identical pair (COH and PLV 1 within the operand rounding;
    Im of the exact FP32 terms is exactly 0, so PLI, WPLI and DSWPLI are exactly 0), and a
    window of one trial (COH and PLV 1, USPLI undefined: NaN, DSWPLI 0 with at most one
    nonzero term)."""
    n, N, K = 36, 100, 5
    x = white_trials(7, K, n, N)
    x[:, 3] = 0.0
    x[:, 7] = x[:, 11]
    with fc.Session(n, N, 100.0, (1.0, 40.0, 128), "hann", fc.FC_SPECTRAL_METRICS, K,
                    mode=fc.FC_MODE_FULL, precision=fc.FC_PREC_BF16) as s:
        s.push(x)
        _check(s, K)
        nets = {m: s.network(m, packed=True)[0] for m in LINEAR + NONLINEAR}
        zero = packed_index(3, np.arange(4, n), n)
        for m in LINEAR + ("PLI", "WPLI", "DSWPLI"):
            assert np.all(nets[m][zero] == 0.0), m
        p = packed_index(7, 11, n)
        assert abs(nets["COH"][p] - 1) < TOL_TC["bf16"] and abs(nets["PLV"][p] - 1) < TOL_TC["bf16"]
        assert nets["PLI"][p] == 0 and nets["WPLI"][p] == 0 and nets["DSWPLI"][p] == 0
    x1 = white_trials(6, 1, 2, 64)
    with fc.Session(2, 64, 128.0, (2.0, 30.0, 64), "hann", fc.FC_SPECTRAL_METRICS, 4,
                    mode=fc.FC_MODE_FULL, precision=fc.FC_PREC_BF16) as s:
        s.push(x1[0])
        nets = {m: s.network(m, packed=True)[0] for m in LINEAR + NONLINEAR}
        assert abs(nets["COH"][0] - 1) < TOL_TC["bf16"] and abs(nets["PLV"][0] - 1) < TOL_TC["bf16"]
        assert np.isnan(nets["USPLI"][0]) and nets["DSWPLI"][0] == 0
        _check(s, 1)


def test_mixed_window_of_two_trials():
    """W = 2, the worst-conditioned debiasing: DSWPLI of a window of two trials is
    2 Im_1 Im_2 / (2 |Im_1| |Im_2|), formed from sums of squares; held to the bound that the
    FP32 chunk sums give (see dswpli_mixed_tolerance), the other metrics as elsewhere."""
    n, N, W = 137, 128, 2
    x = white_trials(75, 6, n, N)
    with fc.Session(n, N, 256.0, (4.0, 60.0, 128), "hann", fc.FC_SPECTRAL_METRICS, W,
                    mode=fc.FC_MODE_FULL, precision=fc.FC_PREC_BF16) as s:
        for t in range(6):
            s.push(x[t])
            _check(s, min(t + 1, W))


def test_mixed_window_longer_than_4096_trials():
    """K = 4200 trials: beyond K = 4096 the non-linear sums form S and S^2 - K of PLI and USPLI
    through integers instead of exactly in FP32 (the packed finalize's other branch), and the
    products take the streaming-operand form (132 K-chunks). Against the oracle, signs exact."""
    n, N, W = 40, 64, 4200
    x = white_trials(31, W, n, N)
    with fc.Session(n, N, 128.0, (8.0, 40.0, 64), "hann", fc.FC_SPECTRAL_METRICS, W,
                    mode=fc.FC_MODE_FULL, precision=fc.FC_PREC_BF16) as s:
        s.push(x)
        _check(s, W)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_mixed_bulk_then_single_pushes_and_band_change(prec):
    """The full-window operands are kept by ring slot: a bulk fill packs the whole window,
    each single push rewrites only its own trial's slot (the slot of the trial that left), a
    band change reuses the operands as they are. Against the oracle on the window's GPU
    spectra after the fill, after single pushes that slide the window past every slot, and
    after a band change (oracle on the selected bins) and one more push."""
    n, N, W = 140, 128, 5
    x = white_trials(23, W + 8, n, N)
    with fc.Session(n, N, 256.0, (4.0, 60.0, 128), "hann", fc.FC_SPECTRAL_METRICS, W,
                    mode=fc.FC_MODE_FULL, precision=PRECISIONS[prec]) as s:
        s.push(x[:W])
        _check(s, W, prec=prec)
        for t in range(W, W + 7):
            s.push(x[t])
        _check(s, W, prec=prec)
        fc.fc_set_band(s.handle, 10.0, 30.0)  # bins 5 .. 14 of the computed 2 .. 29
        sel = slice(5 - 2, 15 - 2)
        for step in range(2):
            X = window_spectra(s, W)[:, :, sel]
            I, J = np.triu_indices(n, 1)
            ref = O.spectral_networks_pairs(X, I, J)
            for m in LINEAR:
                got = s.network(m, packed=True)[0].astype(np.float64)
                assert np.abs(got - ref[m]).max() <= TOL_TC[prec], (m, step)
            for m in NONLINEAR:
                assert_close(s.network(m, packed=True)[0], ref[m], what=f"{m} after the band change")
            if step == 0:
                s.push(x[W + 7])


def test_streaming_tensor_core_precision_needs_a_sliding_window_with_resum():
    """In stream mode a tensor-core precision applies to the drift re-sum of a sliding window:
    a cumulative window (0) or a session without re-sums is refused."""
    for window, period in ((0, 0), (4, -1)):
        with pytest.raises(fc.FcError) as e:
            fc.Session(40, 64, 128.0, (4.0, 40.0, 64), "hann", fc.FC_SPECTRAL_METRICS, window,
                       mode=fc.FC_MODE_STREAM, precision=fc.FC_PREC_BF16, resum_period=period)
        assert e.value.status == fc.FC_ERR_UNSUPPORTED
    with fc.Session(40, 64, 128.0, (4.0, 40.0, 64), "hann", fc.FC_SPECTRAL_METRICS, 4,
                    mode=fc.FC_MODE_STREAM, precision=fc.FC_PREC_BF16) as s:
        assert s.info().precision == fc.FC_PREC_BF16
