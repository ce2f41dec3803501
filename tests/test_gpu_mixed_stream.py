"""Mixed-precision streaming: the exact streaming update with a tensor-core drift re-sum.

A stream-mode session with a tensor-core precision keeps the exact add/subtract update of
every accumulator (FP32 terms, double-float sums); its drift re-sum, one slice of 128-node
tile pairs per push, takes the linear sums (CSD real part, phasor sums) from tcgen05
products over an operand ring of the window and the non-linear sums (sum Im, sum |Im|,
sum Im^2, sign counts) from the non-linear sums kernel of the full-window mixed path (FP32
partial sums of at most 36 trials added into double words; exact signs). After a slice, COH
and PLV carry the operand rounding of the tensor cores; IMAGCOHY (from sum Im), PLI, USPLI,
WPLI and DSWPLI are sums of the exact FP32 terms. Against the oracle on the window's GPU spectra (Supplementary
Information 1): COH and PLV within 5e-3 absolute, the other metrics within 1e-5 with exact
sign sums (the re-sum adds the non-linear terms exactly as the update does, so a trial that
leaves the window leaves no rounding residue behind), through bulk fills, single pushes and more than two re-sum periods; served
sessions give the same networks alone and in the mix.
"""

import numpy as np
import pytest

import oracle as O
from synth import white_trials
from _fc_helpers import assert_close, oracle_spectral, window_spectra

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_03279_gb300 import fc  # noqa: E402

SPECTRAL = ("COH", "IMAGCOHY", "PLV", "PLI", "USPLI", "WPLI", "DSWPLI")
TENSOR = ("COH", "PLV")
PRECISIONS = {"bf16": fc.FC_PREC_BF16, "tf32": fc.FC_PREC_TF32, "tf32x3": fc.FC_PREC_TF32X3}


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fc.load()


def _check(nets, X, K, B, what, prec="bf16"):
    ref = oracle_spectral(X.astype(np.complex128))
    errs = {}
    for m in SPECTRAL:
        got = nets[m].astype(np.float64)
        if m in TENSOR and prec == "tf32x3":  # split TF32: FP32-class products
            assert_close(got, ref[m], what=f"{what} {m}")
            errs[m] = float(np.nanmax(np.abs(got - ref[m])))
        elif m in TENSOR:
            err = np.nanmax(np.abs(got - ref[m]))
            assert err <= 5e-3, (what, m, err)
            errs[m] = err
        else:
            assert_close(got, ref[m], what=f"{what} {m}")
    pli = nets["PLI"].astype(np.float64)
    assert np.array_equal(np.rint(pli * K * B), np.rint(ref["PLI"] * K * B)), what
    return errs


@pytest.mark.parametrize("prec", sorted(PRECISIONS))
def test_mixed_stream_against_oracle(prec):
    """300 nodes (three 128-node tiles, the last ragged; 10 x 10 tiles of 32), W = 8, 20 bins:
    a bulk fill, then 20 single pushes (2.5 re-sum periods), checked after the fill, mid
    period and at the end."""
    n, N, W, T = 300, 256, 8, 28
    x = white_trials(71, T, n, N)
    x[:, 5] += 0.7 * x[:, 290]
    with fc.Session(n, N, 512.0, (10.0, 50.0, 512), "hann", fc.FC_SPECTRAL_METRICS, W,
                    mode=fc.FC_MODE_STREAM, precision=PRECISIONS[prec]) as s:
        B = s.B
        s.push(x[:W])
        for t in range(W, T):
            s.push(x[t])
            if t in (W, W + 5, T - 1):
                nets = {m: s.network(m, packed=True)[0] for m in SPECTRAL}
                errs = _check(nets, window_spectra(s, W), W, B, f"{prec} push {t}", prec)
        print(f"[{prec}] max |gpu - oracle| of the tensor-core metrics:", {k: f"{v:.1e}" for k, v in errs.items()})


def test_mixed_stream_odd_nodes_shortest_window():
    """137 nodes (odd: the non-linear re-sum stages one node per copy; a ragged last 32-node
    and 128-node tile) with the shortest sliding window that re-sums, W = 2 (3 ring slots):
    single pushes from the start, through 3 re-sum periods, against the oracle. With two
    trials a window's debiased differences are as ill-conditioned as they get, so a re-sum
    that rounded its sums would leave residues that the strict tolerance catches."""
    n, N, W, T = 137, 128, 2, 9
    x = white_trials(73, T, n, N)
    with fc.Session(n, N, 256.0, (4.0, 60.0, 128), "hann", fc.FC_SPECTRAL_METRICS, W,
                    mode=fc.FC_MODE_STREAM, precision=fc.FC_PREC_BF16) as s:
        B = s.B
        for t in range(T):
            s.push(x[t])
            if t in (0, 1, 4, T - 1):
                K = min(t + 1, W)
                nets = {m: s.network(m, packed=True)[0] for m in SPECTRAL}
                _check(nets, window_spectra(s, K), K, B, f"push {t}")


def test_mixed_stream_slice_covers_every_block():
    """After one re-sum period the linear sums of every accumulator block come from the
    tensor cores: a BF16 session's COH differs from an FP32 session's (operand rounding) on
    pairs of every 128-node tile pair, while the exact-term metrics agree to 1e-5."""
    n, N, W = 260, 128, 6
    x = white_trials(72, 3 * W + 2, n, N)
    nets = {}
    for prec in (fc.FC_PREC_FP32, fc.FC_PREC_BF16):
        with fc.Session(n, N, 256.0, (8.0, 40.0, 256), "hann", fc.FC_SPECTRAL_METRICS, W,
                        mode=fc.FC_MODE_STREAM, precision=prec) as s:
            for t in range(x.shape[0]):
                s.push(x[t])
            nets[prec] = {m: s.network(m, packed=True)[0].astype(np.float64) for m in SPECTRAL}
    d = np.abs(nets[fc.FC_PREC_FP32]["COH"] - nets[fc.FC_PREC_BF16]["COH"])
    iu = np.triu_indices(n, 1)
    tile_pair = (iu[0] // 128) * 3 + iu[1] // 128
    for tp in np.unique(tile_pair):
        assert d[tile_pair == tp].max() > 0.0, tp  # every tile pair was re-summed on the tensor cores
    assert d.max() <= 5e-3
    for m in ("IMAGCOHY", "PLI", "USPLI", "WPLI", "DSWPLI"):
        assert_close(nets[fc.FC_PREC_BF16][m], nets[fc.FC_PREC_FP32][m], what=m)


SHAPES = [  # n, N, fs, band, W, trials
    (60, 200, 500.0, (1.0, 50.0, 256), 8, 14),
    (200, 200, 500.0, (4.0, 44.0, 250), 6, 15),
]


def _serve(which, xs, launch_blocks=0, precision=fc.FC_PREC_BF16):
    sv = fc.fc_server_create(precision=precision, launch_blocks=launch_blocks)
    try:
        ids = {k: fc.fc_server_open(sv, n, N, fs, band, "hann", fc.FC_SPECTRAL_METRICS, W)
               for k, (n, N, fs, band, W, _) in ((k, SHAPES[k]) for k in which)}
        for t in range(max(SHAPES[k][5] for k in which)):
            for k in which:
                if t < SHAPES[k][5]:
                    fc.fc_server_submit(sv, ids[k], xs[k][t], fc.fc_server_now_ms())
        fc.fc_server_drain(sv, 120000)
        res = fc.fc_server_poll(sv, 4096)
        assert all(r[2] == fc.FC_OK for r in res)
        out = {}
        for k in which:
            n = SHAPES[k][0]
            out[k] = {}
            for m in SPECTRAL:
                buf = np.empty(n * (n - 1) // 2, np.float32)
                fc.fc_server_get_network(sv, ids[k], fc.METRIC_BITS[m], buf)
                out[k][m] = buf
        return out, res
    finally:
        fc.fc_server_destroy(sv)


@pytest.mark.parametrize("prec", ["bf16", "tf32x3"])
def test_served_mixed_precision_sessions(prec):
    """A server whose sessions run the mixed-precision streaming form: each session's
    networks are bit-identical alone and in the mix (with pushes split over launches), and
    match the oracle on the window's GPU spectra within the precision's tolerances."""
    xs = [white_trials(80 + k, T, n, N) for k, (n, N, fs, band, W, T) in enumerate(SHAPES)]
    mixed, res = _serve([0, 1], xs, launch_blocks=50, precision=PRECISIONS[prec])
    assert max(r[5] for r in res) > 1
    for k, (n, N, fs, band, W, T) in enumerate(SHAPES):
        alone, _ = _serve([k], xs, precision=PRECISIONS[prec])
        for m in SPECTRAL:
            assert np.array_equal(alone[k][m], mixed[k][m], equal_nan=True), (k, m)
        with fc.Session(n, N, fs, band, "hann", fc.FC_SPECTRAL_METRICS, W, mode=fc.FC_MODE_STREAM,
                        precision=PRECISIONS[prec]) as s:
            for t in range(T):
                s.push(xs[k][t])
            X = window_spectra(s, W)
            B = s.B
            for m in SPECTRAL:  # the standalone session runs the same kernels in the same order
                assert np.array_equal(s.network(m, packed=True)[0], mixed[k][m], equal_nan=True), (k, m)
        _check(mixed[k], X, W, B, f"served cfg {k}", prec)


def test_mixed_stream_tiny_nodes_exact_signs():
    """Sign sums of the re-sum where Im(X_i X_j*) sits at the rounding level and some nodes
    have spectral components below 2^-50 (there an FMA residual of the exact determinant
    can round, and the FP64 evaluation takes over): nodes 16-31 are real multiples of nodes
    0-15, nodes 32-47 copies of 16-31 scaled by 2^-60 in trials 3, 9 and 10 only, so a node's
    tiny flag comes from a single push. The sign accumulators equal the FP64 signs of the
    window's GPU spectra (exact arithmetic on the same FP32 values) through three re-sum
    periods, with and without a tiny trial in the window."""
    n, N, W, T = 64, 200, 5, 16
    x = white_trials(73, T, n, N)
    rng = np.random.default_rng(9)
    c = rng.uniform(0.3, 3.0, 16) * rng.choice([-1.0, 1.0], 16)
    x[:, 16:32] = (x[:, :16].astype(np.float64) * c[None, :, None]).astype(np.float32)
    x[:, 32:48] = x[:, 16:32]
    for t in (3, 9, 10):
        x[t, 32:48] *= np.float32(2.0 ** -60)
    iu = np.triu_indices(n, 1)
    with fc.Session(n, N, 200.0, (1.0, 60.0, 256), "hann", fc.FC_SPECTRAL_METRICS, W,
                    mode=fc.FC_MODE_STREAM, precision=fc.FC_PREC_BF16) as s:
        checked = 0
        for t in range(T):
            s.push(x[t])
            if t in (W - 1, 9, 11, 14, T - 1):
                X = window_spectra(s, W)
                sums = O.pair_sums_pairs(X, *iu)
                sg = s.accumulators("sign").reshape(s.B, -1)
                assert np.array_equal(sg.astype(np.int64), sums["sign"].T), t
                checked += 1
        tiny = np.abs(X[:, 32:48]).max()
        assert checked == 5 and np.any(sums["sign"] != 0)
    assert tiny > 0
