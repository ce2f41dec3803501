"""XCOR across transform lengths: the shared-memory kernel (trials of at most 32 samples) and
every register-resident size (transforms of 64 .. 8192 points; 4096 points split into two
blocks, 8192 into four, each tested at both ends), against the oracle (values within 1e-5; the
reported lag attains the maximum within 1e-5)."""

import math

import numpy as np
import pytest

import oracle as O
from synth import white_trials

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_03279_gb300 import fc  # noqa: E402
from _fc_helpers import assert_close  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fc.load()


# N -> transform length L = next power of two >= 2N - 1, complex size M = L / 2
@pytest.mark.parametrize("N", [20, 40, 70, 130, 300, 600, 1500, 2048, 2049, 3000, 4096, 4097, 6000, 8192])
def test_xcor_matches_oracle_at_every_transform_length(N):
    n, K = 24, 3
    x = white_trials(100 + N, K, n, N)
    # a shifted copy gives a known lag
    x[:, 1, :] = np.roll(x[:, 0, :], 5)
    with fc.Session(n, N, 1000.0, (1.0, 50.0, max(64, 1 << (N - 1).bit_length())), "hann", fc.FC_XCOR, K) as s:
        s.push(x)
        got = s.network("XCOR", packed=True)[0]
        lags = s.xcor_lags()
    val, _ = O.xcor_network(x)
    iu = np.triu_indices(n, 1)
    assert_close(got, val[iu], what=f"XCOR N={N}")
    # the newest trial's lags attain the maximum
    last = x[-1].astype(np.float64)
    for p in range(0, len(iu[0]), 7):
        i, j = iu[0][p], iu[1][p]
        v, _ = O.xcor_trial_pair(last[i], last[j])
        xi, xj = last[i] - last[i].mean(), last[j] - last[j].mean()
        tau = int(lags[p])
        r = np.dot(xi[tau:], xj[:N - tau]) if tau >= 0 else np.dot(xi[:N + tau], xj[-tau:])
        assert r / math.sqrt(np.dot(xi, xi) * np.dot(xj, xj)) >= v - 1e-5, (N, i, j)


def test_xcor_rejects_trials_longer_than_8192_samples():
    with pytest.raises(fc.FcError):
        fc.Session(8, 8193, 1000.0, (1.0, 50.0, 16384), "hann", fc.FC_XCOR, 2)


@pytest.mark.parametrize("N", [2049, 4096, 4097, 8192])
def test_xcor_streaming_pushes_at_the_split_transform_length(N):
    """Single pushes past the window (the leaving trial's values subtracted) through the
    transforms split into two (4096 points) and four (8192 points) register blocks."""
    n, W, T = 16, 3, 6
    x = white_trials(300 + N, T, n, N)
    x[:, 2, :] = np.roll(x[:, 5, :], -7)
    with fc.Session(n, N, 1000.0, (1.0, 50.0, 1 << (N - 1).bit_length()), "hann", fc.FC_XCOR, W) as s:
        for t in range(T):
            s.push(x[t])
            got = s.network("XCOR", packed=True)[0]
            val, _ = O.xcor_network(x[max(0, t + 1 - W): t + 1])
            assert_close(got, val[np.triu_indices(n, 1)], what=f"XCOR N={N} after push {t}")
        lags = s.xcor_lags()
    p = int(packed_index_of(2, 5, n))
    want = O.xcor_trial_pair(x[-1, 2].astype(np.float64), x[-1, 5].astype(np.float64))[1]
    assert abs(want) == 7 and lags[p] == want, (lags[p], want)


def packed_index_of(i, j, n):
    return i * n - i * (i + 1) // 2 + (j - i - 1)
