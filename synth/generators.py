"""Seeded generators for synthetic trial data (no connectivity arithmetic here)."""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def white_trials(seed: int, n_trials: int, n_nodes: int, n_samples: int) -> np.ndarray:
    """N(0,1) white noise, float32 [trials][nodes][samples]."""
    return _rng(seed).standard_normal((n_trials, n_nodes, n_samples), dtype=np.float32)


def eeg_sinusoid_trials(seed: int, n_trials: int = 20, n_nodes: int = 60, n_samples: int = 500,
                        fs: float = 1000.0, n_pairs: int = 10, f0: float = 10.0,
                        lags=(0.0, math.pi / 4, math.pi / 2)):
    """Sensor-space EEG workload: N(0,1) channels plus ``n_pairs`` disjoint coupled pairs.

    Each coupled pair (a, b) carries ``sin(2*pi*f0*t + theta_k)`` on a and
    ``sin(2*pi*f0*t + theta_k - lag)`` on b, with a fresh uniform phase theta_k
    per trial and the lag cycling through ``lags``.
    Returns (x float32 [K][n][N], pairs list of (a, b, lag)).
    """
    rng = _rng(seed)
    x = rng.standard_normal((n_trials, n_nodes, n_samples))
    nodes = rng.permutation(n_nodes)[: 2 * n_pairs]
    t = np.arange(n_samples) / fs
    pairs = []
    for p in range(n_pairs):
        a, b = int(nodes[2 * p]), int(nodes[2 * p + 1])
        lag = float(lags[p % len(lags)])
        theta = rng.uniform(0.0, 2 * math.pi, n_trials)
        x[:, a, :] += np.sin(2 * math.pi * f0 * t[None, :] + theta[:, None])
        x[:, b, :] += np.sin(2 * math.pi * f0 * t[None, :] + theta[:, None] - lag)
        pairs.append((a, b, lag))
    return x.astype(np.float32), pairs


def meg_pink_trials(seed: int, n_trials: int = 100, n_nodes: int = 306, n_samples: int = 1000,
                    fs: float = 1000.0, n_pairs: int = 40, f_range=(8.0, 30.0)):
    """MEG sensor workload: 1/f-shaped Gaussian noise plus ``n_pairs`` coupled pairs.

    The noise is white Gaussian noise whose spectrum is shaped by 1/sqrt(f)
    (power ~ 1/f), rescaled to unit variance per channel. Each coupled pair gets
    unit-amplitude sinusoids at f ~ U[f_range] with a lag ~ U[0, pi) and a
    random phase per trial. Returns (x float32 [K][n][N], pairs list of (a, b, f, lag)).
    """
    rng = _rng(seed)
    w = rng.standard_normal((n_trials, n_nodes, n_samples))
    spec = np.fft.rfft(w, axis=-1)
    f = np.fft.rfftfreq(n_samples, d=1.0 / fs)
    shape = np.zeros_like(f)
    shape[1:] = 1.0 / np.sqrt(f[1:])
    x = np.fft.irfft(spec * shape, n=n_samples, axis=-1)
    x /= x.std(axis=-1, keepdims=True)
    nodes = rng.permutation(n_nodes)[: 2 * n_pairs]
    t = np.arange(n_samples) / fs
    pairs = []
    for p in range(n_pairs):
        a, b = int(nodes[2 * p]), int(nodes[2 * p + 1])
        f0 = float(rng.uniform(*f_range))
        lag = float(rng.uniform(0.0, math.pi))
        theta = rng.uniform(0.0, 2 * math.pi, n_trials)
        x[:, a, :] += np.sin(2 * math.pi * f0 * t[None, :] + theta[:, None])
        x[:, b, :] += np.sin(2 * math.pi * f0 * t[None, :] + theta[:, None] - lag)
        pairs.append((a, b, f0, lag))
    return x.astype(np.float32), pairs


@dataclass
class AR2Model:
    """Parameters of the AR(2) source model (drawn once per seed)."""
    n_nodes: int
    fs: float
    a1: np.ndarray  # [n] 2 r cos(2 pi f_alpha / fs)
    a2: np.ndarray  # [n] -r^2
    src: np.ndarray  # [E] edge sources
    dst: np.ndarray  # [E] edge targets
    gain: np.ndarray  # [E] coupling c
    delay: np.ndarray  # [E] delay d in samples
    seed: int = 0
    burn_in: int = 200
    extra: dict = field(default_factory=dict)


def ar2_source_model(seed: int, n_nodes: int, fs: float = 1000.0, n_edges: int = 200,
                     f_alpha: float = 10.0, r_range=(0.95, 0.99), c_range=(0.2, 0.5),
                     d_range=(5, 30)) -> AR2Model:
    """Draw the AR(2) alpha oscillators and the seeded directed coupling graph.

    x_t = 2 r cos(2 pi f_alpha / fs) x_{t-1} - r^2 x_{t-2} + eps_t, r ~ U[r_range];
    each of ``n_edges`` edges adds c * x_src(t - d) to x_dst, c ~ U[c_range],
    d ~ U{d_range}.
    """
    rng = _rng(seed)
    r = rng.uniform(*r_range, n_nodes)
    a1 = 2.0 * r * math.cos(2 * math.pi * f_alpha / fs)
    a2 = -(r * r)
    n_edges = min(n_edges, n_nodes * (n_nodes - 1))
    src = rng.integers(0, n_nodes, n_edges)
    off = rng.integers(1, n_nodes, n_edges)
    dst = (src + off) % n_nodes
    gain = rng.uniform(*c_range, n_edges)
    delay = rng.integers(d_range[0], d_range[1] + 1, n_edges)
    return AR2Model(n_nodes, fs, a1, a2, src, dst, gain, delay, seed=seed)


def ar2_source_trials(model: AR2Model, first_trial: int, n_trials: int, n_samples: int) -> np.ndarray:
    """Trials ``first_trial .. first_trial + n_trials - 1`` of the AR(2) source stream.

    Trial k is generated from its own seeded stream (seed, k), so any trial can be
    regenerated independently. Returns float32 [n_trials][n][n_samples].
    """
    n = model.n_nodes
    L = n_samples + model.burn_in
    out = np.empty((n_trials, n, n_samples), dtype=np.float32)
    for k in range(n_trials):
        rng = _rng([model.seed, 7919, first_trial + k])
        eps = rng.standard_normal((L, n))
        y = np.zeros((L, n))
        y[0] = eps[0]
        y[1] = model.a1 * y[0] + eps[1]
        for t in range(2, L):
            y[t] = model.a1 * y[t - 1] + model.a2 * y[t - 2] + eps[t]
        z = y.copy()
        for e in range(len(model.src)):
            d = int(model.delay[e])
            z[d:, model.dst[e]] += model.gain[e] * y[:-d, model.src[e]]
        out[k] = z[model.burn_in:].T
    return out


@dataclass
class ServingSession:
    n_nodes: int
    window: int
    rate_hz: float
    arrivals_s: np.ndarray  # sorted arrival times in seconds


def serving_trace(seed: int, duration_s: float = 2.0,
                  sizes=(60, 60, 60, 60, 128, 128, 128, 128, 306, 306, 306, 306, 1000, 1000, 1000, 5124),
                  window_range=(20, 100), rate_range=(5.0, 50.0)):
    """Serving workload: sessions of mixed node counts with Poisson trial arrivals.

    Each session draws a window W ~ U{window_range} and a rate ~ U[rate_range]
    trials/s; its arrivals are a Poisson process over ``duration_s`` seconds.
    """
    rng = _rng(seed)
    sessions = []
    for n in sizes:
        w = int(rng.integers(window_range[0], window_range[1] + 1))
        rate = float(rng.uniform(*rate_range))
        gaps = rng.exponential(1.0 / rate, int(rate * duration_s * 3) + 8)
        times = np.cumsum(gaps)
        times = times[times < duration_s]
        sessions.append(ServingSession(int(n), w, rate, times))
    return sessions
