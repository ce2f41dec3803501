"""Seeded synthetic trial generators.

These produce the raw trial matrices (float32, ``[trials][nodes][samples]``) that
both the CUDA path and the FP64 oracle consume. This module holds none of the
connectivity method's arithmetic: no taper, no spectrum, no pair sums, no metric.
It only draws random numbers (numpy PCG64) and shapes them like the paper's
workloads:

* sensor-space EEG with sinusoids coupled at fixed lags (60 channels, 10 Hz),
* 1/f-shaped MEG sensor noise with coupled pairs (306 channels, 8-30 Hz),
* AR(2) alpha-band "source" oscillators with a seeded directed coupling graph
  (2000 or 5124 nodes), standing in for RTC-MNE source time courses,
* a serving trace of sessions with Poisson trial arrivals.

The paper's own data (MNE sample data, the MIND median-nerve set) is not
available; these generators stand in for it.
"""

from .generators import (  # noqa: F401
    eeg_sinusoid_trials,
    meg_pink_trials,
    ar2_source_model,
    ar2_source_trials,
    serving_trace,
    white_trials,
)
