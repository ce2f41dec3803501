"""Thin ctypes binding of ``libfc.so`` (include/fc.h), same names as the C ABI.

Argument marshalling only: every step of the connectivity path runs in the CUDA
library. Arrays are passed as pointers: numpy arrays (host) or CUDA torch tensors
(device). If the library is missing it is built with nvcc; if it cannot be built or
loaded, every call raises - there is no CPU fallback.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

# status codes
FC_OK = 0
FC_ERR_INVALID_ARG = -1
FC_ERR_OUT_OF_MEMORY = -2
FC_ERR_CUDA = -3
FC_ERR_NOT_READY = -4
FC_ERR_TIMEOUT = -5
FC_ERR_ADMISSION = -6
FC_ERR_NONFINITE = -7
FC_ERR_UNSUPPORTED = -8

# metric bits
FC_COR, FC_XCOR, FC_COH, FC_IMAGCOHY, FC_PLV, FC_PLI, FC_USPLI, FC_WPLI, FC_DSWPLI = (1 << i for i in range(9))
FC_SPECTRAL_METRICS = FC_COH | FC_IMAGCOHY | FC_PLV | FC_PLI | FC_USPLI | FC_WPLI | FC_DSWPLI
FC_ALL_METRICS = FC_COR | FC_XCOR | FC_SPECTRAL_METRICS
METRIC_BITS = {"COR": FC_COR, "XCOR": FC_XCOR, "COH": FC_COH, "IMAGCOHY": FC_IMAGCOHY, "PLV": FC_PLV,
               "PLI": FC_PLI, "USPLI": FC_USPLI, "WPLI": FC_WPLI, "DSWPLI": FC_DSWPLI}

FC_TAPER_NONE, FC_TAPER_HANN, FC_TAPER_HANN_SYM = 0, 1, 2
TAPERS = {"none": 0, "hann": 1, "hann_sym": 2}
FC_PREC_FP32, FC_PREC_TF32, FC_PREC_BF16, FC_PREC_FP16, FC_PREC_TF32X3 = 0, 1, 2, 3, 4
FC_MODE_STREAM, FC_MODE_FULL = 0, 1
FC_SPECTRUM_AUTO, FC_SPECTRUM_DFT, FC_SPECTRUM_FFT = 0, 1, 2

FC_K_NAMES = ("spectrum", "calibrate", "node", "stream", "window", "herk_tc", "band_reduce",
              "cor", "xcor", "project", "other")
FC_ACC_FIELDS = {"csd_re": 0, "csd_im": 1, "u_re": 2, "u_im": 3, "abs": 4, "sq": 5, "sign": 6,
                 "psd": 7, "cor": 8, "xcor": 9}


class fc_band(C.Structure):
    _fields_ = [("f_lo", C.c_double), ("f_hi", C.c_double), ("nfft", C.c_int)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class fc_config(C.Structure):
    _fields_ = [("precision", C.c_int), ("mode", C.c_int), ("stream", C.c_void_p),
                ("resum_period", C.c_int), ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN),
                ("alloc_ctx", C.c_void_p), ("spectrum", C.c_int)]


class fc_info(C.Structure):
    _fields_ = [("n_nodes", C.c_int), ("n_samples", C.c_int), ("n_bins", C.c_int),
                ("first_bin", C.c_int), ("nfft", C.c_int), ("window", C.c_int), ("k_used", C.c_int),
                ("pushes", C.c_longlong), ("rejected", C.c_longlong), ("pairs", C.c_longlong),
                ("device_bytes", C.c_size_t), ("metric_mask", C.c_uint32), ("mode", C.c_int),
                ("precision", C.c_int), ("spectrum", C.c_int)]


class fc_kernel_time(C.Structure):
    _fields_ = [("launches", C.c_int), ("total_ms", C.c_double)]


class fc_top_info(C.Structure):
    _fields_ = [("max_abs", C.c_float), ("threshold", C.c_float), ("kept", C.c_longlong)]


class fc_server_config(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("max_batch", C.c_int), ("plain", C.c_int),
                ("launch_blocks", C.c_int), ("precision", C.c_int)]


class fc_result(C.Structure):
    _fields_ = [("session", C.c_int), ("seq", C.c_longlong), ("status", C.c_int), ("arrival_ms", C.c_double),
                ("done_ms", C.c_double), ("batch", C.c_int)]


class fc_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("completed", C.c_longlong), ("launches", C.c_longlong),
                ("batched_trials", C.c_longlong), ("pair_bin_updates", C.c_longlong), ("hbm_used", C.c_size_t),
                ("sessions", C.c_int)]


class FcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"fc status {status}: {message}")
        self.status = status


_LIB = None

# (name, restype, argtypes) of every exported entry point
_SIGNATURES = [
    ("fc_config_default", C.c_int, [C.POINTER(fc_config)]),
    ("fc_session_create", C.c_int, [C.c_int, C.c_int, C.c_double, fc_band, C.c_int, C.c_uint32, C.c_int,
                                    C.POINTER(fc_config), C.POINTER(C.c_void_p)]),
    ("fc_session_destroy", C.c_int, [C.c_void_p]),
    ("fc_push_trial", C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    ("fc_push_trials", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    ("fc_get_network", C.c_int, [C.c_void_p, C.c_uint32, C.c_int, C.c_void_p, C.c_size_t, C.c_int,
                                 C.POINTER(C.c_int)]),
    ("fc_get_network_async", C.c_int, [C.c_void_p, C.c_uint32, C.c_void_p, C.c_size_t]),
    ("fc_network_wait", C.c_int, [C.c_void_p]),
    ("fc_get_network_bins", C.c_int, [C.c_void_p, C.c_uint32, C.c_void_p, C.c_size_t, C.c_int]),
    ("fc_get_network_top", C.c_int, [C.c_void_p, C.c_uint32, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_int, C.POINTER(fc_top_info)]),
    ("fc_get_xcor_lags", C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]),
    ("fc_set_metric_mask", C.c_int, [C.c_void_p, C.c_uint32]),
    ("fc_set_band", C.c_int, [C.c_void_p, C.c_double, C.c_double]),
    ("fc_fir_create", C.c_int, [C.c_int, C.c_double, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int,
                                C.c_void_p, C.POINTER(C.c_void_p)]),
    ("fc_fir_get_taps", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    ("fc_fir_process", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    ("fc_fir_reset", C.c_int, [C.c_void_p]),
    ("fc_fir_destroy", C.c_int, [C.c_void_p]),
    ("fc_debug_wait_probe", C.c_int, [C.c_void_p, C.c_double]),
    ("fc_set_projection", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    ("fc_session_snapshot_size", C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    ("fc_session_snapshot", C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    ("fc_session_restore", C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    ("fc_sync", C.c_int, [C.c_void_p]),
    ("fc_session_info", C.c_int, [C.c_void_p, C.POINTER(fc_info)]),
    ("fc_last_error", C.c_char_p, []),
    ("fc_set_profiling", C.c_int, [C.c_void_p, C.c_int]),
    ("fc_kernel_times", C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    ("fc_launch_count", C.c_longlong, [C.c_void_p]),
    ("fc_session_stream", C.c_void_p, [C.c_void_p]),
    ("fc_debug_get_spectra", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t]),
    ("fc_debug_get_scale", C.c_int, [C.c_void_p, C.POINTER(C.c_float)]),
    ("fc_debug_get_accumulators", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t]),
    ("fc_window_networks_noalloc", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_uint32, C.c_void_p,
                                             C.c_size_t, C.c_void_p]),
    ("fc_server_now_ms", C.c_double, []),
    ("fc_server_create", C.c_int, [C.POINTER(fc_server_config), C.POINTER(C.c_void_p)]),
    ("fc_server_open", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_double, fc_band, C.c_int, C.c_uint32, C.c_int,
                                 C.POINTER(C.c_int)]),
    ("fc_server_session_bytes", C.c_int, [C.c_int, C.c_int, C.c_double, fc_band, C.c_uint32, C.c_int, C.c_int,
                                          C.POINTER(C.c_size_t)]),
    ("fc_server_submit", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_double]),
    ("fc_server_poll", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_int]),
    ("fc_server_drain", C.c_int, [C.c_void_p, C.c_int]),
    ("fc_server_get_network", C.c_int, [C.c_void_p, C.c_int, C.c_uint32, C.c_void_p, C.c_size_t]),
    ("fc_server_close", C.c_int, [C.c_void_p, C.c_int]),
    ("fc_server_stats_get", C.c_int, [C.c_void_p, C.POINTER(fc_server_stats)]),
    ("fc_server_destroy", C.c_int, [C.c_void_p]),
]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libfc.so (building it first if needed) and declare every signature."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2303_03279_gb300.build.build()")
    lib = C.CDLL(path)
    for name, res, args in _SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(status: int):
    if status != FC_OK:
        msg = _LIB.fc_last_error().decode(errors="replace")
        raise FcError(status, msg)


def _ptr(arr, dtype):
    """(pointer, on_device, element count) of a numpy array or a CUDA torch tensor."""
    mod = type(arr).__module__
    if mod.startswith("torch"):
        import torch  # noqa: F401  (device memory and streams only)
        if not arr.is_contiguous():
            raise ValueError("tensor must be contiguous")
        want = {np.float32: "torch.float32", np.int32: "torch.int32", np.float64: "torch.float64"}[dtype]
        if str(arr.dtype) != want:
            raise TypeError(f"tensor dtype {arr.dtype}, expected {want}")
        return C.c_void_p(arr.data_ptr()), 1 if arr.is_cuda else 0, arr.numel()
    if not isinstance(arr, np.ndarray) or arr.dtype != dtype or not arr.flags.c_contiguous:
        raise TypeError(f"expected a C-contiguous numpy array of {np.dtype(dtype).name}")
    return C.c_void_p(arr.ctypes.data), 0, arr.size


# ----------------------------------------------------------------- C-ABI mirrors


def fc_config_default() -> fc_config:
    lib = load()
    cfg = fc_config()
    _check(lib.fc_config_default(C.byref(cfg)))
    return cfg


def fc_session_create(n_nodes: int, n_samples: int, fs: float, band, taper, metric_mask: int,
                      window: int, cfg: fc_config | None = None):
    """band: (f_lo, f_hi, nfft); taper: FC_TAPER_* or 'hann' / 'hann_sym' / 'none'."""
    lib = load()
    if isinstance(taper, str):
        taper = TAPERS[taper]
    b = fc_band(float(band[0]), float(band[1]), int(band[2]))
    out = C.c_void_p()
    _check(lib.fc_session_create(int(n_nodes), int(n_samples), float(fs), b, int(taper), int(metric_mask),
                                 int(window), C.byref(cfg) if cfg is not None else None, C.byref(out)))
    return out


def fc_session_destroy(s):
    _check(load().fc_session_destroy(s))


def fc_push_trial(s, x):
    p, dev, _ = _ptr(x, np.float32)
    _check(_LIB.fc_push_trial(s, p, dev))


def fc_push_trials(s, x, count: int):
    p, dev, _ = _ptr(x, np.float32)
    _check(_LIB.fc_push_trials(s, p, int(count), dev))


def fc_get_network(s, metric: int, packed_upper: int, out) -> int:
    p, dev, nel = _ptr(out, np.float32)
    k = C.c_int(0)
    _check(_LIB.fc_get_network(s, int(metric), int(packed_upper), p, nel, dev, C.byref(k) if not dev else None))
    return k.value


def fc_get_network_async(s, metric: int, out):
    """Start reading the packed network into host memory `out` (numpy; pinned memory lets
    the copy overlap later pushes); fc_network_wait waits for the oldest read."""
    p, dev, nel = _ptr(out, np.float32)
    if dev:
        raise ValueError("fc_get_network_async reads into host memory")
    _check(_LIB.fc_get_network_async(s, int(metric), p, nel))


def fc_network_wait(s):
    _check(_LIB.fc_network_wait(s))


def fc_get_network_bins(s, metric: int, out):
    p, dev, nel = _ptr(out, np.float32)
    _check(_LIB.fc_get_network_bins(s, int(metric), p, nel, dev))


def fc_get_network_top(s, metric: int, percent: float, weights=None, degree=None, strength=None) -> dict:
    """Normalized strongest-edge network, node degree and strength (host numpy or device
    tensors, all on the same side); returns the fc_top_info fields."""
    outs = [o for o in (weights, degree, strength) if o is not None]
    on_dev = bool(outs) and type(outs[0]).__module__.startswith("torch") and outs[0].is_cuda
    si = fc_session_info(s)
    ptrs = []
    for o, dt, need in ((weights, np.float32, si.pairs), (degree, np.int32, si.n_nodes),
                        (strength, np.float32, si.n_nodes)):
        if o is None:
            ptrs.append(None)
            continue
        p, dev, nel = _ptr(o, dt)
        if nel < need or bool(dev) != on_dev:
            raise ValueError("outputs: weights [P], degree [n], strength [n], all on the host or all on the device")
        ptrs.append(p)
    pw, pd, ps = ptrs
    info = fc_top_info()
    _check(load().fc_get_network_top(s, int(metric), float(percent), pw, pd, ps, 1 if on_dev else 0, C.byref(info)))
    return {"max_abs": info.max_abs, "threshold": info.threshold, "kept": info.kept}


def fc_get_xcor_lags(s, out):
    p, dev, nel = _ptr(out, np.int32)
    _check(_LIB.fc_get_xcor_lags(s, p, nel, dev))


def fc_set_metric_mask(s, mask: int):
    _check(_LIB.fc_set_metric_mask(s, int(mask)))


def fc_set_band(s, f_lo: float, f_hi: float):
    _check(load().fc_set_band(s, float(f_lo), float(f_hi)))


def fc_session_snapshot(s) -> np.ndarray:
    """The session's state as a host byte array."""
    n = C.c_size_t(0)
    _check(load().fc_session_snapshot_size(s, C.byref(n)))
    buf = np.empty(n.value, np.uint8)
    _check(_LIB.fc_session_snapshot(s, C.c_void_p(buf.ctypes.data), buf.size))
    return buf


def fc_session_restore(s, buf):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(load().fc_session_restore(s, C.c_void_p(buf.ctypes.data), buf.size))


def fc_set_projection(s, op=None):
    """op: [n_nodes][n_channels] float32 (numpy or CUDA tensor), or None to remove it."""
    if op is None:
        _check(load().fc_set_projection(s, None, 0, 0))
        return
    p, dev, _ = _ptr(op, np.float32)
    _check(load().fc_set_projection(s, p, int(op.shape[1]), dev))


def fc_debug_wait_probe(s, limit_ms: float):
    _check(load().fc_debug_wait_probe(s, float(limit_ms)))


FIR_KINDS = {"lowpass": 0, "highpass": 1, "bandpass": 2}


def fc_fir_create(n_channels: int, fs: float, kind, f_lo: float, f_hi: float, transition_hz: float = 0.0,
                  n_taps: int = 0, stream=None):
    k = FIR_KINDS[kind] if isinstance(kind, str) else int(kind)
    out = C.c_void_p()
    _check(load().fc_fir_create(int(n_channels), float(fs), k, float(f_lo), float(f_hi), float(transition_hz),
                                int(n_taps), C.c_void_p(int(stream)) if stream is not None else None, C.byref(out)))
    return out


def fc_fir_get_taps(f) -> np.ndarray:
    n = C.c_int(0)
    _check(load().fc_fir_get_taps(f, None, 0, C.byref(n)))
    taps = np.empty(n.value, np.float64)
    _check(_LIB.fc_fir_get_taps(f, C.c_void_p(taps.ctypes.data), n.value, C.byref(n)))
    return taps


def fc_fir_process(f, x, y):
    """x, y: [n_channels][block_len] float32, both numpy or both CUDA tensors."""
    px, dx, _ = _ptr(x, np.float32)
    py, dy, _ = _ptr(y, np.float32)
    if dx != dy or tuple(x.shape) != tuple(y.shape):
        raise ValueError("x and y: same shape, both on the host or both on the device")
    _check(load().fc_fir_process(f, px, py, int(x.shape[1]), dx))


def fc_fir_reset(f):
    _check(load().fc_fir_reset(f))


def fc_fir_destroy(f):
    _check(load().fc_fir_destroy(f))


def fc_sync(s):
    _check(_LIB.fc_sync(s))


def fc_session_info(s) -> fc_info:
    info = fc_info()
    _check(_LIB.fc_session_info(s, C.byref(info)))
    return info


def fc_last_error() -> str:
    return load().fc_last_error().decode(errors="replace")


def fc_set_profiling(s, enable: bool):
    _check(_LIB.fc_set_profiling(s, 1 if enable else 0))


def fc_kernel_times(s, reset: bool = False) -> dict:
    arr = (fc_kernel_time * len(FC_K_NAMES))()
    _check(_LIB.fc_kernel_times(s, arr, 1 if reset else 0))
    return {FC_K_NAMES[i]: (arr[i].launches, arr[i].total_ms) for i in range(len(FC_K_NAMES))}


def fc_launch_count(s) -> int:
    return int(_LIB.fc_launch_count(s))


def fc_session_stream(s) -> int:
    return int(_LIB.fc_session_stream(s) or 0)


def fc_debug_get_spectra(s, age: int, out):
    p, dev, nel = _ptr(out, np.float32)
    if dev:
        raise ValueError("host output expected")
    _check(_LIB.fc_debug_get_spectra(s, int(age), p, nel))


def fc_debug_get_scale(s) -> float:
    v = C.c_float(0)
    _check(_LIB.fc_debug_get_scale(s, C.byref(v)))
    return v.value


def fc_debug_get_accumulators(s, field, out):
    if isinstance(field, str):
        field = FC_ACC_FIELDS[field]
    p, dev, nel = _ptr(out, np.float64)
    if dev:
        raise ValueError("host output expected")
    _check(_LIB.fc_debug_get_accumulators(s, int(field), p, nel))


def fc_window_networks_noalloc(spectra, n_trials: int, n_bins: int, n_nodes: int, metric_mask: int, out,
                               stream=None):
    """Allocation-free band-averaged spectral networks of one window (device tensors).

    spectra: CUDA float32 tensor [n_trials][n_bins][n_nodes][2]; out: CUDA float32 tensor
    with at least 7 * n_nodes * (n_nodes - 1) / 2 elements; stream: cudaStream_t or None.
    """
    p_in, dev_in, _ = _ptr(spectra, np.float32)
    p_out, dev_out, nel = _ptr(out, np.float32)
    if not (dev_in and dev_out):
        raise ValueError("spectra and out must be CUDA tensors")
    _check(load().fc_window_networks_noalloc(p_in, int(n_trials), int(n_bins), int(n_nodes), int(metric_mask),
                                             p_out, nel, C.c_void_p(int(stream) if stream else 0)))


def fc_server_now_ms() -> float:
    return float(load().fc_server_now_ms())


def fc_server_create(hbm_budget: int = 0, max_batch: int = 0, plain: bool = False, launch_blocks: int = 0,
                     precision: int = 0):
    cfg = fc_server_config(int(hbm_budget), int(max_batch), 1 if plain else 0, int(launch_blocks), int(precision))
    out = C.c_void_p()
    _check(load().fc_server_create(C.byref(cfg), C.byref(out)))
    return out


def fc_server_open(sv, n_nodes, n_samples, fs, band, taper, metric_mask, window) -> int:
    if isinstance(taper, str):
        taper = TAPERS[taper]
    sid = C.c_int(0)
    _check(_LIB.fc_server_open(sv, int(n_nodes), int(n_samples), float(fs), fc_band(float(band[0]), float(band[1]),
                               int(band[2])), int(taper), int(metric_mask), int(window), C.byref(sid)))
    return sid.value


def fc_server_session_bytes(n_nodes, n_samples, fs, band, metric_mask, window, plain=False) -> int:
    out = C.c_size_t(0)
    _check(load().fc_server_session_bytes(int(n_nodes), int(n_samples), float(fs),
                                          fc_band(float(band[0]), float(band[1]), int(band[2])), int(metric_mask),
                                          int(window), 1 if plain else 0, C.byref(out)))
    return int(out.value)


def fc_server_submit(sv, session_id: int, x, arrival_ms: float):
    x = np.ascontiguousarray(x, dtype=np.float32)
    _check(_LIB.fc_server_submit(sv, int(session_id), C.c_void_p(x.ctypes.data), float(arrival_ms)))


def fc_server_poll(sv, max_results: int = 256, wait_ms: int = 0):
    arr = (fc_result * max_results)()
    n = C.c_int(0)
    _check(_LIB.fc_server_poll(sv, arr, int(max_results), C.byref(n), int(wait_ms)))
    return [(r.session, r.seq, r.status, r.arrival_ms, r.done_ms, r.batch) for r in arr[: n.value]]


def fc_server_drain(sv, timeout_ms: int = 60000):
    _check(_LIB.fc_server_drain(sv, int(timeout_ms)))


def fc_server_get_network(sv, session_id: int, metric: int, out):
    p, dev, nel = _ptr(out, np.float32)
    if dev:
        raise ValueError("host output expected")
    _check(_LIB.fc_server_get_network(sv, int(session_id), int(metric), p, nel))


def fc_server_close(sv, session_id: int):
    _check(_LIB.fc_server_close(sv, int(session_id)))


def fc_server_stats_get(sv) -> dict:
    st = fc_server_stats()
    _check(_LIB.fc_server_stats_get(sv, C.byref(st)))
    return {k: getattr(st, k) for k, _ in fc_server_stats._fields_}


def fc_server_destroy(sv):
    _check(load().fc_server_destroy(sv))


# ----------------------------------------------------------------- convenience


class Session:
    """Owning wrapper: ``Session(n, N, fs, band, taper, mask, window, mode=..., ...)``."""

    def __init__(self, n_nodes, n_samples, fs, band, taper="hann", metric_mask=FC_ALL_METRICS,
                 window=0, mode=FC_MODE_STREAM, precision=FC_PREC_FP32, stream=None, resum_period=0,
                 spectrum=FC_SPECTRUM_AUTO):
        cfg = fc_config_default()
        cfg.mode = mode
        cfg.precision = precision
        cfg.resum_period = resum_period
        cfg.spectrum = spectrum
        if stream is not None:
            cfg.stream = C.c_void_p(int(stream))
        self.n, self.N = int(n_nodes), int(n_samples)
        self.handle = fc_session_create(n_nodes, n_samples, fs, band, taper, metric_mask, window, cfg)
        info = fc_session_info(self.handle)
        self.B, self.first_bin, self.P = info.n_bins, info.first_bin, info.pairs
        self.window = window

    def close(self):
        if self.handle:
            fc_session_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def push(self, x):
        x = x if type(x).__module__.startswith("torch") else np.ascontiguousarray(x, dtype=np.float32)
        if x.ndim == 2:
            fc_push_trial(self.handle, x)
        else:
            fc_push_trials(self.handle, x, x.shape[0])

    def network(self, metric, packed=False):
        bit = METRIC_BITS[metric] if isinstance(metric, str) else metric
        out = np.empty(self.P if packed else self.n * self.n, np.float32)
        k = fc_get_network(self.handle, bit, 1 if packed else 0, out)
        return (out if packed else out.reshape(self.n, self.n)), k

    def network_bins(self, metric):
        bit = METRIC_BITS[metric] if isinstance(metric, str) else metric
        out = np.empty(self.B * self.P, np.float32)
        fc_get_network_bins(self.handle, bit, out)
        return out.reshape(self.B, self.P)

    def spectra(self, age=0):
        out = np.empty(self.B * self.n * 2, np.float32)
        fc_debug_get_spectra(self.handle, age, out)
        return out.view(np.complex64).reshape(self.B, self.n).copy()

    def accumulators(self, field):
        f = FC_ACC_FIELDS[field]
        n = self.B * self.n if f == 7 else (self.P if f >= 8 else self.B * self.P)
        out = np.empty(n, np.float64)
        fc_debug_get_accumulators(self.handle, f, out)
        return out

    def xcor_lags(self):
        out = np.empty(self.P, np.int32)
        fc_get_xcor_lags(self.handle, out)
        return out

    def info(self):
        return fc_session_info(self.handle)
