"""The C-ABI library builds for sm_103a, loads, and exports every symbol of include/fc.h.

No compute call is made here (there is no GPU on the build machine); session creation
must fail cleanly with FC_ERR_CUDA instead of falling back to the CPU.
"""

import ctypes
import os
import re

import pytest

from paper_2303_03279_gb300 import build, fc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*(fc_[a-z0-9_]+)\s*\(",
                            text, flags=re.M)
        names += re.findall(r"^\s*(?:long long|const char\s*\*|void\s*\*)\s*(fc_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 19, names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    bound = {s[0] for s in fc._SIGNATURES}
    assert set(names) <= bound, set(names) - bound


def test_binding_declares_only_exported_names():
    lib = fc.load()
    for name, _, _ in fc._SIGNATURES:
        assert hasattr(lib, name)


def test_no_cpu_fallback_without_gpu():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    lib = fc.load()
    with pytest.raises(fc.FcError) as e:
        fc.fc_session_create(8, 16, 100.0, (1.0, 20.0, 16), "hann", fc.FC_COH, 4)
    assert e.value.status == fc.FC_ERR_CUDA
    assert "no CUDA device" in fc.fc_last_error()


def test_argument_errors_are_reported_before_device_use():
    fc.load()
    with pytest.raises(fc.FcError) as e:
        fc.fc_session_create(1, 16, 100.0, (1.0, 20.0, 16), "hann", fc.FC_COH, 4)
    assert e.value.status == fc.FC_ERR_INVALID_ARG
    with pytest.raises(fc.FcError) as e:
        fc.fc_session_create(8, 32, 100.0, (1.0, 20.0, 16), "hann", fc.FC_COH, 4)  # nfft < N
    assert e.value.status == fc.FC_ERR_INVALID_ARG
    with pytest.raises(fc.FcError) as e:
        fc.fc_session_create(8, 16, 100.0, (45.0, 49.0, 16), "hann", fc.FC_COH, 4)  # no bin
    assert e.value.status == fc.FC_ERR_INVALID_ARG
    with pytest.raises(fc.FcError) as e:
        fc.fc_session_create(8, 16, 100.0, (1.0, 20.0, 16), "hann", 1 << 12, 4)
    assert e.value.status == fc.FC_ERR_INVALID_ARG
    # the real-FFT spectrum needs an even nfft in 16 .. 16384 with nfft/2 7-smooth
    for nfft in (1001, 22, 8, 32768, 2 * 11 * 64):
        cfg = fc.fc_config_default()
        cfg.spectrum = fc.FC_SPECTRUM_FFT
        with pytest.raises(fc.FcError) as e:
            fc.fc_session_create(8, 4, 1000.0, (1.0, 200.0, nfft), "hann", fc.FC_COH, 4, cfg)
        assert e.value.status == fc.FC_ERR_UNSUPPORTED, nfft
    cfg = fc.fc_config_default()
    cfg.spectrum = 3
    with pytest.raises(fc.FcError) as e:
        fc.fc_session_create(8, 16, 100.0, (1.0, 20.0, 16), "hann", fc.FC_COH, 4, cfg)
    assert e.value.status == fc.FC_ERR_INVALID_ARG
    for prec in (-1, fc.FC_PREC_TF32X3 + 1):  # outside the precision enum
        cfg = fc.fc_config_default()
        cfg.precision = prec
        with pytest.raises(fc.FcError) as e:
            fc.fc_session_create(8, 16, 100.0, (1.0, 20.0, 16), "hann", fc.FC_COH, 4, cfg)
        assert e.value.status == fc.FC_ERR_INVALID_ARG, prec


def test_header_enum_values_match_the_binding():
    """Every enumerator of include/fc.h written as NAME = <integer> has the same value in
    the Python binding (where the binding names it)."""
    text = open(os.path.join(ROOT, "include", "fc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    checked = 0
    for name, value in re.findall(r"\b(FC_[A-Z0-9_]+)\s*=\s*(-?\d+)\s*[,}\n]", text):
        if hasattr(fc, name):
            assert getattr(fc, name) == int(value), name
            checked += 1
    assert checked >= 10 and fc.FC_PREC_TF32X3 == 4
