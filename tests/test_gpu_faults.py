"""Failure detection without a GPU fault.

* A device wait that runs out: a kernel waits, through the library's bounded-wait routine,
  on a barrier nothing completes; it records a timeout and returns, the call reports
  FC_ERR_TIMEOUT within its budget, and the CUDA context stays usable.
* An allocation that fails (the caller's allocator hook returns NULL): FC_ERR_OUT_OF_MEMORY
  and everything already allocated is handed back.
* A session destroyed with pushes in flight: the other sessions' results are unchanged.
"""

import time

import numpy as np
import pytest

from synth import white_trials

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_03279_gb300 import fc  # noqa: E402

ARGS = (60, 500, 1000.0, (1.0, 50.0, 512), "hann", fc.FC_SPECTRAL_METRICS, 8)


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fc.load()


def _reference_coh(x):
    with fc.Session(*ARGS) as s:
        for t in range(x.shape[0]):
            s.push(x[t])
        return s.network("COH", packed=True)[0]


def test_bounded_wait_runs_out_and_reports_timeout():
    x = white_trials(1, 10, 60, 500)
    want = _reference_coh(x)
    with fc.Session(*ARGS) as probe:
        probe.push(x[0])
        t0 = time.perf_counter()
        with pytest.raises(fc.FcError) as e:
            fc.fc_debug_wait_probe(probe.handle, 20.0)
        assert e.value.status == fc.FC_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 5.0
        with pytest.raises(fc.FcError) as e:  # the session stays flagged
            fc.fc_sync(probe.handle)
        assert e.value.status == fc.FC_ERR_TIMEOUT
    # the context is still usable: a new session computes the same networks
    assert np.array_equal(_reference_coh(x), want)


def test_allocation_failure_returns_out_of_memory_and_frees_everything():
    for fail_after in (0, 3, 7):
        keep, calls = {}, {"n": 0}

        def alloc(nbytes, ctx):
            calls["n"] += 1
            if calls["n"] > fail_after:
                return None
            t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
            keep[t.data_ptr()] = t
            return t.data_ptr()

        def free(ptr, ctx):
            keep.pop(ptr, None)

        cfg = fc.fc_config_default()
        cfg.dev_alloc = fc.ALLOC_FN(alloc)
        cfg.dev_free = fc.FREE_FN(free)
        with pytest.raises(fc.FcError) as e:
            fc.fc_session_create(*ARGS, cfg)
        assert e.value.status == fc.FC_ERR_OUT_OF_MEMORY
        assert keep == {}, fail_after  # every successful allocation was handed back


def test_caller_allocator_runs_a_session_and_gets_everything_back():
    keep = {}

    def alloc(nbytes, ctx):
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        keep[t.data_ptr()] = t
        return t.data_ptr()

    def free(ptr, ctx):
        keep.pop(ptr, None)

    cfg = fc.fc_config_default()
    cfg.dev_alloc = fc.ALLOC_FN(alloc)
    cfg.dev_free = fc.FREE_FN(free)
    x = white_trials(2, 10, 60, 500)
    h = fc.fc_session_create(*ARGS, cfg)
    for t in range(10):
        fc.fc_push_trial(h, x[t])
    got = np.empty(60 * 59 // 2, np.float32)
    fc.fc_get_network(h, fc.FC_COH, 1, got)
    assert keep
    fc.fc_session_destroy(h)
    assert keep == {}
    assert np.array_equal(got, _reference_coh(x))


def test_destroy_with_pushes_in_flight_leaves_other_sessions_intact():
    x = white_trials(3, 12, 60, 500)
    want = _reference_coh(x)
    with fc.Session(*ARGS) as keeper:
        for t in range(12):
            doomed = fc.Session(*ARGS)
            for k in range(6):
                doomed.push(x[k])  # asynchronous: still running when destroyed
            keeper.push(x[t])
            doomed.close()
        assert np.array_equal(keeper.network("COH", packed=True)[0], want)
