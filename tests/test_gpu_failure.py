"""Failure detection on the GPU without a fault: a bounded device-side wait
that nothing completes must end in PIP_E_TIMEOUT, read on the host, with the
context still usable for the next call."""
import numpy as np
import pytest
import torch

import oracle
from paper_2007_15385_gb300 import binding as B
from paper_2007_15385_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()
    yield


def test_wait_that_never_completes_reports_timeout_and_the_context_survives():
    w = wl.vehicle_footprint(m=100_003)
    dev = torch.device("cuda", 0)
    v = torch.from_numpy(w.vertices).to(dev)
    vo = torch.from_numpy(w.vertex_offsets).to(dev)
    p = torch.from_numpy(w.points).to(dev)
    t = B.pip_prepare(v, vo, max_points=w.num_points)
    assert B.pip_get_status(t)[0] == B.PIP_OK
    # about 0.1 ms at 2 GHz; nothing ever completes the awaited phase
    B.pip_selftest_wait_timeout(t, 200_000)
    st, _ = B.pip_get_status(t)
    assert st == B.PIP_E_TIMEOUT
    assert B.pip_get_status(t)[0] == B.PIP_OK  # reported once, then cleared
    # the same tables and context decide the next call exactly
    mask, _ = B.pip_test(t, p)
    st, _ = B.pip_get_status(t)
    assert st == B.PIP_OK
    got = np.unpackbits(mask.cpu().numpy().view(np.uint8), bitorder="little")[:w.num_points]
    want, _ = oracle.inside_exact(w.vertices, w.points)
    np.testing.assert_array_equal(got, want)
    t.close()


def test_selftest_rejects_bad_arguments():
    w = wl.vehicle_footprint(m=64)
    dev = torch.device("cuda", 0)
    t = B.pip_prepare(torch.from_numpy(w.vertices).to(dev), torch.from_numpy(w.vertex_offsets).to(dev),
                      max_points=64)
    scratch = torch.zeros(4096, dtype=torch.uint8, device=dev)
    L = B.lib()
    assert L.pip_selftest_wait_timeout(t, scratch.data_ptr(), 0, None) == B.PIP_E_INVALID_ARG
    assert L.pip_selftest_wait_timeout(t, scratch.data_ptr(), 1 << 40, None) == B.PIP_E_INVALID_ARG
    assert L.pip_selftest_wait_timeout(t, None, 1000, None) == B.PIP_E_INVALID_ARG
    assert L.pip_selftest_wait_timeout(t, scratch.data_ptr() + 8, 1000, None) == B.PIP_E_INVALID_ARG
    assert B.pip_get_status(t)[0] == B.PIP_OK
    t.close()
