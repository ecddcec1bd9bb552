"""Failure detection on the device without a fault: a bounded wait that runs
out, the flag it records, and the host status that reports it.

The test hook of tidas_set_debug_option makes the BF16 GEMM's producer issue
no copies, so its MMA thread's first wait gives up after a short limit with
nothing in flight; the CTA returns, the next tidas_device_status call reports
TIDAS_ERR_TIMEOUT with the wait's code, and the context stays usable: a
normal call afterwards is bit-identical to one made before.
"""
import ctypes
import time

import numpy as np
import pytest

from tidas_workloads import generators

from .gpu_helpers import host, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _gemm(A, B, out):
    from paper_2507_15464_gb300 import capi
    from paper_2507_15464_gb300.ops import _ptr, _stream
    M, K = A.shape
    N = B.shape[0]
    capi.call("tidas_gemm_bf16", _ptr(A), _ptr(B), M, N, K, None, 0, _ptr(out), None, N,
              _stream())


def _status():
    from paper_2507_15464_gb300 import capi
    v = ctypes.c_int32(0)
    rc = capi.load().tidas_device_status(ctypes.byref(v))
    return rc, v.value


def test_wait_that_runs_out_is_reported_and_the_context_stays_usable():
    from paper_2507_15464_gb300 import capi
    M, N, K = 256, 64, 192
    A = to_dev(generators.standard_normal((M, K), (90, 0))).to(torch.bfloat16)
    B = to_dev(generators.standard_normal((N, K), (90, 1))).to(torch.bfloat16)
    before = torch.empty((M, N), device="cuda")
    _gemm(A, B, before)
    assert _status() == (capi.TIDAS_OK, 0)
    out = torch.full((M, N), 7.0, device="cuda")
    try:
        capi.tidas_set_debug_option(capi.DEBUG_WAIT_LIMIT_NS, 1_000_000)  # 1 ms
        capi.tidas_set_debug_option(capi.DEBUG_SKIP_COPIES, 1)
        t0 = time.perf_counter()
        _gemm(A, B, out)  # enqueues fine: the failure is on the device
        rc, code = _status()
        dt = time.perf_counter() - t0
    finally:
        capi.tidas_set_debug_option(capi.DEBUG_SKIP_COPIES, 0)
        capi.tidas_set_debug_option(capi.DEBUG_WAIT_LIMIT_NS, 1_000_000_000)
    assert rc == capi.TIDAS_ERR_TIMEOUT
    assert code == 202  # the MMA thread's wait for its first operand stage
    assert "gave up" in capi.tidas_last_error()
    assert dt < 5.0  # a 1 ms limit, not the default 1 s per wait
    assert torch.all(out == 7.0)  # the abandoned CTAs wrote nothing
    # the flag was cleared by the read, and the context still works
    assert _status() == (capi.TIDAS_OK, 0)
    after = torch.empty((M, N), device="cuda")
    _gemm(A, B, after)
    assert _status() == (capi.TIDAS_OK, 0)
    np.testing.assert_array_equal(host(after), host(before))

