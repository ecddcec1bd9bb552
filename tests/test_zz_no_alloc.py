"""The allocation-free dot product (tidas_dot_noalloc) against tidas_dot.

tidas_dot_noalloc serves callers that cannot let the library allocate device
memory (a pipeline that reserves its device budget up front, a thread that
must not wait on an allocator): its scratch is a fixed array inside the
library.  This file sorts last so that a run stopping at the first failure
has run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from tidas_workloads import generators

pytestmark = pytest.mark.gpu

MAX_N = 16_777_216


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_15464_gb300 import capi
    return torch, capi, capi.load()


def test_noalloc_dot_matches_allocating_dot_on_consecutive_calls():
    torch, capi, L = _setup()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    # two calls in a row with different lengths and data: the second must not
    # see anything the first one left in the shared scratch
    for call, n in enumerate((MAX_N, 123_457)):
        a = torch.from_numpy(generators.standard_normal((n,), (70, call))).cuda()
        b = torch.from_numpy(generators.standard_normal((n,), (71, call))).cuda()
        rc = L.tidas_dot_noalloc(a.data_ptr(), b.data_ptr(), n, out[0:1].data_ptr(), stream)
        assert rc == capi.TIDAS_OK, capi.tidas_last_error()
        rc = L.tidas_dot(a.data_ptr(), b.data_ptr(), n, out[1:2].data_ptr(), stream)
        assert rc == capi.TIDAS_OK, capi.tidas_last_error()
        got, ref = out[:2].cpu().numpy()
        scale = float(torch.linalg.vector_norm(a.double()) * torch.linalg.vector_norm(b.double()))
        assert abs(got - ref) <= 1e-12 * scale
        exact = float(np.dot(a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)))
        assert abs(got - exact) <= 1e-12 * scale


def test_noalloc_dot_rejects_sizes_beyond_its_scratch():
    torch, capi, L = _setup()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    a = torch.zeros(8, device="cuda")
    rc = L.tidas_dot_noalloc(a.data_ptr(), a.data_ptr(), MAX_N + 1, out.data_ptr(), None)
    assert rc == capi.TIDAS_ERR_ARG
    assert "exceeds" in capi.tidas_last_error()
