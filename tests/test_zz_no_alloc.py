"""nmf_error_noalloc: the Frobenius error for callers that cannot allocate device memory.

Such callers (a service that reserved all device memory for its own pool, a
latency-bound loop that cannot pay for cudaMalloc's implicit synchronisation)
get the same value as nmf_error from an entry point that keeps its scratch in
a fixed device array inside the library.  This file is collected last so that
a failure here leaves every other test already run.
"""
import numpy as np
import pytest

from oracle import nmf_oracle as o
from paper_1009_0881_gb300 import native, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def handle():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1009_0881_gb300 import build
    build.build()
    with native.Handle(0) as h:
        yield h


def _case(seed, gh, gw, n, r):
    import torch
    p = synth.make_problem(gh, gw, n, r, data_seed=seed)
    rng = np.random.default_rng(seed)
    V = (rng.random(p.V.shape) / r).astype(np.float32)
    W = rng.random(p.W.shape).astype(np.float32)
    return [torch.from_numpy(x).cuda() for x in (p.M, V, W)]


def test_noalloc_matches_nmf_error_on_two_calls_in_a_row(handle):
    import torch
    # two different problems back to back: the second result must not see the first call's scratch
    cases = [_case(1, 19, 19, 2429, 49), _case(2, 16, 16, 1000, 10)]
    for M, V, W in cases:
        got = native.error_noalloc(M, V, W)
        ref = handle.error(M, V, W)
        assert abs(got - ref) <= 1e-6 * ref, (got, ref)
        # and against the FP64 definition of the norm (problem (NMF), Section 2)
        exact = o.objective(M.cpu().numpy(), V.cpu().numpy(), W.cpu().numpy())
        assert abs(got - exact) <= 1e-6 * exact, (got, exact)
    # and once more on a caller-chosen stream
    s = torch.cuda.Stream()
    M, V, W = cases[0]
    got = native.error_noalloc(M, V, W, s.cuda_stream)
    assert abs(got - handle.error(M, V, W)) <= 1e-6 * got


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    x = torch.zeros(4, device="cuda")
    lib = native.load()
    import ctypes
    out = ctypes.c_double(-1.0)
    # ceil(m/64) * ceil(n/64) = 65537 tiles > 65536: rejected before any work is queued
    rc = lib.nmf_error_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), 64 * 65537, 64, 1, None, ctypes.byref(out))
    assert rc == -7 and out.value == -1.0
    rc = lib.nmf_error_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), 8, 8, 65, None, ctypes.byref(out))
    assert rc == -1


def test_noalloc_rejects_host_pointers():
    import ctypes
    import torch
    x = torch.zeros(64, device="cuda")
    h = np.zeros(64, np.float32)
    lib = native.load()
    out = ctypes.c_double(-1.0)
    hp = h.ctypes.data
    # the kernels read the arrays in place, so host memory is refused instead of staged
    rc = lib.nmf_error_noalloc(hp, x.data_ptr(), x.data_ptr(), 8, 8, 1, None, ctypes.byref(out))
    assert rc == -1 and out.value == -1.0
    rc = lib.nmf_error_noalloc(x.data_ptr(), x.data_ptr(), hp, 8, 8, 1, None, ctypes.byref(out))
    assert rc == -1 and out.value == -1.0
