"""mg_residual_noalloc against mg_residual, through the C ABI.

mg_residual_noalloc serves callers that may not allocate device memory (code
running under another framework's allocator or memory budget, latency-bound
loops where cudaMalloc/cudaFree could stall the device, plug-ins that keep no
workspace): it needs no context and keeps its only scratch, one partial sum
per thread block, in a static device array.  These tests check that two
calls in a row give the residual and squared norm that the context-based
entry point gives, that a smaller call after a larger one does not pick up
the previous call's partial sums, and that sizes beyond the static limit are
refused before anything is launched.  This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_math_9907190_gb300 import Context
from paper_math_9907190_gb300 import _native as N
from paper_math_9907190_gb300 import inputs as I

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

DEV = torch.device("cuda", 0)


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _call(dim, n, order, f, u, r, norm2, pitch=None, h=None):
    pitch = n + 2 if pitch is None else pitch
    h = 1.0 / (n + 1) if h is None else h
    stream = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
    return N.lib().mg_residual_noalloc(dim, n, pitch, h, order, _p(f), _p(u), _p(r) if r is not None else None,
                                       _p(norm2) if norm2 is not None else None, stream)


def _inputs(dim, n, seed):
    f = torch.from_numpy(I.uniform_f(dim, n, seed)).to(DEV)
    u = torch.from_numpy(I.zero_ring(I.uniform_f(dim, n, seed + 100))).to(DEV)
    return f, u


@pytest.mark.parametrize("dim,n,order", [(2, 4095, 2), (2, 63, 4), (3, 255, 2), (3, 31, 4)])
def test_two_calls_match_context_residual(dim, n, order):
    with Context(dim, n, order=order) as c:
        for seed in (11, 12):  # two calls in a row on the shared static scratch
            f, u = _inputs(dim, n, seed)
            r_ref = c.new_grid()
            n2_ref = c.residual(f, u, r_ref)
            r = torch.zeros_like(f)
            n2 = torch.full((1,), -1.0, dtype=torch.float64, device=DEV)
            assert _call(dim, n, order, f, u, r, n2) == N.MG_OK
            torch.cuda.synchronize()
            scale = r_ref.abs().max().item()
            assert (r - r_ref).abs().max().item() <= 1e-12 * scale
            assert n2.item() == pytest.approx(n2_ref, rel=1e-12)


def test_smaller_call_after_larger_call():
    big_f, big_u = _inputs(2, 1023, 21)
    small_f, small_u = _inputs(2, 63, 22)
    n2 = torch.zeros(1, dtype=torch.float64, device=DEV)
    assert _call(2, 1023, 2, big_f, big_u, None, n2) == N.MG_OK
    assert _call(2, 63, 2, small_f, small_u, None, n2) == N.MG_OK
    torch.cuda.synchronize()
    with Context(2, 63) as c:
        want = c.residual(small_f, small_u)
    assert n2.item() == pytest.approx(want, rel=1e-12)


def test_refuses_sizes_beyond_static_limit_and_bad_arguments():
    t = torch.zeros(8, dtype=torch.float64, device=DEV)  # never touched: refused before launch
    assert _call(2, 8191, 2, t, t, None, None) == N.MG_EINVAL
    assert _call(3, 511, 2, t, t, None, None) == N.MG_EINVAL
    assert _call(2, 63, 2, t, t, None, None, h=1.0 / 63) == N.MG_EINVAL
    assert _call(2, 63, 3, t, t, None, None) == N.MG_EINVAL
    assert _call(2, 64, 2, t, t, None, None) == N.MG_EINVAL
    assert _call(2, 63, 2, t, t, None, None, pitch=64) == N.MG_EINVAL


def test_refuses_output_overlapping_an_input():
    """r is written while neighbouring threads still read f and u, so an r
    whose extent overlaps either is refused before anything is launched."""
    n = 63
    f, u = _inputs(2, n, 31)
    big = torch.zeros(2 * (n + 2) ** 2, dtype=torch.float64, device=DEV)
    assert _call(2, n, 2, f, u, f, None) == N.MG_EINVAL
    assert _call(2, n, 2, f, u, u, None) == N.MG_EINVAL
    # r starting inside u's extent
    ub = big[: (n + 2) ** 2].view(n + 2, n + 2)
    ub.copy_(u)
    rb = big[(n + 2) ** 2 // 2: (n + 2) ** 2 // 2 + (n + 2) ** 2]
    assert _call(2, n, 2, f, ub, rb, None) == N.MG_EINVAL


def test_allocates_no_device_memory():
    """After a first call (which may load the library's module on the device),
    further calls leave the device's free memory and torch's reserved memory
    unchanged."""
    f, u = _inputs(2, 1023, 41)
    r = torch.zeros_like(f)
    n2 = torch.zeros(1, dtype=torch.float64, device=DEV)
    assert _call(2, 1023, 2, f, u, r, n2) == N.MG_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(DEV)
    res0 = torch.cuda.memory_reserved(DEV)
    for _ in range(5):
        assert _call(2, 1023, 2, f, u, r, n2) == N.MG_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(DEV)[0] == free0
    assert torch.cuda.memory_reserved(DEV) == res0


_FRESH = r"""
import ctypes, sys, torch
sys.path.insert(0, sys.argv[1])
from paper_math_9907190_gb300 import _native as N
from paper_math_9907190_gb300 import inputs as I
dev = torch.device("cuda", 0)
n = 255
f = torch.from_numpy(I.uniform_f(2, n, 5)).to(dev)
u = torch.from_numpy(I.zero_ring(I.uniform_f(2, n, 6))).to(dev)
r = torch.zeros_like(f)
n2 = torch.zeros(1, dtype=torch.float64, device=dev)
s = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
P = lambda t: ctypes.c_void_p(t.data_ptr())
for _ in range(2):
    assert N.lib().mg_residual_noalloc(2, n, n + 2, 1.0 / (n + 1), 2, P(f), P(u), P(r), P(n2), s) == N.MG_OK
torch.cuda.synchronize()
print(repr(n2.item()))
"""


def test_works_in_a_fresh_process_without_any_context():
    """No mg_create anywhere in the process: the entry point needs nothing
    that a context would have set up."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", _FRESH, root], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    got = float(out.stdout.strip().splitlines()[-1])
    n = 255
    f = torch.from_numpy(I.uniform_f(2, n, 5)).to(DEV)
    u = torch.from_numpy(I.zero_ring(I.uniform_f(2, n, 6))).to(DEV)
    with Context(2, n) as c:
        want = c.residual(f, u)
    assert got == pytest.approx(want, rel=1e-12)
