"""mg_solve_host (the solve with HOST arrays) and mg_fp64_rate, through the C ABI.

mg_solve_host must give the bits of mg_solve on device copies of the same
arrays (it copies, solves with the same graph, copies back), from u = 0 and
from a warm start, and refuse bad arguments before any copy."""

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


@pytest.mark.parametrize("dim,n,prec", [(2, 255, "mixed"), (2, 1023, "fp64"), (3, 63, "mixed")])
def test_host_solve_equals_device_solve(dim, n, prec):
    f = torch.from_numpy(I.uniform_f(dim, n, 71)).pin_memory()
    with Context(dim, n, precision=prec) as c:
        ud, cd, rd, _ = c.solve(f.to(DEV), rtol=1e-10)
        uh = torch.empty_like(f).pin_memory()
        u2, ch, rh = c.solve_host(f, uh, rtol=1e-10)
        assert u2 is uh and ch == cd and rh == rd
        assert np.array_equal(uh.numpy(), ud.cpu().numpy())
        # warm start from a partial solve, result written over the warm start
        up, _, _, _ = c.solve(f.to(DEV), rtol=1e-300, max_cycles=3, raise_on_fail=False)
        w = up.cpu().pin_memory()
        ud2, cd2, rd2, _ = c.solve(f.to(DEV), up.clone(), rtol=1e-10)
        _, ch2, rh2 = c.solve_host(f, w, u0=w, rtol=1e-10)
        assert ch2 == cd2 and rh2 == rd2 and np.array_equal(w.numpy(), ud2.cpu().numpy())


@pytest.mark.parametrize("dim,n", [(2, 1023), (3, 127)])
def test_host_solve_copy_back_waits_for_the_last_cycle(dim, n):
    """On the fused mixed path u is copied back while the closing direct
    residual still runs (from an event the solve's graph records once the
    last cycle has written u).  Alternating two right-hand sides, every result
    must be that of its own solve: a copy that did not wait would return the
    previous call's u."""
    fs = [torch.from_numpy(I.uniform_f(dim, n, 80 + k)).pin_memory() for k in range(2)]
    with Context(dim, n, precision="mixed") as c:
        want = [c.solve(f.to(DEV), rtol=1e-10)[0].cpu().numpy() for f in fs]
        uh = torch.empty_like(fs[0]).pin_memory()
        for k in (0, 1, 0, 1, 1, 0):
            uh.fill_(float("nan"))
            c.solve_host(fs[k], uh, rtol=1e-10)
            assert np.array_equal(uh.numpy(), want[k]), k


@pytest.mark.parametrize("dim,n,prec", [(2, 255, "mixed"), (3, 31, "mixed"), (2, 127, "fp64")])
def test_host_solve_with_padded_pitch_leaves_padding_alone(dim, n, prec):
    """Host arrays in a pitch above n + 2: only the (n+2)^d points move in
    either direction; the padding (NaN here) is neither read nor written."""
    pitch = n + 5 + 2
    f0 = I.uniform_f(dim, n, 77)
    fh = torch.full(f0.shape[:-1] + (pitch,), float("nan"), dtype=torch.float64)
    fh[..., : n + 2] = torch.from_numpy(f0)
    uh = torch.full_like(fh, float("nan"))
    with Context(dim, n, precision=prec, pitch=pitch) as c:
        _, ch, rh = c.solve_host(fh, uh, rtol=1e-10)
    assert torch.isnan(uh[..., n + 2:]).all() and torch.isnan(fh[..., n + 2:]).all()
    with Context(dim, n, precision=prec) as c:
        ud, cd, rd, _ = c.solve(torch.from_numpy(f0).to(DEV), rtol=1e-10)
    assert ch == cd and rh == rd
    assert np.array_equal(uh[..., : n + 2].numpy(), ud.cpu().numpy())


@pytest.mark.parametrize("dim,n,prec,count", [(2, 255, "mixed", 5), (2, 1023, "mixed", 3), (3, 63, "mixed", 4),
                                               (2, 127, "fp64", 3), (2, 255, "mixed", 1)])
def test_host_solve_many_equals_one_call_per_problem(dim, n, prec, count):
    """mg_solve_host_many pipelines the copies and solves of several
    problems over two device buffers; each result must be the bits of
    mg_solve_host on that problem alone (distinct right-hand sides, so a
    result taken from the wrong buffer or too early would show)."""
    fs = [torch.from_numpy(I.uniform_f(dim, n, 90 + k)).pin_memory() for k in range(count)]
    with Context(dim, n, precision=prec) as c:
        want = []
        for f in fs:
            uh = torch.empty_like(f).pin_memory()
            _, ch, rh = c.solve_host(f, uh, rtol=1e-10)
            want.append((uh, ch, rh))
        us = [torch.full_like(f, float("nan")).pin_memory() for f in fs]
        for _ in range(2):  # twice: the second call reuses the graphs and buffers
            for u in us:
                u.fill_(float("nan"))
            _, cyc, rel = c.solve_host_many(fs, us, rtol=1e-10)
            for k in range(count):
                assert cyc[k] == want[k][1] and rel[k] == want[k][2], k
                assert np.array_equal(us[k].numpy(), want[k][0].numpy()), k


def test_host_solve_many_host_driven_loop():
    """With DIAGMG_SOLVE_GRAPH=0 (read when the context is created) the
    problems run one after the other through mg_solve_host: the same bits."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import numpy as np, torch\n"
        "from paper_math_9907190_gb300 import Context\n"
        "from paper_math_9907190_gb300 import inputs as I\n"
        "fs = [torch.from_numpy(I.uniform_f(2, 255, 95 + k)).pin_memory() for k in range(3)]\n"
        "with Context(2, 255, precision='mixed') as c:\n"
        "    want = [c.solve_host(f, torch.empty_like(f), rtol=1e-10) for f in fs]\n"
        "    us, cyc, rel = c.solve_host_many(fs, rtol=1e-10)\n"
        "    for k in range(3):\n"
        "        assert cyc[k] == want[k][1] and rel[k] == want[k][2], k\n"
        "        assert np.array_equal(us[k].numpy(), want[k][0].numpy()), k\n"
        "print('ok')\n")
    env = dict(os.environ, DIAGMG_SOLVE_GRAPH="0", PYTHONPATH=root)
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0 and p.stdout.strip().endswith("ok"), p.stdout + p.stderr


def test_host_solve_many_edge_cases():
    with Context(2, 63) as c:
        assert c.solve_host_many([], []) == ([], [], [])
        f = torch.zeros((65, 65), dtype=torch.float64)
        L = N.lib()
        fp = (N.ctypes.c_void_p * 1)(f.data_ptr())
        assert L.mg_solve_host_many(c._h, 1, fp, fp, 1e-10, 10, None, None, c._stream()) == N.MG_EINVAL  # u over f
        assert L.mg_solve_host_many(c._h, -1, fp, fp, 1e-10, 10, None, None, c._stream()) == N.MG_EINVAL
        # problem 0's output over problem 1's input
        g = torch.zeros_like(f)
        fp2 = (N.ctypes.c_void_p * 2)(f.data_ptr(), g.data_ptr())
        up2 = (N.ctypes.c_void_p * 2)(g.data_ptr(), torch.zeros_like(f).data_ptr())
        assert L.mg_solve_host_many(c._h, 2, fp2, up2, 1e-10, 10, None, None, c._stream()) == N.MG_EINVAL


def test_host_solve_refuses_bad_arguments():
    with Context(2, 63) as c:
        f = torch.zeros((65, 65), dtype=torch.float64)
        L = N.lib()
        P = lambda t: N.ctypes.c_void_p(t.data_ptr())  # noqa: E731
        s = c._stream()
        assert L.mg_solve_host(c._h, None, None, P(f), 1e-10, 10, None, None, s) == N.MG_EINVAL
        assert L.mg_solve_host(c._h, P(f), None, P(f), 1e-10, 10, None, None, s) == N.MG_EINVAL  # u over f
        assert L.mg_solve_host(c._h, P(f), None, N.ctypes.c_void_p(f.data_ptr() + 4), 1e-10, 10, None, None,
                               s) == N.MG_EINVAL
        assert L.mg_solve_host(c._h, P(f), None, P(torch.zeros_like(f)), -1.0, 10, None, None, s) == N.MG_EINVAL


def test_fp64_rate_is_plausible():
    """Measured FP64 pipe rate: between a tenth of and twice the nominal
    152 SMs x 2 FP64 operations per clock x 2.07 GHz (6.3e11 /s)."""
    with Context(2, 63) as c:
        r = c.fp64_rate()
    assert 6.3e10 < r < 1.26e12, r
