"""mg_solve_zero, a solve from u = 0 whose u is output only, against mg_solve
from a zeroed u (Sections 2.3, 3.3: the same V-cycles): the same iterate,
history and residual bit for bit, with u filled with NaN beforehand so that
any read of its old contents would show; zeros when no cycle runs; the graph
cache keeping a solve from zero apart from a warm start on the same arrays;
and the host-driven loop."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_math_9907190_gb300 import Context
from paper_math_9907190_gb300 import inputs as I

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def T(a):
    return torch.from_numpy(a).to("cuda")


CASES = [(2, 127, "mixed", "diag"), (2, 1023, "mixed", "diag"), (3, 63, "mixed", "diag"), (3, 127, "mixed", "diag"),
         (2, 127, "fp64", "diag"), (3, 31, "fp64", "diag"), (2, 255, "mixed", "usual")]


@pytest.mark.parametrize("dim,n,prec,hier", CASES)
def test_zero_start_equals_warm_start_from_zeros(dim, n, prec, hier):
    f = T(I.uniform_f(dim, n, 11))
    with Context(dim, n, precision=prec, hierarchy=hier) as c:
        u1, c1, r1, h1 = c.solve(f, c.new_grid(), rtol=1e-10)
        u2 = torch.full_like(u1, float("nan"))
        u2, c2, r2, h2 = c.solve(f, u2, rtol=1e-10, from_zero=True)
        assert (c1, r1, h1) == (c2, r2, h2)
        assert torch.equal(u1, u2)
        # a new grid (u=None) takes the same path
        u3, c3, r3, _ = c.solve(f, rtol=1e-10)
        assert c3 == c1 and r3 == r1 and torch.equal(u3, u1)


@pytest.mark.parametrize("dim,n", [(2, 255), (3, 63)])
def test_zero_start_without_a_cycle_gives_zeros(dim, n):
    """No cycle runs when max_cycles = 0 or f = 0; u still ends as zeros
    (interior and ring), never as its old contents."""
    f = T(I.uniform_f(dim, n, 12))
    with Context(dim, n, precision="mixed") as c:
        u = torch.full_like(f, float("nan"))
        u, cyc, rel, _ = c.solve(f, u, rtol=1e-10, max_cycles=0, raise_on_fail=False, from_zero=True)
        assert cyc == 0 and abs(rel - 1.0) < 1e-12
        assert torch.count_nonzero(u) == 0
        u = torch.full_like(f, 7.0)
        u, cyc, rel, _ = c.solve(torch.zeros_like(f), u, rtol=1e-10, raise_on_fail=False, from_zero=True)
        assert cyc == 0
        assert torch.count_nonzero(u) == 0


def test_zero_start_and_warm_start_alternate_on_the_same_arrays():
    """The graph cache keys a solve from zero apart from a warm start on the
    same f, u and tolerance: alternating them gives each its own result."""
    n = 255
    f = T(I.uniform_f(2, n, 13))
    with Context(2, n, precision="mixed") as c:
        u, cz, _, _ = c.solve(f, torch.full_like(f, float("nan")), rtol=1e-6, from_zero=True)
        assert cz > 0
        ref = u.clone()
        for _ in range(2):
            u, cw, rw, _ = c.solve(f, u, rtol=1e-6)  # warm start: already converged, u untouched
            assert cw == 0 and rw <= 1e-6 and torch.equal(u, ref)
            u, cz2, _, _ = c.solve(f, u, rtol=1e-6, from_zero=True)
            assert cz2 == cz and torch.equal(u, ref)


def test_zero_start_host_driven_loop():
    """The same through the host-driven loop of the same kernels
    (DIAGMG_SOLVE_GRAPH=0, read when the context is created)."""
    code = (
        "import numpy as np, torch\n"
        "from paper_math_9907190_gb300 import Context\n"
        "from paper_math_9907190_gb300 import inputs as I\n"
        "for dim, n in ((2, 255), (3, 63)):\n"
        "    f = torch.from_numpy(I.uniform_f(dim, n, 14)).cuda()\n"
        "    with Context(dim, n, precision='mixed') as c:\n"
        "        u1, c1, r1, h1 = c.solve(f, c.new_grid(), rtol=1e-10)\n"
        "        u2, c2, r2, h2 = c.solve(f, torch.full_like(f, float('nan')), rtol=1e-10, from_zero=True)\n"
        "        assert (c1, r1, h1) == (c2, r2, h2) and torch.equal(u1, u2), (dim, c1, c2, r1, r2)\n"
        "        u3, c3, _, _ = c.solve(f, torch.full_like(f, float('nan')), rtol=1e-10, max_cycles=0,\n"
        "                               raise_on_fail=False, from_zero=True)\n"
        "        assert c3 == 0 and torch.count_nonzero(u3) == 0\n"
        "print('ok')\n")
    env = dict(os.environ, DIAGMG_SOLVE_GRAPH="0", PYTHONPATH=ROOT)
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0 and p.stdout.strip().endswith("ok"), p.stdout + p.stderr


def test_zero_start_refuses_overlapping_arrays():
    n = 127
    f = T(I.uniform_f(2, n, 15))
    with Context(2, n, precision="mixed") as c:
        with pytest.raises(Exception):
            c.solve(f, f, rtol=1e-10, from_zero=True)
        np.testing.assert_array_equal(f.cpu().numpy(), I.uniform_f(2, n, 15))
