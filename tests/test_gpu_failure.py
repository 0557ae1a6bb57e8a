"""Failure paths of the solvers, driven by inputs (no fault is involved).

A V-cycle whose over-relaxation weight leaves the stable range diverges: the
error on the finest grid's odd-index-sum points is scaled by exactly 1 - p
per cycle (the eigenspace pinned for the oracle), so p = 3 doubles it every
cycle and the residual passes 1e3 times its start.  A right-hand side
carrying a NaN has no defined relative residual.  Both must end the solve with
MG_EDIVERGED -- in the device-driven graph loop, in the host-driven loop
(DIAGMG_SOLVE_GRAPH=0, read when a context is created) and for one problem of
a batch, whose other problems still converge.
"""

import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_math_9907190_gb300 import Batch, Context
from paper_math_9907190_gb300 import _native as N
from paper_math_9907190_gb300 import inputs as I

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

DEV = torch.device("cuda", 0)


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


class _env:
    def __init__(self, **kv):
        self.kv, self.old = kv, {}

    def __enter__(self):
        for k, v in self.kv.items():
            self.old[k] = os.environ.get(k)
            os.environ[k] = v

    def __exit__(self, *exc):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _solve_status(c, f, max_cycles=100):
    u = c.new_grid()
    cyc, rel = N.ctypes.c_int(), N.ctypes.c_double()
    st = N.lib().mg_solve(c._h, c._grid(f, "f"), c._grid(u, "u"), 1e-10, max_cycles, N.ctypes.byref(cyc),
                          N.ctypes.byref(rel), None, c._stream())
    return st, cyc.value, rel.value


@pytest.mark.parametrize("graph", ["1", "0"])
@pytest.mark.parametrize("dim,n,prec", [(2, 255, "fp64"), (2, 255, "mixed"), (3, 31, "fp64"), (3, 63, "mixed")])
def test_unstable_weight_reports_divergence(graph, dim, n, prec):
    f = T(I.uniform_f(dim, n, 61))
    om = (3.0,) if dim == 2 else (1.0, 1.0, 1.0, 3.0)
    with _env(DIAGMG_SOLVE_GRAPH=graph):
        with Context(dim, n, precision=prec, omega=om) as c:
            st, cyc, rel = _solve_status(c, f)
            # the same context still solves a stable problem afterwards
            c.set_omega((1.052,) if dim == 2 else (1.11, 1.42, 1.08, 0.99))
            st2, _, rel2 = _solve_status(c, f)
    assert st == N.MG_EDIVERGED, (st, cyc, rel)
    assert 0 < cyc < 100 and not (rel <= 1.0)
    assert st2 == N.MG_OK and rel2 <= 1e-10


@pytest.mark.parametrize("graph", ["1", "0"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nan_right_hand_side_reports_divergence(graph, prec):
    f = I.uniform_f(2, 127, 62)
    f[40, 50] = math.nan
    with _env(DIAGMG_SOLVE_GRAPH=graph):
        with Context(2, 127, precision=prec) as c:
            st, cyc, rel = _solve_status(c, T(f))
    assert st == N.MG_EDIVERGED and cyc == 0 and math.isnan(rel)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_reports_the_diverging_problem_only(prec):
    sides = [63, 127, 63, 31, 127]
    fs = [I.batch_f(n, b) for b, n in enumerate(sides)]
    bad = 2
    fs[bad][10, 11] = math.nan
    with Batch(2, sides, precision=prec) as bt:
        us, cyc, rel = bt.solve([T(f) for f in fs], rtol=1e-10, max_cycles=60, raise_on_fail=False)
        status = bt.statuses()
        with pytest.raises(N.MGError) as e:
            bt.solve([T(f) for f in fs], rtol=1e-10, max_cycles=60)
        assert e.value.status == N.MG_EDIVERGED
    for b in range(len(sides)):
        if b == bad:
            assert status[b] == N.MG_EDIVERGED and math.isnan(rel[b])
        else:
            assert status[b] == N.MG_OK and rel[b] <= 1e-10, (b, status[b], rel[b])
            with Context(2, sides[b], precision=prec) as c:
                u1, c1, _, _ = c.solve(T(fs[b]), rtol=1e-10, max_cycles=60)
            assert cyc[b] == c1 and torch.equal(us[b], u1)


def test_batch_status_before_any_solve_is_refused():
    with Batch(2, [31, 63]) as bt:
        with pytest.raises(N.MGError):
            bt.statuses()
