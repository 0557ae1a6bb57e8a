"""GPU parity of the extra Jacobi sweeps per level (mg_set_sweeps), the
extension the paper's conclusion leaves open, against the oracle: V-cycle
iterates element by element (max pointwise difference over max |u|: FP64
1e-12, mixed FP32 levels 1e-5, with the L2 ratio 2e-6 as a second bar),
solves cycle by cycle, and the argument checks."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_math_9907190_gb300 import Context
from paper_math_9907190_gb300 import inputs as I
from paper_math_9907190_gb300._native import MGError
from _iterates import assert_iterate

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

DEV = torch.device("cuda", 0)


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def H(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("n,prec,tol,l2", [(63, "fp64", 1e-12, 1e-12), (255, "fp64", 1e-12, 1e-12),
                                           (255, "mixed", 1e-5, 2e-6)])
@pytest.mark.parametrize("extra", [1, 2])
def test_extra_sweeps_vcycle_matches_oracle(n, prec, tol, l2, extra):
    f = I.uniform_f(2, n, 21)
    uo = O.grid(2, n)
    with Context(2, n, precision=prec, omega=(1.052,)) as c:
        c.set_sweeps(extra)
        ug, ft = c.new_grid(), T(f)
        for cyc in range(2):
            O.vcycle(f, uo, omega=[1.052], extra=extra)
            c.vcycle(ft, ug)
            assert_iterate(H(ug), uo, tol, l2_tol=l2, what=f"cycle {cyc}")


def test_extra_sweeps_solve_matches_oracle_fp64():
    n = 127
    f = I.uniform_f(2, n, 22)
    uo, it_o, rel_o, hist_o = O.solve(f, omega=[1.0], extra=1, rtol=1e-10)
    with Context(2, n, omega=(1.0,)) as c:
        c.set_sweeps(1)
        ug, it, rel, hist = c.solve(T(f), rtol=1e-10)
    assert it == it_o and rel <= 1e-10
    np.testing.assert_allclose(hist, hist_o, rtol=1e-8, atol=1e-14)
    assert_iterate(H(ug), uo, 1e-12)


def test_extra_sweeps_solve_mixed_reaches_tolerance():
    """Mixed precision with extra sweeps: FP32 levels, a direct residual every
    cycle; the solution agrees with the oracle's converged one."""
    n = 511
    f = I.uniform_f(2, n, 23)
    uo, _, _, _ = O.solve(f, omega=[1.0], extra=1, rtol=1e-13, max_cycles=200)
    with Context(2, n, precision="mixed", omega=(1.0,)) as c:
        c.set_sweeps(1)
        ug, it, rel, hist = c.solve(T(f), rtol=1e-10)
        assert rel <= 1e-10
        assert_iterate(H(ug), uo, 1e-8)
        c.set_sweeps(0)  # back to the paper's cycle (fused kernels, carried residual)
        _, it0, rel0, _ = c.solve(T(f), rtol=1e-10)
        assert rel0 <= 1e-10


def test_extra_sweeps_rejected_outside_2d_diagonal():
    with Context(3, 15) as c:
        with pytest.raises(MGError):
            c.set_sweeps(1)
        c.set_sweeps(0)
    with Context(2, 63, hierarchy="usual") as c:
        with pytest.raises(MGError):
            c.set_sweeps(1)
    with Context(2, 63) as c:
        with pytest.raises(MGError):
            c.set_sweeps(-1)
        with pytest.raises(MGError):
            c.set_sweeps(65)
