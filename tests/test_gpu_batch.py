"""Batched solves (mg_solve_batched) against single-problem solves and the oracle.

Every problem of a batch runs the same kernels as a single-problem context,
with its data located by the batch offsets; its iterates must therefore match
the single-problem solve exactly (same cycles, same residual history end) and
the oracle to the parity bar."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_math_9907190_gb300 import Batch, Context, default_omega
from paper_math_9907190_gb300 import inputs as I
from _iterates import assert_iterate

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

DEV = torch.device("cuda", 0)


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_2d_matches_single_contexts_and_oracle(precision):
    sides = [31, 63, 127, 31, 255, 63, 7, 3, 511]
    fs = [I.batch_f(n, b) for b, n in enumerate(sides)]
    with Batch(2, sides, precision=precision) as bt:
        us, cyc, rel = bt.solve([T(f) for f in fs], rtol=1e-10, max_cycles=60)
    for b, n in enumerate(sides):
        with Context(2, n, precision=precision) as c:
            u1, c1, r1, _ = c.solve(T(fs[b]), rtol=1e-10, max_cycles=60)
        assert cyc[b] == c1, (b, n)
        assert torch.equal(us[b], u1), (b, n)
        assert rel[b] <= 1e-10
        # FP64: the oracle stopped at the same tolerance (same cycles, iterate parity);
        # mixed: the oracle's converged solution
        uo, co, _, _ = O.solve(fs[b], omega=list(default_omega(2)), rtol=1e-10 if precision == "fp64" else 1e-13,
                               max_cycles=100)
        if precision == "fp64":
            assert co == cyc[b]
        assert_iterate(us[b].cpu().numpy(), uo, 1e-12 if precision == "fp64" else 1e-8, what=f"problem {b} (n={n})")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_3d_matches_oracle(precision):
    sides = [15, 31, 15, 7]
    fs = [I.grad_f(n, b) for b, n in enumerate(sides)]
    om = default_omega(3)
    with Batch(3, sides, precision=precision) as bt:
        us, cyc, rel = bt.solve([T(f) for f in fs], rtol=1e-10, max_cycles=60)
    for b, n in enumerate(sides):
        with Context(3, n, precision=precision) as c:
            u1, c1, _, _ = c.solve(T(fs[b]), rtol=1e-10, max_cycles=60)
        assert cyc[b] == c1 and torch.equal(us[b], u1)
        uo, _, _, _ = O.solve(fs[b], omega=list(om), rtol=1e-10 if precision == "fp64" else 1e-13, max_cycles=100)
        assert_iterate(us[b].cpu().numpy(), uo, 1e-12 if precision == "fp64" else 1e-8, what=f"problem {b} (n={n})")


def test_batch_repeat_and_warm_start():
    sides = [63, 63, 127]
    fs = [T(I.batch_f(n, b)) for b, n in enumerate(sides)]
    with Batch(2, sides) as bt:
        us, cyc, rel = bt.solve(fs, rtol=1e-10)
        us2, cyc2, _ = bt.solve(fs, [u.clone() for u in us], rtol=1e-10)
        assert all(c == 0 for c in cyc2)
        us3, cyc3, _ = bt.solve(fs, [torch.zeros_like(u) for u in us], rtol=1e-10)
        assert cyc3 == cyc and all(torch.equal(a, b) for a, b in zip(us, us3))


@pytest.mark.parametrize("dim,n", [(2, 255), (3, 63)])
def test_batch_mixed_scales_per_problem(dim, n):
    """The quantizer of the mixed path's finest correction is bounded per
    problem: problems of one batch whose right-hand sides differ by 1e-12 ..
    1e12 in scale each converge as they do alone (same cycles, a direct
    residual below the tolerance)."""
    scales = [1e-12, 1.0, 1e12, 1e-4]
    base = I.uniform_f(dim, n, 31)
    fs = [base * s for s in scales]
    with Batch(dim, [n] * len(scales), precision="mixed") as bt:
        us, cyc, rel = bt.solve([T(f) for f in fs], rtol=1e-10, max_cycles=60)
    with Context(dim, n, precision="mixed") as c:
        _, c1, r1, _ = c.solve(T(base), rtol=1e-10, max_cycles=60)
    for b, s in enumerate(scales):
        assert cyc[b] == c1 and rel[b] <= 1e-10, (s, cyc[b], rel[b])
        # scaling f scales u (the quantizer's bound scales with it)
        np.testing.assert_allclose(us[b].cpu().numpy() / s, us[1].cpu().numpy(), rtol=0,
                                   atol=1e-6 * float(us[1].abs().max()))
