"""Two-stage fourth-order solve (second-order V-cycles, then fourth-order
cycles): FP64 iterates against the oracle running the same two stages, and
the gain in fourth-order cycles on a smooth problem the paper describes."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_math_9907190_gb300 import Context, default_omega
from paper_math_9907190_gb300 import inputs as I
from _iterates import assert_iterate

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

DEV = torch.device("cuda", 0)


@pytest.mark.parametrize("dim,n", [(2, 127), (2, 255), (3, 31)])
def test_two_stage_matches_oracle(dim, n):
    f = I.square_small(n) if dim == 2 else I.cube(n)
    om4, om2 = list(default_omega(dim, "diag", 4)), list(default_omega(dim, "diag", 2))
    with Context(dim, n, order=4, precision="fp64") as c:
        u, c2, c4, rel = c.solve_two_stage(torch.from_numpy(f).to(DEV), rtol2=1e-4, rtol=1e-10)
    uo, o2, _, _ = O.solve(f, order=2, omega=om2, rtol=1e-4)
    uo, o4, orel, _ = O.solve(f, uo, order=4, omega=om4, rtol=1e-10)
    assert (c2, c4) == (o2, o4)
    assert rel <= 1e-10
    assert_iterate(u.cpu().numpy(), uo, 1e-12)


def test_two_stage_needs_fewer_fourth_order_cycles_on_smooth_data():
    n = 255
    f = torch.from_numpy(I.square_small(n)).to(DEV)
    with Context(2, n, order=4, precision="mixed") as c:
        _, c4_only, rel1, _ = c.solve(f, rtol=1e-10)
        _, c2, c4, rel2 = c.solve_two_stage(f, rtol2=1e-4, rtol=1e-10)
    assert rel1 <= 1e-10 and rel2 <= 1e-10
    assert c4 < c4_only, (c2, c4, c4_only)
