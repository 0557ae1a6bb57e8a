"""Autograd adjoint of the solve: PoissonSolve.backward against central finite
differences and against the oracle's adjoint solve.

The loss sum((u - u_t)^2) is exactly quadratic in f, so the central
difference has no truncation error; it is evaluated as
sum((u+ - u-)(u+ + u- - 2 u_t)) / (2 eps) from two FP64 solves driven to the
FP64 residual floor, which avoids cancellation."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_math_9907190_gb300 import Context, PoissonSolve
from paper_math_9907190_gb300 import inputs as I

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

DEV = torch.device("cuda", 0)


def _fd(f_b, u_t, coord, eps, n):
    with Context(3, n, precision="fp64") as c:
        out = []
        for sgn in (1.0, -1.0):
            fp = f_b.clone()
            fp[coord] += sgn * eps
            u, _, _, _ = c.solve(fp, rtol=0.0, max_cycles=30, raise_on_fail=False)
            out.append(u)
    up, um = out
    return float(((up - um) * (up + um - 2 * u_t)).sum() / (2 * eps))


@pytest.mark.parametrize("nb,n", [(4, 31), (64, 127)])
def test_gradient_matches_finite_differences_and_oracle(nb, n):
    F = torch.stack([torch.from_numpy(I.grad_f(n, b)) for b in range(nb)]).to(DEV)
    ut = torch.from_numpy(I.grad_target(n)).to(DEV)
    F.requires_grad_(True)
    U = PoissonSolve.apply(F, 1e-10, "mixed")
    loss = ((U - ut) ** 2).sum()
    loss.backward()
    G = F.grad
    rng = np.random.default_rng(7)
    coords = [(int(rng.integers(0, nb)),) + c for c in I.grad_coords(n, 8)]
    for (b, k, j, i) in coords:
        fd = _fd(F.detach()[b], ut, (k, j, i), 1e-6, n)
        g = float(G[b, k, j, i])
        assert abs(g - fd) <= 1e-5 * abs(fd) + 1e-14, (b, k, j, i, g, fd)
    # the oracle's adjoint for one problem: w = L^-1 (2 (u - u_t))
    b0 = coords[0][0]
    rhs = 2.0 * (U.detach()[b0] - ut).cpu().numpy()
    rhs = I.zero_ring(rhs)
    w, _, _, _ = O.solve(np.ascontiguousarray(rhs), omega=[1.11, 1.42, 1.08, 0.99], rtol=1e-12, max_cycles=100)
    gw = G[b0].cpu().numpy()
    inner = (slice(1, -1),) * 3
    err = np.linalg.norm(gw[inner] - w[inner]) / np.linalg.norm(w[inner])
    assert err <= 1e-8, err
    # the ring of f does not enter the second-order solve
    assert float(G[:, 0].abs().max()) == 0.0


def test_single_problem_gradient_2d():
    n = 63
    f = torch.from_numpy(I.uniform_f(2, n, 3)).to(DEV).requires_grad_(True)
    ut = torch.zeros_like(f)
    u = PoissonSolve.apply(f, 1e-12, "fp64")
    (u * u).sum().backward()
    w, _, _, _ = O.solve(np.ascontiguousarray(I.zero_ring(2 * u.detach().cpu().numpy())), omega=[1.052], rtol=1e-13)
    g = f.grad.cpu().numpy()
    assert np.linalg.norm(g[1:-1, 1:-1] - w[1:-1, 1:-1]) / np.linalg.norm(w[1:-1, 1:-1]) <= 1e-10
