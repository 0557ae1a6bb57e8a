"""GPU convergence factors (mg_rho) against the oracle's eigenvalue analysis,
and the weight search of Sections 2.4 / 3.4 on the GPU."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_math_9907190_gb300 import Context
from paper_math_9907190_gb300.omega_search import nelder_mead, search_omega

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _oracle_rho(dim, n, hier, order, omega):
    from scipy.sparse.linalg import LinearOperator, eigs
    N = n ** dim
    f = O.grid(dim, n)
    sl = (slice(1, -1),) * dim

    def mv(x):
        u = O.grid(dim, n)
        u[sl] = x.reshape((n,) * dim)
        O.vcycle(f, u, hier=hier, order=order, omega=omega)
        return u[sl].ravel().copy()

    vals = eigs(LinearOperator((N, N), matvec=mv, dtype=np.float64), k=3, which="LM",
                return_eigenvectors=False, tol=1e-8, maxiter=5000)
    return float(np.max(np.abs(vals)))


@pytest.mark.parametrize("dim,n,order,omega", [(2, 63, 2, (1.052,)), (2, 63, 4, (1.2,)),
                                               (3, 15, 2, (1.11, 1.42, 1.08, 0.99)), (3, 15, 2, (1.0, 1.0, 1.0, 1.0))])
def test_power_iteration_rho_matches_oracle_eigenvalue(dim, n, order, omega):
    with Context(dim, n, order=order, precision="fp64", omega=omega) as c:
        rho = c.rho(cycles=120, skip=80)
    want = _oracle_rho(dim, n, O.DIAG, order, list(omega))
    assert abs(rho - want) <= 0.03 * want, (rho, want)


def test_nelder_mead_on_a_quadratic():
    x, fx, _ = nelder_mead(lambda v: (v[0] - 1.3) ** 2 + 2 * (v[1] + 0.4) ** 2, [0.0, 0.0], step=0.5, iters=200,
                           tol=1e-12)
    assert abs(x[0] - 1.3) < 1e-3 and abs(x[1] + 0.4) < 1e-3


def test_search_finds_paper_quality_weights_3d():
    """Started from p = 1 on the paper's 17^3 grid, the search reaches a factor
    at least as good as the paper's tabulated weights give here."""
    omega, rho, evals = search_omega(3, 15, x0=[1.0, 1.0, 1.0, 1.0], iters=60)
    with Context(3, 15, precision="fp64", omega=(1.11, 1.42, 1.08, 0.99)) as c:
        rho_paper = c.rho(cycles=50, skip=30)
    assert rho <= 1.02 * rho_paper, (omega, rho, rho_paper)
