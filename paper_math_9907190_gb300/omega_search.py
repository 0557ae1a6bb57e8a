"""Search of the over-relaxation weights (Sections 2.4 and 3.4, Table 3).

The paper tuned p (2D) and (p_m, p_r1, p_r2, p_g) (3D) with the Nelder-Mead
simplex method on the largest eigenvalue of the V-cycle, which it could only
afford on a 17^3 grid.  Here each convergence factor comes from mg_rho (power
iteration on the GPU V-cycle), so the same search runs on larger grids.  The
simplex logic below is the textbook Nelder-Mead method (reflection 1,
expansion 2, contraction 1/2, shrink 1/2) written for this module.
"""

from __future__ import annotations

import numpy as np

from .api import Context, default_omega


def nelder_mead(fun, x0, step=0.1, iters=60, tol=1e-4):
    """Minimise fun over R^d from x0; returns (x_best, f_best, evaluations)."""
    d = len(x0)
    pts = [np.array(x0, dtype=float)] + [np.array(x0, dtype=float) + step * np.eye(d)[i] for i in range(d)]
    vals = [fun(p) for p in pts]
    evals = len(vals)
    for _ in range(iters):
        order = np.argsort(vals)
        pts = [pts[i] for i in order]
        vals = [vals[i] for i in order]
        if abs(vals[-1] - vals[0]) <= tol * max(abs(vals[0]), 1e-12):
            break
        centroid = np.mean(pts[:-1], axis=0)
        xr = centroid + (centroid - pts[-1])
        fr = fun(xr); evals += 1
        if fr < vals[0]:
            xe = centroid + 2.0 * (centroid - pts[-1])
            fe = fun(xe); evals += 1
            pts[-1], vals[-1] = (xe, fe) if fe < fr else (xr, fr)
        elif fr < vals[-2]:
            pts[-1], vals[-1] = xr, fr
        else:
            xc = centroid + 0.5 * (pts[-1] - centroid)
            fc = fun(xc); evals += 1
            if fc < vals[-1]:
                pts[-1], vals[-1] = xc, fc
            else:
                for i in range(1, d + 1):
                    pts[i] = pts[0] + 0.5 * (pts[i] - pts[0])
                    vals[i] = fun(pts[i]); evals += 1
    i = int(np.argmin(vals))
    return pts[i], vals[i], evals


def search_omega(dim: int, n: int, order: int = 2, x0=None, iters: int = 40, cycles: int = 50, skip: int = 30):
    """Nelder-Mead over the weights of the diagonal cycle on an n-grid (FP64).
    Returns (omega, rho, evaluations)."""
    x0 = list(default_omega(dim, "diag", order)) if x0 is None else list(x0)
    with Context(dim, n, order=order, precision="fp64", omega=x0) as c:
        def fun(x):
            if np.any(np.asarray(x) <= 0.0) or np.any(np.asarray(x) > 3.0):
                return 10.0
            c.set_omega(list(x))
            return c.rho(cycles=cycles, skip=skip)
        x, fx, evals = nelder_mead(fun, x0, step=0.05, iters=iters)
    return [float(v) for v in x], float(fx), evals
