"""CPU FP64 oracle for the diagonally oriented multigrid V-cycle.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path; the arithmetic lives in ``mg_oracle.c`` (plain C loops in
FP64, compiled without FMA contraction) and this module only marshals numpy
arrays to it.

Array convention: full grids of side n+2 (Dirichlet ring included) as C-ordered
numpy arrays indexed ``[j, i]`` in 2D and ``[k, j, i]`` in 3D, x fastest.

Where each function follows the paper (Roberts, "Fast and accurate multigrid
solution of Poisson's equation using diagonally oriented grids"):

* ``residual``            Eq. Evpois (5/7-point), Eq. Efos2, Eq. Efos4
* ``restrict2d_g2r/r2b``  Eq. Erest2r, Eq. Erest2b
* ``prolong2d_b2r``       Eq. Eajacr then Eq. Eajacb
* ``prolong2d_r2g``       the green-red sweep of Section 2.2 with the weight of Section 2.4
* ``restrict3d_*``        Eq. Erred, Eq. Ermagc + Eq. Ermagm, Eq. Erblu
* ``prolong3d_*``         Eq. Emprolm/Emprolb, Eq. Erprolr/Erprolm, Eq. Egprolg/Egprolr
* ``restrict_fw``, ``prolong_usual``  the conventional cycle of Sections 2.1-2.2, 3.1-3.2
* ``coarse_solve``        exact solve of the coarsest axis grid (the paper is silent)
* ``vcycle``, ``solve``   the V-cycle of Sections 2.3 and 3.3
* ``wcycle``              gamma-cycles of the diagonal hierarchy (Section 5 leaves them open)

Pins (tests/test_oracle_pins.py): closed-form stencil weights and the 17-point
composite restriction, exactness of every Jacobi sweep on quadratics, the
fixed point against a Kronecker-assembled direct solve, O(h^2)/O(h^4)
discretisation error, operator symmetry, the paper's flop counts rebuilt from
level point counts, the convergence factors of the paper's tables, an
eigenspace derived by hand (errors on the odd-index-sum points scaled by
exactly 1 - p; the same one level down on the 2D red and 3D magenta
levels), the spectral radius of the assembled cycle matrix, and linearity
of the cycle in (f, u).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.c")
_LIB = os.path.join(_HERE, "libmg_oracle.so")
_lock = threading.Lock()
_lib = None

DIAG, USUAL = 0, 1


def build(force: bool = False) -> str:
    """Compile mg_oracle.c with gcc (no FMA contraction; OpenMP when the
    compiler has it) and return the .so path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC"]
        if subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], capture_output=True).returncode != 0:
            subprocess.check_call(base + [_SRC, "-o", tmp, "-lm"])  # no OpenMP: the pragmas are ignored
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            i, d = ctypes.c_int, ctypes.c_double
            sig = {
                "orc_residual": (None, [i, i, d, i, dp, dp, dp]),
                "orc_restrict2d_g2r": (None, [i, dp, dp]),
                "orc_restrict2d_r2b": (None, [i, dp, dp]),
                "orc_prolong2d_b2r": (None, [i, d, d, dp, dp, dp]),
                "orc_prolong2d_r2g": (None, [i, d, d, dp, dp, dp]),
                "orc_restrict3d_g2r": (None, [i, dp, dp]),
                "orc_restrict3d_r2m": (None, [i, dp, dp]),
                "orc_restrict3d_m2b": (None, [i, dp, dp]),
                "orc_prolong3d_b2m": (None, [i, d, d, dp, dp, dp]),
                "orc_prolong3d_m2r": (None, [i, d, d, d, dp, dp, dp]),
                "orc_prolong3d_r2g": (None, [i, d, d, dp, dp, dp]),
                "orc_restrict_fw": (None, [i, i, dp, dp]),
                "orc_prolong_usual": (None, [i, i, d, d, dp, dp, dp]),
                "orc_coarse_solve": (i, [i, i, d, dp, dp]),
                "orc_vcycle": (i, [i, i, i, i, i, dp, dp, dp]),
                "orc_vcycle_sweeps": (i, [i, i, i, i, i, dp, i, dp, dp]),
                "orc_sweep2d_red": (None, [i, d, d, dp, dp]),
                "orc_sweep2d_green": (None, [i, d, d, dp, dp]),
                "orc_solve_sweeps": (i, [i, i, i, i, i, dp, i, dp, dp, d, i, dp, dp]),
                "orc_norm2_interior": (d, [i, i, dp]),
                "orc_solve": (i, [i, i, i, i, i, dp, dp, dp, d, i, dp, dp]),
                "orc_set_threads": (i, [i]),
                "orc_wcycle": (i, [i, i, i, i, dp, i, dp, dp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            lib.orc_set_threads(1)
            _lib = lib
    return _lib


def set_threads(t: int) -> int:
    """Threads of the oracle's per-point loops (results do not depend on it);
    returns the count in effect (1 when the library was built without OpenMP)."""
    return int(_load().orc_set_threads(int(t)))


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle arrays are C-contiguous float64"
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dim(a: np.ndarray) -> int:
    return a.ndim


def grid(dim: int, n: int) -> np.ndarray:
    """A zeroed full grid of side n (ring included)."""
    return np.zeros((n + 2,) * dim, dtype=np.float64)


def residual(f: np.ndarray, u: np.ndarray, order: int = 2, h: float | None = None) -> np.ndarray:
    """r = f - L u (order 2) or Mehrstellen / 19-point (order 4); ring of r is 0."""
    dim, n = f.ndim, f.shape[0] - 2
    h = 1.0 / (n + 1) if h is None else h
    r = grid(dim, n)
    _load().orc_residual(dim, n, h, order, _p(f), _p(u), _p(r))
    return r


def restrict2d_g2r(rg: np.ndarray, out: np.ndarray | None = None) -> np.ndarray:
    n = rg.shape[0] - 2
    rr = grid(2, n) if out is None else out
    _load().orc_restrict2d_g2r(n, _p(rg), _p(rr))
    return rr


def restrict2d_r2b(rr: np.ndarray) -> np.ndarray:
    n = rr.shape[0] - 2
    rb = grid(2, (n - 1) // 2)
    _load().orc_restrict2d_r2b(n, _p(rr), _p(rb))
    return rb


def prolong2d_b2r(vb, rr, h, p, out=None):
    n = rr.shape[0] - 2
    vr = grid(2, n) if out is None else out
    _load().orc_prolong2d_b2r(n, h, p, _p(vb), _p(rr), _p(vr))
    return vr


def prolong2d_r2g(vr, rg, h, p, out=None):
    n = rg.shape[0] - 2
    vg = grid(2, n) if out is None else out
    _load().orc_prolong2d_r2g(n, h, p, _p(vr), _p(rg), _p(vg))
    return vg


def restrict3d_g2r(rg, out=None):
    n = rg.shape[0] - 2
    rr = grid(3, n) if out is None else out
    _load().orc_restrict3d_g2r(n, _p(rg), _p(rr))
    return rr


def restrict3d_r2m(rr, out=None):
    n = rr.shape[0] - 2
    rm = grid(3, n) if out is None else out
    _load().orc_restrict3d_r2m(n, _p(rr), _p(rm))
    return rm


def restrict3d_m2b(rm):
    n = rm.shape[0] - 2
    rb = grid(3, (n - 1) // 2)
    _load().orc_restrict3d_m2b(n, _p(rm), _p(rb))
    return rb


def prolong3d_b2m(vb, rm, h, pm, out=None):
    n = rm.shape[0] - 2
    vm = grid(3, n) if out is None else out
    _load().orc_prolong3d_b2m(n, h, pm, _p(vb), _p(rm), _p(vm))
    return vm


def prolong3d_m2r(vm, rr, h, pr1, pr2, out=None):
    n = rr.shape[0] - 2
    vr = grid(3, n) if out is None else out
    _load().orc_prolong3d_m2r(n, h, pr1, pr2, _p(vm), _p(rr), _p(vr))
    return vr


def prolong3d_r2g(vr, rg, h, pg, out=None):
    n = rg.shape[0] - 2
    vg = grid(3, n) if out is None else out
    _load().orc_prolong3d_r2g(n, h, pg, _p(vr), _p(rg), _p(vg))
    return vg


def restrict_fw(rf):
    dim, n = rf.ndim, rf.shape[0] - 2
    rc = grid(dim, (n - 1) // 2)
    _load().orc_restrict_fw(dim, n, _p(rf), _p(rc))
    return rc


def prolong_usual(vc, rf, h, p, out=None):
    dim, n = rf.ndim, rf.shape[0] - 2
    vf = grid(dim, n) if out is None else out
    _load().orc_prolong_usual(dim, n, h, p, _p(vc), _p(rf), _p(vf))
    return vf


def coarse_solve(r, H):
    dim, n = r.ndim, r.shape[0] - 2
    v = grid(dim, n)
    if _load().orc_coarse_solve(dim, n, H, _p(r), _p(v)) != 0:
        raise MemoryError("coarse solve allocation failed")
    return v


def _omega(omega, dim, hier):
    if omega is None:
        omega = [1.0, 1.0, 1.0, 1.0]
    om = np.zeros(4, dtype=np.float64)
    om[: len(omega)] = omega
    return om


def vcycle(f, u, *, hier=DIAG, order=2, coarsest=3, omega=None, extra=0):
    """One V-cycle in place on u (a full-grid float64 array); returns u.
    extra: extra Jacobi sweeps per level (2D diagonal hierarchy)."""
    dim, n = f.ndim, f.shape[0] - 2
    om = _omega(omega, dim, hier)
    rc = _load().orc_vcycle_sweeps(dim, n, hier, order, coarsest, _p(om), extra, _p(f), _p(u))
    if rc != 0:
        raise ValueError(f"orc_vcycle rejected dim={dim} n={n} coarsest={coarsest} order={order}")
    return u


def solve(f, u=None, *, hier=DIAG, order=2, coarsest=3, omega=None, rtol=1e-10, max_cycles=100, extra=0):
    """V-cycles from u (default 0) until the relative residual <= rtol.

    Returns (u, cycles, relres, history)."""
    dim, n = f.ndim, f.shape[0] - 2
    u = grid(dim, n) if u is None else u
    om = _omega(omega, dim, hier)
    hist = np.zeros(max(max_cycles, 1), dtype=np.float64)
    rel = ctypes.c_double(0.0)
    it = _load().orc_solve_sweeps(dim, n, hier, order, coarsest, _p(om), extra, _p(f), _p(u), rtol, max_cycles,
                                  _p(hist), ctypes.byref(rel))
    if it < 0:
        raise ValueError("orc_solve rejected its arguments")
    return u, it, rel.value, hist[:it].copy()


def wcycle(f, u, *, order=2, coarsest=3, omega=None, gamma=2):
    """One gamma-cycle of the diagonal hierarchy in place on u (gamma = 1: the
    V-cycle); omega as for vcycle.  Returns u."""
    dim, n = f.ndim, f.shape[0] - 2
    om = _omega(omega, dim, DIAG)
    if _load().orc_wcycle(dim, n, order, coarsest, _p(om), gamma, _p(f), _p(u)) != 0:
        raise ValueError(f"orc_wcycle rejected dim={dim} n={n} coarsest={coarsest} gamma={gamma}")
    return u


def sweep2d_red(rr, vr, p=1.0, h=None):
    """One extra Jacobi sweep in place on a red (diagonal) level stored on its
    pair's green grid: i,j odd points, then i,j even points."""
    n = vr.shape[0] - 2
    h = 1.0 / (n + 1) if h is None else h
    _load().orc_sweep2d_red(n, h, p, _p(rr), _p(vr))
    return vr


def sweep2d_green(rg, vg, p=1.0, h=None):
    """One extra Jacobi sweep in place on a green (axis) level: i+j odd points,
    then i+j even points."""
    n = vg.shape[0] - 2
    h = 1.0 / (n + 1) if h is None else h
    _load().orc_sweep2d_green(n, h, p, _p(rg), _p(vg))
    return vg


def norm2_interior(x):
    return float(_load().orc_norm2_interior(x.ndim, x.shape[0] - 2, _p(x)))
